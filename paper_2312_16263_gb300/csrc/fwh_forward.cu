// Forward scatter of the FW-H source-time signals onto the observer grids
// ("compute Noise" + "interp pressure signal" + surface integration,
// Sec. III B/C; integrand of Eqs. pT_WT_nd + pL_WT_nd).
//
// For panel p, observer o and source sample k, with the observer-independent
// row X[p][k] (8 series F and their spline moments M) and the per-(p, o)
// record (coefficients c, shift i0, weights a, b, cc, dd):
//   g = c . F[k],   m = c . M[k]                     (source pressure, moment)
//   bin k - i0     += a g + cc m                     (spline, left node)
//   bin k - i0 - 1 += b g + dd m                     (spline, right node)
// which is the natural-spline value at tau = t_j - M0 R for every observer
// bin j (Eq. tau2), summed over panels.  20 FMA per (panel, sample, observer).
//
// Work item = (panel set, observer group, time segment).  A CTA holds NW
// compute warps; warp w owns observers o_begin + w + NW m (m < obs_per_warp)
// of the group and keeps, per observer, a window of `win` bins in shared
// memory.  Lanes map to source samples (k = k0 + lane + 32 j, j < TK), so each
// X row is loaded once per warp and reused for all of the warp's observers,
// the coefficient record is a warp-uniform broadcast, and the window updates
// are conflict-free (consecutive lanes, consecutive bins).  The per-(p, o)
// shift only moves the window offset, never the lane pattern.  After each
// chunk of 32 TK samples the oldest 32 TK bins of every window are complete
// for this panel set: they are flushed to p_out with FP64 atomics (one per bin
// per panel set, not per panel) and the window slides.
//
// Two ways to feed the compute warps:
//  * direct: every warp loads its X rows and coefficient records from global
//    memory (L1/L2) itself;
//  * TMA pipeline: one producer warp streams, per (chunk, panel) step, the X
//    rows (a 2D tensor-map load, 128B swizzled so the per-lane row reads are
//    bank-conflict-free) and the group's coefficient records (a 1D bulk
//    copy) into a ring of shared-memory stages; full/empty mbarriers hand the
//    stages over.  Every wait is bounded by a clock limit: on expiry the
//    kernel raises kErrTimeout, stops issuing copies, waits (bounded) for the
//    copies already in flight and leaves.
//
// Window bound: a panel set's shifts for one observer span S = i0max - i0min;
// slots touched in a chunk are [0, CH + S], so S <= win - CH - 1 is required.
// The host planner bounds S from the set's extent; the plan kernel records,
// per (set, observer), i0max and, per (panel, observer) record, the window
// offset i0max - i0 clamped to [0, win - CH - 1], raising kErrWindow if the
// bound is exceeded; the hot loop adds that offset and can never leave the
// window.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <type_traits>

#include "fwh_internal.cuh"

namespace fwh {

namespace {

constexpr int kMaxObsPerWarp = 16;
constexpr int kMaxObsPerWarpF32 = 9;  // the FP32 consumer unrolls its observer loop to this
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz

template <typename T> struct Vec;
template <> struct Vec<float> {
  using V = float4;
  static constexpr int per = 4;
};
template <> struct Vec<double> {
  using V = double2;
  static constexpr int per = 2;
};

template <typename T> __device__ __forceinline__ int rec_i0_of(T v);
template <> __device__ __forceinline__ int rec_i0_of<float>(float v) {
  return __float_as_int(v);
}
template <> __device__ __forceinline__ int rec_i0_of<double>(double v) { return (int)v; }

template <typename T>
__device__ __forceinline__ void load16(const T *src, T (&dst)[kRec]) {
  using V = typename Vec<T>::V;
  constexpr int per = Vec<T>::per;
  const V *s = reinterpret_cast<const V *>(src);
#pragma unroll
  for (int q = 0; q < kRec / per; ++q) {
    V v = __ldg(s + q);
    if constexpr (per == 4) {
      dst[4 * q] = v.x; dst[4 * q + 1] = v.y; dst[4 * q + 2] = v.z; dst[4 * q + 3] = v.w;
    } else {
      dst[2 * q] = v.x; dst[2 * q + 1] = v.y;
    }
  }
}

// Shared-memory broadcast read of a 16-value record.
template <typename T>
__device__ __forceinline__ void lds16(const T *src, T (&dst)[kRec]) {
  using V = typename Vec<T>::V;
  constexpr int per = Vec<T>::per;
  const V *s = reinterpret_cast<const V *>(src);
#pragma unroll
  for (int q = 0; q < kRec / per; ++q) {
    V v = s[q];
    if constexpr (per == 4) {
      dst[4 * q] = v.x; dst[4 * q + 1] = v.y; dst[4 * q + 2] = v.z; dst[4 * q + 3] = v.w;
    } else {
      dst[2 * q] = v.x; dst[2 * q + 1] = v.y;
    }
  }
}

// One X row from a TMA stage written with SWIZZLE_128B.  The swizzle XORs the
// 16-byte chunk index (address bits 4..6) with address bits 7..9.  FP64 rows
// are 128 B, so chunk q of row r sits at chunk q ^ (r & 7) of that row; FP32
// rows are 64 B, two per 128-byte line, so chunk q of row r is chunk
// (((r & 1) << 2) | q) ^ ((r >> 1) & 7) of line r >> 1.  Consecutive rows read
// by 8 consecutive lanes then hit 8 distinct 16-byte bank groups.
template <typename T>
__device__ __forceinline__ void lds_row_swz(const unsigned char *stg, int r, T (&dst)[kRec]) {
  using V = typename Vec<T>::V;
  constexpr int per = Vec<T>::per;
#pragma unroll
  for (int q = 0; q < kRec / per; ++q) {
    const unsigned char *addr;
    if constexpr (sizeof(T) == 4) {
      addr = stg + (size_t)(r >> 1) * 128 + (((((r & 1) << 2) | q) ^ ((r >> 1) & 7)) << 4);
    } else {
      addr = stg + (size_t)r * 128 + ((q ^ (r & 7)) << 4);
    }
    const V v = *reinterpret_cast<const V *>(addr);
    if constexpr (per == 4) {
      dst[4 * q] = v.x; dst[4 * q + 1] = v.y; dst[4 * q + 2] = v.z; dst[4 * q + 3] = v.w;
    } else {
      dst[2 * q] = v.x; dst[2 * q + 1] = v.y;
    }
  }
}

// ---- mbarrier / TMA primitives (PTX) -------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// Test the phase; a thread whose phase is not complete is suspended until it
// completes or `suspend_ns` pass, so waiting warps do not spin on issue slots.
constexpr unsigned kSuspendNs = 200000;
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity,
                                              unsigned suspend_ns = kSuspendNs) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(suspend_ns)
      : "memory");
  return ok != 0;
}
// Suspend hint of a wait bounded by `limit` clocks: never longer than the bound
// (about 2 clocks per ns at the SM's clock), so a short bound runs out promptly.
__device__ __forceinline__ unsigned suspend_for(long long limit) {
  return limit >= 2LL * kSuspendNs ? kSuspendNs : (unsigned)(limit >> 1);
}
// Bounded wait: false on timeout (flag raised) or when another warp aborted.
// `limit` is the bound in SM clocks (<= 0: kWaitCycles).  The first test uses
// a fixed suspend hint, so that it does not wait on the loads of `limit` and
// `err`: on the usual path, where the phase is already complete, neither is
// needed.  A bound shorter than the hint runs out after the hint instead (a
// test-only case).
constexpr unsigned kFirstSuspendNs = 1000;
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, int *err,
                                          volatile int *abort, long long limit = 0) {
  if (mbar_try_wait(bar, parity, kFirstSuspendNs)) return true;
  if (limit <= 0) limit = kWaitCycles;
  const unsigned ns = suspend_for(limit);
  const long long t0 = clock64();
  for (;;) {
    if (mbar_try_wait(bar, parity, ns)) return true;
    if (*abort) return false;
    if (clock64() - t0 > limit) {
      atomicOr(err, kErrTimeout);
      *abort = 1;
      return false;
    }
  }
}
// The producer's wait for a free stage: it sleeps between polls, so that
// while the compute warps work it takes almost no issue slots from the warps
// that share its SM sub-partition.
__device__ __forceinline__ bool mbar_wait_sleep(uint64_t *bar, unsigned parity, int *err,
                                                volatile int *abort, long long limit = 0) {
  if (mbar_try_wait(bar, parity, kFirstSuspendNs)) return true;
  if (limit <= 0) limit = kWaitCycles;
  const unsigned sus = suspend_for(limit);
  const long long t0 = clock64();
  unsigned ns = 64;
  for (;;) {
    __nanosleep(ns);
    if (mbar_try_wait(bar, parity, sus)) return true;
    if (ns < 512) ns <<= 1;
    if (*abort) return false;
    if (clock64() - t0 > limit) {
      atomicOr(err, kErrTimeout);
      *abort = 1;
      return false;
    }
  }
}
__device__ __forceinline__ void tma_load_2d(void *dst, const void *tmap, int x, int y,
                                            uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(tmap), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
// Warm L2 with a contiguous range ahead of its TMA load (no completion to wait for).
__device__ __forceinline__ void prefetch_l2(const void *src, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes,
                                          uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void atomic_add_f64(double *addr, double v) { atomicAdd(addr, v); }

template <typename T> __device__ __forceinline__ T int_as_rec(int v);
template <> __device__ __forceinline__ float int_as_rec<float>(int v) { return __int_as_float(v); }
template <> __device__ __forceinline__ double int_as_rec<double>(int v) { return (double)v; }

template <typename T>
__global__ void __launch_bounds__(128) k_plan(T *coef, const int *set_begin, int O, int slack,
                                              int half_bytes, int slot_bytes, int *i0max_tab,
                                              int *err) {
  const int sidx = blockIdx.x;
  const int pb = set_begin[sidx], pe = set_begin[sidx + 1];
  for (int o = threadIdx.x; o < O; o += blockDim.x) {
    int lo = 0x7fffffff, hi = -0x7fffffff;
    for (int p = pb; p < pe; ++p) {
      const int i0 = rec_i0_of<T>(coef[((size_t)p * O + o) * kRec + slot::i0]);
      lo = min(lo, i0);
      hi = max(hi, i0);
    }
    if (hi - lo > slack) atomicOr(err, kErrWindow);
    i0max_tab[(size_t)sidx * O + o] = hi;
    for (int p = pb; p < pe; ++p) {
      T *rec = coef + ((size_t)p * O + o) * kRec;
      const int off = min(hi - rec_i0_of<T>(rec[slot::i0]), slack);
      rec[slot::off] = int_as_rec<T>(off);
      if (sizeof(T) == 4) {  // split window: slot x in half x & 1, word x >> 1
        const int x = off + 1, r = x & 1, q = x >> 1;
        rec[slot::w0] = int_as_rec<T>(r * half_bytes + slot_bytes * q);
        rec[slot::w1] = int_as_rec<T>((1 - r) * half_bytes + slot_bytes * (q + r));
      }
    }
  }
}

// Item decomposition shared by both pipelines.
template <typename T, int NW>
struct Item {
  int sidx, p_begin, p_end, o_begin, o_end, opw, nobs, k_begin, k_end;
  __device__ __forceinline__ Item(const FwdArgs<T> &a, int item, int w) {
    const int ng = a.n_obs_groups;
    // observer group fastest (groups share the set's X rows in L2), then the
    // time segments of one set, then the sets, largest first so that the
    // last CTAs to start are the shortest
    const int g = item % ng;
    const int rest = item / ng;
    const int q = a.seg_lo + rest % a.seg_cnt;
    const int r2 = rest / a.seg_cnt;
    sidx = a.set_order ? a.set_order[r2] : r2;
    p_begin = a.set_begin[sidx];
    p_end = a.set_begin[sidx + 1];
    opw = a.obs_per_cta / NW;
    o_begin = g * a.obs_per_cta;
    o_end = min(a.O, o_begin + a.obs_per_cta);
    k_begin = q * a.seg_len;
    k_end = min(a.ntp, k_begin + a.seg_len);
    nobs = 0;
    for (int m = 0; m < opw; ++m)
      if (o_begin + w + NW * m < o_end) nobs = m + 1;
  }
};

// Per-observer largest shift of the panel set (from the plan); zero windows.
template <typename T, int NW>
__device__ __forceinline__ void item_prologue(const FwdArgs<T> &a, const Item<T, NW> &it,
                                              int w, T *wwin, int *s_i0max) {
  const int lane = threadIdx.x & 31;
  if (lane < it.nobs)
    s_i0max[lane] = a.i0max_tab[(size_t)it.sidx * a.O + it.o_begin + w + NW * lane];
  for (int i = lane; i < it.nobs * a.wfl; i += 32) wwin[i] = T(0);
  __syncwarp();
}

// Signal, moment and the two spline-node updates of one (panel, observer),
// one sample per lane per block: read-modify-write of the window; the two
// node updates of neighbouring lanes meet in one bin, so they are separated
// by __syncwarp.
template <typename T, int TK>
__device__ __forceinline__ void accumulate(const T (&x)[TK][kRec], const T (&c)[kRec], T *wm) {
  T gv[TK], mv[TK];
#pragma unroll
  for (int j = 0; j < TK; ++j) {
    T g0 = c[0] * x[j][0], m0 = c[0] * x[j][8];
#pragma unroll
    for (int s = 1; s < 8; ++s) {
      g0 = fma(c[s], x[j][s], g0);
      m0 = fma(c[s], x[j][8 + s], m0);
    }
    gv[j] = g0;
    mv[j] = m0;
  }
#pragma unroll
  for (int j = 0; j < TK; ++j) {
    T v = wm[32 * j];
    v = fma(c[8], gv[j], v);
    v = fma(c[10], mv[j], v);
    wm[32 * j] = v;
  }
  __syncwarp();
#pragma unroll
  for (int j = 0; j < TK; ++j) {
    T v = wm[32 * j - 1];
    v = fma(c[9], gv[j], v);
    v = fma(c[11], mv[j], v);
    wm[32 * j - 1] = v;
  }
  __syncwarp();
}

// Flush the first CH (complete) bins of every window to p_out and slide.
template <typename T, int CH, int NW>
__device__ __forceinline__ void flush_slide(const FwdArgs<T> &a, const Item<T, NW> &it, int w,
                                            T *wwin, const int *s_i0max, int k0) {
  const int lane = threadIdx.x & 31;
  const int win = a.win;
  for (int m = 0; m < it.nobs; ++m) {
    const int o = it.o_begin + w + NW * m;
    T *wm = wwin + (size_t)m * win;
    const int wbase = k0 - s_i0max[m] - 1;
    const int nvalid = a.n_valid[o];
    double *po = a.p_out + (size_t)o * a.nt;
    for (int t = lane; t < CH; t += 32) {
      const int bin = wbase + t;
      const T v = wm[t];
      if (bin >= 0 && bin < nvalid && v != T(0)) atomic_add_f64(po + bin, (double)v);
    }
    __syncwarp();
    for (int t = lane; t < win - CH; t += 32) wm[t] = wm[CH + t];  // win - CH <= CH
    __syncwarp();
    for (int t = win - CH + lane; t < win; t += 32) wm[t] = T(0);
    __syncwarp();
  }
}

// Segment end: the remaining window holds partial bins of the next segment.
template <typename T, int CH, int NW>
__device__ __forceinline__ void flush_tail(const FwdArgs<T> &a, const Item<T, NW> &it, int w,
                                           T *wwin, const int *s_i0max) {
  const int lane = threadIdx.x & 31;
  const int win = a.win;
  for (int m = 0; m < it.nobs; ++m) {
    const int o = it.o_begin + w + NW * m;
    T *wm = wwin + (size_t)m * win;
    const int wbase = it.k_end - s_i0max[m] - 1;
    const int nvalid = a.n_valid[o];
    double *po = a.p_out + (size_t)o * a.nt;
    for (int t = lane; t < win - CH; t += 32) {
      const int bin = wbase + t;
      const T v = wm[t];
      if (bin >= 0 && bin < nvalid && v != T(0)) atomic_add_f64(po + bin, (double)v);
    }
  }
  __syncwarp();
}

// ---- direct-load pipeline --------------------------------------------------
template <typename T, int TK, int NW>
__device__ __forceinline__ void process_item_direct(const FwdArgs<T> &a, int item, T *smem,
                                                    int *st) {
  static_assert(sizeof(T) == 8, "scalar consumers read the 16-value FP64 record");
  constexpr int CH = 32 * TK;
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const Item<T, NW> it(a, item, w);
  T *wwin = smem + (size_t)w * it.opw * a.wfl;
  int *s_i0max = st + w * kMaxObsPerWarp;
  item_prologue<T, NW>(a, it, w, wwin, s_i0max);
  for (int k0 = it.k_begin; k0 < it.k_end; k0 += CH) {
    for (int p = it.p_begin; p < it.p_end; ++p) {
      T x[TK][kRec];
      const T *Xp = a.X + ((size_t)p * a.x_ld + k0 % a.x_ld + lane) * kRec;
#pragma unroll
      for (int j = 0; j < TK; ++j) load16<T>(Xp + (size_t)j * 32 * kRec, x[j]);
      const T *rec0 = a.coef + (size_t)p * a.O * kRec;
      for (int m = 0; m < it.nobs; ++m) {
        const int o = it.o_begin + w + NW * m;
        T c[kRec];
        load16<T>(rec0 + (size_t)o * kRec, c);
        T *wm = wwin + (m * a.win + 1 + lane + rec_i0_of<T>(c[slot::off]));
        accumulate<T, TK>(x, c, wm);
      }
    }
    flush_slide<T, CH, NW>(a, it, w, wwin, s_i0max, k0);
  }
  flush_tail<T, CH, NW>(a, it, w, wwin, s_i0max);
}

// ---- TMA pipeline ------------------------------------------------------------
struct PipeState {
  uint64_t *full, *empty;
  unsigned char *stage0;
  unsigned stage_bytes, x_bytes;
  int nst;
  volatile int *abort;
  int *released;  // in-line producer: per-stage count of warps done with it
  int *issued;    // in-line producer: steps issued so far (for the drain)
  const void *tmap;  // tensor map of the X rows being streamed
  int *err;          // device error flag and the bound of each wait (SM clocks):
  long long wait_cycles;  // the same for every surface of a launch
};

// Threads per CTA: compute warps, plus the producer warp of the TMA pipeline
// (pipe 1); the in-line producer (pipe 2) has none.
template <int NW, int PIPE>
constexpr int cta_threads() { return (NW + (PIPE == 1 ? 1 : 0)) * 32; }

// In-line producer: load step j (in-item index) of `it` into stage `slot`.
// Step j covers panel p_begin + j % np and chunk k_begin + (j / np) CH.
template <typename T, int TK, int NW>
__device__ __forceinline__ void issue_step(const FwdArgs<T> &a, const Item<T, NW> &it,
                                           const PipeState &ps, int j, unsigned slot) {
  constexpr int CH = 32 * TK;
  const int np = it.p_end - it.p_begin;
  const int p = it.p_begin + j % np;
  const int k0 = it.k_begin + (j / np) * CH;
  const unsigned cbytes = (unsigned)((it.o_end - it.o_begin) * kRec * sizeof(T));
  uint64_t *bar = &ps.full[slot];
  unsigned char *dst = ps.stage0 + (size_t)slot * ps.stage_bytes;
  mbar_expect_tx(bar, ps.x_bytes + cbytes);
  const int row = p * a.x_ld + k0 % a.x_ld;  // tensor rows are 128 bytes
  tma_load_2d(dst, ps.tmap, 0, sizeof(T) == 4 ? row >> 1 : row, bar);
  bulk_load(dst + ps.x_bytes, a.coef + ((size_t)p * a.O + it.o_begin) * kRec, cbytes, bar);
}

// Producer (one lane): stream the steps of one item into the stage ring, and
// warm L2 with the rows and records kPrefetchSteps steps beyond the ring so
// that the stage loads hit L2 instead of waiting for HBM.
constexpr int kPrefetchSteps = 8;

template <typename T, int TK, int NW>
__device__ __forceinline__ void produce_item(const FwdArgs<T> &a, const Item<T, 1> &it,
                                             const PipeState &ps, unsigned &step) {
  constexpr int CH = 32 * TK;
  const unsigned cbytes = (unsigned)((it.o_end - it.o_begin) * kRec * sizeof(T));
  const int np = it.p_end - it.p_begin;
  const int nsteps = np * ((it.k_end - it.k_begin) / CH);
  // Step idx covers panel p_begin + idx % np, chunk k_begin + (idx / np) CH.
  // Both cursors (the load and the L2 prefetch running ahead of it) advance
  // incrementally: this lane's per-step work stays short, since it is on the
  // critical path of every stage refill.
  // the item's constants in registers (the batched kernels read their
  // arguments through a pointer, which every copy's memory clobber would make
  // them re-read)
  const T *const X = a.X;
  const T *const coef = a.coef;
  const int x_ld = a.x_ld, O = a.O;
  int *const err = ps.err;
  const long long wait_cycles = ps.wait_cycles;
  auto src_x = [&](int pp, int kc) {
    return X + ((size_t)(it.p_begin + pp) * x_ld + it.k_begin % x_ld + kc * CH) * kRec;
  };
  auto src_c = [&](int pp) {
    return coef + ((size_t)(it.p_begin + pp) * O + it.o_begin) * kRec;
  };
  if (a.withhold) return;  // testing: no copies, so every consumer wait runs out
  int fp = 0, fk = 0;  // prefetch cursor (panel offset, chunk)
  auto prefetch_next = [&]() {
    prefetch_l2(src_x(fp, fk), ps.x_bytes);
    prefetch_l2(src_c(fp), cbytes);
    if (++fp == np) {
      fp = 0;
      ++fk;
    }
  };
  const int lead = min(nsteps, ps.nst + kPrefetchSteps);
  for (int idx = 0; idx < lead; ++idx) prefetch_next();
  int cp = 0, ck = 0;  // load cursor
  unsigned s = step % (unsigned)ps.nst, ph = (step / (unsigned)ps.nst) & 1u;
  for (int idx = 0; idx < nsteps; ++idx, ++step) {
    if (*ps.abort) return;
    if (idx + lead < nsteps) prefetch_next();
    if (step >= (unsigned)ps.nst &&
        !mbar_wait_sleep(&ps.empty[s], ph ^ 1u, err, ps.abort, wait_cycles))
      return;
    unsigned char *dst = ps.stage0 + (size_t)s * ps.stage_bytes;
    mbar_expect_tx(&ps.full[s], ps.x_bytes + cbytes);
    // tensor rows are 128 bytes: two FP32 samples or one FP64 sample
    const int row = (it.p_begin + cp) * x_ld + it.k_begin % x_ld + ck * CH;
    tma_load_2d(dst, ps.tmap, 0, sizeof(T) == 4 ? row >> 1 : row, &ps.full[s]);
    bulk_load(dst + ps.x_bytes, src_c(cp), cbytes, &ps.full[s]);
    if (++cp == np) {
      cp = 0;
      ++ck;
    }
    if (++s == (unsigned)ps.nst) {
      s = 0;
      ph ^= 1u;
    }
  }
}

template <typename T, int TK, int NW>
__device__ __forceinline__ void consume_item(const FwdArgs<T> &a, const Item<T, NW> &it,
                                             const PipeState &ps, unsigned &step, T *wwin,
                                             int *s_i0max, int w) {
  static_assert(sizeof(T) == 8, "scalar consumers read the 16-value FP64 record");
  constexpr int CH = 32 * TK;
  const int lane = threadIdx.x & 31;
  item_prologue<T, NW>(a, it, w, wwin, s_i0max);
  for (int k0 = it.k_begin; k0 < it.k_end; k0 += CH) {
    for (int p = it.p_begin; p < it.p_end; ++p, ++step) {
      const int s = (int)(step % (unsigned)ps.nst);
      const unsigned ph = (step / (unsigned)ps.nst) & 1u;
      if (!mbar_wait(&ps.full[s], ph, ps.err, ps.abort, ps.wait_cycles)) return;
      const unsigned char *stg = ps.stage0 + (size_t)s * ps.stage_bytes;
      T x[TK][kRec];
#pragma unroll
      for (int j = 0; j < TK; ++j) lds_row_swz<T>(stg, lane + 32 * j, x[j]);
      const T *crec = reinterpret_cast<const T *>(stg + ps.x_bytes);
      for (int m = 0; m < it.nobs; ++m) {
        const int o = it.o_begin + w + NW * m;
        T c[kRec];
        lds16<T>(crec + (size_t)(o - it.o_begin) * kRec, c);
        T *wm = wwin + (m * a.win + 1 + lane + rec_i0_of<T>(c[slot::off]));
        accumulate<T, TK>(x, c, wm);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&ps.empty[s]);
    }
    flush_slide<T, CH, NW>(a, it, w, wwin, s_i0max, k0);
  }
  flush_tail<T, CH, NW>(a, it, w, wwin, s_i0max);
}

// ---- FP32 consumer (mixed precision) ----------------------------------------
// FP32 X rows pair the consecutive samples 2r and 2r + 1 of each 64-sample
// block, so the 16-byte chunk c of pair row r holds (x_k[2c], x_k+1[2c],
// x_k[2c+1], x_k+1[2c+1]), k = 64 b + 2 r: one swizzled row read per lane
// gives both samples' series.  Lane l owns pair rows l + 32 t of a chunk
// (samples s = 64 t + 2 l and s + 1) and forms, per observer, G = sum_q c_q
// X_q and M likewise on the moments for both samples at once: (x_k[q],
// x_k+1[q]) is a register pair, and packed fma.rn.f32x2 with c_q in both
// halves computes the two samples' dot products.  A packed FMA issues in one
// slot and occupies the FMA pipe for two cycles, so the 16 multiply-adds of
// the two dot products take 8 issue slots instead of 16: the kernel is bound
// by instruction issue, not by the FMA pipe.  Results are those of scalar
// fmaf (both round each element to nearest).
// Sample s adds a G + cc M (left spline node) to window slot 1 + s + off and
// b G + dd M (right node) to slot s + off, so slot 1 + s + off receives
// a G_s + cc M_s + b G_s+1 + dd M_s+1.  For the first sample of a pair both
// nodes are the lane's own: the old slot value enters a chain of four FMAs.
// For the second, v = b G + dd M of the next sample comes from lane l + 1
// (lane 31: lane 0's pair of block t + 1), one shuffle per pair; the last
// block's lane 31 has no successor in the chunk, and the slot below the
// chunk (v of sample 0) is added by lane 0, so the chunk-crossing node is
// split between two chunks exactly once.
//
// Split windows: slot x of an observer's window lives in half x & 1 at word
// x >> 1, so the two slots of a lane's pair sit in different halves and 32
// lanes touch 32 consecutive words of one half per access: conflict-free for
// every offset.  The planner writes each record's two byte offsets (slots 14,
// 15: the words of slots off + 1 and off + 2 relative to the window), so the
// hot loop adds them to the lane's base and never branches on the shift.
// Within one (panel, observer) no two lanes touch the same slot; one
// __syncwarp per panel orders the next panel's shifted updates.
// Shared-space accesses by 32-bit address (the consumer addresses the stage
// ring and its windows explicitly, so no generic-address arithmetic).
// Window loads are not volatile: the compiler may hoist an observer's loads
// above the previous observer's stores (their windows never overlap), which
// hides their latency.  They stay after the previous panel's stores because
// their addresses derive from a token taken after that panel's __syncwarp.
__device__ __forceinline__ float lds_win(unsigned addr) {
  float v;
  asm("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr));
  return v;
}
__device__ __forceinline__ void sts_f32(unsigned addr, float v) {
  asm volatile("st.shared.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}

// Loads of stage data (X rows, records): not volatile, so the compiler may
// schedule them early; they stay after the stage's full-barrier wait because
// their addresses derive from stage_token(), which that wait orders.
__device__ __forceinline__ float4 lds_v4f32(unsigned addr) {
  float4 v;
  asm("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
      : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
      : "r"(addr));
  return v;
}
__device__ __forceinline__ uint2 lds_v2u32_stage(unsigned addr) {
  uint2 v;
  asm("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(addr));
  return v;
}
// The stage address as an opaque value produced after the barrier wait.
__device__ __forceinline__ unsigned stage_token(unsigned addr) {
  unsigned r;
  asm volatile("mov.u32 %0, %1;" : "=r"(r) : "r"(addr) : "memory");
  return r;
}
// x + (the value of the lane above, if there is one): the last lane keeps x.
__device__ __forceinline__ float add_from_lane_above(float x, float v) {
  float r;
  asm(
      "{\n\t.reg .pred p;\n\t.reg .f32 t;\n\t"
      "shfl.sync.down.b32 t|p, %2, 1, 0x1f, 0xffffffff;\n\t"
      "mov.f32 %0, %1;\n\t"
      "@p add.f32 %0, %1, t;\n\t}"
      : "=f"(r)
      : "f"(x), "f"(v));
  return r;
}

// The slots of one FP32 record that the consumer reads: c0..c7, a, b, cc, dd
// and the two window byte offsets (slots 14, 15).
struct Coef {
  float c[8], wa, wb, wcc, wdd;
  unsigned r0, r1;
};
__device__ __forceinline__ void lds_coef(unsigned rec, Coef &k) {
  static_assert(slot::c == 0 && slot::a == 8 && slot::b == 9 && slot::cc == 10 &&
                    slot::dd == 11 && slot::w0 == 14 && slot::w1 == 15,
                "record read as three 16-byte groups and one 8-byte pair");
  const float4 c0 = lds_v4f32(rec), c1 = lds_v4f32(rec + 16), w = lds_v4f32(rec + 32);
  const uint2 r = lds_v2u32_stage(rec + 4 * slot::w0);
  k.c[0] = c0.x; k.c[1] = c0.y; k.c[2] = c0.z; k.c[3] = c0.w;
  k.c[4] = c1.x; k.c[5] = c1.y; k.c[6] = c1.z; k.c[7] = c1.w;
  k.wa = w.x; k.wb = w.y; k.wcc = w.z; k.wdd = w.w;
  k.r0 = r.x;
  k.r1 = r.y;
}

// Value of a split-window entry: a plain FP32 sum, or a compensated pair
// (sum, compensation) whose value is sum - compensation (formed in FP64).
template <bool KAHAN> struct WinEntry;
template <> struct WinEntry<false> {
  using E = float;
  static __device__ __forceinline__ bool nz(E e) { return e != 0.f; }
  static __device__ __forceinline__ double value(E e) { return (double)e; }
  static __device__ __forceinline__ E zero() { return 0.f; }
};
template <> struct WinEntry<true> {
  using E = float2;
  static __device__ __forceinline__ bool nz(E e) { return e.x != 0.f || e.y != 0.f; }
  static __device__ __forceinline__ double value(E e) { return (double)e.x - (double)e.y; }
  static __device__ __forceinline__ E zero() { return make_float2(0.f, 0.f); }
};

// Flush the first CH (complete) bins of every split window to p_out and slide.
template <int CH, int NW, bool KAHAN>
__device__ __forceinline__ void flush_slide_split(const FwdArgs<float> &a,
                                                  const Item<float, NW> &it, int w, float *wwin,
                                                  const int *s_i0max, int k0) {
  using W = WinEntry<KAHAN>;
  using E = typename W::E;
  const int lane = threadIdx.x & 31;
  const int H = a.win >> 1;
  for (int m = 0; m < it.nobs; ++m) {
    const int o = it.o_begin + w + NW * m;
    E *wm = reinterpret_cast<E *>(wwin + (size_t)m * a.wfl);
    const int wbase = k0 - s_i0max[m] - 1;
    const int nvalid = a.n_valid[o];
    double *po = a.p_out + (size_t)o * a.nt;
#pragma unroll
    for (int hf = 0; hf < 2; ++hf)
      for (int q = lane; q < CH / 2; q += 32) {
        const int bin = wbase + 2 * q + hf;
        const E v = wm[hf * H + q];
        if (bin >= 0 && bin < nvalid && W::nz(v)) atomic_add_f64(po + bin, W::value(v));
      }
    __syncwarp();
#pragma unroll
    for (int hf = 0; hf < 2; ++hf)  // H - CH/2 <= CH/2: no overlap
      for (int q = lane; q < H - CH / 2; q += 32) wm[hf * H + q] = wm[hf * H + CH / 2 + q];
    __syncwarp();
#pragma unroll
    for (int hf = 0; hf < 2; ++hf)
      for (int q = H - CH / 2 + lane; q < H; q += 32) wm[hf * H + q] = W::zero();
    __syncwarp();
  }
}

// Segment end: the remaining split window holds partial bins of the next segment.
template <int CH, int NW, bool KAHAN>
__device__ __forceinline__ void flush_tail_split(const FwdArgs<float> &a,
                                                 const Item<float, NW> &it, int w, float *wwin,
                                                 const int *s_i0max) {
  using W = WinEntry<KAHAN>;
  using E = typename W::E;
  const int lane = threadIdx.x & 31;
  const int H = a.win >> 1;
  for (int m = 0; m < it.nobs; ++m) {
    const int o = it.o_begin + w + NW * m;
    const E *wm = reinterpret_cast<const E *>(wwin + (size_t)m * a.wfl);
    const int wbase = it.k_end - s_i0max[m] - 1;
    const int nvalid = a.n_valid[o];
    double *po = a.p_out + (size_t)o * a.nt;
#pragma unroll
    for (int hf = 0; hf < 2; ++hf)
      for (int q = lane; q < H - CH / 2; q += 32) {
        const int bin = wbase + 2 * q + hf;
        const E v = wm[hf * H + q];
        if (bin >= 0 && bin < nvalid && W::nz(v)) atomic_add_f64(po + bin, W::value(v));
      }
  }
  __syncwarp();
}

// Compensated (Kahan) update of a window entry (sum, compensation) by y.
__device__ __forceinline__ float2 kahan_add(float2 w, float y) {
  const float yc = __fsub_rn(y, w.y);
  const float t = __fadd_rn(w.x, yc);
  return make_float2(t, __fsub_rn(__fsub_rn(t, w.x), yc));
}
__device__ __forceinline__ float2 lds_win2(unsigned addr) {
  float2 v;
  asm("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr));
  return v;
}
__device__ __forceinline__ void sts_f32x2(unsigned addr, float2 v) {
  asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
}

// Packed FP32 pairs (fma.rn.f32x2 and friends): element-wise IEEE round-to-
// nearest operations on two floats held in a 64-bit register pair.  One
// packed FMA issues in one slot and keeps the FMA pipe busy for two cycles.
using f32x2 = unsigned long long;
__device__ __forceinline__ void lds_v2f32x2(unsigned addr, f32x2 &a, f32x2 &b) {
  asm("ld.shared.v2.b64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "r"(addr));
}
__device__ __forceinline__ f32x2 f2_dup(float x) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ f32x2 f2_mul(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f32x2 f2_fma(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ void f2_split(f32x2 v, float &lo, float &hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

template <int TK, int NW, bool PF, int PIPE, bool KAHAN>
__device__ __forceinline__ void consume_item_f32(const FwdArgs<float> &a,
                                                 const Item<float, NW> &it,
                                                 const PipeState &ps, unsigned &step,
                                                 float *wwin, int *s_i0max, int w) {
  constexpr int CH = 32 * TK;
  constexpr int NP = TK / 2;  // pair rows per lane
  constexpr unsigned RB = kRec * 4;  // record bytes
  const int lane = threadIdx.x & 31;
  item_prologue<float, NW>(a, it, w, wwin, s_i0max);
  // Window of observer m starts at win_s + m * win_b; the record's byte
  // offsets r0 / r1 locate slots off + 1 / off + 2 of lane 0, block 0, and
  // block t adds 32 words.
  constexpr unsigned EB = KAHAN ? 8u : 4u;  // bytes per window entry
  const unsigned win_b = (unsigned)a.wfl * 4u;
  const unsigned win_s = smem_u32(wwin) + (unsigned)lane * EB;
  const unsigned stage0 = smem_u32(ps.stage0);
  // X pair row r = lane + 32 t of a stage: 16-byte chunk c at c ^ (lane & 7).
  // Stages are 1024-byte aligned and a pair row is 128 bytes, so bits 4..6 of
  // (stage + 128 lane) are zero and chunk c of the lane's row sits at
  // (stage + 128 lane + 16 (lane & 7)) ^ 16 c: one XOR per chunk.
  const unsigned xrow = (unsigned)lane * 128u + (((unsigned)lane & 7u) << 4);
  const bool first = lane == 0;
  unsigned s = step % (unsigned)ps.nst, ph = (step / (unsigned)ps.nst) & 1u;
  const int nsteps = (it.p_end - it.p_begin) * ((it.k_end - it.k_begin) / CH);
  int j = 0;  // in-item step index
  for (int k0 = it.k_begin; k0 < it.k_end; k0 += CH) {
    for (int p = it.p_begin; p < it.p_end; ++p, ++step, ++j) {
      if (!mbar_wait(&ps.full[s], ph, ps.err, ps.abort, ps.wait_cycles)) return;
      const unsigned stg = stage_token(stage0 + s * ps.stage_bytes);
      // XP[t][q] = (value q of sample 2r, value q of sample 2r + 1): the 16-byte
      // chunk c holds the pairs of values 2c and 2c + 1
      f32x2 XP[NP][kRec];
      const unsigned xb = stg + xrow;
#pragma unroll
      for (int t = 0; t < NP; ++t) {
#pragma unroll
        for (int c = 0; c < 8; ++c)
          lds_v2f32x2((xb ^ ((unsigned)c << 4)) + 4096u * t, XP[t][2 * c], XP[t][2 * c + 1]);
      }
      const unsigned crec = stg + ps.x_bytes + (unsigned)w * RB;
      // window base of this panel's updates, ordered after the previous
      // panel's stores (see lds_win)
      const unsigned wtok = stage_token(win_s);
      // one (panel, observer): the spline-node updates of the lane's samples
      auto observer = [&](int m, const Coef &k) {
        const unsigned base = wtok + (unsigned)m * win_b;
        const unsigned A0 = base + k.r0, A1 = base + k.r1;
        // signal G and moment M of both samples of each pair row: packed dot
        // products c . X with the coefficient in both halves of a register
        // pair (issued after the window loads, which then hide their latency)
        f32x2 Gp[NP], Mp[NP];
        auto dots = [&]() {
          {
            const f32x2 cp = f2_dup(k.c[0]);
#pragma unroll
            for (int t = 0; t < NP; ++t) {
              Gp[t] = f2_mul(cp, XP[t][0]);
              Mp[t] = f2_mul(cp, XP[t][8]);
            }
          }
#pragma unroll
          for (int q = 1; q < 8; ++q) {
            const f32x2 cp = f2_dup(k.c[q]);
#pragma unroll
            for (int t = 0; t < NP; ++t) {
              Gp[t] = f2_fma(cp, XP[t][q], Gp[t]);
              Mp[t] = f2_fma(cp, XP[t][8 + q], Mp[t]);
            }
          }
        };
        if constexpr (!KAHAN) {
          float s0[NP], s1[NP], v0[NP];
#pragma unroll
          for (int t = 0; t < NP; ++t) {
            s0[t] = lds_win(A0 + 128u * t);
            s1[t] = lds_win(A1 + 128u * t);
          }
          // lane 0: the slot below the chunk (other lanes read a slot of the
          // lane below, in the window, and discard it); no lane stores to it
          // before lane 0 does, so it is read early to hide the latency
          const float e_old = lds_win(A1 - 4u);
          dots();
#pragma unroll
          for (int t = 0; t < NP; ++t) {
            float G0, G1, M0, M1;
            f2_split(Gp[t], G0, G1);
            f2_split(Mp[t], M0, M1);
            // slot of the pair's first sample: both spline nodes are this lane's
            s0[t] = fmaf(k.wdd, M1, fmaf(k.wb, G1, fmaf(k.wcc, M0, fmaf(k.wa, G0, s0[t]))));
            // slot of the second: its left node, the right one comes from above
            s1[t] = fmaf(k.wcc, M1, fmaf(k.wa, G1, s1[t]));
            // right node of the pair's first sample, for the lane below
            v0[t] = fmaf(k.wdd, M0, k.wb * G0);
          }
#pragma unroll
          for (int t = 0; t < NP; ++t) sts_f32(A0 + 128u * t, s0[t]);
#pragma unroll
          for (int t = 0; t + 1 < NP; ++t) {
            // lane 0 serves lane 31 with block t + 1's first sample
            const float x = first ? v0[t + 1] : v0[t];
            s1[t] += __shfl_sync(0xffffffffu, x, (lane + 1) & 31);
          }
          s1[NP - 1] = add_from_lane_above(s1[NP - 1], v0[NP - 1]);
#pragma unroll
          for (int t = 0; t < NP; ++t) sts_f32(A1 + 128u * t, s1[t]);
          // lane 0: the slot below the chunk (a C++ condition, so the compiler
          // predicates the store on `first` computed once, not per observer)
          if (first) sts_f32(A1 - 4u, e_old + v0[0]);
        } else {
          // compensated: each slot is (sum, compensation); every panel's
          // contribution to a slot is formed first, then added by Kahan's rule
          float2 w0[NP], w1[NP];
#pragma unroll
          for (int t = 0; t < NP; ++t) {
            w0[t] = lds_win2(A0 + 256u * t);
            w1[t] = lds_win2(A1 + 256u * t);
          }
          const float2 e_old = lds_win2(A1 - 8u);
          dots();
          float y0[NP], y1[NP], v0[NP];
#pragma unroll
          for (int t = 0; t < NP; ++t) {
            float G0, G1, M0, M1;
            f2_split(Gp[t], G0, G1);
            f2_split(Mp[t], M0, M1);
            y0[t] = fmaf(k.wdd, M1, fmaf(k.wb, G1, fmaf(k.wcc, M0, k.wa * G0)));
            y1[t] = fmaf(k.wcc, M1, k.wa * G1);
            v0[t] = fmaf(k.wdd, M0, k.wb * G0);
          }
#pragma unroll
          for (int t = 0; t < NP; ++t) sts_f32x2(A0 + 256u * t, kahan_add(w0[t], y0[t]));
#pragma unroll
          for (int t = 0; t + 1 < NP; ++t) {
            const float x = first ? v0[t + 1] : v0[t];
            y1[t] += __shfl_sync(0xffffffffu, x, (lane + 1) & 31);
          }
          y1[NP - 1] = add_from_lane_above(y1[NP - 1], v0[NP - 1]);
#pragma unroll
          for (int t = 0; t < NP; ++t) sts_f32x2(A1 + 256u * t, kahan_add(w1[t], y1[t]));
          if (first) sts_f32x2(A1 - 8u, kahan_add(e_old, v0[0]));
        }
      };
      // PF: read the next observer's record while this one computes, else
      // read each record right before its use.  A warp with the full count of
      // observers runs them without an exit test, so the compiler may overlap
      // one observer's tail with the next one's loads and arithmetic.
      auto run = [&](auto full) {
        constexpr bool kFull = decltype(full)::value;
        const int n = kFull ? kMaxObsPerWarpF32 : it.nobs;
        auto rec = [&](int m) { return crec + (unsigned)m * NW * RB; };
        Coef k;
        if (PF && n > 0) lds_coef(rec(0), k);
#pragma unroll
        for (int m = 0; m < kMaxObsPerWarpF32; ++m) {
          if (!kFull && m >= n) break;
          if (!PF) lds_coef(rec(m), k);
          Coef kn;
          if (PF && m + 1 < n) lds_coef(rec(m + 1), kn);
          observer(m, k);
          if (PF) k = kn;
        }
      };
      if (it.nobs == kMaxObsPerWarpF32)
        run(std::true_type{});
      else
        run(std::false_type{});
      __syncwarp();
      if constexpr (PIPE == 2) {
        // the last warp done with this stage refills it with step j + nst
        if (lane == 0) {
          __threadfence_block();
          const int done = atomicAdd(&ps.released[s], 1) + 1;
          if (done % NW == 0 && j + ps.nst < nsteps && !a.withhold) {
            __threadfence_block();
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue_step<float, TK, NW>(a, it, ps, j + ps.nst, s);
            atomicMax(ps.issued, (int)step + ps.nst + 1);
          }
        }
      } else {
        if (lane == 0) mbar_arrive(&ps.empty[s]);
      }
      if (++s == (unsigned)ps.nst) {
        s = 0;
        ph ^= 1u;
      }
    }
    flush_slide_split<CH, NW, KAHAN>(a, it, w, wwin, s_i0max, k0);
  }
  flush_tail_split<CH, NW, KAHAN>(a, it, w, wwin, s_i0max);
}

// Wait until every copy the producer issued has landed, always with the full
// bound (never the handle's test bound): the CTA must not exit while a copy
// into its shared memory is in flight.
__device__ __forceinline__ void drain_copies(const PipeState &ps, unsigned step, int *err) {
  const unsigned first = step > (unsigned)ps.nst ? step - (unsigned)ps.nst : 0u;
  volatile int never = 0;
  for (unsigned t = first; t < step; ++t) {
    const int s = (int)(t % (unsigned)ps.nst);
    mbar_wait(&ps.full[s], (t / (unsigned)ps.nst) & 1u, err, &never);
  }
}

template <typename T, int TK, int NW>
__device__ __forceinline__ unsigned char *pipe_setup(unsigned char *raw, int obs_per_cta,
                                                     int nst, uint64_t *bars,
                                                     volatile int *abort, PipeState &ps,
                                                     int *released = nullptr,
                                                     int *issued = nullptr) {
  constexpr int CH = 32 * TK;
  const unsigned base = smem_u32(raw);
  unsigned char *al = raw + ((1024u - (base & 1023u)) & 1023u);
  ps.x_bytes = CH * kRec * sizeof(T);
  ps.stage_bytes = (ps.x_bytes + obs_per_cta * kRec * sizeof(T) + 1023u) & ~1023u;
  ps.nst = nst;
  ps.stage0 = al;
  ps.full = bars;
  ps.empty = bars + nst;
  ps.abort = abort;
  ps.released = released;
  ps.issued = issued;
  if (threadIdx.x == 0) {
    for (int s = 0; s < nst; ++s) {
      mbar_init(&ps.full[s], 1);
      mbar_init(&ps.empty[s], NW);
      if (released) released[s] = 0;
    }
    if (issued) *issued = 0;
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  return al + (size_t)nst * ps.stage_bytes;  // windows follow the stages
}

constexpr int kMaxStages = 8;

// CTAs per SM the register budget is sized for: TMA shapes with 4 compute
// warps run 3 (TK = 4) or 2 (TK = 8) per SM, with 8 compute warps 2 or 1.
template <int TK, int NW, int PIPE>
struct MinBlocks {
  static constexpr int v = !PIPE ? 1
                           : PIPE == 2 ? (NW <= 4 ? (TK <= 4 ? 4 : 2) : (TK <= 4 ? 2 : 1))
                                       : (NW <= 4 ? (TK <= 4 ? 3 : 2) : (TK <= 4 ? 2 : 1));
};

template <typename T, int TK, int NW, int PIPE, int ACC>
__device__ __forceinline__ void forward_cta(const FwdArgs<T> &a, const void *tmap, int nst,
                                            int item, int *err, long long wait_cycles) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int st[NW * kMaxObsPerWarp];
  if constexpr (PIPE == 0) {
    (void)tmap;
    process_item_direct<T, TK, NW>(a, item, reinterpret_cast<T *>(smem_raw), st);
  } else if constexpr (PIPE == 2) {
    static_assert(sizeof(T) == 4 && ACC >= 3, "the in-line producer serves the FP32 consumer");
    __shared__ __align__(8) uint64_t bars[2 * kMaxStages];
    __shared__ int released[kMaxStages];
    __shared__ int issued;
    __shared__ int abort_flag;
    PipeState ps;
    unsigned char *wbase = pipe_setup<T, TK, NW>(smem_raw, a.obs_per_cta, nst, bars,
                                                 &abort_flag, ps, released, &issued);
    ps.tmap = tmap;
    ps.err = err;
    ps.wait_cycles = wait_cycles;
    const int w = threadIdx.x >> 5;
    const Item<T, NW> it(a, item, w);
    if (threadIdx.x == 0 && !a.withhold) {  // fill the ring
      const int nsteps = (it.p_end - it.p_begin) * ((it.k_end - it.k_begin) / (32 * TK));
      const int n0 = min(nst, nsteps);
      for (int j = 0; j < n0; ++j) issue_step<T, TK, NW>(a, it, ps, j, (unsigned)j);
      atomicMax(&issued, n0);
    }
    unsigned step = 0;
    T *wwin = reinterpret_cast<T *>(wbase) + (size_t)w * it.opw * a.wfl;
    consume_item_f32<TK, NW, ACC >= 4, 2, ACC == 5>(a, it, ps, step, wwin, st + w * kMaxObsPerWarp,
                                                      w);
    __syncthreads();
    if (threadIdx.x == 0 && abort_flag) drain_copies(ps, (unsigned)issued, err);
  } else {
    __shared__ __align__(8) uint64_t bars[2 * kMaxStages];
    __shared__ int abort_flag;
    PipeState ps;
    unsigned char *wbase = pipe_setup<T, TK, NW>(smem_raw, a.obs_per_cta, nst, bars,
                                                 &abort_flag, ps);
    ps.tmap = tmap;
    ps.err = err;
    ps.wait_cycles = wait_cycles;
    const int w = threadIdx.x >> 5;
    unsigned step = 0;
    if (w == NW) {
      if ((threadIdx.x & 31) == 0) {
        const Item<T, 1> it(a, item, 0);
        produce_item<T, TK, NW>(a, it, ps, step);
        drain_copies(ps, step, err);
      }
    } else {
      const Item<T, NW> it(a, item, w);
      T *wwin = reinterpret_cast<T *>(wbase) + (size_t)w * it.opw * a.wfl;
      if constexpr (ACC >= 3 && sizeof(T) == 4) {
        consume_item_f32<TK, NW, ACC >= 4, 1, ACC == 5>(a, it, ps, step, wwin, st + w * kMaxObsPerWarp,
                                                        w);
      } else {
        consume_item<T, TK, NW>(a, it, ps, step, wwin, st + w * kMaxObsPerWarp, w);
      }
    }
  }
}


template <typename T, int TK, int NW, int PIPE, int ACC>
__global__ void __launch_bounds__((cta_threads<NW, PIPE>()), (MinBlocks<TK, NW, PIPE>::v))
    k_forward(FwdArgs<T> a, const __grid_constant__ CUtensorMap tm, int nst) {
  forward_cta<T, TK, NW, PIPE, ACC>(a, &tm, nst, blockIdx.x, a.err, a.wait_cycles);
}

// Same CTA program for the long-sample-block shapes (TK = 8), which need
// about 190 registers: capped at 200 so that two CTAs still share an SM.
template <typename T, int TK, int NW, int PIPE, int ACC>
__global__ void __maxnreg__(200) k_forward_wide(FwdArgs<T> a,
                                                const __grid_constant__ CUtensorMap tm, int nst) {
  forward_cta<T, TK, NW, PIPE, ACC>(a, &tm, nst, blockIdx.x, a.err, a.wait_cycles);
}

// Persistent form: CTAs pull work items of several surfaces from one queue.
// The surfaces' arguments, item offsets and X descriptors are one
// __grid_constant__ parameter block (kMaxBatchSurf surfaces at most).
//
// With a producer warp (PIPE = 1) items flow back to back: the producer lane
// claims an item, publishes its index in a small ring (s_q, one mbarrier per
// slot) and streams its steps into the stage ring, whose step count runs on
// across items; each compute warp takes the next published item as soon as it
// has flushed its windows for the previous one.  There is no CTA-wide barrier
// between items, so the copies of an item's first stages are in flight while
// the compute warps finish the item before it.  A slot is rewritten kItemQ
// publications later; the producer can run at most `nst` steps (hence items)
// ahead of the slowest compute warp, so kItemQ > kMaxStages keeps every
// publication readable until each warp has taken it.
constexpr int kItemQ = 16;
// kernel parameters may take up to 32764 bytes (CUDA 12.1 and later)
static_assert(sizeof(BatchParams<double>) + 64 <= 32764, "batched launch parameters too large");
static_assert(kItemQ > kMaxStages, "the item ring must outlast the deepest stage ring");

// Surface of a batched item (prefix[lo] <= item < prefix[lo + 1]).
__device__ __forceinline__ int batch_surface(const int *prefix, int n_surf, int item) {
  int lo = 0, hi = n_surf - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <typename T, int TK, int NW, int PIPE, int ACC>
__device__ __forceinline__ void forward_batch_cta(const BatchParams<T> &P, int *counter, int nst) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int st[NW * kMaxObsPerWarp];
  __shared__ int s_item;
  __shared__ __align__(8) uint64_t bars[2 * kMaxStages];
  __shared__ __align__(8) uint64_t qbar[kItemQ];
  __shared__ int s_q[kItemQ];
  __shared__ int abort_flag;
  __shared__ int released[kMaxStages];
  __shared__ int issued;
  const int n_surf = P.n_surf, total = P.total;
  const int *prefix = P.prefix;   // parameter space: read through the constant cache
  const FwdArgs<T> *args = P.a;
  if (threadIdx.x == 0) {
    s_item = atomicAdd(counter, 1);
    if constexpr (PIPE == 1)
      for (int q = 0; q < kItemQ; ++q) mbar_init(&qbar[q], 1);
  }
  __syncthreads();
  PipeState ps;
  unsigned char *wbase = smem_raw;
  if constexpr (PIPE != 0) {
    int maxo = 0;
    for (int i = 0; i < n_surf; ++i) maxo = max(maxo, args[i].obs_per_cta);
    // (its barrier also orders the item ring's initialisation above)
    wbase = pipe_setup<T, TK, NW>(smem_raw, maxo, nst, bars, &abort_flag, ps,
                                  PIPE == 2 ? released : nullptr, PIPE == 2 ? &issued : nullptr);
    ps.err = args[0].err;
    ps.wait_cycles = args[0].wait_cycles;
  }
  unsigned step = 0;
  if constexpr (PIPE == 1) {
    const int w = threadIdx.x >> 5;
    volatile int *abort = &abort_flag;
    if (w == NW) {
      if ((threadIdx.x & 31) == 0) {
        int item = s_item;
        for (int k = 0;; ++k) {
          s_q[k % kItemQ] = item;
          mbar_arrive(&qbar[k % kItemQ]);  // release: the index is visible to the waiters
          if (item >= total) break;
          const int sf = batch_surface(prefix, n_surf, item);
          const FwdArgs<T> &a = args[sf];
          ps.tmap = &P.tm[sf];
          const Item<T, 1> it(a, item - prefix[sf], 0);
          produce_item<T, TK, NW>(a, it, ps, step);
          // after a timeout, or with copies withheld (testing), end the queue
          // here: the compute warps stop at this sentinel or at the abort flag
          item = (*abort || a.withhold) ? total : atomicAdd(counter, 1);
        }
        drain_copies(ps, step, args[0].err);
      }
    } else {
      for (int k = 0;; ++k) {
        if (!mbar_wait(&qbar[k % kItemQ], (unsigned)(k / kItemQ) & 1u, args[0].err, abort,
                       args[0].wait_cycles))
          break;
        const int item = s_q[k % kItemQ];
        if (item >= total) break;
        const int sf = batch_surface(prefix, n_surf, item);
        const FwdArgs<T> &a = args[sf];
        const Item<T, NW> it(a, item - prefix[sf], w);
        T *wwin = reinterpret_cast<T *>(wbase) + (size_t)w * it.opw * a.wfl;
        if constexpr (ACC >= 3 && sizeof(T) == 4) {
          consume_item_f32<TK, NW, ACC >= 4, 1, ACC == 5>(a, it, ps, step, wwin,
                                                  st + w * kMaxObsPerWarp, w);
        } else {
          consume_item<T, TK, NW>(a, it, ps, step, wwin, st + w * kMaxObsPerWarp, w);
        }
        if (*abort) break;
      }
    }
    return;
  }
  const int w = threadIdx.x >> 5;
  for (;;) {
    __syncthreads();  // the previous item is done; s_item holds this one
    const int item = s_item;
    __syncthreads();  // every thread has read it
    if (item >= total) break;
    const int lo = batch_surface(prefix, n_surf, item);
    // a reference, not a copy: the fields are read from the parameter block
    // where used, instead of holding the whole argument block in registers
    const FwdArgs<T> &a = args[lo];
    const int li = item - prefix[lo];
    if constexpr (PIPE == 0) {
      process_item_direct<T, TK, NW>(a, li, reinterpret_cast<T *>(smem_raw), st);
    } else if constexpr (PIPE == 2) {
      ps.tmap = &P.tm[lo];
      if (abort_flag) break;
      const Item<T, NW> it(a, li, w);
      if (threadIdx.x == 0 && !a.withhold) {  // fill the ring: every stage is free here
        const int nsteps = (it.p_end - it.p_begin) * ((it.k_end - it.k_begin) / (32 * TK));
        const int n0 = min(nst, nsteps);
        for (int j = 0; j < n0; ++j)
          issue_step<T, TK, NW>(a, it, ps, j, (step + (unsigned)j) % (unsigned)nst);
        atomicMax(&issued, (int)step + n0);
      }
      T *wwin = reinterpret_cast<T *>(wbase) + (size_t)w * it.opw * a.wfl;
      consume_item_f32<TK, NW, ACC >= 4, 2, ACC == 5>(a, it, ps, step, wwin, st + w * kMaxObsPerWarp,
                                                      w);
    }
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
  }
  if constexpr (PIPE == 2) {
    __syncthreads();
    if (threadIdx.x == 0 && abort_flag) drain_copies(ps, (unsigned)issued, args[0].err);
  }
}

template <typename T, int TK, int NW, int PIPE, int ACC>
__global__ void __launch_bounds__((cta_threads<NW, PIPE>()), (MinBlocks<TK, NW, PIPE>::v))
    k_forward_batch(const __grid_constant__ BatchParams<T> P, int *counter, int nst) {
  forward_batch_cta<T, TK, NW, PIPE, ACC>(P, counter, nst);
}

template <typename T, int TK, int NW, int PIPE, int ACC>
__global__ void __maxnreg__(200)
    k_forward_batch_wide(const __grid_constant__ BatchParams<T> P, int *counter, int nst) {
  forward_batch_cta<T, TK, NW, PIPE, ACC>(P, counter, nst);
}

// One grid over every surface's items (CTA i takes work item i of the
// concatenated queue): the hardware places each CTA, so each item's warps
// land wherever slots are free.  The persistent kernel keeps each CTA's warp
// placement for the whole launch; on a GB300 its per-scheduler instruction
// counts spread by 12 % (1 % for this grid) and it ran about 3 % slower.
template <typename T, int TK, int NW, int PIPE, int ACC>
__device__ __forceinline__ void forward_multi_cta(const BatchParams<T> &P, int nst) {
  const int item = (int)blockIdx.x;
  const int sf = batch_surface(P.prefix, P.n_surf, item);
  // (the error flag and wait bound are the same for every surface: read at
  // a fixed parameter offset)
  forward_cta<T, TK, NW, PIPE, ACC>(P.a[sf], &P.tm[sf], nst, item - P.prefix[sf], P.a[0].err,
                                    P.a[0].wait_cycles);
}

template <typename T, int TK, int NW, int PIPE, int ACC>
__global__ void __launch_bounds__((cta_threads<NW, PIPE>()), (MinBlocks<TK, NW, PIPE>::v))
    k_forward_multi(const __grid_constant__ BatchParams<T> P, int nst) {
  forward_multi_cta<T, TK, NW, PIPE, ACC>(P, nst);
}

template <typename T, int TK, int NW, int PIPE, int ACC>
__global__ void __maxnreg__(200) k_forward_multi_wide(const __grid_constant__ BatchParams<T> P,
                                                      int nst) {
  forward_multi_cta<T, TK, NW, PIPE, ACC>(P, nst);
}

// Candidate tile shapes {pipe, tk, warps, obs_per_warp, win, seg_chunks,
// stages, acc, wide}.  acc: 0 one sample per lane per block (FP64), 3 a pair
// of consecutive samples per lane per block with split windows and packed
// dot products (FP32; its series rows pair those samples, so every FP32 shape
// is a TMA shape), 4 the same with the next observer's record read ahead, 5
// as 4 with compensated (Kahan) window sums.  wide: register cap 200 instead
// of the launch bounds' occupancy target.
constexpr FwdConfig kCfgF32[] = {
    {1, 4, 4, 9, 224, 4, 3, 4, 0},
    {1, 4, 4, 9, 224, 2, 3, 4, 0},
    {1, 4, 4, 9, 224, 4, 3, 3, 0},
    {2, 4, 4, 9, 224, 4, 2, 4, 0},
    {2, 4, 8, 9, 224, 4, 3, 4, 0},
    {1, 8, 4, 9, 352, 2, 3, 3, 0},
    {1, 4, 4, 9, 224, 4, 3, 4, 1},
    {1, 4, 4, 9, 224, 8, 3, 4, 0},
    {1, 4, 4, 9, 160, 4, 4, 4, 0},
    {1, 4, 4, 9, 224, 4, 2, 4, 0},
    {1, 4, 4, 9, 160, 4, 2, 5, 0},
    {1, 4, 4, 9, 224, 4, 3, 5, 0},
};
constexpr bool f32_obs_fit() {
  for (const FwdConfig &c : kCfgF32)
    if (c.obs_per_warp > kMaxObsPerWarpF32) return false;
  return true;
}
static_assert(f32_obs_fit(), "an FP32 shape has more observers per warp than the unrolled loop");
const FwdConfig kCfgF64[] = {
    {0, 2, 8, 16, 128, 8, 0, 0, 0},
    {1, 2, 8, 9, 128, 8, 3, 0, 0},
    {0, 2, 4, 16, 128, 8, 0, 0, 0},
    {0, 1, 8, 16, 64, 16, 0, 0, 0},
};

template <typename T>
size_t smem_for(const FwdConfig &c, int obs_per_cta) {
  const int opw = obs_per_cta / c.warps;
  size_t win = (size_t)c.warps * opw * c.win * sizeof(T) * (c.acc == 5 ? 2 : 1);
  if (c.pipe == 0) return win;
  const size_t xb = (size_t)32 * c.tk * kRec * sizeof(T);
  const size_t sb =
      (xb + (size_t)obs_per_cta * kRec * sizeof(T) + 1023) & ~size_t(1023);
  return 1024 + (size_t)c.stages * sb + win;
}

template <typename T, int TK, int NW, int PIPE, int ACC>
cudaError_t launch_one(const FwdArgs<T> &a, const CUtensorMap &tm, const FwdConfig &c,
                       cudaStream_t s) {
  const size_t smem = smem_for<T>(c, a.obs_per_cta);
  auto kern = c.wide ? k_forward_wide<T, TK, NW, PIPE, ACC> : k_forward<T, TK, NW, PIPE, ACC>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  if (a.seg_lo < 0 || a.seg_cnt < 1 || a.seg_lo + a.seg_cnt > a.n_segs) return cudaErrorInvalidValue;
  const int items = a.nsets * a.n_obs_groups * a.seg_cnt;
  if (items <= 0) return cudaSuccess;
  kern<<<items, cta_threads<NW, PIPE>(), smem, s>>>(a, tm, c.stages);
  return cudaGetLastError();
}

template <typename T, int TK, int NW, int PIPE, int ACC>
cudaError_t launch_multi_one(const BatchParams<T> &P, size_t smem, bool wide, int nst,
                             cudaStream_t s) {
  auto kern = wide ? k_forward_multi_wide<T, TK, NW, PIPE, ACC>
                   : k_forward_multi<T, TK, NW, PIPE, ACC>;
  cudaError_t e =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)P.total, cta_threads<NW, PIPE>(), smem, s>>>(P, nst);
  return cudaGetLastError();
}

template <typename T, int TK, int NW, int PIPE, int ACC>
cudaError_t launch_batch_one(const BatchParams<T> &P, int *d_counter, size_t smem, int n_ctas,
                             bool wide, int nst, cudaStream_t s) {
  auto kern = wide ? k_forward_batch_wide<T, TK, NW, PIPE, ACC>
                   : k_forward_batch<T, TK, NW, PIPE, ACC>;
  cudaError_t e =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<n_ctas, cta_threads<NW, PIPE>(), smem, s>>>(P, d_counter, nst);
  return cudaGetLastError();
}

}  // namespace

int fwd_num_configs(bool fp64) {
  return fp64 ? (int)(sizeof(kCfgF64) / sizeof(kCfgF64[0]))
              : (int)(sizeof(kCfgF32) / sizeof(kCfgF32[0]));
}

FwdConfig fwd_config(bool fp64, int idx) {
  const int n = fwd_num_configs(fp64);
  if (idx < 0 || idx >= n) idx = 0;
  return fp64 ? kCfgF64[idx] : kCfgF32[idx];
}

size_t fwd_smem_bytes(bool fp64, const FwdConfig &c, int obs_per_cta) {
  return fp64 ? smem_for<double>(c, obs_per_cta) : smem_for<float>(c, obs_per_cta);
}

bool encode_x_tensor_map(void *out128, const void *X, unsigned long long rows, bool fp64,
                         int box_rows) {
  static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
  if (!enc) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return false;
    enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  // Rows of 128 bytes (two FP32 samples or one FP64 sample of 16 values), so
  // the inner box dimension equals the 128-byte swizzle span.
  const unsigned per = fp64 ? 1u : 2u;  // samples per 128-byte row
  const cuuint64_t dims[2] = {fp64 ? 16ull : 32ull, rows / per};
  const cuuint64_t strides[1] = {128ull};
  const cuuint32_t box[2] = {fp64 ? 16u : 32u, (cuuint32_t)(box_rows / per)};
  const cuuint32_t estr[2] = {1, 1};
  CUtensorMap *m = reinterpret_cast<CUtensorMap *>(out128);
  const CUresult r = enc(m, fp64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                         2, const_cast<void *>(X), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Instantiated shapes: FP32 {copy warp: TK 4 with and without the record read
// ahead, TK 8; in-line refill: 4 and 8 warps}; FP64 {direct 2x8, TMA 2x8,
// direct 2x4, direct 1x8}.
#define FWH_DISPATCH(T, c, CALL)                                                        \
  do {                                                                                   \
    if constexpr (sizeof(T) == 4) {                                                      \
      if (c.pipe == 2 && c.tk == 4 && c.warps == 4 && c.acc == 4) return CALL(T, 4, 4, 2, 4); \
      if (c.pipe == 2 && c.tk == 4 && c.warps == 8 && c.acc == 4) return CALL(T, 4, 8, 2, 4); \
      if (c.pipe == 1 && c.tk == 4 && c.warps == 4 && c.acc == 3) return CALL(T, 4, 4, 1, 3); \
      if (c.pipe == 1 && c.tk == 4 && c.warps == 4 && c.acc == 4) return CALL(T, 4, 4, 1, 4); \
      if (c.pipe == 1 && c.tk == 4 && c.warps == 4 && c.acc == 5) return CALL(T, 4, 4, 1, 5); \
      if (c.pipe == 1 && c.tk == 8 && c.warps == 4 && c.acc == 3) return CALL(T, 8, 4, 1, 3); \
    } else {                                                                             \
      if (c.pipe == 0 && c.tk == 2 && c.warps == 8) return CALL(T, 2, 8, 0, 0);          \
      if (c.pipe == 1 && c.tk == 2 && c.warps == 8) return CALL(T, 2, 8, 1, 0);          \
      if (c.pipe == 0 && c.tk == 2 && c.warps == 4) return CALL(T, 2, 4, 0, 0);          \
      if (c.pipe == 0 && c.tk == 1 && c.warps == 8) return CALL(T, 1, 8, 0, 0);          \
    }                                                                                    \
    return cudaErrorInvalidValue;                                                        \
  } while (0)

template <typename T>
cudaError_t launch_forward(const FwdArgs<T> &a, const void *tmap128, int cfg, cudaStream_t s) {
  const FwdConfig c = fwd_config(sizeof(T) == 8, cfg);
  // the X descriptor travels as a kernel parameter (no device copy to make)
  CUtensorMap tm;
  if (tmap128)
    memcpy(&tm, tmap128, sizeof tm);
  else
    memset(&tm, 0, sizeof tm);
#define FWH_CALL_ONE(TT, TK, NW, PIPE, ACC) launch_one<TT, TK, NW, PIPE, ACC>(a, tm, c, s)
  FWH_DISPATCH(T, c, FWH_CALL_ONE);
#undef FWH_CALL_ONE
}

template <typename T>
cudaError_t launch_forward_batch(const BatchParams<T> &P, int *d_counter, int cfg, int n_ctas,
                                 cudaStream_t s) {
  if (P.n_surf < 1 || P.n_surf > kMaxBatchSurf) return cudaErrorInvalidValue;
  const FwdConfig c = fwd_config(sizeof(T) == 8, cfg);
  const size_t smem = smem_for<T>(c, c.warps * c.obs_per_warp);
#define FWH_CALL_BATCH(TT, TK, NW, PIPE, ACC) \
  launch_batch_one<TT, TK, NW, PIPE, ACC>(P, d_counter, smem, n_ctas, c.wide != 0, c.stages, s)
  FWH_DISPATCH(T, c, FWH_CALL_BATCH);
#undef FWH_CALL_BATCH
}

template <typename T>
cudaError_t launch_forward_multi(const BatchParams<T> &P, int cfg, cudaStream_t s) {
  if (P.n_surf < 1 || P.n_surf > kMaxBatchSurf || P.total < 1) return cudaErrorInvalidValue;
  const FwdConfig c = fwd_config(sizeof(T) == 8, cfg);
  const size_t smem = smem_for<T>(c, c.warps * c.obs_per_warp);
#define FWH_CALL_MULTI(TT, TK, NW, PIPE, ACC) \
  launch_multi_one<TT, TK, NW, PIPE, ACC>(P, smem, c.wide != 0, c.stages, s)
  FWH_DISPATCH(T, c, FWH_CALL_MULTI);
#undef FWH_CALL_MULTI
}

// Resident CTAs per SM of the persistent kernel for a config.
template <typename T, int TK, int NW, int PIPE, int ACC>
cudaError_t batch_occupancy_one(const FwdConfig &c, size_t smem, int *per_sm) {
  auto kern = c.wide ? k_forward_batch_wide<T, TK, NW, PIPE, ACC>
                     : k_forward_batch<T, TK, NW, PIPE, ACC>;
  cudaError_t e =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, cta_threads<NW, PIPE>(),
                                                       smem);
}

template <typename T>
cudaError_t forward_batch_occupancy(int cfg, int *per_sm) {
  const FwdConfig c = fwd_config(sizeof(T) == 8, cfg);
  const size_t smem = smem_for<T>(c, c.warps * c.obs_per_warp);
  *per_sm = 0;
#define FWH_CALL_OCC(TT, TK, NW, PIPE, ACC) batch_occupancy_one<TT, TK, NW, PIPE, ACC>(c, smem, per_sm)
  FWH_DISPATCH(T, c, FWH_CALL_OCC);
#undef FWH_CALL_OCC
}

template cudaError_t forward_batch_occupancy<float>(int, int *);
template cudaError_t forward_batch_occupancy<double>(int, int *);

template <typename T>
cudaError_t launch_plan(T *coef, const int *set_begin, int nsets, int O, int slack,
                        int half_bytes, int slot_bytes, int *i0max_tab, int *err,
                        cudaStream_t s) {
  if (nsets <= 0 || O <= 0) return cudaSuccess;
  k_plan<T><<<nsets, 128, 0, s>>>(coef, set_begin, O, slack, half_bytes, slot_bytes, i0max_tab,
                                  err);
  return cudaGetLastError();
}

template cudaError_t launch_plan<float>(float *, const int *, int, int, int, int, int, int *,
                                        int *, cudaStream_t);
template cudaError_t launch_plan<double>(double *, const int *, int, int, int, int, int, int *,
                                         int *, cudaStream_t);
template cudaError_t launch_forward<float>(const FwdArgs<float> &, const void *, int,
                                           cudaStream_t);
template cudaError_t launch_forward<double>(const FwdArgs<double> &, const void *, int,
                                            cudaStream_t);
template cudaError_t launch_forward_multi<float>(const BatchParams<float> &, int, cudaStream_t);
template cudaError_t launch_forward_multi<double>(const BatchParams<double> &, int, cudaStream_t);
template cudaError_t launch_forward_batch<float>(const BatchParams<float> &, int *, int, int,
                                                 cudaStream_t);
template cudaError_t launch_forward_batch<double>(const BatchParams<double> &, int *, int, int,
                                                  cudaStream_t);

}  // namespace fwh
