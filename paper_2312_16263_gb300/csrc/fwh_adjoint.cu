// Adjoint of the forward scatter: a conflict-free gather over observers.
//
// The forward adds, for panel p, observer o and source sample k,
//   a g + cc m  to bin k - i0   and   b g + dd m  to bin k - i0 - 1,
// with g = c . F[k], m = c . M[k].  Its transpose, for the gradient G of the
// loss with respect to p_out (zero outside the valid bins 0 <= j < N_o), is
//   gF = a G[k - i0] + b G[k - i0 - 1],   gM = cc G[k - i0] + dd G[k - i0 - 1]
//   Xbar[p][k][s]     = sum_o c_s gF,     Xbar[p][k][8 + s] = sum_o c_s gM,
// so each (panel, sample) output is owned by one lane and summed over the
// observers in registers, 20 FMA per (panel, sample, observer).  Two forms:
// k_adjoint_set (FP32) gathers per panel set from a window of G staged in
// shared memory, with atomics only to add the partial sums of several
// 36-observer groups; k_adjoint (FP64, and FP32 shapes with 256-sample
// chunks) is one CTA per panel reading G from L2, without atomics.
// Nothing from the forward pass is stored: only the per-(p, o) records
// (geometry, computed once per observer set), the plan and G are read.
#include "fwh_internal.cuh"

namespace fwh {

namespace {

template <typename T> __device__ __forceinline__ int i0_of(T v);
template <> __device__ __forceinline__ int i0_of<float>(float v) { return __float_as_int(v); }
template <> __device__ __forceinline__ int i0_of<double>(double v) { return (int)v; }

// G converted to T with zeros outside [0, N_o): Gt[o][j], j < ntp.
template <typename T>
__global__ void k_grad_pad(const double *grad_p, const int *n_valid, T *Gt, int O, int nt,
                           int ntp) {
  for (int o = blockIdx.y; o < O; o += gridDim.y) {  // grid y is capped at 65535
    const int nv = n_valid[o];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < ntp; j += gridDim.x * blockDim.x)
      Gt[(size_t)o * ntp + j] = (j < nv && j < nt) ? (T)grad_p[(size_t)o * nt + j] : T(0);
  }
}

// One CTA per (panel, group of 8 chunks), one warp per chunk.  The panel's
// records are staged in shared memory in tiles of kObsTile observers (read
// back as broadcasts), and each lane loads the two gradient bins of the next
// observer while it accumulates the current one.
constexpr int kObsTile = 128;

template <typename T, int TK>
__global__ void __launch_bounds__(256) k_adjoint(const T *coef, const T *Gt, T *Xbar, int P,
                                                 int O, int ntp) {
  constexpr int CH = 32 * TK;
  __shared__ __align__(16) T srec[kObsTile * kRec];
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int nch = ntp / CH;
  const int ngrp = (nch + 7) / 8;
  const int p = blockIdx.x / ngrp;
  const int ch = (blockIdx.x % ngrp) * 8 + w;
  const bool live = ch < nch;  // warps past the last chunk only help staging
  const int k0 = ch * CH;
  T acc[TK][kRec];
#pragma unroll
  for (int j = 0; j < TK; ++j)
#pragma unroll
    for (int s = 0; s < kRec; ++s) acc[j][s] = T(0);
  const T *rec0 = coef + (size_t)p * O * kRec;
  for (int ob = 0; ob < O; ob += kObsTile) {
    const int no = min(kObsTile, O - ob);
    __syncthreads();
    for (int idx = threadIdx.x; idx < no * kRec; idx += blockDim.x)
      srec[idx] = rec0[(size_t)ob * kRec + idx];
    __syncthreads();
    if (!live) continue;
    auto bins = [&](int o, T (&g0)[TK], T (&g1)[TK]) {
      const int i0 = i0_of<T>(srec[o * kRec + slot::i0]);
      const T *G = Gt + (size_t)(ob + o) * ntp;
#pragma unroll
      for (int j = 0; j < TK; ++j) {
        const int jb = k0 + lane + 32 * j - i0;  // bin fed by the left spline node
        g0[j] = jb >= 0 ? __ldg(G + jb) : T(0);
        g1[j] = jb >= 1 ? __ldg(G + jb - 1) : T(0);
      }
    };
    T g0[TK], g1[TK];
    bins(0, g0, g1);
    for (int o = 0; o < no; ++o) {
      T n0[TK], n1[TK];
      if (o + 1 < no) bins(o + 1, n0, n1);
      const T *r = srec + o * kRec;
      T c[12];
#pragma unroll
      for (int s = 0; s < 12; ++s) c[s] = r[s];  // c0..c7, then the four weights
#pragma unroll
      for (int j = 0; j < TK; ++j) {
        const T gF = c[slot::a] * g0[j] + c[slot::b] * g1[j];
        const T gM = c[slot::cc] * g0[j] + c[slot::dd] * g1[j];
#pragma unroll
        for (int s = 0; s < 8; ++s) {
          acc[j][s] = fma(c[slot::c + s], gF, acc[j][s]);
          acc[j][8 + s] = fma(c[slot::c + s], gM, acc[j][8 + s]);
        }
      }
      if (o + 1 < no) {
#pragma unroll
        for (int j = 0; j < TK; ++j) {
          g0[j] = n0[j];
          g1[j] = n1[j];
        }
      }
    }
  }
  if (!live) return;
  T *out = Xbar + ((size_t)p * ntp + k0 + lane) * kRec;
#pragma unroll
  for (int j = 0; j < TK; ++j)
#pragma unroll
    for (int s = 0; s < kRec; ++s) out[(size_t)j * 32 * kRec + s] = acc[j][s];
}

// Set form (FP32).  Work item = (panel set, observer group, 128-sample
// chunk), numbered observer group fastest, then chunk, then the sets in
// descending size.  The gradient bins every (panel, observer) of the set can
// touch in the chunk, G[k0 - i0max(o) - 1 + t] for t < win + 1 (the planner
// bounds each record's offset i0max - i0 by the window slack), are staged in
// shared memory once per item; each warp then takes panels of the set in
// turn and, for every observer of the group, reads the two bins of each of
// its samples from that window (conflict-free, consecutive lanes at
// consecutive slots) and accumulates the 16 components of Xbar in registers.
// Each warp stages the group's records of its next panel in shared memory
// (cp.async, a double buffer per warp) while it works on the current one, so
// the inner loop reads every record as a shared-memory broadcast instead of
// waiting on L2.  One observer group writes Xbar directly; several add their
// partial sums with vector atomics into a zeroed Xbar.
constexpr int kAdjGroup = 36;    // observers per item
constexpr int kAdjWarps = 4;
constexpr int kAdjTK = 4;        // samples per lane (chunk 128)

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
// 4-byte copy, zero fill when !ok (src is then not read)
__device__ __forceinline__ void cp_async4_zf(float *dst, const float *src, bool ok) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(ok ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ void red_add_v4(float *addr, float4 v) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};\n" ::"l"(addr), "f"(v.x), "f"(v.y),
               "f"(v.z), "f"(v.w)
               : "memory");
}

template <bool kAtomic>
__global__ void __launch_bounds__(kAdjWarps * 32) k_adjoint_set(AdjArgs<float> a) {
  constexpr int CH = 32 * kAdjTK;
  extern __shared__ __align__(16) float gw[];  // [kAdjGroup][wstride], then the record buffers
  const int wstride = (a.win + 1 + 3) & ~3;
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int ng = (a.O + kAdjGroup - 1) / kAdjGroup;
  const int nch = a.ntp / CH;
  const int item = blockIdx.x;
  const int g = item % ng;
  const int rest = item / ng;
  const int ch = rest % nch;
  const int sidx = a.set_order[rest / nch];
  const int k0 = ch * CH;
  const int o0 = g * kAdjGroup;
  const int no = min(kAdjGroup, a.O - o0);
  const int p_begin = a.set_begin[sidx], p_end = a.set_begin[sidx + 1];
  // stage the window of each observer of the group (cp.async: every copy in
  // flight at once; zero outside the record)
  for (int o = 0; o < no; ++o) {
    const int base = k0 - a.i0max_tab[(size_t)sidx * a.O + o0 + o] - 1;
    const float *G = a.Gt + (size_t)(o0 + o) * a.ntp;
    for (int t = threadIdx.x; t <= a.win; t += blockDim.x) {
      const int j = base + t;
      const bool ok = j >= 0 && j < a.ntp;
      cp_async4_zf(gw + o * wstride + t, G + (ok ? j : 0), ok);
    }
  }
  cp_async_commit();
  // this warp's record double buffer: [2][kAdjGroup][kRec]
  float *rb = gw + (size_t)kAdjGroup * wstride + (size_t)w * 2 * kAdjGroup * kRec;
  auto stage = [&](int p, int buf) {  // the group's records of panel p, 16 bytes a copy
    const float *src = a.coef + ((size_t)p * a.O + o0) * kRec;
    float *dst = rb + (size_t)buf * kAdjGroup * kRec;
    for (int c = lane; c < no * (kRec / 4); c += 32) cp_async16(dst + 4 * c, src + 4 * c);
    cp_async_commit();
  };
  int buf = 0;
  if (p_begin + w < p_end) stage(p_begin + w, 0);
  cp_async_wait<0>();  // the window (and this warp's first records)
  __syncthreads();
  for (int p = p_begin + w; p < p_end; p += kAdjWarps) {
    const bool more = p + kAdjWarps < p_end;
    if (more) {
      stage(p + kAdjWarps, buf ^ 1);
      cp_async_wait<1>();  // this panel's copy has landed (the next one may still fly)
    } else {
      cp_async_wait<0>();
    }
    __syncwarp();
    float acc[kAdjTK][kRec];
#pragma unroll
    for (int j = 0; j < kAdjTK; ++j)
#pragma unroll
      for (int s = 0; s < kRec; ++s) acc[j][s] = 0.f;
    const float4 *rec = reinterpret_cast<const float4 *>(rb + (size_t)buf * kAdjGroup * kRec);
#pragma unroll 2
    for (int o = 0; o < no; ++o) {
      const float4 r0 = rec[4 * o], r1 = rec[4 * o + 1], r2 = rec[4 * o + 2],
                   r3 = rec[4 * o + 3];
      const float c[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
      const float wa = r2.x, wb = r2.y, wcc = r2.z, wdd = r2.w;  // slots a, b, cc, dd
      const int off = __float_as_int(r3.y);                       // slot off = i0max - i0
      // G[k - i0] at window slot (k - k0) + off + 1, G[k - i0 - 1] one below
      const float *gp = gw + o * wstride + off + lane;
#pragma unroll
      for (int j = 0; j < kAdjTK; ++j) {
        const float g1 = gp[32 * j], g0 = gp[32 * j + 1];
        const float gF = wa * g0 + wb * g1;
        const float gM = wcc * g0 + wdd * g1;
#pragma unroll
        for (int s = 0; s < 8; ++s) {
          acc[j][s] = fmaf(c[s], gF, acc[j][s]);
          acc[j][8 + s] = fmaf(c[s], gM, acc[j][8 + s]);
        }
      }
    }
    float *out = a.Xbar + ((size_t)p * a.ntp + k0 + lane) * kRec;
#pragma unroll
    for (int j = 0; j < kAdjTK; ++j)
#pragma unroll
      for (int q = 0; q < kRec / 4; ++q) {
        const float4 v = make_float4(acc[j][4 * q], acc[j][4 * q + 1], acc[j][4 * q + 2],
                                     acc[j][4 * q + 3]);
        float *dst = out + (size_t)j * 32 * kRec + 4 * q;
        if (kAtomic)
          red_add_v4(dst, v);
        else
          *reinterpret_cast<float4 *>(dst) = v;
      }
    __syncwarp();  // every lane is done with this buffer before it is refilled
    buf ^= 1;
  }
}

}  // namespace

template <typename T>
cudaError_t launch_adjoint(const AdjArgs<T> &a, cudaStream_t s) {
  constexpr int TK = sizeof(T) == 4 ? 4 : 2;
  constexpr int CH = 32 * TK;
  T *Gt = a.Gt;
  dim3 gg((a.ntp + 255) / 256, a.O < 65535 ? a.O : 65535);
  k_grad_pad<T><<<gg, 256, 0, s>>>(a.grad_p, a.n_valid, Gt, a.O, a.nt, a.ntp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if constexpr (sizeof(T) == 4) {
    if (a.win > 0) {
      constexpr int SCH = 32 * kAdjTK;
      if (a.ntp % SCH != 0) return cudaErrorInvalidValue;
      const int ng = (a.O + kAdjGroup - 1) / kAdjGroup;
      const long items = (long)a.nsets * ng * (a.ntp / SCH);
      if (items <= 0) return cudaSuccess;
      if (items > INT32_MAX) return cudaErrorInvalidValue;
      const size_t smem = ((size_t)kAdjGroup * ((a.win + 1 + 3) & ~3) +
                           (size_t)kAdjWarps * 2 * kAdjGroup * kRec) * sizeof(float);
      if (ng > 1) {
        e = cudaMemsetAsync(a.Xbar, 0, (size_t)a.P * a.ntp * kRec * sizeof(float), s);
        if (e != cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(k_adjoint_set<true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
          return e;
        k_adjoint_set<true><<<(unsigned)items, kAdjWarps * 32, smem, s>>>(a);
      } else {
        if ((e = cudaFuncSetAttribute(k_adjoint_set<false>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
          return e;
        k_adjoint_set<false><<<(unsigned)items, kAdjWarps * 32, smem, s>>>(a);
      }
      return cudaGetLastError();
    }
  }
  const long blocks = (long)a.P * ((a.ntp / CH + 7) / 8);
  if (blocks <= 0) return cudaSuccess;
  k_adjoint<T, TK><<<(unsigned)blocks, 256, 0, s>>>(a.coef, Gt, a.Xbar, a.P, a.O, a.ntp);
  return cudaGetLastError();
}

template cudaError_t launch_adjoint<float>(const AdjArgs<float> &, cudaStream_t);
template cudaError_t launch_adjoint<double>(const AdjArgs<double> &, cudaStream_t);

}  // namespace fwh
