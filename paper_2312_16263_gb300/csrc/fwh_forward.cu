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
// warps; warp w owns observers o_begin + w + NW m (m < obs_per_warp) of the
// group and keeps, per observer, a window of `win` bins in shared memory.
// Lanes map to source samples (k = k0 + lane + 32 j, j < TK), so each X row
// is loaded once per warp and reused for all of the warp's observers, the
// coefficient record is a warp-uniform broadcast, and the window updates are
// conflict-free (consecutive lanes, consecutive bins).  The per-(p, o) shift
// only moves the window offset, never the lane pattern.  After each chunk of
// 32 TK samples the oldest 32 TK bins of every window are complete for this
// panel set: they are flushed to p_out with FP64 atomics (one per bin per
// panel set, not per panel) and the window slides.
//
// Window bound: a panel set's shifts for one observer span S = i0max - i0min;
// slots touched in a chunk are [0, CH + S], so S <= win - CH - 1 is required
// (the host planner bounds S from the set's extent; a violation is flagged,
// never written out of bounds).
#include "fwh_internal.cuh"

namespace fwh {

namespace {

constexpr int kMaxObsPerWarp = 16;

template <typename T> struct Vec;
template <> struct Vec<float> {
  using V = float4;
  static constexpr int per = 4;
};
template <> struct Vec<double> {
  using V = double2;
  static constexpr int per = 2;
};

template <typename T>
__device__ __forceinline__ int rec_i0(const T *rec);
template <>
__device__ __forceinline__ int rec_i0<float>(const float *rec) {
  return __float_as_int(__ldg(rec + 12));
}
template <>
__device__ __forceinline__ int rec_i0<double>(const double *rec) {
  return (int)__ldg(rec + 12);
}

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

template <typename T> __device__ __forceinline__ int rec_i0_of(T v);
template <> __device__ __forceinline__ int rec_i0_of<float>(float v) {
  return __float_as_int(v);
}
template <> __device__ __forceinline__ int rec_i0_of<double>(double v) { return (int)v; }

__device__ __forceinline__ void atomic_add_f64(double *addr, double v) {
  atomicAdd(addr, v);
}

// One work item.  smem: NW * obs_per_warp * win values of T; st: int state.
template <typename T, int TK, int NW>
__device__ __forceinline__ void process_item(const FwdArgs<T> &a, int item, T *smem,
                                             int *st) {
  constexpr int CH = 32 * TK;
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int ng = a.n_obs_groups;
  const int g = item % ng;
  const int rest = item / ng;
  const int sidx = rest % a.nsets;
  const int q = rest / a.nsets;
  const int p_begin = a.set_begin[sidx], p_end = a.set_begin[sidx + 1];
  const int opw = a.obs_per_cta / NW;
  const int o_begin = g * a.obs_per_cta;
  const int o_end = min(a.O, o_begin + a.obs_per_cta);
  const int k_begin = q * a.seg_len;
  const int k_end = min(a.ntp, k_begin + a.seg_len);
  const int win = a.win;
  T *wwin = smem + (size_t)w * opw * win;
  int *s_i0max = st + w * kMaxObsPerWarp;
  int *s_ok = st + NW * kMaxObsPerWarp + w * kMaxObsPerWarp;

  // observers of this warp
  int nobs = 0;
  for (int m = 0; m < opw; ++m)
    if (o_begin + w + NW * m < o_end) nobs = m + 1;

  // per-observer shift range over the panel set
  for (int m = 0; m < nobs; ++m) {
    const int o = o_begin + w + NW * m;
    int lo = 0x7fffffff, hi = -0x7fffffff;
    for (int p = p_begin + lane; p < p_end; p += 32) {
      const int i0 = rec_i0<T>(a.coef + ((size_t)p * a.O + o) * kRec);
      lo = min(lo, i0);
      hi = max(hi, i0);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, off));
      hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, off));
    }
    const bool ok = (hi - lo) <= win - CH - 1;
    if (lane == 0) {
      s_i0max[m] = hi;
      s_ok[m] = ok ? 1 : 0;
      if (!ok) atomicOr(a.err, kErrWindow);
    }
  }
  for (int i = lane; i < nobs * win; i += 32) wwin[i] = T(0);
  __syncwarp();

  for (int k0 = k_begin; k0 < k_end; k0 += CH) {
    for (int p = p_begin; p < p_end; ++p) {
      // observer-independent rows of this panel for the chunk
      T x[TK][kRec];
      const T *Xp = a.X + ((size_t)p * a.ntp + k0 + lane) * kRec;
#pragma unroll
      for (int j = 0; j < TK; ++j) load16<T>(Xp + (size_t)j * 32 * kRec, x[j]);

      const T *rec0 = a.coef + (size_t)p * a.O * kRec;
      for (int m = 0; m < nobs; ++m) {
        const int o = o_begin + w + NW * m;
        T c[kRec];
        load16<T>(rec0 + (size_t)o * kRec, c);
        const int i0 = rec_i0_of<T>(c[12]);
        if (!s_ok[m]) continue;  // warp-uniform
        // slot of bin (k - i0) relative to the window start
        // (win start = k0 - i0max - 1 for this chunk)
        const int slot = k0 + lane - i0 - (k0 - s_i0max[m] - 1);
        T *wm = wwin + (size_t)m * win + slot;
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
    }
    // the first CH bins of every window are complete: flush and slide
    for (int m = 0; m < nobs; ++m) {
      const int o = o_begin + w + NW * m;
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
      // move live bins [CH, win) to the front (win - CH <= CH), zero the rest
      for (int t = lane; t < win - CH; t += 32) wm[t] = wm[CH + t];
      __syncwarp();
      for (int t = win - CH + lane; t < win; t += 32) wm[t] = T(0);
      __syncwarp();
    }
  }
  // segment end: the remaining window holds partial bins of the next chunk
  for (int m = 0; m < nobs; ++m) {
    const int o = o_begin + w + NW * m;
    T *wm = wwin + (size_t)m * win;
    const int wbase = k_end - s_i0max[m] - 1;
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

template <typename T, int TK, int NW>
__global__ void __launch_bounds__(NW * 32) k_forward(FwdArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int st[2 * NW * kMaxObsPerWarp];
  process_item<T, TK, NW>(a, blockIdx.x, reinterpret_cast<T *>(smem_raw), st);
}

// Persistent form: CTAs pull work items of several surfaces from one queue.
template <typename T, int TK, int NW>
__global__ void __launch_bounds__(NW * 32) k_forward_batch(const FwdArgs<T> *args,
                                                           const int *item_prefix,
                                                           int n_surf, int total,
                                                           int *counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int st[2 * NW * kMaxObsPerWarp];
  __shared__ int s_item;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= total) break;
    int lo = 0, hi = n_surf - 1;  // surface of this item: item_prefix[s] <= item
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (item_prefix[mid] <= item) lo = mid; else hi = mid - 1;
    }
    const FwdArgs<T> a = args[lo];
    process_item<T, TK, NW>(a, item - item_prefix[lo], reinterpret_cast<T *>(smem_raw), st);
  }
}

// Candidate tile shapes: {tk, warps, obs_per_warp (max), win, seg_chunks}.
const FwdConfig kCfgF32[] = {
    {4, 8, 16, 256, 4},
    {4, 4, 16, 256, 4},
    {2, 8, 16, 128, 8},
    {4, 8, 16, 256, 2},
    {4, 8, 16, 256, 8},
};
const FwdConfig kCfgF64[] = {
    {2, 8, 16, 128, 8},
    {2, 4, 16, 128, 8},
    {1, 8, 16, 64, 16},
};

template <typename T, int TK, int NW>
cudaError_t launch_tk_nw(const FwdArgs<T> &a, const FwdConfig &c, cudaStream_t s) {
  const size_t smem = (size_t)NW * (a.obs_per_cta / NW) * a.win * sizeof(T);
  cudaError_t e = cudaFuncSetAttribute(k_forward<T, TK, NW>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int items = a.nsets * a.n_obs_groups * a.n_segs;
  if (items <= 0) return cudaSuccess;
  k_forward<T, TK, NW><<<items, NW * 32, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int TK, int NW>
cudaError_t launch_batch_tk_nw(const FwdArgs<T> *d_args, const int *d_prefix, int n_surf,
                               int total, int *d_counter, size_t smem, int n_ctas,
                               cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(k_forward_batch<T, TK, NW>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_forward_batch<T, TK, NW><<<n_ctas, NW * 32, smem, s>>>(d_args, d_prefix, n_surf, total,
                                                          d_counter);
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

template <>
cudaError_t launch_forward<float>(const FwdArgs<float> &a, int cfg, cudaStream_t s) {
  const FwdConfig c = fwd_config(false, cfg);
  if (c.tk == 4 && c.warps == 8) return launch_tk_nw<float, 4, 8>(a, c, s);
  if (c.tk == 4 && c.warps == 4) return launch_tk_nw<float, 4, 4>(a, c, s);
  if (c.tk == 2 && c.warps == 8) return launch_tk_nw<float, 2, 8>(a, c, s);
  return cudaErrorInvalidValue;
}

template <>
cudaError_t launch_forward<double>(const FwdArgs<double> &a, int cfg, cudaStream_t s) {
  const FwdConfig c = fwd_config(true, cfg);
  if (c.tk == 2 && c.warps == 8) return launch_tk_nw<double, 2, 8>(a, c, s);
  if (c.tk == 2 && c.warps == 4) return launch_tk_nw<double, 2, 4>(a, c, s);
  if (c.tk == 1 && c.warps == 8) return launch_tk_nw<double, 1, 8>(a, c, s);
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_forward_batch(const FwdArgs<T> *d_args, const int *d_prefix, int n_surf,
                                 int total, int *d_counter, int cfg, int n_ctas,
                                 cudaStream_t s);

template <>
cudaError_t launch_forward_batch<float>(const FwdArgs<float> *d_args, const int *d_prefix,
                                        int n_surf, int total, int *d_counter, int cfg,
                                        int n_ctas, cudaStream_t s) {
  const FwdConfig c = fwd_config(false, cfg);
  const size_t smem = (size_t)c.warps * c.obs_per_warp * c.win * sizeof(float);
  if (c.tk == 4 && c.warps == 8)
    return launch_batch_tk_nw<float, 4, 8>(d_args, d_prefix, n_surf, total, d_counter, smem,
                                           n_ctas, s);
  if (c.tk == 4 && c.warps == 4)
    return launch_batch_tk_nw<float, 4, 4>(d_args, d_prefix, n_surf, total, d_counter, smem,
                                           n_ctas, s);
  if (c.tk == 2 && c.warps == 8)
    return launch_batch_tk_nw<float, 2, 8>(d_args, d_prefix, n_surf, total, d_counter, smem,
                                           n_ctas, s);
  return cudaErrorInvalidValue;
}

template <>
cudaError_t launch_forward_batch<double>(const FwdArgs<double> *d_args, const int *d_prefix,
                                         int n_surf, int total, int *d_counter, int cfg,
                                         int n_ctas, cudaStream_t s) {
  const FwdConfig c = fwd_config(true, cfg);
  const size_t smem = (size_t)c.warps * c.obs_per_warp * c.win * sizeof(double);
  if (c.tk == 2 && c.warps == 8)
    return launch_batch_tk_nw<double, 2, 8>(d_args, d_prefix, n_surf, total, d_counter, smem,
                                            n_ctas, s);
  if (c.tk == 2 && c.warps == 4)
    return launch_batch_tk_nw<double, 2, 4>(d_args, d_prefix, n_surf, total, d_counter, smem,
                                            n_ctas, s);
  if (c.tk == 1 && c.warps == 8)
    return launch_batch_tk_nw<double, 1, 8>(d_args, d_prefix, n_surf, total, d_counter, smem,
                                            n_ctas, s);
  return cudaErrorInvalidValue;
}

}  // namespace fwh
