// Power spectral density of the far-field signals (Sec. IV C): Welch's
// method -- segments of L samples with 50 % overlap, a Hanning window on each,
// the squared magnitude of each segment's discrete Fourier transform averaged
// over the segments -- then the span correction of Eq. PSD_corr,
//   PSD_corr = PSD + 10 log10(b_exp / b_m)   (dB),  i.e. PSD x b_exp / b_m.
//
// One CTA per signal.  The segments are transformed two at a time: segment a
// is the real and segment b the imaginary part of one complex sequence z, and
// with Z its transform,
//   A_k = (Z_k + conj Z_{L-k}) / 2,   B_k = (Z_k - conj Z_{L-k}) / (2 i),
// so one complex FFT of length L serves two segments.  The FFT is an
// iterative radix-2 decimation-in-time transform in shared memory (input
// written in bit-reversed order, log2 L butterfly stages, twiddles
// exp(-2 pi i j / L) tabulated once per CTA).  Everything is FP64.
// Bytes per signal: its N valid samples are read once per segment they fall
// in (twice with the 50 % overlap), L / 2 + 1 values are written.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "../../include/fwh.h"
#include "fwh_internal.cuh"

fwh_status fwh_fail_handle(fwh_handle h, fwh_status st, const char *msg);

namespace {

constexpr int kPsdThreads = 256;
constexpr int kPsdMaxSeg = 4096;

struct PsdArgs {
  const double *p;          // [n_sig][ld]
  const long long *n_valid; // [n_sig] or null (every signal has ld samples)
  long long ld;
  int L, log2L;
  double fs, span, p_ref;
  int detrend;
  double *out;              // [n_sig][L / 2 + 1]
};

__device__ __forceinline__ double block_sum(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();  // red may still be read by a previous sum
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];  // same order in every thread
  return s;
}

__global__ void __launch_bounds__(kPsdThreads) k_psd(PsdArgs a) {
  extern __shared__ __align__(16) double2 sm[];
  const int L = a.L, half = L >> 1, tid = threadIdx.x, T = blockDim.x;
  double2 *z = sm;                                        // [L]
  double2 *tw = z + L;                                    // [L / 2]
  double *wv = reinterpret_cast<double *>(tw + half);     // [L]
  double *acc = wv + L;                                   // [L / 2 + 1]
  double *red = acc + half + 1;                           // [T / 32]
  const int sig = blockIdx.x;
  long long n = a.n_valid ? a.n_valid[sig] : a.ld;
  n = n < 0 ? 0 : (n > a.ld ? a.ld : n);
  const int K = n < L ? 0 : (int)((n - L) / half) + 1;  // segments
  for (int j = tid; j < half; j += T) {
    double s, c;
    sincospi(-2.0 * (double)j / (double)L, &s, &c);
    tw[j] = make_double2(c, s);
  }
  double w2 = 0.0;
  for (int i = tid; i < L; i += T) {
    const double w = 0.5 - 0.5 * cospi(2.0 * (double)i / (double)L);  // periodic Hanning
    wv[i] = w;
    w2 += w * w;
  }
  for (int k = tid; k <= half; k += T) acc[k] = 0.0;
  const double wsum2 = block_sum(w2, red);  // also orders the tables before use
  const double *x = a.p + (long long)sig * a.ld;
  for (int s = 0; s < K; s += 2) {
    const bool hb = s + 1 < K;
    const double *xa = x + (long long)s * half, *xb = x + (long long)(s + 1) * half;
    double ma = 0.0, mb = 0.0;
    if (a.detrend) {
      double sa = 0.0, sb = 0.0;
      for (int i = tid; i < L; i += T) {
        sa += xa[i];
        if (hb) sb += xb[i];
      }
      ma = block_sum(sa, red) / L;
      mb = block_sum(sb, red) / L;
    }
    for (int i = tid; i < L; i += T) {
      const double va = wv[i] * (xa[i] - ma);
      const double vb = hb ? wv[i] * (xb[i] - mb) : 0.0;
      z[__brev((unsigned)i) >> (32 - a.log2L)] = make_double2(va, vb);
    }
    __syncthreads();
    for (int h = 1, step = half; h < L; h <<= 1, step >>= 1) {
      for (int b = tid; b < half; b += T) {
        const int pos = b & (h - 1);
        const int i = ((b - pos) << 1) + pos, j = i + h;
        const double2 w = tw[pos * step], zj = z[j], zi = z[i];
        const double tr = w.x * zj.x - w.y * zj.y, ti = w.x * zj.y + w.y * zj.x;
        z[i] = make_double2(zi.x + tr, zi.y + ti);
        z[j] = make_double2(zi.x - tr, zi.y - ti);
      }
      __syncthreads();
    }
    for (int k = tid; k <= half; k += T) {
      const double2 zk = z[k & (L - 1)], zm = z[(L - k) & (L - 1)];
      const double ar = 0.5 * (zk.x + zm.x), ai = 0.5 * (zk.y - zm.y);
      const double br = 0.5 * (zk.y + zm.y), bi = -0.5 * (zk.x - zm.x);
      acc[k] += (ar * ar + ai * ai) + (br * br + bi * bi);
    }
    __syncthreads();
  }
  double *o = a.out + (long long)sig * (half + 1);
  for (int k = tid; k <= half; k += T) {
    double v = nan("");
    if (K > 0) {
      v = acc[k] / ((double)K * a.fs * wsum2);
      if (k > 0 && k < half) v *= 2.0;  // one-sided
      v *= a.span;                       // Eq. PSD_corr
      if (a.p_ref > 0.0) v = 10.0 * log10(v / (a.p_ref * a.p_ref));
    }
    o[k] = v;
  }
}

bool on_device(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

fwh_status fail(fwh_status st, const std::string &m) { return fwh_fail_handle(nullptr, st, m.c_str()); }

}  // namespace

extern "C" fwh_status fwh_psd(int64_t n_sig, const double *p, int64_t ld, const int64_t *n_valid,
                              double fs, int64_t nperseg, int detrend, double span_ratio,
                              double p_ref, double *psd, void *stream) {
  if (n_sig < 1 || n_sig > 0x7fffffff) return fail(FWH_ERR_ARG, "n_sig must be in [1, 2^31)");
  if (!p || !psd) return fail(FWH_ERR_ARG, "p or psd is NULL");
  if (ld < 1) return fail(FWH_ERR_ARG, "ld must be >= 1");
  if (!(fs > 0.0) || !std::isfinite(fs)) return fail(FWH_ERR_ARG, "fs must be > 0");
  if (nperseg < 16 || nperseg > kPsdMaxSeg || (nperseg & (nperseg - 1)))
    return fail(FWH_ERR_ARG, "nperseg must be a power of two in [16, 4096]");
  if (detrend != 0 && detrend != 1) return fail(FWH_ERR_ARG, "detrend must be 0 or 1");
  if (!(span_ratio > 0.0) || !std::isfinite(span_ratio))
    return fail(FWH_ERR_ARG, "span_ratio must be > 0");
  if (!(p_ref >= 0.0) || !std::isfinite(p_ref)) return fail(FWH_ERR_ARG, "p_ref must be >= 0");
  const bool nv_dev = n_valid && on_device(n_valid);
  if (n_valid && !nv_dev)
    for (int64_t i = 0; i < n_sig; ++i)
      if (n_valid[i] < 0 || n_valid[i] > ld)
        return fail(FWH_ERR_ARG, "n_valid[" + std::to_string(i) + "] outside [0, ld]");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int L = (int)nperseg;
  int log2L = 0;
  while ((1 << log2L) < L) ++log2L;
  const size_t in_bytes = (size_t)n_sig * ld * sizeof(double);
  const size_t out_bytes = (size_t)n_sig * (L / 2 + 1) * sizeof(double);
  const bool p_dev = on_device(p), o_dev = on_device(psd);
  void *dp = nullptr, *dn = nullptr, *dout = nullptr;
  cudaError_t e = cudaSuccess;
  auto release = [&]() {
    if (dp) cudaFreeAsync(dp, s);
    if (dn) cudaFreeAsync(dn, s);
    if (dout) cudaFreeAsync(dout, s);
  };
  if (!p_dev && (e = cudaMallocAsync(&dp, in_bytes, s)) == cudaSuccess)
    e = cudaMemcpyAsync(dp, p, in_bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && n_valid && !nv_dev &&
      (e = cudaMallocAsync(&dn, (size_t)n_sig * sizeof(int64_t), s)) == cudaSuccess)
    e = cudaMemcpyAsync(dn, n_valid, (size_t)n_sig * sizeof(int64_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !o_dev) e = cudaMallocAsync(&dout, out_bytes, s);
  PsdArgs a{};
  a.p = p_dev ? p : static_cast<const double *>(dp);
  a.n_valid = reinterpret_cast<const long long *>(n_valid ? (nv_dev ? n_valid : dn) : nullptr);
  a.ld = ld;
  a.L = L;
  a.log2L = log2L;
  a.fs = fs;
  a.span = span_ratio;
  a.p_ref = p_ref;
  a.detrend = detrend;
  a.out = o_dev ? psd : static_cast<double *>(dout);
  const size_t smem = (size_t)L * sizeof(double2) + (size_t)(L / 2) * sizeof(double2) +
                      (size_t)L * sizeof(double) + (size_t)(L / 2 + 1) * sizeof(double) +
                      (kPsdThreads / 32) * sizeof(double);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_psd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) {
    k_psd<<<(unsigned)n_sig, kPsdThreads, smem, s>>>(a);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && !o_dev) e = cudaMemcpyAsync(psd, dout, out_bytes, cudaMemcpyDeviceToHost, s);
  release();
  if (e == cudaSuccess && (!o_dev || !p_dev || (n_valid && !nv_dev))) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? FWH_ERR_OOM : FWH_ERR_CUDA,
                std::string("fwh_psd: ") + cudaGetErrorString(e));
  }
  return FWH_OK;
}
