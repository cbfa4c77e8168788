// Adjoint of the forward scatter: a conflict-free gather over observers.
//
// The forward adds, for panel p, observer o and source sample k,
//   a g + cc m  to bin k - i0   and   b g + dd m  to bin k - i0 - 1,
// with g = c . F[k], m = c . M[k].  Its transpose, for the gradient G of the
// loss with respect to p_out (zero outside the valid bins 0 <= j < N_o), is
//   gF = a G[k - i0] + b G[k - i0 - 1],   gM = cc G[k - i0] + dd G[k - i0 - 1]
//   Xbar[p][k][s]     = sum_o c_s gF,     Xbar[p][k][8 + s] = sum_o c_s gM,
// so each (panel, sample) output is owned by one lane and summed over all
// observers in registers: no atomics, 20 FMA per (panel, sample, observer).
// Nothing from the forward pass is stored: only the per-(p, o) records
// (geometry, computed once per observer set) and G are read.
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
  const long blocks = (long)a.P * ((a.ntp / CH + 7) / 8);
  if (blocks <= 0) return cudaSuccess;
  k_adjoint<T, TK><<<(unsigned)blocks, 256, 0, s>>>(a.coef, Gt, a.Xbar, a.P, a.O, a.ntp);
  return cudaGetLastError();
}

template cudaError_t launch_adjoint<float>(const AdjArgs<float> &, cudaStream_t);
template cudaError_t launch_adjoint<double>(const AdjArgs<double> &, cudaStream_t);

}  // namespace fwh
