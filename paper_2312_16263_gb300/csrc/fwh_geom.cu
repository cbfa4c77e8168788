// Per-(panel, observer) geometry of the wind-tunnel FW-H integral, in FP64.
//
// "compute R" (Sec. III B): the convected distance of the Garrick triangle
// with the angle of attack (Eqs. R_New, R_s_New) in the closed form
//   s = M0 (U.d),  R* = sqrt(s^2 + beta^2 |d|^2),  R = (R* - s) / beta^2,
//   R-hat = (d - M0 R U) / R,
// which is Eqs. R1_prime..R2_New rotated back in one step.  "compute t": per
// observer R_max and R_min over all panels (the paper's MPI_ALLREDUCE), here
// one block-wide reduction per observer.  Then the coefficients of the eight
// observer-independent series in the source-time pressure of Eqs. pT_WT_nd
// and pL_WT_nd, with M = -M0 U, M^2 = M0^2, M_R = M . R-hat, D = 1 - M_R,
// S = dS / (4 pi):
//   Qn_dot : S / (R D^2)
//   Qn     : S (M_R - M0^2) / (M0 R^2 D^3)
//   L_dot  : S M0 R-hat / (R D^2)
//   L      : S [R-hat / (R^2 D^2) - M / (R^2 D^2) + R-hat (M_R - M0^2) / (R^2 D^3)]
// and the arrival shift delta = M0 (R_max - R) = (i0 + f) dt of the source
// sample feeding observer bin j (tau = t_j - M0 R, Eq. tau2) with the
// natural-spline weights a = 1 - f, b = f, (a^3 - a) dt^2/6, (b^3 - b) dt^2/6.
#include "fwh_internal.cuh"

namespace fwh {

namespace {

__device__ __forceinline__ void convected(const double d[3], double mach, double ca,
                                          double sa, double &R, double Rh[3]) {
  const double beta2 = 1.0 - mach * mach;
  const double ud = ca * d[0] + sa * d[1];
  const double s = mach * ud;
  const double dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  const double Rs = sqrt(s * s + beta2 * dd);
  R = (Rs - s) / beta2;
  const double inv = 1.0 / R;
  Rh[0] = (d[0] - mach * R * ca) * inv;
  Rh[1] = (d[1] - mach * R * sa) * inv;
  Rh[2] = d[2] * inv;
}

__global__ void __launch_bounds__(256) k_window(GeomArgs a) {
  const int o = blockIdx.x;
  double x[3] = {a.x[3 * o], a.x[3 * o + 1], a.x[3 * o + 2]};
  double rmax = -1e300, rmin = 1e300;
  for (int p = threadIdx.x; p < a.P; p += blockDim.x) {
    double d[3] = {x[0] - a.y[3 * p], x[1] - a.y[3 * p + 1], x[2] - a.y[3 * p + 2]};
    double R, Rh[3];
    convected(d, a.mach, a.ca, a.sa, R, Rh);
    rmax = fmax(rmax, R);
    rmin = fmin(rmin, R);
  }
  for (int off = 16; off > 0; off >>= 1) {
    rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, off));
    rmin = fmin(rmin, __shfl_xor_sync(0xffffffffu, rmin, off));
  }
  __shared__ double smax[8], smin[8];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    smax[w] = rmax;
    smin[w] = rmin;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
      rmax = fmax(rmax, smax[i]);
      rmin = fmin(rmin, smin[i]);
    }
    a.Rmax[o] = rmax;
    a.Rmin[o] = rmin;
  }
}

template <typename T>
__device__ __forceinline__ void store_i0(T *rec, int i0);
template <>
__device__ __forceinline__ void store_i0<float>(float *slot, int i0) {
  *slot = __int_as_float(i0);
}
template <>
__device__ __forceinline__ void store_i0<double>(double *slot, int i0) {
  *slot = (double)i0;
}

template <typename T>
__global__ void __launch_bounds__(128) k_coef(GeomArgs a, T *coef) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.P) return;
  for (int o = blockIdx.y; o < a.O; o += gridDim.y) {  // grid y is capped at 65535
    const double d[3] = {a.x[3 * o] - a.y[3 * p], a.x[3 * o + 1] - a.y[3 * p + 1],
                         a.x[3 * o + 2] - a.y[3 * p + 2]};
    double R, Rh[3];
    convected(d, a.mach, a.ca, a.sa, R, Rh);
    const double M0 = a.mach;
    const double U[3] = {a.ca, a.sa, 0.0};
    const double URh = U[0] * Rh[0] + U[1] * Rh[1];
    const double MR = -M0 * URh;               // M = -M0 U (surface moves at -U0)
    const double D = 1.0 - MR;
    const double S = a.dS[p] * 0.079577471545947667884441881686257181;  // 1/(4 pi)
    const double iR = 1.0 / R, iD = 1.0 / D;
    const double k1 = S * iR * iD * iD;        // S / (R D^2)
    const double k2 = k1 * iR;                 // S / (R^2 D^2)
    const double mrm = MR - M0 * M0;           // M_R - M^2
    double c[8];
    c[0] = k1;
    c[1] = k2 * mrm * iD / M0;
    for (int i = 0; i < 3; ++i) {
      c[2 + i] = k1 * M0 * Rh[i];
      c[5 + i] = k2 * (Rh[i] + M0 * U[i] + Rh[i] * mrm * iD);
    }
    const double q = M0 * (a.Rmax[o] - R) / a.dt;
    double fl = floor(q);
    double f = q - fl;
    const double aw = 1.0 - f, bw = f;
    const double h26 = a.dt * a.dt / 6.0;
    T *rec = coef + ((size_t)p * a.O + o) * kRec;
    for (int i = 0; i < 8; ++i) rec[slot::c + i] = (T)c[i];
    rec[slot::a] = (T)aw;
    rec[slot::b] = (T)bw;
    rec[slot::cc] = (T)((aw * aw * aw - aw) * h26);
    rec[slot::dd] = (T)((bw * bw * bw - bw) * h26);
    rec[slot::off] = (T)0;
    rec[14] = (T)0;
    rec[15] = (T)0;
    store_i0<T>(rec + slot::i0, (int)fl);
  }
}

// Observer window length N_o = floor((t_end - t_start)/dt) + 1 (Eqs. t_start,
// t_end), clamped to [0, nt]: every operation rounded on its own, as the
// host's planner computes it (no fused multiply-add), so both agree exactly.
__global__ void k_nvalid(const double *Rmax, const double *Rmin, int O, double mach, double dt,
                         int nt, int *n_valid) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= O) return;
  const double tau_max = __dmul_rn((double)(nt - 1), dt);
  const double ts = __dmul_rn(mach, Rmax[o]);
  const double te = __dadd_rn(tau_max, __dmul_rn(mach, Rmin[o]));
  double v = __dadd_rn(floor(__ddiv_rn(__dsub_rn(te, ts), dt)), 1.0);
  v = fmax(0.0, fmin((double)nt, v));
  n_valid[o] = (int)v;
}

}  // namespace

cudaError_t launch_nvalid(const double *Rmax, const double *Rmin, int O, double mach, double dt,
                          int nt, int *n_valid, cudaStream_t s) {
  if (O <= 0) return cudaSuccess;
  k_nvalid<<<(O + 127) / 128, 128, 0, s>>>(Rmax, Rmin, O, mach, dt, nt, n_valid);
  return cudaGetLastError();
}

cudaError_t launch_window(const GeomArgs &a, cudaStream_t s) {
  if (a.O <= 0) return cudaSuccess;
  k_window<<<a.O, 256, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_coef(const GeomArgs &a, T *coef, cudaStream_t s) {
  if (a.O <= 0 || a.P <= 0) return cudaSuccess;
  dim3 grid((a.P + 127) / 128, a.O < 65535 ? a.O : 65535);
  k_coef<T><<<grid, 128, 0, s>>>(a, coef);
  return cudaGetLastError();
}

template cudaError_t launch_coef<float>(const GeomArgs &, float *, cudaStream_t);
template cudaError_t launch_coef<double>(const GeomArgs &, double *, cudaStream_t);

}  // namespace fwh
