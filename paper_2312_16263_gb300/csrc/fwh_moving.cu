// General moving surface (Sec. II B): the permeable-surface Farassat 1A
// integrals of Eqs. pT and pL for panels that move in a medium at rest, with
// the retarded time of Eq. tau, FP64 throughout.
//
// Unlike the wind-tunnel form, the distance r, the radiation direction r-hat
// and the Mach numbers change with source time, so every (panel, observer)
// has its own source-time signal and its own arrival times: the spline that
// carries a panel's signal onto the observer grid cannot be shared between
// observers.  Three kernels:
//  * k_mseries, per (panel, frame): the observer-independent series Q_n
//    (Eq. Qn), L_i (Eq. Li), the surface Mach vector v / c0 and their
//    second-order source-time derivatives (Sec. III B), one 16-value row;
//  * k_mwindow, per observer: the earliest and latest arrival over panels of
//    the first and last frame (the window t_start, t_end and N_o);
//  * k_mscatter, per (observer, tile of 128 panels): a thread per panel
//    evaluates, at every frame, the arrival t_i = tau_i + Delta (the positive
//    root of |b + w Delta| = c0 Delta, b = x0 + w tau - y) and the bracket g_i
//    of Eqs. pT + pL times dS / (4 pi); solves the natural-spline moments of g
//    and of t over source time (tridiagonal elimination in a scratch column);
//    then walks the observer bins: t_j lies in the interval whose arrival
//    times bracket it, tau* solves t(tau*) = t_j there by Newton's method on
//    the spline of t (three steps from the linear estimate reach FP64
//    rounding for subsonic motion), and the spline of g at tau* is reduced
//    over each warp's panels before one FP64 atomic per warp and bin.
// Scratch: four FP64 columns of nt per (panel, observer) of a launch; the
// host splits the observers into launches that fit the scratch budget (16 GiB
// by default: a budget of 2 GiB, four observers per launch on the 8192-panel
// x 2048-step benchmark case, measured 10 % slower, the grid then filling a
// third of the GPU).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/fwh.h"
#include "fwh_internal.cuh"

fwh_status fwh_fail_handle(fwh_handle h, fwh_status st, const char *msg);

namespace {

constexpr int kMRow = 16;     // series row: Qn, Qn', L(3), L'(3), M(3), M'(3), 2 pad
constexpr int kMTile = 128;   // panels per scatter CTA
constexpr double kInv4Pi = 0.079577471545947667884441881686257181;

struct MovArgs {
  const double *y, *n, *v;    // [nt][P][3]
  const double *dS;           // [P]
  const double *fields;       // [nt][5][P]
  const double *x0, *w;       // [O][3], [3]
  double c0, rho0, dt;
  int P, nt, O;
  double *S;                  // [nt][kMRow][P] series (panel fastest)
  double *ts, *te;            // [O] window
  int *nv;                    // [O]
  double *p_out;              // [O][nt]
  double *scratch;            // [4][nt][P * n_obs of the launch]
  int o_lo, n_obs;            // observers of this launch
};

// Q_n (Eq. Qn) and L_i (Eq. Li with P_ij = p' delta_ij) of panel p at frame i.
__device__ __forceinline__ void mv_integrands(const MovArgs &a, int p, int i, double &qn,
                                              double L[3]) {
  const double *n = a.n + ((size_t)i * a.P + p) * 3, *v = a.v + ((size_t)i * a.P + p) * 3;
  const double *f = a.fields + (size_t)i * 5 * a.P + p;
  const double rho = a.rho0 + f[0];
  const double u[3] = {f[(size_t)a.P], f[2 * (size_t)a.P], f[3 * (size_t)a.P]};
  const double pp = f[4 * (size_t)a.P];
  double q = 0.0, un = 0.0, vn = 0.0;
  for (int c = 0; c < 3; ++c) {
    q += (a.rho0 * v[c] + rho * (u[c] - v[c])) * n[c];
    un += u[c] * n[c];
    vn += v[c] * n[c];
  }
  qn = q;
  for (int c = 0; c < 3; ++c) L[c] = pp * n[c] + rho * u[c] * (un - vn);
}

// Second-order source-time derivative weights of Sec. III B at frame i:
// central inside, one-sided three-point at the first and last frame.
__device__ __forceinline__ void fd_stencil(int i, int nt, int idx[3], double wgt[3]) {
  if (i == 0) {
    idx[0] = 0; idx[1] = 1; idx[2] = 2;
    wgt[0] = -3.0; wgt[1] = 4.0; wgt[2] = -1.0;
  } else if (i == nt - 1) {
    idx[0] = nt - 1; idx[1] = nt - 2; idx[2] = nt - 3;
    wgt[0] = 3.0; wgt[1] = -4.0; wgt[2] = 1.0;
  } else {
    idx[0] = i + 1; idx[1] = i - 1; idx[2] = i;
    wgt[0] = 1.0; wgt[1] = -1.0; wgt[2] = 0.0;
  }
}

__global__ void __launch_bounds__(256) k_mseries(MovArgs a) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;  // e = i P + p
  if (e >= (long)a.P * a.nt) return;
  const int p = (int)(e % a.P), i = (int)(e / a.P);
  double qn, L[3];
  mv_integrands(a, p, i, qn, L);
  int idx[3];
  double wgt[3];
  fd_stencil(i, a.nt, idx, wgt);
  const double inv2h = 0.5 / a.dt;
  double qd = 0.0, Ld[3] = {0.0, 0.0, 0.0}, vd[3] = {0.0, 0.0, 0.0};
  for (int s = 0; s < 3; ++s) {
    if (wgt[s] == 0.0) continue;
    double q2, L2[3];
    mv_integrands(a, p, idx[s], q2, L2);
    const double *v2 = a.v + ((size_t)idx[s] * a.P + p) * 3;
    qd += wgt[s] * q2;
    for (int c = 0; c < 3; ++c) {
      Ld[c] += wgt[s] * L2[c];
      vd[c] += wgt[s] * v2[c];
    }
  }
  const double *v = a.v + ((size_t)i * a.P + p) * 3;
  double *row = a.S + (size_t)i * kMRow * a.P + p;  // value q at row[q P]
  const size_t P = a.P;
  row[0] = qn;
  row[P] = qd * inv2h;
  for (int c = 0; c < 3; ++c) {
    row[(2 + c) * P] = L[c];
    row[(5 + c) * P] = Ld[c] * inv2h;
    row[(8 + c) * P] = v[c] / a.c0;              // M
    row[(11 + c) * P] = vd[c] * inv2h / a.c0;    // M-dot
  }
}

// Delay Delta of one source sample: the non-negative root of
// (c0^2 - w.w) Delta^2 - 2 (b.w) Delta - b.b = 0 (Eq. tau, r = c0 Delta).
__device__ __forceinline__ double mv_delay(const MovArgs &a, const double x0[3], double tau,
                                           const double *y, double b[3]) {
  for (int c = 0; c < 3; ++c) b[c] = x0[c] + a.w[c] * tau - y[c];
  const double ww = a.w[0] * a.w[0] + a.w[1] * a.w[1] + a.w[2] * a.w[2];
  const double bw = b[0] * a.w[0] + b[1] * a.w[1] + b[2] * a.w[2];
  const double bb = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
  const double q = a.c0 * a.c0 - ww;
  return (bw + sqrt(bw * bw + q * bb)) / q;
}

__global__ void __launch_bounds__(256) k_mwindow(MovArgs a) {
  const int o = blockIdx.x;
  const double x0[3] = {a.x0[3 * o], a.x0[3 * o + 1], a.x0[3 * o + 2]};
  const double tau1 = (double)(a.nt - 1) * a.dt;
  double ts = -1e300, te = 1e300;
  for (int p = threadIdx.x; p < a.P; p += blockDim.x) {
    double b[3];
    const double d0 = mv_delay(a, x0, 0.0, a.y + (size_t)p * 3, b);
    const double d1 = mv_delay(a, x0, tau1, a.y + ((size_t)(a.nt - 1) * a.P + p) * 3, b);
    ts = fmax(ts, d0);
    te = fmin(te, tau1 + d1);
  }
  for (int off = 16; off > 0; off >>= 1) {
    ts = fmax(ts, __shfl_xor_sync(0xffffffffu, ts, off));
    te = fmin(te, __shfl_xor_sync(0xffffffffu, te, off));
  }
  __shared__ double sts[8], ste[8];
  const int wid = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    sts[wid] = ts;
    ste[wid] = te;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
      ts = fmax(ts, sts[i]);
      te = fmin(te, ste[i]);
    }
    double v = __dadd_rn(floor(__ddiv_rn(__dsub_rn(te, ts), a.dt)), 1.0);
    v = fmax(0.0, fmin((double)a.nt, v));
    a.ts[o] = ts;
    a.te[o] = te;
    a.nv[o] = (int)v;
  }
}

// Natural cubic-spline moments of column c (stride `ld` between samples):
// m_0 = m_{n-1} = 0, m_{i-1} + 4 m_i + m_{i+1} = 6 (c_{i+1} - 2 c_i + c_{i-1})
// / h^2, by tridiagonal elimination; ipiv[i] = 1/pivot of row i (piv_1 = 4,
// piv_i = 4 - 1/piv_{i-1}), constant from row 63 on (it has converged to
// 2 + sqrt 3 to FP64 rounding long before).
constexpr int kPiv = 64;
__device__ void spline_moments(const double *c, double *m, long ld, int n, double h,
                               const double *ipiv) {
  const double s6 = 6.0 / (h * h);
  m[0] = 0.0;
  m[(long)(n - 1) * ld] = 0.0;
  if (n < 3) return;
  double prev = 0.0, cm = c[0], c0 = c[ld];
  for (int i = 1; i <= n - 2; ++i) {
    const double cp1 = c[(long)(i + 1) * ld];
    const double r = s6 * (cp1 - 2.0 * c0 + cm);
    prev = (r - prev) * ipiv[i < kPiv ? i : kPiv - 1];
    m[(long)i * ld] = prev;
    cm = c0;
    c0 = cp1;
  }
  double mn = 0.0;
  for (int i = n - 2; i >= 1; --i) {
    const double v = m[(long)i * ld] - mn * ipiv[i < kPiv ? i : kPiv - 1];
    m[(long)i * ld] = v;
    mn = v;
  }
}

__global__ void __launch_bounds__(kMTile, 8) k_mscatter(MovArgs a) {
  const int ob = blockIdx.y;               // observer within the launch
  const int o = a.o_lo + ob;
  const int p = blockIdx.x * kMTile + threadIdx.x;
  const bool live = p < a.P;
  const int pp = live ? p : a.P - 1;
  const long ld = (long)a.P * a.n_obs;     // scratch column stride
  const long col = (long)ob * a.P + pp;
  double *G = a.scratch + col, *MG = G + (long)a.nt * ld, *TT = MG + (long)a.nt * ld,
         *MT = TT + (long)a.nt * ld;
  const double x0[3] = {a.x0[3 * o], a.x0[3 * o + 1], a.x0[3 * o + 2]};
  const double S4 = a.dS[pp] * kInv4Pi;
  const double c0 = a.c0;
  __shared__ double ipiv[kPiv];
  if (threadIdx.x == 0) {
    double piv = 4.0;
    ipiv[0] = 0.0;
    for (int i = 1; i < kPiv; ++i) {
      if (i > 1) piv = 4.0 - ipiv[i - 1];
      ipiv[i] = 1.0 / piv;
    }
  }
  __syncthreads();
  // signal g and arrival time t at every frame (Eqs. pT, pL, tau); threads
  // past the last panel only join the bin reductions below
  for (int i = 0; live && i < a.nt; ++i) {
    const double tau = (double)i * a.dt;
    const double *rw = a.S + (size_t)i * kMRow * a.P + pp;
    double row[14];
    for (int q = 0; q < 14; ++q) row[q] = rw[(size_t)q * a.P];
    double b[3];
    const double d = mv_delay(a, x0, tau, a.y + ((size_t)i * a.P + pp) * 3, b);
    const double r = c0 * d, ir = 1.0 / r;
    double rh[3];
    for (int c = 0; c < 3; ++c) rh[c] = (b[c] + a.w[c] * d) * ir;
    double Mr = 0.0, Mdr = 0.0, M2 = 0.0, Lr = 0.0, Ldr = 0.0, LM = 0.0;
    for (int c = 0; c < 3; ++c) {
      Mr += row[8 + c] * rh[c];
      Mdr += row[11 + c] * rh[c];
      M2 += row[8 + c] * row[8 + c];
      Lr += row[2 + c] * rh[c];
      Ldr += row[5 + c] * rh[c];
      LM += row[2 + c] * row[8 + c];
    }
    const double D = 1.0 - Mr, iD = 1.0 / D;
    const double k = r * Mdr + c0 * (Mr - M2);
    const double thick = row[1] * ir * iD * iD + row[0] * k * ir * ir * iD * iD * iD;
    const double load = Ldr / c0 * ir * iD * iD + (Lr - LM) * ir * ir * iD * iD +
                        Lr * k / c0 * ir * ir * iD * iD * iD;
    G[(long)i * ld] = S4 * (thick + load);
    TT[(long)i * ld] = tau + d;
  }
  if (live) {
    spline_moments(G, MG, ld, a.nt, a.dt, ipiv);
    spline_moments(TT, MT, ld, a.nt, a.dt, ipiv);
  }
  // observer bins: every thread walks the same j, each warp sums its panels
  // and adds them with one atomic (no CTA barrier per bin)
  const int nv = a.nv[o];
  const double ts = a.ts[o], h = a.dt, h26 = a.dt * a.dt / 6.0;
  int k = 0;
  for (int j = 0; j < nv; ++j) {
    double val = 0.0;
    if (live) {
    const double tj = ts + (double)j * h;
    while (k < a.nt - 2 && TT[(long)(k + 1) * ld] < tj) ++k;
    const double t0 = TT[(long)k * ld], t1 = TT[(long)(k + 1) * ld];
    const double mt0 = MT[(long)k * ld], mt1 = MT[(long)(k + 1) * ld];
    // Newton on S_t(x) = A t0 + B t1 + ((A^3 - A) mt0 + (B^3 - B) mt1) h^2/6 = tj,
    // x = B in [0, 1], A = 1 - B
    double B = (t1 > t0) ? (tj - t0) / (t1 - t0) : 0.0;
    B = fmin(1.0, fmax(0.0, B));
    for (int it = 0; it < 3; ++it) {
      const double A = 1.0 - B;
      const double f = A * t0 + B * t1 + ((A * A * A - A) * mt0 + (B * B * B - B) * mt1) * h26 - tj;
      const double df = (t1 - t0) + ((1.0 - 3.0 * A * A) * mt0 + (3.0 * B * B - 1.0) * mt1) * h26;
      B = fmin(1.0, fmax(0.0, B - f / df));
    }
    const double A = 1.0 - B;
    val = A * G[(long)k * ld] + B * G[(long)(k + 1) * ld] +
          ((A * A * A - A) * MG[(long)k * ld] + (B * B * B - B) * MG[(long)(k + 1) * ld]) * h26;
    }
    for (int off = 16; off > 0; off >>= 1) val += __shfl_xor_sync(0xffffffffu, val, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(a.p_out + (size_t)o * a.nt + j, val);
  }
}

// Scratch budget of one call (bytes; 0: the default of 16 GiB), process-wide.
std::atomic<int64_t> g_mov_scratch{0};
constexpr int64_t kMovScratchDefault = (int64_t)16 << 30;

bool on_device(const void *p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

fwh_status failm(fwh_status st, const std::string &m) {
  return fwh_fail_handle(nullptr, st, m.c_str());
}

}  // namespace

extern "C" fwh_status fwh_set_moving_scratch(int64_t bytes) {
  if (bytes < 0) return failm(FWH_ERR_ARG, "scratch budget must be >= 0 bytes");
  g_mov_scratch.store(bytes);
  return FWH_OK;
}

extern "C" fwh_status fwh_forward_moving(int64_t P, int64_t nt, const double *y,
                                         const double *normals, const double *velocities,
                                         const double *areas, double c0, double rho0,
                                         double dt, const double *fields, int64_t O,
                                         const double *x0, const double *w, double *p_out,
                                         double *t_start, int64_t *n_valid, void *stream) {
  if (P < 1 || P > (1 << 30)) return failm(FWH_ERR_ARG, "n_panels out of range");
  if (nt < 3 || nt > (1 << 24)) return failm(FWH_ERR_ARG, "nt must be in [3, 2^24]");
  if (O < 1 || O > 65535) return failm(FWH_ERR_ARG, "n_obs must be in [1, 65535]");
  if (!y || !normals || !velocities || !areas || !fields || !x0 || !w || !p_out)
    return failm(FWH_ERR_ARG, "NULL argument");
  if (!(c0 > 0.0) || !(rho0 > 0.0) || !(dt > 0.0) || !std::isfinite(c0) || !std::isfinite(dt))
    return failm(FWH_ERR_ARG, "c0, rho0 and dt must be > 0");
  std::vector<double> wh(3);
  if (on_device(w)) {
    if (cudaMemcpy(wh.data(), w, 3 * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
      return failm(FWH_ERR_CUDA, "cannot read w");
  } else {
    wh.assign(w, w + 3);
  }
  if (!(wh[0] * wh[0] + wh[1] * wh[1] + wh[2] * wh[2] < c0 * c0))
    return failm(FWH_ERR_ARG, "observer speed |w| must be below c0");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t geo = (size_t)nt * P * 3 * sizeof(double);
  const size_t fb = (size_t)nt * 5 * P * sizeof(double);
  const size_t ob = (size_t)O * nt * sizeof(double);
  std::vector<void *> tmp;
  cudaError_t e = cudaSuccess;
  auto dev_in = [&](const double *src, size_t bytes) -> const double * {
    if (e != cudaSuccess) return nullptr;
    if (on_device(src)) return src;
    void *d = nullptr;
    if ((e = cudaMallocAsync(&d, bytes, s)) != cudaSuccess) return nullptr;
    tmp.push_back(d);
    e = cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, s);
    return static_cast<const double *>(d);
  };
  auto dev_buf = [&](size_t bytes) -> void * {
    if (e != cudaSuccess) return nullptr;
    void *d = nullptr;
    if ((e = cudaMallocAsync(&d, bytes, s)) != cudaSuccess) return nullptr;
    tmp.push_back(d);
    return d;
  };
  MovArgs a{};
  a.y = dev_in(y, geo);
  a.n = dev_in(normals, geo);
  a.v = dev_in(velocities, geo);
  a.dS = dev_in(areas, (size_t)P * sizeof(double));
  a.fields = dev_in(fields, fb);
  a.x0 = dev_in(x0, (size_t)O * 3 * sizeof(double));
  double *dw = static_cast<double *>(dev_buf(3 * sizeof(double)));
  if (e == cudaSuccess) e = cudaMemcpyAsync(dw, wh.data(), 3 * sizeof(double), cudaMemcpyHostToDevice, s);
  a.w = dw;
  a.c0 = c0;
  a.rho0 = rho0;
  a.dt = dt;
  a.P = (int)P;
  a.nt = (int)nt;
  a.O = (int)O;
  a.S = static_cast<double *>(dev_buf((size_t)P * nt * kMRow * sizeof(double)));
  a.ts = static_cast<double *>(dev_buf((size_t)O * sizeof(double)));
  a.te = static_cast<double *>(dev_buf((size_t)O * sizeof(double)));
  a.nv = static_cast<int *>(dev_buf((size_t)O * sizeof(int)));
  const bool o_dev = on_device(p_out);
  a.p_out = o_dev ? p_out : static_cast<double *>(dev_buf(ob));
  // observers per launch: four scratch columns of nt per (panel, observer)
  // within the scratch budget (at least one observer per launch)
  const size_t per_obs = (size_t)4 * nt * P * sizeof(double);
  const int64_t budget = g_mov_scratch.load() > 0 ? g_mov_scratch.load() : kMovScratchDefault;
  const int n_obs = (int)std::max<size_t>(1, std::min<size_t>((size_t)O, (size_t)budget / per_obs));
  a.scratch = static_cast<double *>(dev_buf(per_obs * n_obs));
  if (e == cudaSuccess) e = cudaMemsetAsync(a.p_out, 0, ob, s);
  if (e == cudaSuccess) {
    const long n = (long)P * nt;
    k_mseries<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_mwindow<<<(unsigned)O, 256, 0, s>>>(a);
    e = cudaGetLastError();
  }
  for (int o0 = 0; e == cudaSuccess && o0 < O; o0 += n_obs) {
    a.o_lo = o0;
    a.n_obs = (int)std::min<int64_t>(n_obs, O - o0);
    dim3 grid((unsigned)((P + kMTile - 1) / kMTile), (unsigned)a.n_obs);
    k_mscatter<<<grid, kMTile, 0, s>>>(a);
    e = cudaGetLastError();
  }
  std::vector<double> hts;
  std::vector<int> hnv;
  if (e == cudaSuccess && (t_start || n_valid)) {
    hts.resize(O);
    hnv.resize(O);
    e = cudaMemcpyAsync(hts.data(), a.ts, O * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(hnv.data(), a.nv, O * sizeof(int), cudaMemcpyDeviceToHost, s);
  }
  if (e == cudaSuccess && !o_dev) e = cudaMemcpyAsync(p_out, a.p_out, ob, cudaMemcpyDeviceToHost, s);
  for (void *d : tmp) cudaFreeAsync(d, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return failm(e == cudaErrorMemoryAllocation ? FWH_ERR_OOM : FWH_ERR_CUDA,
                 std::string("fwh_forward_moving: ") + cudaGetErrorString(e));
  }
  for (int64_t o = 0; o < O; ++o) {
    if (t_start) t_start[o] = hts[o];
    if (n_valid) n_valid[o] = hnv[o];
  }
  return FWH_OK;
}
