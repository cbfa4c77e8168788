// Observer-independent source-time series of the FW-H integrand ("compute
// Noise", Sec. III B), per panel and source sample:
//   Qn  = rho' (U.n) + (1 + rho') (u'.n)                  (Eq. Qn_New_nd)
//   L_c = p' n_c + (1 + rho') u'_c (U.n + u'.n)           (Eq. Li_New_nd)
// in pulsation-expanded form (no cancellation of O(1) terms in FP32), their
// second-order source-time derivatives (central inside, one-sided 3-point at
// the first and last frame), and the natural-cubic-spline second derivatives
// ("moments") of all eight series, used by the spline interpolation onto the
// observer grid ("interp pressure signal").  The spline of the per-panel
// signal sum_s c_s F_s has moments sum_s c_s m(F_s) by linearity, so the
// moments are computed once per panel instead of once per (panel, observer).
//
// FP64 (k_prep): the moments solve, on a window of the chunk plus a halo of H
// samples on each side (clipped to the record), the tridiagonal system
//   m_{j-1} + 4 m_j + m_{j+1} = 6 (F_{j+1} - 2 F_j + F_{j-1}) / dt^2
// with m = 0 at the window ends: at the record ends this is the natural end
// condition itself; at an artificial end the error decays as (2 - sqrt 3)^H
// into the chunk, below the arithmetic's rounding for the chosen H.  A CTA is
// 16 panels x 8 series, one thread per (panel, series), sequential over the
// window in source time; the forward elimination's values for the chunk and
// right halo wait in shared memory for the back substitution.
//
// FP32 (k_prep_iir): the same moments by two first-order recursive filters
// per 64-sample block (see the kernels), written as whole X tiles.
#include "fwh_internal.cuh"

#include <algorithm>

#include <cstdint>

namespace fwh {

__constant__ float c_inv_piv_f[kPivTab];
__constant__ double c_inv_piv_d[kPivTab];

cudaError_t upload_pivots(cudaStream_t s) {
  // 1/pivot of Gaussian elimination of tridiag(1, 4, 1) started at row 1:
  // piv_1 = 4, piv_j = 4 - 1/piv_{j-1}  (converges to 2 + sqrt 3).
  double invd[kPivTab];
  float invf[kPivTab];
  double piv = 4.0;
  invd[0] = 0.0;
  invf[0] = 0.0f;
  for (int j = 1; j < kPivTab; ++j) {
    if (j > 1) piv = 4.0 - invd[j - 1];
    invd[j] = 1.0 / piv;
    invf[j] = (float)invd[j];
  }
  cudaError_t e = cudaMemcpyToSymbolAsync(c_inv_piv_d, invd, sizeof(invd), 0,
                                          cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbolAsync(c_inv_piv_f, invf, sizeof(invf), 0, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

namespace {

template <typename T> __device__ __forceinline__ T inv_piv(int j);
template <> __device__ __forceinline__ float inv_piv<float>(int j) {
  return c_inv_piv_f[j < kPivTab ? j : kPivTab - 1];
}
template <> __device__ __forceinline__ double inv_piv<double>(int j) {
  return c_inv_piv_d[j < kPivTab ? j : kPivTab - 1];
}

constexpr int kPanelsPerCta = 16;     // adjoint-prep tile
constexpr int kThreads = kPanelsPerCta * 8;

template <typename T> struct PrepChunk;
template <> struct PrepChunk<float> { static constexpr int v = 128; };
template <> struct PrepChunk<double> { static constexpr int v = 64; };

// Forward-prep tile: lanes map to panels for coalesced field loads (128 bytes
// of one field component per warp-row), then to (panel, series) pairs.
template <typename T> struct PrepTile;
template <> struct PrepTile<double> { static constexpr int panels = 16, chunk = 64; };

// Integrand `which` (0: Qn, 1..3: L_c) of panel po at sample i.
template <typename T>
struct Integrand {
  const T *f;
  int P, po, which;
  T n0, n1, n2, nc, Un;
  __device__ __forceinline__ T operator()(int i) const {
    const T *b = f + (size_t)i * 5 * P + po;
    const T rho = b[0];
    const T u0 = b[(size_t)P], u1 = b[2 * (size_t)P], u2 = b[3 * (size_t)P];
    const T un = u0 * n0 + u1 * n1 + u2 * n2;
    if (which == 0) return rho * Un + (T(1) + rho) * un;
    const T pp = b[4 * (size_t)P];
    const T uc = which == 1 ? u0 : (which == 2 ? u1 : u2);
    return pp * nc + (T(1) + rho) * uc * (Un + un);
  }
};

// Element (sample i, value q) of a panel's FP64 X rows, plain [i][q].  (The
// FP32 rows, which pair consecutive samples, are written by k_prep_iir.)
template <typename T> __device__ __forceinline__ size_t xidx(int i, int q);
template <> __device__ __forceinline__ size_t xidx<double>(int i, int q) {
  return (size_t)i * kRec + q;
}

// Forward prep.  Phase A stages the four integrands Qn, L_1..3 of the tile's
// panels over the window (plus one sample each side for the FD stencil) in
// shared memory, [row][integrand][panel], computed from coalesced field
// loads.  Phase B runs one thread per (panel, series): the series value (the
// integrand or its FD derivative), the forward elimination of the windowed
// moment system and the back substitution.  Elimination values of the chunk
// wait in the moment slots of X itself (re-read by the same thread), those of
// the right halo in shared memory.
template <typename T>
__global__ void __launch_bounds__(PrepTile<T>::panels * 8) k_prep(PrepArgs<T> a) {
  constexpr int NP = PrepTile<T>::panels;
  constexpr int NT = NP * 8;
  constexpr int H = Prec<T>::halo;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x;
  const int n_pt = (a.P + NP - 1) / NP;  // 1D grid: panel tile fastest, then chunk
  const int p0 = (int)(blockIdx.x % n_pt) * NP;
  const int c0 = (a.c_lo + (int)(blockIdx.x / n_pt)) * a.chunk;
  const int c1 = min(c0 + a.chunk, a.ntp);
  const int nt = a.nt;
  // rows of this chunk sit at c0 mod x_ld in each panel's block of X
  const long xoff = (long)(c0 % a.x_ld) - c0;

  if (c0 >= nt) {  // chunk past the record: zero rows
    for (int idx = tid; idx < NP * (c1 - c0) * kRec; idx += NT) {
      const int pl = idx / ((c1 - c0) * kRec);
      const int r = idx % ((c1 - c0) * kRec);
      if (p0 + pl < a.P) a.X[((size_t)(p0 + pl) * a.x_ld + c0 % a.x_ld) * kRec + r] = T(0);
    }
    return;
  }
  const int ce = min(c1, nt);
  const int wa = max(0, c0 - H), wb = min(nt, ce + H);
  const int ra = max(0, wa - 1), rb = min(nt, wb + 1);  // integrand rows
  T *sb = reinterpret_cast<T *>(smem_raw);              // [rb - ra][4][NP]
  T *zh = sb + (size_t)(rb - ra) * 4 * NP;              // [H][NT] right-halo z

  // ---- phase A: integrands ---------------------------------------------------
  {
    const int lane = tid & 31, warp = tid >> 5;
    constexpr int RPW = 32 / NP;                        // rows per warp pass
    const int pl = lane % NP;
    const int p = p0 + pl;
    const bool live = p < a.P;
    const int po = live ? (a.perm ? a.perm[p] : p) : 0;
    T n0 = 0, n1 = 0, n2 = 0, Un = 0;
    if (live) {
      n0 = (T)a.n[3 * p];
      n1 = (T)a.n[3 * p + 1];
      n2 = (T)a.n[3 * p + 2];
      Un = (T)(a.ca * a.n[3 * p] + a.sa * a.n[3 * p + 1]);
    }
    const int stride = (NT / 32) * RPW;
    auto integrands = [&](int i, T &q, T &l0, T &l1, T &l2) {
      const T *b = a.fields + (size_t)i * 5 * a.P + po;
      const T rho = b[0];
      const T u0 = b[(size_t)a.P], u1 = b[2 * (size_t)a.P], u2 = b[3 * (size_t)a.P];
      const T pp = b[4 * (size_t)a.P];
      const T un = u0 * n0 + u1 * n1 + u2 * n2;
      const T r1 = T(1) + rho;
      const T utn = Un + un;
      q = rho * Un + r1 * un;                 // Qn   (Eq. Qn_New_nd)
      l0 = pp * n0 + r1 * u0 * utn;           // L_1  (Eq. Li_New_nd)
      l1 = pp * n1 + r1 * u1 * utn;
      l2 = pp * n2 + r1 * u2 * utn;
    };
    constexpr int U = 4;  // rows in flight per lane
    for (int i0 = ra + warp * RPW + lane / NP; i0 < rb; i0 += U * stride) {
      T q[U], l0[U], l1[U], l2[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = i0 + u * stride;
        q[u] = l0[u] = l1[u] = l2[u] = T(0);
        if (live && i < rb) integrands(i, q[u], l0[u], l1[u], l2[u]);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = i0 + u * stride;
        if (i < rb) {
          T *row = sb + (size_t)(i - ra) * 4 * NP + pl;
          row[0] = q[u];
          row[NP] = l0[u];
          row[2 * NP] = l1[u];
          row[3 * NP] = l2[u];
        }
      }
    }
  }
  __syncthreads();

  // ---- phase B: series, forward elimination, back substitution ----------------
  // warps 0, 1: the value series (1, 5, 6, 7) of panels 0-7, 8-15; warps 2, 3:
  // the derivative series (0, 2, 3, 4).  Lane = 4 x panel + integrand, so in
  // an interior chunk two whole warps finish after writing their values.
  static_assert(NP == 16 && NT == 128, "phase-B lane map");
  const int pl = ((tid >> 5) & 1) * 8 + ((tid & 31) >> 2);
  const int s = (tid >> 6) ? ((tid & 3) == 0 ? 0 : 1 + (tid & 3)) : ((tid & 3) == 0 ? 1 : 4 + (tid & 3));
  const int p = p0 + pl;
  if (p >= a.P) return;
  T *Xp = a.X + ((long)p * a.x_ld + xoff) * kRec;  // row i of the chunk at Xp + i kRec
  for (int i = max(c0, nt); i < c1; ++i) {  // rows past the record
    Xp[xidx<T>(i, s)] = T(0);
    Xp[xidx<T>(i, 8 + s)] = T(0);
  }
  const bool deriv = (s == 0) || (s >= 2 && s <= 4);
  const int q = (s <= 1) ? 0 : 1 + (s - 2) % 3;
  const T *col = sb + q * NP + pl;  // integrand q of this panel, row stride 4 NP
  auto B = [&](int i) -> T { return col[(size_t)(i - ra) * 4 * NP]; };
  const T inv2h = (T)(0.5 / a.dt);
  const T s6 = (T)(6.0 / (a.dt * a.dt));
  // Interior chunk (window rows inside 1 .. N - 2, so every derivative value
  // in it is a central difference): the moment solve commutes with the
  // central difference, so a derivative series' moments are the central
  // differences of its integrand's value-series moments.  The value-series
  // thread solves and writes both; the derivative-series thread only writes
  // its values.  Uniform across the CTA.
  const bool inner = wa >= 1 && ce + H <= nt - 1;
  if (inner && deriv) {
    for (int i = c0; i < ce; ++i) Xp[xidx<T>(i, s)] = (B(i + 1) - B(i - 1)) * inv2h;
    return;
  }
  const int sd = q == 0 ? 0 : 1 + q;  // the derivative series of integrand q
  auto F = [&](int i) -> T {
    if (!deriv) return B(i);
    if (i == 0) return (T(-3) * B(0) + T(4) * B(1) - B(2)) * inv2h;
    if (i == nt - 1) return (T(3) * B(nt - 1) - T(4) * B(nt - 2) + B(nt - 3)) * inv2h;
    return (B(i + 1) - B(i - 1)) * inv2h;
  };
  const int L = wb - wa;
  T Fprev = T(0), Fcur = F(wa), z = T(0), z_below = T(0);  // z_below: row c0 - 1
#pragma unroll 4
  for (int i = wa; i < wb; ++i) {
    const int j = i - wa;
    const T Fnext = (i + 1 < wb) ? F(i + 1) : T(0);
    if (i >= c0 && i < ce) Xp[xidx<T>(i, s)] = Fcur;
    if (j >= 1 && j <= L - 2) {
      const T r = s6 * (Fnext - T(2) * Fcur + Fprev);
      z = (r - z) * inv_piv<T>(j);
      if (i >= ce) {
        zh[(size_t)(i - ce) * NT + tid] = z;
      } else if (i >= c0) {
        Xp[xidx<T>(i, 8 + s)] = z;
      } else if (i == c0 - 1) {
        z_below = z;
      }
    }
    Fprev = Fcur;
    Fcur = Fnext;
  }
  // back substitution; in an interior chunk m_{i+1}' = (m_{i+2} - m_i) / (2 dt)
  // goes to the derivative series' moment slot as m_i is found
  T mnext = T(0), mnext2 = T(0);
  auto emit = [&](int i, T m) {  // m = m_i, mnext2 = m_{i+2}
    if (inner && i + 1 >= c0 && i + 1 < ce) Xp[xidx<T>(i + 1, 8 + sd)] = (mnext2 - m) * inv2h;
  };
  if (wb - 1 >= c0 && wb - 1 < ce) Xp[xidx<T>(wb - 1, 8 + s)] = T(0);
  const int ilo = max(c0, wa + 1);
  int i = wb - 2;
  // right halo (elimination values in shared memory)
  for (; i >= ilo && i >= ce; --i) {
    const T m = zh[(size_t)(i - ce) * NT + tid] - mnext * inv_piv<T>(i - wa);
    emit(i, m);
    mnext2 = mnext;
    mnext = m;
  }
  // chunk: elimination values come back from X in blocks, loads issued first
  constexpr int BB = 16;
  for (; i - BB + 1 >= ilo; i -= BB) {
    T zb[BB];
#pragma unroll
    for (int u = 0; u < BB; ++u) zb[u] = Xp[xidx<T>(i - u, 8 + s)];
#pragma unroll
    for (int u = 0; u < BB; ++u) {
      const T m = zb[u] - mnext * inv_piv<T>(i - u - wa);
      Xp[xidx<T>(i - u, 8 + s)] = m;
      emit(i - u, m);
      mnext2 = mnext;
      mnext = m;
    }
  }
  for (; i >= ilo; --i) {
    const T m = Xp[xidx<T>(i, 8 + s)] - mnext * inv_piv<T>(i - wa);
    Xp[xidx<T>(i, 8 + s)] = m;
    emit(i, m);
    mnext2 = mnext;
    mnext = m;
  }
  if (inner) emit(c0 - 1, z_below - mnext * inv_piv<T>(c0 - 1 - wa));  // m_{c0-1}: row c0's
  if (wa == c0) Xp[xidx<T>(c0, 8 + s)] = T(0);  // record start: m_0 = 0
}

// ---------------------------------------------------------------------------
// FP32 forward prep by recursive filtering.  The natural-spline moments of a
// record F_0..F_{N-1} solve tridiag(1, 4, 1) m = r on rows 1..N-2 with
// m_0 = m_{N-1} = 0, r_k = 6 (F_{k+1} - 2 F_k + F_{k-1}) / dt^2.  Extending r
// odd-periodically (r_0 = r_{N-1} = 0, r_{-k} = -r_k, period 2 (N - 1)) makes
// the end conditions hold by symmetry, so m is the infinite Toeplitz inverse
// applied to the extended r.  That inverse factors as
//   m = -rho (1 - rho z)^-1 (1 - rho z^-1)^-1 r,   rho = sqrt(3) - 2,
// a causal recursion y_k = r_k + rho y_{k-1} followed by an anti-causal one
// x_k = y_k + rho x_{k+1}, m_k = -rho x_k.  Both recursions start H samples
// outside the 64-sample block they serve (error |rho|^H, below FP32 rounding
// for H = 16), so every block is independent: no sequential sweep over the
// record, no intermediate values in HBM.
//
// Two kernels share the blocks of a record:
//  * k_prep_iir_int, the interior blocks (filter reach inside rows 1..N-2):
//    persistent CTAs walk consecutive blocks of one 16-panel group, with the
//    field rows of the next block in flight (cp.async) while the current one
//    is filtered;
//  * k_prep_iir, the blocks at the record ends (the odd-periodic extension
//    and the one-sided end differences) and the empty blocks past nt.
// The FP32 adjoint k_prep_adj_iir below shares the tile constants.
// ---------------------------------------------------------------------------
constexpr int kIirPanels = 8;
constexpr int kIirChunk = 64;
constexpr int kIirJ = 32;
constexpr int kIirThreads = kIirPanels * 8 * (kIirChunk / kIirJ);
constexpr int kIirH = Prec<float>::halo;
constexpr int kIirRows = kIirChunk + 2 * kIirH + 6;  // bound on the staged rows
constexpr int kIirQ = 8;  // integrand stride in a staged row ([4 integrands][8 panels])
constexpr int kIirRow = 4 * kIirQ;                   // staged row stride (floats)

// ---------------------------------------------------------------------------
// FP32 prep of the interior blocks.  Away from the record ends the moment
// solve and the central time difference are both convolutions, so they
// commute: the moments of a derivative series are the central differences of
// the moments of its value series, m'_k = (m_{k+1} - m_{k-1}) / (2 dt).  Only
// the four value series are filtered, and one thread owns one (panel,
// integrand) over a whole 64-sample block; the four threads of a panel
// assemble each half row of X (the sample pair 2 r, 2 r + 1 of eight slots) and store
// it as four 16-byte pieces.  Blocks whose filter reach touches a record end
// are left to k_prep_iir.
// ---------------------------------------------------------------------------
constexpr int kIntPanels = 16;
constexpr int kIntThreads = kIntPanels * 4;
constexpr int kIntRow = kIntPanels * 4;              // staged row: [panel][integrand]
constexpr int kIntRows = kIirChunk + 2 * kIirH + 4;  // samples c0 - H - 3 .. c0 + 64 + H
constexpr int kIntKeep = kIntRows - kIirChunk;       // rows shared by consecutive blocks
constexpr int kIntUnit = 8;                          // blocks per work unit

__device__ __forceinline__ void cp_async4(float *dst, const float *src, bool ok) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int n = ok ? 4 : 0;  // zero fill
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(n)
               : "memory");
}
__device__ __forceinline__ void cp_async16(float *dst, const float *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

__global__ void __launch_bounds__(kIntThreads, 4) k_prep_iir_int(PrepArgs<float> a) {
  constexpr int NP = kIntPanels, H = kIirH, C = kIirChunk;
  constexpr float rho = -0.267949192431122706f;  // sqrt(3) - 2
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float *sb = reinterpret_cast<float *>(smem_raw);  // [kIntRows][NP][4] integrands
  float *raw = sb + kIntRows * kIntRow;             // [C rows][5][NP] fields in flight
  const int tid = threadIdx.x;
  const int n_pg = (a.P + NP - 1) / NP;
  const int n_blk = a.int_hi - a.int_lo;
  const int n_us = (n_blk + kIntUnit - 1) / kIntUnit;
  const long n_units = (long)n_pg * n_us;
  // phase A thread: panel pa, rows tid / NP + 4 u
  const int pa = tid % NP;
  // phase B thread: integrand qi of panel pl
  const int qi = tid & 3;
  const int pl = tid >> 2;
  const bool q_lo2 = qi < 2, q_is1 = qi == 1, q_is2 = qi == 2;  // lane role in put_row
  const float inv2h = (float)(0.5 / a.dt);
  const float s6 = (float)(6.0 / (a.dt * a.dt));
  const bool vec = a.perm == nullptr && (a.P & 3) == 0 &&
                   ((size_t)a.fields & 15) == 0;  // 16-byte copies of 4 panels
  for (long u = blockIdx.x; u < n_units; u += gridDim.x) {
    // panel group fastest: concurrent units read neighbouring segments of the same rows
    const int p0 = (int)(u % n_pg) * NP;
    const int b0 = a.int_lo + (int)(u / n_pg) * kIntUnit;
    const int b1 = min(a.int_lo + n_blk, b0 + kIntUnit);
    const int p = p0 + pa;
    const bool live = p < a.P;
    float n0 = 0.f, n1 = 0.f, n2 = 0.f, Un = 0.f;
    if (live) {
      n0 = (float)a.n[3 * p];
      n1 = (float)a.n[3 * p + 1];
      n2 = (float)a.n[3 * p + 2];
      Un = (float)(a.ca * a.n[3 * p] + a.sa * a.n[3 * p + 1]);
    }
    const int pb = p0 + pl;
    const bool live_b = pb < a.P;
    // copy field rows [r0, r0 + n) of the group into raw (n <= C)
    auto issue = [&](int r0, int n) {
      if (vec) {
        for (int e = tid; e < n * 5 * (NP / 4); e += kIntThreads) {
          const int q4 = e % (NP / 4), rc = e / (NP / 4);  // rc = row * 5 + component
          const int pq = p0 + 4 * q4;
          if (pq < a.P)
            cp_async16(raw + rc * NP + 4 * q4, a.fields + ((size_t)(r0 * 5) + rc) * a.P + pq);
          else
            *reinterpret_cast<float4 *>(raw + rc * NP + 4 * q4) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      } else {
        const int po = live ? (a.perm ? a.perm[p] : p) : 0;
        for (int rc = tid / NP; rc < n * 5; rc += kIntThreads / NP)
          cp_async4(raw + rc * NP + pa, a.fields + ((size_t)(r0 * 5) + rc) * a.P + po, live);
      }
    };
    // integrands of the n rows in raw into window rows [w0, w0 + n)
    auto integrands = [&](int w0, int n) {
      for (int r = tid / NP; r < n; r += kIntThreads / NP) {
        const float *f = raw + r * 5 * NP + pa;
        const float rho_ = f[0], u0v = f[NP], u1 = f[2 * NP], u2 = f[3 * NP], pp = f[4 * NP];
        const float un = u0v * n0 + u1 * n1 + u2 * n2;
        const float r1 = 1.f + rho_;
        const float utn = Un + un;
        float4 q;
        q.x = rho_ * Un + r1 * un;             // Qn   (Eq. Qn_New_nd)
        q.y = pp * n0 + r1 * u0v * utn;        // L_1  (Eq. Li_New_nd)
        q.z = pp * n1 + r1 * u1 * utn;
        q.w = pp * n2 + r1 * u2 * utn;
        *reinterpret_cast<float4 *>(sb + (size_t)(w0 + r) * kIntRow + pa * 4) = q;
      }
    };
    // window of block b: rows c0 - H - 3 .. c0 + C + H; load its first C rows,
    // then the rest, so that later blocks only add C rows each
    {
      const int lo = b0 * C - H - 3;
      __syncthreads();  // the previous unit is done with raw and sb
      issue(lo, C);
      cp_async_wait_all();
      __syncthreads();
      integrands(0, C);
      __syncthreads();
      issue(lo + C, kIntKeep);
      cp_async_wait_all();
      __syncthreads();
      integrands(C, kIntKeep);
      __syncthreads();
    }
    for (int b = b0; b < b1; ++b) {
      const int c0 = b * C;
      const bool more = b + 1 < b1;
      if (more) issue(c0 + C + H + 1, C);  // rows of the next window, in flight meanwhile
      // ---- phase B: filters of block b ----------------------------------------
      float *xr = a.X + ((size_t)(live_b ? pb : 0) * a.x_ld + c0 % a.x_ld) * kRec;
      // one half row (slots q0 .. q0 + 7 of row r) from the four lanes of a
      // panel: lane qi stores slots q0 + 2 qi, q0 + 2 qi + 1 as one float4 after
      // taking its neighbours' pairs (slot order: d0 v0 d1 d2 | d3 v1 v2 v3)
      auto put_row = [&](int r, int q0, float dl, float dh, float vl, float vh) {
        const float xl = __shfl_down_sync(0xffffffffu, dl, 1);
        const float xh = __shfl_down_sync(0xffffffffu, dh, 1);
        const float yl = __shfl_up_sync(0xffffffffu, vl, 1);
        const float yh = __shfl_up_sync(0xffffffffu, vh, 1);
        const float4 o = make_float4(q_lo2 ? dl : (q_is2 ? xl : yl), q_lo2 ? dh : (q_is2 ? xh : yh),
                                     q_is1 ? xl : (q_is2 ? yl : vl), q_is1 ? xh : (q_is2 ? yh : vh));
        if (live_b) *reinterpret_cast<float4 *>(xr + r * 2 * kRec + (q0 + 2 * qi) * 2) = o;
      };
      const float *bc = sb + (size_t)(H + 3) * kIntRow + pl * 4 + qi;
      auto B = [&](int k) -> float { return bc[k * kIntRow]; };  // k relative to c0
      float y[C + H + 1];
      float yy = 0.f;
      float Bmm = B(-3 - H), Bm = B(-2 - H), B0 = B(-1 - H);
#pragma unroll
      for (int k = -1 - H; k <= C + H - 1; ++k) {
        const float Bp = B(k + 1);
        yy = s6 * (Bp - 2.f * B0 + Bm) + rho * yy;
        if (k >= -1) y[k + 1] = yy;
        if (k >= 1 && k < C && (k & 1)) {  // series of the sample pair (k - 1, k): row (k - 1)/2
          put_row((k - 1) >> 1, 0, (B0 - Bmm) * inv2h, (Bp - Bm) * inv2h, Bm, B0);
        }
        Bmm = Bm;
        Bm = B0;
        B0 = Bp;
      }
      float xx = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f;  // m1, m2, m3: moments at k + 1, k + 2, k + 3
#pragma unroll
      for (int k = C + H - 1; k >= -1; --k) {
        xx = y[k + 1] + rho * xx;
        const float mk = -rho * xx;
        if (k <= C - 3 && (k & 1)) {  // moments of the sample pair (k + 1, k + 2): row (k + 1)/2
          put_row((k + 1) >> 1, 8, (m2 - mk) * inv2h, (m3 - m1) * inv2h, m1, m2);
        }
        m3 = m2;
        m2 = m1;
        m1 = mk;
      }
      if (!more) break;
      // ---- slide the window by C rows and add the rows now in raw --------------
      __syncthreads();  // every thread is done reading the window
      for (int e = tid; e < kIntKeep * kIntRow / 4; e += kIntThreads)
        reinterpret_cast<float4 *>(sb)[e] = reinterpret_cast<const float4 *>(sb + C * kIntRow)[e];
      cp_async_wait_all();
      __syncthreads();
      integrands(kIntKeep, C);
      __syncthreads();
    }
  }
}

// General FP32 prep of a 64-sample block (used for the record ends): thread
// (series, half, panel) filters 32 samples of one of the eight series; the
// two halves of a (panel, series) are lanes 8 apart and store float2 pairs.
__global__ void __launch_bounds__(kIirThreads, 6) k_prep_iir(PrepArgs<float> a) {
  constexpr int NP = kIirPanels, H = kIirH, J = kIirJ;
  constexpr float rho = -0.267949192431122706f;  // sqrt(3) - 2
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // staged integrands, two copies [rows][4 (stride kIirQ)][NP]: the second
  // with its columns rotated by two, read by the threads of the upper half
  // block (rows 32 apart would otherwise share a bank)
  float *sb = reinterpret_cast<float *>(smem_raw);
  float *sb2 = sb + kIirRows * kIirRow;
  const int tid = threadIdx.x;
  // 1D grid over the chunks of [c_lo, c_hi) outside [int_lo, int_hi) (fastest),
  // then panel tiles
  const int na = a.int_lo - a.c_lo, n_edge = na + a.c_hi - a.int_hi;
  const int ei = (int)(blockIdx.x % n_edge);
  const int c0 = (ei < na ? a.c_lo + ei : a.int_hi + ei - na) * kIirChunk;
  const int p0 = (int)(blockIdx.x / n_edge) * NP;
  const int N = a.nt;
  // phase B thread: series s, half h (samples c0 + 32 h ..), panel pl
  const int s = tid & 7;
  const int h = (tid >> 3) & 1;
  const int pl = tid >> 4;
  const int pb = p0 + pl;
  const bool live_b = pb < a.P;
  // X rows of the tile: row r holds the sample pair c0 + 2 r, c0 + 2 r + 1;
  // this thread's samples c0 + 32 h + t fill rows 16 h + t / 2
  float *xr = a.X + ((size_t)(live_b ? pb : 0) * a.x_ld + c0 % a.x_ld + 32 * h) * kRec;
  // slot q of the pair (t0, t0 + 1) (t0 even) as one float2
  auto put2 = [&](int t0, int q, float v0, float v1) {
    if (live_b) *reinterpret_cast<float2 *>(xr + (t0 >> 1) * 2 * kRec + q * 2) = make_float2(v0, v1);
  };
  if (c0 >= N) {
    for (int t = 0; t < J; t += 2) {
      put2(t, s, 0.f, 0.f);
      put2(t, 8 + s, 0.f, 0.f);
    }
    return;
  }
  // staged integrand rows: the tile's filter reach plus FD neighbours, and
  // for a tile at the record end the rows its window folds back onto
  const int reach_lo = c0 - H - 3, reach_hi = c0 + kIirChunk + H + 3;
  const int lo = max(0, min(reach_lo, 2 * (N - 1) - reach_hi));
  const int hi = min(N, reach_hi);
  // ---- phase A: integrands ------------------------------------------------
  {
    const int pl_a = tid % NP;
    const int p = p0 + pl_a;
    const bool live = p < a.P;
    const int po = live ? (a.perm ? a.perm[p] : p) : 0;
    float n0 = 0.f, n1 = 0.f, n2 = 0.f, Un = 0.f;
    if (live) {
      n0 = (float)a.n[3 * p];
      n1 = (float)a.n[3 * p + 1];
      n2 = (float)a.n[3 * p + 2];
      Un = (float)(a.ca * a.n[3 * p] + a.sa * a.n[3 * p + 1]);
    }
    // all field loads of this thread's rows first, then the integrands
    constexpr int RS = kIirThreads / NP;               // row stride between passes
    constexpr int RPT = (kIirRows + RS - 1) / RS;      // passes
    float fv[RPT][5];
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
      const int i = lo + tid / NP + u * RS;
      const bool ok = live && i < hi;
      const float *b = a.fields + (size_t)(ok ? i : 0) * 5 * a.P + po;
#pragma unroll
      for (int c = 0; c < 5; ++c) fv[u][c] = ok ? b[(size_t)c * a.P] : 0.f;
    }
    const int rot = (pl_a + 2) & (NP - 1);
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
      const int i = lo + tid / NP + u * RS;
      if (i >= hi) break;
      const float rho_ = fv[u][0], u0 = fv[u][1], u1 = fv[u][2], u2 = fv[u][3], pp = fv[u][4];
      const float un = u0 * n0 + u1 * n1 + u2 * n2;
      const float r1 = 1.f + rho_;
      const float utn = Un + un;
      const float q0 = rho_ * Un + r1 * un;            // Qn   (Eq. Qn_New_nd)
      const float q1 = pp * n0 + r1 * u0 * utn;        // L_1  (Eq. Li_New_nd)
      const float q2 = pp * n1 + r1 * u1 * utn;
      const float q3 = pp * n2 + r1 * u2 * utn;
      float *row = sb + (size_t)(i - lo) * kIirRow;
      float *row2 = sb2 + (size_t)(i - lo) * kIirRow;
      row[pl_a] = q0;
      row[kIirQ + pl_a] = q1;
      row[2 * kIirQ + pl_a] = q2;
      row[3 * kIirQ + pl_a] = q3;
      row2[rot] = q0;
      row2[kIirQ + rot] = q1;
      row2[2 * kIirQ + rot] = q2;
      row2[3 * kIirQ + rot] = q3;
    }
  }
  __syncthreads();
  // ---- phase B: series and moments, stored straight to X ---------------------
  const int ks = c0 + J * h;
  const bool deriv = (s == 0) || (s >= 2 && s <= 4);
  const int qi = (s <= 1) ? 0 : 1 + (s - 2) % 3;
  const float *col = (h ? sb2 + ((pl + 2) & (NP - 1)) : sb + pl) + qi * kIirQ -
                     (size_t)lo * kIirRow;  // B(i) = col[i * kIirRow]
  const float inv2h = (float)(0.5 / a.dt);
  const float s6 = (float)(6.0 / (a.dt * a.dt));
  auto B = [&](int i) -> float { return col[(size_t)i * kIirRow]; };
  // (each path is taken by the whole CTA, so that the pair exchange in put2
  // runs on full warps)
  // Records of 82 frames or more: every index the filters reach folds back
  // into the record with one reflection, and the odd-periodic extension of r
  // is the second difference of the series point-reflected about its end
  // values, F(-k) = 2 F(0) - F(k), F(N - 1 + k) = 2 F(N - 1) - F(N - 1 - k)
  // (r then also vanishes at both ends).  So the filters run on that
  // extension with the same unrolled recursion as the interior.
  if (N >= 82) {
    float Fs = 0.f, Fe = 0.f;  // series at the first and last frame (one-sided derivatives)
    if (lo == 0) Fs = deriv ? (-3.f * B(0) + 4.f * B(1) - B(2)) * inv2h : B(0);
    if (hi == N) Fe = deriv ? (3.f * B(N - 1) - 4.f * B(N - 2) + B(N - 3)) * inv2h : B(N - 1);
    auto Fx = [&](int kk) -> float {
      const bool neg = kk < 0, big = kk > N - 1;
      const int m = neg ? -kk : (big ? 2 * (N - 1) - kk : kk);
      float v;
      if (deriv) {
        const float c = (B(min(m + 1, N - 1)) - B(max(m - 1, 0))) * inv2h;
        v = m == 0 ? Fs : (m == N - 1 ? Fe : c);
      } else {
        v = B(m);
      }
      return neg ? 2.f * Fs - v : (big ? 2.f * Fe - v : v);
    };
    float y[J + H];
    int k = ks - H;
    float Fm = Fx(k - 1), F0 = Fx(k);
    float yy = 0.f, held = 0.f;
#pragma unroll
    for (int t = 0; t < J + 2 * H; ++t, ++k) {
      const float Fp = Fx(k + 1);
      yy = s6 * (Fp - 2.f * F0 + Fm) + rho * yy;
      if (t >= H) y[t - H] = yy;
      if (t >= H && t < H + J) {
        const float v = k < N ? F0 : 0.f;
        if (((t - H) & 1) == 0)
          held = v;
        else
          put2(t - H - 1, s, held, v);
      }
      Fm = F0;
      F0 = Fp;
    }
    float xx = 0.f;
#pragma unroll
    for (int t = J + H - 1; t >= 0; --t) {
      xx = y[t] + rho * xx;
      if (t < J) {
        const float v = ks + t < N ? -rho * xx : 0.f;
        if (t & 1)
          held = v;
        else
          put2(t, 8 + s, v, held);
      }
    }
  } else {
    // short records (compact code): one-sided derivatives at the first and
    // last frame, r on the odd-periodic extension of any number of periods
    auto F = [&](int i) -> float {
      if (!deriv) return B(i);
      if (i == 0) return (-3.f * B(0) + 4.f * B(1) - B(2)) * inv2h;
      if (i == N - 1) return (3.f * B(N - 1) - 4.f * B(N - 2) + B(N - 3)) * inv2h;
      return (B(i + 1) - B(i - 1)) * inv2h;
    };
    const int L2 = 2 * (N - 1);
    auto r_at = [&](int kk) -> float {
      int km = kk % L2;
      if (km < 0) km += L2;
      float sg = 1.f;
      if (km >= N - 1) {
        km = L2 - km;
        sg = -1.f;
      }
      if (km == 0 || km == N - 1) return 0.f;
      return sg * s6 * (F(km + 1) - 2.f * F(km) + F(km - 1));
    };
    float ye[J + H];
    float yy = 0.f;
#pragma unroll 1
    for (int t = 0; t < J + 2 * H; ++t) {
      yy = r_at(ks - H + t) + rho * yy;
      if (t >= H) ye[t - H] = yy;
    }
#pragma unroll 1
    for (int t = 0; t < J; t += 2)
      put2(t, s, ks + t < N ? F(ks + t) : 0.f, ks + t + 1 < N ? F(ks + t + 1) : 0.f);
    float xx = 0.f, held = 0.f;
#pragma unroll 1
    for (int t = J + H - 1; t >= 0; --t) {
      xx = ye[t] + rho * xx;
      if (t < J) {
        const float v = ks + t < N ? -rho * xx : 0.f;
        if (t & 1)
          held = v;
        else
          put2(t, 8 + s, v, held);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Adjoint of k_prep followed by the Jacobian of the integrands.
// Xbar[p][i][s] = dLoss/dF_s(i), Xbar[p][i][8+s] = dLoss/dm_s(i).  For each
// series: G_s = Xbar_s + (6/dt^2) D2^T T^{-1} mbar (transpose of the moment
// solve; the interior matrix is symmetric), then the integrand gradient is
// G_s (value series) or D1^T G_s (derivative series), summed per integrand
// over the 8 threads of a panel, and mapped to the five field gradients.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) k_prep_adj(PrepAdjArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *zb = reinterpret_cast<T *>(smem_raw);
  const int tid = threadIdx.x;
  const int s = tid & 7;
  const int n_pt = (a.P + kPanelsPerCta - 1) / kPanelsPerCta;  // 1D grid, panel tile fastest
  const int p = (int)(blockIdx.x % n_pt) * kPanelsPerCta + (tid >> 3);
  const bool live = p < a.P;
  const int c0 = (int)(blockIdx.x / n_pt) * a.chunk;
  const int nt = a.nt;
  const int ce = min(c0 + a.chunk, nt);
  if (c0 >= nt) return;  // uniform across the CTA
  const int pp = live ? p : a.P - 1;
  const T *Xb = a.Xbar + (size_t)pp * a.ntp * kRec;
  const bool deriv = (s == 0) || (s >= 2 && s <= 4);
  const T inv2h = (T)(0.5 / a.dt);
  const T s6 = (T)(6.0 / (a.dt * a.dt));
  constexpr int H = Prec<T>::halo;
  // z = T^{-1} mbar is needed on [e0, e1) = [c0 - 3, ce + 3) for G on
  // [c0 - 2, ce + 2) and D1^T on [c0, ce).
  const int e0 = max(0, c0 - 3), e1 = min(nt, ce + 3);
  const int wa = max(0, e0 - H), wb = min(nt, e1 + H);
  const int L = wb - wa;
  // forward elimination; z kept from e0 to the right end of the window
  T z = T(0);
  for (int i = wa + 1; i <= wb - 2; ++i) {
    const int j = i - wa;
    const T mb = Xb[(size_t)i * kRec + 8 + s];
    z = (mb - z) * inv_piv<T>(j);
    if (i >= e0) zb[(size_t)(i - e0) * kThreads + tid] = z;
  }
  // back substitution (window ends and record ends hold z = 0)
  T znext = T(0);
  for (int i = wb - 1; i >= e0; --i) {
    const int j = i - wa;
    T zz;
    if (j == 0 || j == L - 1) {
      zz = T(0);
    } else {
      zz = zb[(size_t)(i - e0) * kThreads + tid] - znext * inv_piv<T>(j);
    }
    zb[(size_t)(i - e0) * kThreads + tid] = zz;
    znext = zz;
  }
  __syncwarp();
  auto zat = [&](int i) -> T {
    if (i < e0 || i >= e1 || i <= 0 || i >= nt - 1) return T(0);
    return zb[(size_t)(i - e0) * kThreads + tid];
  };
  auto Gat = [&](int i) -> T {
    return Xb[(size_t)i * kRec + s] + s6 * (zat(i - 1) - T(2) * zat(i) + zat(i + 1));
  };
  // field gradients for this chunk
  const int po = live ? (a.perm ? a.perm[p] : p) : 0;
  const T n0 = (T)a.n[3 * pp], n1 = (T)a.n[3 * pp + 1], n2 = (T)a.n[3 * pp + 2];
  const T Un = (T)(a.ca * a.n[3 * pp] + a.sa * a.n[3 * pp + 1]);
  for (int i = c0; i < ce; ++i) {
    T c;
    if (!deriv) {
      c = Gat(i);
    } else {
      // transpose of the FD derivative at integrand sample i
      c = T(0);
      if (i - 1 >= 1 && i - 1 <= nt - 2) c += Gat(i - 1) * inv2h;
      if (i + 1 >= 1 && i + 1 <= nt - 2) c -= Gat(i + 1) * inv2h;
      if (i <= 2) {
        const T w0 = (i == 0) ? T(-3) : (i == 1 ? T(4) : T(-1));
        c += w0 * inv2h * Gat(0);
      }
      if (i >= nt - 3) {
        const T w1 = (i == nt - 1) ? T(3) : (i == nt - 2 ? T(-4) : T(1));
        c += w1 * inv2h * Gat(nt - 1);
      }
    }
    // integrand gradients: Qn from series 0,1; L_c from series 2+c and 5+c
    const int base = (tid & 31) & ~7;
    T v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = __shfl_sync(0xffffffffu, c, base + k);
    const T qb = v[0] + v[1];
    const T lb0 = v[2] + v[5], lb1 = v[3] + v[6], lb2 = v[4] + v[7];
    if (live && s < 5) {
      const T *fb = a.fields + (size_t)i * 5 * a.P + po;
      const T rho = fb[0], u0 = fb[(size_t)a.P], u1 = fb[2 * (size_t)a.P],
              u2 = fb[3 * (size_t)a.P];
      const T un = u0 * n0 + u1 * n1 + u2 * n2;
      const T utn = Un + un;  // total u . n
      const T r1 = T(1) + rho;
      const T lu = lb0 * u0 + lb1 * u1 + lb2 * u2;
      T out;
      if (s == 0) {
        // dQn/drho' = U.n + u'.n ; dL_c/drho' = u'_c (U.n + u'.n)
        out = qb * utn + lu * utn;
      } else if (s <= 3) {
        // dQn/du'_k = (1 + rho') n_k ; dL_c/du'_k = (1 + rho')(delta_ck u.n + u'_c n_k)
        const T nk = s == 1 ? n0 : (s == 2 ? n1 : n2);
        const T lk = s == 1 ? lb0 : (s == 2 ? lb1 : lb2);
        out = qb * r1 * nk + lk * r1 * utn + r1 * lu * nk;
      } else {
        out = lb0 * n0 + lb1 * n1 + lb2 * n2;  // dL_c/dp' = n_c
      }
      a.grad_fields[((size_t)i * 5 + s) * a.P + po] = out;
    }
  }
}

// ---------------------------------------------------------------------------
// FP32 adjoint of k_prep_iir followed by the integrand Jacobian.  With
// m = A r, r = (6/dt^2) D2 F on the interior rows and A the symmetric inverse
// of tridiag(1, 4, 1) with natural ends, the gradient of series s is
//   G_s = Xbar_s + (6/dt^2) D2^T A mbar_s,
// where A mbar_s is computed by the same pair of recursive filters on the
// odd-periodic extension of mbar_s (zero at 0 and N-1).  The integrand
// gradient is G_s (value series) or D1^T G_s (derivative series), summed per
// integrand over the series that share it, then mapped to the five field
// gradients.  Tile: 8 panels x 64 samples; thread (half, panel, series)
// filters samples [32 half - 3, 32 half + 35) of the tile; the per-sample
// integrand gradients meet in shared memory and are written per (sample,
// panel) with coalesced stores.
//
// Every CTA first stages in shared memory (cp.async) the moment slots of
// its Xbar rows c0 - 3 - H .. c0 + 64 + H + 2 (the filters' reach) and, at
// the record ends, the value slots of rows c0 - 2 .. c0 + 65.  Per panel the
// rows are 8 floats, the panel stride padded to 8 or 24 mod 32 words so that
// the 4 panels x 8 series one warp reads in a step sit on 32 distinct banks.
// At the record ends the staged moments are the odd-periodic extension
// itself (rows mapped by reflection, zero at 0 and N - 1, negated where
// reflected) and the staged values are zero outside the record, so every
// thread runs the same unrolled filter.  The per-sample integrand gradients
// reuse the staging space once every thread has filtered.
// ---------------------------------------------------------------------------
constexpr int kAdjZ = kIirJ + 6;             // moments-adjoint values a thread keeps
constexpr int kAdjMRows = kIirRows;          // c0 - 3 - H .. c0 + C + H + 2
constexpr int kAdjVRows = kIirChunk + 4;     // c0 - 2 .. c0 + C + 1
constexpr int kAdjMPS = kAdjMRows * 8 + 8;   // panel strides (floats)
constexpr int kAdjVPS = kAdjVRows * 8 + 8;
static_assert((kAdjMPS % 32 == 8 || kAdjMPS % 32 == 24) &&
                  (kAdjVPS % 32 == 8 || kAdjVPS % 32 == 24),
              "bank spread of the staged rows");
static_assert(kIirPanels * kAdjMPS >= kIirChunk * 8 * kIirPanels, "gradients fit the staging");

__device__ __forceinline__ void cp_async16_zfill(float *dst, const float *src, bool ok) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int n = ok ? 16 : 0;  // zero fill
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(n)
               : "memory");
}

// Interior thread: o[t] is the contribution of sample ks + t, from its kAdjZ
// values z (index 0 is sample ks - 3) and the value slot s of Xbar (global).
__device__ __forceinline__ void adj_values(const float (&z)[kAdjZ], const float *Xb, int s,
                                           bool deriv, int ks, float s6, float inv2h,
                                           float (&o)[kIirJ]) {
  constexpr int J = kIirJ;
  float G[J + 4];  // samples ks - 2 .. ks + J + 1
#pragma unroll
  for (int t = 0; t < J + 4; ++t)
    G[t] = Xb[(size_t)(ks - 2 + t) * kRec + s] + s6 * (z[t] - 2.f * z[t + 1] + z[t + 2]);
#pragma unroll
  for (int t = 0; t < J; ++t) o[t] = deriv ? (G[t + 1] - G[t + 3]) * inv2h : G[t + 2];
}

// Record-end thread: the same with the natural ends (no moment at 0 and
// N - 1), D1^T's one-sided end rows, and zero past N - 1.  xv[8 t] is the
// value slot of sample ks - 2 + t (zero outside the record).  ks is a
// multiple of 32, so the start end can only enter as sample 0 = ks; the far
// end's G is picked out of the unrolled G by a select.
__device__ __forceinline__ void adj_values_ends(float (&z)[kAdjZ], const float *xv, bool deriv,
                                                int ks, int N, float s6, float inv2h,
                                                float (&o)[kIirJ]) {
  constexpr int J = kIirJ;
#pragma unroll
  for (int t = 0; t < kAdjZ; ++t) {
    const int i = ks - 3 + t;
    if (i <= 0 || i >= N - 1) z[t] = 0.f;
  }
  float G[J + 4];  // samples ks - 2 .. ks + J + 1
#pragma unroll
  for (int t = 0; t < J + 4; ++t) G[t] = xv[8 * t] + s6 * (z[t] - 2.f * z[t + 1] + z[t + 2]);
  float gN = 0.f;  // G at sample N - 1, when it lies in the thread's range
#pragma unroll
  for (int t = 0; t < J + 4; ++t)
    if (ks - 2 + t == N - 1) gN = G[t];
#pragma unroll
  for (int t = 0; t < J; ++t) {
    const int i = ks + t;
    float c;
    if (!deriv) {
      c = G[t + 2];
    } else {
      c = 0.f;
      if (i - 1 >= 1 && i - 1 <= N - 2) c += G[t + 1] * inv2h;
      if (i + 1 >= 1 && i + 1 <= N - 2) c -= G[t + 3] * inv2h;
      if (i <= 2) c += (i == 0 ? -3.f : (i == 1 ? 4.f : -1.f)) * inv2h * G[2];  // here ks = 0
      if (i >= N - 3) c += (i == N - 1 ? 3.f : (i == N - 2 ? -4.f : 1.f)) * inv2h * gN;
    }
    o[t] = i < N ? c : 0.f;
  }
}

// Blocks [int_lo, int_hi) of each panel tile keep every thread's reach
// inside rows 1 .. N - 2 (ENDS = false); ENDS = true runs the other blocks.
// 1D grid, block fastest.
template <bool ENDS>
__global__ void __launch_bounds__(kIirThreads, ENDS ? 5 : 7) k_prep_adj_iir(PrepAdjArgs<float> a, int int_lo,
                                                              int int_hi) {
  constexpr int NP = kIirPanels, H = kIirH, J = kIirJ;
  constexpr int NR = kAdjZ + 2 * H;  // samples each thread filters
  constexpr float rho = -0.267949192431122706f;  // sqrt(3) - 2
  // staged moments [NP][kAdjMPS] (later the gradients [sample][panel][series]),
  // then, at the record ends, staged values [NP][kAdjVPS]
  __shared__ __align__(16) float sm[NP * kAdjMPS + (ENDS ? NP * kAdjVPS : 0)];
  float *cs = sm;
  const int tid = threadIdx.x;
  const int n_ct = (a.nt + kIirChunk - 1) / kIirChunk;
  const int n_mid = int_hi - int_lo;
  const int n_sel = ENDS ? n_ct - n_mid : n_mid;
  const int e = (int)(blockIdx.x % n_sel);
  const int c0 = (ENDS ? (e < int_lo ? e : e + n_mid) : int_lo + e) * kIirChunk;
  const int p0 = (int)(blockIdx.x / n_sel) * NP;
  const int N = a.nt;
  if (c0 >= N) return;  // uniform across the CTA
  const int L2 = 2 * (N - 1);
  // sample k of the odd-periodic extension as a row of the record: km in
  // [0, N - 1], reflected when the extension's sign is negative
  auto ext_row = [&](int k, bool &reflected) -> int {
    int km = k % L2;
    if (km < 0) km += L2;
    reflected = km > N - 1;
    return reflected ? L2 - km : km;
  };
  if (ENDS) {
    for (int e2 = tid; e2 < NP * 2 * kAdjMRows; e2 += kIirThreads) {
      const int pl = e2 / (2 * kAdjMRows), rq = e2 - pl * (2 * kAdjMRows);
      const float *xp = a.Xbar + (size_t)min(p0 + pl, a.P - 1) * a.ntp * kRec + 8 + 4 * (rq & 1);
      bool refl;
      const int km = ext_row(c0 - 3 - H + (rq >> 1), refl);
      cp_async16_zfill(sm + pl * kAdjMPS + 4 * rq, xp + (size_t)km * kRec, km != 0 && km != N - 1);
    }
  } else {
    // piece rq (row rq / 2, half rq % 2) of every panel: rq = tid and tid + 128
    static_assert(2 * kAdjMRows <= 2 * kIirThreads, "two pieces per thread and panel");
    const int rq1 = tid + kIirThreads;
    const bool two = rq1 < 2 * kAdjMRows;
    const size_t o0 = (size_t)(c0 - 3 - H) * kRec + 8 + (tid >> 1) * kRec + 4 * (tid & 1);
    const size_t o1 = (size_t)(c0 - 3 - H) * kRec + 8 + (rq1 >> 1) * kRec + 4 * (rq1 & 1);
#pragma unroll 1
    for (int pl = 0; pl < NP; ++pl) {
      const float *xp = a.Xbar + (size_t)min(p0 + pl, a.P - 1) * a.ntp * kRec;
      cp_async16(sm + pl * kAdjMPS + 4 * tid, xp + o0);
      if (two) cp_async16(sm + pl * kAdjMPS + 4 * rq1, xp + o1);
    }
  }
  if (ENDS) {
    float *sv = sm + NP * kAdjMPS;
    for (int e2 = tid; e2 < NP * 2 * kAdjVRows; e2 += kIirThreads) {
      const int pl = e2 / (2 * kAdjVRows), rq = e2 - pl * (2 * kAdjVRows);
      const int i = c0 - 2 + (rq >> 1);
      const bool in = i >= 0 && i < N;
      const float *xp = a.Xbar + (size_t)min(p0 + pl, a.P - 1) * a.ntp * kRec + 4 * (rq & 1);
      cp_async16_zfill(sv + pl * kAdjVPS + 4 * rq, xp + (size_t)(in ? i : 0) * kRec, in);
    }
  }
  cp_async_wait_all();
  __syncthreads();
  if (ENDS) {  // negate the reflected rows
    for (int e3 = tid; e3 < NP * kAdjMRows; e3 += kIirThreads) {
      const int pl = e3 / kAdjMRows, r = e3 - pl * kAdjMRows;
      bool refl;
      ext_row(c0 - 3 - H + r, refl);
      if (refl) {
        float4 *q = reinterpret_cast<float4 *>(sm + pl * kAdjMPS + 8 * r);
        const float4 u = q[0], w = q[1];
        q[0] = make_float4(-u.x, -u.y, -u.z, -u.w);
        q[1] = make_float4(-w.x, -w.y, -w.z, -w.w);
      }
    }
    __syncthreads();
  }
  {
    const int s = tid & 7;
    const int pl = (tid >> 3) % NP;
    const int h = tid / (8 * NP);
    const int ks = c0 + J * h;
    const bool deriv = (s == 0) || (s >= 2 && s <= 4);
    const float inv2h = (float)(0.5 / a.dt);
    const float s6 = (float)(6.0 / (a.dt * a.dt));
    // moment slot s of sample ks - 3 - H + t: staged row ks - c0 + t
    const float *xm = sm + pl * kAdjMPS + (ks - c0) * 8 + s;
    float y[kAdjZ + H];
    float yy = 0.f;
#pragma unroll
    for (int t = 0; t < NR; ++t) {
      yy = xm[8 * t] + rho * yy;
      if (t >= H) y[t - H] = yy;
    }
    float xx = 0.f;
    float z[kAdjZ];
#pragma unroll
    for (int t = kAdjZ + H - 1; t >= 0; --t) {
      xx = y[t] + rho * xx;
      if (t < kAdjZ) z[t] = -rho * xx;
    }
    float o[J];
    if (ENDS) {
      // value slot s of sample ks - 2 + t: staged row ks - c0 + t
      adj_values_ends(z, sm + NP * kAdjMPS + pl * kAdjVPS + (ks - c0) * 8 + s, deriv, ks, N, s6,
                      inv2h, o);
    } else {
      adj_values(z, a.Xbar + (size_t)min(p0 + pl, a.P - 1) * a.ntp * kRec, s, deriv, ks, s6,
                 inv2h, o);
    }
    __syncthreads();  // every thread is done with the staged moments
    // [sample][panel][series]: the warp's 4 panels x 8 series on 32 banks
    float *out = cs + (size_t)(ks - c0) * 8 * NP + pl * 8 + s;
#pragma unroll
    for (int t = 0; t < J; ++t) out[t * 8 * NP] = o[t];
  }
  __syncthreads();
  // ---- integrand gradients -> field gradients, per (sample, panel) ----------
  // thread: panel tid % NP, samples tid / NP + 16 it; the field loads of all
  // its samples are issued before any of them is used
  {
    constexpr int IT = kIirChunk * NP / kIirThreads;
    constexpr int RS = kIirThreads / NP;  // sample stride
    const int pl = tid % NP, p = p0 + pl;
    if (p < a.P) {
      const int po = a.perm ? a.perm[p] : p;
      const float n0 = (float)a.n[3 * p], n1 = (float)a.n[3 * p + 1], n2 = (float)a.n[3 * p + 2];
      const float Un = (float)(a.ca * a.n[3 * p] + a.sa * a.n[3 * p + 1]);
      float f[IT][4];
#pragma unroll
      for (int it = 0; it < IT; ++it) {
        const int i = c0 + tid / NP + RS * it;
        const float *fb = a.fields + (size_t)min(i, N - 1) * 5 * a.P + po;
#pragma unroll
        for (int q = 0; q < 4; ++q) f[it][q] = fb[(size_t)q * a.P];
      }
#pragma unroll
      for (int it = 0; it < IT; ++it) {
        const int ir = tid / NP + RS * it;
        const int i = c0 + ir;
        if (i >= N) continue;
        const float4 c03 = *reinterpret_cast<const float4 *>(cs + (size_t)ir * 8 * NP + pl * 8);
        const float4 c47 = *reinterpret_cast<const float4 *>(cs + (size_t)ir * 8 * NP + pl * 8 + 4);
        const float qb = c03.x + c03.y;                      // Qn: series 0 and 1
        const float lb0 = c03.z + c47.y;                     // L_c: series 2 + c and 5 + c
        const float lb1 = c03.w + c47.z;
        const float lb2 = c47.x + c47.w;
        const float rho_ = f[it][0], u0 = f[it][1], u1 = f[it][2], u2 = f[it][3];
        const float un = u0 * n0 + u1 * n1 + u2 * n2;
        const float utn = Un + un;   // total u . n
        const float r1 = 1.f + rho_;
        const float lu = lb0 * u0 + lb1 * u1 + lb2 * u2;
        float *g = a.grad_fields + (size_t)i * 5 * a.P + po;
        g[0] = qb * utn + lu * utn;                               // d/drho'
        g[(size_t)a.P] = r1 * (qb * n0 + lb0 * utn + lu * n0);   // d/du'_1
        g[2 * (size_t)a.P] = r1 * (qb * n1 + lb1 * utn + lu * n1);
        g[3 * (size_t)a.P] = r1 * (qb * n2 + lb2 * utn + lu * n2);
        g[4 * (size_t)a.P] = lb0 * n0 + lb1 * n1 + lb2 * n2;     // d/dp' (dL_c/dp' = n_c)
      }
    }
  }
}

}  // namespace

template <typename T>
cudaError_t launch_prep(const PrepArgs<T> &a0, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (a0.ntp % kIirChunk != 0) return cudaErrorInvalidValue;
    PrepArgs<float> a = a0;
    if (a.c_hi == 0) {
      a.c_lo = 0;
      a.c_hi = a.ntp / kIirChunk;
    }
    if (a.c_lo < 0 || a.c_hi > a.ntp / kIirChunk || a.c_lo >= a.c_hi) return cudaErrorInvalidValue;
    // interior blocks: filter reach inside rows 1 .. N - 2 (c0 >= H + 2 and
    // c0 + C + H + 1 <= N), by the persistent kernel
    const int last_int = a.nt >= kIirChunk + kIirH + 1 ? (a.nt - kIirChunk - kIirH - 1) / kIirChunk : -1;
    a.int_lo = std::max(a.c_lo, (kIirH + 2 + kIirChunk - 1) / kIirChunk);
    a.int_hi = std::min(a.c_hi, last_int + 1);
    if (a.int_lo >= a.int_hi) a.int_lo = a.int_hi = a.c_hi;
    cudaError_t e;
    if (a.int_hi > a.int_lo) {
      const size_t smem_i = ((size_t)kIntRows * kIntRow + (size_t)kIirChunk * 5 * kIntPanels) *
                            sizeof(float);
      e = cudaFuncSetAttribute(k_prep_iir_int, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem_i);
      if (e != cudaSuccess) return e;
      int dev = 0, sms = 0, per_sm = 0;
      if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
      if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
      if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_prep_iir_int, kIntThreads,
                                                             smem_i)) != cudaSuccess)
        return e;
      const long units = (long)((a.P + kIntPanels - 1) / kIntPanels) *
                         ((a.int_hi - a.int_lo + kIntUnit - 1) / kIntUnit);
      const long grid = std::min<long>(units, (long)std::max(per_sm, 1) * sms);
      k_prep_iir_int<<<(unsigned)grid, kIntThreads, smem_i, s>>>(a);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // record-end and empty blocks by the general kernel
    const int n_edge = (a.int_lo - a.c_lo) + (a.c_hi - a.int_hi);
    if (n_edge == 0) return cudaSuccess;
    const size_t smem = (size_t)2 * kIirRows * kIirRow * sizeof(float);
    e = cudaFuncSetAttribute(k_prep_iir, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long eblocks = (long)n_edge * ((a.P + kIirPanels - 1) / kIirPanels);
    if (eblocks > INT32_MAX) return cudaErrorInvalidValue;
    k_prep_iir<<<(unsigned)eblocks, kIirThreads, smem, s>>>(a);
    return cudaGetLastError();
  } else {
    constexpr int NP = PrepTile<T>::panels;
    constexpr int H = Prec<T>::halo;
    PrepArgs<T> a = a0;
    a.chunk = PrepTile<T>::chunk;
    static_assert(PrepTile<T>::chunk == kIirChunk, "chunk ranges count 64-sample chunks");
    if (a.c_hi == 0) {
      a.c_lo = 0;
      a.c_hi = (a.ntp + a.chunk - 1) / a.chunk;
    }
    if (a.c_lo < 0 || a.c_hi > (a.ntp + a.chunk - 1) / a.chunk || a.c_lo >= a.c_hi)
      return cudaErrorInvalidValue;
    // integrand rows (chunk + 2 halos + 2 FD neighbours) x 4 x NP, plus the
    // right-halo elimination values H x (NP * 8)
    const size_t smem =
        ((size_t)(a.chunk + 2 * H + 2) * 4 * NP + (size_t)H * NP * 8) * sizeof(T);
    cudaError_t e = cudaFuncSetAttribute(k_prep<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const long blocks = (long)((a.P + NP - 1) / NP) * (a.c_hi - a.c_lo);
    if (blocks <= 0) return cudaSuccess;
    if (blocks > INT32_MAX) return cudaErrorInvalidValue;
    k_prep<T><<<(unsigned)blocks, NP * 8, smem, s>>>(a);
    return cudaGetLastError();
  }
}

template <typename T>
cudaError_t launch_prep_adjoint(const PrepAdjArgs<T> &a0, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    const int n_ct = (a0.nt + kIirChunk - 1) / kIirChunk;
    const long tiles = (a0.P + kIirPanels - 1) / kIirPanels;
    if (n_ct <= 0 || tiles <= 0) return cudaSuccess;
    // interior blocks: c0 - 3 - H >= 1 and c0 + C + H + 3 <= N - 1
    int int_lo = (kIirH + 4 + kIirChunk - 1) / kIirChunk;
    const int top = a0.nt - 4 - kIirChunk - kIirH;  // largest interior c0
    int int_hi = top >= 0 ? top / kIirChunk + 1 : 0;
    if (int_hi <= int_lo) int_lo = int_hi = 0;
    const long mid = (long)(int_hi - int_lo) * tiles;
    const long ends = (long)(n_ct - (int_hi - int_lo)) * tiles;
    if (mid > INT32_MAX || ends > INT32_MAX) return cudaErrorInvalidValue;
    if (mid > 0) {
      k_prep_adj_iir<false><<<(unsigned)mid, kIirThreads, 0, s>>>(a0, int_lo, int_hi);
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    if (ends > 0) k_prep_adj_iir<true><<<(unsigned)ends, kIirThreads, 0, s>>>(a0, int_lo, int_hi);
    return cudaGetLastError();
  }
  PrepAdjArgs<T> a = a0;
  a.chunk = PrepChunk<T>::v;
  const size_t smem = (size_t)(a.chunk + 6 + Prec<T>::halo) * kThreads * sizeof(T);
  cudaError_t e = cudaFuncSetAttribute(k_prep_adj<T>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long blocks =
      (long)((a.P + kPanelsPerCta - 1) / kPanelsPerCta) * ((a.nt + a.chunk - 1) / a.chunk);
  if (blocks <= 0) return cudaSuccess;
  if (blocks > INT32_MAX) return cudaErrorInvalidValue;
  k_prep_adj<T><<<(unsigned)blocks, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template cudaError_t launch_prep<float>(const PrepArgs<float> &, cudaStream_t);
template cudaError_t launch_prep<double>(const PrepArgs<double> &, cudaStream_t);
template cudaError_t launch_prep_adjoint<float>(const PrepAdjArgs<float> &, cudaStream_t);
template cudaError_t launch_prep_adjoint<double>(const PrepAdjArgs<double> &, cudaStream_t);

}  // namespace fwh
