/*
 * FP64 CPU oracle for the permeable-surface, nondimensional, wind-tunnel FW-H
 * integral (OpenCFD-FWH, arXiv 2312.16263).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
 * includes this file; only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg load it.  It shares no code with the CUDA path.
 *
 * The oracle follows the paper's own order of work (Sec. III B, the
 * "compute R" / "compute Noise" / "compute t" / "interp pressure signal"
 * stages, then the surface sum of Sec. III C), one observer at a time:
 *
 *   1. R, R* and the unit radiation vector by the rotated Garrick-triangle
 *      route: d' (Eqs. d1_prime, d2_prime), R and R* (Eqs. R_New, R_s_New),
 *      R-hat' (Eqs. R1_prime, R2_prime, R3_New) and the rotation back
 *      (Eqs. R1_New, R2_New).
 *   2. For every frame, totals rho = 1 + rho', u = U0-hat + u', and the
 *      literal integrands Q_n = (-U0 + rho u).n and
 *      L_i = p' n_i + rho (u_i - U0_i)(u.n)  (Eqs. Qn_New_nd, Li_New_nd).
 *      Source-time derivatives by second-order finite differences: central
 *      inside, one-sided at the first and last frame (Sec. III B).
 *   3. The source-time pressure of each subface, term by term, from
 *      Eqs. pT_WT_nd and pL_WT_nd, times dS / (4 pi).
 *   4. The observer window t_start = M0 R_max, t_end = tau_max + M0 R_min
 *      (Eqs. t_start, t_end) and a natural cubic spline of each subface's
 *      signal over source time, evaluated at tau = t_j - M0 R.
 *   5. The sum over subfaces (Sec. III C), plain or Neumaier-compensated.
 *
 * Readings where the paper is silent (each listed in the design notes):
 *   - the surface Mach vector in the fluid-at-rest frame is M = -M0 U0-hat,
 *     so M^2 = M0^2 (Sec. II C: the surface moves at -U0);
 *   - inputs are pulsations; totals are rebuilt as 1 + rho', U0-hat + u';
 *   - L-dot is taken per component (L-dot_R = L-dot . R-hat, R-hat fixed);
 *   - tau_0 = 0, tau_max = (nt-1) dt, observer spacing dt,
 *     N_o = floor((t_end - t_start)/dt) + 1, bins j >= N_o are zero;
 *   - the spline is the natural one (zero second derivative at both ends).
 *
 * The adjoint routines are the exact transpose of steps 2-5 (linear in the
 * integrands once geometry is fixed) plus the Jacobian of step 2.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define FWHO_OK 0
#define FWHO_ERR_ARG 1
#define FWHO_ERR_OOM 3

static const double FWHO_PI = 3.14159265358979323846264338327950288;

/* ------------------------------------------------------------------------ */
/* Step 1: convected distance by the paper's rotated route.                  */
/* ------------------------------------------------------------------------ */

/* d = x - y (observer minus source).  Returns R, R* and R-hat (unit). */
static void convected_distance(const double d[3], double mach, double aoa,
                               double *R, double *Rs, double Rhat[3]) {
  const double ca = cos(aoa), sa = sin(aoa);
  const double M1 = mach * ca, M2 = mach * sa;           /* Eqs. M1, M2 */
  const double beta2 = 1.0 - mach * mach;                /* Eq. beta */
  /* Eqs. d1_prime, d2_prime: rotate d into the flow-aligned frame. */
  const double d1p = d[0] * ca + d[1] * sa;
  const double d2p = -d[0] * sa + d[1] * ca;
  const double dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  const double md = M1 * d[0] + M2 * d[1];
  const double rs = sqrt(md * md + beta2 * dd);          /* Eq. R_s_New */
  const double r = (-md + rs) / beta2;                   /* Eq. R_New */
  /* Eqs. R1_prime, R2_prime, R3_New in the rotated frame. */
  const double r1p = (-mach * rs + d1p) / (beta2 * r);
  const double r2p = d2p / r;
  const double r3 = d[2] / r;
  /* Eqs. R1_New, R2_New: rotate back. */
  Rhat[0] = r1p * ca - r2p * sa;
  Rhat[1] = r1p * sa + r2p * ca;
  Rhat[2] = r3;
  *R = r;
  *Rs = rs;
}

int fwho_convected_distance(int64_t n, const double *d, double mach, double aoa,
                            double *R, double *Rs, double *Rhat) {
  if (n < 0 || !(mach > 0.0 && mach < 1.0)) return FWHO_ERR_ARG;
  for (int64_t i = 0; i < n; ++i)
    convected_distance(d + 3 * i, mach, aoa, R + i, Rs + i, Rhat + 3 * i);
  return FWHO_OK;
}

/* ------------------------------------------------------------------------ */
/* Step 2 helpers: finite differences and the natural cubic spline.          */
/* ------------------------------------------------------------------------ */

/* Second-order source-time derivative: central inside, one-sided 3-point at
 * the first and last sample.  Needs n >= 3. */
static void fd_derivative(int64_t n, double h, const double *y, int64_t sy,
                          double *yd) {
  const double inv2h = 1.0 / (2.0 * h);
  yd[0] = (-3.0 * y[0] + 4.0 * y[sy] - y[2 * sy]) * inv2h;
  for (int64_t i = 1; i < n - 1; ++i)
    yd[i] = (y[(i + 1) * sy] - y[(i - 1) * sy]) * inv2h;
  yd[n - 1] = (3.0 * y[(n - 1) * sy] - 4.0 * y[(n - 2) * sy] + y[(n - 3) * sy]) * inv2h;
}

int fwho_fd_derivative(int64_t n, double h, const double *y, double *yd) {
  if (n < 3 || !(h > 0)) return FWHO_ERR_ARG;
  fd_derivative(n, h, y, 1, yd);
  return FWHO_OK;
}

/* Natural cubic spline second derivatives m[0..n-1] of samples y on a grid of
 * spacing h: m_0 = m_{n-1} = 0 and, for 0 < i < n-1,
 *   m_{i-1} + 4 m_i + m_{i+1} = 6 (y_{i+1} - 2 y_i + y_{i-1}) / h^2,
 * solved by plain Gaussian elimination of the tridiagonal system.
 * work must hold n doubles. */
static void natural_spline_moments(int64_t n, double h, const double *y,
                                   double *m, double *work) {
  m[0] = 0.0;
  m[n - 1] = 0.0;
  if (n < 3) return;
  const int64_t k = n - 2; /* unknowns m_1 .. m_{n-2} */
  double *cp = work;       /* modified super-diagonal */
  const double s = 6.0 / (h * h);
  /* forward elimination, rhs kept in m[1..n-2] */
  double piv = 4.0;
  cp[0] = 1.0 / piv;
  m[1] = s * (y[2] - 2.0 * y[1] + y[0]) / piv;
  for (int64_t i = 1; i < k; ++i) {
    piv = 4.0 - cp[i - 1];
    cp[i] = 1.0 / piv;
    const double r = s * (y[i + 2] - 2.0 * y[i + 1] + y[i]);
    m[i + 1] = (r - m[i]) / piv;
  }
  /* back substitution */
  for (int64_t i = k - 2; i >= 0; --i) m[i + 1] -= cp[i] * m[i + 2];
}

int fwho_natural_spline_moments(int64_t n, double h, const double *y, double *m) {
  if (n < 2 || !(h > 0)) return FWHO_ERR_ARG;
  double *work = (double *)malloc(sizeof(double) * (size_t)(n > 2 ? n : 2));
  if (!work) return FWHO_ERR_OOM;
  natural_spline_moments(n, h, y, m, work);
  free(work);
  return FWHO_OK;
}

/* Locate x on the grid tau_i = i h and return the interval index k in
 * [0, n-2] with the two linear weights (A on y_k, B on y_{k+1}). */
static void spline_locate(int64_t n, double h, double x, int64_t *k, double *A,
                          double *B) {
  double u = x / h;
  int64_t kk = (int64_t)floor(u);
  if (kk < 0) kk = 0;
  if (kk > n - 2) kk = n - 2;
  const double b = u - (double)kk;
  *k = kk;
  *B = b;
  *A = 1.0 - b;
}

/* Value of the cubic spline with moments m at x. */
static double spline_eval(int64_t n, double h, const double *y, const double *m,
                          double x) {
  int64_t k;
  double A, B;
  spline_locate(n, h, x, &k, &A, &B);
  return A * y[k] + B * y[k + 1] +
         ((A * A * A - A) * m[k] + (B * B * B - B) * m[k + 1]) * (h * h) / 6.0;
}

int fwho_spline_eval(int64_t n, double h, const double *y, const double *m,
                     int64_t nx, const double *x, double *out) {
  if (n < 2 || !(h > 0)) return FWHO_ERR_ARG;
  for (int64_t i = 0; i < nx; ++i) out[i] = spline_eval(n, h, y, m, x[i]);
  return FWHO_OK;
}

/* ------------------------------------------------------------------------ */
/* Step 2: integrands from pulsations.                                       */
/* ------------------------------------------------------------------------ */

/* fields: [nt][5][P] = rho', u', v', w', p'.  QL: [nt][4][P] = Q_n, L1..L3. */
int fwho_integrands(int64_t P, int64_t nt, const double *normals, double aoa,
                    const double *fields, double *QL) {
  if (P < 0 || nt < 0) return FWHO_ERR_ARG;
  const double U[3] = {cos(aoa), sin(aoa), 0.0}; /* Eq. U_0_nd */
  for (int64_t i = 0; i < nt; ++i) {
    const double *f = fields + i * 5 * P;
    double *q = QL + i * 4 * P;
    for (int64_t p = 0; p < P; ++p) {
      const double *n = normals + 3 * p;
      const double rho = 1.0 + f[0 * P + p];
      const double u[3] = {U[0] + f[1 * P + p], U[1] + f[2 * P + p],
                           U[2] + f[3 * P + p]};
      const double pp = f[4 * P + p];
      /* Eq. Qn_New_nd: Q_n = (-U0_i + rho u_i) n_i */
      double qn = 0.0, un = 0.0;
      for (int c = 0; c < 3; ++c) {
        qn += (-U[c] + rho * u[c]) * n[c];
        un += u[c] * n[c];
      }
      q[0 * P + p] = qn;
      /* Eq. Li_New_nd: L_i = [p' delta_ij + rho (u_i - U0_i) u_j] n_j */
      for (int c = 0; c < 3; ++c)
        q[(1 + c) * P + p] = pp * n[c] + rho * (u[c] - U[c]) * un;
    }
  }
  return FWHO_OK;
}

/* Vector-Jacobian product of fwho_integrands: fields_bar += J^T QL_bar. */
int fwho_integrands_vjp(int64_t P, int64_t nt, const double *normals, double aoa,
                        const double *fields, const double *QL_bar,
                        double *fields_bar) {
  if (P < 0 || nt < 0) return FWHO_ERR_ARG;
  const double U[3] = {cos(aoa), sin(aoa), 0.0};
  for (int64_t i = 0; i < nt; ++i) {
    const double *f = fields + i * 5 * P;
    const double *qb = QL_bar + i * 4 * P;
    double *fb = fields_bar + i * 5 * P;
    for (int64_t p = 0; p < P; ++p) {
      const double *n = normals + 3 * p;
      const double rho = 1.0 + f[0 * P + p];
      const double up[3] = {f[1 * P + p], f[2 * P + p], f[3 * P + p]};
      const double u[3] = {U[0] + up[0], U[1] + up[1], U[2] + up[2]};
      const double un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
      const double qnb = qb[0 * P + p];
      const double lb[3] = {qb[1 * P + p], qb[2 * P + p], qb[3 * P + p]};
      /* dQn/drho = u.n ; dQn/du_c = rho n_c */
      double g_rho = qnb * un;
      double g_u[3] = {qnb * rho * n[0], qnb * rho * n[1], qnb * rho * n[2]};
      double g_p = 0.0;
      /* L_c = p n_c + rho u'_c (u.n):
       * dL_c/dp = n_c ; dL_c/drho = u'_c un ; dL_c/du_k = rho (delta_ck un + u'_c n_k) */
      double lu = 0.0; /* sum_c lb_c u'_c */
      for (int c = 0; c < 3; ++c) {
        g_p += lb[c] * n[c];
        g_rho += lb[c] * up[c] * un;
        g_u[c] += lb[c] * rho * un;
        lu += lb[c] * up[c];
      }
      for (int k = 0; k < 3; ++k) g_u[k] += rho * lu * n[k];
      fb[0 * P + p] += g_rho;
      fb[1 * P + p] += g_u[0];
      fb[2 * P + p] += g_u[1];
      fb[3 * P + p] += g_u[2];
      fb[4 * P + p] += g_p;
    }
  }
  return FWHO_OK;
}

/* ------------------------------------------------------------------------ */
/* Steps 3-5 on given integrands.                                            */
/* ------------------------------------------------------------------------ */

typedef struct {
  double R, Rs, Rhat[3];
} geo_t;

/* Source-time pressure of one subface at one frame, Eqs. pT_WT_nd and
 * pL_WT_nd term by term (the integrand times dS/(4 pi)). */
static double source_pressure(const geo_t *g, double mach, const double M[3],
                              double dS, double qn, double qnd, const double L[3],
                              const double Ld[3]) {
  const double MR = M[0] * g->Rhat[0] + M[1] * g->Rhat[1] + M[2] * g->Rhat[2];
  const double Msq = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
  const double D = 1.0 - MR;
  const double R = g->R;
  const double LR = L[0] * g->Rhat[0] + L[1] * g->Rhat[1] + L[2] * g->Rhat[2];
  const double LRd = Ld[0] * g->Rhat[0] + Ld[1] * g->Rhat[1] + Ld[2] * g->Rhat[2];
  const double LM = L[0] * M[0] + L[1] * M[1] + L[2] * M[2];
  /* thickness, Eq. pT_WT_nd */
  const double t1 = qnd / (R * D * D);
  const double t2 = qn * (MR - Msq) / (mach * R * R * D * D * D);
  /* loading, Eq. pL_WT_nd */
  const double t3 = mach * LRd / (R * D * D);
  const double t4 = (LR - LM) / (R * R * D * D);
  const double t5 = LR * (MR - Msq) / (R * R * D * D * D);
  return (t1 + t2 + t3 + t4 + t5) * dS / (4.0 * FWHO_PI);
}

/* Partial derivatives of source_pressure with respect to
 * (Qn-dot, Qn, L-dot_1..3, L_1..3); used only by the adjoint. */
static void source_pressure_grad(const geo_t *g, double mach, const double M[3],
                                 double dS, double w[8]) {
  const double MR = M[0] * g->Rhat[0] + M[1] * g->Rhat[1] + M[2] * g->Rhat[2];
  const double Msq = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
  const double D = 1.0 - MR;
  const double R = g->R;
  const double S = dS / (4.0 * FWHO_PI);
  w[0] = S / (R * D * D);
  w[1] = S * (MR - Msq) / (mach * R * R * D * D * D);
  for (int c = 0; c < 3; ++c) {
    w[2 + c] = S * mach * g->Rhat[c] / (R * D * D);
    w[5 + c] = S * (g->Rhat[c] / (R * R * D * D) - M[c] / (R * R * D * D) +
                    g->Rhat[c] * (MR - Msq) / (R * R * D * D * D));
  }
}

typedef struct {
  int64_t P, nt, O;
  const double *y, *n, *dS, *x;
  double mach, aoa, dt;
} prob_t;

/* Per-observer window: R for all panels, t_start and N_o. */
static void observer_window(const prob_t *pb, int64_t o, geo_t *geo,
                            double *t_start, int64_t *n_valid) {
  double rmax = -INFINITY, rmin = INFINITY;
  for (int64_t p = 0; p < pb->P; ++p) {
    double d[3];
    for (int c = 0; c < 3; ++c) d[c] = pb->x[3 * o + c] - pb->y[3 * p + c];
    convected_distance(d, pb->mach, pb->aoa, &geo[p].R, &geo[p].Rs, geo[p].Rhat);
    if (geo[p].R > rmax) rmax = geo[p].R;
    if (geo[p].R < rmin) rmin = geo[p].R;
  }
  const double tau_max = (double)(pb->nt - 1) * pb->dt;
  const double ts = rmax * pb->mach;          /* Eq. t_start */
  const double te = tau_max + rmin * pb->mach; /* Eq. t_end */
  int64_t nv = (int64_t)floor((te - ts) / pb->dt) + 1;
  if (nv < 0) nv = 0;
  if (nv > pb->nt) nv = pb->nt;
  *t_start = ts;
  *n_valid = nv;
}

static void neumaier_add(double *s, double *c, double v) {
  const double t = *s + v;
  if (fabs(*s) >= fabs(v))
    *c += (*s - t) + v;
  else
    *c += (v - t) + *s;
  *s = t;
}

/* Forward on integrands QL [nt][4][P]; sums subfaces [p_lo, p_hi). */
static int forward_QL(const prob_t *pb, const double *QL, int64_t p_lo,
                      int64_t p_hi, int compensated, int n_threads,
                      double *p_out, double *t_start, int64_t *n_valid) {
  const int64_t P = pb->P, nt = pb->nt;
  const double M[3] = {-pb->mach * cos(pb->aoa), -pb->mach * sin(pb->aoa), 0.0};
  geo_t *geo = (geo_t *)malloc(sizeof(geo_t) * (size_t)(P > 0 ? P : 1));
  if (!geo) return FWHO_ERR_OOM;
  memset(p_out, 0, sizeof(double) * (size_t)(pb->O * nt));
#ifdef _OPENMP
  if (n_threads <= 0) n_threads = omp_get_max_threads();
#else
  n_threads = 1;
#endif
  for (int64_t o = 0; o < pb->O; ++o) {
    double ts;
    int64_t nv;
    observer_window(pb, o, geo, &ts, &nv);
    t_start[o] = ts;
    n_valid[o] = nv;
    double *acc = (double *)calloc((size_t)(2 * nv * n_threads + 1), sizeof(double));
    if (!acc) {
      free(geo);
      return FWHO_ERR_OOM;
    }
#ifdef _OPENMP
#pragma omp parallel num_threads(n_threads)
#endif
    {
#ifdef _OPENMP
      const int tid = omp_get_thread_num();
#else
      const int tid = 0;
#endif
      double *mys = acc + 2 * nv * tid;
      double *myc = mys + nv;
      double *buf = (double *)malloc(sizeof(double) * (size_t)(12 * nt + 4));
      double *qn = buf, *qnd = buf + nt, *L = buf + 2 * nt, *Ld = buf + 5 * nt;
      double *sig = buf + 8 * nt, *mom = buf + 9 * nt, *work = buf + 10 * nt;
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
      for (int64_t p = p_lo; p < p_hi; ++p) {
        /* "compute Noise": integrands and their source-time derivatives */
        for (int64_t i = 0; i < nt; ++i) {
          qn[i] = QL[i * 4 * P + 0 * P + p];
          for (int c = 0; c < 3; ++c) L[c * nt + i] = QL[i * 4 * P + (1 + c) * P + p];
        }
        fd_derivative(nt, pb->dt, qn, 1, qnd);
        for (int c = 0; c < 3; ++c) fd_derivative(nt, pb->dt, L + c * nt, 1, Ld + c * nt);
        for (int64_t i = 0; i < nt; ++i) {
          const double Li[3] = {L[i], L[nt + i], L[2 * nt + i]};
          const double Ldi[3] = {Ld[i], Ld[nt + i], Ld[2 * nt + i]};
          sig[i] = source_pressure(&geo[p], pb->mach, M, pb->dS[p], qn[i], qnd[i], Li, Ldi);
        }
        /* "interp pressure signal": natural cubic spline onto t_j - M0 R */
        natural_spline_moments(nt, pb->dt, sig, mom, work);
        for (int64_t j = 0; j < nv; ++j) {
          const double tj = ts + (double)j * pb->dt;
          const double tau = tj - pb->mach * geo[p].R; /* Eq. tau2 */
          const double v = spline_eval(nt, pb->dt, sig, mom, tau);
          if (compensated)
            neumaier_add(&mys[j], &myc[j], v);
          else
            mys[j] += v;
        }
      }
      free(buf);
    }
    /* surface integration across threads */
    for (int64_t j = 0; j < nv; ++j) {
      double s = 0.0, c = 0.0;
      for (int t = 0; t < n_threads; ++t) {
        if (compensated) {
          neumaier_add(&s, &c, acc[2 * nv * t + j]);
          neumaier_add(&s, &c, acc[2 * nv * t + nv + j]);
        } else {
          s += acc[2 * nv * t + j];
        }
      }
      p_out[o * nt + j] = s + c;
    }
    free(acc);
  }
  free(geo);
  return FWHO_OK;
}

static int check_prob(const prob_t *pb) {
  if (pb->P < 1 || pb->nt < 3 || pb->O < 0) return FWHO_ERR_ARG;
  if (!(pb->mach > 0.0 && pb->mach < 1.0) || !(pb->dt > 0.0)) return FWHO_ERR_ARG;
  if (!pb->y || !pb->n || !pb->dS || (pb->O > 0 && !pb->x)) return FWHO_ERR_ARG;
  return FWHO_OK;
}

int fwho_forward_QL(int64_t P, const double *centroids, const double *normals,
                    const double *areas, double mach, double aoa, double dt,
                    int64_t nt, const double *QL, int64_t O, const double *obs,
                    int64_t p_lo, int64_t p_hi, int compensated, int n_threads,
                    double *p_out, double *t_start, int64_t *n_valid) {
  prob_t pb = {P, nt, O, centroids, normals, areas, obs, mach, aoa, dt};
  int st = check_prob(&pb);
  if (st) return st;
  if (p_lo < 0 || p_hi > P || p_lo > p_hi) return FWHO_ERR_ARG;
  return forward_QL(&pb, QL, p_lo, p_hi, compensated, n_threads, p_out, t_start,
                    n_valid);
}

int fwho_forward(int64_t P, const double *centroids, const double *normals,
                 const double *areas, double mach, double aoa, double dt, int64_t nt,
                 const double *fields, int64_t O, const double *obs, int64_t p_lo,
                 int64_t p_hi, int compensated, int n_threads, double *p_out,
                 double *t_start, int64_t *n_valid) {
  prob_t pb = {P, nt, O, centroids, normals, areas, obs, mach, aoa, dt};
  int st = check_prob(&pb);
  if (st) return st;
  if (p_lo < 0 || p_hi > P || p_lo > p_hi) return FWHO_ERR_ARG;
  double *QL = (double *)malloc(sizeof(double) * (size_t)(4 * P * nt));
  if (!QL) return FWHO_ERR_OOM;
  fwho_integrands(P, nt, normals, aoa, fields, QL);
  st = forward_QL(&pb, QL, p_lo, p_hi, compensated, n_threads, p_out, t_start, n_valid);
  free(QL);
  return st;
}

/* ------------------------------------------------------------------------ */
/* Adjoint: exact transpose of forward_QL, then the integrand Jacobian.      */
/* ------------------------------------------------------------------------ */

/* grad_p [O][nt] (entries j >= N_o ignored) -> QL_bar [nt][4][P] (overwritten). */
int fwho_backward_QL(int64_t P, const double *centroids, const double *normals,
                     const double *areas, double mach, double aoa, double dt,
                     int64_t nt, int64_t O, const double *obs, const double *grad_p,
                     int n_threads, double *QL_bar) {
  prob_t pb = {P, nt, O, centroids, normals, areas, obs, mach, aoa, dt};
  int st = check_prob(&pb);
  if (st) return st;
  const double M[3] = {-mach * cos(aoa), -mach * sin(aoa), 0.0};
  memset(QL_bar, 0, sizeof(double) * (size_t)(4 * P * nt));
  geo_t *geo = (geo_t *)malloc(sizeof(geo_t) * (size_t)P);
  if (!geo) return FWHO_ERR_OOM;
#ifdef _OPENMP
  if (n_threads <= 0) n_threads = omp_get_max_threads();
#else
  n_threads = 1;
#endif
  const double h = dt, s6 = 6.0 / (dt * dt);
  for (int64_t o = 0; o < O; ++o) {
    double ts;
    int64_t nv;
    observer_window(&pb, o, geo, &ts, &nv);
    const double *gp = grad_p + o * nt;
#ifdef _OPENMP
#pragma omp parallel num_threads(n_threads)
#endif
    {
      double *buf = (double *)malloc(sizeof(double) * (size_t)(6 * nt + 4));
      double *sb = buf, *mb = buf + nt, *rb = buf + 2 * nt, *work = buf + 3 * nt;
      double *qdb = buf + 4 * nt, *tmp = buf + 5 * nt;
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
      for (int64_t p = 0; p < P; ++p) {
        memset(sb, 0, sizeof(double) * (size_t)nt);
        memset(mb, 0, sizeof(double) * (size_t)nt);
        /* transpose of the spline evaluation */
        for (int64_t j = 0; j < nv; ++j) {
          const double tau = ts + (double)j * dt - mach * geo[p].R;
          int64_t k;
          double A, B;
          spline_locate(nt, h, tau, &k, &A, &B);
          const double gb = gp[j];
          sb[k] += A * gb;
          sb[k + 1] += B * gb;
          mb[k] += (A * A * A - A) * h * h / 6.0 * gb;
          mb[k + 1] += (B * B * B - B) * h * h / 6.0 * gb;
        }
        /* transpose of the moment solve: the interior matrix is symmetric, so
         * r_bar = T^{-1} m_bar(interior); boundary moments are fixed zeros. */
        if (nt >= 3) {
          /* reuse the forward solver: solve T z = mb[1..nt-2] */
          const int64_t kk = nt - 2;
          double piv = 4.0;
          work[0] = 1.0 / piv;
          rb[1] = mb[1] / piv;
          for (int64_t i = 1; i < kk; ++i) {
            piv = 4.0 - work[i - 1];
            work[i] = 1.0 / piv;
            rb[i + 1] = (mb[i + 1] - rb[i]) / piv;
          }
          for (int64_t i = kk - 2; i >= 0; --i) rb[i + 1] -= work[i] * rb[i + 2];
          /* r_i = s6 (y_{i+1} - 2 y_i + y_{i-1}) for i = 1..nt-2 */
          for (int64_t i = 1; i <= nt - 2; ++i) {
            const double z = s6 * rb[i];
            sb[i + 1] += z;
            sb[i] -= 2.0 * z;
            sb[i - 1] += z;
          }
        }
        /* transpose of the per-frame source pressure (linear in integrands) */
        double w[8];
        source_pressure_grad(&geo[p], mach, M, areas[p], w);
        /* series 0: Qn (direct w[1], via FD w[0]); series 1..3: L_c (w[5+c], FD w[2+c]) */
        for (int s = 0; s < 4; ++s) {
          const double wd = (s == 0) ? w[0] : w[2 + (s - 1)];
          const double wv = (s == 0) ? w[1] : w[5 + (s - 1)];
          for (int64_t i = 0; i < nt; ++i) qdb[i] = wd * sb[i];
          /* transpose of fd_derivative */
          const double inv2h = 1.0 / (2.0 * dt);
          for (int64_t i = 0; i < nt; ++i) tmp[i] = wv * sb[i];
          tmp[0] += -3.0 * inv2h * qdb[0];
          tmp[1] += 4.0 * inv2h * qdb[0];
          tmp[2] += -1.0 * inv2h * qdb[0];
          for (int64_t i = 1; i < nt - 1; ++i) {
            tmp[i + 1] += inv2h * qdb[i];
            tmp[i - 1] -= inv2h * qdb[i];
          }
          tmp[nt - 1] += 3.0 * inv2h * qdb[nt - 1];
          tmp[nt - 2] += -4.0 * inv2h * qdb[nt - 1];
          tmp[nt - 3] += 1.0 * inv2h * qdb[nt - 1];
          /* each panel p is owned by one thread: no race on QL_bar[.., p] */
          for (int64_t i = 0; i < nt; ++i) QL_bar[i * 4 * P + s * P + p] += tmp[i];
        }
      }
      free(buf);
    }
  }
  free(geo);
  return FWHO_OK;
}

int fwho_backward(int64_t P, const double *centroids, const double *normals,
                  const double *areas, double mach, double aoa, double dt, int64_t nt,
                  const double *fields, int64_t O, const double *obs,
                  const double *grad_p, int n_threads, double *grad_fields) {
  double *QLb = (double *)malloc(sizeof(double) * (size_t)(4 * (P > 0 ? P : 1) * (nt > 0 ? nt : 1)));
  if (!QLb) return FWHO_ERR_OOM;
  int st = fwho_backward_QL(P, centroids, normals, areas, mach, aoa, dt, nt, O, obs,
                            grad_p, n_threads, QLb);
  if (!st) {
    memset(grad_fields, 0, sizeof(double) * (size_t)(5 * P * nt));
    st = fwho_integrands_vjp(P, nt, normals, aoa, fields, QLb, grad_fields);
  }
  free(QLb);
  return st;
}

/* Observer window only (t_start, N_o per observer). */
int fwho_observer_window(int64_t P, const double *centroids, double mach, double aoa,
                         double dt, int64_t nt, int64_t O, const double *obs,
                         double *t_start, int64_t *n_valid) {
  if (P < 1 || nt < 3 || O < 0 || !(mach > 0.0 && mach < 1.0) || !(dt > 0.0))
    return FWHO_ERR_ARG;
  geo_t *geo = (geo_t *)malloc(sizeof(geo_t) * (size_t)P);
  if (!geo) return FWHO_ERR_OOM;
  prob_t pb = {P, nt, O, centroids, NULL, NULL, obs, mach, aoa, dt};
  for (int64_t o = 0; o < O; ++o) observer_window(&pb, o, geo, t_start + o, n_valid + o);
  free(geo);
  return FWHO_OK;
}

int fwho_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ======================================================================== */
/* General moving surface: Eqs. pT and pL of Sec. II B (Farassat 1A for a   */
/* permeable surface moving in a medium at rest), retarded time Eq. tau.    */
/* ======================================================================== */
/*
 * Panels p with per-frame centroid y_p(tau_i), unit normal n_p(tau_i) and
 * velocity v_p(tau_i) ([nt][P][3] each) and a constant area dS_p; a medium at
 * rest with density rho0 and sound speed c0; per frame the density pulsation
 * rho', the fluid velocity u (in the medium's frame) and p' ([nt][5][P]).
 * Observers start at x0_o and move with one constant velocity w (w = 0: at
 * rest; |w| < c0).  For (p, o, i), with b = x0_o + w tau_i - y_p(tau_i):
 *   the delay Delta >= 0 of |b + w Delta| = c0 Delta (Eq. tau, r = c0 (t - tau)),
 *   r = c0 Delta, r-hat = (b + w Delta) / r, arrival t_i = tau_i + Delta;
 *   M = v / c0, M-dot = (dv/dtau) / c0, M_r = M.r-hat (Eq. Mr), M-dot_r =
 *   M-dot.r-hat, M^2 = M.M, D = 1 - M_r;
 *   Q_n = [rho0 v + rho (u - v)].n (Eq. Qn, rho = rho0 + rho'), whose source-time
 *   derivative is the Q-dot_i n_i + Q_i n-dot_i of Eq. pT;
 *   L_i = p' n_i + rho u_i (u.n - v.n) (Eq. Li, P_ij = p' delta_ij), L_r = L.r-hat
 *   (Eq. Lr), L-dot_r = L-dot.r-hat, L_M = L.M (Eq. LM);
 *   g_i = dS / (4 pi) [ Qdot_n / (r D^2) + Q_n (r Mdot_r + c0 (M_r - M^2)) / (r^2 D^3)
 *         + Ldot_r / (c0 r D^2) + (L_r - L_M) / (r^2 D^2)
 *         + L_r (r Mdot_r + c0 (M_r - M^2)) / (c0 r^2 D^3) ].
 * Source-time derivatives by the second-order differences of Sec. III B.
 * Observer window: t_start = max_p t_p(tau_0), t_end = min_p t_p(tau_max),
 * N_o = floor((t_end - t_start) / dt) + 1, t_j = t_start + j dt (the moving-
 * surface generalisation of Eqs. t_start, t_end).  Each panel's g and t are
 * natural cubic splines over tau; for bin j, tau* with t(tau*) = t_j lies in
 * the interval whose arrival times bracket t_j and is found there by
 * bisection on the spline of t; p_j += g-spline(tau*).  Subsonic motion
 * (|M_r| < 1) keeps t increasing in tau.
 */

typedef struct {
  int64_t P, nt, O;
  const double *y, *n, *v, *dS, *x0, *w;
  double c0, rho0, dt;
} mprob_t;

/* Delay, distance and unit radiation vector of one source sample. */
static void moving_arrival(const mprob_t *pb, const double x0[3], double tau,
                           const double y[3], double *delay, double *r, double rh[3]) {
  double b[3];
  for (int c = 0; c < 3; ++c) b[c] = x0[c] + pb->w[c] * tau - y[c];
  const double ww = pb->w[0] * pb->w[0] + pb->w[1] * pb->w[1] + pb->w[2] * pb->w[2];
  const double bw = b[0] * pb->w[0] + b[1] * pb->w[1] + b[2] * pb->w[2];
  const double bb = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
  const double a = pb->c0 * pb->c0 - ww; /* > 0 */
  /* (c0^2 - w.w) D^2 - 2 (b.w) D - b.b = 0, the non-negative root */
  const double d = (bw + sqrt(bw * bw + a * bb)) / a;
  *delay = d;
  *r = pb->c0 * d;
  for (int c = 0; c < 3; ++c) rh[c] = (b[c] + pb->w[c] * d) / *r;
}

/* Arrival time of sample i of panel p at observer o. */
static double moving_t(const mprob_t *pb, int64_t p, int64_t o, int64_t i) {
  double d, r, rh[3];
  moving_arrival(pb, pb->x0 + 3 * o, (double)i * pb->dt, pb->y + (i * pb->P + p) * 3, &d, &r, rh);
  return (double)i * pb->dt + d;
}

int fwho_forward_moving(int64_t P, int64_t nt, const double *y, const double *nrm,
                        const double *vel, const double *areas, double c0, double rho0,
                        double dt, const double *fields, int64_t O, const double *x0,
                        const double *w, int n_threads, double *p_out, double *t_start,
                        int64_t *n_valid) {
  if (P < 1 || nt < 3 || O < 0 || !(c0 > 0.0) || !(dt > 0.0) || !(rho0 > 0.0))
    return FWHO_ERR_ARG;
  if (w[0] * w[0] + w[1] * w[1] + w[2] * w[2] >= c0 * c0) return FWHO_ERR_ARG;
  mprob_t pb = {P, nt, O, y, nrm, vel, areas, x0, w, c0, rho0, dt};
  memset(p_out, 0, sizeof(double) * (size_t)(O * nt));
#ifdef _OPENMP
  if (n_threads <= 0) n_threads = omp_get_max_threads();
#else
  n_threads = 1;
#endif
  for (int64_t o = 0; o < O; ++o) {
    double ts = -INFINITY, te = INFINITY;
    for (int64_t p = 0; p < P; ++p) {
      const double t0 = moving_t(&pb, p, o, 0), t1 = moving_t(&pb, p, o, nt - 1);
      if (t0 > ts) ts = t0;
      if (t1 < te) te = t1;
    }
    int64_t nv = (int64_t)floor((te - ts) / dt) + 1;
    if (nv < 0) nv = 0;
    if (nv > nt) nv = nt;
    t_start[o] = ts;
    n_valid[o] = nv;
    double *acc = (double *)calloc((size_t)(nv * n_threads + 1), sizeof(double));
    if (!acc) return FWHO_ERR_OOM;
#ifdef _OPENMP
#pragma omp parallel num_threads(n_threads)
#endif
    {
#ifdef _OPENMP
      const int tid = omp_get_thread_num();
#else
      const int tid = 0;
#endif
      double *mys = acc + nv * tid;
      double *buf = (double *)malloc(sizeof(double) * (size_t)(20 * nt + 4));
      double *qn = buf, *qnd = buf + nt, *L = buf + 2 * nt, *Ld = buf + 5 * nt;
      double *vv = buf + 8 * nt, *vd = buf + 11 * nt;
      double *g = buf + 14 * nt, *mg = buf + 15 * nt, *tt = buf + 16 * nt;
      double *mt = buf + 17 * nt, *work = buf + 18 * nt;
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
      for (int64_t p = 0; p < P; ++p) {
        /* Eqs. Qn, Li per frame, and the surface velocity, then their FD derivatives */
        for (int64_t i = 0; i < nt; ++i) {
          const double *ni = nrm + (i * P + p) * 3, *vi = vel + (i * P + p) * 3;
          const double rho = rho0 + fields[(i * 5 + 0) * P + p];
          const double u[3] = {fields[(i * 5 + 1) * P + p], fields[(i * 5 + 2) * P + p],
                               fields[(i * 5 + 3) * P + p]};
          const double pp = fields[(i * 5 + 4) * P + p];
          double q = 0.0, un = 0.0, vn = 0.0;
          for (int c = 0; c < 3; ++c) {
            q += (rho0 * vi[c] + rho * (u[c] - vi[c])) * ni[c];
            un += u[c] * ni[c];
            vn += vi[c] * ni[c];
          }
          qn[i] = q;
          for (int c = 0; c < 3; ++c) {
            L[c * nt + i] = pp * ni[c] + rho * u[c] * (un - vn);
            vv[c * nt + i] = vi[c];
          }
        }
        fd_derivative(nt, dt, qn, 1, qnd);
        for (int c = 0; c < 3; ++c) {
          fd_derivative(nt, dt, L + c * nt, 1, Ld + c * nt);
          fd_derivative(nt, dt, vv + c * nt, 1, vd + c * nt);
        }
        /* Eqs. pT + pL at every source sample, with its arrival time (Eq. tau) */
        for (int64_t i = 0; i < nt; ++i) {
          double d, r, rh[3];
          moving_arrival(&pb, x0 + 3 * o, (double)i * dt, y + (i * P + p) * 3, &d, &r, rh);
          double Mr = 0.0, Mdr = 0.0, M2 = 0.0, Lr = 0.0, Ldr = 0.0, LM = 0.0;
          for (int c = 0; c < 3; ++c) {
            const double M = vv[c * nt + i] / c0, Md = vd[c * nt + i] / c0;
            Mr += M * rh[c];
            Mdr += Md * rh[c];
            M2 += M * M;
            Lr += L[c * nt + i] * rh[c];
            Ldr += Ld[c * nt + i] * rh[c];
            LM += L[c * nt + i] * M;
          }
          const double D = 1.0 - Mr;
          const double k = r * Mdr + c0 * (Mr - M2);
          const double thick = qnd[i] / (r * D * D) + qn[i] * k / (r * r * D * D * D);
          const double load = Ldr / (c0 * r * D * D) + (Lr - LM) / (r * r * D * D) +
                              Lr * k / (c0 * r * r * D * D * D);
          g[i] = areas[p] / (4.0 * FWHO_PI) * (thick + load);
          tt[i] = (double)i * dt + d;
        }
        natural_spline_moments(nt, dt, g, mg, work);
        natural_spline_moments(nt, dt, tt, mt, work);
        int64_t k = 0;
        for (int64_t j = 0; j < nv; ++j) {
          const double tj = ts + (double)j * dt;
          while (k < nt - 2 && tt[k + 1] < tj) ++k;
          /* bisection on the spline of t over [tau_k, tau_k+1] */
          double lo = (double)k * dt, hi = (double)(k + 1) * dt;
          for (int it = 0; it < 64; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (spline_eval(nt, dt, tt, mt, mid) < tj)
              lo = mid;
            else
              hi = mid;
          }
          mys[j] += spline_eval(nt, dt, g, mg, 0.5 * (lo + hi));
        }
      }
      free(buf);
    }
    for (int64_t j = 0; j < nv; ++j) {
      double s = 0.0;
      for (int t = 0; t < n_threads; ++t) s += acc[nv * t + j];
      p_out[o * nt + j] = s;
    }
    free(acc);
  }
  return FWHO_OK;
}
