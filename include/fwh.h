/*
 * fwh.h -- C ABI of the GB300 FW-H library (permeable-surface, nondimensional,
 * wind-tunnel Ffowcs Williams-Hawkings integral of OpenCFD-FWH,
 * arXiv 2312.16263).
 *
 * The library evaluates, for every (surface panel, source time, observer),
 * the Farassat-1A-type thickness and loading integrands of the wind-tunnel
 * form (Sec. II C, Eqs. pT_WT and pL_WT, nondimensionalised as Eqs. pT_WT_nd
 * and pL_WT_nd of Sec. II D), with the convected distance from the Garrick
 * triangle and the angle of attack by rotation (Eqs. R_New .. R2_New), and
 * places each subface's source-time signal on the observer-time grid by
 * natural cubic-spline interpolation (Sec. III B, "interp pressure signal"),
 * summed over subfaces (Sec. III C).
 *
 * Conventions for every entry point:
 *  - Everything is nondimensional (Sec. II D): rho* = rho/rho0,
 *    u* = u/U0, p* = p/(rho0 U0^2), c0* = 1/M0, x* = x/Lref, t* = t U0/Lref.
 *  - Fields are PULSATIONS, laid out [nt][5][P]: for frame i and panel p,
 *    fields[(i*5 + c)*P + p] holds c = 0 rho', 1 u', 2 v', 3 w', 4 p'.
 *    Totals are rebuilt as rho = 1 + rho', u = (cos a, sin a, 0) + u'.
 *    FWH_FP64 handles take double fields, FWH_MIXED handles float fields.
 *  - Source time tau_i = i dt, i = 0..nt-1.  Observer o's time grid is
 *    t_j = t_start(o) + j dt with t_start = M0 R_max(o) (Eq. t_start) and
 *    N_o = floor((t_end - t_start)/dt) + 1 valid bins, t_end = tau_max +
 *    M0 R_min(o) (Eq. t_end).  Outputs are [O][nt] doubles, row o holding
 *    p'(t_j) for j < N_o and 0 for j >= N_o.
 *  - The caller owns every buffer it passes; the library copies geometry and
 *    observers into its own device memory.  Buffers may be device pointers
 *    (used in place, on `stream`) or host pointers (pageable or pinned; the
 *    library stages them through device memory it owns and copies results
 *    back before returning).  Host inputs are read by copies that complete
 *    before `stream` passes the call: with a device output the call may
 *    return earlier, and the input must stay unchanged until then.
 *  - `stream` is a cudaStream_t passed as void* (NULL = default stream).
 *    Device work is enqueued on it; calls with host outputs synchronise it.
 *  - Every call returns a status and never aborts; fwh_last_error() gives a
 *    message for the last failing call on that handle.
 *  - Device-side checks (a bounded wait that gave up, a panel set whose
 *    arrival spread exceeded its window) raise a flag on the device.  Calls
 *    with host outputs read it before returning.  Calls whose outputs stay on
 *    the device copy it to pinned host memory behind their work, and the next
 *    call on the handle (forward, backward, batched or allocation-free
 *    forward) that finds that copy complete reports it as its own status
 *    (FWH_ERR_TIMEOUT or FWH_ERR_CUDA, message "an earlier call on this
 *    handle: ...") without running; fwh_check reports it synchronously.
 */
#ifndef FWH_H_
#define FWH_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fwh_ctx *fwh_handle;

typedef enum {
  FWH_OK = 0,
  FWH_ERR_ARG = 1,     /* invalid argument (sizes, ranges, null pointers) */
  FWH_ERR_CUDA = 2,    /* a CUDA runtime call or kernel launch failed */
  FWH_ERR_OOM = 3,     /* device or host allocation failed */
  FWH_ERR_STATE = 4,   /* call out of order (e.g. forward before observers) */
  FWH_ERR_TIMEOUT = 5  /* a bounded device-side wait gave up */
} fwh_status;

enum { FWH_FP64 = 0, FWH_MIXED = 1 };
/* launch forms of batched calls (fwh_set_batch_options) */
enum { FWH_BATCH_PIPELINED = 0, FWH_BATCH_GRID = 1, FWH_BATCH_PERSISTENT = 2 };

/*
 * Create a handle for one permeable surface of n_panels subfaces
 * (the FWH_Surface_Geo.dat content of App. A2, as arrays):
 *   centroids [P][3]  subface centres y_i (double, row-major)
 *   normals   [P][3]  unit outward normals n_i (|n| = 1 within 1e-6)
 *   areas     [P]     subface areas dS (> 0)
 * mach  M0 = U0/c0 in (0, 1) (Eq. M0), aoa_rad the angle of attack in the
 * x-y plane (Eqs. d1_prime, d2_prime), c0 the nondimensional sound speed,
 * which must equal 1/M0 within 1e-12 relative (Sec. II D), dt > 0 the
 * nondimensional sampling interval, precision FWH_FP64 or FWH_MIXED
 * (mixed: FP32 fields and integrand arithmetic, FP64 arrival times and
 * interpolation weights, per-bin FP32 sums over one panel set at a time added
 * into FP64 output bins).
 * Errors: FWH_ERR_ARG on any invalid value (no handle is created),
 * FWH_ERR_OOM / FWH_ERR_CUDA on allocation or device failure.
 */
fwh_status fwh_create(fwh_handle *out, int64_t n_panels, const double *centroids,
                      const double *normals, const double *areas, double mach,
                      double aoa_rad, double c0, double dt, int precision);

/*
 * Set the observers (observers.dat of Sec. III A): xyz [O][3] doubles, host
 * or device.  Computes, once per geometry, the convected distance R and unit
 * radiation vector R-hat of every (panel, observer) pair (Eqs. R_New ..
 * R2_New), the per-observer R_max/R_min (the reductions the paper performs
 * with MPI_ALLREDUCE, Sec. III B "compute t"), the integrand coefficients of
 * Eqs. pT_WT_nd / pL_WT_nd and the arrival-time shift and spline weights, all
 * in FP64.  May be called again to replace the observer set.
 * Errors: FWH_ERR_ARG (n_obs < 1, null xyz, non-finite values).
 */
fwh_status fwh_set_observers(fwh_handle h, int64_t n_obs, const double *xyz);

/*
 * Panel sharding (the paper's Face partition, Sec. III A, with the
 * MPI_ALLREDUCE of R_max / R_min of Sec. III B "compute t"): a handle made on
 * one rank's subset of the subfaces reports, per observer, the largest and
 * smallest convected distance R over its own panels (host arrays [O]); the
 * ranks reduce them (maximum of r_max, minimum of r_min) and each sets the
 * global values on its handle.  Every rank then has the same observer window
 * (t_start = M0 R_max, Eq. t_start; N_o from Eq. t_end), its forward pass
 * yields its panels' share of p_out on that common grid, and a sum over the
 * ranks gives the unsharded result.  fwh_set_observer_extremes recomputes
 * the shifts and spline weights of the records and the panel-set plan; it
 * refuses (FWH_ERR_ARG) extremes that do not enclose the handle's own, and
 * fwh_set_observers restores the handle's own extremes.
 */
fwh_status fwh_observer_extremes(fwh_handle h, double *r_max, double *r_min);
fwh_status fwh_set_observer_extremes(fwh_handle h, const double *r_max, const double *r_min);

/*
 * Forward pass: far-field pressure p_out [O][nt] (double) from the fields
 * [nt][5][P] (double for FWH_FP64, float for FWH_MIXED), nt >= 3.
 * Covers the "compute Noise", "compute t", "interp pressure signal" and
 * surface-integration stages (Sec. III B, III C).  Host FWH_MIXED fields of
 * 256 frames or more are copied in 128-frame slabs on streams the handle owns,
 * overlapped with the preparation and scatter of the frames already copied;
 * the call still returns only when p_out holds the result.
 * Errors: FWH_ERR_STATE before fwh_set_observers, FWH_ERR_ARG for nt outside
 * [3, 2^28], null pointers, or (FWH_MIXED) n_panels x round_up(nt, 256) >= 2^32
 * (series rows are addressed with 32-bit indices; checked before any work, the
 * handle stays usable), FWH_ERR_CUDA / FWH_ERR_OOM on device failure, or the
 * deferred device check of an earlier call (see the conventions above).
 */
fwh_status fwh_forward(fwh_handle h, const void *fields, int64_t nt, double *p_out,
                       void *stream);

/*
 * Observer window for a record of nt frames: t_start [O] (Eq. t_start) and
 * n_valid [O] = N_o (from Eq. t_end).  Host pointers.
 */
fwh_status fwh_observer_window(fwh_handle h, int64_t nt, double *t_start,
                               int64_t *n_valid);

/*
 * Adjoint: given grad_p = dLoss/dp_out [O][nt] (double; entries j >= N_o are
 * ignored), write grad_fields = dLoss/dfields [nt][5][P] (same type as the
 * fields).  It is the exact transpose of fwh_forward's linear stages (spline
 * interpolation, finite differences, integrand coefficients) followed by the
 * Jacobian of the integrands of Eqs. Qn_New_nd / Li_New_nd at `fields`,
 * computed as a gather over observers (no atomics on the gradient).
 * Errors: as fwh_forward.
 */
fwh_status fwh_backward(fwh_handle h, const void *fields, int64_t nt,
                        const double *grad_p, void *grad_fields, void *stream);

/*
 * Batched forward over n handles (several uneven surfaces, each with its own
 * observers, fields, nt and p_out; the surface sum of Sec. III C over the
 * Faces of Sec. III A); all handles must share one precision and take device
 * buffers.  By default the series of every surface are kept for the whole
 * record.  With a ring set on hs[0] (fwh_set_batch_options), the record is
 * streamed instead in rounds of R time segments (512 samples each under the
 * default tile shape): each surface keeps the series of R segments only
 * (P x 512 R rows instead of P x round_up(nt, 256)).  The work items (panel
 * set x time segment x observer group) are scattered in the launch form set
 * on hs[0]: FWH_BATCH_PIPELINED (default) one launch per surface and round,
 * each surface's series prepared on a high-priority stream while the
 * surfaces before it scatter; FWH_BATCH_GRID one grid per round over every
 * surface's items; FWH_BATCH_PERSISTENT one persistent work-queue kernel per
 * round.  The whole sequence is captured once in a CUDA graph keyed on the
 * handle set and the options, and replayed on later calls with the same
 * arguments.  At most 32 surfaces.
 * Errors: FWH_ERR_ARG (n < 1 or > 32, mixed precisions, null entries),
 * FWH_ERR_STATE (a handle without observers), FWH_ERR_CUDA.
 */
fwh_status fwh_batch_forward(int n, const fwh_handle *hs, const void *const *fields,
                             const int64_t *nt, double *const *p_out, void *stream);

/*
 * Options of batched calls led by h (h = hs[0] of fwh_batch_forward).
 * ring_samples = 0 (the default) keeps every surface's series for its whole
 * record; ring_samples > 0 streams records longer than that through a ring
 * of max(1, floor(ring_samples / 512)) time segments of 512 samples (default
 * tile shape), 64 bytes (FP32) or 128 bytes (FP64) per panel and sample.
 * form: FWH_BATCH_PIPELINED, FWH_BATCH_GRID or FWH_BATCH_PERSISTENT (see
 * fwh_batch_forward).  On a GB300 the pipelined form is the fastest; the
 * single grid reads its per-surface arguments from a parameter block by
 * surface index (about 1 % slower per item), and the persistent kernel keeps
 * each CTA's warps on the same schedulers for the whole launch (about 3 %).
 * Results agree to the FP64 rounding of the output sums.
 * Errors: FWH_ERR_ARG for a negative ring length or an unknown form.
 */
fwh_status fwh_set_batch_options(fwh_handle h, int64_t ring_samples, int form);

/*
 * Pipelined forward passes (default off): with device fields and a record of
 * several time segments (512 samples under the default tile shape),
 * fwh_forward prepares the series of each segment on a high-priority stream
 * the handle owns and starts the scatter of a segment as soon as its series
 * are in, so the preparation of later segments runs under the scatter of
 * earlier ones; off, it prepares the whole record first and scatters it in
 * one launch.  Results agree to the FP64 rounding of the output sums.  On a
 * GB300 the pipelined call was slower for device-resident fields (the prep's
 * blocks take SM slots from the arithmetic-bound scatter, and each segment
 * launch has its own tail), hence the default; host fields are always
 * pipelined with their copies.
 */
fwh_status fwh_set_pipeline(fwh_handle h, int enable);

/*
 * Autotune: time the candidate tile shapes of the forward kernel on this
 * handle's geometry for a record of nt frames (synthetic zero fields; the
 * caller's data are not touched) and keep the fastest for later calls.
 * Writes the chosen configuration index to *chosen (may be NULL).
 */
fwh_status fwh_autotune(fwh_handle h, int64_t nt, int *chosen, void *stream);

/*
 * Force a forward tile configuration (index into the candidate table; -1
 * restores the default).  For benchmarking and tests.
 */
fwh_status fwh_set_tile_config(fwh_handle h, int config);

/*
 * Device times (milliseconds, CUDA events recorded on the launching stream,
 * never synchronised by the forward call itself) of fwh_forward calls made
 * while fwh_set_timing(h, 1) is on: [0] integrand preparation, [1] the
 * forward scatter kernel, [2] the whole call.  fwh_last_timings gives the
 * last call; fwh_timing_totals the sums over all timed calls since the last
 * reset and their count.  Both synchronise on the recorded events.  When a
 * FWH_MIXED call takes host fields of 256 frames or more, the copy, the
 * preparation and the scatter overlap in 128-frame slabs: [0] then runs to
 * the start of the first scatter launch and [1] from there to the end.
 */
fwh_status fwh_set_timing(fwh_handle h, int enable);
fwh_status fwh_last_timings(fwh_handle h, float *ms3);
fwh_status fwh_timing_totals(fwh_handle h, double *ms3, int64_t *calls, int reset);

/*
 * Synchronise `stream` and report the device-side checks raised by this
 * handle's kernels since the last check (a panel set whose arrival spread
 * exceeded its window -> FWH_ERR_CUDA; a bounded wait that gave up ->
 * FWH_ERR_TIMEOUT), then clear them.  Calls with host outputs run this check
 * themselves.
 */
fwh_status fwh_check(fwh_handle h, void *stream);

/*
 * Bound, in SM clock cycles, of each wait of the forward kernel's copy
 * pipeline (a compute warp waiting for its stage, the copy warp waiting for a
 * free one); 0 restores the default of 4e9 cycles (about 2 s).  A wait that
 * runs out raises FWH_ERR_TIMEOUT through the device check, the kernel stops
 * issuing copies, waits (always with the default bound) for those in flight
 * and returns; p_out of that call is then incomplete, and the handle stays
 * usable.  withhold_copies != 0 is for testing that error path: the copy
 * pipeline then issues no copies at all, so every stage wait runs out after
 * `cycles` (nothing is in flight when the kernel returns).
 * Errors: FWH_ERR_ARG for a negative bound.
 */
fwh_status fwh_set_wait_limit(fwh_handle h, int64_t cycles, int withhold_copies);

/*
 * Forward pass that allocates no device memory.  The paper has no
 * counterpart: this exists for callers that cannot call cudaMalloc/cudaFree
 * or any allocator while they run (a real-time loop with a memory budget
 * fixed up front, code embedded in a framework that owns the device memory
 * and forbids allocation during a step).  Results equal fwh_forward's.  The
 * handle must have been set up earlier (fwh_create and fwh_set_observers
 * allocate); fields and p_out must be device pointers (FWH_ERR_ARG
 * otherwise: there is no staging).  The call copies nothing from host memory
 * (observer windows are computed on the device, the series descriptor is a
 * kernel parameter) and writes no buffer of the handle besides its device
 * error flag: it reads the handle's panel-set plan, which fwh_set_observers,
 * fwh_set_tile_config and fwh_autotune leave in place for the configured tile
 * shape (FWH_ERR_STATE if a forward call on a huge record replaced it).
 * Scratch: the prepared series and per-call tables live in one file-scope
 * device array of 64 MiB that every GPU loading the library reserves until
 * the process exits; a problem needing more (about P x round_up(nt, 256) x
 * 64 bytes for FWH_MIXED, x 128 for FWH_FP64) is rejected with FWH_ERR_ARG
 * and a message giving both sizes.  The first call on each device looks up
 * the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  All calls on a
 * device share the array (each call writes everything it reads), so calls
 * whose GPU work overlaps race and must be serialised by the caller.
 */
fwh_status fwh_forward_noalloc(fwh_handle h, const void *fields, int64_t nt, double *p_out,
                               void *stream);

/*
 * Power spectral density of far-field signals (Sec. IV C): Welch's method
 * with segments of nperseg samples overlapping by 50 %, a periodic Hanning
 * window w[n] = 0.5 - 0.5 cos(2 pi n / nperseg) on each segment (its mean
 * removed first when detrend = 1), the squared magnitudes of the segments'
 * discrete Fourier transforms averaged over the K = floor((N - nperseg) /
 * (nperseg / 2)) + 1 segments of a signal's N valid samples, divided by
 * fs * sum(w^2) and doubled at 0 < k < nperseg / 2 (one-sided density), then
 * the span correction of Eq. PSD_corr: multiplied by span_ratio = b_exp / b_m,
 * and with p_ref > 0 returned in dB, 10 log10(PSD span_ratio / p_ref^2).
 * Arguments: p [n_sig][ld] doubles (host or device; row s holds signal s),
 * n_valid [n_sig] int64 (host or device; N of each signal, in [0, ld]; NULL:
 * every signal has ld samples -- for fwh_forward output pass the window of
 * fwh_observer_window), fs > 0 the sampling rate (1/dt for the observer
 * grid), nperseg a power of two in [16, 4096], psd [n_sig][nperseg/2 + 1]
 * doubles (host or device) at frequencies k fs / nperseg.  A signal shorter
 * than one segment gets NaN in every bin.  Computed in FP64, one CTA per
 * signal, on `stream`; host buffers are staged and the call then
 * synchronises.  Errors: FWH_ERR_ARG (sizes, ranges, null pointers),
 * FWH_ERR_OOM / FWH_ERR_CUDA (message via fwh_last_error(NULL)).
 */
fwh_status fwh_psd(int64_t n_sig, const double *p, int64_t ld, const int64_t *n_valid,
                   double fs, int64_t nperseg, int detrend, double span_ratio, double p_ref,
                   double *psd, void *stream);

/*
 * General moving surface (Sec. II B): the permeable-surface integrals of
 * Eqs. pT and pL (Farassat 1A) for panels moving in a medium at rest, FP64.
 * The wind-tunnel calls above are this form seen from the surface's frame
 * (Sec. II C); this entry point takes the motion itself.  Arguments:
 *   y, normals, velocities [nt][P][3]: centroid, unit normal and velocity of
 *     every panel at source time tau_i = i dt (host or device);
 *   areas [P]: panel areas (constant);
 *   c0, rho0: sound speed and density of the medium at rest; dt > 0;
 *   fields [nt][5][P]: rho', u_1, u_2, u_3 (fluid velocity in the medium's
 *     frame), p' (host or device);
 *   x0 [O][3], w [3]: observers at x0 + w t (w = 0: at rest; |w| < c0);
 *   p_out [O][nt] (host or device): p' at t_j = t_start + j dt for j < N_o,
 *     0 beyond; t_start, n_valid [O] (host, may be NULL).
 * Per (panel, observer, frame): r = c0 (t - tau) from the non-negative root of
 * |x0 + w t - y(tau)| = c0 (t - tau) (Eq. tau), r-hat, M = v / c0, M-dot by
 * second-order differences, Q_n = [rho0 v + rho (u - v)].n (Eq. Qn) and
 * L_i = p' n_i + rho u_i (u.n - v.n) (Eq. Li) with their source-time
 * derivatives, and the bracket of Eqs. pT + pL times dS / (4 pi).  Observer
 * window: t_start = max over panels of the first frame's arrival, t_end = min
 * of the last frame's, N_o = floor((t_end - t_start) / dt) + 1.  Each panel's
 * signal and arrival time are natural cubic splines over tau; bin j takes the
 * signal at the tau* whose arrival is t_j.  The motion must stay subsonic
 * (|M_r| < 1).  Device scratch of 32 nt P bytes per observer, up to
 * the budget of fwh_set_moving_scratch (16 GiB by default; observers are
 * split over launches that fit it, at least one observer per launch), is
 * taken with cudaMallocAsync on `stream`; the call synchronises.
 * Errors: FWH_ERR_ARG (sizes, |w| >= c0, non-positive c0, rho0, dt),
 * FWH_ERR_OOM / FWH_ERR_CUDA (message via fwh_last_error(NULL)).
 */
/*
 * Scratch budget in bytes of later fwh_forward_moving calls, process-wide
 * (0 restores the default of 16 GiB).  Smaller budgets split the observers
 * over more, smaller launches.  Errors: FWH_ERR_ARG for a negative budget.
 */
fwh_status fwh_set_moving_scratch(int64_t bytes);

fwh_status fwh_forward_moving(int64_t n_panels, int64_t nt, const double *y,
                              const double *normals, const double *velocities,
                              const double *areas, double c0, double rho0, double dt,
                              const double *fields, int64_t n_obs, const double *x0,
                              const double *w, double *p_out, double *t_start,
                              int64_t *n_valid, void *stream);

/*
 * Measured fused multiply-add throughput of the current GPU (TFLOP/s, 2 flop
 * per FMA): FP32 for FWH_MIXED, FP64 for FWH_FP64, from independent FMA
 * chains on every SM timed with CUDA events on `stream` (about 60 ms; the
 * call synchronises).  The forward scatter is bound by this rate, not by
 * memory or a dense contraction, so this is its measured roof.  Not part of
 * the paper's method.  Errors: FWH_ERR_ARG, FWH_ERR_CUDA (message via
 * fwh_last_error(NULL)).
 */
fwh_status fwh_fma_peak(int precision, double *tflops, void *stream);

/* Number of panels, observers and the precision of a handle. */
fwh_status fwh_get_sizes(fwh_handle h, int64_t *n_panels, int64_t *n_obs,
                         int *precision);

/* Destroy a handle and free its device memory (NULL is ignored). */
void fwh_destroy(fwh_handle h);

/* Message of the last failing call on h ("" if none); h may be NULL for
 * errors of fwh_create. The pointer stays valid until the next call. */
const char *fwh_last_error(fwh_handle h);

/* Library version string. */
const char *fwh_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FWH_H_ */
