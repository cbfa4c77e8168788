// Internal declarations of the GB300 FW-H library (not part of the C ABI).
//
// Data layout in HBM (P = panels in the library's spatial order, O =
// observers, ntp = nt rounded up to the forward chunk, T = float or double):
//   fields   [nt][5][P]      caller's pulsations (original panel order)
//   X        [P][ntp][16] T  per panel, per source sample: the eight
//                            observer-independent series
//                              0 Qn_dot 1 Qn 2..4 L_dot 5..7 L
//                            then their natural-spline moments (8..15);
//                            rows >= nt are zero.  FP32 X pairs samples j
//                            and j + 32 of every 64-sample block in one
//                            128-byte row, [ntp/64][32][16][2]
//   coef     [P][O][16] T    per (panel, observer) record (slots in
//                            namespace slot): the 8 integrand coefficients
//                            (same order as X), the interpolation weights
//                            a, b, cc, dd, the integer shift i0 and the
//                            window offset i0max(set) - i0 written by the
//                            planner; integers are bit patterns in FP32
//                            records, values in FP64 ones
//   p_out    [O][nt] double  caller's output
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fwh {

constexpr int kRec = 16;          // values per X row and per coef record

// Slots of a coefficient record (kRec values, both precisions).
namespace slot {
constexpr int c = 0;    // c0..c7: coefficients of the eight series
constexpr int a = 8, b = 9, cc = 10, dd = 11;  // interpolation weights
constexpr int i0 = 12;  // integer shift (bit pattern in FP32 records)
constexpr int off = 13; // window offset i0max(set) - i0, written by the planner
// FP32 records: byte offsets, in an observer's split window (slot x in half
// x & 1, word x >> 1), of the slots off + 1 and off + 2, written by the planner
constexpr int w0 = 14, w1 = 15;
}  // namespace slot
constexpr int kWarp = 32;

// Halo (samples) of the windowed natural-spline solves: the influence of a
// window edge decays as (2 - sqrt 3)^k, below 1e-18 for k = 32 and below
// 1e-9 (under FP32 rounding) for k = 16.
template <typename T> struct Prec;
template <> struct Prec<float> { static constexpr int halo = 16; };
template <> struct Prec<double> { static constexpr int halo = 32; };

constexpr int kPivTab = 64;       // 1/pivot of the tridiag(1,4,1) elimination

// Device error flags (bitmask written by kernels, read by the host).
enum : int {
  kErrWindow = 1,      // a panel set's arrival spread exceeded the window
  kErrTimeout = 2,     // a bounded wait gave up
  kErrQueue = 4,       // persistent queue inconsistency
};

struct GeomArgs {
  const double *y;      // [P][3] sorted centroids
  const double *n;      // [P][3] sorted normals
  const double *dS;     // [P]
  const double *x;      // [O][3]
  int P, O;
  double mach, ca, sa, dt;
  double *Rmax, *Rmin;  // [O]
};

template <typename T>
struct PrepArgs {
  const T *fields;      // [nt][5][P] original order
  const int *perm;      // [P] sorted position -> original panel index
  const double *n;      // [P][3] sorted normals
  T *X;                 // [P][x_ld][16]: sample k of panel p in row p x_ld + k mod x_ld
  int P, nt, ntp, chunk;
  int x_ld;             // X rows per panel: ntp, or a ring of whole time segments
  double ca, sa, dt;
  int c_lo, c_hi;       // 64-sample chunks [c_lo, c_hi) to prepare (0, 0: all)
  int int_lo, int_hi;   // FP32, set by the launcher: the interior chunks within [c_lo, c_hi)
};

template <typename T>
struct FwdArgs {
  const void *tmX;      // batched form: device CUtensorMap over X as [P*ntp rows][16]
                        // (single launches take the descriptor as a kernel parameter)
  const T *X;           // [P][x_ld][16] (sample k in row p x_ld + k mod x_ld)
  const T *coef;        // [P][O][16]
  double *p_out;        // [O][nt]
  const int *n_valid;   // [O]
  const int *set_begin; // [nsets + 1] panel-set boundaries (sorted order)
  const int *set_order; // [nsets] sets by descending panel count (null: index order)
  const int *i0max_tab; // [nsets][O] largest shift of each (panel set, observer)
  int *err;
  int nsets, O, ntp, nt;
  int x_ld;             // X rows per panel (ntp, or a ring of whole time segments)
  int obs_per_cta, n_obs_groups;
  int seg_len, n_segs;
  int seg_lo, seg_cnt;  // this launch covers time segments [seg_lo, seg_lo + seg_cnt)
  int win;              // window slots per observer
  int wfl;              // values per observer window: win, or 2 win for compensated
                        // FP32 windows (a sum and its compensation per slot)
  long long wait_cycles; // bound of each pipeline wait in SM clocks (the handle's limit)
  int withhold;         // testing: the copy pipeline issues no copies (every wait runs out)
};

// Surfaces in one batched call (their arguments sit in each CTA's shared memory).
constexpr int kMaxBatchSurf = 32;

template <typename T>
struct AdjArgs {
  const T *coef;        // [P][O][16]
  T *Gt;                // [O][ntp] workspace: grad_p in T, zero outside [0, N_o)
  const double *grad_p; // [O][nt]
  const int *n_valid;   // [O]
  T *Xbar;              // [P][ntp][16] gradient w.r.t. X
  int P, O, ntp, nt;
  // FP32 set form (win > 0): the forward plan of a 128-sample-chunk shape
  const int *set_begin; // [nsets + 1] panel-set boundaries (sorted order)
  const int *set_order; // [nsets] sets by descending panel count
  const int *i0max_tab; // [nsets][O] largest shift of each (panel set, observer)
  int nsets, win;       // win: window slots per observer (chunk + slack + 1)
};

template <typename T>
struct PrepAdjArgs {
  const T *fields;      // [nt][5][P] original order
  const int *perm;
  const double *n;      // [P][3] sorted normals
  const T *Xbar;        // [P][ntp][16]
  T *grad_fields;       // [nt][5][P] original order
  int P, nt, ntp, chunk;
  double ca, sa, dt;
};

// ---- launchers (defined in the .cu files) --------------------------------
cudaError_t launch_window(const GeomArgs &a, cudaStream_t s);
// N_o per observer (Eq. t_end) from R_max / R_min, rounded as the host does.
cudaError_t launch_nvalid(const double *Rmax, const double *Rmin, int O, double mach, double dt,
                          int nt, int *n_valid, cudaStream_t s);
template <typename T>
cudaError_t launch_coef(const GeomArgs &a, T *coef, cudaStream_t s);
cudaError_t upload_pivots(cudaStream_t s);
template <typename T>
cudaError_t launch_prep(const PrepArgs<T> &a, cudaStream_t s);
template <typename T>
cudaError_t launch_prep_adjoint(const PrepAdjArgs<T> &a, cudaStream_t s);
template <typename T>
cudaError_t launch_adjoint(const AdjArgs<T> &a, cudaStream_t s);

// Forward tile configurations (index into a table in fwh_forward.cu).
struct FwdConfig {
  int pipe;           // 0: direct loads, 1: TMA + mbarrier pipeline (producer warp),
                      // 2: TMA pipeline refilled by the last warp done with a stage
  int tk;             // source samples per lane per chunk (chunk = 32 tk)
  int warps;          // compute warps per CTA
  int obs_per_warp;   // max observers per warp
  int win;            // window slots per observer
  int seg_chunks;     // chunks per time segment
  int stages;         // pipeline stages (pipe = 1)
  int acc;            // 0: one sample per lane per block (FP64); FP32 consecutive sample
                      // pairs with split windows: 3 plain, 4 with the next record read
                      // ahead, 5 read ahead with compensated (Kahan) window sums
  int wide;           // 1: register cap 200 instead of the occupancy launch bound
};
// Bytes of dynamic shared memory a config needs for `obs_per_cta` observers.
size_t fwd_smem_bytes(bool fp64, const FwdConfig &c, int obs_per_cta);
// CTAs of the persistent batch kernel that fit on one SM for config `cfg`.
template <typename T>
cudaError_t forward_batch_occupancy(int cfg, int *per_sm);
// Encode the TMA descriptor of X ([rows][16] elements of 4 or 8 bytes) into a
// host buffer of 128 bytes; returns false if the driver refuses.
bool encode_x_tensor_map(void *out128, const void *X, unsigned long long rows, bool fp64,
                         int box_rows);
int fwd_num_configs(bool fp64);
FwdConfig fwd_config(bool fp64, int idx);
// tmap128: host copy of the X tensor map (128 bytes) for TMA configs, passed
// to the kernel as a parameter; may be null for direct-load configs.
template <typename T>
cudaError_t launch_forward(const FwdArgs<T> &a, const void *tmap128, int cfg_idx,
                           cudaStream_t s);
// Planner kernel: per (panel set, observer) the largest shift i0max into
// i0max_tab and, per record, the window offset i0max - i0 clamped to
// [0, slack] (slack = win - chunk - 1) into slot 13 and, for FP32 records,
// the split-window byte offsets of slots off + 1 and off + 2 into slots 14
// and 15 (half_bytes: bytes of one window half, slot_bytes: bytes per slot);
// a set whose shifts span more than slack raises kErrWindow.
template <typename T>
cudaError_t launch_plan(T *coef, const int *set_begin, int nsets, int O, int slack,
                        int half_bytes, int slot_bytes, int *i0max_tab, int *err,
                        cudaStream_t s);

// Batched persistent forward: the arguments of one launch, passed by value
// as a __grid_constant__ kernel parameter (under 9 KB at kMaxBatchSurf
// surfaces), so that the kernel reads them from the constant bank and hands
// the descriptors' parameter-space addresses to its tensor copies.
struct alignas(64) TmapBytes {
  unsigned char b[128];   // a CUtensorMap (encoded by encode_x_tensor_map)
};
template <typename T>
struct alignas(64) BatchParams {
  TmapBytes tm[kMaxBatchSurf];      // X descriptor of each surface
  FwdArgs<T> a[kMaxBatchSurf];      // arguments of each surface (tmX unused)
  int prefix[kMaxBatchSurf + 1];    // first work item of each surface; [n_surf] = total
  int n_surf, total;
};
template <typename T>
cudaError_t launch_forward_batch(const BatchParams<T> &params, int *d_counter, int cfg_idx,
                                 int n_ctas, cudaStream_t s);
// The same work items as one ordinary grid (one CTA per item, no queue).
template <typename T>
cudaError_t launch_forward_multi(const BatchParams<T> &params, int cfg_idx, cudaStream_t s);

}  // namespace fwh
