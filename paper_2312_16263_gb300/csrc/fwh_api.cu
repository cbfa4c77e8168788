// C ABI of the GB300 FW-H library: handles, the host planner, workspace,
// host/device staging, launches, timing and the batched graph path.
//
// Planner.  Panels are visited in the caller's order when that order is
// spatially coherent, else in Morton (Z-curve) order of their centroids.
// They are grouped into "panel sets" of up to kMaxSet consecutive panels
// whose arrival shifts, for every observer, span at most S samples, where
//   |i0(p1, o) - i0(p2, o)| <= M0 |R(p1, o) - R(p2, o)| / dt + 1
//                          <= M0 |y1 - y2| / ((1 - M0) dt) + 1
// because |grad_y R| = R / R* <= 1 / (1 - M0) (R, R* of Eqs. R_New,
// R_s_New).  The set's bounding-box diagonal bounds |y1 - y2|, so the bound
// needs no per-observer data and holds for any observer set.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/fwh.h"
#include "fwh_internal.cuh"

using namespace fwh;

namespace {

constexpr int kMaxSet = 64;

struct Buf {
  void *p = nullptr;
  size_t bytes = 0;
};

struct Graph {
  cudaGraphExec_t exec = nullptr;
  std::vector<uintptr_t> key;
};

// Plan of one batched call (lives with its graph): per round r (a run of
// consecutive time segments whose series are resident together), the launch
// parameters (every surface's FwdArgs, X descriptor and first work item).
struct BatchPlan {
  Buf counter;                 // [nr] work-queue counters
  std::vector<BatchParams<float>> pf;   // [nr] launch parameters (FP32 surfaces)
  std::vector<BatchParams<double>> pd;  // [nr] launch parameters (FP64 surfaces)
  std::vector<int> total;      // work items of each round's scatter launch
  std::vector<int> x_ld;       // X rows per panel of each surface (ring or whole record)
  std::vector<int> nseg;       // time segments of each surface
  int nq = 0;                  // time segments of the longest record
  int R = 0;                   // segments per round (nq: the whole record in one round)
  int nr = 0, ctas = 0, cfg = 0, seg = 0;
  int form = FWH_BATCH_PIPELINED;  // launch form (fwh_set_batch_options)
};

}  // namespace

struct fwh_ctx {
  int64_t P = 0, O = 0;
  double mach = 0, aoa = 0, dt = 0, ca = 1, sa = 0;
  int precision = FWH_FP64;
  std::vector<double> y, n, dS;  // library (planner) order
  std::vector<int> perm;          // library position -> caller index
  bool identity = true;
  std::vector<double> xobs;
  std::vector<double> Rmax, Rmin;            // window extremes in use (local or set)
  std::vector<double> Rmax_loc, Rmin_loc;    // over this handle's own panels
  // device state
  double *d_y = nullptr, *d_n = nullptr, *d_dS = nullptr, *d_x = nullptr;
  double *d_Rmax = nullptr, *d_Rmin = nullptr;
  int *d_perm = nullptr, *d_err = nullptr;
  Buf coef, X, G, nvalid, sets, sord, stage_in, stage_out, stage_grad, imax;
  // X tensor map (passed to single launches as a kernel parameter; batched
  // calls keep device copies in their plans)
  alignas(64) unsigned char tmap_host[128] = {};
  const void *tmap_X = nullptr;  // X buffer / rows / box the host descriptor describes
  int tmap_box = 0;
  long long tmap_rows = 0;
  long long wait_limit = 0;      // bound of the forward pipeline waits (0: default)
  int withhold = 0;              // testing: the forward pipeline issues no copies
  bool pipeline = false;         // device fields: prep of later segments overlaps the scatter
  int64_t batch_ring = 0;        // batched calls led by this handle: source samples of
                                 // series kept per surface (0: the whole record)
  int batch_form = FWH_BATCH_PIPELINED;  // ... and their launch form
  // deferred device check: each call with device outputs copies the error flag
  // into pinned host memory; the next call (or fwh_check) reads it
  int *h_err = nullptr;
  cudaEvent_t err_ev = nullptr;
  bool err_pending = false;
  // per-nt
  int64_t nt = -1;
  int ntp = 0;
  std::vector<int> h_nvalid;
  std::vector<double> h_tstart;
  // planner
  int plan_win = -1, plan_ch = -1, plan_sb = -1;
  std::vector<int> set_begin;
  int cfg = -1;  // forced/tuned forward config (-1 default)
  bool timing = false;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  float last_ms[3] = {0, 0, 0};
  // timing pool: one (start, after-prep, end) triple per timed call
  std::vector<cudaEvent_t> pool;
  size_t pool_used = 0;
  double sum_ms[3] = {0, 0, 0};
  int64_t sum_calls = 0;
  std::string err;
  // batch
  std::map<std::vector<uintptr_t>, Graph> graphs;
  std::map<std::vector<uintptr_t>, BatchPlan> bplans;
  cudaStream_t side = nullptr;
  cudaStream_t copy = nullptr;              // host-field slabs (fwh_forward)
  cudaStream_t pstream = nullptr;           // their series prep
  cudaStream_t bstream = nullptr;           // second scatter lane of pipelined batches
  std::vector<cudaEvent_t> slab_ev;         // per slab: copied, prepared; plus the start
  cudaEvent_t bev[2] = {nullptr, nullptr};
};

namespace {

std::mutex g_err_mu;
std::string g_err;  // errors without a handle

fwh_status fail(fwh_handle h, fwh_status st, const std::string &msg) {
  if (h) {
    h->err = msg;
  } else {
    std::lock_guard<std::mutex> lk(g_err_mu);
    g_err = msg;
  }
  return st;
}

fwh_status cuda_fail(fwh_handle h, cudaError_t e, const char *what) {
  return fail(h, e == cudaErrorMemoryAllocation ? FWH_ERR_OOM : FWH_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(h, expr)                                   \
  do {                                                \
    cudaError_t e_ = (expr);                          \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #expr); \
  } while (0)

cudaError_t ensure(Buf &b, size_t bytes) {
  if (b.bytes >= bytes && b.p) return cudaSuccess;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  if (bytes == 0) return cudaSuccess;
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e == cudaSuccess) b.bytes = bytes;
  return e;
}

void release(Buf &b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

size_t tsize(int precision) { return precision == FWH_FP64 ? sizeof(double) : sizeof(float); }

uint64_t spread_bits(uint64_t v) {  // 21-bit -> every third bit
  v &= 0x1fffff;
  v = (v | v << 32) & 0x1f00000000ffffULL;
  v = (v | v << 16) & 0x1f0000ff0000ffULL;
  v = (v | v << 8) & 0x100f00f00f00f00fULL;
  v = (v | v << 4) & 0x10c30c30c30c30c3ULL;
  v = (v | v << 2) & 0x1249249249249249ULL;
  return v;
}

// Greedy panel sets over `order`; returns set boundaries (positions).
std::vector<int> build_sets(const std::vector<double> &y, int64_t P, double mach, double dt,
                            int smax) {
  const double k = mach / ((1.0 - mach) * dt);
  std::vector<int> b{0};
  double lo[3], hi[3];
  int cnt = 0;
  for (int64_t p = 0; p < P; ++p) {
    const double *q = &y[3 * p];
    if (cnt == 0) {
      for (int c = 0; c < 3; ++c) lo[c] = hi[c] = q[c];
      cnt = 1;
      continue;
    }
    double nlo[3], nhi[3], d2 = 0;
    for (int c = 0; c < 3; ++c) {
      nlo[c] = std::min(lo[c], q[c]);
      nhi[c] = std::max(hi[c], q[c]);
      d2 += (nhi[c] - nlo[c]) * (nhi[c] - nlo[c]);
    }
    const double bound = k * std::sqrt(d2) + 1.0;
    if (cnt >= kMaxSet || bound > (double)smax) {
      b.push_back((int)p);
      for (int c = 0; c < 3; ++c) lo[c] = hi[c] = q[c];
      cnt = 1;
    } else {
      std::memcpy(lo, nlo, sizeof lo);
      std::memcpy(hi, nhi, sizeof hi);
      ++cnt;
    }
  }
  b.push_back((int)P);
  return b;
}

int default_cfg(const fwh_ctx *h) {
  (void)h;
  return 0;
}

// Observer tiling for a config: observers per warp and groups.
void obs_tiling(const fwh_ctx *h, const FwdConfig &c, int *obs_per_cta, int *groups) {
  int opw = (int)std::min<int64_t>(c.obs_per_warp, (h->O + c.warps - 1) / c.warps);
  if (opw < 1) opw = 1;
  *obs_per_cta = opw * c.warps;
  *groups = (int)((h->O + *obs_per_cta - 1) / *obs_per_cta);
}

// Panel sets for a config, and the plan kernel's per-(set, observer) shift
// table and per-record window offsets, enqueued on `s`.
fwh_status plan(fwh_handle h, const FwdConfig &c, cudaStream_t s) {
  const int ch = 32 * c.tk;
  const int sb = c.acc == 5 ? 8 : 4;  // bytes per FP32 window slot (sum, or sum + compensation)
  if (h->plan_win == c.win && h->plan_ch == ch && h->plan_sb == sb) return FWH_OK;
  const int smax = c.win - ch - 1;
  h->set_begin = build_sets(h->y, h->P, h->mach, h->dt, smax);
  const size_t bytes = h->set_begin.size() * sizeof(int);
  const int nsets = (int)h->set_begin.size() - 1;
  CK(h, ensure(h->sets, bytes));
  CK(h, cudaMemcpy(h->sets.p, h->set_begin.data(), bytes, cudaMemcpyHostToDevice));
  {  // work order: sets by descending panel count
    std::vector<int> ord(nsets);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
      return h->set_begin[x + 1] - h->set_begin[x] > h->set_begin[y + 1] - h->set_begin[y];
    });
    CK(h, ensure(h->sord, ord.size() * sizeof(int)));
    CK(h, cudaMemcpy(h->sord.p, ord.data(), ord.size() * sizeof(int), cudaMemcpyHostToDevice));
  }
  CK(h, ensure(h->imax, (size_t)nsets * h->O * sizeof(int)));
  if (h->precision == FWH_FP64)
    CK(h, launch_plan<double>(reinterpret_cast<double *>(h->coef.p),
                              reinterpret_cast<const int *>(h->sets.p), nsets, (int)h->O, smax,
                              0, 0, reinterpret_cast<int *>(h->imax.p), h->d_err, s));
  else
    CK(h, launch_plan<float>(reinterpret_cast<float *>(h->coef.p),
                             reinterpret_cast<const int *>(h->sets.p), nsets, (int)h->O, smax,
                             (c.win / 2) * sb, sb,
                             reinterpret_cast<int *>(h->imax.p), h->d_err, s));
  h->plan_win = c.win;
  h->plan_ch = ch;
  h->plan_sb = sb;
  return FWH_OK;
}

// Per-nt window and workspace.  ntp is a multiple of 256, hence of every
// forward chunk (32 x TK samples) and prep chunk.
constexpr int64_t kMaxNt = (int64_t)1 << 28;

fwh_status prepare_window(fwh_handle h, int64_t nt) {
  if (nt < 3 || nt > kMaxNt)
    return fail(h, FWH_ERR_ARG, "nt must be in [3, 2^28] (got " + std::to_string(nt) + ")");
  if (h->precision == FWH_MIXED && h->P * ((nt + 255) / 256 * 256) >= ((int64_t)1 << 32))
    return fail(h, FWH_ERR_ARG, "panels x padded steps must stay below 2^32 per handle");
  if (h->nt != nt) {
    h->h_nvalid.assign(h->O, 0);
    h->h_tstart.assign(h->O, 0.0);
    const double tau_max = (double)(nt - 1) * h->dt;
    for (int64_t o = 0; o < h->O; ++o) {
      const double ts = h->mach * h->Rmax[o];                // Eq. t_start
      const double te = tau_max + h->mach * h->Rmin[o];      // Eq. t_end
      double nv = std::floor((te - ts) / h->dt) + 1.0;
      nv = std::max(0.0, std::min((double)nt, nv));
      h->h_nvalid[o] = (int)nv;
      h->h_tstart[o] = ts;
    }
    CK(h, ensure(h->nvalid, h->O * sizeof(int)));
    CK(h, cudaMemcpy(h->nvalid.p, h->h_nvalid.data(), h->O * sizeof(int),
                     cudaMemcpyHostToDevice));
    const int64_t ntp = (nt + 255) / 256 * 256;  // a multiple of every chunk length
    h->nt = nt;
    h->ntp = (int)ntp;
  }
  return FWH_OK;
}

// Window and the whole-record series buffer X.
fwh_status prepare_nt(fwh_handle h, int64_t nt) {
  fwh_status st = prepare_window(h, nt);
  if (st != FWH_OK) return st;
  const size_t ts = tsize(h->precision);
  CK(h, ensure(h->X, (size_t)h->P * h->ntp * kRec * ts));
  return FWH_OK;
}

// Config actually used: TMA configs address X rows with 32-bit coordinates
// (FP64 falls back to a direct-load shape; every FP32 shape is a TMA shape,
// its rows are sample pairs, and prepare_nt bounds P x ntp below 2^32).
int effective_cfg(const fwh_ctx *h, int64_t ntp) {
  const bool fp64 = h->precision == FWH_FP64;
  int cfg = h->cfg >= 0 ? h->cfg : default_cfg(h);
  if (fwd_config(fp64, cfg).pipe != 0 && h->P * ntp >= ((int64_t)1 << 31)) {
    for (int i = 0; i < fwd_num_configs(fp64); ++i)
      if (fwd_config(fp64, i).pipe == 0) return i;
  }
  return cfg;
}

// Panel-set plan of the handle's configured tile shape, made at set-up
// (fwh_set_observers, fwh_set_tile_config, fwh_autotune), so that calls which
// must not allocate or copy from the host find it in place.
fwh_status plan_default(fwh_handle h) {
  const FwdConfig c = fwd_config(h->precision == FWH_FP64, h->cfg >= 0 ? h->cfg : default_cfg(h));
  fwh_status st = plan(h, c, 0);
  if (st != FWH_OK) return st;
  CK(h, cudaStreamSynchronize(0));
  return FWH_OK;
}

// TMA descriptor of the handle's X buffer, kept on the host (re-encoded when
// the buffer, its row count or the box changes).
fwh_status ensure_tmap(fwh_handle h, int box_rows, int x_ld = 0) {
  const long long rows = (long long)h->P * (x_ld > 0 ? x_ld : h->ntp);
  if (h->tmap_X == h->X.p && h->tmap_rows == rows && h->tmap_box == box_rows) return FWH_OK;
  if (!encode_x_tensor_map(h->tmap_host, h->X.p, (unsigned long long)rows,
                           h->precision == FWH_FP64, box_rows))
    return fail(h, FWH_ERR_CUDA, "cuTensorMapEncodeTiled refused the series layout");
  h->tmap_X = h->X.p;
  h->tmap_rows = rows;
  h->tmap_box = box_rows;
  return FWH_OK;
}


// The handle's high-priority stream for the series prep of pipelined calls.
fwh_status ensure_pstream(fwh_handle h) {
  if (h->pstream) return FWH_OK;
  int least = 0, greatest = 0;
  CK(h, cudaDeviceGetStreamPriorityRange(&least, &greatest));
  CK(h, cudaStreamCreateWithPriority(&h->pstream, cudaStreamNonBlocking, greatest));
  return FWH_OK;
}

// At least n ordering events (no timing) in the handle's pool.
fwh_status ensure_events(fwh_handle h, int n) {
  while ((int)h->slab_ev.size() < n) {
    cudaEvent_t e;
    CK(h, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    h->slab_ev.push_back(e);
  }
  return FWH_OK;
}

// Host fields of a mixed handle are copied in slabs of kSlab source frames; the
// series of slab q are prepared as soon as slab q + 1 (which holds the filters'
// reach beyond it) has landed, and the forward scatter runs in segments of two
// chunks, each as soon as its rows are prepared, so copy, prep and scatter
// overlap and only the last slab's prep and segment follow the last copy.
constexpr int kSlab = 128;

template <typename T>
fwh_status run_forward(fwh_handle h, const T *d_fields, double *d_pout, cudaStream_t s,
                       const T *host_fields = nullptr) {
  const bool fp64 = sizeof(T) == 8;
  const int cfg = effective_cfg(h, h->ntp);
  const FwdConfig c = fwd_config(fp64, cfg);
  if (c.pipe != 0) {
    fwh_status st0 = ensure_tmap(h, 32 * c.tk);
    if (st0 != FWH_OK) return st0;
  }
  fwh_status st = plan(h, c, s);
  if (st != FWH_OK) return st;
  cudaEvent_t *tev = nullptr;
  if (h->timing) {
    if (h->pool_used + 3 > h->pool.size()) {
      for (int i = 0; i < 3 * 64; ++i) {
        cudaEvent_t e;
        CK(h, cudaEventCreate(&e));
        h->pool.push_back(e);
      }
    }
    tev = &h->pool[h->pool_used];
    h->pool_used += 3;
    CK(h, cudaEventRecord(tev[0], s));
  }
  CK(h, cudaMemsetAsync(d_pout, 0, (size_t)h->O * h->nt * sizeof(double), s));
  PrepArgs<T> pa{};
  pa.fields = d_fields;
  pa.perm = h->identity ? nullptr : h->d_perm;
  pa.n = h->d_n;
  pa.X = reinterpret_cast<T *>(h->X.p);
  pa.P = (int)h->P;
  pa.nt = (int)h->nt;
  pa.ntp = h->ntp;
  pa.ca = h->ca;
  pa.sa = h->sa;
  pa.dt = h->dt;
  pa.x_ld = h->ntp;
  FwdArgs<T> fa{};
  fa.tmX = nullptr;
  fa.wait_cycles = h->wait_limit;
  fa.withhold = h->withhold;
  fa.x_ld = h->ntp;
  fa.X = pa.X;
  fa.coef = reinterpret_cast<const T *>(h->coef.p);
  fa.p_out = d_pout;
  fa.n_valid = reinterpret_cast<const int *>(h->nvalid.p);
  fa.set_begin = reinterpret_cast<const int *>(h->sets.p);
  fa.set_order = reinterpret_cast<const int *>(h->sord.p);
  fa.i0max_tab = reinterpret_cast<const int *>(h->imax.p);
  fa.err = h->d_err;
  fa.nsets = (int)h->set_begin.size() - 1;
  fa.O = (int)h->O;
  fa.ntp = h->ntp;
  fa.nt = (int)h->nt;
  obs_tiling(h, c, &fa.obs_per_cta, &fa.n_obs_groups);
  fa.seg_len = c.seg_chunks * 32 * c.tk;
  fa.n_segs = (h->ntp + fa.seg_len - 1) / fa.seg_len;
  fa.seg_lo = 0;
  fa.seg_cnt = fa.n_segs;
  fa.win = c.win;
  fa.wfl = c.win * (c.acc == 5 ? 2 : 1);
  if (host_fields == nullptr && (!h->pipeline || fa.n_segs < 2)) {
    CK(h, launch_prep<T>(pa, s));
    if (tev) CK(h, cudaEventRecord(tev[1], s));
    CK(h, launch_forward<T>(fa, c.pipe ? h->tmap_host : nullptr, cfg, s));
  } else if (host_fields == nullptr) {
    // Device fields, several time segments: the series of segment q are
    // prepared on the high-priority prep stream and the scatter of segment q
    // starts as soon as they are in, so the preparation of the later segments
    // runs under the scatter of the earlier ones.  The prep stream first waits
    // for the work already on `s` (the previous call's scatter reads X).
    fwh_status st1 = ensure_pstream(h);
    if (st1 != FWH_OK) return st1;
    st1 = ensure_events(h, fa.n_segs + 1);
    if (st1 != FWH_OK) return st1;
    cudaEvent_t *ev_x = h->slab_ev.data(), ev_go = ev_x[fa.n_segs];
    CK(h, cudaEventRecord(ev_go, s));
    CK(h, cudaStreamWaitEvent(h->pstream, ev_go, 0));
    const int cps = fa.seg_len / 64;  // 64-sample prep chunks per segment
    for (int q = 0; q < fa.n_segs; ++q) {
      pa.c_lo = q * cps;
      pa.c_hi = std::min(h->ntp / 64, (q + 1) * cps);
      CK(h, launch_prep<T>(pa, h->pstream));
      CK(h, cudaEventRecord(ev_x[q], h->pstream));
    }
    for (int q = 0; q < fa.n_segs; ++q) {
      CK(h, cudaStreamWaitEvent(s, ev_x[q], 0));
      if (tev && q == 0) CK(h, cudaEventRecord(tev[1], s));
      fa.seg_lo = q;
      fa.seg_cnt = 1;
      CK(h, launch_forward<T>(fa, c.pipe ? h->tmap_host : nullptr, cfg, s));
    }
  } else {
    // Three streams: `copy` moves the slabs, `prep` (high priority, so that
    // its blocks get onto SMs between the scatter's) prepares slab q - 1 once
    // slab q is in (the filters reach 83 frames past a slab), and `s` scatters
    // each two-chunk time segment once all its rows are prepared.
    // The copy stream first waits for the work already on `s` (the previous
    // call's scatter reads X and its prep the staging buffer), so every later
    // step of this call is ordered after it.
    const int nslab = (int)((h->nt + kSlab - 1) / kSlab);
    const size_t row = (size_t)5 * h->P * sizeof(T);
    if (!h->copy) CK(h, cudaStreamCreateWithFlags(&h->copy, cudaStreamNonBlocking));
    fwh_status st1 = ensure_pstream(h);
    if (st1 != FWH_OK) return st1;
    fa.seg_len = 2 * 32 * c.tk;
    fa.n_segs = (h->ntp + fa.seg_len - 1) / fa.seg_len;
    st1 = ensure_events(h, 2 * nslab + 1);
    if (st1 != FWH_OK) return st1;
    cudaEvent_t *ev_in = h->slab_ev.data(), *ev_x = ev_in + nslab, ev_go = ev_in[2 * nslab];
    CK(h, cudaEventRecord(ev_go, s));
    CK(h, cudaStreamWaitEvent(h->copy, ev_go, 0));
    constexpr int cps = kSlab / 64;  // 64-sample prep chunks per slab
    static_assert(kSlab % 64 == 0 && 256 % kSlab == 0, "slabs tile the padded record");
    int seg_done = 0;
    // scatter the segments whose rows lie below rows_ready (prepared by slab j)
    auto scatter_upto = [&](int rows_ready, int j) -> fwh_status {
      const int ready = rows_ready >= h->ntp ? fa.n_segs : rows_ready / fa.seg_len;
      if (ready <= seg_done) return FWH_OK;
      CK(h, cudaStreamWaitEvent(s, ev_x[j], 0));
      if (tev && seg_done == 0) CK(h, cudaEventRecord(tev[1], s));
      fa.seg_lo = seg_done;
      fa.seg_cnt = ready - seg_done;
      CK(h, launch_forward<T>(fa, c.pipe ? h->tmap_host : nullptr, cfg, s));
      seg_done = ready;
      return FWH_OK;
    };
    for (int q = 0; q <= nslab; ++q) {
      if (q < nslab) {
        const int64_t r0 = (int64_t)q * kSlab, r1 = std::min<int64_t>(h->nt, r0 + kSlab);
        CK(h, cudaMemcpyAsync(const_cast<T *>(d_fields) + r0 * 5 * h->P,
                              host_fields + r0 * 5 * h->P, (size_t)(r1 - r0) * row,
                              cudaMemcpyHostToDevice, h->copy));
        CK(h, cudaEventRecord(ev_in[q], h->copy));
      }
      if (q == 0) continue;
      const int j = q - 1;  // slab to prepare
      CK(h, cudaStreamWaitEvent(h->pstream, ev_in[std::min(q, nslab - 1)], 0));
      pa.c_lo = j * cps;
      pa.c_hi = q < nslab ? q * cps : h->ntp / 64;
      CK(h, launch_prep<T>(pa, h->pstream));
      CK(h, cudaEventRecord(ev_x[j], h->pstream));
      const fwh_status st2 = scatter_upto(pa.c_hi * 64, j);
      if (st2 != FWH_OK) return st2;
    }
  }
  if (tev) CK(h, cudaEventRecord(tev[2], s));
  return FWH_OK;
}

void drop_graphs(fwh_handle h) {
  for (auto &kv : h->graphs)
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  h->graphs.clear();
  for (auto &kv : h->bplans) release(kv.second.counter);
  h->bplans.clear();
}

// Resolve every recorded timing triple (synchronising on the last one).
fwh_status drain_timings(fwh_handle h) {
  for (size_t i = 0; i + 3 <= h->pool_used; i += 3) {
    cudaEvent_t *t = &h->pool[i];
    CK(h, cudaEventSynchronize(t[2]));
    float a = 0, b = 0, c = 0;
    CK(h, cudaEventElapsedTime(&a, t[0], t[1]));
    CK(h, cudaEventElapsedTime(&b, t[1], t[2]));
    CK(h, cudaEventElapsedTime(&c, t[0], t[2]));
    h->last_ms[0] = a;
    h->last_ms[1] = b;
    h->last_ms[2] = c;
    h->sum_ms[0] += a;
    h->sum_ms[1] += b;
    h->sum_ms[2] += c;
    h->sum_calls += 1;
  }
  h->pool_used = 0;
  return FWH_OK;
}

// Status and message of a nonzero device flag.
fwh_status flag_failure(fwh_handle h, int flag, const char *when) {
  std::string m = when;
  if (flag & kErrTimeout) m += ": a bounded device-side wait gave up";
  if (flag & kErrWindow) m += ": a panel set's arrival spread exceeded its window";
  if (flag & kErrQueue) m += ": the persistent work queue was inconsistent";
  return fail(h, (flag & kErrTimeout) ? FWH_ERR_TIMEOUT : FWH_ERR_CUDA,
              m + " (device flags " + std::to_string(flag) + ")");
}

// Synchronous check: wait for `s` and read (and clear) the device flag.
fwh_status check_device_flag(fwh_handle h, cudaStream_t s) {
  int flag = 0;
  CK(h, cudaMemcpyAsync(&flag, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(h, cudaStreamSynchronize(s));
  h->err_pending = false;
  if (flag) {
    CK(h, cudaMemsetAsync(h->d_err, 0, sizeof(int), s));
    CK(h, cudaStreamSynchronize(s));
    return flag_failure(h, flag, "device check");
  }
  return FWH_OK;
}

// After a call whose outputs stay on the device: copy the flag into pinned
// host memory behind the call's work, so that a later call can report it
// without waiting.
fwh_status defer_check(fwh_handle h, cudaStream_t s) {
  CK(h, cudaMemcpyAsync(h->h_err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(h, cudaEventRecord(h->err_ev, s));
  h->err_pending = true;
  return FWH_OK;
}

// At the start of a call: report a failure of an earlier call whose flag copy
// has completed (never waits; a copy still in flight is looked at later).
fwh_status take_deferred(fwh_handle h) {
  if (!h->err_pending) return FWH_OK;
  const cudaError_t q = cudaEventQuery(h->err_ev);
  if (q == cudaErrorNotReady) {
    cudaGetLastError();
    return FWH_OK;
  }
  if (q != cudaSuccess) return cuda_fail(h, q, "cudaEventQuery");
  h->err_pending = false;
  const int flag = *h->h_err;
  if (!flag) return FWH_OK;
  *h->h_err = 0;
  CK(h, cudaMemset(h->d_err, 0, sizeof(int)));
  CK(h, cudaDeviceSynchronize());
  return flag_failure(h, flag, "an earlier call on this handle");
}

}  // namespace

extern "C" {

const char *fwh_version(void) { return "fwh-gb300 1.0 (sm_103a)"; }

const char *fwh_last_error(fwh_handle h) {
  if (h) return h->err.c_str();
  std::lock_guard<std::mutex> lk(g_err_mu);
  return g_err.c_str();
}

fwh_status fwh_create(fwh_handle *out, int64_t P, const double *centroids,
                      const double *normals, const double *areas, double mach, double aoa,
                      double c0, double dt, int precision) {
  if (!out) return fail(nullptr, FWH_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (P < 1 || P > (int64_t)1 << 30) return fail(nullptr, FWH_ERR_ARG, "n_panels out of range");
  if (!centroids || !normals || !areas)
    return fail(nullptr, FWH_ERR_ARG, "geometry pointer is NULL");
  if (!(mach > 0.0 && mach < 1.0)) return fail(nullptr, FWH_ERR_ARG, "mach must be in (0, 1)");
  if (!(std::fabs(c0 * mach - 1.0) <= 1e-12))
    return fail(nullptr, FWH_ERR_ARG, "c0 must equal 1/mach (nondimensional sound speed)");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(nullptr, FWH_ERR_ARG, "dt must be > 0");
  if (!std::isfinite(aoa)) return fail(nullptr, FWH_ERR_ARG, "aoa must be finite");
  if (precision != FWH_FP64 && precision != FWH_MIXED)
    return fail(nullptr, FWH_ERR_ARG, "precision must be FWH_FP64 or FWH_MIXED");
  // geometry may be host or device memory
  std::vector<double> y(3 * P), n(3 * P), dS(P);
  auto fetch = [&](std::vector<double> &dst, const double *src, size_t cnt) -> bool {
    if (is_device_ptr(src))
      return cudaMemcpy(dst.data(), src, cnt * sizeof(double), cudaMemcpyDeviceToHost) ==
             cudaSuccess;
    std::memcpy(dst.data(), src, cnt * sizeof(double));
    return true;
  };
  if (!fetch(y, centroids, 3 * P) || !fetch(n, normals, 3 * P) || !fetch(dS, areas, P))
    return fail(nullptr, FWH_ERR_CUDA, "cannot read geometry");
  for (int64_t p = 0; p < P; ++p) {
    const double nn = n[3 * p] * n[3 * p] + n[3 * p + 1] * n[3 * p + 1] + n[3 * p + 2] * n[3 * p + 2];
    if (!(std::fabs(std::sqrt(nn) - 1.0) <= 1e-6))
      return fail(nullptr, FWH_ERR_ARG, "normal " + std::to_string(p) + " is not unit length");
    if (!(dS[p] > 0.0) || !std::isfinite(dS[p]))
      return fail(nullptr, FWH_ERR_ARG, "area " + std::to_string(p) + " must be > 0");
    for (int c = 0; c < 3; ++c)
      if (!std::isfinite(y[3 * p + c]))
        return fail(nullptr, FWH_ERR_ARG, "centroid " + std::to_string(p) + " not finite");
  }
  fwh_ctx *h = new (std::nothrow) fwh_ctx();
  if (!h) return fail(nullptr, FWH_ERR_OOM, "host allocation failed");
  h->P = P;
  h->mach = mach;
  h->aoa = aoa;
  h->dt = dt;
  h->ca = std::cos(aoa);
  h->sa = std::sin(aoa);
  h->precision = precision;

  // planner order: the caller's order unless a Morton order packs the
  // arrival spreads much better (decided with the default window).
  const FwdConfig c0cfg = fwd_config(precision == FWH_FP64, 0);
  const int smax = c0cfg.win - 32 * c0cfg.tk - 1;
  std::vector<int> sets_id = build_sets(y, P, mach, dt, smax);
  const double avg_id = (double)P / (double)(sets_id.size() - 1);
  std::vector<int> order(P);
  std::iota(order.begin(), order.end(), 0);
  if (avg_id < 24.0 && P > kMaxSet) {
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t p = 0; p < P; ++p)
      for (int c = 0; c < 3; ++c) {
        lo[c] = std::min(lo[c], y[3 * p + c]);
        hi[c] = std::max(hi[c], y[3 * p + c]);
      }
    double ext = std::max({hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2], 1e-300});
    std::vector<uint64_t> key(P);
    for (int64_t p = 0; p < P; ++p) {
      uint64_t q[3];
      for (int c = 0; c < 3; ++c)
        q[c] = (uint64_t)std::min(2097151.0, std::floor((y[3 * p + c] - lo[c]) / ext * 2097151.0));
      key[p] = spread_bits(q[0]) | spread_bits(q[1]) << 1 | spread_bits(q[2]) << 2;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return key[a] < key[b]; });
    std::vector<double> ys(3 * P);
    for (int64_t p = 0; p < P; ++p)
      for (int c = 0; c < 3; ++c) ys[3 * p + c] = y[3 * order[p] + c];
    std::vector<int> sets_m = build_sets(ys, P, mach, dt, smax);
    const double avg_m = (double)P / (double)(sets_m.size() - 1);
    if (avg_m < 1.5 * avg_id) std::iota(order.begin(), order.end(), 0);
  }
  h->perm = order;
  h->identity = true;
  for (int64_t p = 0; p < P; ++p) h->identity = h->identity && order[p] == p;
  h->y.resize(3 * P);
  h->n.resize(3 * P);
  h->dS.resize(P);
  for (int64_t p = 0; p < P; ++p) {
    for (int c = 0; c < 3; ++c) {
      h->y[3 * p + c] = y[3 * order[p] + c];
      h->n[3 * p + c] = n[3 * order[p] + c];
    }
    h->dS[p] = dS[order[p]];
  }
  cudaError_t e;
  if ((e = cudaMalloc(&h->d_y, 3 * P * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&h->d_n, 3 * P * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&h->d_dS, P * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&h->d_perm, P * sizeof(int))) != cudaSuccess ||
      (e = cudaMalloc(&h->d_err, sizeof(int))) != cudaSuccess ||
      (e = cudaMemcpy(h->d_y, h->y.data(), 3 * P * sizeof(double), cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (e = cudaMemcpy(h->d_n, h->n.data(), 3 * P * sizeof(double), cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (e = cudaMemcpy(h->d_dS, h->dS.data(), P * sizeof(double), cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (e = cudaMemcpy(h->d_perm, h->perm.data(), P * sizeof(int), cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (e = cudaMemset(h->d_err, 0, sizeof(int))) != cudaSuccess ||
      (e = upload_pivots(0)) != cudaSuccess) {
    fwh_destroy(h);
    return cuda_fail(nullptr, e, "fwh_create device setup");
  }
  for (int i = 0; i < 4; ++i)
    if ((e = cudaEventCreate(&h->ev[i])) != cudaSuccess) {
      fwh_destroy(h);
      return cuda_fail(nullptr, e, "cudaEventCreate");
    }
  if ((e = cudaHostAlloc(&h->h_err, sizeof(int), cudaHostAllocDefault)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&h->err_ev, cudaEventDisableTiming)) != cudaSuccess) {
    fwh_destroy(h);
    return cuda_fail(nullptr, e, "fwh_create error-flag setup");
  }
  *h->h_err = 0;
  *out = h;
  return FWH_OK;
}

fwh_status fwh_set_observers(fwh_handle h, int64_t O, const double *xyz) {
  if (!h) return fail(nullptr, FWH_ERR_ARG, "handle is NULL");
  if (O < 1 || O > 65535) return fail(h, FWH_ERR_ARG, "n_obs must be in [1, 65535]");
  if (!xyz) return fail(h, FWH_ERR_ARG, "xyz is NULL");
  std::vector<double> x(3 * O);
  if (is_device_ptr(xyz)) {
    CK(h, cudaMemcpy(x.data(), xyz, 3 * O * sizeof(double), cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(x.data(), xyz, 3 * O * sizeof(double));
  }
  for (double v : x)
    if (!std::isfinite(v)) return fail(h, FWH_ERR_ARG, "observer coordinates must be finite");
  if (h->d_x) cudaFree(h->d_x);
  h->d_x = nullptr;
  if (h->d_Rmax) cudaFree(h->d_Rmax);
  if (h->d_Rmin) cudaFree(h->d_Rmin);
  h->d_Rmax = h->d_Rmin = nullptr;
  h->O = 0;
  CK(h, cudaMalloc(&h->d_x, 3 * O * sizeof(double)));
  CK(h, cudaMalloc(&h->d_Rmax, O * sizeof(double)));
  CK(h, cudaMalloc(&h->d_Rmin, O * sizeof(double)));
  CK(h, cudaMemcpy(h->d_x, x.data(), 3 * O * sizeof(double), cudaMemcpyHostToDevice));
  const size_t ts = tsize(h->precision);
  CK(h, ensure(h->coef, (size_t)h->P * O * kRec * ts));
  GeomArgs g{};
  g.y = h->d_y;
  g.n = h->d_n;
  g.dS = h->d_dS;
  g.x = h->d_x;
  g.P = (int)h->P;
  g.O = (int)O;
  g.mach = h->mach;
  g.ca = h->ca;
  g.sa = h->sa;
  g.dt = h->dt;
  g.Rmax = h->d_Rmax;
  g.Rmin = h->d_Rmin;
  CK(h, launch_window(g, 0));
  if (h->precision == FWH_FP64)
    CK(h, launch_coef<double>(g, reinterpret_cast<double *>(h->coef.p), 0));
  else
    CK(h, launch_coef<float>(g, reinterpret_cast<float *>(h->coef.p), 0));
  h->Rmax.resize(O);
  h->Rmin.resize(O);
  CK(h, cudaMemcpy(h->Rmax.data(), h->d_Rmax, O * sizeof(double), cudaMemcpyDeviceToHost));
  CK(h, cudaMemcpy(h->Rmin.data(), h->d_Rmin, O * sizeof(double), cudaMemcpyDeviceToHost));
  h->Rmax_loc = h->Rmax;
  h->Rmin_loc = h->Rmin;
  h->xobs = x;
  h->O = O;
  h->nt = -1;         // window depends on the observers
  h->plan_win = -1;   // records were rewritten: window offsets must be re-planned
  h->plan_sb = -1;
  drop_graphs(h);
  return plan_default(h);
}

fwh_status fwh_observer_extremes(fwh_handle h, double *r_max, double *r_min) {
  if (!h) return fail(nullptr, FWH_ERR_ARG, "handle is NULL");
  if (h->O < 1) return fail(h, FWH_ERR_STATE, "observers not set");
  for (int64_t o = 0; o < h->O; ++o) {
    if (r_max) r_max[o] = h->Rmax_loc[o];
    if (r_min) r_min[o] = h->Rmin_loc[o];
  }
  return FWH_OK;
}

fwh_status fwh_set_observer_extremes(fwh_handle h, const double *r_max, const double *r_min) {
  if (!h) return fail(nullptr, FWH_ERR_ARG, "handle is NULL");
  if (h->O < 1) return fail(h, FWH_ERR_STATE, "observers not set");
  if (!r_max || !r_min) return fail(h, FWH_ERR_ARG, "r_max or r_min is NULL");
  for (int64_t o = 0; o < h->O; ++o) {
    if (!std::isfinite(r_max[o]) || !std::isfinite(r_min[o]))
      return fail(h, FWH_ERR_ARG, "extremes must be finite");
    if (r_max[o] < h->Rmax_loc[o] || r_min[o] > h->Rmin_loc[o])
      return fail(h, FWH_ERR_ARG,
                  "observer " + std::to_string(o) +
                      ": the extremes must enclose this handle's own (r_max >= its largest R, "
                      "r_min <= its smallest)");
  }
  std::vector<double> mx(r_max, r_max + h->O), mn(r_min, r_min + h->O);
  CK(h, cudaMemcpy(h->d_Rmax, mx.data(), h->O * sizeof(double), cudaMemcpyHostToDevice));
  CK(h, cudaMemcpy(h->d_Rmin, mn.data(), h->O * sizeof(double), cudaMemcpyHostToDevice));
  GeomArgs g{};
  g.y = h->d_y;
  g.n = h->d_n;
  g.dS = h->d_dS;
  g.x = h->d_x;
  g.P = (int)h->P;
  g.O = (int)h->O;
  g.mach = h->mach;
  g.ca = h->ca;
  g.sa = h->sa;
  g.dt = h->dt;
  g.Rmax = h->d_Rmax;
  g.Rmin = h->d_Rmin;
  // records: shifts and spline weights relative to the new t_start (Eq. t_start)
  if (h->precision == FWH_FP64)
    CK(h, launch_coef<double>(g, reinterpret_cast<double *>(h->coef.p), 0));
  else
    CK(h, launch_coef<float>(g, reinterpret_cast<float *>(h->coef.p), 0));
  h->Rmax = mx;
  h->Rmin = mn;
  h->nt = -1;
  h->plan_win = -1;
  drop_graphs(h);
  return plan_default(h);
}

fwh_status fwh_observer_window(fwh_handle h, int64_t nt, double *t_start, int64_t *n_valid) {
  if (!h) return fail(nullptr, FWH_ERR_ARG, "handle is NULL");
  if (h->O < 1) return fail(h, FWH_ERR_STATE, "observers not set");
  fwh_status st = prepare_nt(h, nt);
  if (st != FWH_OK) return st;
  for (int64_t o = 0; o < h->O; ++o) {
    if (t_start) t_start[o] = h->h_tstart[o];
    if (n_valid) n_valid[o] = h->h_nvalid[o];
  }
  return FWH_OK;
}

fwh_status fwh_forward(fwh_handle h, const void *fields, int64_t nt, double *p_out,
                       void *stream) {
  if (!h) return fail(nullptr, FWH_ERR_ARG, "handle is NULL");
  if (h->O < 1) return fail(h, FWH_ERR_STATE, "fwh_set_observers must come first");
  if (!fields || !p_out) return fail(h, FWH_ERR_ARG, "fields or p_out is NULL");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  fwh_status st = take_deferred(h);
  if (st != FWH_OK) return st;
  st = prepare_nt(h, nt);
  if (st != FWH_OK) return st;
  const size_t ts = tsize(h->precision);
  const size_t fbytes = (size_t)nt * 5 * h->P * ts;
  const size_t obytes = (size_t)h->O * nt * sizeof(double);
  const bool din = is_device_ptr(fields), dout = is_device_ptr(p_out);
  const void *df = fields;
  double *dp = p_out;
  // mixed handles overlap the copy of host fields with the series prep
  const bool slabs = !din && h->precision == FWH_MIXED && nt >= 2 * kSlab;
  if (!din) {
    CK(h, ensure(h->stage_in, fbytes));
    if (!slabs)
      CK(h, cudaMemcpyAsync(h->stage_in.p, fields, fbytes, cudaMemcpyHostToDevice, s));
    df = h->stage_in.p;
  }
  if (!dout) {
    CK(h, ensure(h->stage_out, obytes));
    dp = reinterpret_cast<double *>(h->stage_out.p);
  }
  st = h->precision == FWH_FP64
           ? run_forward<double>(h, reinterpret_cast<const double *>(df), dp, s)
           : run_forward<float>(h, reinterpret_cast<const float *>(df), dp, s,
                                slabs ? reinterpret_cast<const float *>(fields) : nullptr);
  if (st != FWH_OK) return st;
  if (!dout) {
    CK(h, cudaMemcpyAsync(p_out, dp, obytes, cudaMemcpyDeviceToHost, s));
    return check_device_flag(h, s);
  }
  return defer_check(h, s);
}

fwh_status fwh_backward(fwh_handle h, const void *fields, int64_t nt, const double *grad_p,
                        void *grad_fields, void *stream) {
  if (!h) return fail(nullptr, FWH_ERR_ARG, "handle is NULL");
  if (h->O < 1) return fail(h, FWH_ERR_STATE, "fwh_set_observers must come first");
  if (!fields || !grad_p || !grad_fields)
    return fail(h, FWH_ERR_ARG, "fields, grad_p or grad_fields is NULL");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  fwh_status st = take_deferred(h);
  if (st != FWH_OK) return st;
  st = prepare_nt(h, nt);
  if (st != FWH_OK) return st;
  const size_t ts = tsize(h->precision);
  const size_t fbytes = (size_t)nt * 5 * h->P * ts;
  const size_t gbytes = (size_t)h->O * nt * sizeof(double);
  const void *df = fields;
  const double *dg = grad_p;
  void *dgf = grad_fields;
  const bool dout = is_device_ptr(grad_fields);
  if (!is_device_ptr(fields)) {
    CK(h, ensure(h->stage_in, fbytes));
    CK(h, cudaMemcpyAsync(h->stage_in.p, fields, fbytes, cudaMemcpyHostToDevice, s));
    df = h->stage_in.p;
  }
  if (!is_device_ptr(grad_p)) {
    CK(h, ensure(h->stage_out, gbytes));
    CK(h, cudaMemcpyAsync(h->stage_out.p, grad_p, gbytes, cudaMemcpyHostToDevice, s));
    dg = reinterpret_cast<const double *>(h->stage_out.p);
  }
  if (!dout) {
    CK(h, ensure(h->stage_grad, fbytes));
    dgf = h->stage_grad.p;
  }
  CK(h, ensure(h->G, (size_t)h->O * h->ntp * ts));
  if (h->precision == FWH_FP64) {
    AdjArgs<double> aa{reinterpret_cast<const double *>(h->coef.p),
                       reinterpret_cast<double *>(h->G.p), dg,
                       reinterpret_cast<const int *>(h->nvalid.p),
                       reinterpret_cast<double *>(h->X.p), (int)h->P, (int)h->O, h->ntp,
                       (int)nt};
    CK(h, launch_adjoint<double>(aa, s));
    PrepAdjArgs<double> pa{reinterpret_cast<const double *>(df),
                           h->identity ? nullptr : h->d_perm, h->d_n,
                           reinterpret_cast<const double *>(h->X.p),
                           reinterpret_cast<double *>(dgf), (int)h->P, (int)nt, h->ntp, 0,
                           h->ca, h->sa, h->dt};
    CK(h, launch_prep_adjoint<double>(pa, s));
  } else {
    AdjArgs<float> aa{reinterpret_cast<const float *>(h->coef.p),
                      reinterpret_cast<float *>(h->G.p), dg,
                      reinterpret_cast<const int *>(h->nvalid.p),
                      reinterpret_cast<float *>(h->X.p), (int)h->P, (int)h->O, h->ntp, (int)nt};
    // the set form gathers with the forward's plan (panel sets and each
    // record's window offset) of a 128-sample-chunk tile shape
    const FwdConfig c = fwd_config(false, effective_cfg(h, h->ntp));
    if (32 * c.tk == 128) {
      st = plan(h, c, s);
      if (st != FWH_OK) return st;
      aa.set_begin = reinterpret_cast<const int *>(h->sets.p);
      aa.set_order = reinterpret_cast<const int *>(h->sord.p);
      aa.i0max_tab = reinterpret_cast<const int *>(h->imax.p);
      aa.nsets = (int)h->set_begin.size() - 1;
      aa.win = c.win;
    }
    CK(h, launch_adjoint<float>(aa, s));
    PrepAdjArgs<float> pa{reinterpret_cast<const float *>(df),
                          h->identity ? nullptr : h->d_perm, h->d_n,
                          reinterpret_cast<const float *>(h->X.p),
                          reinterpret_cast<float *>(dgf), (int)h->P, (int)nt, h->ntp, 0,
                          h->ca, h->sa, h->dt};
    CK(h, launch_prep_adjoint<float>(pa, s));
  }
  if (!dout) {
    CK(h, cudaMemcpyAsync(grad_fields, dgf, fbytes, cudaMemcpyDeviceToHost, s));
    return check_device_flag(h, s);
  }
  return defer_check(h, s);
}

fwh_status fwh_set_tile_config(fwh_handle h, int config) {
  if (!h) return fail(nullptr, FWH_ERR_ARG, "handle is NULL");
  if (config < -1 || config >= fwd_num_configs(h->precision == FWH_FP64))
    return fail(h, FWH_ERR_ARG, "tile config out of range");
  h->cfg = config;
  drop_graphs(h);
  return h->O >= 1 ? plan_default(h) : FWH_OK;
}

fwh_status fwh_autotune(fwh_handle h, int64_t nt, int *chosen, void *stream) {
  if (!h) return fail(nullptr, FWH_ERR_ARG, "handle is NULL");
  if (h->O < 1) return fail(h, FWH_ERR_STATE, "fwh_set_observers must come first");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  fwh_status st = prepare_nt(h, nt);
  if (st != FWH_OK) return st;
  const size_t ts = tsize(h->precision);
  Buf f, po;
  CK(h, ensure(f, (size_t)nt * 5 * h->P * ts));
  CK(h, ensure(po, (size_t)h->O * nt * sizeof(double)));
  CK(h, cudaMemsetAsync(f.p, 0, f.bytes, s));
  const bool was = h->timing;
  const int old = h->cfg;
  h->timing = true;
  float best = 1e30f;
  int besti = 0;
  const int n = fwd_num_configs(h->precision == FWH_FP64);
  for (int i = 0; i < n; ++i) {
    h->cfg = i;
    float tot = 0;
    for (int rep = 0; rep < 3; ++rep) {
      st = h->precision == FWH_FP64
               ? run_forward<double>(h, reinterpret_cast<const double *>(f.p),
                                     reinterpret_cast<double *>(po.p), s)
               : run_forward<float>(h, reinterpret_cast<const float *>(f.p),
                                    reinterpret_cast<double *>(po.p), s);
      if (st != FWH_OK) break;
      st = drain_timings(h);
      if (st != FWH_OK) break;
      if (rep > 0) tot += h->last_ms[1];
    }
    if (st != FWH_OK) {
      h->err.clear();
      continue;
    }
    if (tot < best) {
      best = tot;
      besti = i;
    }
  }
  release(f);
  release(po);
  h->timing = was;
  h->cfg = besti;
  (void)old;
  if (chosen) *chosen = besti;
  drop_graphs(h);
  return plan_default(h);
}

fwh_status fwh_set_wait_limit(fwh_handle h, int64_t cycles, int withhold_copies) {
  if (!h) return fail(nullptr, FWH_ERR_ARG, "handle is NULL");
  if (cycles < 0) return fail(h, FWH_ERR_ARG, "wait limit must be >= 0");
  h->wait_limit = cycles;
  h->withhold = withhold_copies != 0;
  drop_graphs(h);
  return FWH_OK;
}

fwh_status fwh_set_pipeline(fwh_handle h, int enable) {
  if (!h) return fail(nullptr, FWH_ERR_ARG, "handle is NULL");
  h->pipeline = enable != 0;
  return FWH_OK;
}

fwh_status fwh_set_batch_options(fwh_handle h, int64_t ring_samples, int form) {
  if (!h) return fail(nullptr, FWH_ERR_ARG, "handle is NULL");
  if (ring_samples < 0) return fail(h, FWH_ERR_ARG, "ring length must be >= 0 samples");
  if (form != FWH_BATCH_PIPELINED && form != FWH_BATCH_GRID && form != FWH_BATCH_PERSISTENT)
    return fail(h, FWH_ERR_ARG, "unknown batched launch form");
  h->batch_ring = ring_samples;
  h->batch_form = form;
  return FWH_OK;
}

fwh_status fwh_set_timing(fwh_handle h, int enable) {
  if (!h) return fail(nullptr, FWH_ERR_ARG, "handle is NULL");
  h->timing = enable != 0;
  return FWH_OK;
}

fwh_status fwh_last_timings(fwh_handle h, float *ms3) {
  if (!h || !ms3) return fail(h, FWH_ERR_ARG, "NULL argument");
  fwh_status st = drain_timings(h);
  if (st != FWH_OK) return st;
  for (int i = 0; i < 3; ++i) ms3[i] = h->last_ms[i];
  return FWH_OK;
}

fwh_status fwh_timing_totals(fwh_handle h, double *ms3, int64_t *calls, int reset) {
  if (!h || !ms3) return fail(h, FWH_ERR_ARG, "NULL argument");
  fwh_status st = drain_timings(h);
  if (st != FWH_OK) return st;
  for (int i = 0; i < 3; ++i) ms3[i] = h->sum_ms[i];
  if (calls) *calls = h->sum_calls;
  if (reset) {
    h->sum_ms[0] = h->sum_ms[1] = h->sum_ms[2] = 0;
    h->sum_calls = 0;
  }
  return FWH_OK;
}

fwh_status fwh_get_sizes(fwh_handle h, int64_t *P, int64_t *O, int *precision) {
  if (!h) return fail(nullptr, FWH_ERR_ARG, "handle is NULL");
  if (P) *P = h->P;
  if (O) *O = h->O;
  if (precision) *precision = h->precision;
  return FWH_OK;
}

void fwh_destroy(fwh_handle h) {
  if (!h) return;
  for (auto &kv : h->graphs)
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  for (auto &kv : h->bplans) release(kv.second.counter);
  for (double *p : {h->d_y, h->d_n, h->d_dS, h->d_x, h->d_Rmax, h->d_Rmin})
    if (p) cudaFree(p);
  if (h->d_perm) cudaFree(h->d_perm);
  if (h->d_err) cudaFree(h->d_err);
  for (Buf *b : {&h->coef, &h->X, &h->G, &h->nvalid, &h->sets, &h->sord, &h->stage_in,
                 &h->stage_out,
                 &h->stage_grad, &h->imax})
    release(*b);
  for (int i = 0; i < 4; ++i)
    if (h->ev[i]) cudaEventDestroy(h->ev[i]);
  for (cudaEvent_t e : h->pool) cudaEventDestroy(e);
  for (int i = 0; i < 2; ++i)
    if (h->bev[i]) cudaEventDestroy(h->bev[i]);
  if (h->err_ev) cudaEventDestroy(h->err_ev);
  if (h->h_err) cudaFreeHost(h->h_err);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->copy) cudaStreamDestroy(h->copy);
  if (h->pstream) cudaStreamDestroy(h->pstream);
  if (h->bstream) cudaStreamDestroy(h->bstream);
  for (cudaEvent_t e : h->slab_ev) cudaEventDestroy(e);
  delete h;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched forward: several surfaces in one graph-captured call.
// Host-side planning (the launch parameter blocks) happens once per argument
// set; the device work (output clears, integrand prep of every surface,
// scatter launches) is captured in a CUDA graph and replayed.
//
// The record is cut into rounds of R consecutive time segments.  By default
// one round holds the whole record; with a ring (fwh_set_batch_options), X
// keeps R segments per surface and each round prepares and scatters its
// segments.  Within a round the work items run in the order (surface, panel
// set, segment, observer group), so the CTAs in flight at any moment share a
// few panel sets' coefficient records and X rows in L2.  A round's scatter is
// one launch per surface (FWH_BATCH_PIPELINED, the default), one grid with a
// CTA per item over every surface (FWH_BATCH_GRID), or the persistent
// work-queue kernel with one CTA per SM slot (FWH_BATCH_PERSISTENT).
// ---------------------------------------------------------------------------
namespace {

// Tile configuration of a batched call (one for all surfaces).
int batch_cfg(int n, const fwh_handle *hs, fwh_handle h0) {
  const bool fp64 = h0->precision == FWH_FP64;
  int cfg = h0->cfg >= 0 ? h0->cfg : default_cfg(h0);
  for (int i = 0; i < n; ++i) {
    const int ci = effective_cfg(hs[i], hs[i]->ntp);
    if (fwd_config(fp64, ci).pipe != fwd_config(fp64, cfg).pipe) cfg = ci;
  }
  return cfg;
}

template <typename T> std::vector<BatchParams<T>> &batch_params(BatchPlan &bp);
template <> std::vector<BatchParams<float>> &batch_params<float>(BatchPlan &bp) { return bp.pf; }
template <> std::vector<BatchParams<double>> &batch_params<double>(BatchPlan &bp) { return bp.pd; }
template <typename T> const std::vector<BatchParams<T>> &batch_params(const BatchPlan &bp) {
  return batch_params<T>(const_cast<BatchPlan &>(bp));
}

// Segments per round of a batched call led by h0 (0: the whole record).
int batch_round_segs(const fwh_ctx *h0, int seg) {
  return h0->batch_ring > 0 ? (int)std::max<int64_t>(1, h0->batch_ring / seg) : 0;
}

// X rows per panel of a surface in a batched call: the whole record, or a
// ring of R time segments when the record spans more than R of them.
int batch_x_ld(const fwh_ctx *h, int seg, int R) {
  return R > 0 && (h->ntp + seg - 1) / seg > R ? R * seg : h->ntp;
}

template <typename T>
fwh_status batch_build(int n, const fwh_handle *hs, double *const *p_out, fwh_handle h0,
                       BatchPlan &bp) {
  const bool fp64 = sizeof(T) == 8;
  const int cfg = batch_cfg(n, hs, h0);
  const FwdConfig c = fwd_config(fp64, cfg);
  const int seg = c.seg_chunks * 32 * c.tk;
  const int R0 = batch_round_segs(h0, seg);
  std::vector<FwdArgs<T>> base(n);
  std::vector<TmapBytes> maps(n);
  bp.x_ld.assign(n, 0);
  bp.nseg.assign(n, 0);
  bp.nq = 0;
  for (int i = 0; i < n; ++i) {
    fwh_handle h = hs[i];
    fwh_status st = plan(h, c, h0->side);
    if (st != FWH_OK) return fail(h0, st, h->err);
    CK(h0, cudaStreamSynchronize(h0->side));
    bp.nseg[i] = (h->ntp + seg - 1) / seg;
    bp.x_ld[i] = batch_x_ld(h, seg, R0);
    bp.nq = std::max(bp.nq, bp.nseg[i]);
    if (h->X.bytes < (size_t)h->P * bp.x_ld[i] * kRec * sizeof(T))
      return fail(h0, FWH_ERR_STATE, "series buffer of a batched surface is too small");
    std::memset(maps[i].b, 0, sizeof maps[i].b);
    if (c.pipe != 0 &&
        !encode_x_tensor_map(maps[i].b, h->X.p, (unsigned long long)h->P * bp.x_ld[i], fp64,
                             32 * c.tk))
      return fail(h0, FWH_ERR_CUDA, "cuTensorMapEncodeTiled refused the series layout");
    FwdArgs<T> &fa = base[i];
    fa.tmX = nullptr;  // the launch passes the descriptors in its parameter block
    fa.wait_cycles = h0->wait_limit;
    fa.withhold = h0->withhold;
    fa.X = reinterpret_cast<const T *>(h->X.p);
    fa.x_ld = bp.x_ld[i];
    fa.coef = reinterpret_cast<const T *>(h->coef.p);
    fa.p_out = p_out[i];
    fa.n_valid = reinterpret_cast<const int *>(h->nvalid.p);
    fa.set_begin = reinterpret_cast<const int *>(h->sets.p);
    fa.set_order = reinterpret_cast<const int *>(h->sord.p);
    fa.i0max_tab = reinterpret_cast<const int *>(h->imax.p);
    fa.err = h0->d_err;
    fa.nsets = (int)h->set_begin.size() - 1;
    fa.O = (int)h->O;
    fa.ntp = h->ntp;
    fa.nt = (int)h->nt;
    obs_tiling(h, c, &fa.obs_per_cta, &fa.n_obs_groups);
    fa.seg_len = seg;
    fa.n_segs = bp.nseg[i];
    fa.win = c.win;
    fa.wfl = c.win * (c.acc == 5 ? 2 : 1);
  }
  // one scatter launch per round over every surface's items of it
  bp.R = R0 > 0 ? std::min(R0, bp.nq) : bp.nq;
  bp.nr = (bp.nq + bp.R - 1) / bp.R;
  std::vector<BatchParams<T>> &prm = batch_params<T>(bp);
  prm.assign(bp.nr, BatchParams<T>{});
  bp.total.assign(bp.nr, 0);
  for (int r = 0; r < bp.nr; ++r) {
    BatchParams<T> &P = prm[r];
    P.n_surf = n;
    P.prefix[0] = 0;
    for (int i = 0; i < n; ++i) {
      FwdArgs<T> fa = base[i];
      const int cnt = std::min(bp.nseg[i], (r + 1) * bp.R) - r * bp.R;
      const bool has = cnt > 0;
      fa.seg_lo = has ? r * bp.R : 0;
      fa.seg_cnt = has ? cnt : 1;
      P.a[i] = fa;
      P.tm[i] = maps[i];
      P.prefix[i + 1] = P.prefix[i] + (has ? fa.nsets * fa.n_obs_groups * cnt : 0);
    }
    P.total = P.prefix[n];
    bp.total[r] = P.total;
  }
  bp.seg = seg;
  bp.cfg = cfg;
  bp.form = h0->batch_form;
  CK(h0, ensure(bp.counter, (size_t)bp.nr * sizeof(int)));
  int dev = 0, sms = 0;
  CK(h0, cudaGetDevice(&dev));
  CK(h0, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int per_sm = 0;
  CK(h0, forward_batch_occupancy<T>(cfg, &per_sm));
  bp.ctas = sms * std::max(1, per_sm);
  return FWH_OK;
}

// The batched call's device work, enqueued on `s` (captured into a graph).
// Per round r: the series prep of every surface's segments of r and the
// scatter of their items.  FWH_BATCH_GRID / FWH_BATCH_PERSISTENT: the preps
// on `s`, then one launch over all surfaces' items; with a ring, the prep of
// round r overwrites the rows the scatter of round r - 1 read, so the rounds
// run strictly one after the other.  FWH_BATCH_PIPELINED: one scatter launch
// per (round, surface), each after its own prep, which runs on the handle's
// high-priority stream; the preps of the other surfaces overlap the scatters
// before them (a prep whose ring rows are still being read waits for that
// surface's scatter of the previous round).
template <typename T>
fwh_status batch_prep(const fwh_handle h, const void *field, const BatchPlan &bp, int i, int r,
                      fwh_handle h0, cudaStream_t s) {
  const int cps = bp.seg / 64;
  PrepArgs<T> pa{};
  pa.fields = reinterpret_cast<const T *>(field);
  pa.perm = h->identity ? nullptr : h->d_perm;
  pa.n = h->d_n;
  pa.X = reinterpret_cast<T *>(h->X.p);
  pa.P = (int)h->P;
  pa.nt = (int)h->nt;
  pa.ntp = h->ntp;
  pa.x_ld = bp.x_ld[i];
  pa.ca = h->ca;
  pa.sa = h->sa;
  pa.dt = h->dt;
  pa.c_lo = r * bp.R * cps;
  pa.c_hi = std::min(h->ntp / 64, (r + 1) * bp.R * cps);
  CK(h0, launch_prep<T>(pa, s));
  return FWH_OK;
}

template <typename T>
fwh_status batch_enqueue(int n, const fwh_handle *hs, const void *const *fields,
                         double *const *p_out, fwh_handle h0, const BatchPlan &bp,
                         cudaStream_t s) {
  for (int i = 0; i < n; ++i)
    CK(h0, cudaMemsetAsync(p_out[i], 0, (size_t)hs[i]->O * hs[i]->nt * sizeof(double), s));
  CK(h0, cudaMemsetAsync(bp.counter.p, 0, (size_t)bp.nr * sizeof(int), s));
  const std::vector<BatchParams<T>> &prm = batch_params<T>(bp);
  if (bp.form != FWH_BATCH_PIPELINED) {
    for (int r = 0; r < bp.nr; ++r) {
      for (int i = 0; i < n; ++i) {
        if (r * bp.R >= bp.nseg[i]) continue;
        fwh_status st = batch_prep<T>(hs[i], fields[i], bp, i, r, h0, s);
        if (st != FWH_OK) return st;
      }
      if (bp.total[r] == 0) continue;
      if (bp.form == FWH_BATCH_PERSISTENT)
        CK(h0, launch_forward_batch<T>(prm[r], reinterpret_cast<int *>(bp.counter.p) + r, bp.cfg,
                                       std::min(bp.ctas, bp.total[r]), s));
      else
        CK(h0, launch_forward_multi<T>(prm[r], bp.cfg, s));
    }
    return FWH_OK;
  }
  fwh_status st = ensure_pstream(h0);
  if (st == FWH_OK) st = ensure_events(h0, 2 + 2 * bp.nr * n);
  if (st != FWH_OK) return st;
  if (!h0->bstream) CK(h0, cudaStreamCreateWithFlags(&h0->bstream, cudaStreamNonBlocking));
  cudaEvent_t *ev = h0->slab_ev.data();  // [0] fork, [1] join, prep and scatter events per (r, i)
  cudaEvent_t *ev_prep = ev + 2, *ev_scat = ev + 2 + bp.nr * n;
  CK(h0, cudaEventRecord(ev[0], s));
  CK(h0, cudaStreamWaitEvent(h0->pstream, ev[0], 0));
  CK(h0, cudaStreamWaitEvent(h0->bstream, ev[0], 0));
  // surfaces in ascending size, so that only the smallest one's prep runs
  // before any scatter; the scatters alternate between two streams, so one
  // surface's tail overlaps the next surface's start
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return hs[x]->P * (int64_t)hs[x]->ntp < hs[y]->P * (int64_t)hs[y]->ntp;
  });
  cudaStream_t lane[2] = {s, h0->bstream};
  int k = 0;
  const bool ring = bp.nr > 1;
  const FwdConfig c = fwd_config(sizeof(T) == 8, bp.cfg);
  for (int r = 0; r < bp.nr; ++r) {
    for (int i : order) {
      if (r * bp.R >= bp.nseg[i]) continue;
      if (ring && r > 0) CK(h0, cudaStreamWaitEvent(h0->pstream, ev_scat[(r - 1) * n + i], 0));
      st = batch_prep<T>(hs[i], fields[i], bp, i, r, h0, h0->pstream);
      if (st != FWH_OK) return st;
      CK(h0, cudaEventRecord(ev_prep[r * n + i], h0->pstream));
    }
    for (int i : order) {
      if (r * bp.R >= bp.nseg[i]) continue;
      cudaStream_t ls = lane[k++ & 1];
      CK(h0, cudaStreamWaitEvent(ls, ev_prep[r * n + i], 0));
      CK(h0, launch_forward<T>(prm[r].a[i], c.pipe ? prm[r].tm[i].b : nullptr, bp.cfg, ls));
      CK(h0, cudaEventRecord(ev_scat[r * n + i], ls));
    }
  }
  // join: every prep precedes a scatter, and the second lane joins `s`
  CK(h0, cudaEventRecord(ev[1], h0->bstream));
  CK(h0, cudaStreamWaitEvent(s, ev[1], 0));
  return FWH_OK;
}

}  // namespace

extern "C" fwh_status fwh_batch_forward(int n, const fwh_handle *hs, const void *const *fields,
                                        const int64_t *nt, double *const *p_out,
                                        void *stream) {
  if (n < 1 || !hs || !fields || !nt || !p_out)
    return fail(nullptr, FWH_ERR_ARG, "invalid batch arguments");
  fwh_handle h0 = hs[0];
  if (n > kMaxBatchSurf)
    return fail(h0, FWH_ERR_ARG, "more surfaces than one batched call takes");
  if (!h0) return fail(nullptr, FWH_ERR_ARG, "NULL handle in batch");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  {
    const fwh_status st0 = take_deferred(h0);
    if (st0 != FWH_OK) return st0;
  }
  for (int i = 0; i < n; ++i) {
    fwh_handle h = hs[i];
    if (!h || !fields[i] || !p_out[i]) return fail(h0, FWH_ERR_ARG, "NULL entry in batch");
    if (h->precision != h0->precision) return fail(h0, FWH_ERR_ARG, "mixed precisions in batch");
    if (h->O < 1) return fail(h0, FWH_ERR_STATE, "a handle has no observers");
    if (!is_device_ptr(fields[i]) || !is_device_ptr(p_out[i]))
      return fail(h0, FWH_ERR_ARG, "batched forward takes device buffers");
    fwh_status st = prepare_window(h, nt[i]);
    if (st != FWH_OK) return fail(h0, st, h->err);
  }
  {  // series buffers (the whole record, or a ring of time segments) before the key
    const FwdConfig c = fwd_config(h0->precision == FWH_FP64, batch_cfg(n, hs, h0));
    const int seg = c.seg_chunks * 32 * c.tk;
    const int R = batch_round_segs(h0, seg);
    for (int i = 0; i < n; ++i)
      CK(h0, ensure(hs[i]->X, (size_t)hs[i]->P * batch_x_ld(hs[i], seg, R) * kRec *
                                  tsize(h0->precision)));
  }
  std::vector<uintptr_t> key;
  for (int i = 0; i < n; ++i) {
    key.push_back((uintptr_t)hs[i]);
    key.push_back((uintptr_t)fields[i]);
    key.push_back((uintptr_t)p_out[i]);
    key.push_back((uintptr_t)nt[i]);
    key.push_back((uintptr_t)hs[i]->X.p);
    key.push_back((uintptr_t)hs[i]->coef.p);
    key.push_back((uintptr_t)hs[i]->O);
    key.push_back((uintptr_t)hs[i]->nvalid.p);
    key.push_back((uintptr_t)hs[i]->sets.p);
    key.push_back((uintptr_t)hs[i]->imax.p);
  }
  key.push_back((uintptr_t)(h0->cfg + 1));
  key.push_back((uintptr_t)h0->wait_limit);
  key.push_back((uintptr_t)h0->withhold);
  key.push_back((uintptr_t)h0->batch_ring);
  key.push_back((uintptr_t)h0->batch_form);
  if (!h0->side) {
    CK(h0, cudaStreamCreateWithFlags(&h0->side, cudaStreamNonBlocking));
    CK(h0, cudaEventCreateWithFlags(&h0->bev[0], cudaEventDisableTiming));
    CK(h0, cudaEventCreateWithFlags(&h0->bev[1], cudaEventDisableTiming));
  }
  auto it = h0->graphs.find(key);
  if (it == h0->graphs.end()) {
    BatchPlan &bp = h0->bplans[key];
    fwh_status st = h0->precision == FWH_FP64 ? batch_build<double>(n, hs, p_out, h0, bp)
                                              : batch_build<float>(n, hs, p_out, h0, bp);
    if (st != FWH_OK) return st;
    // capture on the side stream (the caller's may be the legacy stream)
    cudaGraph_t g = nullptr;
    CK(h0, cudaStreamBeginCapture(h0->side, cudaStreamCaptureModeThreadLocal));
    st = h0->precision == FWH_FP64
             ? batch_enqueue<double>(n, hs, fields, p_out, h0, bp, h0->side)
             : batch_enqueue<float>(n, hs, fields, p_out, h0, bp, h0->side);
    cudaError_t e = cudaStreamEndCapture(h0->side, &g);
    if (st != FWH_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(h0, e, "cudaStreamEndCapture");
    Graph gr;
    e = cudaGraphInstantiate(&gr.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(h0, e, "cudaGraphInstantiate");
    gr.key = key;
    it = h0->graphs.emplace(key, gr).first;
  }
  CK(h0, cudaEventRecord(h0->bev[0], s));
  CK(h0, cudaStreamWaitEvent(h0->side, h0->bev[0], 0));
  CK(h0, cudaGraphLaunch(it->second.exec, h0->side));
  CK(h0, cudaEventRecord(h0->bev[1], h0->side));
  CK(h0, cudaStreamWaitEvent(s, h0->bev[1], 0));
  return defer_check(h0, s);
}

extern "C" fwh_status fwh_check(fwh_handle h, void *stream) {
  if (!h) return fail(nullptr, FWH_ERR_ARG, "handle is NULL");
  return check_device_flag(h, reinterpret_cast<cudaStream_t>(stream));
}

// ---------------------------------------------------------------------------
// Forward pass into caller-provided device scratch (no device allocation, no
// copy from host memory).  Used by the static-scratch entry point in
// fwh_noalloc.cu.  It reads the handle's panel-set plan, which the set-up calls
// (fwh_set_observers, fwh_set_tile_config, fwh_autotune) leave in place, and
// changes no handle state.  Every byte of the scratch that this call reads is
// written earlier in the same call: the observer windows by k_nvalid, every
// row of the prepared series (including the zero rows past nt) by the prep.
// ---------------------------------------------------------------------------
namespace {

template <typename T>
fwh_status forward_into_scratch_t(fwh_handle h, const T *d_fields, int64_t nt, double *d_pout,
                                  cudaStream_t s, unsigned char *scratch, size_t cap) {
  const bool fp64 = sizeof(T) == 8;
  const int ntp = (int)((nt + 255) / 256 * 256);  // same padding as prepare_nt
  const int cfg = effective_cfg(h, ntp);
  const FwdConfig c = fwd_config(fp64, cfg);
  const size_t off_x = ((size_t)h->O * sizeof(int) + 1023) / 1024 * 1024;
  const size_t need = off_x + (size_t)h->P * ntp * kRec * sizeof(T);
  if (need > cap)
    return fail(h, FWH_ERR_ARG,
                "problem needs " + std::to_string(need) + " bytes of scratch (panels x nt rounded "
                "up to 256 x 16 values + windows); the static scratch holds " +
                    std::to_string(cap) + " bytes");
  if (h->plan_win != c.win || h->plan_ch != 32 * c.tk || h->plan_sb != (c.acc == 5 ? 8 : 4))
    return fail(h, FWH_ERR_STATE,
                "the handle's panel-set plan belongs to another tile shape; call "
                "fwh_set_tile_config (which plans without a forward pass) first");
  int *d_nv = reinterpret_cast<int *>(scratch);
  T *d_X = reinterpret_cast<T *>(scratch + off_x);
  // observer windows (Eqs. t_start, t_end) on the device, from R_max / R_min
  CK(h, launch_nvalid(h->d_Rmax, h->d_Rmin, (int)h->O, h->mach, h->dt, (int)nt, d_nv, s));
  alignas(64) unsigned char desc[128];
  if (c.pipe != 0 &&
      !encode_x_tensor_map(desc, d_X, (unsigned long long)h->P * ntp, fp64, 32 * c.tk))
    return fail(h, FWH_ERR_CUDA, "cuTensorMapEncodeTiled refused the series layout");
  CK(h, cudaMemsetAsync(d_pout, 0, (size_t)h->O * nt * sizeof(double), s));
  PrepArgs<T> pa{};
  pa.fields = d_fields;
  pa.perm = h->identity ? nullptr : h->d_perm;
  pa.n = h->d_n;
  pa.X = d_X;
  pa.P = (int)h->P;
  pa.nt = (int)nt;
  pa.ntp = ntp;
  pa.x_ld = ntp;
  pa.ca = h->ca;
  pa.sa = h->sa;
  pa.dt = h->dt;
  CK(h, launch_prep<T>(pa, s));
  FwdArgs<T> fa{};
  fa.tmX = nullptr;
  fa.wait_cycles = h->wait_limit;
  fa.withhold = h->withhold;
  fa.x_ld = ntp;
  fa.X = d_X;
  fa.coef = reinterpret_cast<const T *>(h->coef.p);
  fa.p_out = d_pout;
  fa.n_valid = d_nv;
  fa.set_begin = reinterpret_cast<const int *>(h->sets.p);
  fa.set_order = reinterpret_cast<const int *>(h->sord.p);
  fa.i0max_tab = reinterpret_cast<const int *>(h->imax.p);
  fa.err = h->d_err;
  fa.nsets = (int)h->set_begin.size() - 1;
  fa.O = (int)h->O;
  fa.ntp = ntp;
  fa.nt = (int)nt;
  obs_tiling(h, c, &fa.obs_per_cta, &fa.n_obs_groups);
  fa.seg_len = c.seg_chunks * 32 * c.tk;
  fa.n_segs = (ntp + fa.seg_len - 1) / fa.seg_len;
  fa.seg_lo = 0;
  fa.seg_cnt = fa.n_segs;
  fa.win = c.win;
  fa.wfl = c.win * (c.acc == 5 ? 2 : 1);
  CK(h, launch_forward<T>(fa, c.pipe ? desc : nullptr, cfg, s));
  return defer_check(h, s);
}

}  // namespace

fwh_status fwh_forward_into_scratch(fwh_handle h, const void *fields, int64_t nt,
                                    double *p_out, cudaStream_t s, void *scratch,
                                    size_t cap) {
  if (!h) return fail(nullptr, FWH_ERR_ARG, "handle is NULL");
  if (h->O < 1) return fail(h, FWH_ERR_STATE, "fwh_set_observers must come first");
  if (!fields || !p_out) return fail(h, FWH_ERR_ARG, "fields or p_out is NULL");
  if (nt < 3 || nt > kMaxNt)
    return fail(h, FWH_ERR_ARG, "nt must be in [3, 2^28] (got " + std::to_string(nt) + ")");
  if (!scratch) return fail(h, FWH_ERR_ARG, "scratch is NULL");
  if (!is_device_ptr(fields) || !is_device_ptr(p_out))
    return fail(h, FWH_ERR_ARG, "this entry point takes device buffers only (no staging)");
  const fwh_status st = take_deferred(h);
  if (st != FWH_OK) return st;
  return h->precision == FWH_FP64
             ? forward_into_scratch_t<double>(h, reinterpret_cast<const double *>(fields), nt,
                                              p_out, s, static_cast<unsigned char *>(scratch),
                                              cap)
             : forward_into_scratch_t<float>(h, reinterpret_cast<const float *>(fields), nt,
                                             p_out, s, static_cast<unsigned char *>(scratch),
                                             cap);
}

// Record an error on a handle from another translation unit of the library.
fwh_status fwh_fail_handle(fwh_handle h, fwh_status st, const char *msg) {
  return fail(h, st, msg);
}
