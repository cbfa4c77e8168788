// Allocation-free forward pass: the prepared-series scratch lives in a
// file-scope device array instead of memory the handle allocates.
//
// Who needs this: code that must not call cudaMalloc/cudaFree (or any
// allocator, torch's caching allocator included) while it runs -- for
// example a real-time loop whose memory was budgeted up front, a process whose
// device memory is owned by another framework that forbids allocations during
// a step, or an embedding where an allocation could synchronise the device at
// the wrong moment.  Such a caller sets the handle up earlier (fwh_create and
// fwh_set_observers do allocate) and then calls fwh_forward_noalloc in its
// steady state.  The call copies nothing from host memory either.
//
// Limits and sharing: the array is kStaticScratchBytes (64 MiB) and every
// GPU that loads this library reserves it until the process exits.  All
// calls on a device share it; it keeps the last call's contents, but a call
// never reads anything it has not written itself first.  Calls whose GPU
// work overlaps (different streams, or several host threads) race on the
// array and must be serialised by the caller.
#include <mutex>

#include "../../include/fwh.h"
#include "fwh_internal.cuh"

namespace {
constexpr size_t kStaticScratchBytes = size_t(64) << 20;
constexpr int kMaxDevices = 64;
}  // namespace

static __device__ __align__(256) unsigned char g_fwh_static_scratch[kStaticScratchBytes];

// Device address of the array, looked up once per device (in host code the
// symbol is only a host-side stand-in and must not be passed to a kernel).
static void *g_scratch_addr[kMaxDevices];
static std::mutex g_scratch_mu;

fwh_status fwh_forward_into_scratch(fwh_handle h, const void *fields, int64_t nt,
                                    double *p_out, cudaStream_t s, void *scratch, size_t cap);
fwh_status fwh_fail_handle(fwh_handle h, fwh_status st, const char *msg);

extern "C" fwh_status fwh_forward_noalloc(fwh_handle h, const void *fields, int64_t nt,
                                          double *p_out, void *stream) {
  if (!h) return fwh_fail_handle(nullptr, FWH_ERR_ARG, "handle is NULL");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return fwh_fail_handle(h, FWH_ERR_CUDA, "no usable current CUDA device");
  }
  void *addr = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
      void *p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_fwh_static_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return fwh_fail_handle(h, FWH_ERR_CUDA,
                               "cudaGetSymbolAddress of the static scratch array failed");
      }
      g_scratch_addr[dev] = p;
    }
    addr = g_scratch_addr[dev];
  }
  return fwh_forward_into_scratch(h, fields, nt, p_out, reinterpret_cast<cudaStream_t>(stream),
                                  addr, kStaticScratchBytes);
}
