// nw_noalloc.cu -- nw_all_pairs_topk_noalloc: the all-pairs top-k reduction
// for callers that cannot allocate device memory.  Its scratch (list slots,
// thresholds, task counters, histogram accumulators, error flag) lives in one
// static device array defined here; nothing is allocated per call.
#include <cuda_runtime.h>

#include <mutex>

#include "nw.h"
#include "nw_launch.h"

namespace {

// One copy per device that loads the library, held until the process exits.
// Every call shares it; the host code below only ever hands its device
// address (from cudaGetSymbolAddress) to the kernels.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NW_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 256;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Called by the reduction with `device` current.  The first call on a device
// looks up the array's device address; later calls reuse it.
nw_status scratch_for_device(int device, void** base, size_t* bytes, const char** why) {
  if (device < 0 || device >= kMaxDevices) {
    *why = "device ordinal out of range";
    return NW_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      *why = e != cudaSuccess ? cudaGetErrorString(e) : "null symbol address";
      return NW_ECUDA;
    }
    g_addr[device] = p;
  }
  *base = g_addr[device];
  *bytes = NW_NOALLOC_SCRATCH_BYTES;
  return NW_OK;
}

}  // namespace

extern "C" nw_status nw_all_pairs_topk_noalloc(nw_dict* dict, uint32_t k, uint32_t* nbr_idx, int16_t* nbr_score,
                                               int64_t* hist, int32_t* hist_lo, uint32_t nbins, uint32_t flags) {
  return nw::topk_into_scratch(dict, scratch_for_device, k, nbr_idx, nbr_score, hist, hist_lo, nbins, flags);
}
