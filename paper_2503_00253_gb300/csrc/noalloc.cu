// Allocation-free analysis entry point.
//
// Who needs it: callers that must not allocate device memory themselves,
// for example a plug-in living inside a host application that owns every
// device byte through its own pool, or a real-time cycling loop that cannot
// afford cudaMalloc's implicit device synchronization.  Such callers cannot
// provide the workspace the regular entry points take, so this entry point
// carves it from a fixed array that is part of the library image.
//
// The array is a file-scope __device__ variable: every GPU on which the
// library is loaded holds kNoAllocBytes of it until the process exits.  Host
// code cannot use the symbol itself as a device address, so the first call on
// each device asks the runtime for the array's device address
// (cudaGetSymbolAddress, with that device current) and keeps it.  Make that
// first call before any stream capture on the device.
#include <cuda_runtime.h>

#include <mutex>

#include "info_esrf.h"
#include "info_esrf_stages.h"

namespace {

constexpr size_t kNoAllocBytes = (size_t)32 << 20;   // 32 MiB, the documented maximum
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once.
int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return INFO_ESRF_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return INFO_ESRF_ERR_CUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return INFO_ESRF_OK;
}

}  // namespace

extern "C" int info_esrf_analysis_noalloc(const info_esrf_grid* grid, int64_t N, const double* X_dev, int64_t d,
                                          const int64_t* obs_idx_dev, const double* y_dev,
                                          const double* R_diag_dev, int32_t Q, double tol,
                                          const info_esrf_options* opt, void* stream, double* mu_a_dev,
                                          double* A_a_dev) {
  const size_t need = info_esrf_workspace_size(grid, N, d, Q, opt);
  if (need == 0) return INFO_ESRF_ERR_INVALID_ARG;
  if (need > kNoAllocBytes) return INFO_ESRF_ERR_UNSUPPORTED;
  void* ws = nullptr;
  const int rc = scratch_address(&ws);
  if (rc != INFO_ESRF_OK) return rc;
  // Every scratch word the analysis reads is written earlier in the same
  // call (tables, counters and accumulators are reset by its own kernels), so
  // the previous call's leftovers need no clearing.
  return info_esrf_analysis(grid, N, X_dev, d, obs_idx_dev, y_dev, R_diag_dev, Q, tol, opt, ws, kNoAllocBytes,
                            stream, mu_a_dev, A_a_dev, nullptr);
}
