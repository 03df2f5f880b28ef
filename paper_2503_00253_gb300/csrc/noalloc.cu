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
// code cannot use the symbol itself as a device address, so each call asks
// the runtime for the array's device address in the calling thread's current
// context (cudaGetSymbolAddress).  That address belongs to the context's
// module: a non-primary driver context, or the primary context re-created
// after cudaDeviceReset, has its own copy of the array at its own address.
// A call made while its stream is being captured cannot query the runtime
// safely, so it uses the address recorded by the last uncaptured call in the
// same context; make one uncaptured call in each context before capturing.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "info_esrf.h"
#include "info_esrf_stages.h"

namespace {

constexpr size_t kNoAllocBytes = (size_t)32 << 20;   // 32 MiB, the documented maximum
constexpr int kMaxContexts = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

using CtxGetCurrentFn = CUresult (*)(CUcontext*);

std::mutex g_setup_mutex;
struct Slot {
  CUcontext ctx;
  void* ptr;
};
Slot g_slots[kMaxContexts] = {};
int g_nslots = 0;

// The calling thread's current driver context, through the runtime's driver
// entry-point query (no link against the driver library), or null.
CUcontext current_context() {
  static CtxGetCurrentFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      f = nullptr;
    }
    return reinterpret_cast<CtxGetCurrentFn>(f);
  }();
  CUcontext c = nullptr;
  if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
  return c;
}

// Device address of the scratch array in the current context.  Looked up
// afresh on every call outside stream capture (so a context re-created after
// cudaDeviceReset gets its own address); during capture the address recorded
// for this context by an earlier uncaptured call is used.
int scratch_address(cudaStream_t st, void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return INFO_ESRF_ERR_CUDA;
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
    cudaGetLastError();
    return INFO_ESRF_ERR_CUDA;
  }
  const CUcontext ctx = current_context();
  if (!ctx) return INFO_ESRF_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  int slot = -1;
  for (int i = 0; i < g_nslots; ++i)
    if (g_slots[i].ctx == ctx) slot = i;
  if (cap == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return INFO_ESRF_ERR_CUDA;
    }
    if (slot < 0) {
      if (g_nslots == kMaxContexts) {
        // full: drop the oldest entry (most likely a destroyed context)
        for (int i = 1; i < kMaxContexts; ++i) g_slots[i - 1] = g_slots[i];
        --g_nslots;
      }
      slot = g_nslots++;
      g_slots[slot].ctx = ctx;
    }
    g_slots[slot].ptr = p;
  } else if (slot < 0) {
    return INFO_ESRF_ERR_CUDA;   // first call in this context is being captured
  }
  *out = g_slots[slot].ptr;
  return INFO_ESRF_OK;
}

}  // namespace

extern "C" int info_esrf_analysis_noalloc(const info_esrf_grid* grid, int64_t N, const double* X_dev, int64_t d,
                                          const int64_t* obs_idx_dev, const double* y_dev,
                                          const double* R_diag_dev, int32_t Q, double tol,
                                          const info_esrf_options* opt, void* stream, double* mu_a_dev,
                                          double* A_a_dev) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  void* ws = nullptr;
  const int rc = scratch_address(st, &ws);
  if (rc != INFO_ESRF_OK) return rc;
  const size_t need = info_esrf_workspace_size(grid, N, d, Q, opt);
  // need == 0: the arguments or options are invalid or unsupported; the
  // regular entry point validates them before any kernel touches the array
  // and returns the same code it would for a caller's workspace
  if (need > kNoAllocBytes) return INFO_ESRF_ERR_UNSUPPORTED;
  // Every scratch word the analysis reads is written earlier in the same
  // call (tables, counters and accumulators are reset by its own kernels), so
  // the previous call's leftovers need no clearing.
  return info_esrf_analysis(grid, N, X_dev, d, obs_idx_dev, y_dev, R_diag_dev, Q, tol, opt, ws, kNoAllocBytes,
                            stream, mu_a_dev, A_a_dev, nullptr);
}
