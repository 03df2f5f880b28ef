// FMA throughput probe: the ALU roofline denominator of this GPU, measured.
#include <cuda_runtime.h>

#include "info_esrf.h"
#include "info_esrf_stages.h"
#include "internal.h"

namespace infoesrf {

template <typename T>
__global__ void k_fma_probe(T* out, int64_t iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = (T)(threadIdx.x + j) * (T)1e-3;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = fma(x[j], a, b);
  }
  T s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += x[j];
  if (s == (T)-1.2345) out[0] = s;   // keeps the chains live; practically never stores
}

}  // namespace infoesrf

using namespace infoesrf;

extern "C" int info_esrf_fma_probe(int32_t precision, int64_t iters, double* flops_per_s, double* ms,
                                   void* stream) {
  if ((precision != 0 && precision != 1) || iters < 1 || !flops_per_s || !ms) return INFO_ESRF_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))
    return INFO_ESRF_ERR_CUDA;
  const int blocks = sms * 4, threads = 256;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaGetLastError();
  void* out = nullptr;
  // warm-up and timed launch; the output is never written in practice
  for (int rep = 0; rep < 2; ++rep) {
    if (rep == 1) cudaEventRecord(e0, st);
    if (precision == 1) k_fma_probe<float><<<blocks, threads, 0, st>>>((float*)out, iters, 0.9999999f, 1e-7f);
    else k_fma_probe<double><<<blocks, threads, 0, st>>>((double*)out, iters, 0.9999999999, 1e-12);
    note_launches(1);
  }
  cudaEventRecord(e1, st);
  const cudaError_t err = cudaEventSynchronize(e1);
  float t = 0.f;
  cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess || cudaGetLastError() != cudaSuccess) return INFO_ESRF_ERR_CUDA;
  *ms = t;
  *flops_per_s = 2.0 * 8.0 * (double)iters * blocks * threads / (t * 1e-3);
  return 0;
}
