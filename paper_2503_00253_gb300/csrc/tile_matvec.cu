// a5, BF16 path: the localized-covariance matvec of every PCG iteration,
//     y_j = sigma_j p_j + C p_j   for all systems j at once
// (App. E, Eq. normalized_linear_solve; every shifted system shares the one
// matrix C = R^-1/2 (L_oo o W W^T) R^-1/2 of Sec. 2.3, so the product over
// all systems is one block-sparse matrix product C P with P = [p_1 ... p_J]).
//
// Layout.  Observations are numbered in tile order (the library's own
// permutation, spatially compact tiles).  C is kept only in the 128 x 64
// blocks (row tile, column block) whose bounding boxes come within the
// Gaspari-Cohn support (all other entries are exact zeros), each block
// stored as two BF16 planes hi = bf16(C), lo = bf16(C - hi), row-major
// [tile][128][64].  The directions are BF16, system-major [J][d_pad].
//
// Kernel.  One CTA of 4 warps per (row tile, chunk of H x BN systems).  Warp 0
// lane 0 streams the blocks of the row tile through an S-stage ring of shared
// memory with 2-D TMA loads (128-byte swizzle): the hi and lo planes of the C
// block (the A operand, 128 x 64, K-major) and the 64-row slab of the chunk's
// directions (the B operand, BN x 64, K-major).  Warp 1 lane 0 issues
// tcgen05.mma kind::f16 (BF16 x BF16, FP32 accumulate) into H 128 x BN FP32
// accumulators in tensor memory (H = 2 when more than 256 systems: each C
// block load then serves 512 systems): four K = 16 steps for hi, four for lo,
// per accumulator, then a commit that frees the stage.  After the last block all four warps read the
// accumulator (tcgen05.ld, one TMEM lane = one row per thread), add sigma_j p_j,
// store y and reduce the partial dot products p_j^T y_j of the row tile.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "info_esrf_stages.h"
#include "internal.h"
#include "tile_mma.cuh"

namespace infoesrf {

namespace {

constexpr int kABytes = kTileM * kTileK * 2;   // one BF16 plane of a C block: 16 KB

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// BN systems per accumulator, S pipeline stages, H accumulators (TMEM halves)
// per CTA sharing each C block load.
template <int BN, int S, int H>
struct TileMmShape {
  static constexpr int kStage = 2 * kABytes + H * BN * kTileK * 2;
  static constexpr int kCtrl = 256;   // mbarriers, TMEM slot, flags
  static constexpr size_t kSmem = 1024 + (size_t)S * kStage + kCtrl + 4 * H * BN * sizeof(float);
};

template <int BN, int S, int H>
__global__ void __launch_bounds__(128, 1)
    k_tile_mm(const __grid_constant__ CUtensorMap map_hi, const __grid_constant__ CUtensorMap map_lo,
              const __grid_constant__ CUtensorMap map_p, const TileMmArgs args) {
  using Shape = TileMmShape<BN, S, H>;
  constexpr int kStage = Shape::kStage;
  constexpr int kCols = H * BN;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                         ~static_cast<uintptr_t>(1023));
  unsigned char* ctrl = smem + S * kStage;
  uint64_t* full = reinterpret_cast<uint64_t*>(ctrl);
  uint64_t* empty = full + S;
  uint64_t* accf = empty + S;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(accf + 1);
  int* flags = reinterpret_cast<int*>(tslot + 1);   // [0] abort, [1] loads issued, [2] stages consumed
  float* red = reinterpret_cast<float*>(ctrl + Shape::kCtrl);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int chunk = (int)(blockIdx.x % (unsigned)args.nchunks);
  const int rt = (int)(blockIdx.x / (unsigned)args.nchunks);
  // accumulator h serves systems (chunk H + h) BN ..; skipped when it has none
  // or all of them have converged (args.active has one flag per BN systems)
  bool hact[H];
  int nh = 0;
#pragma unroll
  for (int h = 0; h < H; ++h) {
    const int unit = chunk * H + h;
    hact[h] = unit * BN < args.J && (!args.active || args.active[unit]);
    nh += hact[h];
  }
  if (nh == 0) return;
  const uint32_t stage_bytes = 2 * kABytes + nh * BN * kTileK * 2;
  const int t0 = args.rowptr[rt];
  const int nk = args.rowptr[rt + 1] - t0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accf, 1);
    flags[0] = 0;
    flags[1] = 0;
    flags[2] = 0;
    fence_mbar_init();
    tma_prefetch_map(&map_hi);
    tma_prefetch_map(&map_lo);
    tma_prefetch_map(&map_p);
  }
  if (warp == 2) tmem_alloc(tslot, kCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0 && lane == 0) {
    // producer: C block planes and the directions' slab of each column block
    int kb = 0;
    for (; kb < nk; ++kb) {
      const int s = kb % S;
      if (kb >= S && !mbar_wait(&empty[s], ((kb / S) & 1) ^ 1)) {
        atomicExch(&flags[0], 1);
        break;
      }
      if (*reinterpret_cast<volatile int*>(&flags[0])) break;
      unsigned char* st = smem + s * kStage;
      const int tile = t0 + kb;
      mbar_arrive_expect_tx(&full[s], stage_bytes);
      tma_load_2d(st, &map_hi, &full[s], 0, tile * kTileM);
      tma_load_2d(st + kABytes, &map_lo, &full[s], 0, tile * kTileM);
#pragma unroll
      for (int h = 0; h < H; ++h)
        if (hact[h])
          tma_load_2d(st + 2 * kABytes + h * BN * kTileK * 2, &map_p, &full[s], args.colblk[tile] * kTileK,
                      (chunk * H + h) * BN);
    }
    flags[1] = kb;
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: acc = sum over blocks of (C_hi + C_lo) P, FP32 in TMEM
    constexpr uint32_t idesc = idesc_bf16_f32(kTileM, BN);
    int kb = 0;
    for (; kb < nk; ++kb) {
      const int s = kb % S;
      if (!mbar_wait(&full[s], (kb / S) & 1)) {
        atomicExch(&flags[0], 1);
        break;
      }
      tc_fence_after();
      const uint32_t base = smem_u32(smem + s * kStage);
      const uint64_t dhi = sw128_desc(base), dlo = sw128_desc(base + kABytes);
#pragma unroll
      for (int h = 0; h < H; ++h) {
        if (!hact[h]) continue;
        const uint64_t db = sw128_desc(base + 2 * kABytes + h * BN * kTileK * 2);
        const uint32_t td = tmem + (uint32_t)(h * BN);
#pragma unroll
        for (int k = 0; k < kTileK / 16; ++k)   // K = 16 per MMA: 32 bytes along the swizzled row
          mma_bf16(td, dhi + 2 * k, db + 2 * k, idesc, (kb | k) != 0 ? 1u : 0u);
#pragma unroll
        for (int k = 0; k < kTileK / 16; ++k) mma_bf16(td, dlo + 2 * k, db + 2 * k, idesc, 1u);
      }
      mma_commit(&empty[s]);
    }
    flags[2] = kb;
    mma_commit(accf);
  }
  __syncwarp();
  if (!mbar_wait(accf, 0)) atomicExch(&flags[0], 1);
  tc_fence_after();
  __syncthreads();
  const bool aborted = *reinterpret_cast<volatile int*>(&flags[0]) != 0;
  if (!aborted) {
    const int row = warp * 32 + lane;
    const int64_t a = (int64_t)rt * kTileM + row;
    const uint32_t tbase = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
    for (int h = 0; h < H; ++h) {
      if (!hact[h]) continue;   // uniform across the CTA
      for (int c0 = 0; c0 < BN; c0 += 16) {
        float v[16];
        tmem_ld16(tbase + (uint32_t)(h * BN + c0), v);
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int j = (chunk * H + h) * BN + c0 + c;
          float dot = 0.f;
          if (j < args.J) {
            const float p = __bfloat162float(args.P[(int64_t)j * args.d_pad + a]);
            const float y = fmaf(args.sigma[j], p, v[c]);
            args.Y[(int64_t)j * args.d_pad + a] = y;
            dot = p * y;
          }
          dot = warp_sum_f(dot);
          if (lane == 0) red[warp * kCols + h * BN + c0 + c] = dot;
        }
      }
    }
    __syncthreads();
    if (args.pty)
      for (int t = threadIdx.x; t < kCols; t += blockDim.x) {
        const int j = chunk * kCols + t;
        if (j < args.J && hact[t / BN]) {
          const float v = (red[t] + red[kCols + t]) + (red[2 * kCols + t] + red[3 * kCols + t]);
          if (args.pty_by_system) args.pty[(int64_t)j * args.nrt + rt] = v;
          else args.pty[(int64_t)rt * args.J + j] = v;
        }
      }
  } else if (threadIdx.x == 0) {
    // wait (bounded) for the loads still in flight before the CTA's shared memory goes away
    for (int kb = flags[2]; kb < flags[1]; ++kb) mbar_wait(&full[kb % S], (kb / S) & 1);
    if (args.status) atomicOr(args.status, kStatTimeout);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) tmem_dealloc(tmem, kCols);
}

template <int BN, int S, int H>
int launch_tile_mm_t(TileMmArgs a, const void* chi, const void* clo, int64_t ntiles, cudaStream_t st) {
  using Shape = TileMmShape<BN, S, H>;
  a.nchunks = (a.J + H * BN - 1) / (H * BN);
  CUtensorMap mh, ml, mp;
  if (!encode_bf16(&mh, chi, kTileK, (uint64_t)ntiles * kTileM, kTileK, kTileM) ||
      !encode_bf16(&ml, clo, kTileK, (uint64_t)ntiles * kTileM, kTileK, kTileM) ||
      !encode_bf16(&mp, a.P, (uint64_t)a.d_pad, (uint64_t)a.J, (uint64_t)a.d_pad, BN))
    return INFO_ESRF_ERR_CUDA;
  static thread_local int raised_dev = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (raised_dev != dev) {
    if (cudaFuncSetAttribute(k_tile_mm<BN, S, H>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Shape::kSmem) !=
        cudaSuccess)
      return INFO_ESRF_ERR_CUDA;
    raised_dev = dev;
  }
  const int64_t grid = (int64_t)a.nrt * a.nchunks;
  k_tile_mm<BN, S, H><<<(unsigned)grid, 128, Shape::kSmem, st>>>(mh, ml, mp, a);
  note_launches(1);
  return cudaGetLastError() == cudaSuccess ? INFO_ESRF_OK : INFO_ESRF_ERR_CUDA;
}

}  // namespace

int tile_chunk_width(int32_t J) { return J <= 128 ? 128 : 256; }

int launch_tile_mm(TileMmArgs a, const void* chi, const void* clo, int64_t ntiles, cudaStream_t st) {
  if (a.nrt < 1 || a.J < 1 || a.d_pad % kTileM || (int64_t)a.nrt * kTileM != a.d_pad ||
      ntiles * kTileM >= (int64_t(1) << 31))
    return INFO_ESRF_ERR_INVALID_ARG;
  // up to 128 systems per CTA: one 128-column accumulator, 4 stages; else
  // 256-column accumulators, 3 stages.  (Two accumulators per CTA, so that a
  // C block load serves 512 systems, leave room for two stages only and
  // measured slower: 1225 against 1273 TFLOP/s on the tilemm workload.)
  if (a.J <= 128) return launch_tile_mm_t<128, 4, 1>(a, chi, clo, ntiles, st);
  return launch_tile_mm_t<256, 3, 1>(a, chi, clo, ntiles, st);
}

}  // namespace infoesrf

using namespace infoesrf;

extern "C" int info_esrf_bf16_tile_matvec(int32_t n_row_tiles, const int32_t* rowptr_dev, const int32_t* colblk_dev,
                                          int64_t n_tiles, const uint16_t* C_hi_dev, const uint16_t* C_lo_dev,
                                          int32_t J, const uint16_t* P_dev, const float* sigma_dev, float* Y_dev,
                                          float* pty_dev, int32_t* status_dev, void* stream) {
  if (n_row_tiles < 1 || n_tiles < n_row_tiles || J < 1 || !rowptr_dev || !colblk_dev || !C_hi_dev || !C_lo_dev ||
      !P_dev || !sigma_dev || !Y_dev)
    return INFO_ESRF_ERR_INVALID_ARG;
  TileMmArgs a{};
  a.rowptr = rowptr_dev;
  a.colblk = colblk_dev;
  a.P = reinterpret_cast<const __nv_bfloat16*>(P_dev);
  a.sigma = sigma_dev;
  a.active = nullptr;
  a.Y = Y_dev;
  a.pty = pty_dev;
  a.status = status_dev;
  a.d_pad = (int64_t)n_row_tiles * kTileM;
  a.J = J;
  a.nrt = n_row_tiles;
  cudaGetLastError();
  return launch_tile_mm(a, C_hi_dev, C_lo_dev, n_tiles, reinterpret_cast<cudaStream_t>(stream));
}
