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
// Kernel.  Systems are grouped in units of 16 (one 16-row TMA box of P); a
// launch covers the units that hold an unconverged system, split evenly over
// `nchunks` CTAs per row tile (at most BN / 16 units each), so that converged
// systems cost no tensor-core work.  One CTA of 4 warps per (row tile, chunk):
// warp 0 lane 0 streams the blocks of the row tile through an S-stage ring of
// shared memory with 2-D TMA loads (128-byte swizzle): the hi and lo planes of
// the C block (the A operand, 128 x 64, K-major) and, per run of consecutive
// units, one slab of their directions (together the B operand, 16 u x 64,
// K-major; one tensor map per box height 16 .. 256 rows).  Warp 1
// lane 0 issues tcgen05.mma kind::f16 (BF16 x BF16, FP32 accumulate, N = 16 u)
// into a 128 x 16 u FP32 accumulator in tensor memory: four K = 16 steps for
// hi, four for lo, then a commit that frees the stage.  After the last block
// all four warps read the accumulator (tcgen05.ld, one TMEM lane = one row per
// thread), add sigma_j p_j, store y and reduce the partial dot products
// p_j^T y_j of the row tile.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "info_esrf_stages.h"
#include "internal.h"
#include "tile_mma.cuh"

namespace infoesrf {

namespace {

constexpr int kABytes = kTileM * kTileK * 2;     // one BF16 plane of a C block: 16 KB
constexpr int kUnitBytes = kTileUnit * kTileK * 2;   // one unit's slab of P: 2 KB

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

constexpr int kMaxUnits = 16;                        // units per CTA at most (256 systems)

// At most BN systems (BN / 16 units) per CTA, S pipeline stages.
template <int BN, int S>
struct TileMmShape {
  static constexpr int kUnits = BN / kTileUnit;
  static constexpr int kStage = 2 * kABytes + BN * kTileK * 2;
  static constexpr int kCtrl = 256;   // mbarriers, TMEM slot, flags, the CTA's units and loads
  static_assert(kUnits <= kMaxUnits, "units per CTA");
  static_assert(8 * (2 * S + 1) + 4 + 16 + 8 * kUnits <= kCtrl, "control block");
  static constexpr size_t kSmem = 1024 + (size_t)S * kStage + kCtrl + 4 * BN * sizeof(float);
};

// Tensor maps of P with boxes of 64 columns and 16 (i + 1) rows, i = 0 .. 15.
struct PMaps {
  CUtensorMap m[kMaxUnits];
};

// Ordered list of the units whose flag is set (one CTA of 1024 threads).
__global__ void __launch_bounds__(1024) k_tile_units(const int32_t* flags, int nunits, int32_t* ulist) {
  __shared__ int wsum[32];
  __shared__ int base;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  for (int u0 = 0; u0 < nunits; u0 += 1024) {
    const int u = u0 + (int)threadIdx.x;
    const bool act = u < nunits && flags[u] != 0;
    const unsigned m = __ballot_sync(0xffffffffu, act);
    if (lane == 0) wsum[warp] = __popc(m);
    __syncthreads();
    int off = base;
    for (int w = 0; w < warp; ++w) off += wsum[w];
    if (act) ulist[off + __popc(m & ((1u << lane) - 1u))] = u;
    __syncthreads();
    if (threadIdx.x == 0)
      for (int w = 0; w < 32; ++w) base += wsum[w];
    __syncthreads();
  }
}

template <int BN, int S>
__global__ void __launch_bounds__(128, 1)
    k_tile_mm(const __grid_constant__ CUtensorMap map_hi, const __grid_constant__ CUtensorMap map_lo,
              const __grid_constant__ PMaps maps_p, const TileMmArgs args) {
  using Shape = TileMmShape<BN, S>;
  constexpr int kStage = Shape::kStage;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                         ~static_cast<uintptr_t>(1023));
  unsigned char* ctrl = smem + S * kStage;
  uint64_t* full = reinterpret_cast<uint64_t*>(ctrl);
  uint64_t* empty = full + S;
  uint64_t* accf = empty + S;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(accf + 1);
  int* flags = reinterpret_cast<int*>(tslot + 1);   // [0] abort, [1] loads issued, [2] stages consumed, [3] runs
  int* units = flags + 4;                            // the CTA's units, in order
  int* runs = units + Shape::kUnits;                 // runs of consecutive units: first rank | length << 8
  float* red = reinterpret_cast<float*>(ctrl + Shape::kCtrl);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // an overflowed block pattern is not read (uniform across the grid)
  if (args.status && (*reinterpret_cast<volatile int32_t*>(args.status) & kStatTileOverflow)) return;
  const int chunk = (int)(blockIdx.x % (unsigned)args.nchunks);
  const int rt = (int)(blockIdx.x / (unsigned)args.nchunks);
  // this CTA's units: ranks [chunk T / nchunks, (chunk + 1) T / nchunks) of the T listed units
  // (at most kUnits: nchunks >= T / kUnits)
  const int T = args.units;
  const int lo = (int)((int64_t)chunk * T / args.nchunks);
  const int nu = min((int)((int64_t)(chunk + 1) * T / args.nchunks) - lo, Shape::kUnits);
  if (nu <= 0) return;   // uniform across the CTA, before any barrier or TMEM use
  if (threadIdx.x < nu) units[threadIdx.x] = args.ulist ? args.ulist[lo + threadIdx.x] : lo + (int)threadIdx.x;
  __syncthreads();
  if (threadIdx.x == 0) {
    int nr = 0;
    for (int i = 0; i < nu;) {
      int len = 1;
      while (i + len < nu && units[i + len] == units[i] + len) ++len;
      runs[nr++] = i | (len << 8);
      i += len;
    }
    flags[3] = nr;
  }
  const int ncol = nu * kTileUnit;
  const uint32_t stage_bytes = 2 * kABytes + nu * kUnitBytes;
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
  }
  if (warp == 2) tmem_alloc(tslot, BN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const int nruns = flags[3];

  if (warp == 0 && lane == 0) {
    // producer: C block planes and each unit's slab of the directions for the block's columns
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
      const int xcol = args.colblk[tile] * kTileK;
      mbar_arrive_expect_tx(&full[s], stage_bytes);
      tma_load_2d(st, &map_hi, &full[s], 0, tile * kTileM);
      tma_load_2d(st + kABytes, &map_lo, &full[s], 0, tile * kTileM);
      for (int r = 0; r < nruns; ++r) {
        const int i = runs[r] & 255, len = runs[r] >> 8;
        tma_load_2d(st + 2 * kABytes + i * kUnitBytes, &maps_p.m[len - 1], &full[s], xcol, units[i] * kTileUnit);
      }
    }
    flags[1] = kb;
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: acc = sum over blocks of (C_hi + C_lo) P, FP32 in TMEM
    const uint32_t idesc = idesc_bf16_f32(kTileM, ncol);
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
      const uint64_t db = sw128_desc(base + 2 * kABytes);
#pragma unroll
      for (int k = 0; k < kTileK / 16; ++k)   // K = 16 per MMA: 32 bytes along the swizzled row
        mma_bf16(tmem, dhi + 2 * k, db + 2 * k, idesc, (kb | k) != 0 ? 1u : 0u);
#pragma unroll
      for (int k = 0; k < kTileK / 16; ++k) mma_bf16(tmem, dlo + 2 * k, db + 2 * k, idesc, 1u);
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
    for (int i = 0; i < nu; ++i) {   // one unit = 16 accumulator columns
      float v[16];
      tmem_ld16(tbase + (uint32_t)(i * kTileUnit), v);
      const int jb = units[i] * kTileUnit;
#pragma unroll
      for (int c = 0; c < kTileUnit; ++c) {
        const int j = jb + c;
        float dot = 0.f;
        if (j < args.J) {
          const float p = __bfloat162float(args.P[(int64_t)j * args.d_pad + a]);
          const float y = args.sigma ? fmaf(args.sigma[j], p, v[c]) : v[c];
          args.Y[(int64_t)j * args.d_pad + a] = y;
          dot = p * y;
        }
        dot = warp_sum_f(dot);
        if (lane == 0) red[warp * BN + i * kTileUnit + c] = dot;
      }
    }
    __syncthreads();
    if (args.pty)
      for (int t = threadIdx.x; t < ncol; t += blockDim.x) {
        const int j = units[t / kTileUnit] * kTileUnit + t % kTileUnit;
        if (j < args.J) {
          const float v = (red[t] + red[BN + t]) + (red[2 * BN + t] + red[3 * BN + t]);
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
  if (warp == 2) tmem_dealloc(tmem, BN);
}

template <int BN, int S>
int launch_tile_mm_t(TileMmArgs a, const void* chi, const void* clo, int64_t ntiles, cudaStream_t st) {
  using Shape = TileMmShape<BN, S>;
  a.nchunks = (a.units + Shape::kUnits - 1) / Shape::kUnits;
  CUtensorMap mh, ml;
  PMaps mp;
  if (!encode_bf16(&mh, chi, kTileK, (uint64_t)ntiles * kTileM, kTileK, kTileM) ||
      !encode_bf16(&ml, clo, kTileK, (uint64_t)ntiles * kTileM, kTileK, kTileM))
    return INFO_ESRF_ERR_CUDA;
  for (int i = 0; i < Shape::kUnits; ++i)
    if (!encode_bf16(&mp.m[i], a.P, (uint64_t)a.d_pad, (uint64_t)a.J, (uint64_t)a.d_pad, (uint32_t)(kTileUnit * (i + 1))))
      return INFO_ESRF_ERR_CUDA;
  static thread_local int raised_dev = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (raised_dev != dev) {
    if (cudaFuncSetAttribute(k_tile_mm<BN, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Shape::kSmem) !=
        cudaSuccess)
      return INFO_ESRF_ERR_CUDA;
    raised_dev = dev;
  }
  const int64_t grid = (int64_t)a.nrt * a.nchunks;
  k_tile_mm<BN, S><<<(unsigned)grid, 128, Shape::kSmem, st>>>(mh, ml, mp, a);
  note_launches(1);
  return cudaGetLastError() == cudaSuccess ? INFO_ESRF_OK : INFO_ESRF_ERR_CUDA;
}

}  // namespace

int launch_tile_mm(TileMmArgs a, const void* chi, const void* clo, int64_t ntiles, cudaStream_t st) {
  const int32_t nunits = (a.J + kTileUnit - 1) / kTileUnit;
  if (a.nrt < 1 || a.J < 1 || a.d_pad % kTileM || (int64_t)a.nrt * kTileM != a.d_pad ||
      ntiles * kTileM >= (int64_t(1) << 31) || (a.active && (!a.ulist || a.units < 0 || a.units > nunits)))
    return INFO_ESRF_ERR_INVALID_ARG;
  if (a.active) {
    if (a.units == 0) return INFO_ESRF_OK;
    k_tile_units<<<1, 1024, 0, st>>>(a.active, nunits, a.ulist);
    note_launches(1);
  } else {
    a.units = nunits;
    a.ulist = nullptr;
  }
  // up to 8 units (128 systems): a 128-column accumulator and 4 stages; else
  // up to 16 units per CTA, 3 stages.  (Two 256-column accumulators per CTA,
  // so that a C block load serves 512 systems, leave room for two stages only
  // and measured slower: 1225 against 1273 TFLOP/s on the tilemm workload.)
  if (a.units <= 8) return launch_tile_mm_t<128, 4>(a, chi, clo, ntiles, st);
  return launch_tile_mm_t<256, 3>(a, chi, clo, ntiles, st);
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

namespace infoesrf {
namespace {

// One bounded mbarrier wait, as the tensor-core kernels wait for their copies
// and MMAs: thread 0 initializes a barrier of one arrival, arrives on it first
// when `arrive` is set, then waits for its phase 0 at most `limit` cycles and
// records kStatTimeout in *status when the wait ran out.  Nothing faults or
// hangs: with no arrival the wait ends after the limit.
__global__ void k_wait_probe(long long limit, int arrive, int32_t* status) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  fence_mbar_init();
  if (arrive) mbar_arrive(&bar);
  status[0] = mbar_wait(&bar, 0, limit) ? 0 : kStatTimeout;
}

}  // namespace
}  // namespace infoesrf

extern "C" int info_esrf_wait_probe(int64_t limit_cycles, int32_t arrive, int32_t* status_dev, void* stream) {
  if (!status_dev || limit_cycles < 1 || limit_cycles > infoesrf::kWaitCycles) return INFO_ESRF_ERR_INVALID_ARG;
  cudaGetLastError();
  infoesrf::k_wait_probe<<<1, 32, 0, reinterpret_cast<cudaStream_t>(stream)>>>((long long)limit_cycles,
                                                                                arrive ? 1 : 0, status_dev);
  infoesrf::note_launches(1);
  return cudaGetLastError() == cudaSuccess ? INFO_ESRF_OK : INFO_ESRF_ERR_CUDA;
}
