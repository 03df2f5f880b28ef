// a1-a3 set-up, BF16 path, on the fifth-generation tensor cores: the stored
// 128 x 64 blocks of the normalized localized covariance
//     C(a, b) = GC(r_ab) (w_a . w_b) R_a^-1/2 R_b^-1/2
// (Sec. 2.3, Eq. localized_obs_covar with L_oo the Gaspari-Cohn matrix, and the
// normalization of App. E), for every (row tile, stored column block) of the
// block pattern, as the hi and lo BF16 planes the tensor-core matvec reads.
// Per row tile (128 tile-ordered observations, one CTA) and block (64):
//     S = W_rt W_blk^T        128 x 64, K = members (padded to 128; steps past N skipped)
// as tcgen05.mma kind::f16 with FP32 accumulation in tensor memory, from three
// BF16 planes of W in the six terms hh, hm, mh, hl, lh, mm (about 2^-26
// relative per product, as accurate as the FP32 dot products it replaces).
// The epilogue applies the Gaspari-Cohn weight and R^-1/2 of both ends, splits
// the value into hi = bf16(C), lo = bf16(C - hi), stores both planes, and keeps
// the row sums of |C| (the Gershgorin bound), the diagonal (its minimum and its
// sum) and the count of nonzeros.
//
// CTA of 10 warps: warp 8 lane 0 loads W_rt once and W_blk per block with 2-D
// TMA (128-byte swizzle) and the block's coordinates and R^-1/2 with bulk
// copies; warp 9 lane 0 issues the MMAs; warps 0-7 (two per TMEM lane
// quadrant, one row and 32 of the block's columns per thread) run the
// epilogue.  S has two TMEM buffers and W_blk is free once the product of its
// block is done, so the load and the product of block b + 1 run during the
// epilogue of block b.  All waits are bounded (kStatTimeout).
#include <cuda_bf16.h>

#include "common.cuh"
#include "info_esrf.h"
#include "internal.h"
#include "tile_mma.cuh"

namespace infoesrf {

namespace {

constexpr int kFmThreads = 320;                      // warps 0-7 epilogue, 8 loads, 9 MMAs
constexpr int kFHalf = kTileM * 64 * 2;              // one 64-member half of W_rt: 16 KB
constexpr int kFWHalf = kTileK * 64 * 2;             // one 64-member half of W_blk: 8 KB
constexpr int kFSide = kTileK * 16 + kTileK * 4;     // a block's coordinates and R^-1/2
constexpr int kFD2 = 4096;                           // distance-table entries in shared memory

struct FmLayout {
  uint32_t a, b, side, ctrl, red, d2, total;
};

__host__ __device__ inline FmLayout fm_layout(int nd2) {
  FmLayout L;
  L.a = 0;                          // W_rt: planes h, m, l, two halves each
  L.b = 6 * kFHalf;                 // W_blk: planes h, m, l, two halves each
  L.side = L.b + 6 * kFWHalf;       // two buffers of the block's coordinates and R^-1/2
  L.ctrl = L.side + 2 * kFSide;     // barriers, TMEM slot, flags
  L.red = L.ctrl + 256;             // [128] row sums of the second column half
  L.d2 = L.red + kTileM * 8;        // distance table
  L.total = L.d2 + 4 * (uint32_t)nd2;
  return L;
}

// W in three BF16 planes (members padded to kStK) and the grid coordinates of
// each tile position (w = -1: padding), in tile order.
__global__ void k_tile_form_prep(const ProblemDev* tab) {
  const ProblemDev& pr = tab[blockIdx.y];
  if (pr.precision != 2 || !pr.st_W) return;
  const int64_t N = pr.N, dp = pr.d_pad;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nw = dp * kStK;
  if (i < nw) {
    const int64_t a = i / kStK, k = i % kStK;
    float r = k < N ? pr.Wp[a * N + k] : 0.f;
#pragma unroll
    for (int pl = 0; pl < 3; ++pl) {
      const __nv_bfloat16 h = __float2bfloat16_rn(r);
      pr.st_W[pl * nw + i] = h;
      r -= __bfloat162float(h);
    }
  }
  if (i < dp) {
    const int32_t src = i < pr.d ? pr.tpos_src[i] : -1;
    int4 c = make_int4(0, 0, 0, -1);
    if (src >= 0) {
      const Coord3 cc = flat_to_coord(pr.grid, pr.obs[src]);
      c = make_int4((int)cc.x, (int)cc.y, (int)cc.z, 1);
    }
    pr.st_xyz[i] = c;
  }
}

__global__ void __launch_bounds__(kFmThreads, 1)
    k_tile_form_mma(const __grid_constant__ CUtensorMap map_w0, const __grid_constant__ CUtensorMap map_w1,
                    const __grid_constant__ CUtensorMap map_w2, const ProblemDev* dpr) {
  const ProblemDev& pr = *dpr;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                         ~static_cast<uintptr_t>(1023));
  const GridDev& g = pr.grid;
  const int64_t next = g.ext[0] + g.ext[1] + g.ext[2];   // <= kFD2 (checked by the launcher)
  const FmLayout Lo = fm_layout((int)next);
  // Barriers.  wfull and accf complete once per block / once; xfull, g1done and
  // efree have one barrier per buffer, completing once per two blocks.  Each
  // next completion depends on its waiters having passed, so no waiter falls
  // two phases behind.
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + Lo.ctrl);
  uint64_t* afull = bar + 0;    // W_rt landed (once)
  uint64_t* wfull = bar + 1;    // W_blk(b) landed                                     (MMA)
  uint64_t* xfull = bar + 2;    // [2] side buffer b % 2 landed, phase b / 2           (epilogue)
  uint64_t* g1done = bar + 4;   // [2] S(b) in TMEM buffer b % 2, phase b / 2          (epilogue, loads)
  uint64_t* efree = bar + 6;    // [2] epilogue of b done with TMEM and side buffer b % 2 (MMA, loads; 256)
  uint64_t* accf = bar + 8;     // every MMA done
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 9);
  int* flags = reinterpret_cast<int*>(tslot + 1);   // [0] abort, [1] W_blk/side loads issued, [2] W_rt issued, [3] skip
  double* red = reinterpret_cast<double*>(smem + Lo.red);
  float* d2 = reinterpret_cast<float*>(smem + Lo.d2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t rt = blockIdx.x;
  if (rt >= pr.nrt) return;
  // an overflowed pattern (or a timeout elsewhere) stops the CTA (uniform per CTA)
  if (tid == 0) flags[3] = (pr.status[0] & (kStatTimeout | kStatTileOverflow)) ? 1 : 0;
  __syncthreads();
  if (flags[3]) return;
  const int t0 = pr.rowptr[rt], nk = pr.rowptr[rt + 1] - t0;
  const int N = (int)pr.N;
  if (tid == 0) {
    for (int i = 0; i < 9; ++i) mbar_init(bar + i, (i == 6 || i == 7) ? 256 : 1);
    flags[0] = 0;
    flags[1] = 0;
    flags[2] = 0;
    fence_mbar_init();
    tma_prefetch_map(&map_w0);
    tma_prefetch_map(&map_w1);
    tma_prefetch_map(&map_w2);
  }
  if (warp == 8) tmem_alloc(tslot, 128);
  for (int64_t e = tid; e < next; e += blockDim.x) d2[e] = (float)pr.d2tab[e];
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;   // S buffers at columns 0 and 64

  if (warp == 8) {
    if (lane == 0) {
      // W_rt: three planes, two 64-member halves each, as two 64-row boxes
      mbar_arrive_expect_tx(afull, 6 * kFHalf);
      const CUtensorMap* maps[3] = {&map_w0, &map_w1, &map_w2};
#pragma unroll
      for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int r = 0; r < 2; ++r)
            tma_load_2d(smem + Lo.a + (2 * p + h) * kFHalf + r * (kTileK * 128), maps[p], afull, 64 * h,
                        (int)(rt * kTileM) + r * kTileK);
      flags[2] = 1;
      for (int kb = 0; kb < nk; ++kb) {
        // W_blk is free once the product of kb - 1 is done
        if (kb >= 1 && !mbar_wait(&g1done[(kb - 1) & 1], ((kb - 1) >> 1) & 1)) {
          atomicExch(&flags[0], 1);
          break;
        }
        // side buffer kb % 2 is free once the epilogue of kb - 2 is done
        if (kb >= 2 && !mbar_wait(&efree[kb & 1], ((kb - 2) >> 1) & 1)) {
          atomicExch(&flags[0], 1);
          break;
        }
        if (*reinterpret_cast<volatile int*>(&flags[0])) break;
        const int row = pr.colblk[t0 + kb] * kTileK;
        unsigned char* bp = smem + Lo.b;
        mbar_arrive_expect_tx(wfull, 6 * kFWHalf);
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
          for (int h = 0; h < 2; ++h) tma_load_2d(bp + (2 * p + h) * kFWHalf, maps[p], wfull, 64 * h, row);
        unsigned char* xp = smem + Lo.side + (kb & 1) * kFSide;
        mbar_arrive_expect_tx(&xfull[kb & 1], kFSide);
        bulk_load(xp, pr.st_xyz + row, kTileK * 16, &xfull[kb & 1]);
        bulk_load(xp + kTileK * 16, pr.rinvp + row, kTileK * 4, &xfull[kb & 1]);
        flags[1] = kb + 1;
      }
    }
  } else if (warp == 9) {
    if (lane == 0) {
      // S(it) = W_rt W_blk(it)^T (six terms, two halves) into TMEM buffer it % 2
      const uint32_t id1 = idesc_bf16_f32(kTileM, kTileK);
      const uint32_t ab = smem_u32(smem + Lo.a), bb = smem_u32(smem + Lo.b);
      bool ok = mbar_wait(afull, 0);
      if (!ok) atomicExch(&flags[0], 1);
      for (int it = 0; ok && it < nk; ++it) {
        if (!mbar_wait(wfull, it & 1) || (it >= 2 && !mbar_wait(&efree[it & 1], ((it - 2) >> 1) & 1))) {
          atomicExch(&flags[0], 1);
          break;
        }
        if (*reinterpret_cast<volatile int*>(&flags[0])) break;
        tc_fence_after();
        const uint32_t ts = tmem + (uint32_t)((it & 1) * kTileK);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const uint64_t a0 = sw128_desc(ab + h * kFHalf), a1 = sw128_desc(ab + (2 + h) * kFHalf),
                         a2 = sw128_desc(ab + (4 + h) * kFHalf);
          const uint64_t b0 = sw128_desc(bb + h * kFWHalf), b1 = sw128_desc(bb + (2 + h) * kFWHalf),
                         b2 = sw128_desc(bb + (4 + h) * kFWHalf);
#pragma unroll
          for (int k = 0; k < 4; ++k) {   // K = 16 per MMA: 32 bytes along the swizzled row
            if (16 * (4 * h + k) >= N) break;   // members past N are zero in both operands
            mma_bf16(ts, a0 + 2 * k, b0 + 2 * k, id1, (h | k) != 0 ? 1u : 0u);
            mma_bf16(ts, a0 + 2 * k, b1 + 2 * k, id1, 1u);
            mma_bf16(ts, a1 + 2 * k, b0 + 2 * k, id1, 1u);
            mma_bf16(ts, a0 + 2 * k, b2 + 2 * k, id1, 1u);
            mma_bf16(ts, a2 + 2 * k, b0 + 2 * k, id1, 1u);
            mma_bf16(ts, a1 + 2 * k, b1 + 2 * k, id1, 1u);
          }
        }
        mma_commit(&g1done[it & 1]);
      }
      mma_commit(accf);
    }
  } else {
    // warps 0-7: row `row` of the tile (TMEM lane) and the block's columns half * 32 .. half * 32 + 31
    const int quad = warp & 3, half = warp >> 2;
    const int row = quad * 32 + lane;
    const int64_t a = rt * kTileM + row;
    const int4 ca = pr.st_xyz[a];
    const bool arow = ca.w >= 0;
    const float ra = pr.rinvp[a];
    const int offy = (int)g.ext[0], offz = (int)(g.ext[0] + g.ext[1]);
    const uint32_t trow = (uint32_t)(quad * 32) << 16;
    double rowsum = 0.0;
    int nnz = 0;
    // exits are warp-uniform: the TMEM loads below are warp-collective
    for (int kb = 0; kb < nk; ++kb) {
      const int bf = kb & 1, ph = (kb >> 1) & 1;
      if (!__all_sync(0xffffffffu, mbar_wait(&g1done[bf], ph) && mbar_wait(&xfull[bf], ph))) {
        atomicExch(&flags[0], 1);
        break;
      }
      tc_fence_after();
      float sv[32];
#pragma unroll
      for (int c0 = 0; c0 < 32; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + (uint32_t)(bf * kTileK) + trow + (uint32_t)(half * 32 + c0), v);
#pragma unroll
        for (int i = 0; i < 16; ++i) sv[c0 + i] = v[i];
      }
      const unsigned char* side = smem + Lo.side + bf * kFSide;
      const int4* cs = reinterpret_cast<const int4*>(side);
      const float* rb = reinterpret_cast<const float*>(side + kTileK * 16);
      const int64_t t = t0 + kb;
      const int64_t b0 = (int64_t)pr.colblk[t] * kTileK + half * 32;   // tile position of column 0
      float rs = 0.f;
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const int4 ob = cs[half * 32 + c];
        const float r2 = (d2[abs(ca.x - ob.x)] + d2[offy + abs(ca.y - ob.y)]) + d2[offz + abs(ca.z - ob.z)];
        const bool in = r2 < 4.f;
        const float z = r2 > 0.f ? r2 * rsqrtf(r2) : 0.f;
        const float v = in ? gc_select(z) * sv[c] * ra * rb[half * 32 + c] : 0.f;
        sv[c] = v;
        rs += fabsf(v);
        nnz += (in && arow && ob.w >= 0) ? 1 : 0;
        if (arow && b0 + c == a) {   // the diagonal entry
          atomic_min_nonneg(&pr.scal[1], (double)v);
          atomicAdd(&pr.scal[4], (double)v);
        }
      }
      rowsum += (double)rs;
      uint4* hd = reinterpret_cast<uint4*>(pr.Chi + (t * kTileM + row) * kTileK + half * 32);
      uint4* ld = reinterpret_cast<uint4*>(pr.Clo + (t * kTileM + row) * kTileK + half * 32);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint4 hi, lo;
        split8x2(sv + 8 * q, hi, lo);
        hd[q] = hi;
        ld[q] = lo;
      }
      tc_fence_before();
      mbar_arrive(&efree[bf]);
    }
    // row sums of |C| (half 1 hands its part to half 0) and the count of nonzeros
    if (half == 1) red[row] = rowsum;
    asm volatile("bar.sync 1, 256;" ::: "memory");   // the eight epilogue warps
    if (half == 0 && arow && *reinterpret_cast<volatile int*>(&flags[0]) == 0)
      atomic_max_nonneg(&pr.scal[0], rowsum + red[row]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nnz += __shfl_xor_sync(0xffffffffu, nnz, o);
    if (lane == 0 && nnz) atomicAdd(&pr.scal[3], (double)nnz);   // an exact integer count in FP64
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0 && flags[0]) {
    // wait (bounded) for the copies and MMAs still in flight before the CTA's
    // shared and tensor memory go away: each barrier has at most its last
    // issued phase outstanding
    const int nw = flags[1];
    if (flags[2]) mbar_wait(afull, 0);
    if (nw > 0) mbar_wait(wfull, (nw - 1) & 1);
    for (int b = 0; b < 2; ++b) {
      const int cnt = nw > b ? (nw - b + 1) / 2 : 0;   // side loads into buffer b
      if (cnt > 0) mbar_wait(&xfull[b], (cnt - 1) & 1);
    }
    mbar_wait(accf, 0);
    atomicOr(&pr.status[0], kStatTimeout);
  }
  __syncthreads();
  if (warp == 8) tmem_dealloc(tmem, 128);
}

}  // namespace

// Forms the C blocks of every problem of the table on the tensor cores (all
// BF16 with N <= kStK, grid extents summing to at most kFD2); returns -1
// without launching anything when one of them does not qualify or the device
// cannot be configured, and the caller runs the CUDA-core kernel instead.
int launch_tile_form_mma(const ProblemTable& tab, const ProblemDev* dtab, cudaStream_t st) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  size_t smax = 0;
  int64_t nmax = 0;
  for (int i = 0; i < tab.count; ++i) {
    const ProblemDev& p = tab.p[i];
    const int64_t next = p.grid.ext[0] + p.grid.ext[1] + p.grid.ext[2];
    if (p.precision != 2 || !p.st_W || !p.st_xyz || p.N > kStK || next > kFD2) return -1;
    const size_t need = 1024 + fm_layout((int)next).total;
    smax = need > smax ? need : smax;
    nmax = p.d_pad * kStK > nmax ? p.d_pad * kStK : nmax;
  }
  if (smax > (size_t)optin) return -1;
  CUtensorMap maps[kMaxProblems][3];
  for (int i = 0; i < tab.count; ++i) {
    const ProblemDev& p = tab.p[i];
    const uint64_t dp = (uint64_t)p.d_pad;
    for (int pl = 0; pl < 3; ++pl)
      if (!encode_bf16(&maps[i][pl], p.st_W + pl * dp * kStK, kStK, dp, kStK, kTileK)) return -1;
  }
  static thread_local int raised_dev = -1;
  static thread_local size_t raised_bytes = 0;
  if (raised_dev != dev || raised_bytes < smax) {
    if (cudaFuncSetAttribute(k_tile_form_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax) !=
        cudaSuccess) {
      cudaGetLastError();
      return -1;
    }
    raised_dev = dev;
    raised_bytes = smax;
  }
  k_tile_form_prep<<<dim3((unsigned)((nmax + 255) / 256), tab.count), 256, 0, st>>>(dtab);
  note_launches(1);
  for (int i = 0; i < tab.count; ++i) {
    const ProblemDev& p = tab.p[i];
    if (p.nrt < 1) continue;
    k_tile_form_mma<<<(unsigned)p.nrt, kFmThreads, smax, st>>>(maps[i][0], maps[i][1], maps[i][2], dtab + i);
    note_launches(1);
  }
  return cudaGetLastError() == cudaSuccess ? 0 : INFO_ESRF_ERR_CUDA;
}

}  // namespace infoesrf
