// a10, BF16 path, on the fifth-generation tensor cores: the state update
//     z_a(x) = z(x) - sum_b Sxh(x, b) vbar_b,  Sxh(x, b) = GC(r_xb) (z_x . w_b)
// (Sec. 2.3 model-space localization with Eq. localized_state_covar; vbar
// from the quadrature accumulation).  Per state tile (128 consecutive grid
// points) and stored column block (64 tile-ordered observations within the
// Gaspari-Cohn support), two dense products:
//     S   = Z_tile W_blk^T        128 x 64, K = members (padded to kStK)
//     acc += (GC o S) Vbar_blk    128 x NV, K = 64 observations (the members' columns)
// as tcgen05.mma kind::f16 with FP32 accumulation in tensor memory.
// Precision: z . w sums members' products of both signs, so S is formed from
// three BF16 planes of each operand (h = bf16(a), m = bf16(a - h),
// l = bf16(a - h - m)) in the six terms hh, hm, mh, hl, lh, mm (about 2^-26
// relative per product); the second product takes two planes (hi, lo) in three
// terms.  The mean column, whose sum cancels far more (the innovation
// weights), is accumulated per thread in FP32 from the weighted S in registers
// and across blocks in FP64.
//
// CTA of 18 warps per state tile: warp 16 lane 0 loads W_blk and Vbar_blk^T with
// 2-D TMA (128-byte swizzle) and the block's coordinates and mean-column values
// with bulk copies; warp 17 lane 0 issues the MMAs; warps 0-15 (four per TMEM
// lane quadrant, one state point and 16 of the block's observations per thread)
// read S from tensor memory, apply the Gaspari-Cohn weights, add the mean
// column's terms, split S and write it to shared memory as the A operand of the
// second product, and finally write A_a and mu_a.  Pipelined: S has two TMEM
// buffers and W is free once the first product of its block is done, so the
// loads and the first product of block b + 1 run during the weighting of
// block b; the coordinates have two buffers, Vbar^T and the S planes one.  Z_tile is split and placed in shared memory once
// per CTA.  All waits are bounded (kStatTimeout).
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "info_esrf.h"
#include "internal.h"
#include "tile_mma.cuh"

namespace infoesrf {

namespace {

constexpr int kEpiWarps = 16;                  // epilogue warps: four per TMEM lane quadrant
constexpr int kEpiCols = kTileK * 4 / kEpiWarps;   // columns of S per epilogue thread (16)
constexpr int kLoadWarp = kEpiWarps, kMmaWarp = kEpiWarps + 1;
constexpr int kStThreads = (kEpiWarps + 2) * 32;
constexpr int kSideBytes = kTileK * 16 + kTileK * 4;   // a block's grid coordinates and mean-column values
constexpr int kHalf = kTileM * 64 * 2;         // one 64-member half of a 128-row BF16 operand: 16 KB
constexpr int kWHalf = kTileK * 64 * 2;        // one 64-member half of the W block: 8 KB

struct StLayout {
  int NV;
  uint32_t z, s, stage, w_bytes, v_bytes, side, ctrl, d2, total;
};

__host__ __device__ inline StLayout st_layout(int NV, int nd2) {
  StLayout L;
  L.NV = NV;
  L.z = 0;                                         // Z planes h, m, l (two halves each)
  L.s = 6 * kHalf;                                 // S planes hi, lo
  L.w_bytes = 6 * kWHalf;                          // W planes h, m, l (two halves each)
  L.v_bytes = 2 * (uint32_t)NV * 128;              // Vbar^T hi, lo: NV rows of 64 observations
  L.stage = L.s + 2 * kHalf;                       // W, then Vbar^T, then two side buffers
  L.side = L.stage + L.w_bytes + L.v_bytes;
  L.ctrl = L.side + 2 * kSideBytes;
  L.d2 = L.ctrl + 256;
  L.total = L.d2 + 4 * (uint32_t)nd2;
  return L;
}

// Operand planes of the finish in tile order: W in three planes (members
// padded to kStK), the members' columns of Vbar^T in two (padded to NV), the
// mean column of Vbar in FP32, and the grid coordinates of each tile position.
__global__ void k_tile_state_prep(const ProblemDev* tab) {
  const ProblemDev& pr = tab[blockIdx.y];
  if (pr.precision != 2 || !pr.st_W) return;
  const int64_t N = pr.N, N1 = N + 1, dp = pr.d_pad, NV = pr.st_NV;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nw = dp * kStK, nv = NV * dp;
  const float* Vt = reinterpret_cast<const float*>(pr.VbarT);
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
  if (i < nv) {
    const int64_t m = i / dp, a = i % dp;
    const int32_t src = a < pr.d ? pr.tpos_src[a] : -1;
    const float v = (src >= 0 && m < N) ? Vt[(int64_t)src * N1 + m] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    pr.st_V[i] = h;
    pr.st_V[nv + i] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
  if (i < dp) {
    const int32_t src = i < pr.d ? pr.tpos_src[i] : -1;
    int4 c = make_int4(0, 0, 0, -1);
    if (src >= 0) {
      const Coord3 cc = flat_to_coord(pr.grid, pr.obs[src]);
      c = make_int4((int)cc.x, (int)cc.y, (int)cc.z, 1);
    }
    pr.st_xyz[i] = c;
    pr.st_vm[i] = src >= 0 ? Vt[(int64_t)src * N1 + N] : 0.f;
  }
}

constexpr int kD2St = 4096;   // distance-table entries staged in shared memory (sum of the extents)

__global__ void __launch_bounds__(kStThreads, 1)
    k_tile_state_mma(const __grid_constant__ CUtensorMap map_w0, const __grid_constant__ CUtensorMap map_w1,
                     const __grid_constant__ CUtensorMap map_w2, const __grid_constant__ CUtensorMap map_vh,
                     const __grid_constant__ CUtensorMap map_vl, const ProblemDev* dpr) {
  const ProblemDev& pr = *dpr;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                         ~static_cast<uintptr_t>(1023));
  const GridDev& g = pr.grid;
  const int64_t next = g.ext[0] + g.ext[1] + g.ext[2];
  // the distance table in shared memory (the launcher checks next <= kD2St)
  const int NV = pr.st_NV;
  const StLayout Lo = st_layout(NV, (int)next);
  // Barriers, one phase per block b unless noted.  A waiter never falls two
  // phases behind: each next completion depends on the waiter having passed.
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + Lo.ctrl);
  uint64_t* wfull = bar + 0;     // W(b) landed                                  (MMA)
  uint64_t* vfull = bar + 1;     // Vbar^T(b) landed                             (MMA)
  uint64_t* xfull = bar + 2;     // [2] side buffer b % 2 landed, phase b / 2    (epilogue)
  uint64_t* g1done = bar + 4;    // [2] S(b) in TMEM buffer b % 2, phase b / 2   (epilogue, loads)
  uint64_t* g2done = bar + 6;    // second product of b done: Vbar^T and the S planes free (loads, epilogue)
  uint64_t* sready = bar + 7;    // S planes of b written, TMEM buffer b % 2 read (MMA; every epilogue thread)
  uint64_t* accf = bar + 8;      // every MMA done
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 9);
  int* flags = reinterpret_cast<int*>(tslot + 1);   // [0] abort, [1] W/side loads issued, [2] Vbar loads, [3] skip
  float* d2 = reinterpret_cast<float*>(smem + Lo.d2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t st = blockIdx.x;
  if (st >= pr.nst) return;
  // a timeout anywhere in the grid stops the CTAs that have not started (uniform per CTA)
  if (tid == 0) flags[3] = (pr.status[0] & (kStatTimeout | kStatTileOverflow)) ? 1 : 0;
  __syncthreads();
  if (flags[3]) return;
  const int t0 = pr.st_rowptr[st], nk = pr.st_rowptr[st + 1] - t0;
  const int64_t x0 = st * kTileM;
  const int N = (int)pr.N;
  if (tid == 0) {
    for (int i = 0; i < 9; ++i) mbar_init(bar + i, i == 7 ? kEpiWarps * 32 : 1);
    flags[0] = 0;
    flags[1] = 0;
    flags[2] = 0;
    fence_mbar_init();
    tma_prefetch_map(&map_w0);
    tma_prefetch_map(&map_w1);
    tma_prefetch_map(&map_w2);
    tma_prefetch_map(&map_vh);
    tma_prefetch_map(&map_vl);
  }
  if (warp == kLoadWarp) tmem_alloc(tslot, 256);
  // Z_tile as the A operand of the first product: one state point per thread,
  // members split into three BF16 planes, 128-byte-swizzled 64-member halves
  if (tid < kTileM) {   // warps 0-3
    const int64_t x = x0 + tid;
    const float* Zt = reinterpret_cast<const float*>(pr.Zt);
#pragma unroll 1
    for (int chunk = 0; chunk < kStK / 8; ++chunk) {
      float v[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int k = 8 * chunk + i;
        v[i] = (x < pr.n && k < N) ? Zt[x * N + k] : 0.f;
      }
      uint4 pl[3];
      split8<3>(v, pl);
      const int half = chunk >> 3;
      const uint32_t off = sw128_off(tid, chunk & 7);
#pragma unroll
      for (int p = 0; p < 3; ++p) *reinterpret_cast<uint4*>(smem + Lo.z + (2 * p + half) * kHalf + off) = pl[p];
    }
  }
  for (int64_t e = tid; e < next; e += blockDim.x) d2[e] = (float)pr.d2tab[e];
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t t_s = tmem, t_acc = tmem + 2 * kTileK;   // S buffers at columns 0 and 64, acc at 128

  if (warp == kLoadWarp) {
    if (lane == 0) {
      // loads: W_blk (three planes, two 64-member halves each) with the block's
      // coordinates and mean-column values, then Vbar_blk^T (hi, lo)
      int kb = 0, kv = 0;
      for (; kb < nk; ++kb) {
        // W is free once the first product of kb - 1 is done; side buffer kb % 2 once the
        // weighting of kb - 2 is, which the wait for Vbar below covered in the previous step
        if (kb >= 1 && !mbar_wait(&g1done[(kb - 1) & 1], ((kb - 1) >> 1) & 1)) {
          atomicExch(&flags[0], 1);
          break;
        }
        if (*reinterpret_cast<volatile int*>(&flags[0])) break;
        const int row = pr.st_colblk[t0 + kb] * kTileK;
        unsigned char* wp = smem + Lo.stage;
        mbar_arrive_expect_tx(wfull, Lo.w_bytes);
        tma_load_2d(wp, &map_w0, wfull, 0, row);
        tma_load_2d(wp + kWHalf, &map_w0, wfull, 64, row);
        tma_load_2d(wp + 2 * kWHalf, &map_w1, wfull, 0, row);
        tma_load_2d(wp + 3 * kWHalf, &map_w1, wfull, 64, row);
        tma_load_2d(wp + 4 * kWHalf, &map_w2, wfull, 0, row);
        tma_load_2d(wp + 5 * kWHalf, &map_w2, wfull, 64, row);
        unsigned char* xp = smem + Lo.side + (kb & 1) * kSideBytes;
        mbar_arrive_expect_tx(&xfull[kb & 1], kSideBytes);
        bulk_load(xp, pr.st_xyz + row, kTileK * 16, &xfull[kb & 1]);
        bulk_load(xp + kTileK * 16, pr.st_vm + row, kTileK * 4, &xfull[kb & 1]);
        flags[1] = kb + 1;
        // Vbar^T is free once the second product of kb - 1 is done
        if (kb >= 1 && !mbar_wait(g2done, (kb - 1) & 1)) {
          atomicExch(&flags[0], 1);
          break;
        }
        unsigned char* vp = smem + Lo.stage + Lo.w_bytes;
        mbar_arrive_expect_tx(vfull, Lo.v_bytes);
        tma_load_2d(vp, &map_vh, vfull, row, 0);
        tma_load_2d(vp + NV * 128, &map_vl, vfull, row, 0);
        kv = kb + 1;
        flags[2] = kv;
      }
    }
  } else if (warp == kMmaWarp) {
    if (lane == 0) {
      // MMAs, software-pipelined: the first product of it, then the second of it - 1
      //   S(it) = Z W(it)^T (six terms, two halves) into TMEM buffer it % 2
      //   acc += (GC o S(it - 1)) Vbar(it - 1) (three terms)
      const uint32_t id1 = idesc_bf16_f32(kTileM, kTileK), id2 = idesc_bf16_f32(kTileM, NV);
      const uint32_t zb = smem_u32(smem + Lo.z), sb = smem_u32(smem + Lo.s);
      const uint32_t wb = smem_u32(smem + Lo.stage), vb = wb + Lo.w_bytes;
      for (int it = 0; it <= nk; ++it) {
        if (it < nk) {
          if (!mbar_wait(wfull, it & 1)) {
            atomicExch(&flags[0], 1);
            break;
          }
          if (*reinterpret_cast<volatile int*>(&flags[0])) break;
          tc_fence_after();
          const uint32_t ts = t_s + (uint32_t)((it & 1) * kTileK);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const uint64_t z0 = sw128_desc(zb + h * kHalf), z1 = sw128_desc(zb + (2 + h) * kHalf),
                           z2 = sw128_desc(zb + (4 + h) * kHalf);
            const uint64_t w0 = sw128_desc(wb + h * kWHalf), w1 = sw128_desc(wb + (2 + h) * kWHalf),
                           w2 = sw128_desc(wb + (4 + h) * kWHalf);
#pragma unroll
            for (int k = 0; k < 4; ++k) {   // K = 16 per MMA: 32 bytes along the swizzled row
              if (16 * (4 * h + k) >= N) break;   // members past N are zero in both operands
              mma_bf16(ts, z0 + 2 * k, w0 + 2 * k, id1, (h | k) != 0 ? 1u : 0u);
              mma_bf16(ts, z0 + 2 * k, w1 + 2 * k, id1, 1u);
              mma_bf16(ts, z1 + 2 * k, w0 + 2 * k, id1, 1u);
              mma_bf16(ts, z0 + 2 * k, w2 + 2 * k, id1, 1u);
              mma_bf16(ts, z2 + 2 * k, w0 + 2 * k, id1, 1u);
              mma_bf16(ts, z1 + 2 * k, w1 + 2 * k, id1, 1u);
            }
          }
          mma_commit(&g1done[it & 1]);
        }
        if (it >= 1) {
          const int kb = it - 1;
          if (!mbar_wait(sready, kb & 1) || !mbar_wait(vfull, kb & 1)) {
            atomicExch(&flags[0], 1);
            break;
          }
          tc_fence_after();
          const uint64_t sh = sw128_desc(sb), sl = sw128_desc(sb + kHalf);
          const uint64_t vh = sw128_desc(vb), vl = sw128_desc(vb + NV * 128);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            mma_bf16(t_acc, sh + 2 * k, vh + 2 * k, id2, (kb | k) != 0 ? 1u : 0u);
            mma_bf16(t_acc, sh + 2 * k, vl + 2 * k, id2, 1u);
            mma_bf16(t_acc, sl + 2 * k, vh + 2 * k, id2, 1u);
          }
          mma_commit(g2done);
        }
      }
      mma_commit(accf);
    }
  } else {
    // warps 0-15: state point `row` (TMEM lane) and observations grp * 16 .. grp * 16 + 15
    const int quad = warp & 3, grp = warp >> 2;
    const int row = quad * 32 + lane;
    const int64_t x = x0 + row;
    const bool xin = x < pr.n;
    const Coord3 cx = flat_to_coord(g, xin ? x : 0);
    const int cxi = (int)cx.x, cyi = (int)cx.y, czi = (int)cx.z;
    // offsets of the y and z axes in the distance table; distance 0 has entry 0, so an axis of
    // extent 1 adds nothing
    const int offy = (int)g.ext[0], offz = (int)(g.ext[0] + g.ext[1]);
    const uint32_t trow = (uint32_t)(quad * 32) << 16;
    unsigned char* s_hi = smem + Lo.s;
    double macc = 0.0;   // this group's part of the mean column, FP64 across blocks
    // exits are warp-uniform: the TMEM loads below are warp-collective
    for (int kb = 0; kb < nk; ++kb) {
      const int bf = kb & 1, ph = (kb >> 1) & 1;
      if (!__all_sync(0xffffffffu, mbar_wait(&g1done[bf], ph) && mbar_wait(&xfull[bf], ph))) {
        atomicExch(&flags[0], 1);
        break;
      }
      tc_fence_after();
      const unsigned char* side = smem + Lo.side + bf * kSideBytes;
      const int4* cs = reinterpret_cast<const int4*>(side) + grp * kEpiCols;
      const float* vm = reinterpret_cast<const float*>(side + kTileK * 16) + grp * kEpiCols;
      float sv[kEpiCols];
      tmem_ld16(t_s + (uint32_t)(bf * kTileK) + trow + (uint32_t)(grp * kEpiCols), sv);
      // Gaspari-Cohn weights of the pairs (state point, observation), and the mean column
      float mb = 0.f;
#pragma unroll
      for (int c = 0; c < kEpiCols; ++c) {
        const int4 ob = cs[c];
        const float r2 = (d2[abs(cxi - ob.x)] + d2[offy + abs(cyi - ob.y)]) + d2[offz + abs(czi - ob.z)];
        const float z = r2 > 0.f ? r2 * rsqrtf(r2) : 0.f;
        sv[c] = (ob.w >= 0 && r2 < 4.f) ? gc_select(z) * sv[c] : 0.f;
        mb = fmaf(sv[c], vm[c], mb);
      }
      macc += (double)mb;
      // the second product of the previous block has read the S planes
      if (kb > 0 && !__all_sync(0xffffffffu, mbar_wait(g2done, (kb - 1) & 1))) {
        atomicExch(&flags[0], 1);
        break;
      }
#pragma unroll
      for (int chunk = 0; chunk < kEpiCols / 8; ++chunk) {
        uint4 hi, lo;
        split8x2(sv + 8 * chunk, hi, lo);
        const uint32_t off = sw128_off(row, grp * (kEpiCols / 8) + chunk);
        *reinterpret_cast<uint4*>(s_hi + off) = hi;
        *reinterpret_cast<uint4*>(s_hi + kHalf + off) = lo;
      }
      fence_proxy_async();
      tc_fence_before();
      mbar_arrive(sready);
    }
    const bool got = mbar_wait(accf, 0);
    if (!got) atomicExch(&flags[0], 1);
    tc_fence_after();
    const bool ok = __all_sync(0xffffffffu, got && *reinterpret_cast<volatile int*>(&flags[0]) == 0);
    const double mu = xin ? pr.mu[x] : 0.0;
    for (int c0 = grp * 16; c0 < NV; c0 += 16 * (kEpiWarps / 4)) {   // the groups take alternate 16-column chunks
      float v[16];
      if (nk > 0 && ok) {
        tmem_ld16(t_acc + trow + (uint32_t)c0, v);
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = 0.f;
      }
      if (!xin || !ok) continue;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int col = c0 + i;
        const double inc = (double)v[i];
        if (col < N && pr.do_pert)
          pr.A_a[(int64_t)col * pr.n + x] = (pr.X[(int64_t)col * pr.n + x] - mu) - pr.sqrt_nm1 * inc;
      }
    }
    // the mean column: groups 1.. hand their parts to group 0 (the S planes are free now)
    double* red = reinterpret_cast<double*>(s_hi);   // [groups - 1][128]
    if (grp > 0) red[(grp - 1) * kTileM + row] = macc;
    asm volatile("bar.sync 1, %0;" ::"r"(kEpiWarps * 32) : "memory");   // the epilogue warps
    if (grp == 0 && xin && ok && pr.do_mean) {
      double t = macc;
      for (int q = 1; q < kEpiWarps / 4; ++q) t += red[(q - 1) * kTileM + row];
      pr.mu_a[x] = mu + t;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0 && flags[0]) {
    // wait (bounded) for the loads still in flight before the CTA's shared memory goes away:
    // each barrier has at most its last issued phase outstanding
    const int nw = flags[1], nv = flags[2];
    if (nw > 0) mbar_wait(wfull, (nw - 1) & 1);
    if (nv > 0) mbar_wait(vfull, (nv - 1) & 1);
    for (int b = 0; b < 2; ++b) {
      const int cnt = nw > b ? (nw - b + 1) / 2 : 0;   // side loads into buffer b
      if (cnt > 0) mbar_wait(&xfull[b], (cnt - 1) & 1);
    }
    atomicOr(&pr.status[0], kStatTimeout);
  }
  __syncthreads();
  if (warp == kLoadWarp) tmem_dealloc(tmem, 256);
}

}  // namespace

}  // namespace infoesrf

namespace infoesrf {

// Launches the tensor-core state update for every problem of the table (all
// BF16 with N <= kStK, grid extents summing to at most kD2St, and shared
// memory for one block's operands); returns -1
// without launching anything when one of them does not qualify or the device
// cannot be configured, and the caller runs the CUDA-core kernel instead.
int launch_tile_state_mma(const ProblemTable& tab, const ProblemDev* dtab, cudaStream_t st) {
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
    if (p.precision != 2 || !p.st_W || p.N > kStK || p.st_NV > kStK || p.st_NV < 16 || next > kD2St) return -1;
    const size_t need = 1024 + st_layout(p.st_NV, (int)next).total;
    smax = need > smax ? need : smax;
    const int64_t np = std::max<int64_t>(p.d_pad * kStK, (int64_t)p.st_NV * p.d_pad);
    nmax = np > nmax ? np : nmax;
  }
  if (smax > (size_t)optin) return -1;
  CUtensorMap maps[kMaxProblems][5];
  for (int i = 0; i < tab.count; ++i) {
    const ProblemDev& p = tab.p[i];
    const uint64_t dp = (uint64_t)p.d_pad, NV = (uint64_t)p.st_NV;
    if (!encode_bf16(&maps[i][0], p.st_W, kStK, dp, kStK, kTileK) ||
        !encode_bf16(&maps[i][1], p.st_W + dp * kStK, kStK, dp, kStK, kTileK) ||
        !encode_bf16(&maps[i][2], p.st_W + 2 * dp * kStK, kStK, dp, kStK, kTileK) ||
        !encode_bf16(&maps[i][3], p.st_V, dp, NV, dp, (uint32_t)NV) ||
        !encode_bf16(&maps[i][4], p.st_V + NV * dp, dp, NV, dp, (uint32_t)NV))
      return -1;
  }
  static thread_local int raised_dev = -1;
  static thread_local size_t raised_bytes = 0;
  if (raised_dev != dev || raised_bytes < smax) {
    if (cudaFuncSetAttribute(k_tile_state_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax) !=
        cudaSuccess) {
      cudaGetLastError();
      return -1;
    }
    raised_dev = dev;
    raised_bytes = smax;
  }
  k_tile_state_prep<<<dim3((unsigned)((nmax + 255) / 256), tab.count), 256, 0, st>>>(dtab);
  note_launches(1);
  for (int i = 0; i < tab.count; ++i) {
    const ProblemDev& p = tab.p[i];
    if (p.nst < 1) continue;
    k_tile_state_mma<<<(unsigned)p.nst, kStThreads, smax, st>>>(maps[i][0], maps[i][1], maps[i][2], maps[i][3],
                                                                maps[i][4], dtab + i);
    note_launches(1);
  }
  return cudaGetLastError() == cudaSuccess ? 0 : INFO_ESRF_ERR_CUDA;
}

}  // namespace infoesrf
