// Set-up and finish of the BF16 block-tile path (precision 2).
//
// a1  Tile order of the observations: every observation gets the rank of the
//     Morton code of its grid point (axes of extent 1 skipped), by a bitonic
//     sort of (code, index) pairs.  Codes of distinct grid points differ, so
//     the order is unique.  128 consecutive positions form a row tile, 64 a
//     column block; on 2-D and layered grids both are compact patches, on
//     1-D grids the order is the natural one.  W and R^-1/2 are copied into
//     this order (Wp, rinvp), zero at the padding positions d .. d_pad - 1.
// a5  Block pattern: the bounding box of each column block; a (row tile,
//     column block) pair is stored when the boxes come within the
//     Gaspari-Cohn support (r < 2, Sec. 2.3, Sec. 5.2).  Box distances are
//     lower bounds of every pair distance inside, so every entry with
//     GC(r) > 0 lies in a stored block and all others are exact zeros.  The
//     same test pairs state tiles (128 consecutive grid points) with column
//     blocks for the state update.
//     C entries: C(a, b) = GC(r_ab) (w_a . w_b) R_a^-1/2 R_b^-1/2
//     (Sec. 3.1 with Eq. localized_state_covar), in FP32, stored as
//     hi = bf16(C), lo = bf16(C - hi).  The same pass takes the Gershgorin
//     bound of C, min_a C(a, a) and sum_a C(a, a) (App. D, App. E).
// a4  Ritz stage: C X for the l test vectors of the randomized eigensolver,
//     from the stored blocks (hi + lo in FP32) on the CUDA cores.
// a9  vbar = R^-1/2 sum_q p_q u_q from the tile-ordered iterates (FP64 sum).
// a10 z_a = z - Sxh vbar, Sxh(x, b) = GC(r_xb) (z_x . w_b): per state tile
//     and stored column block, S = (GC o Z W^T) in shared memory, then S Vbar.
#include <cuda_bf16.h>

#include "common.cuh"
#include "internal.h"

namespace infoesrf {

namespace {

__device__ __forceinline__ uint64_t morton_code(const GridDev& g, const Coord3& c) {
  const uint64_t v[3] = {(uint64_t)c.x, (uint64_t)c.y, (uint64_t)c.z};
  int bits[3];
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) bits[ax] = g.ext[ax] > 1 ? 64 - __clzll((long long)(g.ext[ax] - 1)) : 0;
  uint64_t key = 0;
  int out = 0;
  for (int b = 0; b < 64 && out < 64; ++b) {
    bool any = false;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      if (b < bits[ax] && out < 64) {
        key |= ((v[ax] >> b) & 1ull) << out;
        ++out;
        any = true;
      }
    }
    if (!any) break;
  }
  return key;
}

__global__ void k_tile_keys(const ProblemDev* tab) {
  const ProblemDev& pr = tab[blockIdx.y];
  if (pr.precision != 2) return;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= pr.nsort) return;
  if (i < pr.d) {
    int64_t o = pr.obs[i];
    o = o < 0 ? 0 : (o >= pr.n ? pr.n - 1 : o);   // bad indices are reported by the observe kernel
    pr.skey[i] = morton_code(pr.grid, flat_to_coord(pr.grid, o));
    pr.sidx[i] = (int32_t)i;
  } else {
    pr.skey[i] = ~0ull;
    pr.sidx[i] = -1;
  }
}

__device__ __forceinline__ void cmp_swap(uint64_t& ka, int32_t& ia, uint64_t& kb, int32_t& ib, bool up) {
  if ((ka > kb) == up) {
    const uint64_t tk = ka;
    ka = kb;
    kb = tk;
    const int32_t ti = ia;
    ia = ib;
    ib = ti;
  }
}

// Bitonic steps with stride j >= 1024 (one compare-exchange per thread).
__global__ void k_bitonic_global(const ProblemDev* tab, int64_t k, int64_t j) {
  const ProblemDev& pr = tab[blockIdx.y];
  if (pr.precision != 2 || k > pr.nsort) return;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= pr.nsort / 2) return;
  const int64_t a = ((t & ~(j - 1)) << 1) | (t & (j - 1));
  const int64_t b = a + j;
  cmp_swap(pr.skey[a], pr.sidx[a], pr.skey[b], pr.sidx[b], (a & k) == 0);
}

// All steps with stride j < 1024 of sequence sizes k in [k_lo, k_hi], on
// 1024-element chunks in shared memory (512 threads).
__global__ void __launch_bounds__(512) k_bitonic_chunk(const ProblemDev* tab, int64_t k_lo, int64_t k_hi) {
  const ProblemDev& pr = tab[blockIdx.y];
  if (pr.precision != 2) return;
  const int64_t base = (int64_t)blockIdx.x * 1024;
  if (base >= pr.nsort) return;
  __shared__ uint64_t sk[1024];
  __shared__ int32_t si[1024];
  for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
    sk[e] = pr.skey[base + e];
    si[e] = pr.sidx[base + e];
  }
  __syncthreads();
  for (int64_t k = k_lo; k <= k_hi && k <= pr.nsort; k <<= 1) {
    for (int64_t j = (k >> 1) < 512 ? (k >> 1) : 512; j >= 1; j >>= 1) {
      const int t = threadIdx.x;
      const int a = ((t & ~(int)(j - 1)) << 1) | (t & (int)(j - 1));
      const int b = a + (int)j;
      cmp_swap(sk[a], si[a], sk[b], si[b], ((base + a) & k) == 0);
      __syncthreads();
    }
  }
  for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
    pr.skey[base + e] = sk[e];
    pr.sidx[base + e] = si[e];
  }
}

// Tile-ordered copies of W and R^-1/2, and both directions of the permutation.
__global__ void k_tile_order(const ProblemDev* tab) {
  const ProblemDev& pr = tab[blockIdx.y];
  if (pr.precision != 2) return;
  const int64_t N = pr.N;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= pr.d_pad * N) return;
  const int64_t a = i / N, k = i % N;
  const int32_t src = a < pr.d ? pr.sidx[a] : -1;
  const float* W = reinterpret_cast<const float*>(pr.W);
  pr.Wp[i] = src >= 0 ? W[(int64_t)src * N + k] : 0.f;
  if (k == 0) {
    pr.tpos_src[a] = src;
    pr.rinvp[a] = src >= 0 ? (float)pr.rinv[src] : 0.f;
    if (src >= 0) pr.obs_tpos[src] = (int32_t)a;
  }
}

struct Box {
  int32_t lo[3], hi[3];
};

__device__ __forceinline__ Box empty_box() {
  Box b;
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    b.lo[ax] = INT32_MAX;
    b.hi[ax] = INT32_MIN;
  }
  return b;
}

__device__ __forceinline__ void box_add(Box& b, const Coord3& c) {
  const int32_t v[3] = {(int32_t)c.x, (int32_t)c.y, (int32_t)c.z};
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    b.lo[ax] = min(b.lo[ax], v[ax]);
    b.hi[ax] = max(b.hi[ax], v[ax]);
  }
}

__device__ __forceinline__ void box_merge(Box& b, const Box& o) {
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    b.lo[ax] = min(b.lo[ax], o.lo[ax]);
    b.hi[ax] = max(b.hi[ax], o.hi[ax]);
  }
}

__device__ __forceinline__ Box warp_box(Box b) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      b.lo[ax] = min(b.lo[ax], __shfl_xor_sync(0xffffffffu, b.lo[ax], o));
      b.hi[ax] = max(b.hi[ax], __shfl_xor_sync(0xffffffffu, b.hi[ax], o));
    }
  }
  return b;
}

__device__ __forceinline__ Box load_box(const int32_t* t) {
  Box b;
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    b.lo[ax] = t[2 * ax];
    b.hi[ax] = t[2 * ax + 1];
  }
  return b;
}

// True when some pair of points of the two boxes may be closer than the
// Gaspari-Cohn support (r < 2).  The interval gap on each axis (the nearest
// periodic image on periodic axes) bounds every pair's axis distance from
// below; the chordal distance grows with the gap.  A margin of 1e-9 keeps
// pairs at r = 2 up to rounding on the stored side.
__device__ __forceinline__ bool boxes_within_support(const GridDev& g, const Box& A, const Box& B) {
  double r2 = 0.0;
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const int64_t e = g.ext[ax];
    if (A.lo[ax] > A.hi[ax] || B.lo[ax] > B.hi[ax]) return false;   // a box without points
    if (e <= 1) continue;
    int64_t gap;
    if (g.periodic[ax]) {
      gap = INT64_MAX;
      for (int s = -1; s <= 1; ++s) {
        const int64_t lo2 = B.lo[ax] + s * e, hi2 = B.hi[ax] + s * e;
        int64_t gp = lo2 - A.hi[ax];
        const int64_t g2 = A.lo[ax] - hi2;
        gp = gp > g2 ? gp : g2;
        gp = gp > 0 ? gp : 0;
        gap = gp < gap ? gp : gap;
      }
    } else {
      int64_t gp = B.lo[ax] - A.hi[ax];
      const int64_t g2 = A.lo[ax] - B.hi[ax];
      gp = gp > g2 ? gp : g2;
      gap = gp > 0 ? gp : 0;
    }
    double dist = (double)gap;
    if (g.periodic[ax] && g.chordal) dist = ((double)e / kPi) * sin(kPi * (double)gap / (double)e);
    const double dd = dist * g.inv_c[ax];
    r2 += dd * dd;
  }
  return r2 < 4.0 * (1.0 + 1e-9);
}

// Bounding box of each column block (one warp per block).
__global__ void k_tile_boxes(const ProblemDev* tab) {
  const ProblemDev& pr = tab[blockIdx.y];
  if (pr.precision != 2) return;
  const int64_t blk = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (blk >= pr.nblk) return;
  Box b = empty_box();
  for (int e = lane; e < kTileK; e += 32) {
    const int32_t src = pr.tpos_src[blk * kTileK + e];
    if (src >= 0) box_add(b, flat_to_coord(pr.grid, pr.obs[src]));
  }
  b = warp_box(b);
  if (lane < 6) pr.tbox[blk * 6 + lane] = lane & 1 ? b.hi[lane >> 1] : b.lo[lane >> 1];
}

// Box of row tile `row` (mode 0: blocks 2 row, 2 row + 1) or of state tile
// `row` (mode 1: grid points 128 row .. 128 row + 127), by warp 0 into *out.
__device__ void row_box(const ProblemDev& pr, int mode, int64_t row, Box* out) {
  if (threadIdx.x >= 32) return;
  Box b = empty_box();
  if (mode == 0) {
    if (threadIdx.x == 0) {
      box_merge(b, load_box(pr.tbox + (2 * row) * 6));
      if (2 * row + 1 < pr.nblk) box_merge(b, load_box(pr.tbox + (2 * row + 1) * 6));
    }
  } else {
    for (int e = threadIdx.x; e < kTileM; e += 32) {
      const int64_t x = row * kTileM + e;
      if (x < pr.n) box_add(b, flat_to_coord(pr.grid, x));
    }
  }
  b = warp_box(b);
  if (threadIdx.x == 0) *out = b;
}

// Pass 0 counts the stored blocks of each row (row tiles, then state tiles);
// pass 1 writes their column blocks in increasing order at the row's offset.
// The diagonal block of a row tile is always stored (so every row tile has one).
__global__ void __launch_bounds__(256) k_tile_pattern(const ProblemDev* tab, int mode, int pass) {
  const ProblemDev& pr = tab[blockIdx.y];
  if (pr.precision != 2) return;
  const int64_t row = blockIdx.x;
  const int64_t rows = mode == 0 ? pr.nrt : pr.nst;
  if (row >= rows) return;
  if (pass == 1 && (pr.status[0] & kStatTileOverflow)) return;
  __shared__ Box rb;
  __shared__ int wcount[8];
  row_box(pr, mode, row, &rb);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int32_t* rowptr = mode == 0 ? pr.rowptr : pr.st_rowptr;
  int32_t* cols = mode == 0 ? pr.colblk : pr.st_colblk;
  int64_t written = pass == 1 ? rowptr[row] : 0;
  int64_t count = 0;
  for (int64_t b0 = 0; b0 < pr.nblk; b0 += blockDim.x) {
    const int64_t blk = b0 + threadIdx.x;
    bool keep = false;
    if (blk < pr.nblk) {
      keep = boxes_within_support(pr.grid, rb, load_box(pr.tbox + blk * 6));
      if (mode == 0 && blk == 2 * row) keep = true;
    }
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) wcount[warp] = __popc(m);
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < 8; ++w) {
      before += w < warp ? wcount[w] : 0;
      total += wcount[w];
    }
    if (pass == 1 && keep) cols[written + count + before + __popc(m & ((1u << lane) - 1u))] = (int32_t)blk;
    count += total;
    __syncthreads();
  }
  if (pass == 0 && threadIdx.x == 0) pr.tcount[(mode == 0 ? 0 : pr.nrt) + row] = (int32_t)count;
}

// Exclusive scans of the counts into rowptr / st_rowptr, checked against the
// capacities (one CTA per problem).
__global__ void __launch_bounds__(1024) k_tile_scan(const ProblemDev* tab) {
  const ProblemDev& pr = tab[blockIdx.x];
  if (pr.precision != 2) return;
  __shared__ int64_t carry;
  __shared__ int64_t part[1024];
  for (int mode = 0; mode < 2; ++mode) {
    const int64_t rows = mode == 0 ? pr.nrt : pr.nst;
    const int32_t* cnt = pr.tcount + (mode == 0 ? 0 : pr.nrt);
    int32_t* out = mode == 0 ? pr.rowptr : pr.st_rowptr;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b0 = 0; b0 < rows; b0 += 1024) {
      const int64_t i = b0 + threadIdx.x;
      part[threadIdx.x] = i < rows ? cnt[i] : 0;
      __syncthreads();
      for (int o = 1; o < 1024; o <<= 1) {   // inclusive Hillis-Steele scan
        const int64_t v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
      }
      if (i < rows) {
        const int64_t incl = carry + part[threadIdx.x];
        out[i + 1] = (int32_t)(incl < INT32_MAX ? incl : INT32_MAX);
      }
      __syncthreads();
      if (threadIdx.x == 1023) carry += part[1023];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      out[0] = 0;
      const int64_t cap = mode == 0 ? pr.tile_cap : pr.st_cap;
      if (carry > cap) atomicOr(&pr.status[0], kStatTileOverflow);
    }
    __syncthreads();
  }
}

// C blocks of one row tile (one thread per row), 16 columns per pass.
__global__ void __launch_bounds__(kTileM) k_tile_form(const ProblemDev* tab) {
  const ProblemDev& pr = tab[blockIdx.y];
  if (pr.precision != 2 || blockIdx.x >= pr.nrt) return;
  if (pr.status[0] & kStatTileOverflow) return;
  extern __shared__ __align__(16) float fsm[];
  const int N = (int)pr.N, NS = N + 1;
  float* Wr = fsm;                     // [128][N + 1] this row tile's W
  float* Wb = Wr + kTileM * NS;        // [64][N + 1] the block's W
  int32_t* cb = reinterpret_cast<int32_t*>(Wb + kTileK * NS);   // [64][3] block coordinates
  float* rb = reinterpret_cast<float*>(cb + 3 * kTileK);         // [64] block R^-1/2
  const int r = threadIdx.x;
  const int64_t row = (int64_t)blockIdx.x;
  const int64_t a = row * kTileM + r;
  for (int e = threadIdx.x; e < kTileM * N; e += blockDim.x) {
    const int rr = e / N, k = e % N;
    Wr[rr * NS + k] = pr.Wp[(row * kTileM + rr) * N + k];
  }
  const int32_t srca = pr.tpos_src[a];
  const Coord3 ca = flat_to_coord(pr.grid, srca >= 0 ? pr.obs[srca] : 0);
  const float ra = pr.rinvp[a];
  double rowsum = 0.0;
  int64_t nnz = 0;
  const int t0 = pr.rowptr[row], t1 = pr.rowptr[row + 1];
  for (int t = t0; t < t1; ++t) {
    const int64_t blk = pr.colblk[t];
    __syncthreads();
    for (int e = threadIdx.x; e < kTileK * N; e += blockDim.x) {
      const int c = e / N, k = e % N;
      Wb[c * NS + k] = pr.Wp[(blk * kTileK + c) * N + k];
    }
    if (threadIdx.x < kTileK) {
      const int64_t b = blk * kTileK + threadIdx.x;
      const int32_t sb = pr.tpos_src[b];
      const Coord3 c = flat_to_coord(pr.grid, sb >= 0 ? pr.obs[sb] : 0);
      cb[3 * threadIdx.x] = (int32_t)c.x;
      cb[3 * threadIdx.x + 1] = (int32_t)c.y;
      cb[3 * threadIdx.x + 2] = (int32_t)c.z;
      rb[threadIdx.x] = pr.rinvp[b];
    }
    __syncthreads();
    __nv_bfloat16* hi = pr.Chi + ((int64_t)t * kTileM + r) * kTileK;
    __nv_bfloat16* lo = pr.Clo + ((int64_t)t * kTileM + r) * kTileK;
    for (int c0 = 0; c0 < kTileK; c0 += 16) {
      float acc[16];
#pragma unroll
      for (int cc = 0; cc < 16; ++cc) acc[cc] = 0.f;
      for (int k = 0; k < N; ++k) {
        const float w = Wr[r * NS + k];
#pragma unroll
        for (int cc = 0; cc < 16; ++cc) acc[cc] = fmaf(w, Wb[(c0 + cc) * NS + k], acc[cc]);
      }
      __align__(16) __nv_bfloat16 h16[16], l16[16];
#pragma unroll
      for (int cc = 0; cc < 16; ++cc) {
        const int c = c0 + cc;
        const Coord3 cbc{cb[3 * c], cb[3 * c + 1], cb[3 * c + 2]};
        const double r2 = scaled_r2_tab(pr.grid, pr.d2tab, ca, cbc);
        float v = 0.f;
        if (r2 < 4.0) v = gaspari_cohn_f(sqrtf((float)r2)) * acc[cc] * ra * rb[c];
        nnz += (r2 < 4.0 && srca >= 0 && pr.tpos_src[blk * kTileK + c] >= 0) ? 1 : 0;
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        h16[cc] = h;
        l16[cc] = __float2bfloat16_rn(v - __bfloat162float(h));
        rowsum += fabs((double)v);
        if (srca >= 0 && blk * kTileK + c == a) {
          atomic_min_nonneg(&pr.scal[1], (double)v);
          atomicAdd(&pr.scal[4], (double)v);
        }
      }
      const uint4* h4 = reinterpret_cast<const uint4*>(h16);
      const uint4* l4 = reinterpret_cast<const uint4*>(l16);
      uint4* hd = reinterpret_cast<uint4*>(hi + c0);
      uint4* ld = reinterpret_cast<uint4*>(lo + c0);
      hd[0] = h4[0];
      hd[1] = h4[1];
      ld[0] = l4[0];
      ld[1] = l4[1];
    }
  }
  if (srca >= 0) atomic_max_nonneg(&pr.scal[0], rowsum);
  if (nnz) atomicAdd(&pr.scal[3], (double)nnz);   // nonzeros of C (an exact integer count in FP64)
}

// Y = C X for the Ritz basis: X, Y [d][l] FP32 in tile order (Om / Yb), one
// thread per row of a row tile, the block's rows of X staged in shared memory.
__global__ void __launch_bounds__(kTileM) k_tile_ritz_matvec(const ProblemDev* tab, int src) {
  const ProblemDev& pr = tab[blockIdx.y];
  if (pr.precision != 2 || pr.l <= 0 || blockIdx.x >= pr.nrt) return;
  if (pr.status[0] & kStatTileOverflow) return;
  __shared__ float xs[kTileK][kMaxRitz + 1];
  const int l = pr.l;
  const float* X = reinterpret_cast<const float*>(src == 0 ? pr.Om : pr.Yb);
  float* Y = reinterpret_cast<float*>(src == 0 ? pr.Yb : pr.Om);
  const int64_t row = blockIdx.x, a = row * kTileM + threadIdx.x;
  float acc[kMaxRitz];
#pragma unroll
  for (int m = 0; m < kMaxRitz; ++m) acc[m] = 0.f;
  for (int t = pr.rowptr[row]; t < pr.rowptr[row + 1]; ++t) {
    const int64_t blk = pr.colblk[t];
    __syncthreads();
    for (int e = threadIdx.x; e < kTileK * l; e += blockDim.x) {
      const int c = e / l, m = e % l;
      const int64_t b = blk * kTileK + c;
      xs[c][m] = b < pr.d ? X[b * l + m] : 0.f;
    }
    __syncthreads();
    const uint4* h4 = reinterpret_cast<const uint4*>(pr.Chi + ((int64_t)t * kTileM + threadIdx.x) * kTileK);
    const uint4* l4 = reinterpret_cast<const uint4*>(pr.Clo + ((int64_t)t * kTileM + threadIdx.x) * kTileK);
    for (int q = 0; q < kTileK / 8; ++q) {
      const uint4 hv = h4[q], lv = l4[q];
      const __nv_bfloat16* hb = reinterpret_cast<const __nv_bfloat16*>(&hv);
      const __nv_bfloat16* lb = reinterpret_cast<const __nv_bfloat16*>(&lv);
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const float cv = __bfloat162float(hb[e]) + __bfloat162float(lb[e]);
        const int c = q * 8 + e;
#pragma unroll
        for (int m = 0; m < kMaxRitz; ++m)
          if (m < l) acc[m] = fmaf(cv, xs[c][m], acc[m]);
      }
    }
  }
  if (a < pr.d) {
#pragma unroll
    for (int m = 0; m < kMaxRitz; ++m)   // unrolled: acc stays in registers
      if (m < l) Y[a * l + m] = acc[m];
  }
}

// vbar (natural order, FP64 and the FP32 copy) from the tile-ordered iterates.
__global__ void k_tile_accumulate(const ProblemDev* tab) {
  const ProblemDev& pr = tab[blockIdx.y];
  if (pr.precision != 2) return;
  const int64_t N1 = pr.N + 1;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= pr.d * N1) return;
  const int64_t a = i / N1, m = i % N1;
  const int64_t ap = pr.obs_tpos[a];
  double acc = 0.0;
  if (m < pr.N) {
    if (pr.do_pert)
      for (int q = 0; q < pr.Q; ++q) {
        const int64_t sid = pr.mean_sys + (int64_t)q * pr.N + m;
        acc += pr.p[q] * (double)pr.Xv[sid * pr.d_pad + ap];
      }
  } else if (pr.do_mean) {
    acc = (double)pr.Xv[ap];
  }
  const double v = pr.rinv[a] * acc;
  pr.Vbar[a * N1 + m] = v;
  reinterpret_cast<float*>(pr.VbarT)[a * N1 + m] = (float)v;
}

// State update over state tiles (256 threads).  For each stored column block:
//   S = GC o (Z_tile W_blk^T)   (128 x 64; thread: 4 points x 8 observations)
//   acc += S Vbar_blk           (128 x (N + 1); thread: 4 points x up to 17 columns)
// Operands sit k-major in shared memory so a thread's 4 points or 8
// observations are one or two 16-byte loads; the per-axis distance table is
// staged in FP32.  Register-blocked so each shared-memory load feeds 3-4 FMAs.
constexpr int kStCols = 17;     // columns per thread in the S Vbar product: 8 groups cover N + 1 <= 136
constexpr int kD2Max = 4096;    // distance-table entries staged in shared memory (sum of the extents)
__global__ void __launch_bounds__(256, 1) k_tile_state_apply(const ProblemDev* tab) {
  const ProblemDev& pr = tab[blockIdx.y];
  if (pr.precision != 2 || blockIdx.x >= pr.nst) return;
  if (pr.status[0] & kStatTileOverflow) return;
  extern __shared__ __align__(16) float fsm[];
  const int N = (int)pr.N, N1 = N + 1;
  const int cpg = (N1 + 7) / 8;           // columns per column group (<= kStCols)
  const int N1p = 8 * cpg;
  float* Zs = fsm;                        // [N][128]
  float* Wb = Zs + N * kTileM;            // [N][64]
  float* S = Wb + N * kTileK;             // [64][128]
  float* Vb = S + kTileK * kTileM;        // [64][N1p]
  float* d2 = Vb + kTileK * N1p;          // [ext0 + ext1 + ext2] (when <= kD2Max)
  int32_t* cb = reinterpret_cast<int32_t*>(d2 + kD2Max);   // [64][3]
  const GridDev& g = pr.grid;
  const int64_t next = g.ext[0] + g.ext[1] + g.ext[2];
  const bool d2s = next <= kD2Max;
  const int64_t st = blockIdx.x, x0 = st * kTileM;
  const float* Zt = reinterpret_cast<const float*>(pr.Zt);
  const float* VbT = reinterpret_cast<const float*>(pr.VbarT);
  for (int e = threadIdx.x; e < kTileM * N; e += blockDim.x) {
    const int i = e / N, k = e % N;
    const int64_t x = x0 + i;
    Zs[k * kTileM + i] = x < pr.n ? Zt[x * N + k] : 0.f;
  }
  if (d2s)
    for (int e = threadIdx.x; e < next; e += blockDim.x) d2[e] = (float)pr.d2tab[e];
  const int tid = threadIdx.x;
  const int rg = tid >> 3, cg = tid & 7;  // 32 row groups of 4 points x 8 column groups
  Coord3 cx[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t x = x0 + 4 * rg + i;
    cx[i] = flat_to_coord(g, x < pr.n ? x : 0);
  }
  float acc[4][kStCols];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < kStCols; ++j) acc[i][j] = 0.f;
  for (int t = pr.st_rowptr[st]; t < pr.st_rowptr[st + 1]; ++t) {
    const int64_t blk = pr.st_colblk[t];
    __syncthreads();
    for (int e = tid; e < kTileK * N; e += blockDim.x) {
      const int c = e / N, k = e % N;
      Wb[k * kTileK + c] = pr.Wp[(blk * kTileK + c) * N + k];
    }
    for (int e = tid; e < kTileK * N1p; e += blockDim.x) {
      const int c = e / N1p, m = e % N1p;
      const int32_t src = pr.tpos_src[blk * kTileK + c];
      Vb[c * N1p + m] = (src >= 0 && m < N1) ? VbT[(int64_t)src * N1 + m] : 0.f;
    }
    if (tid < kTileK) {
      const int32_t src = pr.tpos_src[blk * kTileK + tid];
      const Coord3 c = flat_to_coord(g, src >= 0 ? pr.obs[src] : 0);
      cb[3 * tid] = src >= 0 ? (int32_t)c.x : -1;   // -1: padding column
      cb[3 * tid + 1] = (int32_t)c.y;
      cb[3 * tid + 2] = (int32_t)c.z;
    }
    __syncthreads();
    // S for points 4 rg .. 4 rg + 3 and observations 8 cg .. 8 cg + 7
    {
      float sa[4][8];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) sa[i][j] = 0.f;
      for (int k = 0; k < N; ++k) {
        const float4 z = *reinterpret_cast<const float4*>(Zs + k * kTileM + 4 * rg);
        const float4 w0 = *reinterpret_cast<const float4*>(Wb + k * kTileK + 8 * cg);
        const float4 w1 = *reinterpret_cast<const float4*>(Wb + k * kTileK + 8 * cg + 4);
        const float zz[4] = {z.x, z.y, z.z, z.w};
        const float ww[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) sa[i][j] = fmaf(zz[i], ww[j], sa[i][j]);
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int c = 8 * cg + j;
        const int32_t bc[3] = {cb[3 * c], cb[3 * c + 1], cb[3 * c + 2]};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          float v = 0.f;
          if (bc[0] >= 0) {
            const int64_t ca[3] = {cx[i].x, cx[i].y, cx[i].z};
            float r2 = 0.f;
            int64_t off = 0;
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
              if (g.ext[ax] > 1) {
                const int64_t dl = ca[ax] > bc[ax] ? ca[ax] - bc[ax] : bc[ax] - ca[ax];
                r2 += d2s ? d2[off + dl] : (float)pr.d2tab[off + dl];
              }
              off += g.ext[ax];
            }
            if (r2 < 4.f) v = gaspari_cohn_f(sqrtf(r2)) * sa[i][j];
          }
          S[c * kTileM + 4 * rg + i] = v;
        }
      }
    }
    __syncthreads();
    // acc += S Vbar for columns cg * cpg .. cg * cpg + cpg - 1
    for (int c = 0; c < kTileK; ++c) {
      const float4 sv = *reinterpret_cast<const float4*>(S + c * kTileM + 4 * rg);
      const float ss[4] = {sv.x, sv.y, sv.z, sv.w};
      const float* vr = Vb + c * N1p + cg * cpg;
#pragma unroll
      for (int j = 0; j < kStCols; ++j) {
        if (j < cpg) {
          const float v = vr[j];
#pragma unroll
          for (int i = 0; i < 4; ++i) acc[i][j] = fmaf(ss[i], v, acc[i][j]);
        }
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t x = x0 + 4 * rg + i;
    if (x >= pr.n) continue;
    const double mu = pr.mu[x];
#pragma unroll
    for (int j = 0; j < kStCols; ++j) {   // unrolled: acc stays in registers
      const int col = cg * cpg + j;
      if (j < cpg && col < N1) {
        const double inc = (double)acc[i][j];
        if (col < N) {
          if (pr.do_pert)
            pr.A_a[(int64_t)col * pr.n + x] = (pr.X[(int64_t)col * pr.n + x] - mu) - pr.sqrt_nm1 * inc;
        } else if (pr.do_mean) {
          pr.mu_a[x] = mu + inc;
        }
      }
    }
  }
}

size_t form_smem(int64_t N) {
  return (size_t)(kTileM + kTileK) * (N + 1) * 4 + 3 * kTileK * 4 + kTileK * 4;
}
size_t state_smem(int64_t N) {
  const int64_t n1p = 8 * ((N + 1 + 7) / 8);
  return (size_t)(kTileM + kTileK) * N * 4 + (size_t)kTileK * kTileM * 4 + (size_t)kTileK * n1p * 4 + kD2Max * 4 +
         3 * kTileK * 4;
}

}  // namespace

// Largest ensemble the tile kernels take (shared-memory staging of W and Z rows).
constexpr int64_t kTileMaxN = 128;
int64_t tile_max_members() { return kTileMaxN; }

void launch_tile_setup(const ProblemTable& tab, const ProblemDev* dtab, cudaStream_t st) {
  int64_t nsort = 0, dpn = 0, nblk = 0, nrt = 0, nst = 0, Nmax = 0;
  for (int i = 0; i < tab.count; ++i) {
    const ProblemDev& p = tab.p[i];
    nsort = p.nsort > nsort ? p.nsort : nsort;
    dpn = p.d_pad * p.N > dpn ? p.d_pad * p.N : dpn;
    nblk = p.nblk > nblk ? p.nblk : nblk;
    nrt = p.nrt > nrt ? p.nrt : nrt;
    nst = p.nst > nst ? p.nst : nst;
    Nmax = p.N > Nmax ? p.N : Nmax;
  }
  const unsigned P = (unsigned)tab.count;
  k_tile_keys<<<dim3((unsigned)((nsort + 255) / 256), P), 256, 0, st>>>(dtab);
  k_bitonic_chunk<<<dim3((unsigned)(nsort / 1024), P), 512, 0, st>>>(dtab, 2, 1024);
  int launches = 2;
  for (int64_t k = 2048; k <= nsort; k <<= 1) {
    for (int64_t j = k >> 1; j >= 1024; j >>= 1) {
      k_bitonic_global<<<dim3((unsigned)((nsort / 2 + 255) / 256), P), 256, 0, st>>>(dtab, k, j);
      ++launches;
    }
    k_bitonic_chunk<<<dim3((unsigned)(nsort / 1024), P), 512, 0, st>>>(dtab, k, k);
    ++launches;
  }
  k_tile_order<<<dim3((unsigned)((dpn + 255) / 256), P), 256, 0, st>>>(dtab);
  k_tile_boxes<<<dim3((unsigned)((nblk * 32 + 255) / 256), P), 256, 0, st>>>(dtab);
  k_tile_pattern<<<dim3((unsigned)nrt, P), 256, 0, st>>>(dtab, 0, 0);
  k_tile_pattern<<<dim3((unsigned)nst, P), 256, 0, st>>>(dtab, 1, 0);
  k_tile_scan<<<P, 1024, 0, st>>>(dtab);
  k_tile_pattern<<<dim3((unsigned)nrt, P), 256, 0, st>>>(dtab, 0, 1);
  k_tile_pattern<<<dim3((unsigned)nst, P), 256, 0, st>>>(dtab, 1, 1);
  const size_t fs = form_smem(Nmax);
  static thread_local int raised = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (raised != dev) {
    cudaFuncSetAttribute(k_tile_form, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)form_smem(kTileMaxN));
    cudaFuncSetAttribute(k_tile_state_apply, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)state_smem(kTileMaxN));
    raised = dev;
  }
  note_launches(launches + 7);
  // the C blocks on the tensor cores where every problem qualifies, else on the CUDA cores
  if (launch_tile_form_mma(tab, dtab, st) != 0) {
    cudaGetLastError();
    k_tile_form<<<dim3((unsigned)nrt, P), kTileM, fs, st>>>(dtab);
    note_launches(1);
  }
}

// Y = C X of the Ritz basis on the tensor cores: X [d][l] (tile order) split
// exactly into BF16 planes Xh = bf16(X), Xl = bf16(X - Xh), stored as the 2 l
// "systems" [Xh; Xl] of the tile matvec in the PCG's direction buffer (free
// during the set-up); then Y = C Xh + C Xl.
__global__ void k_ritz_split(const ProblemDev* dp, int src) {
  const ProblemDev& pr = *dp;
  const int l = pr.l;
  const int64_t dpad = pr.d_pad;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)l * dpad) return;
  const int64_t m = i / dpad, a = i % dpad;
  const float* X = reinterpret_cast<const float*>(src == 0 ? pr.Om : pr.Yb);
  const float x = a < pr.d ? X[a * l + m] : 0.f;
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  pr.Pdir[i] = h;
  pr.Pdir[(int64_t)l * dpad + i] = __float2bfloat16_rn(x - __bfloat162float(h));
}

__global__ void k_ritz_sum(const ProblemDev* dp, int src) {
  const ProblemDev& pr = *dp;
  const int l = pr.l;
  const int64_t dpad = pr.d_pad;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= pr.d * l) return;
  const int64_t a = i / l, m = i % l;
  float* Y = reinterpret_cast<float*>(src == 0 ? pr.Yb : pr.Om);
  Y[i] = pr.Yv[m * dpad + a] + pr.Yv[(l + m) * dpad + a];
}

void launch_tile_ritz_matvec(const ProblemTable& tab, const ProblemDev* dtab, int src, cudaStream_t st) {
  // the tensor-core form needs room for 2 l systems in the direction buffer
  bool tc = true;
  for (int i = 0; i < tab.count; ++i) {
    const ProblemDev& p = tab.p[i];
    if (p.precision == 2 && p.l > 0 && p.nsys < 2 * (int64_t)p.l) tc = false;
  }
  for (int i = 0; tc && i < tab.count; ++i) {
    const ProblemDev& p = tab.p[i];
    if (p.precision != 2 || p.l <= 0) continue;
    k_ritz_split<<<(unsigned)(((int64_t)p.l * p.d_pad + 255) / 256), 256, 0, st>>>(dtab + i, src);
    TileMmArgs a{};
    a.rowptr = p.rowptr;
    a.colblk = p.colblk;
    a.P = p.Pdir;
    a.sigma = nullptr;
    a.active = nullptr;
    a.Y = p.Yv;
    a.pty = nullptr;
    a.status = p.status;
    a.d_pad = p.d_pad;
    a.J = 2 * p.l;
    a.nrt = (int32_t)p.nrt;
    if (launch_tile_mm(a, p.Chi, p.Clo, p.tile_cap, st) != 0) {
      cudaGetLastError();
      tc = false;   // the CUDA-core kernel below recomputes every problem
      break;
    }
    k_ritz_sum<<<(unsigned)((p.d * p.l + 255) / 256), 256, 0, st>>>(dtab + i, src);
    note_launches(2);
  }
  if (tc) return;
  int64_t nrt = 0;
  for (int i = 0; i < tab.count; ++i) nrt = tab.p[i].nrt > nrt ? tab.p[i].nrt : nrt;
  k_tile_ritz_matvec<<<dim3((unsigned)nrt, tab.count), kTileM, 0, st>>>(dtab, src);
  note_launches(1);
}

void launch_tile_finish(const ProblemTable& tab, const ProblemDev* dtab, cudaStream_t st) {
  int64_t dn1 = 0, nst = 0, Nmax = 0;
  for (int i = 0; i < tab.count; ++i) {
    const ProblemDev& p = tab.p[i];
    dn1 = p.d * (p.N + 1) > dn1 ? p.d * (p.N + 1) : dn1;
    nst = p.nst > nst ? p.nst : nst;
    Nmax = p.N > Nmax ? p.N : Nmax;
  }
  k_tile_accumulate<<<dim3((unsigned)((dn1 + 255) / 256), tab.count), 256, 0, st>>>(dtab);
  note_launches(1);
  // the state update on the tensor cores (tile_state.cu) where every problem
  // qualifies, else on the CUDA cores
  if (launch_tile_state_mma(tab, dtab, st) == -1) {
    k_tile_state_apply<<<dim3((unsigned)nst, tab.count), 256, state_smem(Nmax), st>>>(dtab);
    note_launches(1);
  }
}

}  // namespace infoesrf
