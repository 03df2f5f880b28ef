// a5-a7 for one-dimensional observation networks: cluster-resident batched
// shifted PCG (App. E, Eq. normalized_linear_solve; Golub & Van Loan Alg. 11.5.1)
// with the band of C held in shared memory for the whole launch.
//
// Why: every (node, member) system uses the same C, and C is re-read once
// per iteration per system group.  Streaming it from L2 each iteration made
// the first kernel L2-latency bound.  Here a thread-block cluster of CS CTAs
// splits the rows of C: CTA c owns rows [c R_s, (c+1) R_s) and keeps them,
// as dense 16-row tiles over each tile's column window (zeros outside a
// row's band), in shared memory for the whole launch.  The cluster iterates
// kJ = 32 systems at once (the "lanes"); each CTA holds the lanes' vectors on
// its own rows, plus a window of p widened by the band's reach, whose halo
// rows are copied from the owning CTAs through distributed shared memory.
//
// On a 1-D grid the observations within the Gaspari-Cohn support of an
// observation form a contiguous cyclic range of (sorted) observation
// indices, which is what makes the row tiles dense; the kernel checks this
// and the shared-memory budget at start-up and, if either fails, sets a
// flag and exits so that the general kernel solves the systems instead.
//
// The band matvec runs on the tensor cores (mma.sync, FP16 operands split
// into hi + lo pairs after power-of-two scaling, FP32 accumulation; see the
// matvec step below for why this keeps FP32 accuracy).
//
// Per iteration (three cluster barriers, a fourth for the learned term's r
// halo):
//   matvec y = sigma p + C p and partial p^T y      -> barrier 1 -> alpha
//   x += alpha p, r -= alpha y, partial r^T r, Phi^T r, A^T r -> barrier 2
//   convergence, preconditioner scalars, refills;  p = z + beta p, the lanes'
//   max |p| (the next matvec's scale)               -> barrier 3
//   new lanes start, halo of p copied from the neighbours.
// Every CTA sums the CS partials in rank order, so all CTAs of a cluster
// take identical decisions without further communication.  A lane whose
// system converges is refilled with the next system of a global queue
// ordered hardest (smallest shift) first, so no lane idles while work
// remains.  Dot products of the FP32 vectors are float-float sums (FP64
// accuracy without the FP64 pipe); the CG scalars formed from them and the
// k x k algebra of the limited-memory preconditioner are FP32.
#include <cooperative_groups.h>
#include <cuda_fp16.h>
#include <math.h>
#include <stddef.h>

#include "common.cuh"
#include "info_esrf.h"
#include "info_esrf_stages.h"
#include "internal.h"

namespace cg = cooperative_groups;

namespace infoesrf {

namespace {

constexpr int kJ = 32;          // lanes (systems) per cluster
constexpr int kLD = kJ + 4;     // padded row stride (floats) of lane-major row vectors
constexpr int kTile = 16;       // rows per matvec tile
constexpr int kNW = kThreads / 32;
constexpr int kK = 10;          // Ritz vectors handled by this kernel
constexpr int kNR = 4 + 2 * kK; // residual reduction values per lane: rr (hi, lo), uu (hi, lo), f[k], g[k]
constexpr int kKP = (kK + 3) & ~3;   // kK rounded up to a multiple of 4
constexpr int kRetry = 1 << 30; // queue id flag: solve this system again without the learned term
constexpr int kTH = 2 * kLearnH;          // half-width of T = S^T S (autocorrelation of the taps)
constexpr int kTT = 2 * kTH + 1;          // taps of T
constexpr int kStRows = 16;               // own rows per warp in the learned stencil (kNW kStRows >= R_s)
constexpr int kMaxTiles = 128;  // rows per CTA <= 2048
constexpr int kMaxCS = 8;       // CTAs per cluster
constexpr int kQTab = 65;       // shift slots (Q + 1) whose lane scalars are staged in shared memory

enum : int { kEmpty = 0, kStart = 1, kActive = 2 };

// Phase clocks (built only with -DINFO_ESRF_PHASE_CLOCKS, a separate build of
// the library): thread 0 of every CTA sums clock64() deltas per phase of a
// round in shared memory and adds them, with the round count and its set-up
// cycles, into g_band_phase at exit; info_esrf_band_phase_clocks reads them.
constexpr int kPhases = 10;
[[maybe_unused]] constexpr int kPhaseSlots = kPhases + 3;   // phases, rounds, set-up cycles, CTAs
#ifdef INFO_ESRF_PHASE_CLOCKS
#define BAND_PHASE(i)                 \
  if (tid == 0) {                     \
    const long long now_ = clock64(); \
    s_ph[i] += now_ - ph_t;           \
    ph_t = now_;                      \
  }
#else
#define BAND_PHASE(i)
#endif

struct LaneState {
  int sid[kJ], state[kJ], it[kJ], newsid[kJ], fin[kJ];
  int qs[kJ];                         // coefficient slot of the learned term (q, Q: mean), -1: none
  float rho[kJ];                      // r^T M r of the current iterate
  float rrh[kJ], rrl[kJ];             // r^T r as a float-float pair (FP64-accurate)
  float bn2[kJ];                      // b^T b
  float sigf[kJ], alpha[kJ], beta[kJ];
  float t[kJ][kKP], c[kJ][kKP];       // LMP coefficients, rows padded for 16-byte loads
  float la[kJ], ltT[kTT][kJ];         // learned correction: a and the taps of T = S^T S (tap-major)
  float bmf[kJ];                      // beta_q - sigma_q of the preconditioner (App. E)
  int learn[kJ];
  int mem[kJ];                        // ensemble member of the lane's system, -1 for the mean system
};

static_assert(offsetof(LaneState, t) % 16 == 0 && offsetof(LaneState, c) % 16 == 0, "16-byte rows of t and c");

// Problem fields read inside the iteration loop, copied to shared memory once:
// global loads after a cluster barrier (acquire at cluster scope) cannot be
// served from a stale L1 line, so every ProblemDev access there would be an
// L2 round trip on the critical path.
struct LoopArgs {
  const float* learn_T;
  const double* bmean;
  float* U;
  int32_t* iters;
  double* relres;
  int32_t* status;
  int mean_sys, Q, nsys, fixed_iters;
};

struct Setup {
  int hl, hr, bad, tilesz;
  int xchg[4];
  int npush;       // halo rows of p this CTA pushes to the cluster
  int nrpush;      // halo rows of r (learned term)
};

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }

// 4-byte asynchronous copy global -> shared (completion: cp_async_wait_all + a barrier).
__device__ __forceinline__ void cp_async4(float* dst_smem, const float* src_global) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst_smem);
  const size_t g = __cvta_generic_to_global(src_global);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
// Split cluster barrier: arrive (releasing this thread's earlier shared and
// distributed shared-memory writes), independent work, then wait (acquiring
// every CTA's).  All threads of the cluster execute both, in the same order.
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory"); }

// Two FP32 values (already scaled into FP16 range) as hi + lo pairs of
// packed FP16: hi = the values rounded to FP16, lo = the remainders rounded to
// FP16 (the remainder itself is exact in FP32).  The lower half holds x0.
__device__ __forceinline__ void f16_split2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  const __half2 h = __floats2half2_rn(x0, x1);
  const float2 hf = __half22float2(h);
  const __half2 l = __floats2half2_rn(x0 - hf.x, x1 - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// D += A B for one 16 x 8 x 16 FP16 tile, FP32 accumulation.  Fragments
// (g = lane / 4, q = lane % 4; a register holds two consecutive k, the lower
// k in its lower half): a = A[g][2q..], A[g+8][2q..], A[g][2q+8..],
// A[g+8][2q+8..]; b = B[2q..][g], B[2q+8..][g]; d = D[g][2q], D[g][2q+1],
// D[g+8][2q], D[g+8][2q+1].
__device__ __forceinline__ void mma_f16(float& d0, float& d1, float& d2, float& d3, const uint4& a, uint32_t b0,
                                        uint32_t b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d0), "+f"(d1), "+f"(d2), "+f"(d3)
      : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
}

// Cyclic offset col - a folded into (-d/2, d/2] (0 <= col, a < d < 2^31).
__device__ __forceinline__ int wrap_delta(int col, int a, int d) {
  int dl = col - a;
  if (dl < 0) dl += d;
  if (2 * dl > d) dl -= d;
  return dl;
}

// Power-of-two scale that brings |m| into [0.5, 1) (1 when m is 0 or not finite).
__device__ __forceinline__ void pow2_scale(float m, float& scale, float& inv) {
  if (m > 0.f && isfinite(m)) {
    int e = 0;
    frexpf(m, &e);
    e = e < -100 ? -100 : (e > 100 ? 100 : e);
    scale = ldexpf(1.f, -e);
    inv = ldexpf(1.f, e);
  } else {
    scale = 1.f;
    inv = 1.f;
  }
}

#ifdef INFO_ESRF_PHASE_CLOCKS
__device__ unsigned long long g_band_phase[kPhaseSlots];
#endif

}  // namespace

__global__ void __launch_bounds__(kThreads, 1)
k_pcg_band1d(const ProblemDev* tab, int32_t* queue, int32_t* fallback, int dyn_floats) {
  extern __shared__ __align__(16) float dyn[];
  __shared__ __align__(16) LaneState L;
  __shared__ Setup S;
  __shared__ int s_klo[kMaxTiles], s_w[kMaxTiles], s_off[kMaxTiles];
  __shared__ __align__(16) float s_pmax_in[kMaxCS][kJ];     // max |p| per lane over each CTA's own rows
  __shared__ __align__(16) float s_pscale[kJ], s_pinv[kJ];  // power-of-two scale of p per lane
  __shared__ float s_gram[3][kK * kK];
  __shared__ float s_theta[kK];
  // partial sums pushed by every CTA of the cluster into every CTA (slot = source rank)
  __shared__ __align__(16) float s_pap_in[kMaxCS][kJ][2];      // p^T y (float-float)
  __shared__ __align__(16) float s_res_in[kMaxCS][kJ][kNR];    // rr (float-float), Phi^T r, A^T r
  __shared__ float s_wpap[kNW][kJ][2];
  __shared__ int s_lo_min, s_hi_max, s_bad;

  cg::cluster_group cluster = cg::this_cluster();
  const int CS = (int)cluster.num_blocks();
  const int crank = (int)cluster.block_rank();
  const int cl_id = blockIdx.x / CS;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#ifdef INFO_ESRF_PHASE_CLOCKS
  __shared__ long long s_ph[kPhaseSlots];
  long long ph_t = clock64();
  if (tid < kPhaseSlots) s_ph[tid] = 0;
#endif
  const ProblemDev& pr = tab[0];
  const int64_t d = pr.d, N = pr.N;
  const int k = pr.kR < kK ? pr.kR : kK;
  const int pk = pr.kR;
  const int R_s = (int)((d + CS - 1) / CS);
  const int64_t s0 = (int64_t)crank * R_s;
  const int nrows = (int)(d - s0 < 0 ? 0 : (d - s0 < R_s ? d - s0 : R_s));
  const int ntiles = (nrows + kTile - 1) / kTile;

  // ---------------- set-up: band reach of the own rows ----------------
  if (tid == 0) { s_lo_min = 1 << 30; s_hi_max = -(1 << 30); s_bad = (R_s > kMaxTiles * kTile) ? 1 : 0; }
  __syncthreads();
  // per-row window [lo, hi] relative to s0, kept in the dynamic buffer's tail
  int* rlo = reinterpret_cast<int*>(dyn);
  int* rhi = rlo + R_s;
  float* ramax = dyn + 2 * R_s;   // max |C| of each own row (its FP16 scale)
  if (3 * R_s > dyn_floats) s_bad = 1;
  __syncthreads();
  if (!s_bad) {
    // two threads per row (alternate entries), combined by a shuffle; the same
    // pass takes each row's max |C| (the FP16 scale of its row)
    const float* cval = reinterpret_cast<const float*>(pr.oo_val);
    for (int base = 0; base < nrows; base += (int)blockDim.x / 2) {
      const int row = base + (tid >> 1), part = tid & 1;
      int dmin = 1 << 30, dmax = -(1 << 30), nnz = 0;
      float amax = 0.f;
      if (row < nrows) {
        const int64_t a = s0 + row;
        nnz = pr.oo_nnz[a];
#pragma unroll 8
        for (int e = part; e < nnz; e += 2) {   // eight entries' loads in flight
          const int dl = wrap_delta(pr.oo_col[(int64_t)e * d + a], (int)a, (int)d);
          dmin = dl < dmin ? dl : dmin;
          dmax = dl > dmax ? dl : dmax;
          amax = fmaxf(amax, fabsf(cval[(int64_t)e * d + a]));
        }
      }
      amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, 1));
      if (row < nrows && part == 0) ramax[row] = amax;
      dmin = min(dmin, __shfl_xor_sync(0xffffffffu, dmin, 1));
      dmax = max(dmax, __shfl_xor_sync(0xffffffffu, dmax, 1));
      if (row < nrows && part == 0) {
        bool ok = nnz >= 1 && (dmax - dmin + 1) == nnz && 2 * (int64_t)(dmax - dmin + 1) < d;
        if (!ok) atomicOr(&s_bad, 1);
        rlo[row] = row + dmin;
        rhi[row] = row + dmax;
        atomicMin(&s_lo_min, row + dmin);
        atomicMax(&s_hi_max, row + dmax);
      }
    }
  }
  __syncthreads();
  // tile windows
  if (!s_bad) {
    for (int t = warp; t < ntiles; t += kNW) {
      const int row = t * kTile + (lane & 15);
      int lo = 1 << 30, hi = -(1 << 30);
      if (lane < 16 && row < nrows) { lo = rlo[row]; hi = rhi[row]; }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
      }
      if (lane == 0) { s_klo[t] = lo; s_w[t] = (hi - lo + 1 + 15) & ~15; }   // whole 16-column chunks
    }
  }
  __syncthreads();
  if (tid == 0) {
    int off = 0;
    if (!s_bad)
      for (int t = 0; t < ntiles; ++t) { s_off[t] = off; off += s_w[t] * kTile; }
    S.tilesz = off;
    S.hl = nrows > 0 ? (s_lo_min < 0 ? -s_lo_min : 0) : 0;
    S.hr = nrows > 0 ? (s_hi_max > R_s - 1 ? s_hi_max - (R_s - 1) : 0) : 0;
    S.bad = s_bad;
    S.xchg[0] = S.hl; S.xchg[1] = S.hr; S.xchg[2] = S.bad; S.xchg[3] = S.tilesz;
  }
  cluster.sync();
  int hl = 0, hr = 0, bad = 0, tilesz = 0;
  for (int c = 0; c < CS; ++c) {
    const Setup* rs = cluster.map_shared_rank(&S, c);
    hl = max(hl, rs->xchg[0]);
    hr = max(hr, rs->xchg[1]);
    bad |= rs->xchg[2];
    tilesz = max(tilesz, rs->xchg[3]);
  }
  // halo rows of every CTA that this CTA owns: (own row, destination, window row)
  auto nrows_of = [&](int c2) {
    const int64_t s02 = (int64_t)c2 * R_s;
    return (int)(d - s02 < 0 ? 0 : (d - s02 < R_s ? d - s02 : R_s));
  };
  auto for_each_push_w = [&](int wl, int wr, auto&& f) {   // window [-wl, R_s + wr), thread-strided
    const int per = wl + R_s + wr;           // window rows per CTA (own rows skipped)
    for (int e = tid; e < CS * per; e += blockDim.x) {
      const int c2 = e / per, wrow = e % per;  // wrow = rel2 + wl
      const int rel2 = wrow - wl;
      const int nr2 = nrows_of(c2);
      if (rel2 >= 0 && rel2 < nr2) continue;   // own row of c2, not a halo row
      int g = c2 * R_s + rel2;          // |rel2| < d, so one fold is enough
      if (g < 0) g += (int)d;
      if (g >= d) g -= (int)d;
      const int owner = g / R_s;
      if (owner != crank) continue;
      f((int)(g - s0), c2, wrow);
    }
  };
  auto for_each_push = [&](auto&& f) { for_each_push_w(hl, hr, f); };
  // learned term: T r needs r on a window of +-kTH rows around the own rows
  const bool learn_ok = pr.learned_model != nullptr && R_s <= kNW * kStRows;
  if (tid == 0) { S.npush = 0; S.nrpush = 0; }
  __syncthreads();
  {
    int cnt = 0, cnt2 = 0;
    for_each_push([&](int, int, int) { ++cnt; });
    if (learn_ok) for_each_push_w(kTH, kTH, [&](int, int, int) { ++cnt2; });
    if (cnt) atomicAdd(&S.npush, cnt);
    if (cnt2) atomicAdd(&S.nrpush, cnt2);
  }
  cluster.sync();
  int npush_max = 0, nrpush_max = 0;
  for (int c = 0; c < CS; ++c) {
    npush_max = max(npush_max, cluster.map_shared_rank(&S, c)->npush);
    nrpush_max = max(nrpush_max, cluster.map_shared_rank(&S, c)->nrpush);
  }
  // shared-memory carve (floats): tiles | p window | r | x | y | Phi^T | A^T | push table
  const int W_p = R_s + hl + hr;
  const int o_pw = (tilesz + 3) & ~3;
  const int o_r = o_pw + (W_p + 16) * kLD;         // p window + 16 zero rows read by padded chunks
  const int o_x = o_r + R_s * kLD;
  const int o_y = o_x + R_s * kLD;                 // y, then the r window, own rows at +kTH
  const int o_ph = o_y + (R_s + 2 * kTH) * kLD;
  const int o_at = o_ph + k * R_s;
  const int o_push = (o_at + k * R_s + 1) & ~1;
  const int o_rpush = o_push + 2 * npush_max;
  const int o_rinv = o_rpush + 2 * nrpush_max;     // R^-1/2 of the own rows
  const int o_rsc = o_rinv + R_s;                  // power-of-two scale of each row of C, and its inverse
  const int need = o_rsc + 2 * R_s;
  if (need > dyn_floats || o_rsc < 3 * R_s) bad = 1;   // the scales are copied out of the head region
  cluster.sync();                                   // remote reads of S done before anyone exits
  if (bad) {
    if (cl_id == 0 && crank == 0 && tid == 0) *fallback = 1;
    return;
  }
  if (cl_id == 0 && crank == 0 && tid == 0) atomicOr(&pr.status[1], 1);
  float* Ct = dyn;
  float* __restrict__ pw = dyn + o_pw;   // the six vector regions are disjoint
  float* __restrict__ vr = dyn + o_r;
  float* __restrict__ vx = dyn + o_x;
  float* __restrict__ vy = dyn + o_y;
  float* __restrict__ phT = dyn + o_ph;
  float* __restrict__ aT = dyn + o_at;
  int2* push = reinterpret_cast<int2*>(dyn + o_push);
  int2* rpush = reinterpret_cast<int2*>(dyn + o_rpush);
  float* s_rinv = dyn + o_rinv;
  float* rsc = dyn + o_rsc;
  float* rsi = rsc + R_s;
  const float* val = reinterpret_cast<const float*>(pr.oo_val);
  const float* Phi = reinterpret_cast<const float*>(pr.Phi);
  const float* CPhi = reinterpret_cast<const float*>(pr.CPhi);
  const float* W = reinterpret_cast<const float*>(pr.W);

  // ---------------- set-up: fill tiles and the constant arrays ----------------
  // the row scales leave the head of the buffer before the tiles overwrite it
  for (int row = tid; row < R_s; row += blockDim.x) pow2_scale(row < nrows ? ramax[row] : 0.f, rsc[row], rsi[row]);
  __syncthreads();
  for (int i = tid; i < tilesz; i += blockDim.x) Ct[i] = 0.f;
  for (int i = o_pw + tid; i < o_ph; i += blockDim.x) dyn[i] = 0.f;
  __syncthreads();
  // C is stored tile by tile as FP16 hi + lo pairs of C with each row scaled by a
  // power of two (the row's max |C| into [0.5, 1)), in MMA fragment order: per
  // 16-column chunk, the hi halves of the 32 lanes (8 each), then the lo halves.
  // Scaling row i of A scales row i of A B, so the matvec undoes it per output
  // row; rows of very different size (observation errors of very different
  // size) each keep FP16's relative precision.
  {
    __half* Ch = reinterpret_cast<__half*>(Ct);
    for (int base = 0; base < nrows; base += (int)blockDim.x / 2) {
      const int row = base + (tid >> 1), part = tid & 1;
      if (row >= nrows) continue;
      const int64_t a = s0 + row;
      const int nnz = pr.oo_nnz[a];
      const int t = row / kTile, r = row % kTile;
      const float sc = rsc[row];
#pragma unroll 8
      for (int e = part; e < nnz; e += 2) {   // eight entries' loads in flight
        const int rel = row + wrap_delta(pr.oo_col[(int64_t)e * d + a], (int)a, (int)d);
        const int kk = rel - s_klo[t], kc = kk & 15;
        const int ln = (r & 7) * 4 + ((kc & 7) >> 1);         // lane holding this element
        const int h = (r >> 3) * 2 + (kc >> 3) * 4 + (kc & 1);  // half within the lane's 8
        const float v = val[(int64_t)e * d + a] * sc;
        const __half hv = __float2half_rn(v);
        const int64_t at = 2 * (int64_t)s_off[t] + (kk >> 4) * 512 + ln * 8 + h;
        Ch[at] = hv;
        Ch[at + 256] = __float2half_rn(v - __half2float(hv));
      }
    }
  }
  for (int row = tid; row < R_s; row += blockDim.x) s_rinv[row] = row < nrows ? (float)pr.rinv[s0 + row] : 0.f;
  for (int i = tid; i < k * R_s; i += blockDim.x) {
    const int m = i / R_s, row = i % R_s;
    const bool ok = row < nrows;
    phT[i] = ok ? Phi[(s0 + row) * pk + m] : 0.f;
    aT[i] = ok ? CPhi[(s0 + row) * pk + m] : 0.f;
  }
  for (int i = tid; i < 3 * k * k; i += blockDim.x) {
    const int w3 = i / (k * k), e = i % (k * k), ii = e / k, jj = e % k;
    s_gram[w3][e] = (float)pr.gram[w3 * pk * pk + ii * pk + jj];
  }
  for (int m = tid; m < k; m += blockDim.x) s_theta[m] = (float)pr.theta[m];
  __shared__ int s_npush, s_nrpush;
  if (tid == 0) { s_npush = 0; s_nrpush = 0; }
  __syncthreads();
  for_each_push([&](int row, int c2, int wrow) {
    const int slot = atomicAdd(&s_npush, 1);
    push[slot] = make_int2(row | (c2 << 16), wrow);
  });
  if (learn_ok)
    for_each_push_w(kTH, kTH, [&](int row, int c2, int wrow) {
      const int slot = atomicAdd(&s_nrpush, 1);
      rpush[slot] = make_int2(row | (c2 << 16), wrow);
    });
  const double cmin = pr.scal[1];
  const int maxit = pr.fixed_iters > 0 ? pr.fixed_iters : pr.max_iter;
  const float tol2f = (float)(pr.tol * pr.tol);

  // Per-shift lane scalars, staged once: sigma = s_q + 1 as FP32, the
  // preconditioner's beta - sigma (App. E) and the learned scale a_q (> 0 when
  // the term applies to shift q); slot Q is the mean system (sigma = 1).
  __shared__ float s_qsigf[kQTab], s_qbmf[kQTab], s_qla[kQTab];
  const bool qtab = pr.Q + 1 <= kQTab;
  auto shift_scalars = [&](int qs, float& sgf, float& bmf, float& la0) {
    const double sg = qs >= pr.Q ? 1.0 : pr.s[qs] + 1.0;
    sgf = (float)sg;
    bmf = (float)(sg + cmin) - sgf;
    la0 = pr.learn_coef[(int64_t)qs * kLearnOut];
  };
  if (qtab)
    for (int qs = tid; qs <= pr.Q; qs += blockDim.x) shift_scalars(qs, s_qsigf[qs], s_qbmf[qs], s_qla[qs]);
  __shared__ LoopArgs LA;
  if (tid == 0) {
    LA.learn_T = pr.learn_T;
    LA.bmean = pr.bmean;
    LA.U = reinterpret_cast<float*>(pr.U);
    LA.iters = pr.iters;
    LA.relres = pr.relres;
    LA.status = pr.status;
    LA.mean_sys = (int)pr.mean_sys;
    LA.Q = pr.Q;
    LA.nsys = (int)pr.nsys;
    LA.fixed_iters = pr.fixed_iters;
  }
  __syncthreads();
  // Starts system sid in lane j (scalars; the taps of the learned term follow
  // with the lane's right-hand side in lane_vectors_all).
  auto lane_scalars = [&](int j, int code) {
    const bool retry = code >= kRetry;
    const int sid = retry ? code - kRetry : code;
    L.sid[j] = sid;
    L.fin[j] = 0;
    L.learn[j] = 0;
    L.la[j] = 1.f;
    L.qs[j] = -1;
    L.mem[j] = -1;
    float sgf = 1.f, bmf = (float)(1.0 + cmin) - 1.f;
    if (sid < 0) {
      L.state[j] = kEmpty;
    } else {
      L.state[j] = kStart;
      const int q = sid < LA.mean_sys ? -1 : (sid - LA.mean_sys) / (int)N;
      if (q >= 0) L.mem[j] = sid - LA.mean_sys - q * (int)N;
      const int qs = q < 0 ? LA.Q : q;
      float la0;
      if (qtab) {
        sgf = s_qsigf[qs];
        bmf = s_qbmf[qs];
        la0 = s_qla[qs];
      } else {
        shift_scalars(qs, sgf, bmf, la0);
      }
      if (learn_ok && !retry && la0 > 0.f) {
        L.learn[j] = 1;
        L.la[j] = la0;
        L.qs[j] = qs;
      }
    }
    L.sigf[j] = sgf;
    L.bmf[j] = bmf;
    L.it[j] = 0;
    L.alpha[j] = 0.f;
    L.beta[j] = 0.f;
    L.rho[j] = 0.f;
  };
  // Own rows of r and x for every lane in state kStart: x = 0, and r receives the
  // member's observed anomalies by asynchronous copies that complete during the
  // matvec; the residual step scales them by R^-1/2 (the mean system's
  // right-hand side, already scaled, is stored directly).
  __shared__ int s_start[kJ], s_nstart, s_live, s_anyl;
  auto lane_masks = [&]() {           // warp 0: which lanes are live / just started / use the learned term
    if (tid < kJ) {
      const unsigned lm = __ballot_sync(0xffffffffu, L.state[tid] != kEmpty);
      const unsigned sm = __ballot_sync(0xffffffffu, L.state[tid] == kStart);
      const unsigned ll = __ballot_sync(0xffffffffu, L.learn[tid] != 0);
      if (sm & (1u << tid)) s_start[__popc(sm & ((1u << tid) - 1u))] = tid;
      if (tid == 0) { s_live = lm != 0u; s_nstart = __popc(sm); s_anyl = ll != 0u; }
    }
  };
  auto lane_vectors_all = [&]() {
    const int ns = s_nstart;
    // taps of T = S^T S of the started lanes (zero without the learned term)
    for (int e = tid; e < ns * kTT; e += blockDim.x) {
      const int j = s_start[e / kTT], u = e % kTT, qs = L.qs[j];
      if (qs >= 0) cp_async4(&L.ltT[u][j], LA.learn_T + (int64_t)qs * kLearnT + u);
      else L.ltT[u][j] = 0.f;
    }
    for (int is = 0; is < ns; ++is) {
      const int j = s_start[is], i = L.mem[j];
      for (int row = tid; row < R_s; row += blockDim.x) {
        float* dst = vr + row * kLD + j;
        vx[row * kLD + j] = 0.f;
        if (row >= nrows) { *dst = 0.f; continue; }
        const int64_t a = s0 + row;
        if (i < 0) *dst = (float)LA.bmean[a];
        else cp_async4(dst, W + a * N + i);
      }
    }
    cp_async_commit();
  };
  // first lanes: rank 0 takes kJ systems and pushes their ids to every CTA
  if (crank == 0 && warp == 0) {
    int base = 0;
    if (lane == 0) base = atomicAdd(queue, kJ);
    base = __shfl_sync(0xffffffffu, base, 0);
    const int v = base + lane < pr.nsys ? base + lane : -1;
    for (int dst = 0; dst < CS; ++dst) cluster.map_shared_rank(&L.newsid[0], dst)[lane] = v;
  }
  cluster.sync();
  if (tid < kJ) lane_scalars(tid, L.newsid[tid]);
  if (tid < kJ) { s_pscale[tid] = 1.f; s_pinv[tid] = 1.f; }
  lane_masks();
  __syncthreads();
  lane_vectors_all();
  cluster.sync();   // all CTAs initialized before anyone pushes into their windows
  BAND_PHASE(kPhases + 1);

  for (;;) {
    // ---------------- A: y = sigma p + C p on the own rows, partial p^T y ----------------
    // On the tensor cores: mma.sync m16n8k16 with FP16 operands and FP32
    // accumulation.  C (per row) and p (per lane, over the whole cluster) are
    // scaled by powers of two into [0.5, 1) and split into FP16 hi + lo, and
    // each product is taken in three terms, a b = a_h b_h + (a_h b_l + a_l b_h),
    // which keeps it near FP32 accuracy; the scales are undone exactly.  A warp
    // takes one 16-row tile (its A operand) and runs over the tile's 16-column
    // chunks (the k steps) for all kJ lanes.  Column n of n-block nb is lane
    // 4 n + nb: a thread's B operands for the four n-blocks then come from one
    // 16-byte load per k row, and its results are lanes 8 q .. 8 q + 7 of rows
    // g and g + 8 (g = lane / 4, q = lane % 4).
    {
      const int g = lane >> 2, q = lane & 3;
      const float4 ps4 = ld4(&s_pscale[4 * g]);   // scales of this thread's B columns (lanes 4 g + nb)
      const float psc[4] = {ps4.x, ps4.y, ps4.z, ps4.w};
      DotAcc<float> pp[8];   // p^T y of lanes 8 q + i over this warp's rows
      for (int t = warp; t < ntiles; t += kNW) {
        const int rA = t * kTile + g, rB = rA + 8;
        float dA[8], dB[8], eA[8], eB[8];   // a_h b_h and the correction terms, lanes 8 q + i
#pragma unroll
        for (int i = 0; i < 8; ++i) { dA[i] = 0.f; dB[i] = 0.f; eA[i] = 0.f; eB[i] = 0.f; }
        const float* ct = Ct + s_off[t] + 4 * lane;
        const float* pb = pw + (s_klo[t] + hl + 2 * q) * kLD + 4 * g;
        const int nch = s_w[t] >> 4;
#pragma unroll 2
        for (int c = 0; c < nch; ++c) {
          const uint4 ah = *reinterpret_cast<const uint4*>(ct + c * 256);
          const uint4 al = *reinterpret_cast<const uint4*>(ct + c * 256 + 128);
          const float* pc = pb + (16 * c) * kLD;
          const float4 k0 = ld4(pc), k1 = ld4(pc + kLD);                // B rows 2q, 2q + 1
          const float4 k8 = ld4(pc + 8 * kLD), k9 = ld4(pc + 9 * kLD);  // B rows 2q + 8, 2q + 9
          const float b0[4] = {k0.x, k0.y, k0.z, k0.w}, b1[4] = {k1.x, k1.y, k1.z, k1.w};
          const float b8[4] = {k8.x, k8.y, k8.z, k8.w}, b9[4] = {k9.x, k9.y, k9.z, k9.w};
#pragma unroll
          for (int nb = 0; nb < 4; ++nb) {
            uint32_t h0, l0, h1, l1;
            f16_split2(b0[nb] * psc[nb], b1[nb] * psc[nb], h0, l0);
            f16_split2(b8[nb] * psc[nb], b9[nb] * psc[nb], h1, l1);
            mma_f16(dA[nb], dA[4 + nb], dB[nb], dB[4 + nb], ah, h0, h1);
            mma_f16(eA[nb], eA[4 + nb], eB[nb], eB[4 + nb], ah, l0, l1);
            mma_f16(eA[nb], eA[4 + nb], eB[nb], eB[4 + nb], al, h0, h1);
          }
        }
        // D element i of a row is lane 8 q + i after the permutation above
        const float4 si0 = ld4(&s_pinv[8 * q]), si1 = ld4(&s_pinv[8 * q + 4]);
        const float4 sg0 = ld4(&L.sigf[8 * q]), sg1 = ld4(&L.sigf[8 * q + 4]);
        const float un[8] = {si0.x, si0.y, si0.z, si0.w, si1.x, si1.y, si1.z, si1.w};
        const float sg[8] = {sg0.x, sg0.y, sg0.z, sg0.w, sg1.x, sg1.y, sg1.z, sg1.w};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int row = h ? rB : rA;
          if (row < nrows) {
            const float ir = rsi[row];   // inverse scale of this row of C
            const float4 p0 = ld4(pw + (row + hl) * kLD + 8 * q), p1 = ld4(pw + (row + hl) * kLD + 8 * q + 4);
            const float pv[8] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
            float y[8];
#pragma unroll
            for (int i = 0; i < 8; ++i)
              y[i] = fmaf(sg[i], pv[i], ((h ? dB[i] : dA[i]) + (h ? eB[i] : eA[i])) * (ir * un[i]));
            st4(vy + (row + kTH) * kLD + 8 * q, make_float4(y[0], y[1], y[2], y[3]));
            st4(vy + (row + kTH) * kLD + 8 * q + 4, make_float4(y[4], y[5], y[6], y[7]));
#pragma unroll
            for (int i = 0; i < 8; ++i) pp[i].add_prod(pv[i], y[i]);
          }
        }
      }
      // reduce-scatter the eight float-float sums over g (lane bits 4, 3, 2):
      // lane (g, q) ends with the sum of lane 8 q + g
      float vh[8], vl[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) { vh[i] = pp[i].hi; vl[i] = pp[i].lo; }
#pragma unroll
      for (int lev = 0; lev < 3; ++lev) {
        const int off = 16 >> lev, half = 4 >> lev;
        const bool up = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
          const float sh = up ? vh[i] : vh[i + half], sl = up ? vl[i] : vl[i + half];
          float kh = up ? vh[i + half] : vh[i], kl = up ? vl[i + half] : vl[i];
          ff_merge(kh, kl, __shfl_xor_sync(0xffffffffu, sh, off), __shfl_xor_sync(0xffffffffu, sl, off));
          vh[i] = kh;
          vl[i] = kl;
        }
      }
      s_wpap[warp][8 * q + g][0] = vh[0];
      s_wpap[warp][8 * q + g][1] = vl[0];
    }
    BAND_PHASE(0);
    __syncthreads();
    if (tid < (kJ / 2) * CS) {   // two lanes per thread: one 16-byte store per destination
      const int j = 2 * (tid % (kJ / 2)), dst = tid / (kJ / 2);
      float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
      for (int w = 0; w < kNW; ++w) {
        ff_merge(h0, l0, s_wpap[w][j][0], s_wpap[w][j][1]);
        ff_merge(h1, l1, s_wpap[w][j + 1][0], s_wpap[w][j + 1][1]);
      }
      st4(cluster.map_shared_rank(&s_pap_in[crank][j][0], dst), make_float4(h0, l0, h1, l1));
    }
    cluster_arrive();
    cp_async_wait_all();   // right-hand sides of lanes started in the previous step
    cluster_wait();   // (1)
    BAND_PHASE(1);
    // ---------------- alpha ----------------
    if (tid < kJ) {
      const int j = tid;
      float hi = 0.f, lo = 0.f;
      for (int c = 0; c < CS; ++c) ff_merge(hi, lo, s_pap_in[c][j][0], s_pap_in[c][j][1]);
      const float pAp = hi + lo;          // alpha is FP32: no FP64 division here
      float alpha = 0.f;
      if (L.state[j] == kActive) {
        if (pAp > 0.f && isfinite(pAp)) {
          alpha = L.rho[j] / pAp;
          L.it[j] += 1;
        } else {
          L.fin[j] = 2;   // breakdown: finished with a flag
        }
      }
      L.alpha[j] = alpha;
    }
    __syncthreads();
    BAND_PHASE(2);
    // ---------------- x += alpha p, r -= alpha y; partial rr, Phi^T r, A^T r ----------------
    {
      const int j0 = 4 * warp;   // this warp's four lanes
      const float a0 = L.alpha[j0], a1 = L.alpha[j0 + 1], a2 = L.alpha[j0 + 2], a3 = L.alpha[j0 + 3];
      DotAcc<float> rr[4];
      // partial Phi^T r and A^T r of the four lanes: value jj * 2kK + (m | kK + m),
      // 80 values held as two blocks of 32 and one of 16
      float v0[32], v1[32], v2[16];
#pragma unroll
      for (int i = 0; i < 32; ++i) { v0[i] = 0.f; v1[i] = 0.f; }
#pragma unroll
      for (int i = 0; i < 16; ++i) v2[i] = 0.f;
      bool sc[4];
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) sc[jj] = L.state[j0 + jj] == kStart && L.mem[j0 + jj] >= 0;
      const bool any_sc = sc[0] | sc[1] | sc[2] | sc[3];
      // two rows (row, row + 32) per iteration, every shared-memory load of
      // both issued before their arithmetic; sums run in row order
      const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int row = lane; row < nrows; row += 64) {
        const int rb = row + 32;
        const bool hb = rb < nrows;
        const float4 p4a = ld4(pw + (row + hl) * kLD + j0), y4a = ld4(vy + (row + kTH) * kLD + j0);
        const float4 x4a = ld4(vx + row * kLD + j0), r4a0 = ld4(vr + row * kLD + j0);
        const float4 p4b = hb ? ld4(pw + (rb + hl) * kLD + j0) : zero4;
        const float4 y4b = hb ? ld4(vy + (rb + kTH) * kLD + j0) : zero4;
        const float4 x4b = hb ? ld4(vx + rb * kLD + j0) : zero4, r4b0 = hb ? ld4(vr + rb * kLD + j0) : zero4;
        float ra[4] = {r4a0.x, r4a0.y, r4a0.z, r4a0.w}, rb4[4] = {r4b0.x, r4b0.y, r4b0.z, r4b0.w};
        if (any_sc) {                                   // b = R^-1/2 w of a lane started last step
          const float ria = s_rinv[row], rib = hb ? s_rinv[rb] : 0.f;
#pragma unroll
          for (int jj = 0; jj < 4; ++jj)
            if (sc[jj]) { ra[jj] *= ria; rb4[jj] *= rib; }
        }
        const float al[4] = {a0, a1, a2, a3};
        const float pa[4] = {p4a.x, p4a.y, p4a.z, p4a.w}, pb[4] = {p4b.x, p4b.y, p4b.z, p4b.w};
        const float ya[4] = {y4a.x, y4a.y, y4a.z, y4a.w}, yb[4] = {y4b.x, y4b.y, y4b.z, y4b.w};
        float xa[4] = {x4a.x, x4a.y, x4a.z, x4a.w}, xb[4] = {x4b.x, x4b.y, x4b.z, x4b.w};
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
          xa[jj] = fmaf(al[jj], pa[jj], xa[jj]);
          xb[jj] = fmaf(al[jj], pb[jj], xb[jj]);
          ra[jj] = fmaf(-al[jj], ya[jj], ra[jj]);
          rb4[jj] = fmaf(-al[jj], yb[jj], rb4[jj]);
        }
        const float4 r4a = make_float4(ra[0], ra[1], ra[2], ra[3]), r4b = make_float4(rb4[0], rb4[1], rb4[2], rb4[3]);
        st4(vx + row * kLD + j0, make_float4(xa[0], xa[1], xa[2], xa[3]));
        st4(vr + row * kLD + j0, r4a);
        st4(vy + (row + kTH) * kLD + j0, r4a);     // r window (y is no longer needed)
        if (hb) {
          st4(vx + rb * kLD + j0, make_float4(xb[0], xb[1], xb[2], xb[3]));
          st4(vr + rb * kLD + j0, r4b);
          st4(vy + (rb + kTH) * kLD + j0, r4b);
        }
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
          rr[jj].add_prod(ra[jj], ra[jj]);
          rr[jj].add_prod(rb4[jj], rb4[jj]);   // zero for a missing second row
        }
#pragma unroll
        for (int m = 0; m < kK; ++m) {
          if (m < k) {
            const float pha = phT[m * R_s + row], ata = aT[m * R_s + row];
            const float phb = hb ? phT[m * R_s + rb] : 0.f, atb = hb ? aT[m * R_s + rb] : 0.f;
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
              const int idx = jj * 2 * kK + m, idg = idx + kK;
              float& vf = idx < 32 ? v0[idx] : idx < 64 ? v1[idx - 32] : v2[idx - 64];
              vf = fmaf(phb, rb4[jj], fmaf(pha, ra[jj], vf));
              float& vg = idg < 32 ? v0[idg] : idg < 64 ? v1[idg - 32] : v2[idg - 64];
              vg = fmaf(atb, rb4[jj], fmaf(ata, ra[jj], vg));
            }
          }
        }
      }
      BAND_PHASE(3);
      // learned term, applied periodically across the slices: the halo rows of
      // the r window go to the CTAs that hold them (split barrier 2a: the
      // warp reductions below run while the rows are in flight)
      if (s_anyl) {
        __syncthreads();
        const int nrp = s_nrpush;
        for (int e = tid; e < nrp * (kJ / 4); e += blockDim.x) {
          const int2 t = rpush[e / (kJ / 4)];
          const int q4 = e % (kJ / 4);
          const int row = t.x & 0xffff, c2 = t.x >> 16;
          st4(cluster.map_shared_rank(vy, c2) + t.y * kLD + 4 * q4, ld4(vy + (row + kTH) * kLD + 4 * q4));
        }
        cluster_arrive();   // (2a)
      }
      // the warp's partial Phi^T r and A^T r are reduced first, which frees
      // their 80 registers before the learned term's stencil
      const float s0v = warp_reduce_scatter32<float>(v0, lane);
      const float s1v = warp_reduce_scatter32<float>(v1, lane);
      // 16-value block: fold the warp halves, then reduce-scatter over 16 lanes
#pragma unroll
      for (int i = 0; i < 16; ++i) v2[i] += __shfl_xor_sync(0xffffffffu, v2[i], 16);
#pragma unroll
      for (int off = 8; off >= 1; off >>= 1) {
        const bool up = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < off; ++i) {
          const float send = up ? v2[i] : v2[i + off];
          const float keep = up ? v2[i + off] : v2[i];
          v2[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
      }
      const float sv[3] = {s0v, s1v, v2[0]};
      // r^T r of the four lanes: four float-float values reduce-scattered over
      // the lane bits 4, 3 and summed over bits 2, 1, 0; lane L ends with r^T r
      // of lane j0 + qj, qj = 2 b4 + b3.  Lanes with bit 2 set carry r^T T r
      // of the same lane instead (learned term, below).
      float vh[4], vl[4];
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) { vh[jj] = rr[jj].hi; vl[jj] = rr[jj].lo; }
#pragma unroll
      for (int lev = 0; lev < 2; ++lev) {
        const int off = 16 >> lev, half = 2 >> lev;
        const bool up = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
          const float sh = up ? vh[i] : vh[i + half], sl = up ? vl[i] : vl[i + half];
          float kh = up ? vh[i + half] : vh[i], kl = up ? vl[i + half] : vl[i];
          ff_merge(kh, kl, __shfl_xor_sync(0xffffffffu, sh, off), __shfl_xor_sync(0xffffffffu, sl, off));
          vh[i] = kh;
          vl[i] = kl;
        }
      }
      float qh = vh[0], ql = vl[0];
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, qh, o);
        const float l2 = __shfl_xor_sync(0xffffffffu, ql, o);
        ff_merge(qh, ql, h2, l2);
      }
      const int qj = ((lane >> 4) & 1) * 2 + ((lane >> 3) & 1);
      const bool q_uu = (lane & 4) != 0;
      if (q_uu) { qh = 0.f; ql = 0.f; }
      // T r = S^T S r then replaces r on the own rows of the window, where the
      // direction update reads it
      if (s_anyl) {
        cluster_wait();   // (2a) r windows complete
        // thread = (system lane `lane`, own rows kStRows warp ..): the
        // kStRows + 2 kTH rows of its window are read once into registers,
        // one conflict-free wavefront per row for the warp (lanes without the
        // term have zero taps and produce zeros)
        const int jl = lane, r0 = kStRows * warp;
        DotAcc<float> ua;
        float tr[kStRows];
        if (r0 < R_s) {
          float tap[kTT], win[kStRows + 2 * kTH];
#pragma unroll
          for (int tp = 0; tp < kTT; ++tp) tap[tp] = L.ltT[tp][jl];
#pragma unroll
          for (int i = 0; i < kStRows + 2 * kTH; ++i)
            win[i] = r0 + i < R_s + 2 * kTH ? vy[(r0 + i) * kLD + jl] : 0.f;
#pragma unroll
          for (int o = 0; o < kStRows; ++o) {
            float acc = 0.f;
#pragma unroll
            for (int tp = 0; tp < kTT; ++tp) acc = fmaf(tap[tp], win[o + tp], acc);   // r[row + tp - kTH]
            tr[o] = acc;
            if (r0 + o < nrows) ua.add_prod(win[o + kTH], acc);
          }
        }
        s_wpap[warp][jl][0] = ua.hi;   // p^T y partials were consumed by alpha
        s_wpap[warp][jl][1] = ua.lo;
        __syncthreads();   // every window read
        if (r0 < R_s) {
#pragma unroll
          for (int o = 0; o < kStRows; ++o)
            if (r0 + o < R_s) vy[(r0 + o + kTH) * kLD + jl] = tr[o];
        }
        if (q_uu) {
          float uh = 0.f, ul = 0.f;
          for (int w = 0; w < kNW; ++w) ff_merge(uh, ul, s_wpap[w][j0 + qj][0], s_wpap[w][j0 + qj][1]);
          qh = uh;
          ql = ul;
        }
      }
      BAND_PHASE(4);
      const int qdst = (j0 + qj) * kNR + (q_uu ? 2 : 0);
      // push this warp's four lanes to every CTA of the cluster.  Distributed
      // shared-memory stores are separate transactions, so the four lanes of
      // a group 4 k .. 4 k + 3 gather values 4 k .. 4 k + 3 of each block into
      // one 16-byte word (2 kK is a multiple of 4, so a group never straddles
      // two lanes' rows) and share the destinations: lane 4 k + c stores to
      // ranks c, c + 4, ...
      float4 sv4[3];
      const int gbase = lane & ~3;
#pragma unroll
      for (int b = 0; b < 3; ++b)
        sv4[b] = make_float4(__shfl_sync(0xffffffffu, sv[b], gbase), __shfl_sync(0xffffffffu, sv[b], gbase + 1),
                             __shfl_sync(0xffffffffu, sv[b], gbase + 2), __shfl_sync(0xffffffffu, sv[b], gbase + 3));
      static_assert((2 * kK) % 4 == 0 && kNR % 4 == 0, "16-byte groups of the residual partials");
      for (int dst = lane & 3; dst < CS; dst += 4) {
        float* base = cluster.map_shared_rank(&s_res_in[crank][0][0], dst);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          const int idx = 32 * b + gbase;          // = jj * 2kK + (m or kK + m)
          if (idx >= 4 * 2 * kK) continue;
          const int jj = idx / (2 * kK), w = idx % (2 * kK);
          st4(base + (j0 + jj) * kNR + 4 + w, sv4[b]);
        }
        *reinterpret_cast<float2*>(base + qdst) = make_float2(qh, ql);
      }
    }
    cluster.sync();   // (2)
    BAND_PHASE(5);
    // ---------------- decisions, then z = P^-1 r and p = z + beta p ----------------
    // Each warp handles its four lanes (the lanes of the residual step), so no
    // block barrier is needed until the queue.  Sums over the cluster are taken
    // in rank order from the local receive buffers, identically in every CTA.
    // Preconditioner algebra: t = T^-1 f, t2 = g + sigma f - G_q t,
    // c = (beta - sigma) t - T^-1 t2, with G_q = (C_q Phi)^T (C_q Phi).
    {
      const int j0 = 4 * warp;
      static_assert(kK <= 16, "two Ritz indices per thread");
      {
        // eight threads per lane: thread m0 = lane % 8 of lane j holds Ritz
        // indices m0 and m0 + 8
        const int j = j0 + (lane >> 3);
        const int mA = lane & 7, mB = mA + 8;
        const bool vA = mA < k, vB = mB < k;
        // pairwise (tree) sums over the cluster's partials, the same order in every CTA
        float fa[kMaxCS], ga[kMaxCS], fb[kMaxCS], gb[kMaxCS];
#pragma unroll
        for (int c = 0; c < kMaxCS; ++c) {
          fa[c] = (vA && c < CS) ? s_res_in[c][j][4 + mA] : 0.f;
          ga[c] = (vA && c < CS) ? s_res_in[c][j][4 + kK + mA] : 0.f;
          fb[c] = (vB && c < CS) ? s_res_in[c][j][4 + mB] : 0.f;
          gb[c] = (vB && c < CS) ? s_res_in[c][j][4 + kK + mB] : 0.f;
        }
#pragma unroll
        for (int w2 = 1; w2 < kMaxCS; w2 <<= 1)
#pragma unroll
          for (int c = 0; c + w2 < kMaxCS; c += 2 * w2) {
            fa[c] += fa[c + w2];
            ga[c] += ga[c + w2];
            fb[c] += fb[c + w2];
            gb[c] += gb[c + w2];
          }
        const float sg = L.sigf[j];
        const float rthA = vA ? __frcp_rn(s_theta[mA] + sg) : 0.f;   // (T_q)^-1 entries
        const float rthB = vB ? __frcp_rn(s_theta[mB] + sg) : 0.f;
        const float tA = fa[0] * rthA, tB = fb[0] * rthB;
        float t2A = ga[0] + sg * fa[0], t2B = gb[0] + sg * fb[0];
        auto gq = [&](int mm, int i) {   // (G_q)_{mm i}
          return s_gram[2][mm * k + i] + sg * (s_gram[1][mm * k + i] + s_gram[1][i * k + mm]) +
                 sg * sg * s_gram[0][mm * k + i];
        };
#pragma unroll
        for (int i = 0; i < kK; ++i) {
          const float ti = __shfl_sync(0xffffffffu, i < 8 ? tA : tB, (lane & 24) + (i & 7));
          if (i < k) {
            if (vA) t2A = fmaf(-gq(mA, i), ti, t2A);
            if (vB) t2B = fmaf(-gq(mB, i), ti, t2B);
          }
        }
        const float bm = L.bmf[j];
        const float ccA = vA ? fmaf(bm, tA, -t2A * rthA) : 0.f;
        const float ccB = vB ? fmaf(bm, tB, -t2B * rthB) : 0.f;
        if (vA) { L.t[j][mA] = tA; L.c[j][mA] = ccA; }
        if (vB) { L.t[j][mB] = tB; L.c[j][mB] = ccB; }
        // rho = r^T M r = a r^T P^-1 r + r^T S^T S r.  The dot products are
        // float-float (FP64-accurate); rho, alpha and beta multiply FP32
        // vectors and are formed in FP32, and so is the k-term LMP correction.
        float corr = (vA ? fmaf(fa[0], ccA, -ga[0] * tA) : 0.f) + (vB ? fmaf(fb[0], ccB, -gb[0] * tB) : 0.f);
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) corr += __shfl_xor_sync(0xffffffffu, corr, o);
        const int m = mA;
        if (m == 0) {
          float rh[kMaxCS], rl[kMaxCS], uh[kMaxCS], ul[kMaxCS];
#pragma unroll
          for (int c = 0; c < kMaxCS; ++c) {
            const bool in = c < CS;
            rh[c] = in ? s_res_in[c][j][0] : 0.f;
            rl[c] = in ? s_res_in[c][j][1] : 0.f;
            uh[c] = in ? s_res_in[c][j][2] : 0.f;
            ul[c] = in ? s_res_in[c][j][3] : 0.f;
          }
#pragma unroll
          for (int w2 = 1; w2 < kMaxCS; w2 <<= 1)
#pragma unroll
            for (int c = 0; c + w2 < kMaxCS; c += 2 * w2) {
              ff_merge(rh[c], rl[c], rh[c + w2], rl[c + w2]);
              ff_merge(uh[c], ul[c], uh[c + w2], ul[c + w2]);
            }
          const float hi = rh[0], lo = rl[0], hu = uh[0], lu = ul[0];
          L.rrh[j] = hi;
          L.rrl[j] = lo;
          const float rr = hi + lo;
          const float rho = L.la[j] * (rr + corr) + (L.learn[j] ? hu + lu : 0.f);
          const int st = L.state[j];
          if (st == kStart) {
            L.bn2[j] = rr;
            if (!(rr > 0.f) || !isfinite(rr)) {
              L.fin[j] = isfinite(rr) ? 1 : 2;
            } else {
              L.state[j] = kActive;
              L.rho[j] = rho;
              L.beta[j] = 0.f;
            }
          } else if (st == kActive && L.fin[j] == 0) {
            bool done = false;
            if (!isfinite(rr)) { done = true; L.fin[j] = 2; }
            else if (LA.fixed_iters > 0) done = L.it[j] >= LA.fixed_iters || !(rr > 0.f);
            else done = !(rr > tol2f * L.bn2[j]) || L.it[j] >= maxit;
            if (done) {
              if (L.fin[j] == 0) L.fin[j] = 1;
            } else {
              L.beta[j] = rho / L.rho[j];
              L.rho[j] = rho;
            }
          }
        }
      }
      __syncwarp();
      BAND_PHASE(6);
      float tj[4][kK], cj[4][kK];
#pragma unroll
      for (int jj = 0; jj < 4; ++jj)
#pragma unroll
        for (int q4 = 0; q4 < kKP / 4; ++q4) {
          const float4 t4 = ld4(&L.t[j0 + jj][4 * q4]), c4 = ld4(&L.c[j0 + jj][4 * q4]);
          const float tv[4] = {t4.x, t4.y, t4.z, t4.w}, cv[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int mm = 4 * q4 + e;
            if (mm < kK) {
              tj[jj][mm] = mm < k ? tv[e] : 0.f;
              cj[jj][mm] = mm < k ? cv[e] : 0.f;
            }
          }
        }
      bool act[4], fin[4];
      float bj[4], aj[4];
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        act[jj] = L.state[j0 + jj] == kActive && L.fin[j0 + jj] == 0;
        fin[jj] = L.fin[j0 + jj] != 0;
        bj[jj] = L.beta[j0 + jj];
        aj[jj] = L.la[j0 + jj];
      }
      const bool any_learn2 = L.learn[j0] | L.learn[j0 + 1] | L.learn[j0 + 2] | L.learn[j0 + 3];
      float pmx[4] = {0.f, 0.f, 0.f, 0.f};   // max |p| of the four lanes over this thread's rows
      float* U = LA.U;
      // two rows (row, row + 32) per iteration, every shared-memory load of
      // both issued before their arithmetic
      const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int row = lane; row < nrows; row += 64) {
        const int rb = row + 32;
        const bool hb = rb < nrows;
        const float4 r4a = ld4(vr + row * kLD + j0), p4a = ld4(pw + (row + hl) * kLD + j0);
        const float4 r4b = hb ? ld4(vr + rb * kLD + j0) : zero4, p4b = hb ? ld4(pw + (rb + hl) * kLD + j0) : zero4;
        float4 w4a = zero4, w4b = zero4;   // (T r)_row from the learned step
        if (any_learn2) {
          w4a = ld4(vy + (row + kTH) * kLD + j0);
          if (hb) w4b = ld4(vy + (rb + kTH) * kLD + j0);
        }
        float za[4] = {r4a.x, r4a.y, r4a.z, r4a.w}, zb[4] = {r4b.x, r4b.y, r4b.z, r4b.w};
#pragma unroll
        for (int mm = 0; mm < kK; ++mm) {
          if (mm < k) {
            const float pha = phT[mm * R_s + row], ata = aT[mm * R_s + row];
            const float phb = hb ? phT[mm * R_s + rb] : 0.f, atb = hb ? aT[mm * R_s + rb] : 0.f;
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
              za[jj] = fmaf(pha, cj[jj][mm], fmaf(-ata, tj[jj][mm], za[jj]));
              zb[jj] = fmaf(phb, cj[jj][mm], fmaf(-atb, tj[jj][mm], zb[jj]));
            }
          }
        }
        if (any_learn2) {
          const float wa[4] = {w4a.x, w4a.y, w4a.z, w4a.w}, wb[4] = {w4b.x, w4b.y, w4b.z, w4b.w};
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) {
            za[jj] = fmaf(aj[jj], za[jj], wa[jj]);
            zb[jj] = fmaf(aj[jj], zb[jj], wb[jj]);
          }
        }
        const float pva[4] = {p4a.x, p4a.y, p4a.z, p4a.w}, pvb[4] = {p4b.x, p4b.y, p4b.z, p4b.w};
        float pna[4], pnb[4];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
          pna[jj] = act[jj] ? fmaf(bj[jj], pva[jj], za[jj]) : 0.f;
          pnb[jj] = (act[jj] && hb) ? fmaf(bj[jj], pvb[jj], zb[jj]) : 0.f;
          pmx[jj] = fmaxf(pmx[jj], fmaxf(fabsf(pna[jj]), fabsf(pnb[jj])));
        }
        st4(pw + (row + hl) * kLD + j0, make_float4(pna[0], pna[1], pna[2], pna[3]));
        if (hb) st4(pw + (rb + hl) * kLD + j0, make_float4(pnb[0], pnb[1], pnb[2], pnb[3]));
#pragma unroll
        for (int jj = 0; jj < 4; ++jj)
          if (fin[jj]) {
            U[(int64_t)L.sid[j0 + jj] * d + s0 + row] = vx[row * kLD + j0 + jj];
            if (hb) U[(int64_t)L.sid[j0 + jj] * d + s0 + rb] = vx[rb * kLD + j0 + jj];
          }
      }
      // the lanes' max |p| over the own rows, to every CTA (the scale of p in the next matvec)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) pmx[jj] = fmaxf(pmx[jj], __shfl_xor_sync(0xffffffffu, pmx[jj], o));
      if (lane < CS) st4(cluster.map_shared_rank(&s_pmax_in[crank][j0], lane), make_float4(pmx[0], pmx[1], pmx[2], pmx[3]));
      BAND_PHASE(7);
    }
    __syncthreads();
    // finished lanes: stats, and rank 0 takes the next systems off the queue
    if (crank == 0 && warp == 0) {
      const int j = lane;
      const bool f = L.fin[j] != 0;
      const float bn = L.bn2[j];
      const float rrj = L.rrh[j] + L.rrl[j];
      const bool failed = f && (L.fin[j] == 2 || (LA.fixed_iters <= 0 && !(rrj <= tol2f * bn)));
      const bool retry = failed && L.learn[j];          // plain PCG solves it again
      const bool take = f && !retry;
      const unsigned fm = __ballot_sync(0xffffffffu, take);
      int base = 0;
      if (lane == 0 && fm) base = atomicAdd(queue, __popc(fm));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (f) {
        const int sid = L.sid[j];
        int v;
        if (retry) {
          v = sid + kRetry;
        } else {
          LA.iters[sid] = L.it[j];
          LA.relres[sid] = bn > 0.f ? (double)sqrtf(rrj / bn) : 0.0;
          if (L.fin[j] == 2) atomicOr(&LA.status[0], kStatBreakdown);
          else if (failed) atomicOr(&LA.status[0], kStatNotConverged);
          const int nid = base + __popc(fm & ((1u << j) - 1u));
          v = nid < LA.nsys ? nid : -1;
        }
        for (int dst = 0; dst < CS; ++dst) cluster.map_shared_rank(&L.newsid[0], dst)[j] = v;
      }
    }
    // push the own rows that other windows hold as halo rows
    {
      const int np = s_npush;
      for (int e = tid; e < np * (kJ / 4); e += blockDim.x) {
        const int2 t = push[e / (kJ / 4)];
        const int q4 = e % (kJ / 4);
        const int row = t.x & 0xffff, c2 = t.x >> 16;
        st4(cluster.map_shared_rank(pw, c2) + t.y * kLD + 4 * q4, ld4(pw + (row + hl) * kLD + 4 * q4));
      }
    }
    cluster.sync();   // (3)
    BAND_PHASE(8);
    // ---------------- refills, exit test, halo ----------------
    if (tid < kJ && L.fin[tid]) lane_scalars(tid, L.newsid[tid]);
    if (tid < kJ) {
      float m = 0.f;
      for (int c = 0; c < CS; ++c) m = fmaxf(m, s_pmax_in[c][tid]);
      pow2_scale(m, s_pscale[tid], s_pinv[tid]);
    }
    lane_masks();
    __syncthreads();
    if (!s_live) break;
    lane_vectors_all();   // lanes started in this step: own rows of r and x
    __syncthreads();
    BAND_PHASE(9);
#ifdef INFO_ESRF_PHASE_CLOCKS
    if (tid == 0) s_ph[kPhases] += 1;
#endif
  }
  cluster.sync();   // no CTA leaves while another may still read its shared memory
#ifdef INFO_ESRF_PHASE_CLOCKS
  if (tid < kPhaseSlots - 1) atomicAdd(&g_band_phase[tid], (unsigned long long)s_ph[tid]);
  if (tid == 0) atomicAdd(&g_band_phase[kPhaseSlots - 1], 1ull);
#endif
}

// Whether the band kernel above can take problem p (FP32, at most kK Ritz
// vectors, a one-dimensional grid); the kernel itself checks the band reach
// and the shared-memory budget and otherwise sets the fall-back flag.
bool band1d_eligible(const ProblemDev& p) {
  if (p.precision != 1 || p.kR > kK || p.nsys < 1 || p.H_rowptr) return false;   // dense C: the general kernel
  int active = 0;
  for (int ax = 0; ax < 3; ++ax) active += p.grid.ext[ax] > 1;
  return active == 1 && p.grid.ext[0] > 1;
}

// Cluster size for problem p: the requested one (0: 8), halved while a CTA
// would own fewer than two row tiles.
int band1d_cluster_size(const ProblemDev& p, int requested) {
  int CS = requested > 0 ? requested : kMaxCS;
  while (CS > 1 && (p.d + CS - 1) / CS < 2 * kTile) CS >>= 1;
  return CS;
}

// Launch facts that depend only on the device (the dynamic shared-memory
// size and its function attribute) or on the device and the cluster size (the
// co-resident cluster count), looked up once per thread and device.
struct BandLaunchInfo {
  bool ready = false;
  int dyn_bytes = 0;                  // <= 0: the kernel cannot be configured on this device
  int max_clusters[kMaxCS + 1] = {};  // 0: not looked up yet, -1: this cluster shape cannot run
};

int launch_pcg_band1d(const ProblemDev& p, const ProblemDev* dp, int CS, int32_t* queue, int32_t* fallback,
                      int num_sms, cudaStream_t st) {
  int clusters = (p.nsys + kJ - 1) / kJ;
  if (clusters > num_sms / CS) clusters = num_sms / CS;
  if (clusters < 1) clusters = 1;
  constexpr int kMaxDev = 64;
  static thread_local BandLaunchInfo info_by_dev[kMaxDev];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev || CS < 1 || CS > kMaxCS) {
    cudaGetLastError();
    return -1;
  }
  BandLaunchInfo& info = info_by_dev[dev];
  if (!info.ready) {
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    cudaFuncGetAttributes(&fa, k_pcg_band1d);
    info.dyn_bytes = (optin - (int)fa.sharedSizeBytes - 1024) & ~15;
    if (info.dyn_bytes <= 0 ||
        cudaFuncSetAttribute(k_pcg_band1d, cudaFuncAttributeMaxDynamicSharedMemorySize, info.dyn_bytes) !=
            cudaSuccess) {
      cudaGetLastError();
      info.dyn_bytes = 0;
    }
    info.ready = true;
  }
  const int dyn_bytes = info.dyn_bytes;
  if (dyn_bytes <= 0) return -1;
  cudaMemsetAsync(queue, 0, sizeof(int32_t), st);
  cudaMemsetAsync(fallback, 0, sizeof(int32_t), st);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(clusters * CS, 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = dyn_bytes;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // A cluster shape this GPU cannot co-schedule is left to the general kernel;
  // launch no more clusters than can run at once (later ones would only find
  // the queue drained).
  if (info.max_clusters[CS] == 0) {
    int mc = 0;
    if (cudaOccupancyMaxActiveClusters(&mc, k_pcg_band1d, &cfg) != cudaSuccess || mc < 1) {
      cudaGetLastError();
      mc = -1;
    }
    info.max_clusters[CS] = mc;
  }
  const int max_clusters = info.max_clusters[CS];
  if (max_clusters < 1) return -1;
  if (clusters > max_clusters) {
    clusters = max_clusters;
    cfg.gridDim = dim3(clusters * CS, 1, 1);
  }
  const cudaError_t err = cudaLaunchKernelEx(&cfg, k_pcg_band1d, dp, queue, fallback, dyn_bytes / 4);
  if (err != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  note_launches(1);
  return 0;
}

}  // namespace infoesrf

extern "C" int info_esrf_band_phase_clocks(int64_t* out, int32_t n, int32_t reset) {
#ifdef INFO_ESRF_PHASE_CLOCKS
  using namespace infoesrf;
  if (!out || n < 1) return INFO_ESRF_ERR_INVALID_ARG;
  unsigned long long h[kPhaseSlots] = {};
  if (cudaMemcpyFromSymbol(h, g_band_phase, sizeof(h)) != cudaSuccess) {
    cudaGetLastError();
    return INFO_ESRF_ERR_CUDA;
  }
  for (int i = 0; i < n && i < kPhaseSlots; ++i) out[i] = (int64_t)h[i];
  if (reset) {
    const unsigned long long z[kPhaseSlots] = {};
    if (cudaMemcpyToSymbol(g_band_phase, z, sizeof(z)) != cudaSuccess) {
      cudaGetLastError();
      return INFO_ESRF_ERR_CUDA;
    }
  }
  return 0;
#else
  (void)out;
  (void)n;
  (void)reset;
  return INFO_ESRF_ERR_UNSUPPORTED;
#endif
}
