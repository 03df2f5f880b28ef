// a6-a8, BF16 path: batched shifted PCG over every (node, member) system and
// the mean system (App. E, Eq. normalized_linear_solve; Golub & Van Loan
// Alg. 11.5.1) with the limited-memory preconditioner of App. E, as a
// sequence of kernels per iteration over all systems at once:
//
//   1. y_j = sigma_j p_j + C p_j and row-tile partials of p_j^T y_j
//      (tensor-core block-tile matvec, tile_matvec.cu);
//   2. alpha_j = rho_j / p_j^T y_j (FP64, partials summed in a fixed order);
//   3. x_j += alpha_j p_j, r_j -= alpha_j y_j, and partials of r^T r,
//      f = Phi^T r, g = (C Phi)^T r (FP32 per thread, FP64 across threads);
//   4. per system: convergence test ||r|| <= tol ||b||, the preconditioner
//      coefficients t = T^-1 f, c = (beta_lmp - sigma) t - T^-1 (g + sigma f - G_q t)
//      with G_q = (C_q Phi)^T (C_q Phi), rho' = r^T z = r^T r - g.t + f.c and
//      beta = rho' / rho (FP64);
//   5. p_j = bf16(z_j + beta_j p_j), z = r - (C Phi) t + Phi c.
//
// Learned correction (2-D observation lattices with a model; tile_learn.cu):
// after step 3, u = S r and u^T u; step 4 takes rho = a (r^T P^-1 r) + u^T u,
// step 5 z = a P^-1 r + S u.  A learned system that breaks down or reaches
// the iteration cap is solved again from the start without the term (plain
// PCG as the fallback), after the other systems.
//
// The directions are stored in BF16 and the same BF16 vector enters the
// matvec and the update of x (step 3), so x and r stay consistent:
// r = b - C_q x up to the accuracy of the product (C kept as hi + lo BF16
// planes, about 16 significant bits; products exact, FP32 accumulation).
// Rounding p only perturbs the conjugacy of the directions, not the system
// that is solved.  Converged systems stop updating; a 256-system chunk whose
// systems have all stopped is skipped by the matvec.  The host reads the
// count of running systems after every iteration (one stream synchronization
// per iteration).
#include <cuda_bf16.h>
#include <math.h>

#include "common.cuh"
#include "info_esrf.h"
#include "internal.h"

namespace infoesrf {

namespace {

constexpr int kSys = 16;           // systems per CTA in the vector kernels
constexpr int kDotRows = kTileDotRows;   // rows per CTA (and per partial dot product)
constexpr int kVecThreads = 256;   // 16 row lanes per system, four rows per lane and step
// per-system FP64 scalars in sysd[j][8]
enum { kRho = 0, kAlpha = 1, kBeta = 2, kBn2 = 3, kRr = 4, kFirst = 5 };

__device__ __forceinline__ double sys_sigma(const ProblemDev& pr, int64_t j) {
  if (j < pr.mean_sys) return 1.0;
  const int64_t q = (j - pr.mean_sys) / pr.N;
  return pr.s[q] + 1.0;
}

// x = 0, r = b, p = 0 and the per-system state (mode 0), or (mode 1) the
// per-system state of the systems marked for a retry without the learned
// term, whose vectors k_tpcg_retry_vectors has reset.
__global__ void k_tpcg_init(const ProblemDev* dpr, int mode, int allow_learn) {
  const ProblemDev& pr = *dpr;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t J = pr.nsys;
  if (i < J && (mode == 0 || pr.learn_on[i] == 2)) {
    double* sd = pr.sysd + i * 8;
    sd[kRho] = 0.0;
    sd[kAlpha] = 0.0;
    sd[kBeta] = 0.0;
    sd[kBn2] = 0.0;
    sd[kRr] = 0.0;
    sd[kFirst] = 1.0;
    pr.sigmaf[i] = (float)sys_sigma(pr, i);
    pr.active[i] = 1;
    pr.iters[i] = 0;
    pr.relres[i] = 0.0;
    if (pr.learn_on) {
      int on = 0;
      if (mode == 0 && allow_learn && pr.learned_model && pr.lat_info[0] == 1) {
        const int64_t q = i < pr.mean_sys ? pr.Q : (i - pr.mean_sys) / pr.N;
        on = pr.learn_coef[q * kLearnOut] > 0.f ? 1 : 0;
        if (on) atomicAdd(&pr.lat_info[8], 1);
      }
      pr.learn_on[i] = on;
    }
  }
  if (mode != 0 || i >= J * pr.d_pad) return;
  const int64_t j = i / pr.d_pad, a = i % pr.d_pad;
  float b = 0.f;
  const int32_t src = a < pr.d ? pr.tpos_src[a] : -1;
  if (src >= 0) {
    if (j < pr.mean_sys) b = (float)pr.bmean[src];
    else b = pr.Wp[a * pr.N + (j - pr.mean_sys) % pr.N] * pr.rinvp[a];
  }
  pr.Xv[i] = 0.f;
  pr.Rv[i] = b;
  pr.Pdir[i] = __float2bfloat16_rn(0.f);
}

// x = 0, r = b, p = 0 for the systems marked for a retry (learn_on == 2).
__global__ void k_tpcg_retry_vectors(const ProblemDev* dpr) {
  const ProblemDev& pr = *dpr;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= pr.nsys * pr.d_pad) return;
  const int64_t j = i / pr.d_pad, a = i % pr.d_pad;
  if (pr.learn_on[j] != 2) return;
  float b = 0.f;
  const int32_t src = a < pr.d ? pr.tpos_src[a] : -1;
  if (src >= 0) {
    if (j < pr.mean_sys) b = (float)pr.bmean[src];
    else b = pr.Wp[a * pr.N + (j - pr.mean_sys) % pr.N] * pr.rinvp[a];
  }
  pr.Xv[i] = 0.f;
  pr.Rv[i] = b;
  pr.Pdir[i] = __float2bfloat16_rn(0.f);
}

// A learned system that failed: stop it and mark it for the retry.
__device__ __forceinline__ void mark_retry(const ProblemDev& pr, int64_t j) {
  pr.active[j] = 0;
  pr.learn_on[j] = 2;
  atomicAdd(&pr.lat_info[7], 1);
}

// alpha_j = rho_j / p_j^T y_j (one warp per system: lanes over the row-tile
// partials, a fixed shuffle tree); resets the unit flags and the running counts.
__global__ void k_tpcg_alpha(const ProblemDev* dpr, int it, int nunits, int reset_only) {
  const ProblemDev& pr = *dpr;
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gt < nunits) pr.unit_active[gt] = 0;
  if (gt == 0) {
    pr.nactive[0] = 0;
    pr.nactive[2] = 0;
  }
  const int lane = threadIdx.x & 31;
  const int64_t j = gt >> 5;
  if (j >= pr.nsys || reset_only) return;
  double* sd = pr.sysd + j * 8;
  if (!pr.active[j]) {
    if (lane == 0) sd[kAlpha] = 0.0;
    return;
  }
  double pap = 0.0;
  const float* src = pr.pty + j * pr.nrt;
  for (int64_t t = lane; t < pr.nrt; t += 32) pap += (double)src[t];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) pap += __shfl_xor_sync(0xffffffffu, pap, o);
  if (lane != 0) return;
  if (pap > 0.0 && isfinite(pap)) {
    sd[kAlpha] = sd[kRho] / pap;
    pr.iters[j] = it;
  } else {
    sd[kAlpha] = 0.0;
    if (pr.learn_on && pr.learn_on[j] == 1) {
      mark_retry(pr, j);
    } else {
      pr.active[j] = 0;
      atomicOr(&pr.status[0], kStatBreakdown);
    }
  }
}

// Step 3 (update = 1) or the dot products of r alone (update = 0): CTA =
// (block of kDotRows rows, group of kSys systems); Phi and C Phi of the rows
// are staged in shared memory once and reused by every system of the group.
// Systems: list[blockIdx.y * kSys + s] for positions below count (list = NULL:
// systems blockIdx.y * kSys + s).
__device__ __forceinline__ int64_t listed_system(const int32_t* list, int64_t count, int64_t pos, int64_t J) {
  if (pos >= count) return J;   // past the end: no system
  return list ? list[pos] : pos;
}

// Column stride (floats) of the staged [Phi | C Phi]: the block's rows plus
// 4, so that a column is read along the rows with 16-byte loads (four
// consecutive rows per thread, consecutive threads on consecutive rows: no
// bank conflict) and the transposing writes of the staging spread over the
// banks.
constexpr int kPhCol = kDotRows + 4;
__host__ __device__ __forceinline__ size_t phi_stage_bytes(int k) { return (size_t)2 * k * kPhCol * sizeof(float); }

// Stages rows abase .. abase + kDotRows - 1 of [Phi | C Phi] transposed into
// shared memory: pht[m * kPhCol + row] (m < k: Phi, k <= m < 2k: C Phi).
// Phi and C Phi are contiguous [d][k] blocks, so each is read with 16-byte
// loads that are all independent (a block of rows starts at a multiple of 4
// floats); rows at or past d are zero.
__device__ __forceinline__ void stage_phi(const ProblemDev& pr, int64_t abase, int k, float* pht) {
  const int64_t a1 = abase + kDotRows < pr.d ? abase + kDotRows : pr.d;
  const int nrows = a1 > abase ? (int)(a1 - abase) : 0;
  const int tot = nrows * k, ntail = kDotRows - nrows;
  for (int e = threadIdx.x; e < 2 * k * ntail; e += blockDim.x) {
    const int m = e / ntail, row = nrows + e % ntail;
    pht[m * kPhCol + row] = 0.f;
  }
#pragma unroll
  for (int which = 0; which < 2; ++which) {
    const float* src = reinterpret_cast<const float*>(which == 0 ? pr.Phi : pr.CPhi) + abase * k;
    const float4* src4 = reinterpret_cast<const float4*>(src);
    float* dst = pht + which * k * kPhCol;
#pragma unroll 4
    for (int q = threadIdx.x; q < tot / 4; q += blockDim.x) {
      const float4 v = src4[q];
      const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int e = 4 * q + i, row = e / k, m = e - row * k;
        dst[m * kPhCol + row] = vv[i];
      }
    }
    for (int e = (tot & ~3) + threadIdx.x; e < tot; e += blockDim.x) {
      const int row = e / k, m = e - row * k;
      dst[m * kPhCol + row] = src[e];
    }
  }
}

// CTA layout of steps 3 and 5: thread t serves system t / kRowLanes of the
// group and rows t % kRowLanes, t % kRowLanes + kRowLanes, ... of the block,
// so the kSys systems advance side by side and each thread runs a long loop
// of independent rows.
constexpr int kRowLanes = kVecThreads / kSys;   // 16

// Step 3 (update = 1) or the dot products of r alone (update = 0).
// NV32: 32-value chunks of the dot vector (r^T r, f, g): 1 for k <= 14 (the
// float4 loop then covers 28 columns of [Phi | C Phi]), else 2 (k <= 24).
template <int NV32>
__global__ void __launch_bounds__(kVecThreads) k_tpcg_update(const ProblemDev* dpr, int update,
                                                             const int32_t* list, int64_t count) {
  const ProblemDev& pr = *dpr;
  const int64_t sb = blockIdx.x;
  const int64_t g0 = (int64_t)blockIdx.y * kSys;
  const int k = pr.kR, NV = 2 * k + 1, NVD = tile_dot_values(k);
  const int64_t J = pr.nsys, dp = pr.d_pad;
  extern __shared__ float4 phs_dyn4[];   // [2 k][kPhCol / 4]
  float* phs = reinterpret_cast<float*>(phs_dyn4);
  __shared__ float part[kSys][2][32 * NV32];   // per system: the two half-lanes' reduce-scatter results
  __shared__ int64_t sys[kSys];
  __shared__ float als[kSys];
  if (threadIdx.x < kSys) {
    const int64_t j = listed_system(list, count, g0 + threadIdx.x, J);
    const bool run = j < J && pr.active[j];
    sys[threadIdx.x] = run ? j : -1;
    als[threadIdx.x] = run ? (float)pr.sysd[j * 8 + kAlpha] : 0.f;
  }
  __syncthreads();
  bool any = false;
  for (int s = 0; s < kSys; ++s) any |= sys[s] >= 0;
  if (!any) return;
  const int64_t abase = sb * kDotRows;
  stage_phi(pr, abase, k, phs);
  __syncthreads();
  const int s = threadIdx.x / kRowLanes, r0 = threadIdx.x % kRowLanes;
  const int64_t j = sys[s];
  float acc[32 * NV32];
#pragma unroll
  for (int v = 0; v < 32 * NV32; ++v) acc[v] = 0.f;
  if (j >= 0) {
    const float al = als[s];
    // four consecutive rows per step: 16-byte loads of r, y, x and 8 bytes of p
    // (d_pad and the row block are multiples of 4, so a group never straddles dp)
    for (int r4 = 4 * r0; r4 < kDotRows; r4 += 4 * kRowLanes) {
      const int64_t a = abase + r4;
      if (a >= dp) break;
      const int64_t e = j * dp + a;
      float4 rv = *reinterpret_cast<const float4*>(pr.Rv + e);
      if (update) {
        const uint2 pw = *reinterpret_cast<const uint2*>(pr.Pdir + e);
        const __nv_bfloat162* pp = reinterpret_cast<const __nv_bfloat162*>(&pw);
        const float2 p01 = __bfloat1622float2(pp[0]), p23 = __bfloat1622float2(pp[1]);
        float4 xv = *reinterpret_cast<const float4*>(pr.Xv + e);
        const float4 yv = *reinterpret_cast<const float4*>(pr.Yv + e);
        xv.x = fmaf(al, p01.x, xv.x);
        xv.y = fmaf(al, p01.y, xv.y);
        xv.z = fmaf(al, p23.x, xv.z);
        xv.w = fmaf(al, p23.y, xv.w);
        rv.x = fmaf(-al, yv.x, rv.x);
        rv.y = fmaf(-al, yv.y, rv.y);
        rv.z = fmaf(-al, yv.z, rv.z);
        rv.w = fmaf(-al, yv.w, rv.w);
        *reinterpret_cast<float4*>(pr.Xv + e) = xv;
        *reinterpret_cast<float4*>(pr.Rv + e) = rv;
      }
      acc[0] = fmaf(rv.x, rv.x, acc[0]);
      acc[0] = fmaf(rv.y, rv.y, acc[0]);
      acc[0] = fmaf(rv.z, rv.z, acc[0]);
      acc[0] = fmaf(rv.w, rv.w, acc[0]);
      // column m of [Phi | C Phi] at the four rows: one 16-byte load
      const float4* col4 = phs_dyn4 + r4 / 4;
#pragma unroll
      for (int m = 0; m < 32 * NV32 - 1; ++m) {
        if (m < 2 * k) {
          const float4 f = col4[m * (kPhCol / 4)];
          float t = acc[1 + m];
          t = fmaf(f.x, rv.x, t);
          t = fmaf(f.y, rv.y, t);
          t = fmaf(f.z, rv.z, t);
          acc[1 + m] = fmaf(f.w, rv.w, t);
        }
      }
    }
  }
  // reduce over the 16 row lanes of each system (a half-warp): a reduce-scatter
  // with offsets 8, 4, 2, 1 leaves lane l of the half with values 2 l and 2 l + 1
  // of each 32-value chunk (fixed order of additions)
  const int hl = r0;   // lane within the half-warp
#pragma unroll
  for (int c = 0; c < NV32; ++c) {
    float* v = acc + 32 * c;
#pragma unroll
    for (int off = 8, width = 16; off >= 1; off >>= 1, width >>= 1) {
      const bool up = (hl & off) != 0;
#pragma unroll
      for (int i = 0; i < width; ++i) {
        const float send = up ? v[i] : v[i + width];
        const float keep = up ? v[i + width] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
      }
    }
    // after the rounds lane hl holds the sums of values 2 hl', 2 hl' + 1 with hl' the
    // bit-reversal-free index: value index = 16 b3 + 8 b2 + 4 b1 + 2 b0 + i, i in {0, 1}
    const int vbase = 32 * c + 16 * ((hl >> 3) & 1) + 8 * ((hl >> 2) & 1) + 4 * ((hl >> 1) & 1) + 2 * (hl & 1);
    part[s][0][vbase] = v[0];
    part[s][0][vbase + 1] = v[1];
  }
  __syncthreads();
  const int64_t nsub = gridDim.x;
  for (int e = threadIdx.x; e < kSys * NV; e += blockDim.x) {
    const int ss = e / NV, v = e % NV;
    if (sys[ss] >= 0) pr.dots[(sys[ss] * NVD + v) * nsub + sb] = (double)part[ss][0][v];
  }
}

// Sums of the row-block partials: one CTA per listed system, one warp per
// value (r^T r, f, g), lanes over the row blocks (contiguous), then a fixed
// shuffle tree: the same order every call.
__global__ void __launch_bounds__(256) k_tpcg_reduce(const ProblemDev* dpr, int nsub, const int32_t* list,
                                                     int64_t count) {
  const ProblemDev& pr = *dpr;
  const int64_t j = listed_system(list, count, blockIdx.x, pr.nsys);
  if (j >= pr.nsys || !pr.active[j]) return;
  const int NV = tile_dot_values(pr.kR);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int v = warp; v < NV; v += blockDim.x >> 5) {
    const double* src = pr.dots + (j * NV + v) * (int64_t)nsub;
    double t = 0.0;
    for (int sb = lane; sb < nsub; sb += 32) t += src[sb];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) pr.dsum[j * NV + v] = t;
  }
}

// Step 4: one thread per system.
__global__ void k_tpcg_scalars(const ProblemDev* dpr, int nsub, int last) {
  const ProblemDev& pr = *dpr;
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j == 0) pr.nactive[1] = pr.status[0];   // timeouts and overflow are set by earlier kernels
  if (j >= pr.nsys || !pr.active[j]) return;
  const int k = pr.kR, NVD = tile_dot_values(k);
  const double* v = pr.dsum + j * NVD;   // r^T r, f = Phi^T r, g = (C Phi)^T r, u^T u
  (void)nsub;
  double* sd = pr.sysd + j * 8;
  const double rr = v[0];
  const bool first = sd[kFirst] != 0.0;
  if (first) sd[kBn2] = rr;
  sd[kRr] = rr;
  const double bn2 = sd[kBn2];
  pr.relres[j] = bn2 > 0.0 ? sqrt(rr / bn2) : 0.0;
  const bool lrn = pr.learn_on && pr.learn_on[j] == 1;
  bool act = true;
  if (pr.fixed_iters <= 0 && !(rr > pr.tol * pr.tol * bn2)) act = false;
  if (!isfinite(rr) && lrn) {
    mark_retry(pr, j);
    return;
  }
  if (!(rr > 0.0) || !isfinite(rr)) act = false;
  if (last && act) {
    // iteration cap reached with the system still running
    if (lrn && pr.fixed_iters <= 0) {
      mark_retry(pr, j);
      return;
    }
    if (pr.fixed_iters <= 0) atomicOr(&pr.status[0], kStatNotConverged);
    act = false;
  }
  if (!act) {
    pr.active[j] = 0;
    return;
  }
  const double sigma = sys_sigma(pr, j);
  const double beta_lmp = sigma + pr.scal[1];
  double rho = rr;
  float* lc = pr.lcoef + j * 2 * kMaxK;
  if (k > 0) {
    double t[kMaxK], t2[kMaxK];
    for (int m = 0; m < k; ++m) t[m] = v[1 + m] / (pr.theta[m] + sigma);
    double gt = 0.0, fc = 0.0;
    for (int m = 0; m < k; ++m) {
      double acc = v[1 + k + m] + sigma * v[1 + m];
      for (int i2 = 0; i2 < k; ++i2) {
        const int ge = m * k + i2, gtr = i2 * k + m;
        const double G = pr.gram[2 * k * k + ge] + sigma * (pr.gram[k * k + ge] + pr.gram[k * k + gtr]) +
                         sigma * sigma * pr.gram[ge];
        acc -= G * t[i2];
      }
      t2[m] = acc;
    }
    for (int m = 0; m < k; ++m) {
      const double c = (beta_lmp - sigma) * t[m] - t2[m] / (pr.theta[m] + sigma);
      gt += v[1 + k + m] * t[m];
      fc += v[1 + m] * c;
      lc[m] = (float)t[m];
      lc[kMaxK + m] = (float)c;
    }
    rho = rr - gt + fc;
  }
  if (lrn) {   // rho = r^T (a P^-1 + S S) r = a r^T P^-1 r + u^T u
    const int64_t q = j < pr.mean_sys ? pr.Q : (j - pr.mean_sys) / pr.N;
    rho = (double)pr.learn_coef[q * kLearnOut] * rho + v[2 * k + 1];
  }
  sd[kBeta] = first ? 0.0 : rho / sd[kRho];
  sd[kRho] = rho;
  sd[kFirst] = 0.0;
  if (atomicExch(&pr.unit_active[j / kTileUnit], 1) == 0) atomicAdd(&pr.nactive[2], 1);
  pr.alist[atomicAdd(&pr.nactive[0], 1)] = (int32_t)j;
}

// Step 5: p = bf16(r - (C Phi) t + Phi c + beta p) for the running systems;
// same CTA layout as step 3, the coefficients of all its systems staged once.
// learned != 0: the dynamic buffer also holds the block's stencil table, and
// a learned system takes z = a (r - (C Phi) t + Phi c) + S u.
__global__ void __launch_bounds__(kVecThreads) k_tpcg_direction(const ProblemDev* dpr, int learned) {
  const ProblemDev& pr = *dpr;
  const int64_t sb = blockIdx.x;
  const int64_t g0 = (int64_t)blockIdx.y * kSys;
  const int k = pr.kR;
  const int64_t J = pr.nsys, dp = pr.d_pad;
  const int64_t count = pr.nactive[0];   // the list the scalars kernel just built
  extern __shared__ float4 phs_dyn4[];   // [2 k][kPhCol / 4]
  float* phs = reinterpret_cast<float*>(phs_dyn4);
  __shared__ float4 tc4[kSys][2 * kMaxK / 4];   // per system: c (Phi coefficients), then -t (C Phi)
  __shared__ int64_t sys[kSys];
  __shared__ float bes[kSys];
  __shared__ int lon[kSys];
  __shared__ float las[kSys], ltap[kSys][kLatBins];
  if (threadIdx.x < kSys) {
    const int64_t j = listed_system(pr.alist, count, g0 + threadIdx.x, J);
    const bool run = j < J && pr.active[j];
    sys[threadIdx.x] = run ? j : -1;
    bes[threadIdx.x] = run ? (float)pr.sysd[j * 8 + kBeta] : 0.f;
    const bool on = learned && run && pr.learn_on[j] == 1;
    lon[threadIdx.x] = on ? 1 : 0;
    las[threadIdx.x] = 1.f;
    if (on) {
      const int64_t q = j < pr.mean_sys ? pr.Q : (j - pr.mean_sys) / pr.N;
      las[threadIdx.x] = pr.learn_coef[q * kLearnOut];
      for (int b = 0; b < kLatBins; ++b) ltap[threadIdx.x][b] = pr.learn_coef[q * kLearnOut + 1 + b];
    }
  }
  __syncthreads();
  bool any = false, anyl = false;
  for (int s = 0; s < kSys; ++s) {
    any |= sys[s] >= 0;
    anyl |= lon[s] != 0;
  }
  if (!any) return;
  const int64_t abase = sb * kDotRows;
  stage_phi(pr, abase, k, phs);
  int32_t* nbr_s = reinterpret_cast<int32_t*>(phs + 2 * k * kPhCol);   // [kDotRows][kLatPts]
  if (anyl) {
    const int64_t nrow = dp - abase < kDotRows ? dp - abase : kDotRows;
    for (int64_t e = threadIdx.x; e < nrow * kLatPts; e += blockDim.x) nbr_s[e] = pr.lat_nbr[abase * kLatPts + e];
  }
  float* tcf = reinterpret_cast<float*>(tc4);
  for (int e = threadIdx.x; e < kSys * 2 * kMaxK; e += blockDim.x) {
    const int s = e / (2 * kMaxK), m = e % (2 * kMaxK);
    float v = 0.f;
    if (sys[s] >= 0) {
      // aligned with the staged columns: Phi columns take c, C Phi columns take -t
      if (m < k) v = pr.lcoef[sys[s] * 2 * kMaxK + kMaxK + m];
      else if (m < 2 * k) v = -pr.lcoef[sys[s] * 2 * kMaxK + (m - k)];
    }
    tcf[e] = v;
  }
  __syncthreads();
  const int s = threadIdx.x / kRowLanes, r0 = threadIdx.x % kRowLanes;
  const int64_t j = sys[s];
  if (j < 0) return;
  const float be = bes[s];
  const bool sl = lon[s] != 0;
  const float la = las[s];
  float w[kLatPts];
#pragma unroll
  for (int n = 0; n < kLatPts; ++n) w[n] = sl ? ltap[s][lat_bin(n)] : 0.f;
  const float* u = pr.learn_u + j * dp;
  for (int r4 = 4 * r0; r4 < kDotRows; r4 += 4 * kRowLanes) {   // four rows per step
    const int64_t a = abase + r4;
    if (a >= dp) break;
    const int64_t e = j * dp + a;
    const float4 rv = *reinterpret_cast<const float4*>(pr.Rv + e);
    const uint2 pw = *reinterpret_cast<const uint2*>(pr.Pdir + e);
    const __nv_bfloat162* pp = reinterpret_cast<const __nv_bfloat162*>(&pw);
    const float2 p01 = __bfloat1622float2(pp[0]), p23 = __bfloat1622float2(pp[1]);
    float z[4] = {rv.x, rv.y, rv.z, rv.w};
    const float pv[4] = {p01.x, p01.y, p23.x, p23.y};
    // column m of [Phi | C Phi] at the four rows: one 16-byte load
    const float4* col4 = phs_dyn4 + r4 / 4;
#pragma unroll
    for (int q = 0; q < 2 * kMaxK / 4; ++q) {
      if (4 * q < 2 * k) {
        const float4 c4 = tc4[s][q];   // four coefficients (a broadcast load)
        const float cq[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if (4 * q + i >= 2 * k) break;   // only 2 k columns are staged
          const float4 f = col4[(4 * q + i) * (kPhCol / 4)];
          z[0] = fmaf(f.x, cq[i], z[0]);
          z[1] = fmaf(f.y, cq[i], z[1]);
          z[2] = fmaf(f.z, cq[i], z[2]);
          z[3] = fmaf(f.w, cq[i], z[3]);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (sl) {   // z = a P^-1 r + S u
        const int32_t* nb = nbr_s + (r4 + i) * kLatPts;
        float su = 0.f;
#pragma unroll
        for (int n = 0; n < kLatPts; ++n) su = fmaf(w[n], __ldg(u + nb[n]), su);
        z[i] = fmaf(la, z[i], su);
      }
      z[i] = (a + i < pr.d) ? fmaf(be, pv[i], z[i]) : 0.f;
    }
    __nv_bfloat162 out[2] = {__floats2bfloat162_rn(z[0], z[1]), __floats2bfloat162_rn(z[2], z[3])};
    *reinterpret_cast<uint2*>(pr.Pdir + e) = *reinterpret_cast<const uint2*>(out);
  }
}

}  // namespace

// Runs the PCG of one BF16 problem (host copy p, device copy dp) to
// convergence or the iteration cap.  Synchronizes the stream once per
// iteration to read the number of running systems.  cap != NULL: records the
// Krylov samples of its systems at iterations 1..cap->K and stops after K
// iterations, without the learned term.
static int tile_pcg_loop(const ProblemDev& p, const ProblemDev* dp, cudaStream_t st, double* mm_ms, int* mm_count,
                         const TileCapture* cap) {
  const int64_t J = p.nsys;
  if (J < 1) return 0;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  if (mm_ms && (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess)) {
    cudaGetLastError();
    if (ev[0]) cudaEventDestroy(ev[0]);
    return INFO_ESRF_ERR_CUDA;
  }
  bool timed = false;   // an event pair of the previous iteration awaits reading
  auto read_time = [&]() {
    if (!timed) return;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ev[0], ev[1]) == cudaSuccess) {
      *mm_ms += ms;
      ++*mm_count;
    }
    timed = false;
  };
  struct Destroy {
    cudaEvent_t* e;
    ~Destroy() {
      if (e[0]) cudaEventDestroy(e[0]);
      if (e[1]) cudaEventDestroy(e[1]);
    }
  } destroy{ev};
  const int nunits = (int)((J + kTileUnit - 1) / kTileUnit);
  const int nsub = (int)((p.d_pad + kDotRows - 1) / kDotRows);
  const dim3 gsys((unsigned)((J + 127) / 128));
  const dim3 gall((unsigned)((J * p.d_pad + 255) / 256));
  const dim3 gvec((unsigned)nsub, (unsigned)((J + kSys - 1) / kSys));
  TileMmArgs ta{};
  ta.rowptr = p.rowptr;
  ta.colblk = p.colblk;
  ta.P = p.Pdir;
  ta.sigma = p.sigmaf;
  ta.active = p.unit_active;
  ta.ulist = p.unit_list;
  ta.Y = p.Yv;
  ta.pty = p.pty;
  ta.status = p.status;
  ta.d_pad = p.d_pad;
  ta.J = (int32_t)J;
  ta.nrt = p.nrt;
  ta.pty_by_system = 1;
  int maxit = p.fixed_iters > 0 ? p.fixed_iters : p.max_iter;
  if (cap) maxit = cap->K;
  // the learned term is possible when the problem has a model and its tables
  bool learned = !cap && p.learned_model && p.learn_on && p.lat_info;
  const size_t vsm = phi_stage_bytes(p.kR);
  size_t dsm = vsm;   // + the stencil table while learned systems run (set below)
  const bool wide = 2 * p.kR > 28;   // k > 14: 64-value dot vectors (the 32-value loop covers 28 columns)
  static thread_local int raised = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (raised != dev) {
    const int mx = (int)phi_stage_bytes(kMaxK);
    const int mxd = mx + kDotRows * kLatPts * (int)sizeof(int32_t);
    if (cudaFuncSetAttribute(k_tpcg_update<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx) != cudaSuccess ||
        cudaFuncSetAttribute(k_tpcg_update<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx) != cudaSuccess ||
        cudaFuncSetAttribute(k_tpcg_direction, cudaFuncAttributeMaxDynamicSharedMemorySize, mxd) != cudaSuccess)
      return INFO_ESRF_ERR_CUDA;
    raised = dev;
  }
  int32_t host[3] = {0, 0, 0};   // running systems, status bits, active units
  auto update = [&](dim3 grid, int upd, const int32_t* list, int64_t count) {
    if (wide) k_tpcg_update<2><<<grid, kVecThreads, vsm, st>>>(dp, upd, list, count);
    else k_tpcg_update<1><<<grid, kVecThreads, vsm, st>>>(dp, upd, list, count);
  };
  const dim3 galpha((unsigned)(((32 * J > nunits ? 32 * J : nunits) + 255) / 256));
  // the first direction of every running system: r = b, z = M r, p = z
  auto start = [&]() {
    update(gvec, 0, nullptr, J);
    if (learned) launch_tile_learn_u(p, dp, nullptr, J, nsub, st);
    k_tpcg_reduce<<<(unsigned)J, 256, 0, st>>>(dp, nsub, nullptr, J);
    k_tpcg_alpha<<<galpha, 256, 0, st>>>(dp, 0, nunits, 1);   // resets the unit flags and the counts
    k_tpcg_scalars<<<gsys, 128, 0, st>>>(dp, nsub, maxit <= 0 ? 1 : 0);
    k_tpcg_direction<<<gvec, kVecThreads, dsm, st>>>(dp, learned ? 1 : 0);
    note_launches(5);
  };
  auto iterate = [&]() -> int {
    for (int it = 1; it <= maxit; ++it) {
      // running systems (and the status word) after the previous iteration
      if (cudaMemcpyAsync(host, p.nactive, sizeof(host), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        return INFO_ESRF_ERR_CUDA;
      read_time();   // the previous launch has completed (stream synchronized)
      if (host[0] == 0) break;
      if (host[1] & (kStatTimeout | kStatTileOverflow)) break;
      const int64_t nrun = host[0];
      ta.units = host[2];
      const dim3 glist((unsigned)nsub, (unsigned)((nrun + kSys - 1) / kSys));
      if (mm_ms) cudaEventRecord(ev[0], st);
      if (launch_tile_mm(ta, p.Chi, p.Clo, p.tile_cap, st) != 0) return INFO_ESRF_ERR_CUDA;
      if (mm_ms) {
        cudaEventRecord(ev[1], st);
        timed = true;
      }
      if (cap) launch_tile_capture_record(p, dp, *cap, it, st);
      k_tpcg_alpha<<<galpha, 256, 0, st>>>(dp, it, nunits, 0);
      update(glist, 1, p.alist, nrun);
      if (learned) launch_tile_learn_u(p, dp, p.alist, nrun, nsub, st);
      k_tpcg_reduce<<<(unsigned)nrun, 256, 0, st>>>(dp, nsub, p.alist, nrun);
      k_tpcg_scalars<<<gsys, 128, 0, st>>>(dp, nsub, it == maxit ? 1 : 0);
      k_tpcg_direction<<<glist, kVecThreads, dsm, st>>>(dp, learned ? 1 : 0);
      note_launches(5);
    }
    return 0;
  };
  k_tpcg_init<<<gall, 256, 0, st>>>(dp, 0, learned ? 1 : 0);
  note_launches(1);
  if (learned) {   // systems that use the term (none: the plain loop)
    int32_t nl = 0;
    if (cudaMemcpyAsync(&nl, p.lat_info + 8, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return INFO_ESRF_ERR_CUDA;
    learned = nl > 0;
  }
  if (learned) dsm = vsm + (size_t)kDotRows * kLatPts * sizeof(int32_t);
  start();
  int rc = iterate();
  if (rc) return rc;
  if (learned) {
    // plain PCG for the learned systems that broke down or hit the cap
    int32_t retries = 0;
    if (cudaMemcpyAsync(&retries, p.lat_info + 7, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return INFO_ESRF_ERR_CUDA;
    read_time();
    if (retries > 0) {
      k_tpcg_retry_vectors<<<gall, 256, 0, st>>>(dp);
      k_tpcg_init<<<gsys, 128, 0, st>>>(dp, 1, 0);
      note_launches(2);
      start();
      rc = iterate();
      if (rc) return rc;
    }
  }
  if (timed) {
    if (cudaEventSynchronize(ev[1]) != cudaSuccess) return INFO_ESRF_ERR_CUDA;
    read_time();
  }
  return cudaGetLastError() == cudaSuccess ? 0 : INFO_ESRF_ERR_CUDA;
}

int run_tile_pcg(const ProblemDev& p, const ProblemDev* dp, cudaStream_t st, double* mm_ms, int* mm_count) {
  return tile_pcg_loop(p, dp, st, mm_ms, mm_count, nullptr);
}

int run_tile_pcg_capture(const ProblemDev& p, const ProblemDev* dp, const TileCapture& cap, float* Z, float* feat,
                         cudaStream_t st) {
  const int rc = tile_pcg_loop(p, dp, st, nullptr, nullptr, &cap);
  if (rc) return rc;
  launch_tile_capture_finish(p, dp, cap, Z, feat, st);
  return cudaGetLastError() == cudaSuccess ? 0 : INFO_ESRF_ERR_CUDA;
}

}  // namespace infoesrf
