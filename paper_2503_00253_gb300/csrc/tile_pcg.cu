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

constexpr int kSys = 8;            // systems per CTA in the vector kernels
constexpr int kDotRows = kTileDotRows;   // rows per CTA (and per partial dot product)
constexpr int kVecThreads = 256;   // two rows per thread
// per-system FP64 scalars in sysd[j][8]
enum { kRho = 0, kAlpha = 1, kBeta = 2, kBn2 = 3, kRr = 4, kFirst = 5 };

__device__ __forceinline__ double sys_sigma(const ProblemDev& pr, int64_t j) {
  if (j < pr.mean_sys) return 1.0;
  const int64_t q = (j - pr.mean_sys) / pr.N;
  return pr.s[q] + 1.0;
}

// x = 0, r = b, p = 0 and the per-system state.
__global__ void k_tpcg_init(const ProblemDev* dpr) {
  const ProblemDev& pr = *dpr;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t J = pr.nsys;
  if (i < J) {
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
  }
  if (i >= J * pr.d_pad) return;
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

// alpha_j = rho_j / p_j^T y_j; resets the chunk flags and the running count.
__global__ void k_tpcg_alpha(const ProblemDev* dpr, int it, int nchunks, int reset_only) {
  const ProblemDev& pr = *dpr;
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < nchunks) pr.chunk_active[j] = 0;
  if (j == 0) pr.nactive[0] = 0;
  if (j >= pr.nsys || reset_only) return;
  double* sd = pr.sysd + j * 8;
  if (!pr.active[j]) {
    sd[kAlpha] = 0.0;
    return;
  }
  double pap = 0.0;
  for (int64_t t = 0; t < pr.nrt; ++t) pap += (double)pr.pty[t * pr.nsys + j];
  if (pap > 0.0 && isfinite(pap)) {
    sd[kAlpha] = sd[kRho] / pap;
    pr.iters[j] = it;
  } else {
    sd[kAlpha] = 0.0;
    pr.active[j] = 0;
    atomicOr(&pr.status[0], kStatBreakdown);
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

__global__ void __launch_bounds__(kVecThreads) k_tpcg_update(const ProblemDev* dpr, int update,
                                                             const int32_t* list, int64_t count) {
  const ProblemDev& pr = *dpr;
  const int64_t sb = blockIdx.x;
  const int64_t g0 = (int64_t)blockIdx.y * kSys;
  const int k = pr.kR, NV = 2 * k + 1;
  const int64_t J = pr.nsys, dp = pr.d_pad;
  extern __shared__ float phs_dyn[];   // [kDotRows][2 k + 1]
  __shared__ float wred[kVecThreads / 32][2 * kMaxK + 1];
  bool any = false;
  for (int s = 0; s < kSys; ++s) {
    const int64_t j = listed_system(list, count, g0 + s, J);
    any |= j < J && pr.active[j];
  }
  if (!any) return;
  const float* Phi = reinterpret_cast<const float*>(pr.Phi);
  const float* CPhi = reinterpret_cast<const float*>(pr.CPhi);
  const int64_t abase = sb * kDotRows;
  for (int e = threadIdx.x; e < kDotRows * 2 * k; e += blockDim.x) {
    const int row = e / (2 * k), m = e % (2 * k);
    const int64_t a = abase + row;
    float v = 0.f;
    if (a < pr.d) v = m < k ? Phi[a * k + m] : CPhi[a * k + (m - k)];
    phs_dyn[row * (2 * k + 1) + m] = v;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int s = 0; s < kSys; ++s) {
    const int64_t j = listed_system(list, count, g0 + s, J);
    if (j >= J || !pr.active[j]) continue;   // uniform across the CTA
    const float al = (float)pr.sysd[j * 8 + kAlpha];
    float acc[2 * kMaxK + 1];
#pragma unroll
    for (int v = 0; v < 2 * kMaxK + 1; ++v) acc[v] = 0.f;
    for (int rr = threadIdx.x; rr < kDotRows; rr += blockDim.x) {
      const int64_t a = abase + rr;
      if (a >= dp) break;
      const int64_t e = j * dp + a;
      float r = pr.Rv[e];
      if (update) {
        const float p = __bfloat162float(pr.Pdir[e]);
        pr.Xv[e] = fmaf(al, p, pr.Xv[e]);
        r = fmaf(-al, pr.Yv[e], r);
        pr.Rv[e] = r;
      }
      acc[0] = fmaf(r, r, acc[0]);
#pragma unroll
      for (int m = 0; m < 2 * kMaxK; ++m)
        if (m < 2 * k) acc[1 + m] = fmaf(phs_dyn[rr * (2 * k + 1) + m], r, acc[1 + m]);
    }
#pragma unroll
    for (int v = 0; v < 2 * kMaxK + 1; ++v) {
      if (v >= NV) break;
      float x = acc[v];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) wred[warp][v] = x;
    }
    __syncthreads();
    for (int v = threadIdx.x; v < NV; v += blockDim.x) {
      double t = 0.0;
      for (int w = 0; w < kVecThreads / 32; ++w) t += (double)wred[w][v];
      pr.dots[(sb * J + j) * NV + v] = t;
    }
    __syncthreads();
  }
}

// Step 4: one thread per system.
__global__ void k_tpcg_scalars(const ProblemDev* dpr, int nsub, int bn, int last) {
  const ProblemDev& pr = *dpr;
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j == 0) pr.nactive[1] = pr.status[0];   // timeouts and overflow are set by earlier kernels
  if (j >= pr.nsys || !pr.active[j]) return;
  const int k = pr.kR, NV = 2 * k + 1;
  double v[2 * kMaxK + 1];
  for (int e = 0; e < NV; ++e) v[e] = 0.0;
  for (int s = 0; s < nsub; ++s)
    for (int e = 0; e < NV; ++e) v[e] += pr.dots[((int64_t)s * pr.nsys + j) * NV + e];
  double* sd = pr.sysd + j * 8;
  const double rr = v[0];
  const bool first = sd[kFirst] != 0.0;
  if (first) sd[kBn2] = rr;
  sd[kRr] = rr;
  const double bn2 = sd[kBn2];
  pr.relres[j] = bn2 > 0.0 ? sqrt(rr / bn2) : 0.0;
  bool act = true;
  if (pr.fixed_iters <= 0 && !(rr > pr.tol * pr.tol * bn2)) act = false;
  if (!(rr > 0.0) || !isfinite(rr)) act = false;
  if (last && act) {
    // iteration cap reached with the system still running
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
  sd[kBeta] = first ? 0.0 : rho / sd[kRho];
  sd[kRho] = rho;
  sd[kFirst] = 0.0;
  pr.chunk_active[j / bn] = 1;
  pr.alist[atomicAdd(&pr.nactive[0], 1)] = (int32_t)j;
}

// Step 5: p = bf16(r - (C Phi) t + Phi c + beta p) for the running systems;
// same CTA shape as step 3.
__global__ void __launch_bounds__(kVecThreads) k_tpcg_direction(const ProblemDev* dpr) {
  const ProblemDev& pr = *dpr;
  const int64_t sb = blockIdx.x;
  const int64_t g0 = (int64_t)blockIdx.y * kSys;
  const int k = pr.kR;
  const int64_t J = pr.nsys, dp = pr.d_pad;
  const int64_t count = pr.nactive[0];   // the list the scalars kernel just built
  extern __shared__ float phs_dyn[];   // [kDotRows][2 k + 1]
  __shared__ float tc[2 * kMaxK];
  bool any = false;
  for (int s = 0; s < kSys; ++s) {
    const int64_t j = listed_system(pr.alist, count, g0 + s, J);
    any |= j < J && pr.active[j];
  }
  if (!any) return;
  const float* Phi = reinterpret_cast<const float*>(pr.Phi);
  const float* CPhi = reinterpret_cast<const float*>(pr.CPhi);
  const int64_t abase = sb * kDotRows;
  for (int e = threadIdx.x; e < kDotRows * 2 * k; e += blockDim.x) {
    const int row = e / (2 * k), m = e % (2 * k);
    const int64_t a = abase + row;
    float v = 0.f;
    if (a < pr.d) v = m < k ? Phi[a * k + m] : CPhi[a * k + (m - k)];
    phs_dyn[row * (2 * k + 1) + m] = v;
  }
  for (int s = 0; s < kSys; ++s) {
    const int64_t j = listed_system(pr.alist, count, g0 + s, J);
    if (j >= J || !pr.active[j]) continue;   // uniform across the CTA
    __syncthreads();
    for (int m = threadIdx.x; m < 2 * k; m += blockDim.x)
      tc[m] = pr.lcoef[j * 2 * kMaxK + (m < k ? m : kMaxK + (m - k))];   // t then c
    __syncthreads();
    const float be = (float)pr.sysd[j * 8 + kBeta];
    for (int rr = threadIdx.x; rr < kDotRows; rr += blockDim.x) {
      const int64_t a = abase + rr;
      if (a >= dp) break;
      const int64_t e = j * dp + a;
      float z = pr.Rv[e];
#pragma unroll
      for (int m = 0; m < kMaxK; ++m)
        if (m < k) z += phs_dyn[rr * (2 * k + 1) + m] * tc[k + m] - phs_dyn[rr * (2 * k + 1) + k + m] * tc[m];
      const float p = __bfloat162float(pr.Pdir[e]);
      pr.Pdir[e] = __float2bfloat16_rn(a < pr.d ? fmaf(be, p, z) : 0.f);
    }
  }
}

}  // namespace

// Runs the PCG of one BF16 problem (host copy p, device copy dp) to
// convergence or the iteration cap.  Synchronizes the stream once per
// iteration to read the number of running systems.
int run_tile_pcg(const ProblemDev& p, const ProblemDev* dp, cudaStream_t st, double* mm_ms, int* mm_count) {
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
  const int bn = tile_chunk_width((int32_t)J);
  const int nchunks = (int)((J + bn - 1) / bn);
  const int nsub = (int)((p.d_pad + kDotRows - 1) / kDotRows);
  const dim3 gsys((unsigned)((J + 127) / 128));
  const dim3 gall((unsigned)((J * p.d_pad + 255) / 256));
  const dim3 gvec((unsigned)nsub, (unsigned)((J + kSys - 1) / kSys));
  TileMmArgs ta{};
  ta.rowptr = p.rowptr;
  ta.colblk = p.colblk;
  ta.P = p.Pdir;
  ta.sigma = p.sigmaf;
  ta.active = p.chunk_active;
  ta.Y = p.Yv;
  ta.pty = p.pty;
  ta.status = p.status;
  ta.d_pad = p.d_pad;
  ta.J = (int32_t)J;
  ta.nrt = p.nrt;
  const int maxit = p.fixed_iters > 0 ? p.fixed_iters : p.max_iter;
  const size_t vsm = (size_t)kDotRows * (2 * p.kR + 1) * sizeof(float);
  static thread_local int raised = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (raised != dev) {
    const int mx = (int)((size_t)kDotRows * (2 * kMaxK + 1) * sizeof(float));
    if (cudaFuncSetAttribute(k_tpcg_update, cudaFuncAttributeMaxDynamicSharedMemorySize, mx) != cudaSuccess ||
        cudaFuncSetAttribute(k_tpcg_direction, cudaFuncAttributeMaxDynamicSharedMemorySize, mx) != cudaSuccess)
      return INFO_ESRF_ERR_CUDA;
    raised = dev;
  }
  int32_t host[2] = {0, 0};
  k_tpcg_init<<<gall, 256, 0, st>>>(dp);
  k_tpcg_update<<<gvec, kVecThreads, vsm, st>>>(dp, 0, nullptr, J);
  const dim3 galpha((unsigned)(((J > nchunks ? J : nchunks) + 127) / 128));
  k_tpcg_alpha<<<galpha, 128, 0, st>>>(dp, 0, nchunks, 1);   // resets the chunk flags and the count
  k_tpcg_scalars<<<gsys, 128, 0, st>>>(dp, nsub, bn, maxit <= 0 ? 1 : 0);
  k_tpcg_direction<<<gvec, kVecThreads, vsm, st>>>(dp);
  note_launches(5);
  for (int it = 1; it <= maxit; ++it) {
    // running systems (and the status word) after the previous iteration
    if (cudaMemcpyAsync(host, p.nactive, sizeof(host), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return INFO_ESRF_ERR_CUDA;
    read_time();   // the previous launch has completed (stream synchronized)
    if (host[0] == 0) break;
    if (host[1] & (kStatTimeout | kStatTileOverflow)) break;
    const int64_t nrun = host[0];
    const dim3 glist((unsigned)nsub, (unsigned)((nrun + kSys - 1) / kSys));
    if (mm_ms) cudaEventRecord(ev[0], st);
    if (launch_tile_mm(ta, p.Chi, p.Clo, p.tile_cap, st) != 0) return INFO_ESRF_ERR_CUDA;
    if (mm_ms) {
      cudaEventRecord(ev[1], st);
      timed = true;
    }
    k_tpcg_alpha<<<galpha, 128, 0, st>>>(dp, it, nchunks, 0);
    k_tpcg_update<<<glist, kVecThreads, vsm, st>>>(dp, 1, p.alist, nrun);
    k_tpcg_scalars<<<gsys, 128, 0, st>>>(dp, nsub, bn, it == maxit ? 1 : 0);
    k_tpcg_direction<<<glist, kVecThreads, vsm, st>>>(dp);
    note_launches(4);
  }
  if (timed) {
    if (cudaEventSynchronize(ev[1]) != cudaSuccess) return INFO_ESRF_ERR_CUDA;
    read_time();
  }
  return cudaGetLastError() == cudaSuccess ? 0 : INFO_ESRF_ERR_CUDA;
}

}  // namespace infoesrf
