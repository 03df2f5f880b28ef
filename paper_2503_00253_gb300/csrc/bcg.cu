// Block CG across members (Sec. 3.3, second alternative; O'Leary 1980) for
// the normalized shifted systems of App. E, Eq. normalized_linear_solve:
// for every node q the N members' systems ((s_q + 1) I + C) U_q = R^-1/2 W
// form one block of N columns sharing the block Krylov space
// span{B, C_q B, ..., C_q^(k-1) B}; the mean system is a block of one column
// (plain CG).  With X_0 = 0, R_0 = P_0 = B and Q = C_q P:
//
//     alpha = (P^T Q)^-1 (R^T R),  X += P alpha,  R' = R - Q alpha,
//     beta = (R^T R)^-1 (R'^T R'),  P = R' + P beta.
//
// A block stops when every column has ||r_i|| <= tol ||b_i|| (or after
// fixed_iters iterations).  The members' right-hand sides sum to zero, so a
// node's block runs on N - 1 columns and the last member's solution is minus
// the sum of the others (the same block Krylov space, so the same iterates in
// exact arithmetic); pivots of the s x s Gram matrices at rounding level are
// taken as zero (semidefinite Cholesky), which deflates converged columns.  Kernels per iteration, over all running blocks at once:
// the banded product Q = sigma P + C P (the ELL band of C from set-up), the
// Gram matrices P^T Q and R^T R (FP64 sums in a fixed order), one CTA per
// block for the s x s Cholesky solves (FP64), and the block updates of X, R
// and P.  The host reads the number of running blocks after each iteration.
// Vectors are system-major [nsys][d] (X is the solution array U of the
// finish), in the bulk precision T.
#include <math.h>

#include "common.cuh"
#include "info_esrf.h"
#include "internal.h"

namespace infoesrf {

namespace {

struct BlockInfo {
  int64_t sid0;   // first system
  int s;          // columns
  double sigma;
};

__device__ __forceinline__ BlockInfo block_info(const ProblemDev& pr, int b) {
  BlockInfo bi;
  if (b < pr.mean_sys) {
    bi.sid0 = 0;
    bi.s = 1;
    bi.sigma = 1.0;
  } else {
    // the members' right-hand sides sum to zero (anomalies of the ensemble
    // mean), so the last member's system is minus the sum of the others and
    // shares their block Krylov space: the block iterates over N - 1 columns
    // and k_bcg_complete fills in the last
    const int q = b - pr.mean_sys;
    bi.sid0 = pr.mean_sys + (int64_t)q * pr.N;
    bi.s = (int)pr.N - 1;
    bi.sigma = pr.s[q] + 1.0;
  }
  return bi;
}

// The last member of every perturbation block: x_N = -(x_1 + ... + x_(N-1)),
// with the block's iteration count and the largest relative residual.
template <typename T>
__global__ void k_bcg_complete(const ProblemDev* dp) {
  const ProblemDev& pr = *dp;
  const int b = pr.mean_sys + blockIdx.y;
  if (b >= pr.bcg_nblocks) return;
  const BlockInfo bi = block_info(pr, b);
  const int64_t d = pr.d, last = bi.sid0 + bi.s;
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  T* X = reinterpret_cast<T*>(pr.U);
  if (a < d) {
    double acc = 0.0;
    for (int i = 0; i < bi.s; ++i) acc += (double)X[(bi.sid0 + i) * d + a];
    X[last * d + a] = to_t<T>(-acc);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double rmax = 0.0;
    for (int i = 0; i < bi.s; ++i) rmax = fmax(rmax, pr.relres[bi.sid0 + i]);
    pr.relres[last] = rmax;
    pr.iters[last] = bi.s > 0 ? pr.iters[bi.sid0] : 0;
  }
}

// X = 0, R = P = b for every system.
template <typename T>
__global__ void k_bcg_init(const ProblemDev* dp) {
  const ProblemDev& pr = *dp;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)pr.nsys * pr.d) return;
  const int64_t sid = i / pr.d, a = i % pr.d;
  T b;
  if (sid < pr.mean_sys) b = to_t<T>(pr.bmean[a]);
  else b = reinterpret_cast<const T*>(pr.W)[a * pr.N + (sid - pr.mean_sys) % pr.N] * to_t<T>(pr.rinv[a]);
  reinterpret_cast<T*>(pr.U)[i] = T(0);
  reinterpret_cast<T*>(pr.bcg_R)[i] = b;
  reinterpret_cast<T*>(pr.bcg_P)[i] = b;
}

// Q = sigma P + C P for the systems of running blocks (thread per row, CTA row per system).
template <typename T>
__global__ void k_bcg_matvec(const ProblemDev* dp) {
  const ProblemDev& pr = *dp;
  const int64_t sid = blockIdx.y;
  const int b = sid < pr.mean_sys ? 0 : pr.mean_sys + (int)((sid - pr.mean_sys) / pr.N);
  if (pr.bcg_state[b] != 0) return;
  if (sid >= pr.mean_sys && (sid - pr.mean_sys) % pr.N == pr.N - 1) return;   // completed at the end
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= pr.d) return;
  const int64_t d = pr.d;
  const T* P = reinterpret_cast<const T*>(pr.bcg_P) + sid * d;
  const T* val = reinterpret_cast<const T*>(pr.oo_val);
  const double sigma = block_info(pr, b).sigma;
  T acc = to_t<T>(sigma) * P[a];
  const int nnz = pr.oo_nnz[a];
  for (int e = 0; e < nnz; ++e) acc += val[(int64_t)e * d + a] * P[pr.oo_col[(int64_t)e * d + a]];
  reinterpret_cast<T*>(pr.bcg_Q)[sid * d + a] = acc;
}

// Row i of a Gram matrix of block b: which = 0: G1 = P^T Q; 1: G2 = R^T R.
// Threads over the rows, one FP64 accumulator per column j; the per-thread
// sums are combined in shared memory in thread order.
constexpr int kGramThreads = 128;
template <typename T>
__global__ void __launch_bounds__(kGramThreads) k_bcg_gram(const ProblemDev* dp, int which) {
  const ProblemDev& pr = *dp;
  const int b = blockIdx.y, i = blockIdx.x;
  if (b >= pr.bcg_nblocks || pr.bcg_state[b] != 0) return;
  const BlockInfo bi = block_info(pr, b);
  if (i >= bi.s) return;
  extern __shared__ double gsm[];   // [kGramThreads][s]
  const int64_t d = pr.d;
  const T* L = reinterpret_cast<const T*>(which == 0 ? pr.bcg_P : pr.bcg_R) + (bi.sid0 + i) * d;
  const T* Rm = reinterpret_cast<const T*>(which == 0 ? pr.bcg_Q : pr.bcg_R) + bi.sid0 * d;
  double acc[kBcgMaxS];
#pragma unroll
  for (int j = 0; j < kBcgMaxS; ++j) acc[j] = 0.0;
  for (int64_t a = threadIdx.x; a < d; a += blockDim.x) {
    const double l = (double)L[a];
#pragma unroll
    for (int j = 0; j < kBcgMaxS; ++j)
      if (j < bi.s) acc[j] = fma(l, (double)Rm[j * d + a], acc[j]);
  }
#pragma unroll
  for (int j = 0; j < kBcgMaxS; ++j)
    if (j < bi.s) gsm[threadIdx.x * bi.s + j] = acc[j];
  __syncthreads();
  double* G = (which == 0 ? pr.bcg_G1 : pr.bcg_G2) + (int64_t)b * kBcgMaxS * kBcgMaxS;
  for (int j = threadIdx.x; j < bi.s; j += blockDim.x) {
    double t = 0.0;
    for (int r = 0; r < kGramThreads; ++r) t += gsm[r * bi.s + j];
    G[i * kBcgMaxS + j] = t;
  }
}

// In-place Cholesky A = L L^T of an s x s symmetric positive semidefinite
// matrix (row stride kBcgMaxS) in shared memory by the whole CTA.  The
// members' anomalies sum to zero, so a block's residual and direction Gram
// matrices are singular in exact arithmetic (rank N - 1), and columns that
// have converged make them nearly so.  A pivot at or below eps times the
// largest diagonal entry is therefore taken as zero: its column of L is
// zeroed and null[k] set, and the solve gives that unknown the value 0 (the
// minimum-norm choice in the determined subspace; the oracle's dense LU solve
// differs from it only by rounding).  False (for every thread) on a
// non-finite pivot.
__device__ bool chol_smem(double* A, int s, double eps, int* null_col, int* fail) {
  __shared__ double maxd;
  if (threadIdx.x == 0) {
    *fail = 0;
    double m = 0.0;
    for (int k = 0; k < s; ++k) m = fmax(m, A[k * kBcgMaxS + k]);
    maxd = m;
  }
  __syncthreads();
  for (int k = 0; k < s; ++k) {
    if (threadIdx.x == 0) {
      const double piv = A[k * kBcgMaxS + k];
      null_col[k] = 0;
      if (!isfinite(piv)) {
        *fail = 1;
      } else if (!(piv > eps * maxd)) {
        null_col[k] = 1;
        A[k * kBcgMaxS + k] = 1.0;
      } else {
        A[k * kBcgMaxS + k] = sqrt(piv);
      }
    }
    __syncthreads();
    if (*fail) return false;
    if (null_col[k]) {
      for (int i = k + 1 + threadIdx.x; i < s; i += blockDim.x) A[i * kBcgMaxS + k] = 0.0;
      __syncthreads();
      continue;
    }
    const double lkk = A[k * kBcgMaxS + k];
    for (int i = k + 1 + threadIdx.x; i < s; i += blockDim.x) A[i * kBcgMaxS + k] /= lkk;
    __syncthreads();
    for (int e = threadIdx.x; e < (s - k - 1) * (s - k - 1); e += blockDim.x) {
      const int i = k + 1 + e / (s - k - 1), j = k + 1 + e % (s - k - 1);
      if (j <= i) A[i * kBcgMaxS + j] -= A[i * kBcgMaxS + k] * A[j * kBcgMaxS + k];
    }
    __syncthreads();
  }
  return true;
}

// X = A^+ B for the factor L of A from chol_smem (null columns give 0), B
// and X s x s (row stride kBcgMaxS): one thread per column of B, forward then
// backward substitution.
__device__ void chol_solve_smem(const double* Lf, const int* null_col, const double* B, double* X, int s) {
  for (int c = threadIdx.x; c < s; c += blockDim.x) {
    for (int i = 0; i < s; ++i) {
      double t = B[i * kBcgMaxS + c];
      for (int k = 0; k < i; ++k) t -= Lf[i * kBcgMaxS + k] * X[k * kBcgMaxS + c];
      X[i * kBcgMaxS + c] = null_col[i] ? 0.0 : t / Lf[i * kBcgMaxS + i];
    }
    for (int i = s - 1; i >= 0; --i) {
      double t = X[i * kBcgMaxS + c];
      for (int k = i + 1; k < s; ++k) t -= Lf[k * kBcgMaxS + i] * X[k * kBcgMaxS + c];
      X[i * kBcgMaxS + c] = null_col[i] ? 0.0 : t / Lf[i * kBcgMaxS + i];
    }
  }
}

// One CTA per block.  phase 0: alpha = G1^-1 RR.  phase 1 (after R^T R of the
// new residual in G2; first = the initial residual): record ||b_i||^2 on the
// first call, test convergence, beta = RR^-1 G2, RR = G2, count running blocks.
__global__ void __launch_bounds__(128) k_bcg_solve(const ProblemDev* dp, int phase, int it, int last) {
  const ProblemDev& pr = *dp;
  const int b = blockIdx.x;
  if (b >= pr.bcg_nblocks || pr.bcg_state[b] != 0) return;
  const BlockInfo bi = block_info(pr, b);
  const int s = bi.s;
  extern __shared__ double ssm[];
  double* A = ssm;                              // factor
  double* Bm = A + kBcgMaxS * kBcgMaxS;         // right-hand side
  double* X = Bm + kBcgMaxS * kBcgMaxS;         // solution
  __shared__ int fail, all_conv;
  __shared__ int null_col[kBcgMaxS];
  // pivots below this fraction of the largest are zero (rounding level of the
  // Gram matrices: FP64 vectors 1e-12, FP32 vectors 1e-10)
  const double eps = pr.precision == 0 ? 1e-12 : 1e-10;
  double* RR = pr.bcg_RR + (int64_t)b * kBcgMaxS * kBcgMaxS;
  const double* G1 = pr.bcg_G1 + (int64_t)b * kBcgMaxS * kBcgMaxS;
  const double* G2 = pr.bcg_G2 + (int64_t)b * kBcgMaxS * kBcgMaxS;
  double* out = (phase == 0 ? pr.bcg_alpha : pr.bcg_beta) + (int64_t)b * kBcgMaxS * kBcgMaxS;
  if (phase == 1) {
    if (threadIdx.x == 0) all_conv = 1;
    __syncthreads();
    for (int i = threadIdx.x; i < s; i += blockDim.x) {
      const int64_t sid = bi.sid0 + i;
      const double rr = G2[i * kBcgMaxS + i];
      if (it == 0) pr.bcg_bn2[sid] = rr;
      const double bn2 = pr.bcg_bn2[sid];
      pr.relres[sid] = bn2 > 0.0 ? sqrt(rr / bn2) : 0.0;
      pr.iters[sid] = it;
      if (!(rr <= pr.tol * pr.tol * bn2)) atomicAnd(&all_conv, 0);
    }
    __syncthreads();
    bool stop = pr.fixed_iters > 0 ? (it >= pr.fixed_iters) : (all_conv != 0);
    if (!stop && last) {   // iteration cap reached with a column still running
      if (pr.fixed_iters <= 0 && threadIdx.x == 0) atomicOr(&pr.status[0], kStatNotConverged);
      stop = true;
    }
    if (stop) {
      if (threadIdx.x == 0) pr.bcg_state[b] = 1;
      return;
    }
    if (it == 0) {   // initial residual: RR = R^T R (P = R needs no beta)
      for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
        const int i = e / s, j = e % s;
        RR[i * kBcgMaxS + j] = G2[i * kBcgMaxS + j];
      }
      if (threadIdx.x == 0) atomicAdd(pr.bcg_running, 1);
      return;
    }
  }
  // factor the matrix (phase 0: P^T Q, phase 1: the old R^T R), solve for the new coefficients
  for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
    const int i = e / s, j = e % s;
    A[i * kBcgMaxS + j] = phase == 0 ? G1[i * kBcgMaxS + j] : RR[i * kBcgMaxS + j];
    Bm[i * kBcgMaxS + j] = phase == 0 ? RR[i * kBcgMaxS + j] : G2[i * kBcgMaxS + j];
  }
  __syncthreads();
  if (!chol_smem(A, s, eps, null_col, &fail)) {
    if (threadIdx.x == 0) {
      pr.bcg_state[b] = 2;
      atomicOr(&pr.status[0], kStatBreakdown);
    }
    return;
  }
  __syncthreads();
  chol_solve_smem(A, null_col, Bm, X, s);
  __syncthreads();
  for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
    const int i = e / s, j = e % s;
    out[i * kBcgMaxS + j] = X[i * kBcgMaxS + j];
    if (phase == 1) RR[i * kBcgMaxS + j] = G2[i * kBcgMaxS + j];
  }
  if (phase == 1 && threadIdx.x == 0) atomicAdd(pr.bcg_running, 1);
}

// phase 0: X += P alpha, R -= Q alpha.  phase 1: P = R + P beta.  CTA per
// (row chunk, block), the s x s coefficients in shared memory, thread per row.
template <typename T>
__global__ void __launch_bounds__(128) k_bcg_update(const ProblemDev* dp, int phase) {
  const ProblemDev& pr = *dp;
  const int b = blockIdx.y;
  if (b >= pr.bcg_nblocks || pr.bcg_state[b] != 0) return;
  const BlockInfo bi = block_info(pr, b);
  const int s = bi.s;
  __shared__ double cf[kBcgMaxS * kBcgMaxS];
  const double* src = (phase == 0 ? pr.bcg_alpha : pr.bcg_beta) + (int64_t)b * kBcgMaxS * kBcgMaxS;
  for (int e = threadIdx.x; e < s * s; e += blockDim.x) cf[(e / s) * kBcgMaxS + e % s] = src[(e / s) * kBcgMaxS + e % s];
  __syncthreads();
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= pr.d) return;
  const int64_t d = pr.d;
  T* X = reinterpret_cast<T*>(pr.U) + bi.sid0 * d;
  T* R = reinterpret_cast<T*>(pr.bcg_R) + bi.sid0 * d;
  T* P = reinterpret_cast<T*>(pr.bcg_P) + bi.sid0 * d;
  const T* Qm = reinterpret_cast<const T*>(pr.bcg_Q) + bi.sid0 * d;
  T pv[kBcgMaxS], qv[kBcgMaxS];
#pragma unroll
  for (int i = 0; i < kBcgMaxS; ++i) {
    pv[i] = i < s ? P[i * d + a] : T(0);
    qv[i] = (phase == 0 && i < s) ? Qm[i * d + a] : T(0);
  }
  for (int j = 0; j < s; ++j) {
    double sp = 0.0, sq = 0.0;
#pragma unroll
    for (int i = 0; i < kBcgMaxS; ++i) {
      if (i < s) {
        sp = fma((double)pv[i], cf[i * kBcgMaxS + j], sp);
        if (phase == 0) sq = fma((double)qv[i], cf[i * kBcgMaxS + j], sq);
      }
    }
    if (phase == 0) {
      X[j * d + a] += to_t<T>(sp);
      R[j * d + a] -= to_t<T>(sq);
    } else {
      P[j * d + a] = R[j * d + a] + to_t<T>(sp);
    }
  }
}

__global__ void k_bcg_reset(const ProblemDev* dp) {
  const ProblemDev& pr = *dp;
  for (int b = threadIdx.x; b < pr.bcg_nblocks; b += blockDim.x) pr.bcg_state[b] = 0;
  if (threadIdx.x == 0) *pr.bcg_running = 0;
}

__global__ void k_bcg_zero_running(const ProblemDev* dp) { *dp->bcg_running = 0; }

template <typename T>
int run_bcg_t(const ProblemDev& p, const ProblemDev* dp, cudaStream_t st) {
  const int nb = p.bcg_nblocks;
  const int smax = p.do_pert ? (int)p.N : 1;
  const dim3 gall((unsigned)(((int64_t)p.nsys * p.d + 255) / 256));
  const dim3 gmv((unsigned)((p.d + 127) / 128), (unsigned)p.nsys);
  const dim3 ggram((unsigned)smax, (unsigned)nb);
  const size_t gsm = (size_t)kGramThreads * smax * sizeof(double);
  const size_t ssm = 3 * (size_t)kBcgMaxS * kBcgMaxS * sizeof(double);
  const dim3 gupd((unsigned)((p.d + 127) / 128), (unsigned)nb);
  static thread_local int raised = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (raised != dev) {
    const int gmax = (int)((size_t)kGramThreads * kBcgMaxS * sizeof(double));
    if (cudaFuncSetAttribute(k_bcg_gram<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, gmax) != cudaSuccess ||
        cudaFuncSetAttribute(k_bcg_gram<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, gmax) != cudaSuccess ||
        cudaFuncSetAttribute(k_bcg_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssm) != cudaSuccess)
      return INFO_ESRF_ERR_CUDA;
    raised = dev;
  }
  const int maxit = p.fixed_iters > 0 ? p.fixed_iters : p.max_iter;
  k_bcg_reset<<<1, 256, 0, st>>>(dp);
  k_bcg_init<T><<<gall, 256, 0, st>>>(dp);
  k_bcg_gram<T><<<ggram, kGramThreads, gsm, st>>>(dp, 1);        // R^T R of the initial residual
  k_bcg_solve<<<nb, 128, ssm, st>>>(dp, 1, 0, 0);               // ||b_i||, convergence test, RR
  note_launches(4);
  int32_t running = 0;
  for (int it = 1; it <= maxit; ++it) {
    if (cudaMemcpyAsync(&running, p.bcg_running, sizeof(running), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return INFO_ESRF_ERR_CUDA;
    if (running == 0) break;
    k_bcg_zero_running<<<1, 1, 0, st>>>(dp);
    k_bcg_matvec<T><<<gmv, 128, 0, st>>>(dp);
    k_bcg_gram<T><<<ggram, kGramThreads, gsm, st>>>(dp, 0);     // P^T Q
    k_bcg_solve<<<nb, 128, ssm, st>>>(dp, 0, it, 0);            // alpha
    k_bcg_update<T><<<gupd, 128, 0, st>>>(dp, 0);               // X, R
    k_bcg_gram<T><<<ggram, kGramThreads, gsm, st>>>(dp, 1);     // R^T R
    k_bcg_solve<<<nb, 128, ssm, st>>>(dp, 1, it, it == maxit);  // convergence, beta
    k_bcg_update<T><<<gupd, 128, 0, st>>>(dp, 1);               // P
    note_launches(8);
  }
  if (p.do_pert) {
    k_bcg_complete<T><<<dim3((unsigned)((p.d + 255) / 256), (unsigned)p.Q), 256, 0, st>>>(dp);
    note_launches(1);
  }
  return cudaGetLastError() == cudaSuccess ? 0 : INFO_ESRF_ERR_CUDA;
}

}  // namespace

int run_bcg(const ProblemDev& p, const ProblemDev* dp, cudaStream_t st) {
  if (p.nsys < 1) return 0;
  return p.precision == 0 ? run_bcg_t<double>(p, dp, st) : run_bcg_t<float>(p, dp, st);
}

}  // namespace infoesrf
