// a9-a11: quadrature-weighted accumulation and the state-space update.
//
//   vbar^(i) = R^-1/2 sum_q p_q u_q^(i)                       (Sec. 3.2, App. E)
//   z_a^(i)  = z^(i) - Sxh vbar^(i),  A_a = sqrt(N-1) Z_a       (Sec. 3.2)
//   mu_a     = mu + Sxh R^-1/2 u_mean                           (Eq. info_esrf_mean_solve)
//
// The quadrature sum is FP64.  Sxh is the state-obs band formed in setup, so
// the state update is one banded product with N + 1 right-hand sides.
#include "common.cuh"
#include "internal.h"

namespace infoesrf {

template <typename T>
__global__ void k_accumulate(const ProblemDev* tab) {
  const ProblemDev& pr = tab[blockIdx.y];
  const int64_t N1 = pr.N + 1;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= pr.d * N1) return;
  const int64_t a = i / N1, m = i % N1;
  const int64_t d = pr.d;
  const T* U = reinterpret_cast<const T*>(pr.U);
  double acc = 0.0;
  if (m < pr.N) {
    if (pr.do_pert) {
      for (int q = 0; q < pr.Q; ++q) {
        const int64_t sid = pr.mean_sys + (int64_t)q * pr.N + m;
        acc += pr.p[q] * (double)U[sid * d + a];
      }
    }
  } else if (pr.do_mean) {
    acc = (double)U[a];   // sid 0
  }
  const double v = pr.rinv[a] * acc;
  pr.Vbar[a * N1 + m] = v;
  reinterpret_cast<T*>(pr.VbarT)[a * N1 + m] = to_t<T>(v);
}

// One thread per (state point, pair of columns: member m < N, or the mean
// m == N), state points fastest so that band loads and output stores are
// coalesced; each band entry is read once for both columns of the pair (one
// column per thread left the band reads doubled, four left too few warps to
// hide the gathers).
constexpr int kStateCols = 2;
template <typename T>
__global__ void k_state_apply(const ProblemDev* tab) {
  const ProblemDev& pr = tab[blockIdx.z];
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = pr.n, N = pr.N, N1 = N + 1;
  const int64_t m0 = (int64_t)blockIdx.y * kStateCols;
  if (x >= n || m0 > N) return;
  const T* __restrict__ val = reinterpret_cast<const T*>(pr.xo_val);
  const int32_t* __restrict__ col = pr.xo_col;
  const T* __restrict__ Vb = reinterpret_cast<const T*>(pr.VbarT);
  const int nnz = pr.xo_nnz[x];
  const int nc = (int)(N1 - m0 < kStateCols ? N1 - m0 : kStateCols);
  T acc[kStateCols];
#pragma unroll
  for (int j = 0; j < kStateCols; ++j) acc[j] = T(0);
#pragma unroll 4
  for (int e = 0; e < nnz; ++e) {
    const T v = val[(int64_t)e * n + x];
    const T* vb = Vb + (int64_t)col[(int64_t)e * n + x] * N1 + m0;
#pragma unroll
    for (int j = 0; j < kStateCols; ++j)
      if (j < nc) acc[j] += v * vb[j];
  }
  const double mu = pr.mu[x];
#pragma unroll
  for (int j = 0; j < kStateCols; ++j) {
    if (j >= nc) break;
    const int64_t m = m0 + j;
    const double inc = (double)acc[j];
    if (m < N) {
      if (pr.do_pert) pr.A_a[m * n + x] = (pr.X[m * n + x] - mu) - pr.sqrt_nm1 * inc;
    } else if (pr.do_mean) {
      pr.mu_a[x] = mu + inc;
    }
  }
}

void launch_finish(const ProblemTable& tab, const ProblemDev* dtab, cudaStream_t st, bool accumulate) {
  int64_t dn1 = 0, nmax = 0, Nmax = 0;
  for (int i = 0; i < tab.count; ++i) {
    const ProblemDev& p = tab.p[i];
    dn1 = p.d * (p.N + 1) > dn1 ? p.d * (p.N + 1) : dn1;
    nmax = p.n > nmax ? p.n : nmax;
    Nmax = p.N > Nmax ? p.N : Nmax;
  }
  const dim3 ga((unsigned)((dn1 + 255) / 256), tab.count);
  const dim3 gs((unsigned)((nmax + 127) / 128), (unsigned)((Nmax + kStateCols) / kStateCols), tab.count);
  if (tab.p[0].precision == 0) {
    if (accumulate) { k_accumulate<double><<<ga, 256, 0, st>>>(dtab); note_launches(1); }
    k_state_apply<double><<<gs, 128, 0, st>>>(dtab); note_launches(1);
  } else {
    if (accumulate) { k_accumulate<float><<<ga, 256, 0, st>>>(dtab); note_launches(1); }
    k_state_apply<float><<<gs, 128, 0, st>>>(dtab); note_launches(1);
  }
}

}  // namespace infoesrf
