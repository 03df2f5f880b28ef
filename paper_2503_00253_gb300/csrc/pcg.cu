// a5-a8: persistent batched shifted PCG over every (quadrature node, member)
// system of every problem, plus the mean system (App. E, Eq.
// normalized_linear_solve; Golub & Van Loan Alg. 11.5.1):
//
//     C_q u = b,   C_q = (s_q + 1) I + C,   C = R^-1/2 (L_oo o W W^T) R^-1/2,
//     b = R^-1/2 w_f^(i)  (perturbation)   or   R^-1/2 (y - H mu)  (mean, s = 0).
//
// All systems share the band of C, formed once per analysis, so the matvec
// is a banded sparse-times-dense product over a group of JT systems that
// share one shift.  Each CTA owns one group at a time: its PCG vectors sit
// in shared memory (or in a private global slice when d is large), so a
// group iterates to convergence without any grid-wide synchronization.
// Groups come from an atomic queue, so CTAs that finish early take more.
//
// Preconditioner: the limited-memory preconditioner of App. E,
//   P_q^-1 = (I - Phi T^-1 Phi^T C_q)(I - C_q Phi T^-1 Phi^T) + beta Phi T^-1 Phi^T,
// applied with f = Phi^T r, g = A^T r (A = C Phi) and the k x k matrix
// G_q = (C_q Phi)^T (C_q Phi):  t = T^-1 f,  t2 = g + sigma f - G_q t,
// c = (beta - sigma) t - T^-1 t2,  z = r - A t + Phi c,  r^T z = r^T r - g.t + f.c.
// So f, g and r^T r come out of the same block reduction as the residual
// norm, and one PCG iteration needs two block reductions.
//
// Scalars (rho, alpha, beta, norms, the k x k preconditioner algebra) are FP64
// and handled by one thread per system; dot products of FP32 vectors are
// accumulated as float-float pairs.
#include <math.h>

#include "common.cuh"
#include "internal.h"

namespace infoesrf {

template <typename T, int JT>
struct Row {
  T v[JT];
};

template <typename T, int JT>
__device__ __forceinline__ Row<T, JT> ld_row(const T* base, int64_t a) {
  static_assert((sizeof(T) * JT) % 16 == 0, "row must be a multiple of 16 bytes");
  Row<T, JT> r;
  const uint4* src = reinterpret_cast<const uint4*>(base + a * JT);
  uint4* dst = reinterpret_cast<uint4*>(r.v);
#pragma unroll
  for (int i = 0; i < (int)(sizeof(T) * JT / 16); ++i) dst[i] = src[i];
  return r;
}

template <typename T, int JT>
__device__ __forceinline__ void st_row(T* base, int64_t a, const Row<T, JT>& r) {
  uint4* dst = reinterpret_cast<uint4*>(base + a * JT);
  const uint4* src = reinterpret_cast<const uint4*>(r.v);
#pragma unroll
  for (int i = 0; i < (int)(sizeof(T) * JT / 16); ++i) dst[i] = src[i];
}

struct GroupInfo {
  int prob;
  int lanes;     // active systems in this group
  int i0;        // first member (perturbation groups)
  int q;         // quadrature index, -1 for the mean system
  int lg;        // group index inside the problem
};

__device__ __forceinline__ GroupInfo decode_group(const ProblemDev* tab, int count, int gg) {
  GroupInfo gi;
  int p = 0;
  while (p + 1 < count && tab[p + 1].group_base <= gg) ++p;
  const ProblemDev& pr = tab[p];
  gi.prob = p;
  gi.lg = gg - pr.group_base;
  if (gi.lg < pr.mean_sys) {         // the mean system comes first (hardest shift)
    gi.q = -1;
    gi.i0 = 0;
    gi.lanes = 1;
  } else {
    const int pg = gi.lg - pr.mean_sys;
    gi.q = pg / pr.groups_per_q;
    gi.i0 = (pg % pr.groups_per_q) * pr.JT;
    const int left = (int)pr.N - gi.i0;
    gi.lanes = left < pr.JT ? left : pr.JT;
  }
  return gi;
}

template <typename T, int JT, int KMAX>
struct PcgShared {
  double rho[JT], bn2[JT], rr[JT];
  double Gq[KMAX * KMAX + 1];
  double thq[KMAX + 1];
  T alpha[JT], beta[JT];
  T tco[JT][KMAX + 1], cco[JT][KMAX + 1];
  int active[JT];
  int iters[JT];
  int any_active;
  int group;
  double sigma, beta_lmp;
};

// Warp-level partial of a DotAcc into shared memory (lane 0 writes).
template <typename T>
__device__ __forceinline__ void warp_partial(const DotAcc<T>& acc, float* ff, double* dd, int lane) {
  if constexpr (sizeof(T) == 4) {
    float hi = acc.hi, lo = acc.lo;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
      const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
      ff_merge(hi, lo, h2, l2);
    }
    if (lane == 0) { ff[0] = hi; ff[1] = lo; }
  } else {
    const double s = warp_sum(acc.value());
    if (lane == 0) dd[0] = s;
  }
}

// Sum of the NW warp partials written by warp_partial (called by one thread).
template <typename T, int NW>
__device__ __forceinline__ double combine_partials(const float (*ff)[2], const double* dd) {
  if constexpr (sizeof(T) == 4) {
    float hi = 0.f, lo = 0.f;
    for (int w = 0; w < NW; ++w) ff_merge(hi, lo, ff[w][0], ff[w][1]);
    return (double)hi + (double)lo;
  } else {
    double s = 0.0;
    for (int w = 0; w < NW; ++w) s += dd[w];
    return s;
  }
}

// CTAs per SM the kernel is compiled for: kPcgFp32CtasPerSm for the FP32 path
// with a small Ritz rank (the register budget a thread then gets lets that
// many 256-thread CTAs share an SM), one otherwise.  The grid is sized by the
// measured occupancy at launch, and the vector scratch by this count.
constexpr int kPcgFp32CtasPerSm = 2;
template <typename T, int KMAX>
constexpr int pcg_ctas_per_sm() { return (sizeof(T) == 4 && KMAX <= 12) ? kPcgFp32CtasPerSm : 1; }

template <typename T, int JT, int KMAX>
__global__ void __launch_bounds__(kThreads, pcg_ctas_per_sm<T, KMAX>())
k_pcg(const ProblemDev* tab, int count, int total_groups, int32_t* counter, T* gscratch,
      int64_t scratch_stride, int use_smem, uint64_t band_mask, const int32_t* band_fb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int NW = kThreads / 32;
  constexpr int NVCAP = KMAX <= 12 ? 32 : 64;    // rr, f[k], g[k]
  __shared__ PcgShared<T, JT, KMAX> sh;
  __shared__ T red[JT][NVCAP][NW];
  __shared__ double redd[JT][NVCAP];
  __shared__ float wpf[JT][NW][2];
  __shared__ double wpd[JT][NW];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // Problems in band_mask were given to the band kernel first; this kernel
  // solves them only where it fell back (band_fb[p] != 0).
  auto band_solved = [&](int p) { return ((band_mask >> p) & 1ull) && band_fb[p] == 0; };
  if (band_mask) {
    bool all = true;
    for (int p = 0; p < count && all; ++p) all = band_solved(p);
    if (all) return;
  }

  for (;;) {
    if (tid == 0) sh.group = atomicAdd(counter, 1);
    __syncthreads();
    const int gg = sh.group;
    if (gg >= total_groups) break;
    const GroupInfo gi = decode_group(tab, count, gg);
    const ProblemDev& pr = tab[gi.prob];
    if (band_mask && band_solved(gi.prob)) {
      // skip the rest of this problem's groups at once (the queue only grows)
      if (tid == 0) atomicMax(counter, pr.group_base + pr.num_groups);
      __syncthreads();
      continue;
    }
    const int64_t d = pr.d, N = pr.N;
    const int k = pr.kR < KMAX ? pr.kR : KMAX;

    T* base = use_smem ? reinterpret_cast<T*>(smem_raw) : gscratch + (int64_t)blockIdx.x * scratch_stride;
    T* vr = base;
    T* vp = base + d * JT;
    T* vy = base + 2 * d * JT;
    T* vx = base + 3 * d * JT;
    const T* val = reinterpret_cast<const T*>(pr.oo_val);
    const T* Phi = reinterpret_cast<const T*>(pr.Phi);
    const T* CPhi = reinterpret_cast<const T*>(pr.CPhi);
    const T* W = reinterpret_cast<const T*>(pr.W);

    // ---- group setup: shift, LMP constants, G_q ----
    if (tid == 0) {
      const double s = gi.q < 0 ? 0.0 : pr.s[gi.q];
      sh.sigma = s + 1.0;
      sh.beta_lmp = sh.sigma + pr.scal[1];
    }
    __syncthreads();
    const double sigma = sh.sigma;
    const T sigma_t = to_t<T>(sigma);
    for (int e = tid; e < k * k; e += blockDim.x) {
      const int i = e / k, j = e % k;
      const int kk = pr.kR;   // gram matrices are stored with the problem's k
      const int ge = i * kk + j, gt = j * kk + i;
      // G_q = A^T A + sigma (A^T Phi + Phi^T A) + sigma^2 Phi^T Phi
      sh.Gq[e] = pr.gram[2 * kk * kk + ge] + sigma * (pr.gram[kk * kk + ge] + pr.gram[kk * kk + gt]) +
                 sigma * sigma * pr.gram[ge];
    }
    for (int m = tid; m < k; m += blockDim.x) sh.thq[m] = pr.theta[m] + sigma;
    if (tid < JT) {
      sh.active[tid] = tid < gi.lanes;
      sh.iters[tid] = 0;
      sh.beta[tid] = T(0);
      sh.rr[tid] = 0.0;
    }

    // ---- x = 0, r = b, p = 0 ----
    for (int64_t a = tid; a < d; a += blockDim.x) {
      Row<T, JT> rb, zero;
      const T ri = to_t<T>(pr.rinv[a]);
#pragma unroll
      for (int j = 0; j < JT; ++j) {
        zero.v[j] = T(0);
        T b = T(0);
        if (j < gi.lanes) {
          if (gi.q < 0) b = to_t<T>(pr.bmean[a]);
          else b = W[a * N + gi.i0 + j] * ri;
        }
        rb.v[j] = b;
      }
      st_row<T, JT>(vr, a, rb);
      st_row<T, JT>(vp, a, zero);
      st_row<T, JT>(vx, a, zero);
    }
    __syncthreads();

    bool first = true;
    const int maxit = pr.fixed_iters > 0 ? pr.fixed_iters : pr.max_iter;
    const int pk = pr.kR;   // row stride of Phi / CPhi

    // rr, f = Phi^T r, g = A^T r -> preconditioner scalars
    auto reduce_residual = [&]() {
#pragma unroll 1
      for (int j = 0; j < JT; ++j) {
        T v[NVCAP];
#pragma unroll
        for (int i = 0; i < NVCAP; ++i) v[i] = T(0);
        DotAcc<T> rr;
        for (int64_t a = tid; a < d; a += blockDim.x) {
          const T r = vr[a * JT + j];
          rr.add_prod(r, r);
#pragma unroll
          for (int m = 0; m < KMAX; ++m) {
            if (m < k) {
              v[1 + m] += Phi[a * pk + m] * r;
              v[1 + KMAX + m] += CPhi[a * pk + m] * r;
            }
          }
        }
        const T s0 = warp_reduce_scatter32<T>(*reinterpret_cast<T(*)[32]>(&v[0]), lane);
        red[j][lane][warp] = s0;
        if constexpr (NVCAP == 64) {
          const T s1 = warp_reduce_scatter32<T>(*reinterpret_cast<T(*)[32]>(&v[32]), lane);
          red[j][32 + lane][warp] = s1;
        }
        warp_partial<T>(rr, wpf[j][warp], &wpd[j][warp], lane);
      }
      __syncthreads();
      for (int e = tid; e < JT * NVCAP; e += blockDim.x) {
        const int j = e / NVCAP, vi = e % NVCAP;
        if (vi == 0) {
          redd[j][0] = combine_partials<T, NW>(wpf[j], wpd[j]);
        } else {
          T s = T(0);
#pragma unroll
          for (int w = 0; w < NW; ++w) s += red[j][vi][w];
          redd[j][vi] = (double)s;
        }
      }
      __syncthreads();
      if (tid < JT) {
        const int j = tid;
        const double rr = redd[j][0];
        if (first) sh.bn2[j] = rr;
        const bool was_active = sh.active[j];
        bool act = was_active;
        if (act && pr.fixed_iters <= 0 && !(rr > pr.tol * pr.tol * sh.bn2[j])) act = false;
        if (act && !(rr > 0.0)) act = false;
        if (act && !isfinite(rr)) act = false;
        double rho = rr;
        if (k > 0) {
          double t[KMAX], t2[KMAX];
          for (int m = 0; m < k; ++m) t[m] = redd[j][1 + m] / sh.thq[m];
          double gt = 0.0, fc = 0.0;
          for (int m = 0; m < k; ++m) {
            double acc = redd[j][1 + KMAX + m] + sigma * redd[j][1 + m];
            for (int i2 = 0; i2 < k; ++i2) acc -= sh.Gq[m * k + i2] * t[i2];
            t2[m] = acc;
          }
          for (int m = 0; m < k; ++m) {
            const double c = (sh.beta_lmp - sigma) * t[m] - t2[m] / sh.thq[m];
            gt += redd[j][1 + KMAX + m] * t[m];
            fc += redd[j][1 + m] * c;
            sh.tco[j][m] = to_t<T>(t[m]);
            sh.cco[j][m] = to_t<T>(c);
          }
          rho = rr - gt + fc;
        }
        if (!act) {
          sh.beta[j] = T(0);
          for (int m = 0; m < k; ++m) { sh.tco[j][m] = T(0); sh.cco[j][m] = T(0); }
        } else if (first) {
          sh.beta[j] = T(0);
          sh.rho[j] = rho;
        } else {
          sh.beta[j] = to_t<T>(rho / sh.rho[j]);
          sh.rho[j] = rho;
        }
        if (was_active || first) sh.rr[j] = rr;
        sh.active[j] = act;
      }
      __syncthreads();
      if (tid == 0) {
        int any = 0;
        for (int j = 0; j < JT; ++j) any |= sh.active[j];
        sh.any_active = any;
      }
      __syncthreads();
    };

    // z = P^-1 r, p = z + beta p
    auto update_direction = [&]() {
      for (int64_t a = tid; a < d; a += blockDim.x) {
        const Row<T, JT> r = ld_row<T, JT>(vr, a);
        Row<T, JT> p = ld_row<T, JT>(vp, a);
        T z[JT];
#pragma unroll
        for (int j = 0; j < JT; ++j) z[j] = r.v[j];
        for (int m = 0; m < k; ++m) {
          const T ph = Phi[a * pk + m], cp = CPhi[a * pk + m];
#pragma unroll
          for (int j = 0; j < JT; ++j) z[j] += ph * sh.cco[j][m] - cp * sh.tco[j][m];
        }
#pragma unroll
        for (int j = 0; j < JT; ++j) p.v[j] = sh.active[j] ? z[j] + sh.beta[j] * p.v[j] : p.v[j];
        st_row<T, JT>(vp, a, p);
      }
      __syncthreads();
    };

    reduce_residual();
    first = false;
    if (sh.any_active) update_direction();

    int it = 0;
    while (sh.any_active && it < maxit) {
      ++it;
      // ---- y = C_q p, p^T y ----
      DotAcc<T> pap[JT];
      for (int64_t a = tid; a < d; a += blockDim.x) {
        const Row<T, JT> p = ld_row<T, JT>(vp, a);
        T acc[JT];
#pragma unroll
        for (int j = 0; j < JT; ++j) acc[j] = sigma_t * p.v[j];
        const int nnz = pr.oo_nnz[a];
        for (int e = 0; e < nnz; ++e) {
          const T c = val[(int64_t)e * d + a];
          const int b = pr.oo_col[(int64_t)e * d + a];
          const Row<T, JT> pb = ld_row<T, JT>(vp, b);
#pragma unroll
          for (int j = 0; j < JT; ++j) acc[j] += c * pb.v[j];
        }
        Row<T, JT> y;
#pragma unroll
        for (int j = 0; j < JT; ++j) {
          y.v[j] = acc[j];
          pap[j].add_prod(p.v[j], acc[j]);
        }
        st_row<T, JT>(vy, a, y);
      }
#pragma unroll
      for (int j = 0; j < JT; ++j) warp_partial<T>(pap[j], wpf[j][warp], &wpd[j][warp], lane);
      __syncthreads();
      if (tid < JT) {
        const int j = tid;
        T alpha = T(0);
        if (sh.active[j]) {
          const double pAp = combine_partials<T, NW>(wpf[j], wpd[j]);
          if (pAp > 0.0 && isfinite(pAp)) {
            alpha = to_t<T>(sh.rho[j] / pAp);
            sh.iters[j] = it;
          } else {
            sh.active[j] = 0;
            atomicOr(&pr.status[0], kStatBreakdown);
          }
        }
        sh.alpha[j] = alpha;
      }
      __syncthreads();
      // ---- x += alpha p, r -= alpha y ----
      for (int64_t a = tid; a < d; a += blockDim.x) {
        const Row<T, JT> p = ld_row<T, JT>(vp, a);
        const Row<T, JT> y = ld_row<T, JT>(vy, a);
        Row<T, JT> x = ld_row<T, JT>(vx, a);
        Row<T, JT> r = ld_row<T, JT>(vr, a);
#pragma unroll
        for (int j = 0; j < JT; ++j) {
          x.v[j] += sh.alpha[j] * p.v[j];
          r.v[j] -= sh.alpha[j] * y.v[j];
        }
        st_row<T, JT>(vx, a, x);
        st_row<T, JT>(vr, a, r);
      }
      __syncthreads();
      reduce_residual();
      if (!sh.any_active) break;
      update_direction();
    }

    // ---- results ----
    // lane j holds system sid0 + j (the mean group has one lane, sid 0)
    const int64_t sid0 = gi.q < 0 ? 0 : pr.mean_sys + (int64_t)gi.q * N + gi.i0;
    T* U = reinterpret_cast<T*>(pr.U);
    for (int j = 0; j < gi.lanes; ++j)
      for (int64_t a = tid; a < d; a += blockDim.x) U[(sid0 + j) * d + a] = vx[a * JT + j];
    if (tid < gi.lanes) {
      const int64_t sidx = sid0 + tid;
      pr.iters[sidx] = sh.iters[tid];
      const double bn = sh.bn2[tid];
      pr.relres[sidx] = bn > 0 ? sqrt(sh.rr[tid] / bn) : 0.0;
      if (sh.active[tid] && pr.fixed_iters <= 0) atomicOr(&pr.status[0], kStatNotConverged);
    }
    __syncthreads();
  }
}

int pcg_jt(int precision) { return precision == 0 ? 4 : 8; }

static size_t vec_bytes(const ProblemTable& tab) {
  int64_t dmax = 0;
  for (int i = 0; i < tab.count; ++i) dmax = tab.p[i].d > dmax ? tab.p[i].d : dmax;
  const int jt = pcg_jt(tab.p[0].precision);
  const size_t esz = tab.p[0].precision == 0 ? 8 : 4;
  return (size_t)4 * (size_t)dmax * jt * esz;
}

static constexpr size_t kSmemVecLimit = 160 * 1024;

size_t pcg_scratch_bytes(const ProblemTable& tab, int num_sms) {
  const size_t vb = vec_bytes(tab);
  if (vb <= kSmemVecLimit) return 0;
  int kmax = 0;
  for (int i = 0; i < tab.count; ++i) kmax = tab.p[i].kR > kmax ? tab.p[i].kR : kmax;
  const int per_sm = (tab.p[0].precision == 1 && kmax <= 12) ? kPcgFp32CtasPerSm : 1;
  return vb * (size_t)num_sms * (size_t)per_sm;   // one slice per resident CTA
}

template <typename T, int JT, int KMAX>
static int launch_pcg_t(const ProblemTable& tab, const ProblemDev* dtab, int32_t* counter, void* scratch,
                        size_t scratch_bytes, int num_sms, cudaStream_t st, uint64_t band_mask,
                        const int32_t* band_fb) {
  const size_t vb = vec_bytes(tab);
  const int use_smem = vb <= kSmemVecLimit;
  const size_t dyn = use_smem ? vb : 0;
  // the attribute once per thread and device, the occupancy per dynamic size
  constexpr int kMaxDev = 64;
  static thread_local bool attr_set[kMaxDev] = {};
  static thread_local size_t occ_dyn[kMaxDev] = {};
  static thread_local int occ_per_sm[kMaxDev] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
    cudaGetLastError();
    dev = -1;
  }
  if (dev < 0 || !attr_set[dev]) {
    cudaFuncSetAttribute(k_pcg<T, JT, KMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemVecLimit);
    if (dev >= 0) attr_set[dev] = true;
  }
  int per_sm = 0;
  if (dev >= 0 && occ_per_sm[dev] > 0 && occ_dyn[dev] == dyn) per_sm = occ_per_sm[dev];
  if (per_sm < 1) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg<T, JT, KMAX>, kThreads, dyn) != cudaSuccess ||
        per_sm < 1) {
      cudaGetLastError();
      per_sm = 1;
    }
    if (dev >= 0) {
      occ_dyn[dev] = dyn;
      occ_per_sm[dev] = per_sm;
    }
  }
  int64_t want = (int64_t)per_sm * num_sms;
  if (!use_smem && vb > 0) want = std::min<int64_t>(want, (int64_t)(scratch_bytes / vb));   // scratch slices
  int grid = (int)std::min<int64_t>(tab.total_groups, want);
  if (!use_smem && grid < 1 && tab.total_groups > 0) return -1;
  if (grid <= 0) return 0;
  cudaMemsetAsync(counter, 0, sizeof(int32_t), st);
  k_pcg<T, JT, KMAX><<<grid, kThreads, dyn, st>>>(dtab, tab.count, tab.total_groups, counter,
                                            reinterpret_cast<T*>(scratch), (int64_t)(vb / sizeof(T)),
                                            use_smem, band_mask, band_fb);
  note_launches(1);
  return 0;
}

int launch_pcg(const ProblemTable& tab, const ProblemDev* dtab, int32_t* counter, void* scratch,
               size_t scratch_bytes, int num_sms, cudaStream_t st) {
  int kmax = 0;
  for (int i = 0; i < tab.count; ++i) kmax = tab.p[i].kR > kmax ? tab.p[i].kR : kmax;
  const bool small = kmax <= 12;
  // Problems the band kernel can take are launched there first, one launch
  // per problem (each with its own queue and fall-back flag in the counter
  // area); the general kernel then solves the rest and any that fell back.
  // cluster_size 0 uses the band kernel for a single problem only: in a batch
  // the general kernel packs the systems of many small problems onto all SMs
  // at once, while band launches run one after another, each with its own
  // drain (on 64 uneven problems the two came out within 2%, general first).
  const bool use_band = tab.cluster_size > 0 || (tab.cluster_size == 0 && tab.count == 1);
  int32_t* band_q = counter + 1;
  int32_t* band_fb = counter + 1 + kMaxProblems;
  uint64_t mask = 0;
  for (int i = 0; i < tab.count && use_band; ++i) {
    const ProblemDev& p = tab.p[i];
    if (!band1d_eligible(p)) continue;
    const int CS = band1d_cluster_size(p, tab.cluster_size);
    if (launch_pcg_band1d(p, dtab + i, CS, band_q + i, band_fb + i, num_sms, st) == 0) mask |= 1ull << i;
  }
  if (tab.p[0].precision == 0) {
    if (small) return launch_pcg_t<double, 4, 12>(tab, dtab, counter, scratch, scratch_bytes, num_sms, st, mask, band_fb);
    return launch_pcg_t<double, 4, 24>(tab, dtab, counter, scratch, scratch_bytes, num_sms, st, mask, band_fb);
  }
  if (small) return launch_pcg_t<float, 8, 12>(tab, dtab, counter, scratch, scratch_bytes, num_sms, st, mask, band_fb);
  return launch_pcg_t<float, 8, 24>(tab, dtab, counter, scratch, scratch_bytes, num_sms, st, mask, band_fb);
}

// ---------------------------------------------------------------------------
// Stage entry points for testing: Y = sigma P + C P and Z = P_q^-1 R for
// FP64 vectors [nvec][d] against the prepared band and Ritz pairs.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_obs_matvec(const ProblemDev* pr, int32_t nvec, const double* P, const double* sigma,
                             double* Y) {
  const int64_t d = pr->d;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d * nvec) return;
  const int64_t v = i / d, a = i % d;
  const T* val = reinterpret_cast<const T*>(pr->oo_val);
  const T* Pv = nullptr;
  (void)Pv;
  T acc = to_t<T>(sigma[v]) * to_t<T>(P[v * d + a]);
  const int nnz = pr->oo_nnz[a];
  for (int e = 0; e < nnz; ++e)
    acc += val[(int64_t)e * d + a] * to_t<T>(P[v * d + pr->oo_col[(int64_t)e * d + a]]);
  Y[v * d + a] = (double)acc;
}

void launch_obs_matvec(const ProblemDev& pr, const ProblemDev* dpr, int32_t nvec, const double* P,
                       const double* sigma, double* Y, cudaStream_t st) {
  const int64_t tot = pr.d * nvec;
  if (tot <= 0) return;
  if (pr.precision == 0)
    k_obs_matvec<double><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(dpr, nvec, P, sigma, Y);
  else
    k_obs_matvec<float><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(dpr, nvec, P, sigma, Y);
  note_launches(1);
}

// One block per vector; same algebra as the PCG kernel, FP64 throughout.
template <typename T>
__global__ void k_lmp_apply(const ProblemDev* prp, int32_t nvec, const double* Rv, const double* sigma_in,
                            double* Z) {
  const ProblemDev& pr = *prp;
  const int64_t d = pr.d;
  const int k = pr.kR;
  const int v = blockIdx.x;
  const double* r = Rv + (int64_t)v * d;
  double* z = Z + (int64_t)v * d;
  const double sigma = sigma_in[v];
  const T* Phi = reinterpret_cast<const T*>(pr.Phi);
  const T* A = reinterpret_cast<const T*>(pr.CPhi);
  __shared__ double fg[2 * kMaxK][kThreads / 32];
  __shared__ double cc[2][kMaxK];
  for (int m = 0; m < 2 * k; ++m) {
    double acc = 0.0;
    for (int64_t a = threadIdx.x; a < d; a += blockDim.x)
      acc += (double)(m < k ? Phi[a * k + m] : A[a * k + (m - k)]) * r[a];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) fg[m][threadIdx.x >> 5] = acc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double f[kMaxK], g[kMaxK], t[kMaxK];
    for (int m = 0; m < 2 * k; ++m) {
      double s = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += fg[m][w];
      if (m < k) f[m] = s; else g[m - k] = s;
    }
    const double beta = sigma + pr.scal[1];
    for (int m = 0; m < k; ++m) t[m] = f[m] / (pr.theta[m] + sigma);
    for (int m = 0; m < k; ++m) {
      double t2 = g[m] + sigma * f[m];
      for (int i = 0; i < k; ++i) {
        const int e = m * k + i;
        const double G = pr.gram[2 * k * k + e] + sigma * (pr.gram[k * k + e] + pr.gram[k * k + i * k + m]) +
                         sigma * sigma * pr.gram[e];
        t2 -= G * t[i];
      }
      cc[0][m] = t[m];
      cc[1][m] = (beta - sigma) * t[m] - t2 / (pr.theta[m] + sigma);
    }
  }
  __syncthreads();
  for (int64_t a = threadIdx.x; a < d; a += blockDim.x) {
    double acc = r[a];
    for (int m = 0; m < k; ++m) acc += (double)Phi[a * k + m] * cc[1][m] - (double)A[a * k + m] * cc[0][m];
    z[a] = acc;
  }
}

void launch_lmp_apply(const ProblemDev& pr, const ProblemDev* dpr, int32_t nvec, const double* Rv,
                      const double* sigma, double* Z, cudaStream_t st) {
  if (nvec <= 0) return;
  if (pr.precision == 0) k_lmp_apply<double><<<nvec, kThreads, 0, st>>>(dpr, nvec, Rv, sigma, Z);
  else k_lmp_apply<float><<<nvec, kThreads, 0, st>>>(dpr, nvec, Rv, sigma, Z);
  note_launches(1);
}

}  // namespace infoesrf
