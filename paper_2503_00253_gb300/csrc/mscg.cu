// a5-a7 and a9 by multi-shift CG (Sec. 3.3, the first alternative to one PCG
// run per system).  In normalized form every system of member i,
//
//     ((s_q + 1) I + C) u_q = b = R^-1/2 w^(i),    q = 1..Q,
//
// is the same C shifted by sigma_q = s_q + 1, and Krylov subspaces are
// invariant under shifts.  So one CG run on the base system
// (C + sigma_0 I) u = b, sigma_0 = min_q sigma_q, gives every shifted iterate:
// the shifted residuals stay collinear with the base residual,
// r_k^(q) = zeta_k^(q) r_k, and with delta_q = sigma_q - sigma_0
//
//   zeta_{k+1} = zeta_k zeta_{k-1} alpha_{k-1} /
//                (alpha_k beta_{k-1} (zeta_{k-1} - zeta_k) + zeta_{k-1} alpha_{k-1} (1 + delta_q alpha_k)),
//   alpha_k^(q) = alpha_k zeta_{k+1} / zeta_k,   beta_k^(q) = beta_k (zeta_{k+1} / zeta_k)^2,
//   u_q += alpha_k^(q) p_q,   p_q <- zeta_{k+1} r_{k+1} + beta_k^(q) p_q
//
// (Frommer & Glassner 1998; Jegerlehner 1996).  No preconditioner (the LMP
// of App. E is not shift-invariant).  Only sum_q p_q u_q is needed (Sec. 3.2),
// so it is accumulated in place of the Q solutions.  Shift q stops once
// |zeta^(q)| ||r|| <= tol ||b|| (1e-30 ||b|| in fixed-iteration mode, so that
// zeta never underflows); the mean system is a chain with the single shift 1.
//
// GB300 mapping: one thread-block cluster of CS CTAs per group of LC chains
// (members) of one problem.  CTA c of the cluster owns rows [c Rc, (c+1) Rc) of
// the observation space: their residuals, shifted directions, quadrature sums
// and their rows of C's band (staged in shared memory once per problem when
// they fit, else read from L2).  Every CTA keeps a full copy of each chain's
// base direction p in shared memory; after each update the owner pushes its
// rows, as 16-byte distributed-shared-memory stores, to the CTAs whose rows of
// C read them (on a 1-D band: itself and its two neighbours).  An iteration has
// three cluster barriers: the partial sums of p^T (C + sigma_0) p, those of
// r^T r, and the p exchange.  Every CTA then forms the same scalars from the
// same partials in the same order, so the cluster stays in lockstep without a
// leader.  The scalars are FP64 on the FP64 path and float-float (about 48
// bits, FP32 instructions only) on the FP32 path, where FP64 throughput would
// dominate an iteration; the coefficients that scale FP32 vectors are FP32.
#include <cooperative_groups.h>
#include <math.h>
#include <string.h>

#include "common.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace infoesrf {

constexpr int kMsThreads = 256;
constexpr int kMsWarps = kMsThreads / 32;
constexpr int kMsMaxCS = 8;
constexpr int kMsMaxLC = 4;
// Dynamic shared memory the plan may use per CTA (the rest of the 227 KB
// opt-in limit is left for the static arrays).
constexpr size_t kMsSmemBudget = 224 * 1024;

// Threads per matvec row (a power of two <= 8 that keeps a CTA of kMsThreads
// busy) and the row stride of the staged slice of C: a multiple of 32 plus
// 32 / sub, so that the sub threads of a row, which read neighbouring slots,
// fall in different banks.
__host__ __device__ __forceinline__ int ms_sub(int Rc) {
  int sub = 1;
  while (sub < 8 && Rc * sub * 2 <= kMsThreads) sub <<= 1;
  return sub;
}
__host__ __device__ __forceinline__ int ms_cstride(int Rc) {
  const int sub = ms_sub(Rc);
  return (Rc + 31) / 32 * 32 + (sub > 1 ? 32 / sub : 0);
}

// Bytes of dynamic shared memory for LC chains (layout in k_mscg).
static size_t ms_dyn_bytes(int LC, int Rc, int dall, int Qs, int cap, size_t esz, bool c_smem, bool ps_smem) {
  size_t b = esz * ((size_t)LC * dall + 4 * (size_t)LC * Rc + 7 * (size_t)LC * Qs);
  b += 8 * 6 * (size_t)LC * Qs + 4 * 4 * (size_t)LC * Qs + 4 * (size_t)Rc;
  if (c_smem) b += (esz + 4) * (size_t)cap * ms_cstride(Rc);
  if (ps_smem) b += esz * (size_t)LC * Qs * Rc;
  return b;
}

__host__ __device__ __forceinline__ int chains_of(const ProblemDev& p) {
  return p.do_mean + (p.do_pert ? (int)p.N : 0);
}

// Cluster-wide sums of LC per-thread partials: warp shuffles, one partial per
// warp in shared memory, then thread (j, dst) combines the warps of chain j and
// stores the CTA's sum into slot [crank][j] of CTA dst (a float-float pair for
// FP32 vectors, a double for FP64).  Ends with the cluster barrier, after which
// red[c * LC + j] holds CTA c's partial on every CTA.
template <typename T, int LC>
__device__ __forceinline__ void ms_push_partials(DotAcc<T> (&acc)[LC], double* red, float (*wff)[kMsMaxLC][2],
                                                 double (*wdd)[kMsMaxLC], cg::cluster_group& cluster, int CS,
                                                 int crank) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < LC; ++j) {
    if constexpr (sizeof(T) == 4) {
      float hi = acc[j].hi, lo = acc[j].lo;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
        const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        ff_merge(hi, lo, h2, l2);
      }
      if (lane == 0) {
        wff[warp][j][0] = hi;
        wff[warp][j][1] = lo;
      }
    } else {
      const double s = warp_sum(acc[j].value());
      if (lane == 0) wdd[warp][j] = s;
    }
  }
  __syncthreads();
  if ((int)threadIdx.x < LC * CS) {
    const int j = threadIdx.x % LC, dst = threadIdx.x / LC;
    double* slot = cluster.map_shared_rank(red, dst) + crank * LC + j;
    if constexpr (sizeof(T) == 4) {
      float hi = 0.f, lo = 0.f;
      for (int w = 0; w < kMsWarps; ++w) ff_merge(hi, lo, wff[w][j][0], wff[w][j][1]);
      *reinterpret_cast<float2*>(slot) = make_float2(hi, lo);
    } else {
      double v = 0.0;
      for (int w = 0; w < kMsWarps; ++w) v += wdd[w][j];
      *slot = v;
    }
  }
  cluster.sync();
}

// Sum over the cluster's CTAs of chain j's partials, in rank order.
__device__ __forceinline__ FF ms_sum_ff(const double* red, int CS, int LC, int j) {
  float hi = 0.f, lo = 0.f;
  for (int c = 0; c < CS; ++c) {
    const float2 v = reinterpret_cast<const float2*>(red)[c * LC + j];
    ff_merge(hi, lo, v.x, v.y);
  }
  return ff_norm(hi, lo);
}
__device__ __forceinline__ double ms_sum_d(const double* red, int CS, int LC, int j) {
  double s = 0.0;
  for (int c = 0; c < CS; ++c) s += red[c * LC + j];
  return s;
}
__device__ __forceinline__ double ff_to_d(FF a) { return (double)a.h + (double)a.l; }

// A shift index carried in the packed coefficient entry as the bits of a T.
template <typename T>
__device__ __forceinline__ T ms_q_bits(int q) {
  if constexpr (sizeof(T) == 4) return __int_as_float(q);
  else return __longlong_as_double((long long)q);
}
__device__ __forceinline__ int ms_q_of(float v) { return __float_as_int(v); }
__device__ __forceinline__ int ms_q_of(double v) { return (int)__double_as_longlong(v); }

// beta = r'^T r' / r^T r (as double and as T) and ||r'|| of chain j from the
// cluster's partials; also r'^T r' itself (float-float and double) for the
// next step.
template <typename T>
__device__ __forceinline__ void ms_beta(const double* red, int CS, int LC, int j, float rrh, float rrl, double rr,
                                        double& beta, T& beta_t, double& srr, float& rnh, float& rnl,
                                        double& rnd) {
  if constexpr (sizeof(T) == 4) {
    const FF rn = ms_sum_ff(red, CS, LC, j);
    const FF b = ff_div(rn, FF{rrh, rrl});
    const FF sr = rn.h > 0.f ? ff_mul(rn, ff_rsqrt(rn)) : FF{0.f, 0.f};
    beta = ff_to_d(b);
    beta_t = b.h + b.l;
    srr = ff_to_d(sr);
    rnh = rn.h;
    rnl = rn.l;
    rnd = ff_to_d(rn);
  } else {
    const double rn = ms_sum_d(red, CS, LC, j);
    beta = rn / rr;
    beta_t = to_t<T>(beta);
    srr = sqrt(rn);
    rnh = rnl = 0.f;
    rnd = rn;
  }
}

// Four consecutive elements from 16-byte-aligned shared memory.
template <typename T>
__device__ __forceinline__ void ms_ld4(const T* src, T (&v)[4]) {
  if constexpr (sizeof(T) == 4) {
    const float4 x = *reinterpret_cast<const float4*>(src);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
  } else {
    const double2 x = reinterpret_cast<const double2*>(src)[0], y = reinterpret_cast<const double2*>(src)[1];
    v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
  }
}

// Four consecutive elements to 16-byte-aligned shared (or global) memory.
template <typename T>
__device__ __forceinline__ void ms_st4(T* dst, const T (&v)[4]) {
  if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(dst) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
    reinterpret_cast<double2*>(dst)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(dst)[1] = make_double2(v[2], v[3]);
  }
}

// Shift t of the flattened active lists of the chains in `step`: chain j and
// position in its list.
template <int LC>
__device__ __forceinline__ int ms_locate(int t, unsigned step, const int* nact, int& off) {
  int j = 0;
  for (; j < LC - 1; ++j) {
    const int nj = (step >> j & 1u) ? nact[j] : 0;
    if (t < nj) break;
    t -= nj;
  }
  off = t;
  return j;
}

constexpr int kMsZetaWarps = 4;   // warps that run the shifted recurrences while the others update r

// Dynamic shared memory (T arrays first, all sizes multiples of 16 bytes):
//   pfull [LC][dall]   full copy of each chain's base direction p
//   rv, apv [LC][Rc]   own rows of r and (C + sigma_0 I) p
//   ahi, alo [LC][Rc]  own rows of sum_q p_q u_q (float-float for FP32)
//   pk [LC][Qs][4]     this step's p_q alpha^(q), zeta_{k+1}, beta^(q) and q of the
//                      i-th active shift of each chain (one 16- or 32-byte load)
//   wqt, ratt, zt [LC][Qs]  p_q, zeta_{k+1} / zeta_k and zeta_{k+1} in T, for the
//                      coefficients (which only scale T vectors)
//   zeta, zprev, delta, wq, res, rat [LC][Qs] (FP64; res = |zeta| ||r||, rat = zeta_{k+1} / zeta_k)
//   act, itq [LC][Qs], lst [2][LC][Qs] (int): active flags, iteration counts,
//                      and the active shifts of this step and the next
//   snnz [Rc] (int)
//   sval [cap][Cs], scol [cap][Cs]  the CTA's rows of the band of C (if c_smem;
//                      staged once per problem, read every iteration; row
//                      stride Cs = ms_cstride(Rc))
//   ps [LC][Qs][Rc]    shifted directions (here, or in the CTA's scratch slice)
template <typename T, int LC>
__global__ void __launch_bounds__(kMsThreads, 1)
    k_mscg(const ProblemDev* __restrict__ tab, int count, int Rc, int dall, int Qs, int cap, int c_smem,
           int ps_smem, T* __restrict__ ps_scratch) {
  cg::cluster_group cluster = cg::this_cluster();
  const int CS = (int)cluster.num_blocks();
  const int crank = (int)cluster.block_rank();
  const int cl = blockIdx.x / CS, ncl = gridDim.x / CS;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  extern __shared__ __align__(16) unsigned char ms_dyn[];
  T* pfull = reinterpret_cast<T*>(ms_dyn);
  T* rv = pfull + (size_t)LC * dall;
  T* apv = rv + LC * Rc;
  T* ahi = apv + LC * Rc;
  T* alo = ahi + LC * Rc;
  T* pk = alo + LC * Rc;
  T* wqt = pk + 4 * LC * Qs;
  T* ratt = wqt + LC * Qs;
  T* zt = ratt + LC * Qs;
  double* zeta = reinterpret_cast<double*>(zt + LC * Qs);
  double* zprev = zeta + LC * Qs;
  double* delta = zprev + LC * Qs;
  double* wq = delta + LC * Qs;
  double* res = wq + LC * Qs;
  double* rat = res + LC * Qs;
  int* act = reinterpret_cast<int*>(rat + LC * Qs);
  int* itq = act + LC * Qs;
  int* lst = itq + LC * Qs;
  int* snnz = lst + 2 * LC * Qs;
  T* sval = reinterpret_cast<T*>(snnz + Rc);
  const int Cs = ms_cstride(Rc);
  int32_t* scol = reinterpret_cast<int32_t*>(sval + (c_smem ? (size_t)cap * Cs : 0));
  T* ps_s = reinterpret_cast<T*>(scol + (c_smem ? (size_t)cap * Cs : 0));
  T* ps_g = ps_scratch ? ps_scratch + (size_t)blockIdx.x * LC * Qs * Rc : nullptr;

  __shared__ double s_red_pap[kMsMaxCS * kMsMaxLC];
  __shared__ double s_red_rr[kMsMaxCS * kMsMaxLC];
  __shared__ float s_wff[kMsWarps][kMsMaxLC][2];
  __shared__ double s_wdd[kMsWarps][kMsMaxLC];
  __shared__ double s_rr[2][LC], s_alpha[LC], s_aprev[LC], s_bprev[LC], s_beta[LC];
  // the FP32 path keeps the CG scalars of the shifted recurrences as
  // float-float pairs (about 48 bits) and issues no FP64 instruction per step
  __shared__ float2 s_alpha2[LC], s_aprev2[LC], s_bprev2[LC], s_beta2[LC];
  __shared__ double s_bn[LC], s_sig0[LC], s_stop[LC];
  __shared__ float s_stop_f[LC];
  __shared__ float s_rrh[2][LC], s_rrl[2][LC];   // r^T r as float-float, this step's and the next
  __shared__ T s_alpha_t[LC], s_beta_t[LC];
  __shared__ int s_live[LC], s_done[LC], s_qc[LC], s_mem[LC], s_k[LC];
  __shared__ int s_nact[2][LC];
  __shared__ int s_cprob;   // problem whose rows of C are staged
  __shared__ unsigned s_needs[kMsMaxCS];   // bit s of entry c: CTA c's rows read slice s of p
  __shared__ unsigned s_need, s_pushmask;  // slices this CTA reads; CTAs that read its slice
  if (tid == 0) s_cprob = -1;

  const int sub = ms_sub(Rc);

  int G = 0;
  for (int p = 0; p < count; ++p) G += (chains_of(tab[p]) + LC - 1) / LC;

  for (int g = cl; g < G; g += ncl) {
    int p = 0, gb = 0, nch = 0;
    for (; p < count; ++p) {
      nch = chains_of(tab[p]);
      const int ng = (nch + LC - 1) / LC;
      if (g < gb + ng) break;
      gb += ng;
    }
    const ProblemDev& pr = tab[p];
    const int c0 = (g - gb) * LC;
    const int d = (int)pr.d;
    const int64_t N = pr.N, N1 = pr.N + 1;
    const int r0 = crank * Rc;
    const int nrows = max(0, min(d - r0, Rc));
    const bool fixed = pr.fixed_iters > 0;
    const int limit = fixed ? pr.fixed_iters : pr.max_iter;

    if (tid < LC) {
      const int c = c0 + tid;
      const bool live = c < nch;
      const bool mean = live && pr.do_mean && c == 0;
      s_live[tid] = live;
      s_mem[tid] = live ? (mean ? -1 : c - pr.do_mean) : -2;
      s_qc[tid] = live ? (mean ? 1 : pr.Q) : 0;
      double sg0 = 1.0;
      if (live && !mean) {
        sg0 = pr.s[0] + 1.0;
        for (int q = 1; q < pr.Q; ++q) sg0 = fmin(sg0, pr.s[q] + 1.0);
      }
      s_sig0[tid] = sg0;
      s_aprev[tid] = 1.0;
      s_bprev[tid] = 0.0;
      s_aprev2[tid] = make_float2(1.f, 0.f);
      s_bprev2[tid] = make_float2(0.f, 0.f);
      s_k[tid] = 0;
    }
    __syncthreads();

    // the CTA's rows of the band of C, once per problem
    if (s_cprob != p) {
      const T* __restrict__ gv = reinterpret_cast<const T*>(pr.oo_val);
      const int cp = (int)pr.max_oo;
      for (int row = tid; row < Rc; row += kMsThreads) snnz[row] = row < nrows ? pr.oo_nnz[r0 + row] : 0;
      if (c_smem) {
        for (int idx = tid; idx < cp * Rc; idx += kMsThreads) {
          const int e = idx / Rc, row = idx % Rc;
          if (row < nrows) {
            sval[e * Cs + row] = gv[(int64_t)e * d + r0 + row];
            scol[e * Cs + row] = pr.oo_col[(int64_t)e * d + r0 + row];
          }
        }
      }
      // which slices of p the own rows of C read, and so which CTAs need this
      // CTA's slice after each update (on a 1-D band: itself and its neighbours)
      if (tid == 0) s_need = 1u << crank;
      __syncthreads();
      unsigned need = 0;
      for (int idx = tid; idx < cp * Rc; idx += kMsThreads) {
        const int e = idx / Rc, row = idx % Rc;
        if (row < nrows && e < snnz[row]) need |= 1u << (pr.oo_col[(int64_t)e * d + r0 + row] / Rc);
      }
      if (need) atomicOr(&s_need, need);
      __syncthreads();
      if (tid < CS) cluster.map_shared_rank(s_needs, tid)[crank] = s_need;
      cluster.sync();
      if (tid == 0) {
        unsigned m = 0;
        for (int c = 0; c < CS; ++c) m |= (s_needs[c] >> crank & 1u) << c;
        s_pushmask = m;
      }
    }
    // p_0 = b for every chain, in full: b = R^-1/2 w^(i), or R^-1/2 (y - H mu)
    const T* W = reinterpret_cast<const T*>(pr.W);
    for (int idx = tid; idx < LC * dall; idx += kMsThreads) {
      const int j = idx / dall, a = idx % dall;
      const int m = s_mem[j];
      T v = T(0);
      if (a < d && m >= -1) v = m == -1 ? to_t<T>(pr.bmean[a]) : to_t<T>(pr.rinv[a]) * W[(int64_t)a * N + m];
      pfull[idx] = v;
    }
    __syncthreads();
    {
      DotAcc<T> bb[LC];
      T* psb = ps_smem ? ps_s : ps_g;
      for (int idx = tid; idx < LC * Rc; idx += kMsThreads) {
        const int j = idx / Rc, row = idx % Rc;
        const T v = row < nrows ? pfull[(size_t)j * dall + r0 + row] : T(0);
        rv[idx] = v;
        apv[idx] = T(0);
        ahi[idx] = T(0);
        alo[idx] = T(0);
        T* psj = psb + (size_t)j * Qs * Rc + row;
        for (int q = 0; q < s_qc[j]; ++q) psj[(size_t)q * Rc] = v;
#pragma unroll
        for (int jj = 0; jj < LC; ++jj)
          if (jj == j) bb[jj].add_prod(v, v);
      }
      ms_push_partials<T, LC>(bb, s_red_rr, s_wff, s_wdd, cluster, CS, crank);
    }
    if (tid < LC) {
      double rr;
      if constexpr (sizeof(T) == 4) {
        const FF f = ms_sum_ff(s_red_rr, CS, LC, tid);
        s_rrh[0][tid] = f.h;
        s_rrl[0][tid] = f.l;
        rr = ff_to_d(f);
      } else {
        rr = ms_sum_d(s_red_rr, CS, LC, tid);
      }
      const double bn = sqrt(rr);
      s_rr[0][tid] = rr;
      s_bn[tid] = bn;
      s_stop[tid] = (fixed ? 1e-30 : pr.tol) * bn;
      s_stop_f[tid] = (float)s_stop[tid];
      const bool on = s_live[tid] && bn > 0.0;
      s_done[tid] = !on;
      s_nact[0][tid] = on ? s_qc[tid] : 0;
    }
    __syncthreads();
    for (int idx = tid; idx < LC * Qs; idx += kMsThreads) {
      const int j = idx / Qs, q = idx % Qs;
      const bool has = q < s_qc[j];
      double sg = 1.0, w = 1.0;
      if (has && s_mem[j] >= 0) {
        sg = pr.s[q] + 1.0;
        w = pr.p[q];
      }
      if constexpr (sizeof(T) == 4) {
        const FF dl = ff_from(sg - s_sig0[j]);
        reinterpret_cast<float2*>(zeta)[idx] = make_float2(1.f, 0.f);
        reinterpret_cast<float2*>(zprev)[idx] = make_float2(1.f, 0.f);
        reinterpret_cast<float2*>(delta)[idx] = make_float2(dl.h, dl.l);
      } else {
        zeta[idx] = 1.0;
        zprev[idx] = 1.0;
        delta[idx] = sg - s_sig0[j];
      }
      wq[idx] = w;
      wqt[idx] = to_t<T>(w);
      res[idx] = (has && s_bn[j] > 0.0) ? s_bn[j] : 0.0;
      act[idx] = has && !s_done[j];
      itq[idx] = 0;
      lst[idx] = q;   // buffer 0: every shift of a live chain, in order
    }
    __syncthreads();

    T sg0[LC];
#pragma unroll
    for (int j = 0; j < LC; ++j) sg0[j] = to_t<T>(s_sig0[j]);
    const T* __restrict__ cval = reinterpret_cast<const T*>(pr.oo_val);
    const int32_t* __restrict__ ccol = pr.oo_col;
    const unsigned pushmask = s_pushmask;
    int buf = 0;

    for (;;) {
      // identical on every CTA: the flags come from identical scalars
      unsigned step = 0;
#pragma unroll
      for (int j = 0; j < LC; ++j) step |= (s_done[j] == 0 ? 1u : 0u) << j;
      if (step == 0) break;
      const int* nact = s_nact[buf];
      const int* lcur = lst + buf * LC * Qs;

      // q = (C + sigma_0 I) p over the own rows, and the partials of p^T q
      DotAcc<T> pap[LC];
      const int rows_per_pass = kMsThreads / sub;
      for (int base = 0; base < nrows; base += rows_per_pass) {
        const int rl = base + tid / sub, part = tid % sub;
        const bool valid = rl < nrows;
        const int a = r0 + rl;
        T y[LC];
#pragma unroll
        for (int j = 0; j < LC; ++j) y[j] = T(0);
        const int nnz = valid ? snnz[rl] : 0;
        if (c_smem) {
#pragma unroll 8
          for (int e = part; e < nnz; e += sub) {
            const T v = sval[e * Cs + rl];
            const int c = scol[e * Cs + rl];
#pragma unroll
            for (int j = 0; j < LC; ++j) y[j] = fma(v, pfull[(size_t)j * dall + c], y[j]);
          }
        } else {
#pragma unroll 8
          for (int e = part; e < nnz; e += sub) {
            const T v = __ldg(cval + (int64_t)e * d + a);
            const int c = __ldg(ccol + (int64_t)e * d + a);
#pragma unroll
            for (int j = 0; j < LC; ++j) y[j] = fma(v, pfull[(size_t)j * dall + c], y[j]);
          }
        }
        for (int o = sub >> 1; o > 0; o >>= 1) {
#pragma unroll
          for (int j = 0; j < LC; ++j) y[j] += __shfl_xor_sync(0xffffffffu, y[j], o);
        }
        if (valid && part == 0) {
#pragma unroll
          for (int j = 0; j < LC; ++j) {
            const T pa = pfull[(size_t)j * dall + a];
            const T yy = fma(sg0[j], pa, y[j]);
            apv[j * Rc + rl] = yy;
            if (step >> j & 1u) pap[j].add_prod(pa, yy);
          }
        }
      }
      ms_push_partials<T, LC>(pap, s_red_pap, s_wff, s_wdd, cluster, CS, crank);   // (1)

      // alpha = r^T r / p^T q
      if (tid < LC && (step >> tid & 1u)) {
        bool bad;
        double al = 0.0;
        if constexpr (sizeof(T) == 4) {
          const FF pq = ms_sum_ff(s_red_pap, CS, LC, tid);
          bad = !(pq.h > 0.f) || !isfinite(pq.h);
          if (!bad) {
            const FF a = ff_div(FF{s_rrh[buf][tid], s_rrl[buf][tid]}, pq);
            s_alpha2[tid] = make_float2(a.h, a.l);
            s_alpha_t[tid] = a.h + a.l;
          }
        } else {
          const double pq = ms_sum_d(s_red_pap, CS, LC, tid);
          bad = !(pq > 0.0) || !isfinite(pq);
          if (!bad) {
            al = s_rr[buf][tid] / pq;
            s_alpha_t[tid] = to_t<T>(al);
          }
        }
        if (bad) {
          s_done[tid] = 2;   // breakdown
          s_alpha_t[tid] = T(0);
        }
        s_alpha[tid] = al;
      }
      __syncthreads();
      step = 0;
#pragma unroll
      for (int j = 0; j < LC; ++j) step |= (s_done[j] == 0 ? 1u : 0u) << j;

      DotAcc<T> rra[LC];
      if (warp < kMsZetaWarps) {
        // zeta_{k+1} / zeta_k of every active shift (FP64, or float-float on
        // the FP32 path)
        int tot = 0;
#pragma unroll
        for (int j = 0; j < LC; ++j) tot += (step >> j & 1u) ? nact[j] : 0;
        for (int t = tid; t < tot; t += kMsZetaWarps * 32) {
          int off;
          const int j = ms_locate<LC>(t, step, nact, off);
          const int idx = j * Qs + lcur[j * Qs + off];
          if constexpr (sizeof(T) == 4) {
            const float2 z0v = reinterpret_cast<const float2*>(zeta)[idx];
            const float2 zmv = reinterpret_cast<const float2*>(zprev)[idx];
            const float2 dv = reinterpret_cast<const float2*>(delta)[idx];
            const FF z0{z0v.x, z0v.y}, zm{zmv.x, zmv.y}, dl{dv.x, dv.y};
            const FF al{s_alpha2[j].x, s_alpha2[j].y}, ap{s_aprev2[j].x, s_aprev2[j].y};
            const FF bp{s_bprev2[j].x, s_bprev2[j].y};
            const FF A = ff_mul(zm, ap);
            const FF den = ff_add(ff_mul(ff_mul(al, bp), ff_sub(zm, z0)),
                                  ff_mul(A, ff_add(FF{1.f, 0.f}, ff_mul(dl, al))));
            const FF ratio = ff_div(A, den);
            const FF z1 = ff_mul(z0, ratio);
            ratt[idx] = ratio.h + ratio.l;
            zt[idx] = z1.h + z1.l;
            reinterpret_cast<float2*>(zprev)[idx] = z0v;
            reinterpret_cast<float2*>(zeta)[idx] = make_float2(z1.h, z1.l);
          } else {
            const double z0 = zeta[idx], zm = zprev[idx];
            const double al = s_alpha[j], ap = s_aprev[j], bp = s_bprev[j];
            const double ratio = zm * ap / (al * bp * (zm - z0) + zm * ap * (1.0 + delta[idx] * al));
            const double z1 = z0 * ratio;
            rat[idx] = ratio;
            ratt[idx] = to_t<T>(ratio);
            zt[idx] = to_t<T>(z1);
            zprev[idx] = z0;
            zeta[idx] = z1;
          }
        }
      } else {
        // r <- r - alpha q and the partials of r^T r
        T alpha_t[LC];
#pragma unroll
        for (int j = 0; j < LC; ++j) alpha_t[j] = s_alpha_t[j];
        for (int idx = tid - kMsZetaWarps * 32; idx < LC * Rc; idx += kMsThreads - kMsZetaWarps * 32) {
          const int j = idx / Rc;
          if (!(step >> j & 1u)) continue;
          T al = T(0);
#pragma unroll
          for (int jj = 0; jj < LC; ++jj)
            if (jj == j) al = alpha_t[jj];
          const T rn = fma(-al, apv[idx], rv[idx]);
          rv[idx] = rn;
#pragma unroll
          for (int jj = 0; jj < LC; ++jj)
            if (jj == j) rra[jj].add_prod(rn, rn);
        }
      }
      ms_push_partials<T, LC>(rra, s_red_rr, s_wff, s_wdd, cluster, CS, crank);   // (2)

      // beta = r'^T r' / r^T r and ||r'||, formed from the same partials by the
      // chain's owner (lane 0 of warp kMsWarps - 1 - j, which has no shift to
      // update while there are at most 32 (kMsWarps - LC) active shifts) and by
      // every thread of an active shift; then the packed coefficients, the
      // stopping test and the iteration count of every active shift
      {
        const int nb = buf ^ 1;
        const int jo = kMsWarps - 1 - warp;
        if (lane == 0 && jo >= 0 && jo < LC && (step >> jo & 1u)) {
          if constexpr (sizeof(T) == 4) {
            const FF rn = ms_sum_ff(s_red_rr, CS, LC, jo);
            const FF b = ff_div(rn, FF{s_rrh[buf][jo], s_rrl[buf][jo]});
            s_beta2[jo] = make_float2(b.h, b.l);
            s_beta_t[jo] = b.h + b.l;
            s_rrh[nb][jo] = rn.h;
            s_rrl[nb][jo] = rn.l;
          } else {
            double bd, srr;
            T bt;
            ms_beta<T>(s_red_rr, CS, LC, jo, s_rrh[buf][jo], s_rrl[buf][jo], s_rr[buf][jo], bd, bt, srr,
                       s_rrh[nb][jo], s_rrl[nb][jo], s_rr[nb][jo]);
            s_beta[jo] = bd;
            s_beta_t[jo] = bt;
          }
        }
        int tot = 0;
#pragma unroll
        for (int j = 0; j < LC; ++j) tot += (step >> j & 1u) ? nact[j] : 0;
        for (int t = tid; t < tot; t += kMsThreads) {
          int off;
          const int j = ms_locate<LC>(t, step, nact, off);
          const int q = lcur[j * Qs + off], idx = j * Qs + q;
          T* e = pk + 4 * (j * Qs + off);
          itq[idx] = s_k[j] + 1;
          if constexpr (sizeof(T) == 4) {
            // FP32 coefficients of FP32 vectors: no FP64 instruction here
            const FF rn = ms_sum_ff(s_red_rr, CS, LC, j);
            const FF b = ff_div(rn, FF{s_rrh[buf][j], s_rrl[buf][j]});
            const FF sr = rn.h > 0.f ? ff_mul(rn, ff_rsqrt(rn)) : FF{0.f, 0.f};
            const float bt = b.h + b.l, ra = ratt[idx];
            e[0] = wqt[idx] * s_alpha_t[j] * ra;
            e[1] = zt[idx];
            e[2] = bt * ra * ra;
            e[3] = ms_q_bits<T>(q);
            const float rq = fabsf(zt[idx]) * (sr.h + sr.l);
            res[idx] = (double)rq;
            if (!(rq > s_stop_f[j])) act[idx] = 0;
          } else {
            double bd, srr, rd;
            T bt;
            float rh, rl;
            ms_beta<T>(s_red_rr, CS, LC, j, s_rrh[buf][j], s_rrl[buf][j], s_rr[buf][j], bd, bt, srr, rh, rl, rd);
            const double ratio = rat[idx];
            e[0] = to_t<T>(wq[idx] * s_alpha[j] * ratio);
            e[1] = to_t<T>(zeta[idx]);
            e[2] = to_t<T>(bd * ratio * ratio);
            e[3] = ms_q_bits<T>(q);
            const double rq = fabs(zeta[idx]) * srr;
            res[idx] = rq;
            if (!(rq > s_stop[j])) act[idx] = 0;
          }
        }
      }
      __syncthreads();

      // next step's active lists and the chain bookkeeping (read again only
      // after barrier (3)): chain j by warp kMsWarps - 1 - j, the warps with the
      // least update work; everyone else goes straight to the update
      {
        const int j = kMsWarps - 1 - warp;
        if (j >= 0 && j < LC && (step >> j & 1u)) {
          const int nb = buf ^ 1;
          int n = 0;
          for (int q0 = 0; q0 < s_qc[j]; q0 += 32) {
            const int q = q0 + lane;
            const bool a = q < s_qc[j] && act[j * Qs + q];
            const unsigned m = __ballot_sync(0xffffffffu, a);
            if (a) lst[(nb * LC + j) * Qs + n + __popc(m & ((1u << lane) - 1u))] = q;
            n += __popc(m);
          }
          if (lane == 0) {
            s_nact[nb][j] = n;
            s_aprev[j] = s_alpha[j];
            s_bprev[j] = s_beta[j];
            s_aprev2[j] = s_alpha2[j];
            s_bprev2[j] = s_beta2[j];
            s_k[j] += 1;
            if (n == 0 || s_k[j] >= limit) s_done[j] = 1;
          }
        }
      }

      // shifted directions, quadrature sum, base direction, and its exchange
      T beta_t[LC];
#pragma unroll
      for (int j = 0; j < LC; ++j) beta_t[j] = s_beta_t[j];
      // four consecutive rows of one chain per thread: 16-byte (FP32) accesses
      // to r, the shifted directions, the quadrature sums and p, four
      // independent FMA chains, and p pushed without a gather
      auto update = [&](T* psb) {
        const int R4 = Rc / 4;
        for (int it = tid; it < LC * R4; it += kMsThreads) {
          const int j = it / R4, row = (it % R4) * 4;
          if (!(step >> j & 1u)) continue;
          const int idx = j * Rc + row;
          T rn[4], sum[4] = {T(0), T(0), T(0), T(0)};
          ms_ld4(rv + idx, rn);
          T* pc = psb + (size_t)j * Qs * Rc + row;
          const T* ej = pk + 4 * j * Qs;
          const int n = nact[j];
          int i = 0;
          for (; i + 2 <= n; i += 2) {
            T c0[4], c1[4], p0[4], p1[4];
            ms_ld4(ej + 4 * i, c0);
            ms_ld4(ej + 4 * i + 4, c1);
            T* a0 = pc + (size_t)ms_q_of(c0[3]) * Rc;
            T* a1 = pc + (size_t)ms_q_of(c1[3]) * Rc;
            ms_ld4(a0, p0);
            ms_ld4(a1, p1);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
              sum[r] = fma(c0[0], p0[r], sum[r]);
              sum[r] = fma(c1[0], p1[r], sum[r]);
              p0[r] = fma(c0[1], rn[r], c0[2] * p0[r]);
              p1[r] = fma(c1[1], rn[r], c1[2] * p1[r]);
            }
            ms_st4(a0, p0);
            ms_st4(a1, p1);
          }
          if (i < n) {
            T c0[4], p0[4];
            ms_ld4(ej + 4 * i, c0);
            T* a0 = pc + (size_t)ms_q_of(c0[3]) * Rc;
            ms_ld4(a0, p0);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
              sum[r] = fma(c0[0], p0[r], sum[r]);
              p0[r] = fma(c0[1], rn[r], c0[2] * p0[r]);
            }
            ms_st4(a0, p0);
          }
          T hi[4], lo[4], pn[4];
          ms_ld4(ahi + idx, hi);
          ms_ld4(alo + idx, lo);
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            if constexpr (sizeof(T) == 4) {
              float sh, e;
              two_sum(hi[r], sum[r], sh, e);
              hi[r] = sh;
              lo[r] += e;
            } else {
              hi[r] += sum[r];
            }
          }
          ms_st4(ahi + idx, hi);
          ms_st4(alo + idx, lo);
          T bt = T(0);
#pragma unroll
          for (int jj = 0; jj < LC; ++jj)
            if (jj == j) bt = beta_t[jj];
          T* pf = pfull + (size_t)j * dall + r0 + row;
          ms_ld4(pf, pn);
#pragma unroll
          for (int r = 0; r < 4; ++r) pn[r] = fma(bt, pn[r], rn[r]);
          for (int c = 0; c < CS; ++c)
            if (pushmask >> c & 1u) ms_st4(c == crank ? pf : cluster.map_shared_rank(pf, c), pn);
        }
      };
      if (ps_smem) update(ps_s);
      else update(ps_g);
      cluster.sync();   // (3)
      buf ^= 1;
    }

    // vbar = R^-1/2 sum_q p_q u_q (FP64) for the state update
    for (int idx = tid; idx < LC * Rc; idx += kMsThreads) {
      const int j = idx / Rc, row = idx % Rc;
      if (!s_live[j] || row >= nrows) continue;
      const int a = r0 + row;
      const int64_t m = s_mem[j] == -1 ? N : (int64_t)s_mem[j];
      const double u = (double)ahi[idx] + (double)alo[idx];
      const double v = pr.rinv[a] * u;
      pr.Vbar[(int64_t)a * N1 + m] = v;
      reinterpret_cast<T*>(pr.VbarT)[(int64_t)a * N1 + m] = to_t<T>(v);
    }
    if (crank == 0) {
      for (int idx = tid; idx < LC * Qs; idx += kMsThreads) {
        const int j = idx / Qs, q = idx % Qs;
        if (!s_live[j] || q >= s_qc[j]) continue;
        const int64_t sid = s_mem[j] == -1 ? 0 : pr.mean_sys + (int64_t)q * N + s_mem[j];
        pr.iters[sid] = itq[idx];
        pr.relres[sid] = s_bn[j] > 0.0 ? res[idx] / s_bn[j] : 0.0;
        if (act[idx] && !fixed) atomicOr(&pr.status[0], kStatNotConverged);
      }
      if (tid < LC && s_done[tid] == 2) atomicOr(&pr.status[0], kStatBreakdown);
      if (tid == 0) atomicOr(&pr.status[1], 2);
    }
    if (tid == 0) s_cprob = p;
    __syncthreads();
  }
  cluster.sync();   // no CTA leaves while another may still write to its shared memory
}

int mscg_plan(const ProblemTable& tab, int num_sms, int requested_cs, MsPlan* out) {
  int64_t dmax = 1, cap = 1;
  int qmax = 1;
  for (int i = 0; i < tab.count; ++i) {
    const ProblemDev& p = tab.p[i];
    dmax = p.d > dmax ? p.d : dmax;
    cap = p.max_oo > cap ? p.max_oo : cap;
    if (p.do_pert) qmax = p.Q > qmax ? p.Q : qmax;
  }
  int CS = requested_cs > 0 ? requested_cs : kMsMaxCS;
  if (requested_cs <= 0)
    while (CS > 1 && (dmax + CS - 1) / CS < 64) CS >>= 1;
  if (CS > num_sms) CS = 1;
  MsPlan pl;
  memset(&pl, 0, sizeof(pl));
  pl.CS = CS;
  pl.Rc = (int)((((dmax + CS - 1) / CS) + 3) / 4 * 4);
  pl.dall = CS * pl.Rc;
  pl.Qs = (qmax + 3) / 4 * 4;
  pl.cap = (int)cap;
  pl.esz = tab.p[0].precision == 0 ? 8 : 4;
  // the slice of C (read every iteration by every thread) before the shifted
  // directions (one read and one write per active shift)
  const bool order[4][2] = {{true, true}, {true, false}, {false, true}, {false, false}};
  for (int lc = 1; lc <= kMsMaxLC; ++lc) {
    for (int o = 0; o < 4; ++o) {
      const size_t b = ms_dyn_bytes(lc, pl.Rc, pl.dall, pl.Qs, pl.cap, pl.esz, order[o][0], order[o][1]);
      if (b <= kMsSmemBudget) {
        pl.c_smem[lc] = order[o][0];
        pl.ps_smem[lc] = order[o][1];
        pl.dyn[lc] = b;
        pl.LCmax = lc;
        if (!order[o][1]) {
          const size_t sb = (size_t)num_sms * lc * pl.Qs * pl.Rc * pl.esz;
          pl.scratch_bytes = sb > pl.scratch_bytes ? sb : pl.scratch_bytes;
        }
        break;
      }
    }
  }
  if (!pl.LCmax) return -1;
  *out = pl;
  return 0;
}

namespace {

// Co-resident clusters per (device, instantiation, cluster size, dynamic
// bytes), looked up once per host thread; the function attribute is raised to
// the largest dynamic size the plan can ask for on first use.
struct MsOcc {
  int dev, esz, LC, CS;
  size_t dyn;
  int clusters;
};

template <typename T, int LC>
int ms_max_clusters(int CS, size_t dyn) {
  constexpr int kMaxDev = 64;
  static thread_local MsOcc cache[32];
  static thread_local int ncache = 0;
  static thread_local bool attr_set[kMaxDev] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
    cudaGetLastError();
    return -1;
  }
  for (int i = 0; i < ncache; ++i) {
    const MsOcc& c = cache[i];
    if (c.dev == dev && c.esz == (int)sizeof(T) && c.LC == LC && c.CS == CS && c.dyn == dyn) return c.clusters;
  }
  if (!attr_set[dev]) {
    if (cudaFuncSetAttribute(k_mscg<T, LC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMsSmemBudget) !=
        cudaSuccess) {
      cudaGetLastError();
      return -1;
    }
    attr_set[dev] = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CS, 1, 1);
  cfg.blockDim = dim3(kMsThreads, 1, 1);
  cfg.dynamicSmemBytes = dyn;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int mc = 0;
  if (cudaOccupancyMaxActiveClusters(&mc, k_mscg<T, LC>, &cfg) != cudaSuccess || mc < 1) {
    cudaGetLastError();
    mc = -1;
  }
  MsOcc& e = cache[ncache < 32 ? ncache++ : 31];
  e = MsOcc{dev, (int)sizeof(T), LC, CS, dyn, mc};
  return mc;
}

template <typename T, int LC>
int ms_launch(const ProblemTable& tab, const ProblemDev* dtab, const MsPlan& pl, int clusters, size_t dyn,
              cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(clusters * pl.CS, 1, 1);
  cfg.blockDim = dim3(kMsThreads, 1, 1);
  cfg.dynamicSmemBytes = dyn;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = pl.CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  T* scratch = reinterpret_cast<T*>(tab.ms_scratch);
  if (!pl.ps_smem[LC] && !scratch) return -1;
  if (cudaLaunchKernelEx(&cfg, k_mscg<T, LC>, dtab, (int)tab.count, pl.Rc, pl.dall, pl.Qs, pl.cap,
                         pl.c_smem[LC], pl.ps_smem[LC], scratch) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  note_launches(1);
  return 0;
}

template <typename T>
int ms_dispatch(const ProblemTable& tab, const ProblemDev* dtab, const MsPlan& pl, int num_sms, cudaStream_t st) {
  // the smallest chain group that still fits one wave of co-resident clusters
  int pick = 0, clusters = 0;
  size_t dyn = 0;
  for (int lc = 1; lc <= pl.LCmax; ++lc) {
    if (!pl.dyn[lc]) continue;
    const size_t b = pl.dyn[lc];
    int mc = lc == 1 ? ms_max_clusters<T, 1>(pl.CS, b)
             : lc == 2 ? ms_max_clusters<T, 2>(pl.CS, b)
             : lc == 3 ? ms_max_clusters<T, 3>(pl.CS, b)
                       : ms_max_clusters<T, 4>(pl.CS, b);
    if (mc < 1) continue;
    if (mc > num_sms / pl.CS) mc = num_sms / pl.CS;
    if (mc < 1) continue;
    int groups = 0;
    for (int i = 0; i < tab.count; ++i) groups += (chains_of(tab.p[i]) + lc - 1) / lc;
    pick = lc;
    dyn = b;
    clusters = groups < mc ? groups : mc;
    if (groups <= mc) break;
  }
  if (!pick || clusters < 1) return -1;
  switch (pick) {
    case 1: return ms_launch<T, 1>(tab, dtab, pl, clusters, dyn, st);
    case 2: return ms_launch<T, 2>(tab, dtab, pl, clusters, dyn, st);
    case 3: return ms_launch<T, 3>(tab, dtab, pl, clusters, dyn, st);
    default: return ms_launch<T, 4>(tab, dtab, pl, clusters, dyn, st);
  }
}

}  // namespace

int launch_mscg(const ProblemTable& tab, const ProblemDev* dtab, const MsPlan& pl, int num_sms, cudaStream_t st) {
  return tab.p[0].precision == 0 ? ms_dispatch<double>(tab, dtab, pl, num_sms, st)
                                 : ms_dispatch<float>(tab, dtab, pl, num_sms, st);
}

}  // namespace infoesrf
