// a4 for the FP32 path in one launch: the randomized Ritz pairs of C (App. E;
// Halko, Martinsson & Tropp Alg. 5.3) by one thread-block cluster per problem.
//
// The multi-kernel sequence (test matrix, band matvecs, CholeskyQR2 passes,
// Rayleigh-Ritz, vectors, Gram matrices) is a chain of a dozen short
// kernels whose launch boundaries cost as much as their work.  Here CTA c of
// the cluster owns rows [c R, (c+1) R) of the d x l blocks: it forms its rows
// of Omega and of every product C X (X read from global memory, which stays
// in L2), its float-float partial Gram matrices, and its rows of every
// triangular solve.  Partial Grams are combined through distributed shared
// memory in rank order, and every CTA factors the same Gram matrix, so all
// CTAs hold identical factors without another exchange.  Cluster barriers
// (release/acquire at cluster scope) order the global-memory phases.
//
// Same outputs as the multi-kernel path: Phi, C Phi, theta, the Gram matrices
// of Phi and C Phi (pr.gram), and ev / Rm / Gm for the stage exports.
#include <cooperative_groups.h>
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "info_esrf.h"
#include "internal.h"

namespace cg = cooperative_groups;

namespace infoesrf {

namespace {
constexpr int kRC = 8;                              // CTAs per cluster (at most)
constexpr int kRT = 512;                            // threads per CTA (128 registers each)
constexpr int kRW = kRT / 32;
constexpr int kRL = kMaxRitz;                       // columns l <= 32
constexpr int kRTmp = 1024;                         // (entry, chunk) partials
constexpr int kRParts = 4;                          // threads per row in the band product
constexpr int kRMaxRows = kRT / kRParts;            // own rows per CTA (128)
constexpr size_t kRStageBytes = 144 * 1024;         // shared staging of a full d x l block
// Phase clocks (built only with -DINFO_ESRF_PHASE_CLOCKS, a separate build of
// the library): thread 0 of cluster rank 0 sums clock64() deltas per stage
// and adds them, with a launch count, into g_ritz_phase at exit;
// info_esrf_ritz_phase_clocks reads them.
constexpr int kRitzPhases = 10;
}  // namespace
#ifdef INFO_ESRF_PHASE_CLOCKS
__device__ unsigned long long g_ritz_phase[kRitzPhases + 1];
#define RITZ_PHASE(i)                 \
  if (tid == 0 && crank == 0) {       \
    const long long now_ = clock64(); \
    ph_c[i] += now_ - ph_t;           \
    ph_t = now_;                      \
  }
#else
#define RITZ_PHASE(i)
#endif

// Whether the fused kernel takes a problem: the whole d x l block must fit the
// shared staging area and the own rows of a CTA one pass of the band product.
bool ritz_cluster_fits(int64_t d, int l) {
  return (size_t)d * (size_t)l * 4 <= kRStageBytes && (d + kRC - 1) / kRC <= kRMaxRows;
}

__global__ void __launch_bounds__(kRT, 1) k_ritz_cluster(const ProblemDev* tab) {
  extern __shared__ __align__(16) float xs[];      // full d x l staging (gathers of the band product)
  cg::cluster_group cluster = cg::this_cluster();
  const int CS = (int)cluster.num_blocks();
  const int crank = (int)cluster.block_rank();
  const ProblemDev& pr = tab[blockIdx.x / CS];
  const int l = pr.l, k = pr.kR;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t d = pr.d;
  const int64_t R = (d + CS - 1) / CS;
  const int64_t r0 = (int64_t)crank * R < d ? (int64_t)crank * R : d;
  const int64_t r1 = r0 + R < d ? r0 + R : d;
  const int nrow = (int)(r1 - r0);
  float* buf[2] = {reinterpret_cast<float*>(pr.Om), reinterpret_cast<float*>(pr.Yb)};
  const float* val = reinterpret_cast<const float*>(pr.oo_val);

  __shared__ float Gp_h[kRTmp], Gp_l[kRTmp];        // this CTA's partial Gram (float-float)
  __shared__ float Tp_h[kRTmp], Tp_l[kRTmp];        // (entry, chunk) scratch
  __shared__ FF G[kRL][kRL + 1];                    // merged Gram (upper triangle)
  __shared__ float Rt[kRL][kRL + 1], rinv[kRL];
  __shared__ float ys[kRMaxRows][kRL + 1];          // own rows of the working block
  __shared__ float zs[kRMaxRows][kRL + 1];          // own rows of its image under C
  __shared__ float U[kRL][kRL + 1], V[kRL][kRL + 1], nrm[kRL], lam[kRL];
  __shared__ int8_t pair_p[kRL][kRL / 2], pair_q[kRL][kRL / 2];
  __shared__ float Vk[kRL][kMaxK];
  __shared__ float s_scale, s_tiny, s_trw[kRW];
  if (l <= 0 || k <= 0) return;                     // uniform over the cluster
#ifdef INFO_ESRF_PHASE_CLOCKS
  long long ph_c[kRitzPhases] = {};
  long long ph_t = clock64();
#endif

  // ---- partial Gram of the own rows from shared memory: entries (i, j) of A^T B ----
  auto gram_partial = [&](const float (*A)[kRL + 1], const float (*Bm)[kRL + 1], int nc, bool sym) {
    const int nent = sym ? nc * (nc + 1) / 2 : nc * nc;
    int chunks = kRT / nent;
    if (chunks < 1) chunks = 1;
    if (chunks * nent > kRTmp) chunks = kRTmp / nent;
    for (int e = tid; e < nent * chunks; e += kRT) {
      const int ent = e / chunks, ch = e % chunks;
      int i, j;
      if (sym) {                                    // ent -> (i, j), i <= j, row-major upper triangle
        i = 0;
        int rem = ent;
        while (rem >= nc - i) { rem -= nc - i; ++i; }
        j = i + rem;
      } else {
        i = ent / nc;
        j = ent % nc;
      }
      DotAcc<float> acc;
      for (int a = ch; a < nrow; a += chunks) acc.add_prod(A[a][i], Bm[a][j]);
      Tp_h[e] = acc.hi;
      Tp_l[e] = acc.lo;
    }
    __syncthreads();
    for (int ent = tid; ent < nent; ent += kRT) {
      float h = 0.f, lo = 0.f;
      for (int ch = 0; ch < chunks; ++ch) ff_merge(h, lo, Tp_h[ent * chunks + ch], Tp_l[ent * chunks + ch]);
      Gp_h[ent] = h;
      Gp_l[ent] = lo;
    }
  };
  // ---- merge of the cluster's partials, in rank order (call after a cluster barrier) ----
  auto gram_merge = [&](int nent, float* out_h, float* out_l) {
    for (int ent = tid; ent < nent; ent += kRT) {
      float h[kRC], lo[kRC];
#pragma unroll
      for (int c = 0; c < kRC; ++c) {
        h[c] = c < CS ? cluster.map_shared_rank(Gp_h, c)[ent] : 0.f;
        lo[c] = c < CS ? cluster.map_shared_rank(Gp_l, c)[ent] : 0.f;
      }
      float sh = 0.f, sl = 0.f;
#pragma unroll
      for (int c = 0; c < kRC; ++c) ff_merge(sh, sl, h[c], lo[c]);
      out_h[ent] = sh;
      out_l[ent] = sl;
    }
  };
  // ---- own rows of C src into out (shared) and dst (global); src complete in global ----
  auto matvec = [&](const float* src, float* dst, float (*out)[kRL + 1]) {
    const int nv4 = (int)(d * l / 4);               // l * d is a multiple of 4 (checked at launch)
    for (int e = tid; e < nv4; e += kRT)
      reinterpret_cast<float4*>(xs)[e] = reinterpret_cast<const float4*>(src)[e];
    __syncthreads();
    const int row = tid / kRParts, part = tid % kRParts;
    float acc[kRL];
#pragma unroll
    for (int m = 0; m < kRL; ++m) acc[m] = 0.f;
    if (row < nrow) {
      const int64_t a = r0 + row;
      const int nnz = pr.oo_nnz[a];
      for (int e = part; e < nnz; e += kRParts) {
        const float c = val[(int64_t)e * d + a];
        const float* xr = xs + (int64_t)pr.oo_col[(int64_t)e * d + a] * l;   // 16-byte aligned (l % 4 == 0)
#pragma unroll
        for (int m4 = 0; m4 < kRL / 4; ++m4) {
          if (4 * m4 < l) {
            const float4 v = *reinterpret_cast<const float4*>(xr + 4 * m4);
            acc[4 * m4 + 0] = fmaf(c, v.x, acc[4 * m4 + 0]);
            acc[4 * m4 + 1] = fmaf(c, v.y, acc[4 * m4 + 1]);
            acc[4 * m4 + 2] = fmaf(c, v.z, acc[4 * m4 + 2]);
            acc[4 * m4 + 3] = fmaf(c, v.w, acc[4 * m4 + 3]);
          }
        }
      }
    }
#pragma unroll
    for (int m = 0; m < kRL; ++m) {
      acc[m] += __shfl_xor_sync(0xffffffffu, acc[m], 1);
      acc[m] += __shfl_xor_sync(0xffffffffu, acc[m], 2);
    }
    if (row < nrow) {
      for (int m = part; m < l; m += kRParts) {
        out[row][m] = acc[m];
        dst[(r0 + row) * l + m] = acc[m];
      }
    }
    __syncthreads();
  };
  // ---- one CholeskyQR pass on the own rows (ys): ys <- ys R^-1 (also to dst) ----
  auto cholqr_pass = [&](float* dst) {
    gram_partial(ys, ys, l, true);
    cluster.sync();                                  // partials complete
    gram_merge(l * (l + 1) / 2, Tp_h, Tp_l);
    __syncthreads();
    float tr = 0.f;
    for (int ent = tid; ent < l * (l + 1) / 2; ent += kRT) {
      int i = 0, rem = ent;
      while (rem >= l - i) { rem -= l - i; ++i; }
      G[i][i + rem] = FF{Tp_h[ent], Tp_l[ent]};
      if (rem == 0) tr += Tp_h[ent];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
    if (lane == 0) s_trw[warp] = tr;
    __syncthreads();
    if (tid == 0) {
      float t2 = 0.f;
      for (int w = 0; w < kRW; ++w) t2 += s_trw[w];
      s_tiny = 1e-28f * (t2 > 0.f ? t2 : 1.f);
    }
    __syncthreads();
    // right-looking Cholesky in float-float arithmetic: every thread forms the
    // pivot's reciprocal root itself, so one barrier per column suffices
    const float tiny = s_tiny;
    for (int j = 0; j < l; ++j) {
      const FF gjj = G[j][j];
      const bool ok = gjj.h > tiny;
      const FF inv = ok ? ff_rsqrt(gjj) : FF{0.f, 0.f};
      const int mrem = l - 1 - j;
      if (tid == 0) {
        const FF rjj = ff_mul(gjj, inv);
        Rt[j][j] = rjj.h + rjj.l;
        rinv[j] = inv.h + inv.l;
        if (!ok && crank == 0) atomicOr(&pr.status[0], kStatEigFail);
      }
      if (tid < j) Rt[j][tid] = 0.f;
      if (tid < mrem) {
        const FF r = ff_mul(G[j][j + 1 + tid], inv);
        Rt[j][j + 1 + tid] = r.h + r.l;
      }
      for (int e = tid; e < mrem * mrem; e += kRT) {
        const int c2 = j + 1 + e / mrem, c = j + 1 + e % mrem;
        if (c2 <= c) {
          const FF a2 = ff_mul(G[j][c2], inv), a1 = ff_mul(G[j][c], inv);
          G[c2][c] = ff_sub(G[c2][c], ff_mul(a2, a1));
        }
      }
      __syncthreads();
    }
    for (int a = tid; a < nrow; a += kRT) {
      float row[kRL];
#pragma unroll
      for (int j = 0; j < kRL; ++j) {
        if (j < l) {
          float t = ys[a][j];
#pragma unroll
          for (int i = 0; i < j; ++i) t = fmaf(-row[i], Rt[i][j], t);
          row[j] = t * rinv[j];
        } else {
          row[j] = 0.f;
        }
      }
#pragma unroll
      for (int j = 0; j < kRL; ++j)
        if (j < l) {
          ys[a][j] = row[j];
          dst[(r0 + a) * l + j] = row[j];
        }
    }
    cluster.sync();                                  // dst rows visible; partial reads done
  };

  // ---- test matrix (element (a, j) uses counter j d + a), own rows ----
  for (int e = tid; e < nrow * l; e += kRT) {
    const int64_t a = r0 + e / l;
    const int j = e % l;
    buf[0][a * l + j] = philox_normal_f(pr.seed, (uint64_t)j * (uint64_t)d + (uint64_t)a);
  }
  cluster.sync();
  RITZ_PHASE(0);
  matvec(buf[0], buf[1], ys);                        // Y = C Omega (own rows in ys)
  RITZ_PHASE(1);
  for (int it = 0; it < pr.power_iters; ++it) {
    cholqr_pass(buf[0]);
    RITZ_PHASE(2);
    cholqr_pass(buf[1]);                             // Q in ys and buf[1]
    RITZ_PHASE(3);
    matvec(buf[1], buf[0], ys);                      // C Q
    cluster.sync();
    RITZ_PHASE(1);
    // the next block lives in buf[0]; keep buf[1] as the spare
    float* t = buf[0]; buf[0] = buf[1]; buf[1] = t;
  }
  cholqr_pass(buf[0]);
  RITZ_PHASE(2);
  cholqr_pass(buf[1]);                               // basis Q: ys, buf[1]
  RITZ_PHASE(3);
  matvec(buf[1], buf[0], zs);                        // C Q: zs, buf[0]
  cluster.sync();
  RITZ_PHASE(4);
  // ---- Rayleigh-Ritz: B = Q^T (C Q), eigenpairs by one-sided Jacobi in CTA 0 ----
  gram_partial(ys, zs, l, false);
  cluster.sync();
  RITZ_PHASE(5);
  if (crank == 0) {
    gram_merge(l * l, Tp_h, Tp_l);
    __syncthreads();
    for (int e = tid; e < l * l; e += kRT) {
      const int i = e / l, c = e % l;
      pr.Gm[e] = (double)Tp_h[e] + (double)Tp_l[e];
      U[i][c] = 0.5f * ((Tp_h[e] + Tp_l[e]) + (Tp_h[c * l + i] + Tp_l[c * l + i]));
      V[i][c] = i == c ? 1.f : 0.f;
    }
    const int m = (l + 1) & ~1, npairs = m / 2;
    for (int e = tid; e < (m - 1) * npairs; e += kRT) {
      const int round = e / npairs, w = e % npairs;
      const int s1 = w, s2 = m - 1 - w;
      int p = s1 == 0 ? 0 : ((s1 - 1 + round) % (m - 1)) + 1;
      int q = ((s2 - 1 + round) % (m - 1)) + 1;
      if (p > q) { const int x = p; p = q; q = x; }
      pair_p[round][w] = (int8_t)p;
      pair_q[round][w] = (int8_t)q;
    }
    __syncthreads();
    for (int c = warp; c < l; c += kRW) {
      const float u = lane < l ? U[lane][c] : 0.f;
      float a = u * u;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      if (lane == 0) nrm[c] = a;
    }
    __syncthreads();
    if (tid == 0) {
      float mx = 0.f;
      for (int c = 0; c < l; ++c) mx = fmaxf(mx, nrm[c]);
      s_scale = mx;
    }
    __syncthreads();
    const float gabs = 2e-6f * s_scale;
    for (int sweep = 0; sweep < 4; ++sweep) {
      int busy = 0;
      for (int round = 0; round < m - 1; ++round) {
        for (int w = warp; w < npairs; w += kRW) {
          const int p = pair_p[round][w], q = pair_q[round][w];
          if (q >= l) continue;
          const float up = lane < l ? U[lane][p] : 0.f, uq = lane < l ? U[lane][q] : 0.f;
          float g = up * uq;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
          const float al = nrm[p], be = nrm[q];
          if (g == 0.f) continue;
          busy |= fabsf(g) > gabs && fabsf(g) > 1e-5f * sqrtf(al * be);
          const float zeta = __fdividef(be - al, 2.f * g);
          const float z2 = fmaf(zeta, zeta, 1.f);
          const float tt = copysignf(1.f, zeta) * __fdividef(1.f, fabsf(zeta) + z2 * rsqrtf(z2));
          const float cs = rsqrtf(fmaf(tt, tt, 1.f)), sn = cs * tt;
          if (lane < l) {
            U[lane][p] = cs * up - sn * uq;
            U[lane][q] = sn * up + cs * uq;
            const float vp = V[lane][p], vq = V[lane][q];
            V[lane][p] = cs * vp - sn * vq;
            V[lane][q] = sn * vp + cs * vq;
          }
          if (lane == 0) {
            nrm[p] = fmaxf(al - tt * g, 0.f);
            nrm[q] = fmaxf(be + tt * g, 0.f);
          }
        }
        __syncthreads();
      }
      for (int c = warp; c < l; c += kRW) {
        const float u = lane < l ? U[lane][c] : 0.f;
        float a = u * u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) nrm[c] = a;
      }
      if (!__syncthreads_or(busy)) break;
    }
    for (int c = warp; c < l; c += kRW) {
      float a = lane < l ? V[lane][c] * U[lane][c] : 0.f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      if (lane == 0) lam[c] = a;
    }
    __syncthreads();
    if (tid < l) {
      const float di = lam[tid];
      int rank = 0;
      for (int u = 0; u < l; ++u) rank += (lam[u] > di) || (lam[u] == di && u < tid);
      pr.ev[rank] = (double)di;
      if (rank < k) pr.theta[rank] = (double)di;
      for (int u = 0; u < l; ++u) {
        pr.Rm[u * l + rank] = (double)V[u][tid];
        if (rank < k) Vk[u][rank] = V[u][tid];
      }
    }
  }
  RITZ_PHASE(6);
  cluster.sync();                                    // Vk of CTA 0 complete
  {
    const float* Vk0 = cluster.map_shared_rank(&Vk[0][0], 0);
    for (int e = tid; e < l * kMaxK; e += kRT) (&Vk[0][0])[e] = Vk0[e];
  }
  cluster.sync();                                    // copies done before CTA 0 moves on
  RITZ_PHASE(7);
  // ---- Ritz vectors on the own rows: Phi = Q V_k, C Phi = (C Q) V_k ----
  float* Phi = reinterpret_cast<float*>(pr.Phi);
  float* CPhi = reinterpret_cast<float*>(pr.CPhi);
  float (*ph_s)[kRL + 1] = reinterpret_cast<float (*)[kRL + 1]>(xs);             // own rows of Phi
  float (*cp_s)[kRL + 1] = reinterpret_cast<float (*)[kRL + 1]>(xs) + kRMaxRows; // and of C Phi
  for (int e = tid; e < nrow * k; e += kRT) {
    const int a = e / k, j = e % k;
    float ph = 0.f, cp = 0.f;
    for (int i = 0; i < l; ++i) {
      ph = fmaf(ys[a][i], Vk[i][j], ph);
      cp = fmaf(zs[a][i], Vk[i][j], cp);
    }
    ph_s[a][j] = ph;
    cp_s[a][j] = cp;
    Phi[(r0 + a) * k + j] = ph;
    CPhi[(r0 + a) * k + j] = cp;
  }
  __syncthreads();
  RITZ_PHASE(8);
  // ---- Gram matrices of Phi and A = C Phi: gram[0] = Phi^T Phi, [1] = A^T Phi, [2] = A^T A ----
  for (int w3 = 0; w3 < 3; ++w3) {
    gram_partial(w3 == 0 ? ph_s : cp_s, w3 == 2 ? cp_s : ph_s, k, false);
    cluster.sync();
    if (crank == 0) {
      gram_merge(k * k, Tp_h, Tp_l);
      __syncthreads();
      for (int e = tid; e < k * k; e += kRT) pr.gram[w3 * k * k + e] = (double)Tp_h[e] + (double)Tp_l[e];
    }
    cluster.sync();                                  // partial reads done before the next overwrite
  }
  RITZ_PHASE(9);
#ifdef INFO_ESRF_PHASE_CLOCKS
  if (tid == 0 && crank == 0) {
    for (int i = 0; i < kRitzPhases; ++i) atomicAdd(&g_ritz_phase[i], (unsigned long long)ph_c[i]);
    atomicAdd(&g_ritz_phase[kRitzPhases], 1ull);
  }
#endif
}

int launch_ritz_cluster(const ProblemTable& tab, const ProblemDev* dtab, cudaStream_t st) {
  int64_t dmin = INT64_MAX;
  for (int i = 0; i < tab.count; ++i) dmin = tab.p[i].d < dmin ? tab.p[i].d : dmin;
  int CS = kRC;
  while (CS > 1 && dmin < (int64_t)CS * 64) CS >>= 1;
  for (int i = 0; i < tab.count; ++i)
    if (!ritz_cluster_fits(tab.p[i].d, tab.p[i].l) || (tab.p[i].l & 3) != 0 ||
        (tab.p[i].d + CS - 1) / CS > kRMaxRows)
      return -1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(tab.count * CS), 1, 1);
  cfg.blockDim = dim3(kRT, 1, 1);
  size_t dyn = 0;
  for (int i = 0; i < tab.count; ++i) dyn = std::max(dyn, (size_t)tab.p[i].d * (size_t)tab.p[i].l * 4);
  dyn = std::max(dyn, (size_t)2 * kRMaxRows * (kRL + 1) * 4);   // Phi / C Phi own rows reuse the area
  // the attribute allows the largest staging area once per thread and device
  constexpr int kMaxDev = 64;
  static thread_local bool attr_set[kMaxDev] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
    cudaGetLastError();
    return -1;
  }
  if (!attr_set[dev]) {
    const size_t most = std::max(kRStageBytes, (size_t)2 * kRMaxRows * (kRL + 1) * 4);
    if (cudaFuncSetAttribute(k_ritz_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most) != cudaSuccess) {
      cudaGetLastError();
      return -1;
    }
    attr_set[dev] = true;
  }
  cfg.dynamicSmemBytes = dyn;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t err = cudaLaunchKernelEx(&cfg, k_ritz_cluster, dtab);
  if (err != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  note_launches(1);
  return 0;
}

}  // namespace infoesrf

extern "C" int info_esrf_ritz_phase_clocks(int64_t* out, int32_t n, int32_t reset) {
#ifdef INFO_ESRF_PHASE_CLOCKS
  using namespace infoesrf;
  if (!out || n < 1) return INFO_ESRF_ERR_INVALID_ARG;
  unsigned long long h[kRitzPhases + 1] = {};
  if (cudaMemcpyFromSymbol(h, g_ritz_phase, sizeof(h)) != cudaSuccess) {
    cudaGetLastError();
    return INFO_ESRF_ERR_CUDA;
  }
  for (int i = 0; i < n && i < kRitzPhases + 1; ++i) out[i] = (int64_t)h[i];
  if (reset) {
    const unsigned long long z[kRitzPhases + 1] = {};
    if (cudaMemcpyToSymbol(g_ritz_phase, z, sizeof(z)) != cudaSuccess) {
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
