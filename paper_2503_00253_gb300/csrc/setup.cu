// Setup stages of one InFo-ESRF analysis, batched over problems (blockIdx.y).
//
//  * anomalies and observation gather   (Eq. normalized_perturbations, W = H Z)
//  * localized obs covariance band C    (Eq. localized_state_covar, Sec. 2.3,
//    normalized by R^-1/2 as in App. E) and the state-obs band Sxh
//  * quadrature nodes and weights       (App. D)
//  * randomized Ritz pairs of C         (App. E, Halko et al. Alg. 5.3)
//
// Precision: T is the bulk type (double on the FP64 path, float on the mixed
// path).  Sums that feed scalars use DotAcc<T> (float-float for float).
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace infoesrf {

template <typename T>
__device__ __forceinline__ T* tp(void* p) { return reinterpret_cast<T*>(p); }
template <typename T>
__device__ __forceinline__ const T* tp(const void* p) { return reinterpret_cast<const T*>(p); }

// ---------------------------------------------------------------------------
// Problem table upload: chunks of the host table travel as kernel parameters,
// so the upload is stream-ordered and graph-capturable.
// ---------------------------------------------------------------------------
constexpr int kChunk = 4;
struct TableChunk {
  int32_t first, count;
  ProblemDev p[kChunk];
};

// One launch per chunk of problems: block (0, i) writes problem i's table entry
// and clears its scalars and status; every block fills part of its per-axis
// table of (axis distance / half-width)^2 for every index offset, which the
// band kernels use instead of a transcendental per candidate pair.  Only the
// parameter copy of the table is read, so no block waits for the upload.
__global__ void k_prepare(const TableChunk c, ProblemDev* dst) {
  const int i = blockIdx.y;
  if (i >= c.count) return;
  const ProblemDev& pc = c.p[i];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    dst[c.first + i] = pc;
    pc.scal[0] = 0.0;
    pc.scal[1] = __longlong_as_double(0x7ff0000000000000LL);  // +inf, atomically lowered
    for (int u = 2; u < 8; ++u) pc.scal[u] = 0.0;
    for (int u = 0; u < 4; ++u) pc.status[u] = 0;
  }
  const GridDev& g = pc.grid;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t total = g.ext[0] + g.ext[1] + g.ext[2];
  if (e >= total) return;
  const int ax = e < g.ext[0] ? 0 : (e < g.ext[0] + g.ext[1] ? 1 : 2);
  const int64_t delta = e - (ax == 0 ? 0 : ax == 1 ? g.ext[0] : g.ext[0] + g.ext[1]);
  const double dd = axis_distance(g, ax, 0, delta) * g.inv_c[ax];
  pc.d2tab[e] = dd * dd;
}

void launch_prepare(const ProblemTable& tab, ProblemDev* dtab, cudaStream_t st) {
  for (int first = 0; first < tab.count; first += kChunk) {
    TableChunk c;
    c.first = first;
    c.count = tab.count - first < kChunk ? tab.count - first : kChunk;
    int64_t emax = 1;
    for (int i = 0; i < c.count; ++i) {
      c.p[i] = tab.p[first + i];
      const GridDev& g = tab.p[first + i].grid;
      emax = std::max<int64_t>(emax, g.ext[0] + g.ext[1] + g.ext[2]);
    }
    k_prepare<<<dim3((unsigned)((emax + 255) / 256), (unsigned)c.count), 256, 0, st>>>(c, dtab);
    note_launches(1);
  }
}

// ---------------------------------------------------------------------------
// a1: ensemble mean and normalized anomalies Z (Eq. normalized_perturbations)
// ---------------------------------------------------------------------------
// One CTA per 32 consecutive state points (kAnomPts); warp w of the 8 takes
// the members w, w + 8, ...  Reads of X are coalesced over the points, the
// member sum is FP64 in a fixed order (per warp, then over the warps), and
// Z^T [n][N] is written through a shared-memory transpose, 32 members at a
// time, so that each point's member run is contiguous.
constexpr int kAnomPts = 32;
template <typename T>
__global__ void __launch_bounds__(256) k_anomalies(const ProblemDev* tab) {
  const ProblemDev& pr = tab[blockIdx.y];
  const int64_t x0 = (int64_t)blockIdx.x * kAnomPts;
  if (x0 >= pr.n) return;
  const int64_t N = pr.N, n = pr.n;
  const int lx = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t x = x0 + lx;
  const bool in = x < n;
  __shared__ double s_part[8][kAnomPts];
  __shared__ double s_mu[kAnomPts];
  __shared__ T s_tile[kAnomPts][33];
  __shared__ int s_bad;
  if (threadIdx.x == 0) s_bad = 0;
  double sum = 0.0;
  bool bad = false;
  if (in)
    for (int64_t k = w; k < N; k += 8) {
      const double v = pr.X[k * n + x];
      bad |= !isfinite(v);
      sum += v;
    }
  s_part[w][lx] = sum;
  __syncthreads();
  if (bad) s_bad = 1;
  if (w == 0) {
    double t = 0.0;
    for (int u = 0; u < 8; ++u) t += s_part[u][lx];
    const double mu = t / (double)N;
    s_mu[lx] = mu;
    if (in) pr.mu[x] = mu;
  }
  __syncthreads();
  const double mu = s_mu[lx];
  const double scale = 1.0 / pr.sqrt_nm1;
  T* Zt = tp<T>(pr.Zt);
  const int np = (int)(n - x0 < kAnomPts ? n - x0 : kAnomPts);
  for (int64_t c0 = 0; c0 < N; c0 += 32) {
    const int nk = (int)(N - c0 < 32 ? N - c0 : 32);
    for (int kk = w; kk < nk; kk += 8)
      s_tile[lx][kk] = in ? to_t<T>((pr.X[(c0 + kk) * n + x] - mu) * scale) : to_t<T>(0.0);
    __syncthreads();
    for (int e = threadIdx.x; e < np * 32; e += blockDim.x) {
      const int xi = e >> 5, kk = e & 31;
      if (kk < nk) Zt[(x0 + xi) * N + c0 + kk] = s_tile[xi][kk];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && s_bad) atomicOr(&pr.status[0], kStatNonFinite);
}

// W = H Z (rows of Z at the observed points), one thread per (observation,
// member) element so that the copy is coalesced; the member-0 thread of each
// observation also checks its index, forms R^-1/2 and the mean right-hand side.
template <typename T>
__global__ void k_observe(const ProblemDev* tab) {
  const ProblemDev& pr = tab[blockIdx.y];
  if (pr.H_rowptr) return;   // general observation operator: k_observe_H
  const int64_t N = pr.N;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= pr.d * N) return;
  const int64_t a = i / N, k = i - a * N;
  int64_t o = pr.obs[a];
  const bool bad_obs = o < 0 || o >= pr.n || (a > 0 && pr.obs[a - 1] >= o);
  if (o < 0) o = 0;
  if (o >= pr.n) o = pr.n - 1;
  tp<T>(pr.W)[i] = tp<const T>(pr.Zt)[o * N + k];
  if (k != 0) return;
  const double r = pr.R[a];
  const bool bad_r = !(r > 0.0) || !isfinite(r);
  const double ri = bad_r ? 0.0 : 1.0 / sqrt(r);
  pr.rinv[a] = ri;
  if (pr.do_mean) pr.bmean[a] = ri * (pr.y[a] - pr.mu[o]);
  if (bad_obs) atomicOr(&pr.status[0], kStatBadObs);
  if (bad_r) atomicOr(&pr.status[0], kStatBadR);
}

// ---------------------------------------------------------------------------
// General linear observation operator H (CSR, one row per observation; the
// paper's weighted sums, Sec. 4.1 and Sec. 5.1).  With h linearized and
// model-space localization (Sec. 2.3): W = H Z, Sxh = (L o Z Z^T) H^T,
// Shh = H Sxh, so C = R^-1/2 H Sxh R^-1/2.  Both are dense ([n][d], [d][d])
// and stored in the ELL layouts of the subsampling path with every column
// present, so the later stages run unchanged.  Row pointers and columns are
// checked before any entry is read.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool h_row(const ProblemDev& pr, int64_t a, int64_t& e0, int64_t& e1) {
  e0 = pr.H_rowptr[a];
  e1 = pr.H_rowptr[a + 1];
  if (e0 < 0 || e1 < e0 || e1 > pr.H_nnz || (a == 0 && e0 != 0)) {
    e0 = 0;
    e1 = 0;
    return false;
  }
  return true;
}

// W = H Z, one thread per (observation, member); the member-0 thread of each
// observation also forms R^-1/2 and the mean right-hand side R^-1/2 (y - H mu).
template <typename T>
__global__ void k_observe_H(const ProblemDev* tab) {
  const ProblemDev& pr = tab[blockIdx.y];
  if (!pr.H_rowptr) return;
  const int64_t N = pr.N;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= pr.d * N) return;
  const int64_t a = i / N, k = i - a * N;
  int64_t e0, e1;
  bool bad = !h_row(pr, a, e0, e1);
  const T* Zt = tp<const T>(pr.Zt);
  double w = 0.0, hmu = 0.0;
  for (int64_t e = e0; e < e1; ++e) {
    const int64_t c = pr.H_col[e];
    if (c < 0 || c >= pr.n) {
      bad = true;
      continue;
    }
    const double h = pr.H_val[e];
    w += h * (double)Zt[c * N + k];
    if (k == 0) hmu += h * pr.mu[c];
  }
  tp<T>(pr.W)[i] = to_t<T>(w);
  if (k != 0) return;
  const double r = pr.R[a];
  const bool bad_r = !(r > 0.0) || !isfinite(r);
  const double ri = bad_r ? 0.0 : 1.0 / sqrt(r);
  pr.rinv[a] = ri;
  if (pr.do_mean) pr.bmean[a] = ri * (pr.y[a] - hmu);
  if (bad) atomicOr(&pr.status[0], kStatBadObs);
  if (bad_r) atomicOr(&pr.status[0], kStatBadR);
}

// Sxh(x, b) = sum_j H(b, j) L(x, j) z_x . z_j, thread x (consecutive, so that
// the ELL writes are coalesced) of observation column b = blockIdx.y.
template <typename T>
__global__ void k_sxh_H(const ProblemDev* tab) {
  const ProblemDev& pr = tab[blockIdx.z];
  if (!pr.H_rowptr) return;
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t b = blockIdx.y;
  const int64_t n = pr.n, N = pr.N;
  if (x >= n || b >= pr.d) return;
  const GridDev& g = pr.grid;
  const Coord3 px = flat_to_coord(g, x);
  const T* Zt = tp<const T>(pr.Zt);
  const T* zx = Zt + x * N;
  int64_t e0, e1;
  h_row(pr, b, e0, e1);
  double acc = 0.0;
  for (int64_t e = e0; e < e1; ++e) {
    const int64_t c = pr.H_col[e];
    if (c < 0 || c >= n) continue;
    const double r2 = scaled_r2_tab(g, pr.d2tab, px, flat_to_coord(g, c));
    if (!(r2 < 4.0)) continue;
    DotAcc<T> dot;
    const T* zc = Zt + c * N;
    for (int64_t k = 0; k < N; ++k) dot.add_prod(zx[k], zc[k]);
    const double gc = sizeof(T) == 8 ? gaspari_cohn(sqrt(r2)) : (double)gaspari_cohn_f(sqrtf((float)r2));
    acc += pr.H_val[e] * gc * dot.value();
  }
  tp<T>(pr.xo_val)[b * n + x] = to_t<T>(acc);
  pr.xo_col[b * n + x] = (int32_t)b;
  if (b == 0) pr.xo_nnz[x] = (int32_t)pr.d;
}

// C(a, b) = R_a^-1/2 R_b^-1/2 sum_x H(a, x) Sxh(x, b), one warp per row a with
// the lanes over b; the Gershgorin bound, the minimum and the sum of the
// diagonal as in k_band.
template <typename T>
__global__ void k_c_H(const ProblemDev* tab) {
  const ProblemDev& pr = tab[blockIdx.y];
  if (!pr.H_rowptr) return;
  const int lane = threadIdx.x & 31;
  const int64_t a = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t n = pr.n, d = pr.d;
  if (a >= d) return;
  int64_t e0, e1;
  h_row(pr, a, e0, e1);
  const T* S = tp<const T>(pr.xo_val);
  const double ra = pr.rinv[a];
  double rowsum = 0.0;
  for (int64_t b = lane; b < d; b += 32) {
    double acc = 0.0;
    for (int64_t e = e0; e < e1; ++e) {
      const int64_t c = pr.H_col[e];
      if (c < 0 || c >= n) continue;
      acc += pr.H_val[e] * (double)S[b * n + c];
    }
    const double v = ra * pr.rinv[b] * acc;
    tp<T>(pr.oo_val)[b * d + a] = to_t<T>(v);
    pr.oo_col[b * d + a] = (int32_t)b;
    rowsum += fabs(v);
    if (b == a) {
      atomic_min_nonneg(&pr.scal[1], fmax(v, 0.0));
      atomicAdd(&pr.scal[4], v);
    }
  }
  rowsum = warp_sum(rowsum);
  if (lane == 0) {
    pr.oo_nnz[a] = (int32_t)d;
    atomic_max_nonneg(&pr.scal[0], rowsum);
  }
}

static bool any_general_h(const ProblemTable& tab) {
  for (int i = 0; i < tab.count; ++i)
    if (tab.p[i].H_rowptr) return true;
  return false;
}

void launch_anomalies(const ProblemTable& tab, const ProblemDev* dtab, cudaStream_t st) {
  int64_t nmax = 0, dnmax = 0;
  for (int i = 0; i < tab.count; ++i) {
    nmax = tab.p[i].n > nmax ? tab.p[i].n : nmax;
    dnmax = tab.p[i].d * tab.p[i].N > dnmax ? tab.p[i].d * tab.p[i].N : dnmax;
  }
  const bool f64 = tab.p[0].precision == 0;
  dim3 g1((unsigned)((nmax + kAnomPts - 1) / kAnomPts), tab.count);
  dim3 g2((unsigned)((dnmax + 255) / 256), tab.count);
  if (f64) {
    k_anomalies<double><<<g1, 256, 0, st>>>(dtab); note_launches(1);
    k_observe<double><<<g2, 256, 0, st>>>(dtab); note_launches(1);
    if (any_general_h(tab)) { k_observe_H<double><<<g2, 256, 0, st>>>(dtab); note_launches(1); }
  } else {
    k_anomalies<float><<<g1, 256, 0, st>>>(dtab); note_launches(1);
    k_observe<float><<<g2, 256, 0, st>>>(dtab); note_launches(1);
    if (any_general_h(tab)) { k_observe_H<float><<<g2, 256, 0, st>>>(dtab); note_launches(1); }
  }
}

// ---------------------------------------------------------------------------
// Bands.  One warp per row.  Lanes take consecutive candidate obs b from the
// geometry's candidate ranges, keep those with r < 2, and append
//   C(a, b) = GC(r) (w_a . w_b) R_a^-1/2 R_b^-1/2        (obs-obs, rows = obs)
//   Sxh(x, b) = GC(r) (z_x . w_b)                        (state-obs, rows = state)
// in increasing candidate order to the ELL row (column-major: entry e of row
// a at e * rows + a).
// ---------------------------------------------------------------------------
template <typename T, bool OBS_ROWS>
__global__ void k_band(const ProblemDev* tab) {
  const ProblemDev& pr = tab[blockIdx.y];
  if (pr.H_rowptr) return;   // general observation operator: k_sxh_H and k_c_H
  const int lane = threadIdx.x & 31;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t rows = OBS_ROWS ? pr.d : pr.n;
  if (row >= rows) return;
  const int64_t N = pr.N, d = pr.d;
  const GridDev& g = pr.grid;
  int64_t pidx = OBS_ROWS ? pr.obs[row] : row;
  if (pidx < 0) pidx = 0;
  if (pidx >= pr.n) pidx = pr.n - 1;
  const Coord3 pc = flat_to_coord(g, pidx);
  const T* W = tp<const T>(pr.W);
  const T* src = OBS_ROWS ? W + row * N : tp<const T>(pr.Zt) + row * N;
  const int64_t cap = OBS_ROWS ? pr.max_oo : pr.max_xo;
  T* val = OBS_ROWS ? tp<T>(pr.oo_val) : tp<T>(pr.xo_val);
  int32_t* col = OBS_ROWS ? pr.oo_col : pr.xo_col;
  const double ra = OBS_ROWS ? pr.rinv[row] : 1.0;
  int64_t count = 0;
  double rowsum = 0.0;
  for_each_candidate_range(g, pr.obs, d, pc, [&](int64_t b0, int64_t b1) {
    for (int64_t base = b0; base < b1; base += 32) {
      const int64_t b = base + lane;
      double v = 0.0;
      bool keep = false;
      if (b < b1) {
        const Coord3 bc = flat_to_coord(g, pr.obs[b]);
        const double r2 = scaled_r2_tab(g, pr.d2tab, pc, bc);
        if (r2 < 4.0) {
          keep = true;
          DotAcc<T> acc;
          const T* wb = W + b * N;
          // 16-byte loads when the member rows allow them (same order of terms)
          if (sizeof(T) == 4 && (N & 3) == 0) {
            const float4* s4 = reinterpret_cast<const float4*>(src);
            const float4* w4 = reinterpret_cast<const float4*>(wb);
            for (int64_t k = 0; k < N / 4; ++k) {
              const float4 u = s4[k], v4 = w4[k];
              acc.add_prod((T)u.x, (T)v4.x);
              acc.add_prod((T)u.y, (T)v4.y);
              acc.add_prod((T)u.z, (T)v4.z);
              acc.add_prod((T)u.w, (T)v4.w);
            }
          } else if (sizeof(T) == 8 && (N & 1) == 0) {
            const double2* s2 = reinterpret_cast<const double2*>(src);
            const double2* w2 = reinterpret_cast<const double2*>(wb);
            for (int64_t k = 0; k < N / 2; ++k) {
              const double2 u = s2[k], v2 = w2[k];
              acc.add_prod((T)u.x, (T)v2.x);
              acc.add_prod((T)u.y, (T)v2.y);
            }
          } else {
            for (int64_t k = 0; k < N; ++k) acc.add_prod(src[k], wb[k]);
          }
          const double gc = sizeof(T) == 8 ? gaspari_cohn(sqrt(r2)) : (double)gaspari_cohn_f(sqrtf((float)r2));
          v = gc * acc.value();
          if (OBS_ROWS) v *= ra * pr.rinv[b];
        }
      }
      const unsigned mask = __ballot_sync(0xffffffffu, keep);
      const int before = __popc(mask & ((1u << lane) - 1u));
      if (keep) {
        const int64_t e = count + before;
        if (e < cap) {
          val[e * rows + row] = to_t<T>(v);
          col[e * rows + row] = (int32_t)b;
        }
        rowsum += fabs(v);
        if (OBS_ROWS && b == row) {
          atomic_min_nonneg(&pr.scal[1], v);
          atomicAdd(&pr.scal[4], v);
        }
      }
      count += __popc(mask);
    }
  });
  rowsum = warp_sum(rowsum);
  if (lane == 0) {
    int32_t* nnz = OBS_ROWS ? pr.oo_nnz : pr.xo_nnz;
    nnz[row] = (int32_t)(count < cap ? count : cap);
    if (count > cap) atomicOr(&pr.status[0], kStatBandOverflow);
    if (OBS_ROWS) atomic_max_nonneg(&pr.scal[0], rowsum);
  }
}

// Band of C (obs rows); the distance table comes from launch_prepare.
void launch_band_obs(const ProblemTable& tab, const ProblemDev* dtab, cudaStream_t st) {
  int64_t dmax = 0;
  for (int i = 0; i < tab.count; ++i) dmax = tab.p[i].d > dmax ? tab.p[i].d : dmax;
  dim3 go((unsigned)((dmax * 32 + 255) / 256), tab.count);
  if (tab.p[0].precision == 0) k_band<double, true><<<go, 256, 0, st>>>(dtab);
  else k_band<float, true><<<go, 256, 0, st>>>(dtab);
  note_launches(1);
  if (any_general_h(tab)) {
    // dense Sxh first (C is formed from it), then C
    int64_t nmax = 0, dh = 0;
    for (int i = 0; i < tab.count; ++i)
      if (tab.p[i].H_rowptr) {
        nmax = std::max<int64_t>(nmax, tab.p[i].n);
        dh = std::max<int64_t>(dh, tab.p[i].d);
      }
    const dim3 gs((unsigned)((nmax + 127) / 128), (unsigned)dh, tab.count);
    const dim3 gc((unsigned)((dh * 32 + 255) / 256), tab.count);
    if (tab.p[0].precision == 0) {
      k_sxh_H<double><<<gs, 128, 0, st>>>(dtab);
      k_c_H<double><<<gc, 256, 0, st>>>(dtab);
    } else {
      k_sxh_H<float><<<gs, 128, 0, st>>>(dtab);
      k_c_H<float><<<gc, 256, 0, st>>>(dtab);
    }
    note_launches(2);
  }
}

// Band of Sxh (state rows); needed only by the state update.
void launch_band_state(const ProblemTable& tab, const ProblemDev* dtab, cudaStream_t st) {
  int64_t nmax = 0;
  for (int i = 0; i < tab.count; ++i) nmax = tab.p[i].n > nmax ? tab.p[i].n : nmax;
  dim3 gx((unsigned)((nmax * 32 + 255) / 256), tab.count);
  if (tab.p[0].precision == 0) k_band<double, false><<<gx, 256, 0, st>>>(dtab);
  else k_band<float, false><<<gx, 256, 0, st>>>(dtab);
  note_launches(1);
}

void launch_bands(const ProblemTable& tab, const ProblemDev* dtab, cudaStream_t st) {
  launch_band_obs(tab, dtab, st);
  launch_band_state(tab, dtab, st);
}

// Counts neighbours to size the bands: out2[0] = max obs per obs row,
// out2[1] = max obs per state row.
__global__ void k_count_neighbours(const GridDev g, const int64_t* obs, int64_t d, int64_t n,
                                   unsigned long long* out2) {
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n + d) return;
  const bool is_obs = row >= n;
  int64_t pidx = is_obs ? obs[row - n] : row;
  if (pidx < 0) pidx = 0;
  if (pidx >= n) pidx = n - 1;
  const Coord3 pc = flat_to_coord(g, pidx);
  unsigned long long count = 0;
  for_each_candidate_range(g, obs, d, pc, [&](int64_t b0, int64_t b1) {
    for (int64_t b = b0; b < b1; ++b) {
      if (scaled_distance(g, pc, flat_to_coord(g, obs[b])) < 2.0) ++count;
    }
  });
  atomicMax(&out2[is_obs ? 0 : 1], count);
}

void launch_count_neighbours(const GridDev& g, const int64_t* obs, int64_t d, int64_t n,
                             int64_t* out2, cudaStream_t st) {
  cudaMemsetAsync(out2, 0, 2 * sizeof(int64_t), st);
  const int64_t rows = n + d;
  k_count_neighbours<<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(
      g, obs, d, n, reinterpret_cast<unsigned long long*>(out2));
  note_launches(1);
}

// ---------------------------------------------------------------------------
// a2: quadrature (App. D).  Elliptic rule with modulus g = sqrt(ell/(1+ell)):
//   s_q = sc(u_q | g)^2,  p_q = (2 K / (pi Q)) dn(u_q | g),  u_q = (q - 1/2) K / Q,
// which is r_q / (s_q + 1) with r_q = (2K/(pi Q)) nc dc (d sc/du = dc nc and
// sc^2 + 1 = nc^2).  K and the Jacobi functions come from one descending
// Landen ladder in float-float (quadrature_node); nodes past K/2 use
// sn(K - v) = cd(v), cn(K - v) = g' sd(v), dn(K - v) = g' nd(v) so that small
// cn values keep full relative precision.
// ---------------------------------------------------------------------------
// pi / 2 as a float-float pair, and the Taylor coefficients (-1)^j / (2j+1)! and
// (-1)^j / (2j)!, j = 0..9, as exact float-float pairs (hexadecimal literals).
constexpr float kPiHalfHi = 0x1.921fb6p+0f, kPiHalfLo = -0x1.777a5cp-25f;
__constant__ float kSinH[10] = {0x1p+0f, -0x1.555556p-3f, 0x1.111112p-7f, -0x1.a01a02p-13f, 0x1.71de3ap-19f,
                                -0x1.ae6456p-26f, 0x1.612462p-33f, -0x1.ae7f3ep-41f, 0x1.952c78p-49f,
                                -0x1.2f49b4p-57f};
__constant__ float kSinL[10] = {0.f, 0x1.555556p-28f, -0x1.dddddep-32f, 0x1.7f97fap-39f, 0x1.55b1ccp-45f,
                                -0x1.fd5138p-52f, -0x1.8af25ep-58f, -0x1.ccee08p-67f, -0x1.f9ea56p-74f,
                                -0x1.a05056p-83f};
__constant__ float kCosH[10] = {0x1p+0f, -0x1p-1f, 0x1.555556p-5f, -0x1.6c16c2p-10f, 0x1.a01a02p-16f,
                                -0x1.27e4fcp-22f, 0x1.1eed8ep-29f, -0x1.93974ap-37f, 0x1.ae7f3ep-45f,
                                -0x1.682786p-53f};
__constant__ float kCosL[10] = {0.f, 0.f, -0x1.555556p-30f, 0x1.27d27ep-35f, -0x1.7f97fap-42f, 0x1.10ec14p-47f,
                                0x1.ff1b14p-54f, -0x1.180f94p-62f, 0x1.ccee08p-71f, -0x1.dcbeccp-80f};

// sin x and cos x for |x| <= pi/4 in float-float: Taylor series by Horner's
// rule in x^2, truncated after x^19 (sin) and x^18 (cos), below 1e-17 there.
__device__ void ff_sincos_small(FF x, FF& sn, FF& cn) {
  const FF x2 = ff_mul(x, x);
  FF as{kSinH[9], kSinL[9]}, ac{kCosH[9], kCosL[9]};
  for (int j = 8; j >= 0; --j) {
    as = ff_add(FF{kSinH[j], kSinL[j]}, ff_mul(as, x2));
    ac = ff_add(FF{kCosH[j], kCosL[j]}, ff_mul(ac, x2));
  }
  sn = ff_mul(x, as);
  cn = ac;
}

__device__ void quadrature_node(int32_t Q, double ell, int32_t rule, int q, double& s, double& p) {
  if (rule == 1) {
    // Gauss-Legendre on (0,1) for the trigonometric form (Eq. gaussian_quadrature_rule);
    // Newton iteration on P_Q with the three-term recurrence.
    double x = cos(kPi * (q + 0.75) / (Q + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= Q; ++k) {
        const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (Q == 1) { p1 = x; p0 = 1.0; }
      dp = Q * (x * p1 - p0) / (x * x - 1.0);
      const double dx = p1 / dp;
      x -= dx;
      if (fabs(dx) < 1e-16) {
        break;
      }
    }
    {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= Q; ++k) {
        const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = Q * (x * p1 - p0) / (x * x - 1.0);
    }
    const double v = 2.0 / ((1.0 - x * x) * dp * dp);
    const double lam = 0.5 * (1.0 - x);   // ascending order in q
    const double tn = tan(0.5 * kPi * lam);
    s = tn * tn;
    p = 0.5 * v;
    return;
  }
  // Elliptic rule in float-float (about 48 bits, FP32 instructions only; a
  // chain of FP64 instructions is slow on this GPU).  Descending Landen
  // ladder of the modulus g (g^2 = ell / (1 + ell), g' = (1 + ell)^-1/2):
  //   k_{n+1} = k_n^2 / (1 + k'_n)^2 = (1 - k'_n) / (1 + k'_n),  k'_{n+1} = 2 sqrt(k'_n) / (1 + k'_n),
  // free of cancellation for k near 1, with K = (pi/2) prod_n (1 + k_n).  The
  // argument at the bottom of the ladder is u prod_n (1 + k_n)^-1 = t pi / 2
  // for u = t K, so sin and cos are of a known angle <= pi/4 (Taylor series);
  // sn, cn, dn then ascend the ladder by the descending Landen (Gauss)
  // transformation (Abramowitz & Stegun 16.12): with s2 = k_{n+1} sn^2,
  //   sn <- (1 + k_{n+1}) sn / (1 + s2),  cn <- cn dn / (1 + s2),  dn <- (1 - s2) / (1 + s2).
  // Nodes past K/2 use the reflection below.
  const FF one{1.f, 0.f};
  const FF L = ff_from(ell);
  const FF kp0 = ff_rsqrt(ff_add(one, L));
  FF k = ff_mul(ff_sqrt(L), kp0), kp = kp0, prod = one;
  FF ks[24];
  int nk = 0;
  while (k.h > 1e-17f && nk < 24) {
    const FF opk = ff_add(one, kp);
    const FF k1 = ff_div(ff_mul(k, k), ff_mul(opk, opk));
    ks[nk++] = k1;
    prod = ff_mul(prod, ff_add(one, k1));
    kp = ff_div(ff_mul(FF{2.f, 0.f}, ff_sqrt(kp)), opk);
    k = k1;
  }
  const double t = (q + 0.5) / Q;
  const bool refl = t > 0.5;
  const double tt = refl ? ((Q - q) - 0.5) / Q : t;   // K - u_q, formed without cancellation
  FF sn, cn;
  ff_sincos_small(ff_mul(FF{kPiHalfHi, kPiHalfLo}, ff_from(tt)), sn, cn);
  FF dn = one;
  for (int i = nk - 1; i >= 0; --i) {
    const FF s2 = ff_mul(ks[i], ff_mul(sn, sn));
    const FF den = ff_div(one, ff_add(one, s2));
    const FF s_new = ff_mul(ff_mul(ff_add(one, ks[i]), sn), den);
    const FF c_new = ff_mul(ff_mul(cn, dn), den);
    dn = ff_mul(ff_sub(one, s2), den);
    sn = s_new;
    cn = c_new;
  }
  const FF scale = ff_div(prod, ff_from((double)Q));   // 2 K / (pi Q)
  FF sq, pq;
  if (!refl) {
    const FF r = ff_div(sn, cn);                       // sc(u_q)
    sq = ff_mul(r, r);
    pq = ff_mul(scale, dn);
  } else {
    const FF r = ff_div(cn, ff_mul(kp0, sn));          // sc(K - v) = cd(v) / (g' sd(v))
    sq = ff_mul(r, r);
    pq = ff_div(ff_mul(scale, kp0), dn);               // dn(K - v) = g' / dn(v)
  }
  s = (double)sq.h + (double)sq.l;
  p = (double)pq.h + (double)pq.l;
}

__global__ void k_quadrature(ProblemDev* tab) {
  ProblemDev& pr = tab[blockIdx.x];
  __shared__ double ell_s;
  if (threadIdx.x == 0) {
    double ell = pr.ell_fixed;
    if (!(ell > 0.0)) {
      const double b = fmax(pr.scal[0], 1.0);
      ell = exp10(floor(log10(b)) + 1.0);
    }
    ell_s = ell;
    pr.scal[2] = ell;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < pr.Q; q += blockDim.x) {
    double s, p;
    quadrature_node(pr.Q, ell_s, pr.rule, q, s, p);
    pr.s[q] = s;
    pr.p[q] = p;
  }
}

void launch_quadrature(const ProblemTable& tab, const ProblemDev* dtab, cudaStream_t st) {
  k_quadrature<<<tab.count, 64, 0, st>>>(const_cast<ProblemDev*>(dtab)); note_launches(1);
}

__global__ void k_quadrature_nodes(int32_t Q, double ell, int32_t rule, double* s, double* p) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < Q) quadrature_node(Q, ell, rule, q, s[q], p[q]);
}

void launch_quadrature_nodes(int32_t Q, double ell, int32_t rule, double* s, double* p, cudaStream_t st) {
  k_quadrature_nodes<<<(Q + 63) / 64, 64, 0, st>>>(Q, ell, rule, s, p); note_launches(1);
}

__global__ void k_philox(uint64_t seed, int64_t count, double* out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < count) out[e] = philox_normal(seed, (uint64_t)e);
}

void launch_philox(uint64_t seed, int64_t count, double* out, cudaStream_t st) {
  if (count > 0) {
    k_philox<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(seed, count, out);
    note_launches(1);
  }
}

// ---------------------------------------------------------------------------
// a4: randomized Ritz pairs of C (App. E; Halko, Martinsson, Tropp Alg. 5.3
// on a range basis from their Alg. 4.3 with power_iters power iterations).
//
// Two [d][l] buffers of the bulk type T (Om and Yb) hold the basis and its
// image under C; `src` selects which one a kernel reads.  Gram matrices are
// summed with DotAcc<T> and kept in FP64.  Orthonormalization is CholeskyQR2
// (each pass: G = X^T X, G = R^T R, X <- X R^-1, the Cholesky factor formed
// redundantly by every row block).  The l x l eigenproblem uses cyclic
// Jacobi with one thread per matrix entry and l/2 disjoint rotations per
// round (round-robin ordering), in the bulk precision.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T* ritz_buf(const ProblemDev& pr, int which) {
  return reinterpret_cast<T*>(which == 0 ? pr.Om : pr.Yb);
}

template <typename T>
__global__ void k_ritz_omega(const ProblemDev* tab) {
  const ProblemDev& pr = tab[blockIdx.y];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (pr.l <= 0 || i >= pr.d * pr.l) return;
  const int64_t a = i / pr.l, j = i % pr.l;
  ritz_buf<T>(pr, 0)[i] = to_t<T>(philox_normal(pr.seed, (uint64_t)(j * pr.d + a)));
}

// dst = C src: one warp per row, lanes over the row's band entries; each lane
// accumulates all l columns of its entries, then a butterfly reduce-scatter
// leaves column j's sum in lane j.
template <typename T>
__global__ void k_ritz_matvec(const ProblemDev* tab, int src) {
  const ProblemDev& pr = tab[blockIdx.y];
  const int l = pr.l;
  const int lane = threadIdx.x & 31;
  const int64_t a = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (l <= 0 || a >= pr.d) return;
  const int64_t d = pr.d;
  const T* __restrict__ V = ritz_buf<T>(pr, src);
  T* Y = ritz_buf<T>(pr, 1 - src);
  const T* __restrict__ val = tp<const T>(pr.oo_val);
  const int32_t* __restrict__ col = pr.oo_col;
  const int nnz = pr.oo_nnz[a];
  T acc[32];
#pragma unroll
  for (int m = 0; m < 32; ++m) acc[m] = T(0);
  const bool vec4 = sizeof(T) == 4 && (l & 3) == 0;
  for (int e = lane; e < nnz; e += 32) {
    const T c = val[(int64_t)e * d + a];
    const T* vr = V + (int64_t)col[(int64_t)e * d + a] * l;
    if (vec4) {
#pragma unroll
      for (int m4 = 0; m4 < 8; ++m4) {
        if (4 * m4 < l) {
          const float4 v = *reinterpret_cast<const float4*>(reinterpret_cast<const float*>(vr) + 4 * m4);
          acc[4 * m4 + 0] += c * (T)v.x;
          acc[4 * m4 + 1] += c * (T)v.y;
          acc[4 * m4 + 2] += c * (T)v.z;
          acc[4 * m4 + 3] += c * (T)v.w;
        }
      }
    } else {
#pragma unroll
      for (int m = 0; m < 32; ++m)
        if (m < l) acc[m] += c * vr[m];
    }
  }
  const T sum = warp_reduce_scatter32<T>(acc, lane);
  if (lane < l) Y[a * l + lane] = sum;
}

// G[i][j] = sum_a A[a][i] B[a][j] (FP64 result), one block per entry.
// sym: A = B = buf(src) and only j >= i is computed (mirrored).
template <typename T>
__global__ void k_ritz_gram(const ProblemDev* tab, int srcA, int srcB, int sym) {
  const ProblemDev& pr = tab[blockIdx.y];
  const int l = pr.l;
  const int pair = blockIdx.x;
  if (l <= 0 || pair >= l * l) return;
  const int i = pair / l, j = pair % l;
  if (sym && j < i) return;
  const T* A = ritz_buf<T>(pr, srcA);
  const T* Bm = ritz_buf<T>(pr, srcB);
  DotAcc<T> acc;
  for (int64_t a = threadIdx.x; a < pr.d; a += blockDim.x) acc.add_prod(A[a * l + i], Bm[a * l + j]);
  DotAcc<T> accs[1] = {acc};
  double out[1];
  __shared__ double scratch[2 * kThreads / 32];
  block_sum<1>(accs, out, scratch);
  if (threadIdx.x == 0) {
    pr.Gm[i * l + j] = out[0];
    if (sym) pr.Gm[j * l + i] = out[0];
  }
}

// X_dst = X_src R^-1 with G = R^T R the Cholesky factorization of the Gram
// matrix in Gm.  Right-looking factorization in float-float arithmetic by four
// warps: warp 0 takes the pivot's reciprocal square root, all threads scale
// row j and update the trailing upper triangle.  A non-positive pivot zeroes
// that column (rank loss) and flags kStatEigFail.  R goes to shared memory in
// the bulk type for the triangular solve, one thread per row.
template <typename T>
__global__ void k_ritz_orth(const ProblemDev* tab, int src) {
  const ProblemDev& pr = tab[blockIdx.y];
  const int l = pr.l;
  if (l <= 0) return;
  __shared__ FF G[kMaxRitz][kMaxRitz + 1];
  __shared__ FF Rrow[kMaxRitz];
  __shared__ FF s_inv;
  __shared__ float s_tiny;
  __shared__ T Rt[kMaxRitz][kMaxRitz + 1];
  __shared__ T rinv[kMaxRitz];
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
    const int i = e / l, c = e % l;
    if (i <= c) G[i][c] = ff_from(pr.Gm[e]);
  }
  if (threadIdx.x < 32) {
    float tr = threadIdx.x < l ? (float)pr.Gm[threadIdx.x * (l + 1)] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
    if (threadIdx.x == 0) s_tiny = 1e-28f * (tr > 0.f ? tr : 1.f);
  }
  __syncthreads();
  constexpr int kCT = 128;
  const int t = threadIdx.x;
  if (t < kCT) {
    const float tiny = s_tiny;
    for (int j = 0; j < l; ++j) {
      if (t == 0) {
        const FF gjj = G[j][j];
        const bool ok = gjj.h > tiny;
        const FF inv = ok ? ff_rsqrt(gjj) : FF{0.f, 0.f};
        s_inv = inv;
        const FF rjj = ff_mul(gjj, inv);
        Rt[j][j] = (T)rjj.h + (T)rjj.l;
        rinv[j] = (T)inv.h + (T)inv.l;
        if (!ok && blockIdx.x == 0) atomicOr(&pr.status[0], kStatEigFail);
      }
      asm volatile("bar.sync 1, 128;" ::: "memory");
      const FF inv = s_inv;
      for (int c = j + 1 + t; c < l; c += kCT) {
        const FF r = ff_mul(G[j][c], inv);
        Rrow[c] = r;
        Rt[j][c] = (T)r.h + (T)r.l;
      }
      if (t < j) Rt[j][t] = T(0);
      asm volatile("bar.sync 1, 128;" ::: "memory");
      const int mrem = l - 1 - j;
      for (int e = t; e < mrem * mrem; e += kCT) {
        const int c2 = j + 1 + e / mrem, c = j + 1 + e % mrem;
        if (c2 <= c) G[c2][c] = ff_sub(G[c2][c], ff_mul(Rrow[c2], Rrow[c]));
      }
      asm volatile("bar.sync 1, 128;" ::: "memory");
    }
  }
  __syncthreads();
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= pr.d) return;
  const T* X = ritz_buf<T>(pr, src);
  T* Y = ritz_buf<T>(pr, 1 - src);
  T row[kMaxRitz];
#pragma unroll
  for (int j = 0; j < kMaxRitz; ++j) {
    if (j < l) {
      T t = X[a * l + j];
#pragma unroll
      for (int k = 0; k < j; ++k) t -= row[k] * Rt[k][j];
      row[j] = t * rinv[j];
    } else {
      row[j] = T(0);
    }
  }
#pragma unroll
  for (int j = 0; j < kMaxRitz; ++j)
    if (j < l) Y[a * l + j] = row[j];
}

// Element-parallel cyclic Jacobi on B = sym(Om^T C Om) (Gm holds Om^T (C Om)),
// one thread per entry.  The round-robin pairing of every round is tabulated
// once; a round is then two barriers (rotations, then the two-sided update).
// Output: ev (descending) and Rm (eigenvectors).
template <typename T>
__device__ __forceinline__ void jacobi_rotation(T app, T aqq, T apq, T& c, T& s) {
  c = T(1);
  s = T(0);
  if (apq != T(0)) {
    const T theta = (aqq - app) / (T(2) * apq);
    const T t = (theta >= T(0) ? T(1) : T(-1)) / (fabs(theta) + sqrt(theta * theta + T(1)));
    c = T(1) / sqrt(t * t + T(1));
    s = t * c;
  }
}
template <>
__device__ __forceinline__ void jacobi_rotation<float>(float app, float aqq, float apq, float& c, float& s) {
  c = 1.f;
  s = 0.f;
  if (apq != 0.f) {
    const float theta = __fdividef(aqq - app, 2.f * apq);
    const float t = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(fmaf(theta, theta, 1.f)));
    c = rsqrtf(fmaf(t, t, 1.f));
    s = t * c;
  }
}

template <typename T>
__global__ void k_ritz_jacobi(const ProblemDev* tab) {
  const ProblemDev& pr = tab[blockIdx.x];
  const int l = pr.l;
  if (l <= 0) return;
  __shared__ T A[2][kMaxRitz][kMaxRitz + 1];
  __shared__ T V[2][kMaxRitz][kMaxRitz + 1];
  __shared__ T cs[kMaxRitz][2];                 // (c, s) of the pair containing index x
  __shared__ int8_t partner[kMaxRitz][kMaxRitz];  // [round][x]
  __shared__ T red_off[kMaxRitz], red_tot[kMaxRitz];
  __shared__ int go_on;
  const int tid = threadIdx.x;
  const int i = tid / kMaxRitz, j = tid % kMaxRitz;
  const bool mine = i < l && j < l;
  const int m = (l + 1) & ~1;   // even count; index l is a dummy when l is odd
  if (mine) {
    const double b = 0.5 * (pr.Gm[i * l + j] + pr.Gm[j * l + i]);
    A[0][i][j] = to_t<T>(b);
    V[0][i][j] = i == j ? T(1) : T(0);
  }
  // circle method: position 0 fixed, the others rotate by one per round
  if (i < m - 1 && j < m) {
    const int round = i, x = j;
    const int pos = x == 0 ? 0 : ((x - 1 - round) % (m - 1) + (m - 1)) % (m - 1) + 1;
    const int ppos = m - 1 - pos;
    partner[round][x] = (int8_t)(ppos == 0 ? 0 : ((ppos - 1 + round) % (m - 1)) + 1);
  }
  int cur = 0;
  __syncthreads();
  // cyclic Jacobi converges quadratically; six sweeps reach FP32 rounding for
  // l <= 32 (the Ritz pairs only shape the preconditioner)
  const int max_sweeps = sizeof(T) == 4 ? 6 : 30;
  const T eps = sizeof(T) == 4 ? T(1e-11) : T(1e-30);
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    {
      // off-diagonal and total squared norms: warp i holds row i
      T v = mine ? A[cur][i][j] * A[cur][i][j] : T(0);
      T o = (mine && i != j) ? v : T(0);
#pragma unroll
      for (int sh = 16; sh > 0; sh >>= 1) {
        v += __shfl_xor_sync(0xffffffffu, v, sh);
        o += __shfl_xor_sync(0xffffffffu, o, sh);
      }
      if (j == 0) { red_tot[i] = v; red_off[i] = o; }
      __syncthreads();
      if (tid < 32) {
        T to = red_tot[tid], of = red_off[tid];
#pragma unroll
        for (int sh = 16; sh > 0; sh >>= 1) {
          to += __shfl_xor_sync(0xffffffffu, to, sh);
          of += __shfl_xor_sync(0xffffffffu, of, sh);
        }
        if (tid == 0) go_on = of > eps * to;
      }
      __syncthreads();
    }
    if (!go_on) break;
    for (int round = 0; round < m - 1; ++round) {
      if (tid < l) {
        const int x = tid, y = partner[round][x];
        if (x < y && y < l) {
          T c, s;
          jacobi_rotation<T>(A[cur][x][x], A[cur][y][y], A[cur][x][y], c, s);
          cs[x][0] = c; cs[x][1] = s;
          cs[y][0] = c; cs[y][1] = s;
        } else if (y >= l) {
          cs[x][0] = T(1); cs[x][1] = T(0);
        }
      }
      __syncthreads();
      if (mine) {
        // coefficients of row/column index u: new_u = al * X_p + be * X_q for its pair (p < q)
        auto coef = [&](int u, int& p, int& q, T& al, T& be) {
          const int v2 = partner[round][u];
          if (v2 >= l) { p = u; q = u; al = T(1); be = T(0); return; }
          const T c = cs[u][0], s = cs[u][1];
          if (u < v2) { p = u; q = v2; al = c; be = -s; }
          else { p = v2; q = u; al = s; be = c; }
        };
        int pi, qi, pj, qj;
        T ai, bi, aj, bj;
        coef(i, pi, qi, ai, bi);
        coef(j, pj, qj, aj, bj);
        const T(*Ac)[kMaxRitz + 1] = A[cur];
        T nv;
        if (pi == qi && pj == qj) nv = Ac[i][j];
        else if (pi == qi) nv = aj * Ac[i][pj] + bj * Ac[i][qj];
        else if (pj == qj) nv = ai * Ac[pi][j] + bi * Ac[qi][j];
        else nv = ai * (aj * Ac[pi][pj] + bj * Ac[pi][qj]) + bi * (aj * Ac[qi][pj] + bj * Ac[qi][qj]);
        A[1 - cur][i][j] = nv;
        V[1 - cur][i][j] = pj == qj ? V[cur][i][j] : aj * V[cur][i][pj] + bj * V[cur][i][qj];
      }
      __syncthreads();
      cur = 1 - cur;
    }
  }
  // descending order: rank of each diagonal entry
  if (tid < l) {
    const T di = A[cur][tid][tid];
    int rank = 0;
    for (int u = 0; u < l; ++u) {
      const T du = A[cur][u][u];
      rank += (du > di) || (du == di && u < tid);
    }
    pr.ev[rank] = (double)di;
    for (int u = 0; u < l; ++u) pr.Rm[u * l + rank] = (double)V[cur][u][tid];
  }
}

// One-sided (Hestenes) cyclic Jacobi for the FP32 path: one warp per column
// pair of a round (lane i holds row i), U = B, V = I initially; each round
// rotates its pairs so that their columns of U become orthogonal.  At
// convergence B V = U with orthogonal columns, so the columns of V are
// eigenvectors and lambda_c = v_c . u_c (sign kept).  Squared column norms are
// carried through the rotations (alpha' = alpha - t g, beta' = beta + t g) and
// recomputed once per sweep.
__global__ void k_ritz_jacobi_pairs(const ProblemDev* tab) {
  const ProblemDev& pr = tab[blockIdx.x];
  const int l = pr.l;
  if (l <= 0) return;
  __shared__ float U[kMaxRitz][kMaxRitz + 1], V[kMaxRitz][kMaxRitz + 1];
  __shared__ float nrm[kMaxRitz];
  __shared__ float s_scale;
  __shared__ int8_t pair_p[kMaxRitz][kMaxRitz / 2], pair_q[kMaxRitz][kMaxRitz / 2];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int e = tid; e < l * l; e += blockDim.x) {
    const int i = e / l, c = e % l;
    U[i][c] = (float)(0.5 * (pr.Gm[i * l + c] + pr.Gm[c * l + i]));
    V[i][c] = i == c ? 1.f : 0.f;
  }
  const int m = (l + 1) & ~1, npairs = m / 2;
  // round-robin schedule (circle method): slot 0 fixed, slot s > 0 holds
  // ((s - 1 + round) mod (m - 1)) + 1; pair w of a round joins slots w and m - 1 - w
  for (int e = tid; e < (m - 1) * npairs; e += blockDim.x) {
    const int round = e / npairs, w = e % npairs;
    const int s1 = w, s2 = m - 1 - w;
    int p = s1 == 0 ? 0 : ((s1 - 1 + round) % (m - 1)) + 1;
    int q = ((s2 - 1 + round) % (m - 1)) + 1;
    if (p > q) { const int x = p; p = q; q = x; }
    pair_p[round][w] = (int8_t)p;
    pair_q[round][w] = (int8_t)q;
  }
  __syncthreads();
  auto refresh_norms = [&]() {
    for (int c = warp; c < l; c += nw) {
      const float u = lane < l ? U[lane][c] : 0.f;
      float a = u * u;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      if (lane == 0) nrm[c] = a;
    }
  };
  refresh_norms();
  __syncthreads();
  if (tid == 0) {
    float mx = 0.f;
    for (int c = 0; c < l; ++c) mx = fmaxf(mx, nrm[c]);
    s_scale = mx;
  }
  __syncthreads();
  // a pair stays unconverged while the cosine of its columns exceeds 1e-5 and
  // |u_p . u_q| exceeds 2e-6 of the largest squared column norm (below that it
  // is FP32 rounding noise of the small columns)
  const float gabs = 2e-6f * s_scale;
  // four sweeps: cyclic Jacobi is quadratically convergent, and the Ritz pairs
  // only shape the preconditioner (a round costs a few hundred cycles of
  // dependent latency, so the sweep count is the cost)
  for (int sweep = 0; sweep < 4; ++sweep) {
    int busy = 0;
    for (int round = 0; round < m - 1; ++round) {
      for (int w = warp; w < npairs; w += nw) {
        const int p = pair_p[round][w], q = pair_q[round][w];
        if (q >= l) continue;
        const float up = lane < l ? U[lane][p] : 0.f, uq = lane < l ? U[lane][q] : 0.f;
        float g = up * uq;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
        const float al = nrm[p], be = nrm[q];
        if (g == 0.f) continue;
        busy |= fabsf(g) > gabs && fabsf(g) > 1e-5f * sqrtf(al * be);
        // rotation from approximate reciprocals and roots: any orthogonal rotation
        // keeps B V = U exact; these only change how fast the pair converges
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
    refresh_norms();
    if (!__syncthreads_or(busy)) break;
  }
  // eigenvalues (Rayleigh quotients) and the descending order
  __shared__ float lam[kMaxRitz];
  for (int c = warp; c < l; c += nw) {
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
    for (int u = 0; u < l; ++u) pr.Rm[u * l + rank] = (double)V[u][tid];
  }
}

// Phi = basis V_k, C Phi = image V_k (stored in T), theta = top k eigenvalues.
template <typename T>
__global__ void k_ritz_vectors(const ProblemDev* tab, int basis) {
  const ProblemDev& pr = tab[blockIdx.y];
  const int l = pr.l, k = pr.kR;
  if (k <= 0) return;
  __shared__ T Vk[kMaxRitz][kMaxK];
  for (int e = threadIdx.x; e < l * k; e += blockDim.x) Vk[e / k][e % k] = to_t<T>(pr.Rm[(e / k) * l + e % k]);
  __syncthreads();
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= pr.d) return;
  const T* Qb = ritz_buf<T>(pr, basis);
  const T* Pb = ritz_buf<T>(pr, 1 - basis);
  T* Phi = tp<T>(pr.Phi);
  T* CPhi = tp<T>(pr.CPhi);
  T q[kMaxRitz], c[kMaxRitz];
#pragma unroll
  for (int i = 0; i < kMaxRitz; ++i) {
    q[i] = i < l ? Qb[a * l + i] : T(0);
    c[i] = i < l ? Pb[a * l + i] : T(0);
  }
  for (int j = 0; j < k; ++j) {
    T ph = T(0), cp = T(0);
#pragma unroll
    for (int i = 0; i < kMaxRitz; ++i) {
      if (i < l) {
        ph += q[i] * Vk[i][j];
        cp += c[i] * Vk[i][j];
      }
    }
    Phi[a * k + j] = ph;
    CPhi[a * k + j] = cp;
  }
  if (a == 0)
    for (int j = 0; j < k; ++j) pr.theta[j] = pr.ev[j];
}

// Gram matrices of the stored Phi and A = C Phi in FP64:
// gram[0] = Phi^T Phi, gram[1] = A^T Phi, gram[2] = A^T A.  One block per entry.
template <typename T>
__global__ void k_ritz_grams(const ProblemDev* tab) {
  const ProblemDev& pr = tab[blockIdx.y];
  const int k = pr.kR;
  const int e = blockIdx.x;
  if (k <= 0 || e >= 3 * k * k) return;
  const int which = e / (k * k), i = (e / k) % k, j = e % k;
  const T* Phi = tp<const T>(pr.Phi);
  const T* A = tp<const T>(pr.CPhi);
  const T* L = which == 0 ? Phi : A;
  const T* Rr = which == 2 ? A : Phi;
  DotAcc<T> acc;
  for (int64_t a = threadIdx.x; a < pr.d; a += blockDim.x) acc.add_prod(L[a * k + i], Rr[a * k + j]);
  DotAcc<T> accs[1] = {acc};
  double out[1];
  __shared__ double scratch[2 * kThreads / 32];
  block_sum<1>(accs, out, scratch);
  if (threadIdx.x == 0) pr.gram[e] = out[0];
}

// tile = true: the BF16 block-tile path, whose C exists only as stored blocks;
// the matvec of the range finder then runs over those blocks (FP32 basis).
template <typename T>
static void launch_ritz_t(const ProblemTable& tab, const ProblemDev* dtab, cudaStream_t st, bool tile = false) {
  int64_t dl = 0, dmax = 0;
  int lmax = 0, kmax = 0;
  for (int i = 0; i < tab.count; ++i) {
    const ProblemDev& p = tab.p[i];
    dl = p.d * p.l > dl ? p.d * p.l : dl;
    dmax = p.d > dmax ? p.d : dmax;
    lmax = p.l > lmax ? p.l : lmax;
    kmax = p.kR > kmax ? p.kR : kmax;
  }
  if (lmax <= 0 || kmax <= 0) return;
  const dim3 gdl((unsigned)((dl + 255) / 256), tab.count);
  const dim3 gd((unsigned)((dmax + 255) / 256), tab.count);
  const dim3 gdw((unsigned)((dmax * 32 + 255) / 256), tab.count);   // one warp per row
  const dim3 gll((unsigned)(lmax * lmax), tab.count);
  int cur = 0;   // buffer holding the current basis candidate
  auto matvec = [&]() {   // buf[1 - cur] = C buf[cur]
    if (tile) {
      launch_tile_ritz_matvec(tab, dtab, cur, st);
      return;
    }
    k_ritz_matvec<T><<<gdw, 256, 0, st>>>(dtab, cur);
    note_launches(1);
  };
  auto orth2 = [&](int x) {   // orthonormalize buf[x] in place (scratch: the other buffer)
    k_ritz_gram<T><<<gll, 256, 0, st>>>(dtab, x, x, 1);
    k_ritz_orth<T><<<gd, 256, 0, st>>>(dtab, x);          // buf[1-x] = buf[x] R^-1
    k_ritz_gram<T><<<gll, 256, 0, st>>>(dtab, 1 - x, 1 - x, 1);
    k_ritz_orth<T><<<gd, 256, 0, st>>>(dtab, 1 - x);      // buf[x] = buf[1-x] R^-1
    note_launches(4);
  };
  k_ritz_omega<T><<<gdl, 256, 0, st>>>(dtab);               // buf0 = Omega
  note_launches(1);
  matvec();                                                 // buf1 = C buf0
  cur = 1;
  for (int it = 0; it < tab.p[0].power_iters; ++it) {
    orth2(cur);                                             // buf[cur] orthonormal
    matvec();                                               // buf[1-cur] = C buf[cur]
    cur = 1 - cur;
  }
  orth2(cur);                                               // basis in buf[cur]
  matvec();                                                 // image in buf[1-cur]
  k_ritz_gram<T><<<gll, 256, 0, st>>>(dtab, cur, 1 - cur, 0);   // Gm = Q^T (C Q)
  if (sizeof(T) == 4) k_ritz_jacobi_pairs<<<tab.count, 32 * ((lmax + 1) / 2), 0, st>>>(dtab);
  else k_ritz_jacobi<T><<<tab.count, kMaxRitz * kMaxRitz, 0, st>>>(dtab);
  k_ritz_vectors<T><<<gd, 256, 0, st>>>(dtab, cur);
  k_ritz_grams<T><<<dim3(3 * kmax * kmax, tab.count), 256, 0, st>>>(dtab);
  note_launches(4);
}

void launch_ritz(const ProblemTable& tab, const ProblemDev* dtab, cudaStream_t st) {
  if (tab.p[0].precision == 0) {
    launch_ritz_t<double>(tab, dtab, st);
    return;
  }
  if (tab.p[0].precision == 2) {
    launch_ritz_t<float>(tab, dtab, st, true);
    return;
  }
  // FP32: one cluster launch for the whole stage when every problem fits it
  bool fused = true;
  for (int i = 0; i < tab.count; ++i) {
    const ProblemDev& p = tab.p[i];
    fused &= p.l > 0 && p.kR > 0 && p.l <= kMaxRitz && p.kR <= kMaxK && ritz_cluster_fits(p.d, p.l);
  }
  if (fused && launch_ritz_cluster(tab, dtab, st) == 0) return;
  launch_ritz_t<float>(tab, dtab, st);
}

}  // namespace infoesrf
