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

__global__ void k_write_table(const TableChunk c, ProblemDev* dst) {
  const int i = threadIdx.x;
  if (i < c.count) dst[c.first + i] = c.p[i];
}

__global__ void k_clear_scalars(ProblemDev* tab) {
  const ProblemDev& pr = tab[blockIdx.x];
  if (threadIdx.x == 0) {
    pr.scal[0] = 0.0;
    pr.scal[1] = __longlong_as_double(0x7ff0000000000000LL);  // +inf, atomically lowered
    pr.scal[2] = 0.0;
    pr.scal[3] = 0.0;
    for (int i = 0; i < 4; ++i) pr.status[i] = 0;
  }
}

void launch_prepare(const ProblemTable& tab, ProblemDev* dtab, cudaStream_t st) {
  for (int first = 0; first < tab.count; first += kChunk) {
    TableChunk c;
    c.first = first;
    c.count = tab.count - first < kChunk ? tab.count - first : kChunk;
    for (int i = 0; i < c.count; ++i) c.p[i] = tab.p[first + i];
    k_write_table<<<1, 32, 0, st>>>(c, dtab); note_launches(1);
  }
  k_clear_scalars<<<tab.count, 32, 0, st>>>(dtab); note_launches(1);
}

// ---------------------------------------------------------------------------
// a1: ensemble mean and normalized anomalies Z (Eq. normalized_perturbations)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_anomalies(const ProblemDev* tab) {
  const ProblemDev& pr = tab[blockIdx.y];
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= pr.n) return;
  const int64_t N = pr.N, n = pr.n;
  double sum = 0.0;
  bool bad = false;
  for (int64_t k = 0; k < N; ++k) {
    const double v = pr.X[k * n + x];
    bad |= !isfinite(v);
    sum += v;
  }
  const double mu = sum / (double)N;
  pr.mu[x] = mu;
  const double scale = 1.0 / pr.sqrt_nm1;
  T* Zt = tp<T>(pr.Zt);
  for (int64_t k = 0; k < N; ++k) Zt[x * N + k] = to_t<T>((pr.X[k * n + x] - mu) * scale);
  if (bad) atomicOr(&pr.status[0], kStatNonFinite);
}

// W = H Z (rows of Z at the observed points), R^-1/2 and the mean right-hand side.
template <typename T>
__global__ void k_observe(const ProblemDev* tab) {
  const ProblemDev& pr = tab[blockIdx.y];
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= pr.d) return;
  int64_t o = pr.obs[a];
  bool bad_obs = o < 0 || o >= pr.n || (a > 0 && pr.obs[a - 1] >= o);
  if (o < 0) o = 0;
  if (o >= pr.n) o = pr.n - 1;
  const double r = pr.R[a];
  const bool bad_r = !(r > 0.0) || !isfinite(r);
  const double ri = bad_r ? 0.0 : 1.0 / sqrt(r);
  pr.rinv[a] = ri;
  const T* Zt = tp<const T>(pr.Zt);
  T* W = tp<T>(pr.W);
  for (int64_t k = 0; k < pr.N; ++k) W[a * pr.N + k] = Zt[o * pr.N + k];
  if (pr.do_mean) pr.bmean[a] = ri * (pr.y[a] - pr.mu[o]);
  if (bad_obs) atomicOr(&pr.status[0], kStatBadObs);
  if (bad_r) atomicOr(&pr.status[0], kStatBadR);
}

void launch_anomalies(const ProblemTable& tab, const ProblemDev* dtab, cudaStream_t st) {
  int64_t nmax = 0, dmax = 0;
  for (int i = 0; i < tab.count; ++i) {
    nmax = tab.p[i].n > nmax ? tab.p[i].n : nmax;
    dmax = tab.p[i].d > dmax ? tab.p[i].d : dmax;
  }
  const bool f64 = tab.p[0].precision == 0;
  dim3 g1((unsigned)((nmax + 255) / 256), tab.count);
  dim3 g2((unsigned)((dmax + 255) / 256), tab.count);
  if (f64) {
    k_anomalies<double><<<g1, 256, 0, st>>>(dtab); note_launches(1);
    k_observe<double><<<g2, 256, 0, st>>>(dtab); note_launches(1);
  } else {
    k_anomalies<float><<<g1, 256, 0, st>>>(dtab); note_launches(1);
    k_observe<float><<<g2, 256, 0, st>>>(dtab); note_launches(1);
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
        const double r = scaled_distance(g, pc, bc);
        if (r < 2.0) {
          keep = true;
          DotAcc<T> acc;
          const T* wb = W + b * N;
          for (int64_t k = 0; k < N; ++k) acc.add_prod(src[k], wb[k]);
          v = gaspari_cohn(r) * acc.value();
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
        if (OBS_ROWS && b == row) atomic_min_nonneg(&pr.scal[1], v);
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

void launch_bands(const ProblemTable& tab, const ProblemDev* dtab, cudaStream_t st) {
  int64_t nmax = 0, dmax = 0;
  for (int i = 0; i < tab.count; ++i) {
    nmax = tab.p[i].n > nmax ? tab.p[i].n : nmax;
    dmax = tab.p[i].d > dmax ? tab.p[i].d : dmax;
  }
  dim3 go((unsigned)((dmax * 32 + 255) / 256), tab.count);
  dim3 gx((unsigned)((nmax * 32 + 255) / 256), tab.count);
  if (tab.p[0].precision == 0) {
    k_band<double, true><<<go, 256, 0, st>>>(dtab); note_launches(1);
    k_band<double, false><<<gx, 256, 0, st>>>(dtab); note_launches(1);
  } else {
    k_band<float, true><<<go, 256, 0, st>>>(dtab); note_launches(1);
    k_band<float, false><<<gx, 256, 0, st>>>(dtab); note_launches(1);
  }
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
// sc^2 + 1 = nc^2).  Jacobi functions by the arithmetic-geometric mean
// (descending Landen transformation, Abramowitz & Stegun 16.4); nodes past
// K/2 use sn(K - v) = cd(v), cn(K - v) = g' sd(v), dn(K - v) = g' nd(v) so that
// small cn values keep full relative precision.
// ---------------------------------------------------------------------------
__device__ double ellip_k(double m) {
  double a = 1.0, b = sqrt(1.0 - m);
  for (int i = 0; i < 64 && fabs(a - b) > 1e-16 * a; ++i) {
    const double an = 0.5 * (a + b);
    b = sqrt(a * b);
    a = an;
  }
  return kPi / (2.0 * a);
}

__device__ void ellip_jacobi(double u, double m, double& sn, double& cn, double& dn) {
  double a[40], c[40];
  a[0] = 1.0;
  c[0] = sqrt(m);
  double b = sqrt(1.0 - m);
  int nn = 0;
  while (nn < 38 && fabs(c[nn]) > 1e-17) {
    a[nn + 1] = 0.5 * (a[nn] + b);
    c[nn + 1] = 0.5 * (a[nn] - b);
    b = sqrt(a[nn] * b);
    ++nn;
  }
  double phi = ldexp(a[nn] * u, nn);
  double phi_prev = phi;
  for (int i = nn; i > 0; --i) {
    phi_prev = phi;
    phi = 0.5 * (phi + asin(c[i] * sin(phi) / a[i]));
  }
  sn = sin(phi);
  cn = cos(phi);
  dn = nn > 0 ? cn / cos(phi_prev - phi) : 1.0;
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
  const double m = ell / (1.0 + ell);
  const double kp = sqrt(1.0 / (1.0 + ell));   // complementary modulus g'
  const double K = ellip_k(m);
  const double scale = 2.0 * K / (kPi * Q);
  const double t = (q + 0.5) / Q;
  double sn, cn, dn;
  if (t <= 0.5) {
    ellip_jacobi(t * K, m, sn, cn, dn);
    s = (sn / cn) * (sn / cn);
    p = scale * dn;
  } else {
    const double v = ((Q - q) - 0.5) / Q * K;   // K - u_q, formed without cancellation
    ellip_jacobi(v, m, sn, cn, dn);
    const double sc = cn / (kp * sn);         // sc(K - v) = cd(v) / (g' sd(v))
    s = sc * sc;
    p = scale * kp / dn;                       // dn(K - v) = g' / dn(v)
  }
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
// on a range basis from Alg. 4.3 with power_iters power iterations).
// Vectors here are FP64 [d][l]; the band is read in its stored type.
// ---------------------------------------------------------------------------
__global__ void k_ritz_omega(const ProblemDev* tab) {
  const ProblemDev& pr = tab[blockIdx.y];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (pr.l <= 0 || i >= pr.d * pr.l) return;
  const int64_t a = i / pr.l, j = i % pr.l;
  pr.Om[i] = philox_normal(pr.seed, (uint64_t)(j * pr.d + a));
}

// Y[a][j] = sum_b C(a, b) V[b][j], one thread per (a, j).
template <typename T>
__global__ void k_ritz_matvec(const ProblemDev* tab, int from_om) {
  const ProblemDev& pr = tab[blockIdx.y];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (pr.l <= 0 || i >= pr.d * pr.l) return;
  const int64_t a = i / pr.l, j = i % pr.l, d = pr.d, l = pr.l;
  const double* V = from_om ? pr.Om : pr.Yb;
  double* Y = from_om ? pr.Yb : pr.Om;
  const T* val = tp<const T>(pr.oo_val);
  double acc = 0.0;
  const int nnz = pr.oo_nnz[a];
  for (int e = 0; e < nnz; ++e) acc += (double)val[e * d + a] * V[(int64_t)pr.oo_col[e * d + a] * l + j];
  Y[a * l + j] = acc;
}

// G = A^T B for [d][l] FP64 matrices, one block per (i, j) with j >= i.
__global__ void k_ritz_gram(const ProblemDev* tab, int which) {
  const ProblemDev& pr = tab[blockIdx.y];
  const int l = pr.l;
  const int pair = blockIdx.x;
  if (l <= 0 || pair >= l * l) return;
  const int i = pair / l, j = pair % l;
  if (j < i) return;
  // which: 0 -> G = Y^T Y (Y = Yb); 1 -> G = Om^T Yb
  const double* A = which == 0 ? pr.Yb : pr.Om;
  const double* B = pr.Yb;
  double acc = 0.0;
  for (int64_t a = threadIdx.x; a < pr.d; a += blockDim.x) acc += A[a * l + i] * B[a * l + j];
  __shared__ double red[32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    if (which == 1) {
      // symmetric part of Om^T C Om: (i,j) and (j,i) accumulate separately below
      pr.Gm[i * l + j] = s;
    } else {
      pr.Gm[i * l + j] = s;
      pr.Gm[j * l + i] = s;
    }
  }
}

// Lower-triangular entries (i > j) of Om^T Yb for symmetrization.
__global__ void k_ritz_gram_lower(const ProblemDev* tab) {
  const ProblemDev& pr = tab[blockIdx.y];
  const int l = pr.l;
  const int pair = blockIdx.x;
  if (l <= 0 || pair >= l * l) return;
  const int i = pair / l, j = pair % l;
  if (j >= i) return;
  double acc = 0.0;
  for (int64_t a = threadIdx.x; a < pr.d; a += blockDim.x) acc += pr.Om[a * l + i] * pr.Yb[a * l + j];
  __shared__ double red[32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    pr.Rm[i * l + j] = s;   // stash; combined in the eigensolver
  }
}

// Cholesky G = R^T R (upper R) in one thread; a non-positive pivot zeroes the
// column (rank loss) and flags kStatEigFail.
__global__ void k_ritz_cholesky(const ProblemDev* tab) {
  const ProblemDev& pr = tab[blockIdx.x];
  const int l = pr.l;
  if (threadIdx.x != 0 || l <= 0) return;
  double* G = pr.Gm;
  double* Rr = pr.Rm;
  for (int i = 0; i < l * l; ++i) Rr[i] = 0.0;
  double tr = 0.0;
  for (int i = 0; i < l; ++i) tr += G[i * l + i];
  const double tiny = 1e-28 * (tr > 0 ? tr : 1.0);
  for (int j = 0; j < l; ++j) {
    double s = G[j * l + j];
    for (int k = 0; k < j; ++k) s -= Rr[k * l + j] * Rr[k * l + j];
    if (!(s > tiny)) {
      for (int c = j; c < l; ++c) Rr[j * l + c] = 0.0;
      atomicOr(&pr.status[0], kStatEigFail);
      continue;
    }
    const double rjj = sqrt(s);
    Rr[j * l + j] = rjj;
    for (int c = j + 1; c < l; ++c) {
      double t = G[j * l + c];
      for (int k = 0; k < j; ++k) t -= Rr[k * l + j] * Rr[k * l + c];
      Rr[j * l + c] = t / rjj;
    }
  }
}

// Om[a][:] = Yb[a][:] R^-1 (row-wise forward substitution); zero pivots give zero columns.
__global__ void k_ritz_trsm(const ProblemDev* tab) {
  const ProblemDev& pr = tab[blockIdx.y];
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int l = pr.l;
  if (l <= 0 || a >= pr.d) return;
  double row[kMaxRitz];
  for (int j = 0; j < l; ++j) {
    double t = pr.Yb[a * l + j];
    for (int k = 0; k < j; ++k) t -= row[k] * pr.Rm[k * l + j];
    const double rjj = pr.Rm[j * l + j];
    row[j] = rjj > 0.0 ? t / rjj : 0.0;
  }
  for (int j = 0; j < l; ++j) pr.Om[a * l + j] = row[j];
}

// Copies Om -> Yb (so that the next orthonormalization reads Yb).
__global__ void k_ritz_copy(const ProblemDev* tab) {
  const ProblemDev& pr = tab[blockIdx.y];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (pr.l <= 0 || i >= pr.d * pr.l) return;
  pr.Yb[i] = pr.Om[i];
}

// Symmetric Jacobi eigensolver for B = (Om^T C Om + its transpose) / 2 (l x l),
// one block per problem, cyclic sweeps with l/2 disjoint rotations per round
// (round-robin ordering).  Output: ev (descending), Rm = eigenvectors (columns).
__global__ void k_ritz_jacobi(const ProblemDev* tab) {
  const ProblemDev& pr = tab[blockIdx.x];
  const int l = pr.l;
  if (l <= 0) return;
  __shared__ double A[kMaxRitz][kMaxRitz + 1];
  __shared__ double V[kMaxRitz][kMaxRitz + 1];
  __shared__ double cs[kMaxRitz / 2 + 1][2];
  __shared__ int pq[kMaxRitz / 2 + 1][2];
  __shared__ int perm[kMaxRitz + 1];
  __shared__ double off_s;
  const int tid = threadIdx.x;
  for (int i = tid; i < l * l; i += blockDim.x) {
    const int r = i / l, c = i % l;
    double v;
    if (r == c) v = pr.Gm[r * l + c];
    else if (r < c) v = 0.5 * (pr.Gm[r * l + c] + pr.Rm[c * l + r]);
    else v = 0.5 * (pr.Gm[c * l + r] + pr.Rm[r * l + c]);
    A[r][c] = v;
    V[r][c] = (r == c) ? 1.0 : 0.0;
  }
  const int m = (l + 1) & ~1;   // even count for round-robin, index l is a dummy
  if (tid < m) perm[tid] = tid;
  __syncthreads();
  for (int sweep = 0; sweep < 30; ++sweep) {
    if (tid == 0) {
      double off = 0.0, tot = 0.0;
      for (int r = 0; r < l; ++r)
        for (int c = 0; c < l; ++c) {
          const double v = A[r][c] * A[r][c];
          tot += v;
          if (r != c) off += v;
        }
      off_s = (off <= 1e-30 * tot) ? -1.0 : off;
    }
    __syncthreads();
    if (off_s < 0.0) break;
    for (int round = 0; round < m - 1; ++round) {
      const int npairs = m / 2;
      if (tid < npairs) {
        int p = perm[tid], q = perm[m - 1 - tid];
        if (p > q) { const int t = p; p = q; q = t; }
        double c = 1.0, s = 0.0;
        if (q < l && A[p][q] != 0.0) {
          const double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
          const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
          c = 1.0 / sqrt(t * t + 1.0);
          s = t * c;
        }
        pq[tid][0] = p;
        pq[tid][1] = q;
        cs[tid][0] = c;
        cs[tid][1] = s;
      }
      __syncthreads();
      // rows: A <- J^T A
      for (int i = tid; i < npairs * l; i += blockDim.x) {
        const int k = i / l, col = i % l;
        const int p = pq[k][0], q = pq[k][1];
        if (q >= l) continue;
        const double c = cs[k][0], s = cs[k][1];
        const double ap = A[p][col], aq = A[q][col];
        A[p][col] = c * ap - s * aq;
        A[q][col] = s * ap + c * aq;
      }
      __syncthreads();
      // columns: A <- A J, V <- V J
      for (int i = tid; i < npairs * l; i += blockDim.x) {
        const int k = i / l, row = i % l;
        const int p = pq[k][0], q = pq[k][1];
        if (q >= l) continue;
        const double c = cs[k][0], s = cs[k][1];
        const double ap = A[row][p], aq = A[row][q];
        A[row][p] = c * ap - s * aq;
        A[row][q] = s * ap + c * aq;
        const double vp = V[row][p], vq = V[row][q];
        V[row][p] = c * vp - s * vq;
        V[row][q] = s * vp + c * vq;
      }
      __syncthreads();
      if (tid == 0) {   // round-robin rotation keeping perm[0] fixed
        const int last = perm[m - 1];
        for (int i = m - 1; i > 1; --i) perm[i] = perm[i - 1];
        perm[1] = last;
      }
      __syncthreads();
    }
  }
  // sort eigenvalues descending (selection by one thread; l <= 32)
  if (tid == 0) {
    int order[kMaxRitz];
    bool used[kMaxRitz];
    for (int i = 0; i < l; ++i) used[i] = false;
    for (int r = 0; r < l; ++r) {
      int best = -1;
      for (int i = 0; i < l; ++i)
        if (!used[i] && (best < 0 || A[i][i] > A[best][best])) best = i;
      used[best] = true;
      order[r] = best;
    }
    for (int r = 0; r < l; ++r) {
      pr.ev[r] = A[order[r]][order[r]];
      for (int i = 0; i < l; ++i) pr.Rm[i * l + r] = V[i][order[r]];
    }
  }
}

// Phi = Om V_k, C Phi = Yb V_k (stored in T), theta = top k eigenvalues.
template <typename T>
__global__ void k_ritz_vectors(const ProblemDev* tab) {
  const ProblemDev& pr = tab[blockIdx.y];
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int l = pr.l, k = pr.kR;
  if (k <= 0 || a >= pr.d) return;
  T* Phi = tp<T>(pr.Phi);
  T* CPhi = tp<T>(pr.CPhi);
  for (int j = 0; j < k; ++j) {
    double ph = 0.0, cp = 0.0;
    for (int i = 0; i < l; ++i) {
      const double v = pr.Rm[i * l + j];
      ph += pr.Om[a * l + i] * v;
      cp += pr.Yb[a * l + i] * v;
    }
    Phi[a * k + j] = to_t<T>(ph);
    CPhi[a * k + j] = to_t<T>(cp);
  }
  if (a == 0)
    for (int j = 0; j < k; ++j) pr.theta[j] = pr.ev[j];
}

// Gram matrices of the stored (rounded) Phi and A = C Phi in FP64:
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
  double acc = 0.0;
  for (int64_t a = threadIdx.x; a < pr.d; a += blockDim.x) acc += (double)L[a * k + i] * (double)Rr[a * k + j];
  __shared__ double red[32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    pr.gram[e] = s;
  }
}

void launch_ritz(const ProblemTable& tab, const ProblemDev* dtab, cudaStream_t st) {
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
  const bool f64 = tab.p[0].precision == 0;
  const dim3 gdl((unsigned)((dl + 255) / 256), tab.count);
  const dim3 gd((unsigned)((dmax + 255) / 256), tab.count);
  const dim3 gll((unsigned)(lmax * lmax), tab.count);
  auto matvec = [&](int from_om) {
    if (f64) k_ritz_matvec<double><<<gdl, 256, 0, st>>>(dtab, from_om);
    else k_ritz_matvec<float><<<gdl, 256, 0, st>>>(dtab, from_om);
    note_launches(1);
  };
  auto orthonormalize = [&]() {   // Yb -> Om with CholeskyQR2
    for (int pass = 0; pass < 2; ++pass) {
      k_ritz_gram<<<gll, 256, 0, st>>>(dtab, 0); note_launches(1);
      k_ritz_cholesky<<<tab.count, 32, 0, st>>>(dtab); note_launches(1);
      k_ritz_trsm<<<gd, 256, 0, st>>>(dtab); note_launches(1);
      if (pass == 0) {
        k_ritz_copy<<<gdl, 256, 0, st>>>(dtab);
        note_launches(1);
      }
    }
  };
  k_ritz_omega<<<gdl, 256, 0, st>>>(dtab); note_launches(1);
  matvec(1);                                   // Yb = C Om
  int power = tab.p[0].power_iters;
  for (int it = 0; it < power; ++it) {
    orthonormalize();                          // Om = orth(Yb)
    matvec(1);                                 // Yb = C Om
  }
  orthonormalize();                            // Om = orth(Yb): range basis
  matvec(1);                                   // Yb = C Om
  k_ritz_gram<<<gll, 256, 0, st>>>(dtab, 1);   // Gm (upper) = Om^T Yb
  note_launches(1);
  k_ritz_gram_lower<<<gll, 256, 0, st>>>(dtab); note_launches(1);
  k_ritz_jacobi<<<tab.count, 128, 0, st>>>(dtab); note_launches(1);
  if (f64) {
    k_ritz_vectors<double><<<gd, 256, 0, st>>>(dtab); note_launches(1);
    k_ritz_grams<double><<<dim3(3 * kmax * kmax, tab.count), 256, 0, st>>>(dtab); note_launches(1);
  } else {
    k_ritz_vectors<float><<<gd, 256, 0, st>>>(dtab); note_launches(1);
    k_ritz_grams<float><<<dim3(3 * kmax * kmax, tab.count), 256, 0, st>>>(dtab); note_launches(1);
  }
}

}  // namespace infoesrf
