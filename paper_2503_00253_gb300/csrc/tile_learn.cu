// Learned preconditioner correction on the BF16 path, for observations that
// fill a periodic 2-D lattice, and the Krylov capture of that path.  Not in
// the paper: its preconditioner is the limited-memory one of App. E.
//
// Lattice: the observations are exactly the points (x0 + i sx, y0 + j sy),
// i < Lx, j < Ly, of the two axes of extent > 1 of the grid, both periodic,
// with Lx sx and Ly sy the axis extents; lattice index i + Lx j.  The
// correction is M_q = a_q P_q^-1 + S_q S_q with S_q the symmetric stencil over
// the lattice offsets (dx, dy) with dx^2 + dy^2 <= 8 (the 5 x 5 square), one
// tap per squared length 0, 1, 2, 4, 5, 8 (the first kLatBins taps of the
// network's output), so S_q^T S_q = S_q S_q and M_q is SPD for a_q > 0.
//
// In the PCG (tile_pcg.cu): after the residual update, u = S r and u^T u
// (this file); rho = r^T M r = a r^T P^-1 r + u^T u; the direction update
// adds S u to a P^-1 r.  Vectors are in tile order, so S is applied through
// a table of the 25 tile positions of each row's stencil points.
#include <cuda_bf16.h>
#include <math.h>

#include "common.cuh"
#include "info_esrf.h"
#include "internal.h"

namespace infoesrf {

namespace {

constexpr int kVecThreads = 128;      // 8 systems per CTA, 16 row lanes each
constexpr int kSys = 8;
constexpr int kRowLanes = kVecThreads / kSys;
constexpr int kRows = kTileDotRows;   // rows per CTA (and per partial sum)

__device__ __forceinline__ int64_t gcd64(int64_t a, int64_t b) {
  while (b != 0) {
    const int64_t t = a % b;
    a = b;
    b = t;
  }
  return a;
}

// The two axes of extent > 1 (ax[0] < ax[1]); false unless there are exactly two.
__device__ __forceinline__ bool lattice_axes(const GridDev& g, int* ax) {
  int n = 0;
  for (int a = 0; a < 3; ++a)
    if (g.ext[a] > 1) {
      if (n < 2) ax[n] = a;
      ++n;
    }
  return n == 2;
}

__device__ __forceinline__ int64_t coord_on(const Coord3& c, int axis) {
  return axis == 0 ? c.x : (axis == 1 ? c.y : c.z);
}

// Lattice detection, one CTA per problem: origin (minimum coordinates) and
// spacings (gcd of the offsets from the origin) on the two axes; the
// observations form the lattice when the spacings divide the extents and
// the lattice has exactly d points (duplicates are caught by k_lat_map).
__global__ void __launch_bounds__(1024) k_lat_scan(const ProblemDev* tab) {
  const ProblemDev& pr = tab[blockIdx.y];
  if (pr.precision != 2 || !pr.lat_info) return;
  __shared__ int64_t red[1024];
  __shared__ int ax[2];
  __shared__ int ok;
  if (threadIdx.x == 0) {
    int a2[2] = {0, 1};
    ok = lattice_axes(pr.grid, a2) && pr.grid.periodic[a2[0]] && pr.grid.periodic[a2[1]] && pr.d > 0 &&
         pr.obs != nullptr;
    ax[0] = a2[0];
    ax[1] = a2[1];
  }
  __syncthreads();
  if (!ok) {
    if (threadIdx.x < 16) pr.lat_info[threadIdx.x] = 0;
    return;
  }
  int64_t org[2], gap[2];
  for (int w = 0; w < 2; ++w) {
    int64_t m = INT64_MAX;
    for (int64_t a = threadIdx.x; a < pr.d; a += blockDim.x) {
      const int64_t o = pr.obs[a];
      const int64_t c = (o >= 0 && o < pr.n) ? coord_on(flat_to_coord(pr.grid, o), ax[w]) : 0;
      m = c < m ? c : m;
    }
    red[threadIdx.x] = m;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if ((int)threadIdx.x < s) red[threadIdx.x] = red[threadIdx.x + s] < red[threadIdx.x] ? red[threadIdx.x + s]
                                                                                          : red[threadIdx.x];
      __syncthreads();
    }
    org[w] = red[0];
    __syncthreads();
    int64_t gg = 0;
    for (int64_t a = threadIdx.x; a < pr.d; a += blockDim.x) {
      const int64_t o = pr.obs[a];
      const int64_t c = (o >= 0 && o < pr.n) ? coord_on(flat_to_coord(pr.grid, o), ax[w]) : org[w];
      gg = gcd64(gg, c - org[w]);
    }
    red[threadIdx.x] = gg;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if ((int)threadIdx.x < s) red[threadIdx.x] = gcd64(red[threadIdx.x], red[threadIdx.x + s]);
      __syncthreads();
    }
    gap[w] = red[0];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int64_t e0 = pr.grid.ext[ax[0]], e1 = pr.grid.ext[ax[1]];
    const int64_t sx = gap[0] > 0 ? gap[0] : e0, sy = gap[1] > 0 ? gap[1] : e1;
    const bool good = e0 % sx == 0 && e1 % sy == 0 && (e0 / sx) * (e1 / sy) == pr.d;
    pr.lat_info[0] = good ? 1 : 0;
    pr.lat_info[1] = (int32_t)(e0 / sx);
    pr.lat_info[2] = (int32_t)(e1 / sy);
    pr.lat_info[3] = (int32_t)org[0];
    pr.lat_info[4] = (int32_t)org[1];
    pr.lat_info[5] = (int32_t)sx;
    pr.lat_info[6] = (int32_t)sy;
    pr.lat_info[7] = 0;
    pr.lat_info[8] = 0;
  }
}

__device__ __forceinline__ void lattice_ij(const ProblemDev& pr, int64_t obs, int64_t& i, int64_t& j) {
  int ax[2] = {0, 1};
  lattice_axes(pr.grid, ax);
  const Coord3 c = flat_to_coord(pr.grid, obs);
  i = (coord_on(c, ax[0]) - pr.lat_info[3]) / pr.lat_info[5];
  j = (coord_on(c, ax[1]) - pr.lat_info[4]) / pr.lat_info[6];
}

// lat_tpos[i + Lx j] = tile position of the observation at lattice point (i, j)
// (lat_tpos is -1 beforehand; a second observation at a point spoils the lattice).
__global__ void k_lat_map(const ProblemDev* tab) {
  const ProblemDev& pr = tab[blockIdx.y];
  if (pr.precision != 2 || !pr.lat_info || pr.lat_info[0] != 1) return;
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= pr.d) return;
  int64_t i, j;
  lattice_ij(pr, pr.obs[a], i, j);
  const int64_t Lx = pr.lat_info[1];
  const int32_t old = atomicCAS(&pr.lat_tpos[i + Lx * j], -1, pr.obs_tpos[a]);
  if (old != -1) atomicExch(&pr.lat_info[0], 0);
}

// lat_nbr[a][n] = tile position of stencil point n of tile row a (a itself at
// the padding rows, whose entries of every vector are zero).
__global__ void k_lat_nbr(const ProblemDev* tab) {
  const ProblemDev& pr = tab[blockIdx.y];
  if (pr.precision != 2 || !pr.lat_info || pr.lat_info[0] != 1) return;
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= pr.d_pad) return;
  int32_t* out = pr.lat_nbr + a * kLatPts;
  if (a >= pr.d) {
    for (int n = 0; n < kLatPts; ++n) out[n] = (int32_t)a;
    return;
  }
  int64_t i, j;
  lattice_ij(pr, pr.obs[pr.tpos_src[a]], i, j);
  const int64_t Lx = pr.lat_info[1], Ly = pr.lat_info[2];
  for (int n = 0; n < kLatPts; ++n) {
    int64_t ii = (i + lat_dx(n)) % Lx, jj = (j + lat_dy(n)) % Ly;
    ii = ii < 0 ? ii + Lx : ii;
    jj = jj < 0 ? jj + Ly : jj;
    out[n] = pr.lat_tpos[ii + Lx * jj];
  }
}

// u_j = S_j r_j on the listed learned systems (learn_on == 1), and the
// row-block partial sums of u^T u (dot value 2 k + 1).  CTA = (block of kRows
// rows, group of kSys systems), the block's stencil table staged once.
__global__ void __launch_bounds__(kVecThreads) k_tpcg_learn_u(const ProblemDev* dpr, const int32_t* list,
                                                             int64_t count) {
  const ProblemDev& pr = *dpr;
  const int64_t sb = blockIdx.x, g0 = (int64_t)blockIdx.y * kSys;
  const int64_t J = pr.nsys, dp = pr.d_pad;
  const int k = pr.kR, NVD = tile_dot_values(k);
  extern __shared__ int32_t nbr_s[];   // [kRows][kLatPts]
  __shared__ int64_t sys[kSys];
  __shared__ float taps[kSys][kLatBins];
  if (threadIdx.x < kSys) {
    const int64_t pos = g0 + threadIdx.x;
    int64_t j = pos < count ? (list ? list[pos] : pos) : J;
    if (j < J && !(pr.active[j] && pr.learn_on[j] == 1)) j = J;
    sys[threadIdx.x] = j < J ? j : -1;
    if (j < J) {
      const int64_t q = j < pr.mean_sys ? pr.Q : (j - pr.mean_sys) / pr.N;
      for (int b = 0; b < kLatBins; ++b) taps[threadIdx.x][b] = pr.learn_coef[q * kLearnOut + 1 + b];
    }
  }
  __syncthreads();
  bool any = false;
  for (int s = 0; s < kSys; ++s) any |= sys[s] >= 0;
  if (!any) return;
  const int64_t abase = sb * kRows;
  const int64_t nrow = dp - abase < kRows ? dp - abase : kRows;
  for (int64_t e = threadIdx.x; e < nrow * kLatPts; e += blockDim.x) nbr_s[e] = pr.lat_nbr[abase * kLatPts + e];
  __syncthreads();
  const int s = threadIdx.x / kRowLanes, r0 = threadIdx.x % kRowLanes;
  const int64_t j = sys[s];
  float acc = 0.f;
  if (j >= 0) {
    float w[kLatPts];
#pragma unroll
    for (int n = 0; n < kLatPts; ++n) w[n] = taps[s][lat_bin(n)];
    const float* r = pr.Rv + j * dp;
    float* u = pr.learn_u + j * dp;
    for (int64_t row = r0; row < nrow; row += kRowLanes) {
      const int32_t* nb = nbr_s + row * kLatPts;
      float v = 0.f;
#pragma unroll
      for (int n = 0; n < kLatPts; ++n) v = fmaf(w[n], __ldg(r + nb[n]), v);
      u[abase + row] = v;
      acc = fmaf(v, v, acc);
    }
  }
#pragma unroll
  for (int o = kRowLanes / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (j >= 0 && r0 == 0) pr.dots[(j * NVD + 2 * k + 1) * (int64_t)gridDim.x + sb] = (double)acc;
}

// Capture: the directions p (as the matvec used them, BF16) and images
// y = sigma p + C p of the selected systems at iteration it, in lattice order;
// zero for a system that no longer runs.
__global__ void k_tcap_record(const ProblemDev* dpr, const int32_t* sel, int nsel, int it, int K, float* V,
                              float* Y) {
  const ProblemDev& pr = *dpr;
  const int s = blockIdx.y;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsel || i >= pr.d) return;
  const int64_t j = pr.mean_sys + sel[s];
  const int64_t row = (int64_t)s * K + (it - 1);
  float v = 0.f, y = 0.f;
  if (j < pr.nsys && pr.active[j]) {
    const int64_t a = j * pr.d_pad + pr.lat_tpos[i];
    v = __bfloat162float(pr.Pdir[a]);
    y = pr.Yv[a];
  }
  V[row * pr.d + i] = v;
  Y[row * pr.d + i] = y;
}

// Capture finish, one CTA per sample: v = p / ||p||, y = y / ||p||,
// z = P_q^-1 y (App. E, the paper's preconditioner: t = T^-1 Phi^T y,
// c = (beta - sigma) t - T^-1 (g + sigma f - G_q t)) and the features.
__global__ void __launch_bounds__(256) k_tcap_finish(const ProblemDev* dpr, const int32_t* sel, int K, float* V,
                                                     float* Y, float* Z, float* feat) {
  const ProblemDev& pr = *dpr;
  const int64_t row = blockIdx.x;
  const int s = (int)(row / K);
  const int64_t d = pr.d;
  const int k = pr.kR < kMaxK ? pr.kR : kMaxK;
  const int64_t q = sel[s] / pr.N;
  const double sigma = pr.s[q] + 1.0;
  float* v = V + row * d;
  float* y = Y + row * d;
  float* z = Z + row * d;
  const float* Phi = reinterpret_cast<const float*>(pr.Phi);
  const float* A = reinterpret_cast<const float*>(pr.CPhi);
  constexpr int NV = 1 + 2 * kMaxK;
  __shared__ double red[NV][8];
  __shared__ float tco[kMaxK], cco[kMaxK];
  __shared__ double nrm;
  DotAcc<float> acc[NV];
  for (int64_t i = threadIdx.x; i < d; i += blockDim.x) {
    const float vi = v[i], yi = y[i];
    acc[0].add_prod(vi, vi);
    const int64_t a = pr.lat_tpos[i];
    for (int m = 0; m < k; ++m) {
      acc[1 + m].add_prod(Phi[a * pr.kR + m], yi);
      acc[1 + kMaxK + m].add_prod(A[a * pr.kR + m], yi);
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int e = 0; e < NV; ++e) {
    double t = acc[e].value();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) red[e][warp] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sums[NV];
    for (int e = 0; e < NV; ++e) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[e][w];
      sums[e] = t;
    }
    nrm = sums[0] > 0.0 ? sqrt(sums[0]) : 0.0;
    double t[kMaxK];
    for (int m = 0; m < k; ++m) t[m] = sums[1 + m] / (pr.theta[m] + sigma);
    const int kk = pr.kR;
    for (int m = 0; m < k; ++m) {
      double t2 = sums[1 + kMaxK + m] + sigma * sums[1 + m];
      for (int i2 = 0; i2 < k; ++i2) {
        const double G = pr.gram[2 * kk * kk + m * kk + i2] +
                         sigma * (pr.gram[kk * kk + m * kk + i2] + pr.gram[kk * kk + i2 * kk + m]) +
                         sigma * sigma * pr.gram[m * kk + i2];
        t2 -= G * t[i2];
      }
      tco[m] = (float)t[m];
      cco[m] = (float)(pr.scal[1] * t[m] - t2 / (pr.theta[m] + sigma));
    }
    float phi[4];
    learn_features(sigma, pr.scal[4] / (double)d, pr.scal[0], phi);
    for (int c = 0; c < 4; ++c) feat[row * 4 + c] = phi[c];
  }
  __syncthreads();
  const float inv = nrm > 0.0 ? (float)(1.0 / nrm) : 0.f;
  for (int64_t i = threadIdx.x; i < d; i += blockDim.x) {
    const int64_t a = pr.lat_tpos[i];
    const float yi = y[i];
    float zi = yi;
    for (int m = 0; m < k; ++m) zi += Phi[a * pr.kR + m] * cco[m] - A[a * pr.kR + m] * tco[m];
    v[i] *= inv;
    y[i] = yi * inv;
    z[i] = zi * inv;
  }
}

}  // namespace

void launch_tile_lattice(const ProblemTable& tab, const ProblemDev* dtab, cudaStream_t st) {
  int64_t dmax = 0, dpmax = 0;
  bool any = false;
  for (int i = 0; i < tab.count; ++i) {
    const ProblemDev& p = tab.p[i];
    if (p.precision != 2 || !p.lat_info) continue;
    any = true;
    dmax = p.d > dmax ? p.d : dmax;
    dpmax = p.d_pad > dpmax ? p.d_pad : dpmax;
    cudaMemsetAsync(p.lat_tpos, 0xff, (size_t)p.d * sizeof(int32_t), st);
  }
  if (!any || dmax < 1) return;
  k_lat_scan<<<dim3(1, tab.count), 1024, 0, st>>>(dtab);
  k_lat_map<<<dim3((unsigned)((dmax + 255) / 256), tab.count), 256, 0, st>>>(dtab);
  k_lat_nbr<<<dim3((unsigned)((dpmax + 255) / 256), tab.count), 256, 0, st>>>(dtab);
  note_launches(3);
}

void launch_tile_learn_u(const ProblemDev& p, const ProblemDev* dp, const int32_t* list, int64_t count, int nsub,
                         cudaStream_t st) {
  if (count < 1) return;
  static thread_local int raised = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  const int smem = kRows * kLatPts * (int)sizeof(int32_t);
  if (raised != dev) {
    cudaFuncSetAttribute(k_tpcg_learn_u, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    raised = dev;
  }
  const dim3 grid((unsigned)nsub, (unsigned)((count + kSys - 1) / kSys));
  k_tpcg_learn_u<<<grid, kVecThreads, smem, st>>>(dp, list, count);
  note_launches(1);
}

void launch_tile_capture_record(const ProblemDev& p, const ProblemDev* dp, const TileCapture& cap, int it,
                                cudaStream_t st) {
  const dim3 grid((unsigned)((p.d + 255) / 256), (unsigned)cap.nsel);
  k_tcap_record<<<grid, 256, 0, st>>>(dp, cap.sel, cap.nsel, it, cap.K, cap.V, cap.Y);
  note_launches(1);
}

void launch_tile_capture_finish(const ProblemDev& p, const ProblemDev* dp, const TileCapture& cap, float* Z,
                                float* feat, cudaStream_t st) {
  (void)p;
  k_tcap_finish<<<(unsigned)cap.nsel * cap.K, 256, 0, st>>>(dp, cap.sel, cap.K, cap.V, cap.Y, Z, feat);
  note_launches(1);
}

}  // namespace infoesrf
