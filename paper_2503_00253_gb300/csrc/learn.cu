// Learned preconditioner correction (not in the paper; the paper's
// preconditioner is the limited-memory one of App. E):
//
//     M_q = a_q P_q^-1 + S_q^T S_q,   S_q a circulant stencil over the
//     observation index with taps w_q[delta], delta = -kLearnH..kLearnH,
//
// symmetric positive definite by construction (a_q > 0).  A small network
// maps per-shift features to out, and a_q = exp(out_0) / sigma,
// w_q = out_1.. / sqrt(sigma) (relative to C_q^-1 ~ I / sigma, so that every
// shift contributes an O(1) loss):
//   phi = (log(sigma)/5, (log(sigma)/5)^2, log(mean diag C)/5, log(Gershgorin(C))/10)
//   h1 = tanh(W1 phi + b1), h2 = tanh(W2 h1 + b2), out = W3 h2 + b3.
// Parameters are one flat float vector (W1 [32][4], b1, W2 [32][32], b2,
// W3 [18][32], b3).  Training minimizes the mean over Krylov vectors v of
// ||a z + S^T S y - v||^2 / ||v||^2 with y = C_q v and z = P_q^-1 y; the
// vectors come from the method's own PCG runs (Krylov capture below).
//
// Kernels here: inference (per-shift coefficients), Krylov capture,
// per-sample loss and gradient (forward and hand-written backward through
// the stencil and the network), a fixed-order reduction over samples, Adam.
#include <math.h>

#include "common.cuh"
#include "info_esrf.h"
#include "info_esrf_stages.h"
#include "internal.h"

namespace infoesrf {

namespace {
constexpr int kHid = 32;
constexpr int kIn = 4;
constexpr int kOW1 = 0, kOB1 = kOW1 + kHid * kIn, kOW2 = kOB1 + kHid, kOB2 = kOW2 + kHid * kHid,
              kOW3 = kOB2 + kHid, kOB3 = kOW3 + kLearnOut * kHid;
static_assert(kOB3 + kLearnOut == kLearnParams, "parameter layout");
}  // namespace


// Forward pass by one thread (inference: a handful of shifts).
__device__ void learn_forward_thread(const float* th, const float* phi, float* out) {
  float h1[kHid], h2[kHid];
  for (int i = 0; i < kHid; ++i) {
    float a = th[kOB1 + i];
    for (int c = 0; c < kIn; ++c) a = fmaf(th[kOW1 + i * kIn + c], phi[c], a);
    h1[i] = tanhf(a);
  }
  for (int i = 0; i < kHid; ++i) {
    float a = th[kOB2 + i];
    for (int j = 0; j < kHid; ++j) a = fmaf(th[kOW2 + i * kHid + j], h1[j], a);
    h2[i] = tanhf(a);
  }
  for (int o = 0; o < kLearnOut; ++o) {
    float a = th[kOB3 + o];
    for (int j = 0; j < kHid; ++j) a = fmaf(th[kOW3 + o * kHid + j], h2[j], a);
    out[o] = a;
  }
}

// Forward pass by one warp (lane i computes hidden unit i; kHid = 32); the
// same sums in the same order as learn_forward_thread.  Lane o < kLearnOut
// returns out[o].
__device__ __forceinline__ float learn_forward_warp(const float* th, const float* phi, int lane) {
  static_assert(kHid == 32, "one hidden unit per lane");
  float a = th[kOB1 + lane];
  for (int c = 0; c < kIn; ++c) a = fmaf(th[kOW1 + lane * kIn + c], phi[c], a);
  const float h1 = tanhf(a);
  float b = th[kOB2 + lane];
#pragma unroll 8
  for (int j = 0; j < kHid; ++j) b = fmaf(th[kOW2 + lane * kHid + j], __shfl_sync(0xffffffffu, h1, j), b);
  const float h2 = tanhf(b);
  const int o = lane < kLearnOut ? lane : 0;
  float r = th[kOB3 + o];
#pragma unroll 8
  for (int j = 0; j < kHid; ++j) r = fmaf(th[kOW3 + o * kHid + j], __shfl_sync(0xffffffffu, h2, j), r);
  return r;
}

// Per-shift coefficients of one problem: coef[q] = (a_q, w_q[17]) for q < Q,
// slot Q for the mean system (sigma = 1).  One warp per shift.
__global__ void k_learn_coef_problem(const ProblemDev* tab) {
  const ProblemDev& pr = tab[blockIdx.y];
  if (!pr.learned_model) return;
  const int lane = threadIdx.x & 31;
  const int q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (q > pr.Q) return;
  const double sigma = q < pr.Q ? pr.s[q] + 1.0 : 1.0;
  float* cq = pr.learn_coef + (int64_t)q * kLearnOut;
  float* tq = pr.learn_T + (int64_t)q * kLearnT;
  if (pr.learned_max_shift > 0.0 && sigma > pr.learned_max_shift) {
    if (lane < kLearnOut) cq[lane] = 0.f;   // a = 0: this shift uses P_q^-1 alone
    tq[lane] = 0.f;
    if (lane == 0) tq[kLearnT - 1] = 0.f;
    return;
  }
  float phi[kIn];
  if (lane == 0) learn_features(sigma, pr.scal[4] / (double)pr.d, pr.scal[0], phi);
#pragma unroll
  for (int c = 0; c < kIn; ++c) phi[c] = __shfl_sync(0xffffffffu, phi[c], 0);
  const float out = learn_forward_warp(pr.learned_model, phi, lane);
  const float rs = rsqrtf((float)sigma);
  if (lane == 0) cq[0] = expf(out) * rs * rs;
  else if (lane < kLearnOut) cq[lane] = out * rs;
  // T = S^T S: t[D] = sum_u w[u] w[u - D], D = -2h..2h; pass 0 gives D = lane - 2h,
  // pass 1 gives D = lane + 32 - 2h (only D = 2h, on lane 0, is in range)
  const float w = lane >= 1 && lane < kLearnOut ? out * rs : 0.f;   // lane 1 + u holds w[u]
#pragma unroll
  for (int pass = 0; pass < 2; ++pass) {
    const int Dl = lane + 32 * pass - 2 * kLearnH;
    float acc = 0.f;
    for (int u = 0; u < kLearnTaps; ++u) {
      const float wu = __shfl_sync(0xffffffffu, w, 1 + u);
      const int v2 = u - Dl;
      const bool in = v2 >= 0 && v2 < kLearnTaps;
      const float wv = __shfl_sync(0xffffffffu, w, 1 + (in ? v2 : 0));
      if (in) acc = fmaf(wu, wv, acc);
    }
    if (Dl <= 2 * kLearnH) tq[Dl + 2 * kLearnH] = acc;
  }
}

void launch_learn_coef(const ProblemTable& tab, const ProblemDev* dtab, cudaStream_t st) {
  int qmax = 0;
  bool any = false;
  for (int i = 0; i < tab.count; ++i) {
    qmax = tab.p[i].Q > qmax ? tab.p[i].Q : qmax;
    any |= tab.p[i].learned_model != nullptr;
  }
  if (!any) return;
  constexpr int kWarps = 8;
  k_learn_coef_problem<<<dim3((qmax + 1 + kWarps - 1) / kWarps, tab.count), 32 * kWarps, 0, st>>>(dtab);
  note_launches(1);
}

__global__ void k_learn_coef(const float* theta, int nshift, const float* feat, float* coef) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nshift) return;
  float out[kLearnOut];
  learn_forward_thread(theta, feat + (int64_t)s * kIn, out);
  const float rs = expf(-2.5f * feat[(int64_t)s * kIn]);   // sigma^-1/2, sigma = exp(5 phi_0)
  coef[(int64_t)s * kLearnOut] = expf(out[0]) * rs * rs;
  for (int j = 1; j < kLearnOut; ++j) coef[(int64_t)s * kLearnOut + j] = out[j] * rs;
}

// ---------------------------------------------------------------------------
// Loss and gradient, one block per sample.  Vectors in dynamic shared memory.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
k_learn_loss_grad(const float* theta, int nsamp, int64_t d, const float* feat, const float* V, const float* Y,
                  const float* Z, float* G, double* sample_loss) {
  extern __shared__ __align__(16) float sm[];
  float* y = sm;
  float* z = y + d;
  float* v = z + d;
  float* u = v + d;
  float* e = u + d;
  float* se = e + d;
  __shared__ float h1[kHid], h2[kHid], out[kLearnOut], gout[kLearnOut], ga2[kHid], ga1[kHid];
  __shared__ float phi[kIn];
  __shared__ double red_scratch[2 * (3 + 2 * kLearnTaps) * (kThreads / 32)];
  const int s = blockIdx.x;
  const int tid = threadIdx.x;
  if (s >= nsamp) return;
  const float* th = theta;
  if (tid < kIn) phi[tid] = feat[(int64_t)s * kIn + tid];
  __syncthreads();
  if (tid < kHid) {
    float a = th[kOB1 + tid];
    for (int c = 0; c < kIn; ++c) a = fmaf(th[kOW1 + tid * kIn + c], phi[c], a);
    h1[tid] = tanhf(a);
  }
  __syncthreads();
  if (tid < kHid) {
    float a = th[kOB2 + tid];
    for (int j = 0; j < kHid; ++j) a = fmaf(th[kOW2 + tid * kHid + j], h1[j], a);
    h2[tid] = tanhf(a);
  }
  __syncthreads();
  if (tid < kLearnOut) {
    float a = th[kOB3 + tid];
    for (int j = 0; j < kHid; ++j) a = fmaf(th[kOW3 + tid * kHid + j], h2[j], a);
    out[tid] = a;
  }
  for (int64_t a = tid; a < d; a += blockDim.x) {
    y[a] = Y[s * d + a];
    z[a] = Z[s * d + a];
    v[a] = V[s * d + a];
  }
  __shared__ float wsc[kLearnTaps];
  const float rs = expf(-2.5f * phi[0]);       // sigma^-1/2
  if (tid < kLearnTaps) wsc[tid] = out[1 + tid] * rs;
  __syncthreads();
  const float sa = expf(out[0]) * rs * rs;
  const float* w = wsc;
  // u = S y
  for (int64_t a = tid; a < d; a += blockDim.x) {
    float acc = 0.f;
    for (int j = 0; j < kLearnTaps; ++j) {
      int64_t b = (a + j - kLearnH) % d;
      if (b < 0) b += d;
      acc = fmaf(w[j], y[b], acc);
    }
    u[a] = acc;
  }
  __syncthreads();
  // e = a z + S^T u - v
  for (int64_t a = tid; a < d; a += blockDim.x) {
    float acc = 0.f;
    for (int j = 0; j < kLearnTaps; ++j) {
      int64_t b = (a - (j - kLearnH)) % d;
      if (b < 0) b += d;
      acc = fmaf(w[j], u[b], acc);
    }
    e[a] = sa * z[a] + acc - v[a];
  }
  __syncthreads();
  // S e
  for (int64_t a = tid; a < d; a += blockDim.x) {
    float acc = 0.f;
    for (int j = 0; j < kLearnTaps; ++j) {
      int64_t b = (a + j - kLearnH) % d;
      if (b < 0) b += d;
      acc = fmaf(w[j], e[b], acc);
    }
    se[a] = acc;
  }
  __syncthreads();
  // sums: ||v||^2, ||e||^2, e.z, and per tap c1 = sum e_a u_{a-delta}, c2 = sum (Se)_b y_{b+delta}
  constexpr int NV = 3 + 2 * kLearnTaps;
  DotAcc<float> acc[NV];
  for (int64_t a = tid; a < d; a += blockDim.x) {
    acc[0].add_prod(v[a], v[a]);
    acc[1].add_prod(e[a], e[a]);
    acc[2].add_prod(e[a], z[a]);
#pragma unroll
    for (int j = 0; j < kLearnTaps; ++j) {
      const int dl = j - kLearnH;
      int64_t am = (a - dl) % d;
      if (am < 0) am += d;
      int64_t bp = (a + dl) % d;
      if (bp < 0) bp += d;
      acc[3 + j].add_prod(e[a], u[am]);
      acc[3 + kLearnTaps + j].add_prod(se[a], y[bp]);
    }
  }
  double sums[NV];
  block_sum<NV>(acc, sums, red_scratch);
  const double vv = sums[0] > 0 ? sums[0] : 1.0;
  const double scale = 2.0 / ((double)nsamp * vv);
  if (tid == 0) {
    sample_loss[s] = sums[1] / vv / (double)nsamp;
    gout[0] = (float)(scale * (double)sa * sums[2]);
  }
  if (tid < kLearnTaps) gout[1 + tid] = (float)(scale * (sums[3 + tid] + sums[3 + kLearnTaps + tid])) * rs;
  __syncthreads();
  // backward through the network
  float* g = G + (int64_t)s * kLearnParams;
  for (int e2 = tid; e2 < kLearnOut * kHid; e2 += blockDim.x) {
    const int o = e2 / kHid, j = e2 % kHid;
    g[kOW3 + e2] = gout[o] * h2[j];
  }
  if (tid < kLearnOut) g[kOB3 + tid] = gout[tid];
  if (tid < kHid) {
    float gh = 0.f;
    for (int o = 0; o < kLearnOut; ++o) gh = fmaf(th[kOW3 + o * kHid + tid], gout[o], gh);
    ga2[tid] = gh * (1.f - h2[tid] * h2[tid]);
  }
  __syncthreads();
  for (int e2 = tid; e2 < kHid * kHid; e2 += blockDim.x) {
    const int i = e2 / kHid, j = e2 % kHid;
    g[kOW2 + e2] = ga2[i] * h1[j];
  }
  if (tid < kHid) {
    g[kOB2 + tid] = ga2[tid];
    float gh = 0.f;
    for (int i = 0; i < kHid; ++i) gh = fmaf(th[kOW2 + i * kHid + tid], ga2[i], gh);
    ga1[tid] = gh * (1.f - h1[tid] * h1[tid]);
  }
  __syncthreads();
  for (int e2 = tid; e2 < kHid * kIn; e2 += blockDim.x) {
    const int i = e2 / kIn, c = e2 % kIn;
    g[kOW1 + e2] = ga1[i] * phi[c];
  }
  if (tid < kHid) g[kOB1 + tid] = ga1[tid];
}

// ---------------------------------------------------------------------------
// Loss and gradient of the 2-D lattice form (tile_learn.cu): S symmetric over
// the 5 x 5 lattice offsets with one tap per squared length, so
// e = a z + S S y - v and dL/dw_b = 2 (e^T B_b u + (S e)^T B_b y) / ||v||^2
// with u = S y and B_b the 0/1 stencil of bin b.  One block per sample;
// vectors (lattice order, i + Lx j) in global memory, u, e and S e in the
// sample's slice of tmp.
// ---------------------------------------------------------------------------
// The 25 stencil points of lattice point a = i + Lx j (periodic), nb[n]:
// a + dx + Lx dy away from the lattice edges, wrapped near them.
__device__ __forceinline__ void lat_points(int a, int Lx, int Ly, const int (&off)[kLatPts], int (&nb)[kLatPts]) {
  const int i = a % Lx, j = a / Lx;
  if (i >= 2 && i < Lx - 2 && j >= 2 && j < Ly - 2) {
#pragma unroll
    for (int n = 0; n < kLatPts; ++n) nb[n] = a + off[n];
  } else {
#pragma unroll
    for (int n = 0; n < kLatPts; ++n) {
      int ii = (i + lat_dx(n)) % Lx, jj = (j + lat_dy(n)) % Ly;
      ii = ii < 0 ? ii + Lx : ii;
      jj = jj < 0 ? jj + Ly : jj;
      nb[n] = ii + Lx * jj;
    }
  }
}

__global__ void __launch_bounds__(kThreads)
k_learn_loss_grad_lat(const float* theta, int nsamp, int Lx, int Ly, const float* feat, const float* V,
                      const float* Y, const float* Z, float* G, double* sample_loss, float* tmp) {
  __shared__ float h1[kHid], h2[kHid], out[kLearnOut], gout[kLearnOut], ga2[kHid], ga1[kHid];
  __shared__ float phi[kIn];
  __shared__ float wsc[kLatBins];
  constexpr int NV = 3 + kLatBins;
  __shared__ double red_scratch[NV * (kThreads / 32)];
  const int s = blockIdx.x;
  const int tid = threadIdx.x;
  if (s >= nsamp) return;
  const int d = Lx * Ly;   // < 2^31 (checked by the host)
  const float* th = theta;
  if (tid < kIn) phi[tid] = feat[(int64_t)s * kIn + tid];
  __syncthreads();
  if (tid < kHid) {
    float a = th[kOB1 + tid];
    for (int c = 0; c < kIn; ++c) a = fmaf(th[kOW1 + tid * kIn + c], phi[c], a);
    h1[tid] = tanhf(a);
  }
  __syncthreads();
  if (tid < kHid) {
    float a = th[kOB2 + tid];
    for (int j = 0; j < kHid; ++j) a = fmaf(th[kOW2 + tid * kHid + j], h1[j], a);
    h2[tid] = tanhf(a);
  }
  __syncthreads();
  if (tid < kLearnOut) {
    float a = th[kOB3 + tid];
    for (int j = 0; j < kHid; ++j) a = fmaf(th[kOW3 + tid * kHid + j], h2[j], a);
    out[tid] = a;
  }
  __syncthreads();
  const float rs = expf(-2.5f * phi[0]);       // sigma^-1/2
  if (tid < kLatBins) wsc[tid] = out[1 + tid] * rs;
  __syncthreads();
  const float sa = expf(out[0]) * rs * rs;
  float w[kLatPts];
  int off[kLatPts], nb[kLatPts];
#pragma unroll
  for (int n = 0; n < kLatPts; ++n) {
    w[n] = wsc[lat_bin(n)];
    off[n] = lat_dx(n) + Lx * lat_dy(n);
  }
  const float* y = Y + (int64_t)s * d;
  const float* z = Z + (int64_t)s * d;
  const float* v = V + (int64_t)s * d;
  float* u = tmp + (int64_t)s * 3 * d;
  float* e = u + d;
  float* se = e + d;
  for (int a = tid; a < d; a += blockDim.x) {   // u = S y
    lat_points(a, Lx, Ly, off, nb);
    float acc = 0.f;
#pragma unroll
    for (int n = 0; n < kLatPts; ++n) acc = fmaf(w[n], y[nb[n]], acc);
    u[a] = acc;
  }
  __syncthreads();
  for (int a = tid; a < d; a += blockDim.x) {   // e = a z + S u - v
    lat_points(a, Lx, Ly, off, nb);
    float acc = 0.f;
#pragma unroll
    for (int n = 0; n < kLatPts; ++n) acc = fmaf(w[n], u[nb[n]], acc);
    e[a] = sa * z[a] + acc - v[a];
  }
  __syncthreads();
  for (int a = tid; a < d; a += blockDim.x) {   // S e
    lat_points(a, Lx, Ly, off, nb);
    float acc = 0.f;
#pragma unroll
    for (int n = 0; n < kLatPts; ++n) acc = fmaf(w[n], e[nb[n]], acc);
    se[a] = acc;
  }
  __syncthreads();
  // ||v||^2, ||e||^2, e.z and per bin sum_{delta in bin} sum_a e_a u_{a+delta} + (S e)_a y_{a+delta}
  DotAcc<float> acc[NV];
  for (int a = tid; a < d; a += blockDim.x) {
    acc[0].add_prod(v[a], v[a]);
    acc[1].add_prod(e[a], e[a]);
    acc[2].add_prod(e[a], z[a]);
    lat_points(a, Lx, Ly, off, nb);
    float bsum[kLatBins];
#pragma unroll
    for (int b = 0; b < kLatBins; ++b) bsum[b] = 0.f;
#pragma unroll
    for (int n = 0; n < kLatPts; ++n)
      bsum[lat_bin(n)] = fmaf(e[a], u[nb[n]], fmaf(se[a], y[nb[n]], bsum[lat_bin(n)]));
#pragma unroll
    for (int b = 0; b < kLatBins; ++b) acc[3 + b].add(bsum[b]);
  }
  double sums[NV];
  block_sum<NV>(acc, sums, red_scratch);
  const double vv = sums[0] > 0 ? sums[0] : 1.0;
  const double scale = 2.0 / ((double)nsamp * vv);
  if (tid == 0) {
    sample_loss[s] = sums[0] > 0 ? sums[1] / vv / (double)nsamp : 0.0;
    gout[0] = sums[0] > 0 ? (float)(scale * (double)sa * sums[2]) : 0.f;
  }
  if (tid < kLearnTaps) gout[1 + tid] = (tid < kLatBins && sums[0] > 0) ? (float)(scale * sums[3 + tid]) * rs : 0.f;
  __syncthreads();
  // backward through the network
  float* g = G + (int64_t)s * kLearnParams;
  for (int e2 = tid; e2 < kLearnOut * kHid; e2 += blockDim.x) {
    const int o = e2 / kHid, j = e2 % kHid;
    g[kOW3 + e2] = gout[o] * h2[j];
  }
  if (tid < kLearnOut) g[kOB3 + tid] = gout[tid];
  if (tid < kHid) {
    float gh = 0.f;
    for (int o = 0; o < kLearnOut; ++o) gh = fmaf(th[kOW3 + o * kHid + tid], gout[o], gh);
    ga2[tid] = gh * (1.f - h2[tid] * h2[tid]);
  }
  __syncthreads();
  for (int e2 = tid; e2 < kHid * kHid; e2 += blockDim.x) {
    const int i = e2 / kHid, j = e2 % kHid;
    g[kOW2 + e2] = ga2[i] * h1[j];
  }
  if (tid < kHid) {
    g[kOB2 + tid] = ga2[tid];
    float gh = 0.f;
    for (int i = 0; i < kHid; ++i) gh = fmaf(th[kOW2 + i * kHid + tid], ga2[i], gh);
    ga1[tid] = gh * (1.f - h1[tid] * h1[tid]);
  }
  __syncthreads();
  for (int e2 = tid; e2 < kHid * kIn; e2 += blockDim.x) {
    const int i = e2 / kIn, c = e2 % kIn;
    g[kOW1 + e2] = ga1[i] * phi[c];
  }
  if (tid < kHid) g[kOB1 + tid] = ga1[tid];
}

// grad[p] = sum_s G[s][p] in sample order; loss = sum_s sample_loss[s].
__global__ void k_learn_reduce(int nsamp, const float* G, const double* sample_loss, float* grad, double* loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < kLearnParams) {
    float acc = 0.f;
    for (int s = 0; s < nsamp; ++s) acc += G[(int64_t)s * kLearnParams + p];
    grad[p] = acc;
  }
  if (p == 0 && loss) {
    double l = 0.0;
    for (int s = 0; s < nsamp; ++s) l += sample_loss[s];
    *loss = l;
  }
}

__global__ void k_learn_adam(float* theta, float* m, float* v, const float* grad, int step, float lr, float b1,
                             float b2, float eps) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kLearnParams) return;
  const float g = grad[p];
  const float mn = b1 * m[p] + (1.f - b1) * g;
  const float vn = b2 * v[p] + (1.f - b2) * g * g;
  m[p] = mn;
  v[p] = vn;
  const float mh = mn / (1.f - powf(b1, (float)step));
  const float vh = vn / (1.f - powf(b2, (float)step));
  theta[p] -= lr * mh / (sqrtf(vh) + eps);
}

// ---------------------------------------------------------------------------
// Krylov capture: one block per selected system runs the method's PCG (the
// limited-memory preconditioner of App. E, FP32 vectors, FP64 scalars) on the
// system's shifted matrix for K iterations and records v = p / ||p||,
// y = C_q v and z = P_q^-1 y.  The right-hand side is random (Philox keyed by
// the options' seed and the system) and is drawn again whenever the residual
// falls below 1e-6, so each selected system yields K informative directions.
// ---------------------------------------------------------------------------
template <int NV>
__device__ void block_dots(const float* a, const float* const* bs, int nb, int64_t d, double (&out)[NV],
                           double* scratch) {
  DotAcc<float> acc[NV];
  for (int64_t i = threadIdx.x; i < d; i += blockDim.x) {
    const float ai = a[i];
#pragma unroll
    for (int j = 0; j < NV; ++j)
      if (j < nb) acc[j].add_prod(ai, bs[j][i]);
  }
  block_sum<NV>(acc, out, scratch);
}

// z = P^-1 r for the shift sigma; Phi/A from the prepared problem (float).
__device__ void lmp_apply_block(const ProblemDev& pr, double sigma, const float* r, float* z, double* scratch,
                                float* tco, float* cco) {
  const int64_t d = pr.d;
  const int k = pr.kR < kMaxK ? pr.kR : kMaxK;
  const float* Phi = reinterpret_cast<const float*>(pr.Phi);
  const float* A = reinterpret_cast<const float*>(pr.CPhi);
  if (k > 0) {
    DotAcc<float> acc[2 * kMaxK];
    for (int64_t a = threadIdx.x; a < d; a += blockDim.x) {
      const float ra = r[a];
      for (int m = 0; m < k; ++m) {
        acc[m].add_prod(Phi[a * pr.kR + m], ra);
        acc[kMaxK + m].add_prod(A[a * pr.kR + m], ra);
      }
    }
    double fg[2 * kMaxK];
    block_sum<2 * kMaxK>(acc, fg, scratch);
    if (threadIdx.x == 0) {
      double t[kMaxK];
      for (int m = 0; m < k; ++m) t[m] = fg[m] / (pr.theta[m] + sigma);
      const int kk = pr.kR;
      for (int m = 0; m < k; ++m) {
        double t2 = fg[kMaxK + m] + sigma * fg[m];
        for (int i = 0; i < k; ++i) {
          const double Gm = pr.gram[2 * kk * kk + m * kk + i] +
                            sigma * (pr.gram[kk * kk + m * kk + i] + pr.gram[kk * kk + i * kk + m]) +
                            sigma * sigma * pr.gram[m * kk + i];
          t2 -= Gm * t[i];
        }
        tco[m] = (float)t[m];
        cco[m] = (float)((sigma + pr.scal[1] - sigma) * t[m] - t2 / (pr.theta[m] + sigma));
      }
    }
    __syncthreads();
  }
  for (int64_t a = threadIdx.x; a < d; a += blockDim.x) {
    float acc = r[a];
    for (int m = 0; m < k; ++m) acc += Phi[a * pr.kR + m] * cco[m] - A[a * pr.kR + m] * tco[m];
    z[a] = acc;
  }
  __syncthreads();
}

__device__ void matvec_block(const ProblemDev& pr, float sigma, const float* p, float* y) {
  const int64_t d = pr.d;
  const float* val = reinterpret_cast<const float*>(pr.oo_val);
  for (int64_t a = threadIdx.x; a < d; a += blockDim.x) {
    float acc = sigma * p[a];
    const int nnz = pr.oo_nnz[a];
    for (int e = 0; e < nnz; ++e) acc += val[(int64_t)e * d + a] * p[pr.oo_col[(int64_t)e * d + a]];
    y[a] = acc;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kThreads)
k_krylov_capture(const ProblemDev* tab, int nsel, const int32_t* sel, int K, float* V, float* Y, float* Z,
                 float* feat) {
  extern __shared__ __align__(16) float sm[];
  const ProblemDev& pr = tab[0];
  const int64_t d = pr.d, N = pr.N;
  const int s = blockIdx.x;
  if (s >= nsel) return;
  float* x = sm;
  float* r = x + d;
  float* p = r + d;
  float* y = p + d;
  float* z = y + d;
  __shared__ double scratch[2 * 2 * kMaxK * (kThreads / 32)];
  __shared__ float tco[kMaxK], cco[kMaxK];
  __shared__ double sc[4];
  const int sid = sel[s];
  const int q = (int)(sid / N);
  const double sigma = pr.s[q < pr.Q ? q : pr.Q - 1] + 1.0;
  // start (and, once converged, restart) from a random right-hand side, so that
  // every shift contributes K directions spanning its whole spectrum
  int start = 0;
  auto restart = [&]() {
    const uint64_t key = pr.seed ^ (0x9E3779B97F4A7C15ull * (uint64_t)(sid + 1)) ^ ((uint64_t)start << 48);
    for (int64_t a = threadIdx.x; a < d; a += blockDim.x) {
      x[a] = 0.f;
      r[a] = (float)philox_normal(key, (uint64_t)a);
    }
    ++start;
    __syncthreads();
    lmp_apply_block(pr, sigma, r, z, scratch, tco, cco);
    const float* bs[2] = {z, r};
    double o[2];
    block_dots<2>(r, bs, 2, d, o, scratch);
    if (threadIdx.x == 0) { sc[0] = o[0]; sc[1] = o[1]; }   // rho, ||b||^2
    for (int64_t a = threadIdx.x; a < d; a += blockDim.x) p[a] = z[a];
    __syncthreads();
  };
  restart();
  for (int it = 0; it < K; ++it) {
    matvec_block(pr, (float)sigma, p, y);
    double o2[2];
    {
      const float* bs[2] = {p, y};
      block_dots<2>(p, bs, 2, d, o2, scratch);   // p.p, p.y
    }
    const double pn = sqrt(o2[0] > 0 ? o2[0] : 1.0);
    const int64_t row = (int64_t)s * K + it;
    // record v = p/|p|, y/|p|; z = P^-1 y / |p| (z buffer reused)
    for (int64_t a = threadIdx.x; a < d; a += blockDim.x) {
      V[row * d + a] = (float)(p[a] / pn);
      Y[row * d + a] = (float)(y[a] / pn);
    }
    lmp_apply_block(pr, sigma, y, z, scratch, tco, cco);
    for (int64_t a = threadIdx.x; a < d; a += blockDim.x) Z[row * d + a] = (float)(z[a] / pn);
    if (threadIdx.x == 0) {
      float phi[kIn];
      learn_features(sigma, pr.scal[4] / (double)d, pr.scal[0], phi);
      for (int c = 0; c < kIn; ++c) feat[row * kIn + c] = phi[c];
    }
    // PCG step
    const double alpha = o2[1] > 0 ? sc[0] / o2[1] : 0.0;
    for (int64_t a = threadIdx.x; a < d; a += blockDim.x) {
      x[a] += (float)alpha * p[a];
      r[a] -= (float)alpha * y[a];
    }
    __syncthreads();
    lmp_apply_block(pr, sigma, r, z, scratch, tco, cco);
    double o1[2];
    {
      const float* bs[2] = {z, r};
      block_dots<2>(r, bs, 2, d, o1, scratch);
    }
    const bool conv = !(o1[1] > 1e-12 * sc[1]);           // ||r|| <= 1e-6 ||b||
    const double beta = sc[0] > 0 ? o1[0] / sc[0] : 0.0;
    __syncthreads();
    if (conv) {
      restart();
    } else {
      if (threadIdx.x == 0) sc[0] = o1[0];
      for (int64_t a = threadIdx.x; a < d; a += blockDim.x) p[a] = z[a] + (float)beta * p[a];
      __syncthreads();
    }
  }
}

int launch_krylov_capture(const ProblemTable& tab, const ProblemDev* dtab, int nsel, const int32_t* sel, int K,
                          float* V, float* Y, float* Z, float* feat, cudaStream_t st) {
  const size_t dyn = (size_t)5 * tab.p[0].d * sizeof(float);
  if (dyn > 200 * 1024) return INFO_ESRF_ERR_UNSUPPORTED;
  cudaFuncSetAttribute(k_krylov_capture, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  k_krylov_capture<<<nsel, kThreads, dyn, st>>>(dtab, nsel, sel, K, V, Y, Z, feat);
  note_launches(1);
  return 0;
}

}  // namespace infoesrf

using namespace infoesrf;

extern "C" {

int32_t info_esrf_learn_nparams(void) { return kLearnParams; }
int32_t info_esrf_learn_halfwidth(void) { return kLearnH; }

int info_esrf_learn_coefficients(const float* theta_dev, int32_t nshift, const float* feat_dev, float* coef_dev,
                                 void* stream) {
  if (!theta_dev || nshift < 0 || (nshift > 0 && (!feat_dev || !coef_dev))) return INFO_ESRF_ERR_INVALID_ARG;
  if (nshift == 0) return 0;
  cudaGetLastError();
  k_learn_coef<<<(nshift + 63) / 64, 64, 0, reinterpret_cast<cudaStream_t>(stream)>>>(theta_dev, nshift, feat_dev,
                                                                                     coef_dev);
  note_launches(1);
  return cudaGetLastError() == cudaSuccess ? 0 : INFO_ESRF_ERR_CUDA;
}

int info_esrf_learn_loss_grad(const float* theta_dev, int32_t nsamp, int64_t d, const float* feat_dev,
                              const float* V_dev, const float* Y_dev, const float* Z_dev, float* grad_dev,
                              double* loss_dev, void* scratch_dev, size_t scratch_bytes, void* stream) {
  if (!theta_dev || nsamp < 1 || d < 1 || !feat_dev || !V_dev || !Y_dev || !Z_dev || !grad_dev)
    return INFO_ESRF_ERR_INVALID_ARG;
  const size_t need = (size_t)nsamp * kLearnParams * sizeof(float) + (size_t)nsamp * sizeof(double);
  if (!scratch_dev || scratch_bytes < need || (reinterpret_cast<uintptr_t>(scratch_dev) % 16) != 0)
    return INFO_ESRF_ERR_WORKSPACE;
  const size_t dyn = (size_t)6 * d * sizeof(float);
  if (dyn > 200 * 1024) return INFO_ESRF_ERR_UNSUPPORTED;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  float* G = reinterpret_cast<float*>(scratch_dev);
  double* sl = reinterpret_cast<double*>(G + (size_t)nsamp * kLearnParams);
  cudaGetLastError();
  cudaFuncSetAttribute(k_learn_loss_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  k_learn_loss_grad<<<nsamp, kThreads, dyn, st>>>(theta_dev, nsamp, d, feat_dev, V_dev, Y_dev, Z_dev, G, sl);
  k_learn_reduce<<<(kLearnParams + 255) / 256, 256, 0, st>>>(nsamp, G, sl, grad_dev, loss_dev);
  note_launches(2);
  return cudaGetLastError() == cudaSuccess ? 0 : INFO_ESRF_ERR_CUDA;
}

size_t info_esrf_learn_lattice_scratch_size(int32_t nsamp, int64_t d) {
  if (nsamp < 1 || d < 1) return 0;
  return (size_t)nsamp * kLearnParams * sizeof(float) + (size_t)nsamp * sizeof(double) +
         (size_t)nsamp * 3 * (size_t)d * sizeof(float) + 512;
}

int info_esrf_learn_loss_grad_lattice(const float* theta_dev, int32_t nsamp, int32_t Lx, int32_t Ly,
                                      const float* feat_dev, const float* V_dev, const float* Y_dev,
                                      const float* Z_dev, float* grad_dev, double* loss_dev, void* scratch_dev,
                                      size_t scratch_bytes, void* stream) {
  if (!theta_dev || nsamp < 1 || Lx < 1 || Ly < 1 || !feat_dev || !V_dev || !Y_dev || !Z_dev || !grad_dev)
    return INFO_ESRF_ERR_INVALID_ARG;
  const int64_t d = (int64_t)Lx * Ly;
  if (d >= ((int64_t)1 << 31)) return INFO_ESRF_ERR_UNSUPPORTED;
  if (!scratch_dev || scratch_bytes < info_esrf_learn_lattice_scratch_size(nsamp, d) ||
      (reinterpret_cast<uintptr_t>(scratch_dev) % 16) != 0)
    return INFO_ESRF_ERR_WORKSPACE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  float* G = reinterpret_cast<float*>(scratch_dev);
  double* sl = reinterpret_cast<double*>(G + (size_t)nsamp * kLearnParams);
  uintptr_t t = reinterpret_cast<uintptr_t>(sl + nsamp);
  t = (t + 255) & ~(uintptr_t)255;
  float* tmp = reinterpret_cast<float*>(t);
  cudaGetLastError();
  k_learn_loss_grad_lat<<<nsamp, kThreads, 0, st>>>(theta_dev, nsamp, Lx, Ly, feat_dev, V_dev, Y_dev, Z_dev, G, sl,
                                                     tmp);
  k_learn_reduce<<<(kLearnParams + 255) / 256, 256, 0, st>>>(nsamp, G, sl, grad_dev, loss_dev);
  note_launches(2);
  return cudaGetLastError() == cudaSuccess ? 0 : INFO_ESRF_ERR_CUDA;
}

int info_esrf_learn_train_lattice(float* theta_dev, float* m_dev, float* v_dev, int32_t first_step, int32_t steps,
                                  float lr, int32_t nsamp, int32_t Lx, int32_t Ly, const float* feat_dev,
                                  const float* V_dev, const float* Y_dev, const float* Z_dev, float* grad_dev,
                                  double* loss_hist_dev, void* scratch_dev, size_t scratch_bytes, void* stream) {
  if (steps < 1 || first_step < 1) return INFO_ESRF_ERR_INVALID_ARG;
  for (int t = 0; t < steps; ++t) {
    int rc = info_esrf_learn_loss_grad_lattice(theta_dev, nsamp, Lx, Ly, feat_dev, V_dev, Y_dev, Z_dev, grad_dev,
                                               loss_hist_dev ? loss_hist_dev + t : nullptr, scratch_dev,
                                               scratch_bytes, stream);
    if (rc) return rc;
    rc = info_esrf_learn_adam_step(theta_dev, m_dev, v_dev, grad_dev, first_step + t, lr, stream);
    if (rc) return rc;
  }
  return 0;
}

size_t info_esrf_learn_scratch_size(int32_t nsamp) {
  return nsamp < 1 ? 0 : (size_t)nsamp * kLearnParams * sizeof(float) + (size_t)nsamp * sizeof(double) + 256;
}

int info_esrf_learn_adam_step(float* theta_dev, float* m_dev, float* v_dev, const float* grad_dev, int32_t step,
                              float lr, void* stream) {
  if (!theta_dev || !m_dev || !v_dev || !grad_dev || step < 1 || !(lr > 0.f)) return INFO_ESRF_ERR_INVALID_ARG;
  cudaGetLastError();
  k_learn_adam<<<(kLearnParams + 255) / 256, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      theta_dev, m_dev, v_dev, grad_dev, step, lr, 0.9f, 0.999f, 1e-8f);
  note_launches(1);
  return cudaGetLastError() == cudaSuccess ? 0 : INFO_ESRF_ERR_CUDA;
}

int info_esrf_learn_train(float* theta_dev, float* m_dev, float* v_dev, int32_t first_step, int32_t steps, float lr,
                          int32_t nsamp, int64_t d, const float* feat_dev, const float* V_dev, const float* Y_dev,
                          const float* Z_dev, float* grad_dev, double* loss_hist_dev, void* scratch_dev,
                          size_t scratch_bytes, void* stream) {
  if (steps < 1 || first_step < 1) return INFO_ESRF_ERR_INVALID_ARG;
  for (int t = 0; t < steps; ++t) {
    int rc = info_esrf_learn_loss_grad(theta_dev, nsamp, d, feat_dev, V_dev, Y_dev, Z_dev, grad_dev,
                                       loss_hist_dev ? loss_hist_dev + t : nullptr, scratch_dev, scratch_bytes,
                                       stream);
    if (rc) return rc;
    rc = info_esrf_learn_adam_step(theta_dev, m_dev, v_dev, grad_dev, first_step + t, lr, stream);
    if (rc) return rc;
  }
  return 0;
}

}  // extern "C"
