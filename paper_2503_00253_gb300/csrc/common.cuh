// Device-side building blocks shared by the InFo-ESRF kernels.
//
// Geometry and Gaspari-Cohn localization (Sec. 2.3, Sec. 5.2), the
// Philox4x32-10 generator (Salmon et al., SC'11) used by the randomized
// eigensolver of App. E, float-float accumulation for FP64-accurate dot
// products of FP32 vectors, and block reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace infoesrf {

constexpr double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------------------
// Geometry: flat index = (z * ny + y) * nx + x.
// ---------------------------------------------------------------------------
struct Coord3 {
  int64_t x, y, z;
};

__device__ __forceinline__ Coord3 flat_to_coord(const GridDev& g, int64_t idx) {
  Coord3 c;
  c.x = idx % g.ext[0];
  int64_t t = idx / g.ext[0];
  c.y = t % g.ext[1];
  c.z = t / g.ext[1];
  return c;
}

__device__ __forceinline__ double axis_distance(const GridDev& g, int ax, int64_t a, int64_t b) {
  int64_t delta = a > b ? a - b : b - a;
  const int64_t e = g.ext[ax];
  if (g.periodic[ax]) {
    if (g.chordal) return ((double)e / kPi) * sin(kPi * (double)delta / (double)e);
    return (double)(delta < e - delta ? delta : e - delta);
  }
  return (double)delta;
}

// r = sqrt(sum_axes (dist / c)^2) between two grid points.
__device__ __forceinline__ double scaled_distance(const GridDev& g, const Coord3& a, const Coord3& b) {
  double r2 = 0.0;
  const int64_t ca[3] = {a.x, a.y, a.z};
  const int64_t cb[3] = {b.x, b.y, b.z};
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    if (g.ext[ax] > 1) {
      const double dd = axis_distance(g, ax, ca[ax], cb[ax]) * g.inv_c[ax];
      r2 += dd * dd;
    }
  }
  return sqrt(r2);
}

// Gaspari & Cohn (1999) Eq. 4.10, z = distance / half-width; zero for z >= 2.
__device__ __forceinline__ double gaspari_cohn(double z) {
  z = fabs(z);
  if (z <= 1.0) {
    return (((-0.25 * z + 0.5) * z + 0.625) * z - 5.0 / 3.0) * z * z + 1.0;
  }
  if (z < 2.0) {
    return ((((z / 12.0 - 0.5) * z + 0.625) * z + 5.0 / 3.0) * z - 5.0) * z + 4.0 - (2.0 / 3.0) / z;
  }
  return 0.0;
}

// r^2 from the per-axis table tab[off_ax + |a_ax - b_ax|] = (dist_ax / c_ax)^2,
// off = (0, ext0, ext0 + ext1); filled by k_prepare with axis_distance.
__device__ __forceinline__ double scaled_r2_tab(const GridDev& g, const double* tab, const Coord3& a,
                                                const Coord3& b) {
  double r2 = 0.0;
  const int64_t ca[3] = {a.x, a.y, a.z};
  const int64_t cb[3] = {b.x, b.y, b.z};
  int64_t off = 0;
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    if (g.ext[ax] > 1) {
      const int64_t delta = ca[ax] > cb[ax] ? ca[ax] - cb[ax] : cb[ax] - ca[ax];
      r2 += tab[off + delta];
    }
    off += g.ext[ax];
  }
  return r2;
}

// Gaspari-Cohn in single precision (the FP32 path's band values).
__device__ __forceinline__ float gaspari_cohn_f(float z) {
  z = fabsf(z);
  if (z <= 1.f) return (((-0.25f * z + 0.5f) * z + 0.625f) * z - 5.f / 3.f) * z * z + 1.f;
  if (z < 2.f) return ((((z / 12.f - 0.5f) * z + 0.625f) * z + 5.f / 3.f) * z - 5.f) * z + 4.f - (2.f / 3.f) / z;
  return 0.f;
}

// First index i in sorted a[lo, hi) with a[i] >= key.
__device__ __forceinline__ int64_t lower_bound_i64(const int64_t* a, int64_t lo, int64_t hi, int64_t key) {
  while (lo < hi) {
    const int64_t mid = lo + ((hi - lo) >> 1);
    if (a[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Visits the obs-index ranges [b0, b1) whose grid points can lie inside the
// Gaspari-Cohn support of point p: one box row (z, y) at a time, with the x
// window split at the periodic seam.  Candidates are supersets; callers test
// r < 2 exactly.  f(b0, b1) is called with increasing flat index within a row.
template <typename F>
__device__ __forceinline__ void for_each_candidate_range(const GridDev& g, const int64_t* obs, int64_t d,
                                                         const Coord3& p, F&& f) {
  const int64_t nx = g.ext[0], ny = g.ext[1], nz = g.ext[2];
  const int64_t rz = g.reach[2], ry = g.reach[1], rx = g.reach[0];
  const bool wz = g.whole[2], wy = g.whole[1], wx = g.whole[0];
  const int64_t z_lo = wz ? 0 : -rz, z_hi = wz ? nz - 1 : rz;
  const int64_t y_lo = wy ? 0 : -ry, y_hi = wy ? ny - 1 : ry;
  for (int64_t iz = z_lo; iz <= z_hi; ++iz) {
    int64_t z;
    if (wz) z = iz;
    else {
      z = p.z + iz;
      if (g.periodic[2]) { z %= nz; if (z < 0) z += nz; }
      else if (z < 0 || z >= nz) continue;
    }
    for (int64_t iy = y_lo; iy <= y_hi; ++iy) {
      int64_t y;
      if (wy) y = iy;
      else {
        y = p.y + iy;
        if (g.periodic[1]) { y %= ny; if (y < 0) y += ny; }
        else if (y < 0 || y >= ny) continue;
      }
      const int64_t base = (z * ny + y) * nx;
      int64_t lo[2], hi[2];
      int nint = 0;
      if (wx) { lo[0] = 0; hi[0] = nx - 1; nint = 1; }
      else {
        const int64_t a = p.x - rx, b = p.x + rx;
        if (g.periodic[0]) {
          if (a < 0) { lo[0] = 0; hi[0] = b; lo[1] = nx + a; hi[1] = nx - 1; nint = 2; }
          else if (b >= nx) { lo[0] = 0; hi[0] = b - nx; lo[1] = a; hi[1] = nx - 1; nint = 2; }
          else { lo[0] = a; hi[0] = b; nint = 1; }
        } else {
          lo[0] = a < 0 ? 0 : a; hi[0] = b >= nx ? nx - 1 : b; nint = 1;
        }
      }
      for (int k = 0; k < nint; ++k) {
        const int64_t b0 = lower_bound_i64(obs, 0, d, base + lo[k]);
        const int64_t b1 = lower_bound_i64(obs, b0, d, base + hi[k] + 1);
        if (b1 > b0) f(b0, b1);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// Standard normals: element e comes from pair t = e / 2 (Box-Muller).
__device__ __forceinline__ double philox_normal(uint64_t seed, uint64_t e) {
  const uint64_t t = e >> 1;
  const uint4 o = philox4x32_10(make_uint4((uint32_t)t, (uint32_t)(t >> 32), 0u, 0u),
                                make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  const double u1 = ((double)o.x + 0.5) * 2.3283064365386963e-10;   // 2^-32
  const double u2 = ((double)o.y + 0.5) * 2.3283064365386963e-10;
  const double rad = sqrt(-2.0 * log(u1));
  return (e & 1) ? rad * sin(2.0 * kPi * u2) : rad * cos(2.0 * kPi * u2);
}

// Standard normals in FP32 arithmetic from the same counter scheme (the
// mixed-precision path stores the test matrix in FP32 anyway).
__device__ __forceinline__ float philox_normal_f(uint64_t seed, uint64_t e) {
  const uint64_t t = e >> 1;
  const uint4 o = philox4x32_10(make_uint4((uint32_t)t, (uint32_t)(t >> 32), 0u, 0u),
                                make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  const float u1 = fmaf((float)o.x, 2.3283064365386963e-10f, 1.1641532182693481e-10f);
  const float u2 = fmaf((float)o.y, 2.3283064365386963e-10f, 1.1641532182693481e-10f);
  const float rad = sqrtf(-2.f * logf(u1));
  float sv, cv;
  sincospif(2.f * u2, &sv, &cv);
  return (e & 1) ? rad * sv : rad * cv;
}

// Float-float arithmetic (a value is hi + lo, |lo| <= ulp(hi) / 2): about 48
// significant bits from FP32 operations (Dekker's TwoProd through fma,
// Knuth's TwoSum), used where FP64 instruction latency would dominate.
struct FF {
  float h, l;
};
__device__ __forceinline__ FF ff_norm(float s, float e) {
  const float h = s + e;
  return FF{h, e - (h - s)};
}
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
  const float p = a.h * b.h;
  const float e = fmaf(a.h, b.h, -p) + fmaf(a.h, b.l, a.l * b.h);
  return ff_norm(p, e);
}
__device__ __forceinline__ FF ff_sub(FF a, FF b) {
  const float s = a.h - b.h;
  const float v = s - a.h;
  const float e = ((a.h - (s - v)) - (b.h + v)) + (a.l - b.l);
  return ff_norm(s, e);
}
__device__ __forceinline__ FF ff_from(double x) {
  const float h = (float)x;
  return FF{h, (float)(x - (double)h)};
}
__device__ __forceinline__ FF ff_add(FF a, FF b) { return ff_sub(a, FF{-b.h, -b.l}); }
// a / b (b != 0): the FP32 quotient of the leading parts, corrected once by the
// residual a - q b formed in float-float.
__device__ __forceinline__ FF ff_div(FF a, FF b) {
  const float q1 = a.h / b.h;
  const FF r = ff_sub(a, ff_mul(FF{q1, 0.f}, b));
  return ff_norm(q1, r.h / b.h);
}
// 1 / sqrt(g) for g > 0: FP32 seed, one Newton step with the residual
// 1 - g y0^2 formed exactly enough in float-float arithmetic.
__device__ __forceinline__ FF ff_rsqrt(FF g) {
  const float y0 = rsqrtf(g.h);
  const float p = y0 * y0, pe = fmaf(y0, y0, -p);      // y0^2 = p + pe exactly
  const float t = g.h * p, te = fmaf(g.h, p, -t);      // g.h p = t + te exactly
  const float r = (1.f - t) - (te + fmaf(g.h, pe, g.l * p));
  return ff_norm(y0, 0.5f * y0 * r);
}
__device__ __forceinline__ FF ff_sqrt(FF g) { return ff_mul(g, ff_rsqrt(g)); }

// ---------------------------------------------------------------------------
// Accumulators.  For FP64 vectors a plain double sum.  For FP32 vectors a
// float-float (hi, lo) pair: products are split exactly with an FMA and
// summed with Knuth's TwoSum, so the dot product carries about 48 bits,
// without issuing FP64 instructions in the inner loop.
// ---------------------------------------------------------------------------
// Features of the learned correction's network for shift sigma (learn.cu):
// (log(sigma)/5, (log(sigma)/5)^2, log(mean diag C)/5, log(Gershgorin(C))/10),
// single-precision logarithms (features of a small network; FP64 is slow here).
__device__ __forceinline__ void learn_features(double sigma, double mean_diag, double gersh, float* phi) {
  const float ls = logf((float)sigma) * 0.2f;
  phi[0] = ls;
  phi[1] = ls * ls;
  phi[2] = logf(fmaxf((float)mean_diag, 1e-30f)) * 0.2f;
  phi[3] = logf(fmaxf((float)gersh, 1e-30f)) * 0.1f;
}

template <typename T> struct DotAcc;

template <> struct DotAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add_prod(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ void add(double a) { s += a; }
  __device__ __forceinline__ double value() const { return s; }
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

template <> struct DotAcc<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add_prod(float a, float b) {
    const float p = a * b;
    const float pe = fmaf(a, b, -p);
    float s, e;
    two_sum(hi, p, s, e);
    hi = s;
    lo += e + pe;
  }
  __device__ __forceinline__ void add(float a) {
    float s, e;
    two_sum(hi, a, s, e);
    hi = s;
    lo += e;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Combines two float-float values (hi, lo) + (h2, l2).
__device__ __forceinline__ void ff_merge(float& hi, float& lo, float h2, float l2) {
  float s, e;
  two_sum(hi, h2, s, e);
  hi = s;
  lo += e + l2;
}

// Block-wide sums of NV values per thread, results in FP64 broadcast to all
// threads.  FP32 inputs are reduced as float-float pairs.  scratch must hold
// 2 * NV * (blockDim/32) floats-or-doubles.
template <int NV>
__device__ __forceinline__ void block_sum(DotAcc<double> (&acc)[NV], double (&out)[NV], double* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    double s = acc[v].s;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) scratch[v * nw + warp] = s;
  }
  __syncthreads();
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += scratch[v * nw + w];
    out[v] = s;
  }
  __syncthreads();
}

template <int NV>
__device__ __forceinline__ void block_sum(DotAcc<float> (&acc)[NV], double (&out)[NV], double* scratch_d) {
  float* scratch = reinterpret_cast<float*>(scratch_d);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    float hi = acc[v].hi, lo = acc[v].lo;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
      const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
      ff_merge(hi, lo, h2, l2);
    }
    if (lane == 0) { scratch[2 * (v * nw + warp)] = hi; scratch[2 * (v * nw + warp) + 1] = lo; }
  }
  __syncthreads();
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    float hi = 0.f, lo = 0.f;
    for (int w = 0; w < nw; ++w) ff_merge(hi, lo, scratch[2 * (v * nw + w)], scratch[2 * (v * nw + w) + 1]);
    out[v] = (double)hi + (double)lo;
  }
  __syncthreads();
}

// Butterfly reduce-scatter of 32 values per lane: afterwards lane l holds
// the warp-wide sum of value l (31 shuffles instead of 32 x 5).
template <typename T>
__device__ __forceinline__ T warp_reduce_scatter32(T (&v)[32], int lane) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    const bool up = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < off; ++i) {
      const T send = up ? v[i] : v[i + off];
      const T keep = up ? v[i + off] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
  return v[0];
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Atomic max/min on non-negative doubles through their ordered bit patterns.
__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}
__device__ __forceinline__ void atomic_min_nonneg(double* addr, double v) {
  atomicMin(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

template <typename T> __device__ __forceinline__ T to_t(double v);
template <> __device__ __forceinline__ double to_t<double>(double v) { return v; }
template <> __device__ __forceinline__ float to_t<float>(double v) { return (float)v; }

}  // namespace infoesrf
