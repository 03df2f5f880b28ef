// Host side of the C ABI: argument checks, workspace layout, the launch
// sequence of one analysis and the optional stats read-back.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <vector>

#include "info_esrf.h"
#include "info_esrf_stages.h"
#include "internal.h"

using namespace infoesrf;

namespace infoesrf {
static std::atomic<long long> g_launches{0};
void note_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace infoesrf

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct Carver {
  char* base;        // may be null while sizing
  size_t off = 0;
  template <typename P>
  P* take(size_t bytes) {
    P* p = base ? reinterpret_cast<P*>(base + off) : nullptr;
    off = align_up(off + (bytes ? bytes : 1));
    return p;
  }
};

int num_sms_current() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 160;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
    cudaGetLastError();
    return 160;
  }
  return sms;
}

// Geometry -> device grid descriptor; candidate reach per axis.
int make_grid(const info_esrf_grid* g, GridDev* out) {
  if (!g) return INFO_ESRF_ERR_INVALID_ARG;
  memset(out, 0, sizeof(*out));
  out->chordal = g->chordal ? 1 : 0;
  for (int ax = 0; ax < 3; ++ax) {
    const int64_t e = g->shape[ax];
    if (e < 1) return INFO_ESRF_ERR_INVALID_ARG;
    out->ext[ax] = e;
    out->periodic[ax] = g->periodic[ax] ? 1 : 0;
    if (e == 1) {
      out->reach[ax] = 0;
      out->whole[ax] = 1;
      out->inv_c[ax] = 0.0;
      continue;
    }
    const double c = g->half_width[ax];
    if (!(c > 0.0) || !isfinite(c)) return INFO_ESRF_ERR_INVALID_ARG;
    out->inv_c[ax] = 1.0 / c;
    // candidates: every offset whose axis distance alone can be below 2c
    double lim = 2.0 * c;
    int64_t reach;
    if (out->periodic[ax] && out->chordal) {
      const double top = (double)e / M_PI;        // largest chordal distance
      if (lim >= top) reach = e;                  // whole axis
      else reach = (int64_t)floor((double)e / M_PI * asin(lim * M_PI / (double)e)) + 1;
    } else {
      reach = (int64_t)ceil(lim);
    }
    if (out->periodic[ax]) {
      if (2 * reach + 1 >= e) { out->whole[ax] = 1; reach = e; }
    } else if (reach >= e) {
      reach = e - 1;
    }
    out->reach[ax] = reach;
  }
  return 0;
}

int64_t geometric_bound(const GridDev& g, int64_t d) {
  double count = 1.0;
  for (int ax = 0; ax < 3; ++ax) {
    if (g.ext[ax] <= 1) continue;
    count *= g.whole[ax] ? (double)g.ext[ax] : (double)(2 * g.reach[ax] + 1);
  }
  return (int64_t)std::min<double>(count, (double)d);
}

int check_options(const info_esrf_options* in, info_esrf_options* out) {
  info_esrf_default_options(out);
  if (in) *out = *in;
  if (out->precision != 0 && out->precision != 1 && out->precision != 2) return INFO_ESRF_ERR_INVALID_ARG;
  if (out->precision == 2 && out->solver != INFO_ESRF_SOLVER_PCG) return INFO_ESRF_ERR_UNSUPPORTED;
  if (out->ritz_rank < 0 || out->ritz_rank > kMaxK) return INFO_ESRF_ERR_UNSUPPORTED;
  if (out->oversample < 0) return INFO_ESRF_ERR_INVALID_ARG;
  if (out->power_iters < 0 || out->power_iters > 8) return INFO_ESRF_ERR_INVALID_ARG;
  if (out->max_iter < 1 && out->fixed_iters <= 0) return INFO_ESRF_ERR_INVALID_ARG;
  if (out->rule != 0 && out->rule != 1) return INFO_ESRF_ERR_INVALID_ARG;
  if (out->cluster_size != 0 && out->cluster_size != -1 && out->cluster_size != 2 && out->cluster_size != 4 &&
      out->cluster_size != 8)
    return INFO_ESRF_ERR_INVALID_ARG;
  if (out->solver != INFO_ESRF_SOLVER_PCG && out->solver != INFO_ESRF_SOLVER_MULTISHIFT &&
      out->solver != INFO_ESRF_SOLVER_BLOCK)
    return INFO_ESRF_ERR_INVALID_ARG;
  return 0;
}

// Fills pr (sizes, options) and carves its workspace slice.
// Volume (cells) of a box of extents P dilated by the axis-aligned ellipsoid
// of half-axes R (Steiner formula: sum over axis subsets S of the box's
// extents outside S times the |S|-ball volume times prod R over S).
double dilated_volume(const double* P, const double* R, int na) {
  static const double omega[4] = {1.0, 2.0, M_PI, 4.0 * M_PI / 3.0};
  double vol = 0.0;
  for (int mask = 0; mask < (1 << na); ++mask) {
    double v = 1.0;
    int k = 0;
    for (int a = 0; a < na; ++a) {
      if (mask & (1 << a)) {
        v *= R[a];
        ++k;
      } else {
        v *= P[a];
      }
    }
    vol += omega[k] * v;
  }
  return vol;
}

// Estimated stored blocks per row of the BF16 path: a row tile (state = false,
// a Morton patch of kTileM observations) or a state tile (kTileM consecutive
// grid points) against column blocks (Morton patches of kTileK observations),
// for observations spread evenly at density d / n; 1.3 x plus 4 of margin.
int64_t tile_blocks_estimate(const GridDev& g, int64_t n, int64_t d, bool state) {
  const double rho = (double)d / (double)n;
  auto patch = [&](double cnt, double* e) {
    for (int ax = 0; ax < 3; ++ax) e[ax] = 1.0;
    for (int guard = 0; guard < 200; ++guard) {
      double cells = 1.0;
      for (int ax = 0; ax < 3; ++ax) cells *= e[ax];
      if (cells * rho >= cnt) break;
      int best = -1;
      for (int ax = 0; ax < 3; ++ax)
        if (g.ext[ax] > 1 && e[ax] < (double)g.ext[ax] && (best < 0 || e[ax] < e[best])) best = ax;
      if (best < 0) break;
      e[best] = std::min(2.0 * e[best], (double)g.ext[best]);
    }
  };
  double Pr[3], Pb[3];
  patch((double)kTileK, Pb);
  if (state) {
    double left = (double)kTileM;
    for (int ax = 0; ax < 3; ++ax) {
      Pr[ax] = std::min(left, (double)g.ext[ax]);
      left = std::ceil(left / (double)g.ext[ax]);
    }
  } else {
    patch((double)kTileM, Pr);
  }
  double P[3], R[3], whole = 1.0;
  int na = 0;
  for (int ax = 0; ax < 3; ++ax) {
    if (g.ext[ax] <= 1) continue;
    const double span = Pr[ax] + Pb[ax] + 2.0 * (double)g.reach[ax];
    if (g.whole[ax] || span >= (double)g.ext[ax]) {
      whole *= (double)g.ext[ax];   // the support wraps this axis: all of it
      continue;
    }
    P[na] = Pr[ax] + Pb[ax];
    R[na] = (double)g.reach[ax];
    ++na;
  }
  const double cells = whole * (na ? dilated_volume(P, R, na) : 1.0);
  return (int64_t)std::ceil(1.3 * cells * rho / (double)kTileK) + 4;
}

int64_t next_pow2(int64_t v) {
  int64_t p = 1;
  while (p < v) p <<= 1;
  return p;
}

void carve_problem(Carver& cv, ProblemDev& pr, const info_esrf_options& o) {
  const size_t esz = o.precision == 0 ? 8 : 4;
  const int64_t n = pr.n, N = pr.N, d = pr.d;
  const int l = pr.l, k = pr.kR;
  pr.mu = cv.take<double>(n * 8);
  pr.d2tab = cv.take<double>((size_t)(pr.grid.ext[0] + pr.grid.ext[1] + pr.grid.ext[2]) * 8);
  pr.Zt = cv.take<void>(n * N * esz);
  pr.W = cv.take<void>(d * N * esz);
  pr.rinv = cv.take<double>(d * 8);
  pr.bmean = cv.take<double>(d * 8);
  pr.scal = cv.take<double>(8 * 8);
  pr.status = cv.take<int32_t>(4 * 4);
  pr.s = cv.take<double>((size_t)std::max(pr.Q, 1) * 8);
  pr.p = cv.take<double>((size_t)std::max(pr.Q, 1) * 8);
  pr.oo_val = cv.take<void>((size_t)pr.max_oo * d * esz);
  pr.oo_col = cv.take<int32_t>((size_t)pr.max_oo * d * 4);
  pr.oo_nnz = cv.take<int32_t>(d * 4);
  pr.xo_val = cv.take<void>((size_t)pr.max_xo * n * esz);
  pr.xo_col = cv.take<int32_t>((size_t)pr.max_xo * n * 4);
  pr.xo_nnz = cv.take<int32_t>(n * 4);
  pr.Om = cv.take<void>((size_t)d * l * esz);
  pr.Yb = cv.take<void>((size_t)d * l * esz);
  pr.Gm = cv.take<double>((size_t)l * l * 8);
  pr.Rm = cv.take<double>((size_t)l * l * 8);
  pr.ev = cv.take<double>((size_t)l * 8);
  pr.Phi = cv.take<void>((size_t)d * k * esz);
  pr.CPhi = cv.take<void>((size_t)d * k * esz);
  pr.theta = cv.take<double>((size_t)k * 8);
  pr.gram = cv.take<double>((size_t)3 * k * k * 8);
  pr.U = cv.take<void>(o.precision == 2 ? 0 : (size_t)pr.nsys * d * esz);
  pr.iters = cv.take<int32_t>((size_t)pr.nsys * 4);
  pr.relres = cv.take<double>((size_t)pr.nsys * 8);
  pr.Vbar = cv.take<double>((size_t)d * (N + 1) * 8);
  pr.VbarT = cv.take<void>((size_t)d * (N + 1) * esz);
  pr.learn_coef = cv.take<float>((size_t)(pr.Q + 1) * kLearnOut * 4);
  pr.learn_T = cv.take<float>((size_t)(pr.Q + 1) * kLearnT * 4);
  if (o.solver == INFO_ESRF_SOLVER_BLOCK) {
    pr.bcg_nblocks = pr.mean_sys + (pr.do_pert ? pr.Q : 0);
    const size_t vec = (size_t)pr.nsys * d * esz, mat = (size_t)pr.bcg_nblocks * kBcgMaxS * kBcgMaxS * 8;
    pr.bcg_R = cv.take<void>(vec);
    pr.bcg_P = cv.take<void>(vec);
    pr.bcg_Q = cv.take<void>(vec);
    pr.bcg_G1 = cv.take<double>(mat);
    pr.bcg_G2 = cv.take<double>(mat);
    pr.bcg_RR = cv.take<double>(mat);
    pr.bcg_alpha = cv.take<double>(mat);
    pr.bcg_beta = cv.take<double>(mat);
    pr.bcg_bn2 = cv.take<double>((size_t)pr.nsys * 8);
    pr.bcg_state = cv.take<int32_t>((size_t)pr.bcg_nblocks * 4);
    pr.bcg_running = cv.take<int32_t>(4);
  }
  if (o.precision == 2) {
    const int64_t J = pr.nsys, dp = pr.d_pad, kk = pr.kR;
    const int64_t nsub = (dp + kTileDotRows - 1) / kTileDotRows;
    pr.skey = cv.take<uint64_t>((size_t)pr.nsort * 8);
    pr.sidx = cv.take<int32_t>((size_t)pr.nsort * 4);
    pr.tpos_src = cv.take<int32_t>((size_t)dp * 4);
    pr.obs_tpos = cv.take<int32_t>((size_t)pr.d * 4);
    pr.tbox = cv.take<int32_t>((size_t)pr.nblk * 6 * 4);
    pr.tcount = cv.take<int32_t>((size_t)(pr.nrt + pr.nst) * 4);
    pr.rowptr = cv.take<int32_t>((size_t)(pr.nrt + 1) * 4);
    pr.colblk = cv.take<int32_t>((size_t)pr.tile_cap * 4);
    pr.st_rowptr = cv.take<int32_t>((size_t)(pr.nst + 1) * 4);
    pr.st_colblk = cv.take<int32_t>((size_t)pr.st_cap * 4);
    pr.Chi = cv.take<__nv_bfloat16>((size_t)pr.tile_cap * kTileM * kTileK * 2);
    pr.Clo = cv.take<__nv_bfloat16>((size_t)pr.tile_cap * kTileM * kTileK * 2);
    pr.Wp = cv.take<float>((size_t)dp * N * 4);
    pr.rinvp = cv.take<float>((size_t)dp * 4);
    pr.Pdir = cv.take<__nv_bfloat16>((size_t)J * dp * 2);
    pr.Yv = cv.take<float>((size_t)J * dp * 4);
    pr.Xv = cv.take<float>((size_t)J * dp * 4);
    pr.Rv = cv.take<float>((size_t)J * dp * 4);
    pr.pty = cv.take<float>((size_t)pr.nrt * J * 4);
    pr.dots = cv.take<double>((size_t)nsub * J * tile_dot_values((int)kk) * 8);
    pr.dsum = cv.take<double>((size_t)J * tile_dot_values((int)kk) * 8);
    pr.sysd = cv.take<double>((size_t)J * 8 * 8);
    pr.lcoef = cv.take<float>((size_t)J * 2 * kMaxK * 4);
    pr.sigmaf = cv.take<float>((size_t)J * 4);
    pr.active = cv.take<int32_t>((size_t)J * 4);
    pr.unit_active = cv.take<int32_t>((size_t)((J + kTileUnit - 1) / kTileUnit) * 4);
    pr.unit_list = cv.take<int32_t>((size_t)((J + kTileUnit - 1) / kTileUnit) * 4);
    pr.nactive = cv.take<int32_t>(4 * 4);
    pr.alist = cv.take<int32_t>((size_t)J * 4);
    // operand planes of the tensor-core state update (tile_state.cu)
    pr.st_NV = (int32_t)((N + 15) / 16 * 16);
    pr.st_W = cv.take<__nv_bfloat16>((size_t)3 * dp * kStK * 2);
    pr.st_V = cv.take<__nv_bfloat16>((size_t)2 * pr.st_NV * dp * 2);
    pr.st_vm = cv.take<float>((size_t)dp * 4);
    pr.st_xyz = cv.take<int4>((size_t)dp * 16);
    // observation lattice and the learned term's vectors (tile_learn.cu)
    pr.lat_info = cv.take<int32_t>(16 * 4);
    pr.lat_tpos = cv.take<int32_t>((size_t)pr.d * 4);
    pr.lat_nbr = cv.take<int32_t>((size_t)dp * kLatPts * 4);
    if (o.learned_model) {
      pr.learn_u = cv.take<float>((size_t)J * dp * 4);
      pr.learn_on = cv.take<int32_t>((size_t)J * 4);
    }
  }
}

// Builds the host table for a batch; with ws == nullptr only sizes it.
int build_table(const info_esrf_problem* probs, int32_t count, const info_esrf_options& o, void* ws,
                ProblemTable& tab, size_t* bytes_out, ProblemDev** dtab_out, int32_t** counter_out,
                void** scratch_out, size_t* scratch_bytes_out, int num_sms) {
  if (count < 1) return INFO_ESRF_ERR_INVALID_ARG;
  if (count > kMaxProblems) return INFO_ESRF_ERR_UNSUPPORTED;
  memset(&tab, 0, sizeof(tab));
  tab.count = count;
  tab.cluster_size = o.cluster_size;
  Carver cv{reinterpret_cast<char*>(ws)};
  ProblemDev* dtab = cv.take<ProblemDev>(sizeof(ProblemDev) * count);
  int32_t* counter = cv.take<int32_t>(kCounterInts * sizeof(int32_t));
  int group_base = 0, sys_base = 0;
  const int JT = pcg_jt(o.precision);
  for (int i = 0; i < count; ++i) {
    const info_esrf_problem& P = probs[i];
    ProblemDev& pr = tab.p[i];
    int rc = make_grid(&P.grid, &pr.grid);
    if (rc) return rc;
    pr.n = P.grid.shape[0] * P.grid.shape[1] * P.grid.shape[2];
    pr.N = P.N;
    pr.d = P.d;
    pr.do_mean = P.mu_a != nullptr;
    pr.do_pert = P.A_a != nullptr;
    if (!pr.do_mean && !pr.do_pert) return INFO_ESRF_ERR_INVALID_ARG;
    if (pr.N < 2 || pr.d < 1 || pr.n < 1 || pr.d > pr.n) return INFO_ESRF_ERR_INVALID_ARG;
    if (pr.n > INT32_MAX || pr.d > INT32_MAX) return INFO_ESRF_ERR_UNSUPPORTED;
    pr.Q = pr.do_pert ? P.Q : 0;
    if (pr.do_pert && P.Q < 1) return INFO_ESRF_ERR_INVALID_ARG;
    if (o.fixed_iters <= 0 && !(P.tol > 0.0)) return INFO_ESRF_ERR_INVALID_ARG;
    const bool general_h = P.H_rowptr != nullptr;
    if (!P.X || (!P.obs_idx && !general_h) || !P.R_diag || (pr.do_mean && !P.y)) return INFO_ESRF_ERR_INVALID_ARG;
    if (general_h && (!P.H_col || !P.H_val || P.H_nnz < 0)) return INFO_ESRF_ERR_INVALID_ARG;
    pr.tol = P.tol;
    pr.kR = (int32_t)std::min<int64_t>(o.ritz_rank, pr.d);
    pr.l = pr.kR > 0 ? (int32_t)std::min<int64_t>(std::min<int64_t>(pr.kR + o.oversample, kMaxRitz), pr.d) : 0;
    pr.rule = o.rule;
    pr.precision = o.precision;
    pr.fixed_iters = o.fixed_iters;
    pr.max_iter = o.max_iter;
    pr.power_iters = o.power_iters;
    pr.learned_model = o.learned_model;
    pr.learned_max_shift = o.learned_max_shift;
    pr.ell_fixed = o.ell;
    pr.seed = o.seed;
    pr.sqrt_nm1 = sqrt((double)(pr.N - 1));
    if (o.solver == INFO_ESRF_SOLVER_BLOCK && pr.do_pert && pr.N > kBcgMaxS) return INFO_ESRF_ERR_UNSUPPORTED;
    if (o.precision == 2) {
      // BF16 block-tile path: no bands; tile counts and capacities
      if (general_h || pr.N > tile_max_members()) return INFO_ESRF_ERR_UNSUPPORTED;
      pr.max_oo = 0;
      pr.max_xo = 0;
      pr.d_pad = (pr.d + kTileM - 1) / kTileM * kTileM;
      pr.nrt = (int32_t)(pr.d_pad / kTileM);
      pr.nblk = (int32_t)(pr.d_pad / kTileK);
      pr.nst = (int32_t)((pr.n + kTileM - 1) / kTileM);
      pr.nsort = std::max<int64_t>(1024, next_pow2(pr.d));
      const int64_t est_c = std::min<int64_t>(pr.nblk, tile_blocks_estimate(pr.grid, pr.n, pr.d, false));
      const int64_t est_s = std::min<int64_t>(pr.nblk, tile_blocks_estimate(pr.grid, pr.n, pr.d, true));
      pr.tile_cap = o.tile_capacity > 0 ? o.tile_capacity : (int64_t)pr.nrt * est_c;
      pr.st_cap = o.state_tile_capacity > 0 ? o.state_tile_capacity : (int64_t)pr.nst * est_s;
      pr.tile_cap = std::max<int64_t>(pr.tile_cap, pr.nrt);
      pr.st_cap = std::max<int64_t>(pr.st_cap, 1);
      if (pr.tile_cap * kTileM >= (int64_t(1) << 31) || pr.st_cap >= INT32_MAX) return INFO_ESRF_ERR_UNSUPPORTED;
    } else if (general_h) {
      // dense covariances: every row of C and of Sxh holds all d columns
      if (pr.n * pr.d > (int64_t(1) << 28)) return INFO_ESRF_ERR_UNSUPPORTED;
      pr.max_oo = pr.d;
      pr.max_xo = pr.d;
    } else {
      const int64_t gb = geometric_bound(pr.grid, pr.d);
      int64_t cap_oo = P.max_oo > 0 ? P.max_oo : (o.max_neighbors > 0 ? o.max_neighbors : gb);
      int64_t cap_xo = P.max_xo > 0 ? P.max_xo : (o.max_neighbors > 0 ? o.max_neighbors : gb);
      pr.max_oo = std::min(cap_oo, pr.d);
      pr.max_xo = std::min(cap_xo, pr.d);
    }
    pr.X = P.X;
    pr.obs = general_h ? nullptr : P.obs_idx;
    pr.H_rowptr = P.H_rowptr;
    pr.H_col = general_h ? P.H_col : nullptr;
    pr.H_val = general_h ? P.H_val : nullptr;
    pr.H_nnz = general_h ? P.H_nnz : 0;
    pr.y = P.y;
    pr.R = P.R_diag;
    pr.mu_a = P.mu_a;
    pr.A_a = P.A_a;
    pr.JT = JT;
    pr.groups_per_q = (int32_t)((pr.N + JT - 1) / JT);
    pr.num_groups = (pr.do_pert ? pr.Q * pr.groups_per_q : 0) + (pr.do_mean ? 1 : 0);
    pr.group_base = group_base;
    group_base += pr.num_groups;
    pr.mean_sys = pr.do_mean ? 1 : 0;
    pr.nsys = pr.mean_sys + (pr.do_pert ? pr.Q * (int32_t)pr.N : 0);
    pr.sys_base = sys_base;
    sys_base += pr.nsys;
    carve_problem(cv, pr, o);
  }
  tab.total_groups = group_base;
  tab.total_sys = sys_base;
  tab.solver = o.solver;
  const size_t sb = o.solver == INFO_ESRF_SOLVER_PCG ? pcg_scratch_bytes(tab, num_sms) : 0;
  void* scratch = cv.take<void>(sb);
  if (o.solver == INFO_ESRF_SOLVER_MULTISHIFT) {
    if (mscg_plan(tab, num_sms, o.cluster_size, &tab.ms) != 0) return INFO_ESRF_ERR_UNSUPPORTED;
    tab.ms_scratch = tab.ms.scratch_bytes ? cv.take<void>(tab.ms.scratch_bytes) : nullptr;
  }
  *bytes_out = cv.off;
  if (dtab_out) *dtab_out = dtab;
  if (counter_out) *counter_out = counter;
  if (scratch_out) *scratch_out = scratch;
  if (scratch_bytes_out) *scratch_bytes_out = sb;
  return 0;
}

int status_to_code(int32_t bits) {
  if (bits & kStatBadObs) return INFO_ESRF_ERR_BAD_OBS_INDEX;
  if (bits & kStatBadR) return INFO_ESRF_ERR_NONPOSITIVE_R;
  if (bits & kStatNonFinite) return INFO_ESRF_ERR_NONFINITE;
  if (bits & kStatBandOverflow) return INFO_ESRF_ERR_BAND_OVERFLOW;
  if (bits & kStatTimeout) return INFO_ESRF_ERR_TIMEOUT;
  if (bits & kStatTileOverflow) return INFO_ESRF_ERR_BAND_OVERFLOW;
  if (bits & kStatBreakdown) return INFO_ESRF_ERR_BREAKDOWN;
  if (bits & kStatNotConverged) return INFO_ESRF_NOT_CONVERGED;
  return INFO_ESRF_OK;
}

// Side stream and events, per host thread and device, for the work that
// overlaps the main sequence: the quadrature and the state-obs band run while
// the Ritz pairs are computed.  Created on first use and kept for the life of
// the thread (like a library handle).
struct AuxStream {
  cudaStream_t s = nullptr;
  cudaEvent_t mid = nullptr, jq = nullptr, jb = nullptr;
};

AuxStream* aux_stream() {
  constexpr int kMaxDev = 64;
  static thread_local AuxStream aux[kMaxDev];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
    cudaGetLastError();
    return nullptr;
  }
  AuxStream& a = aux[dev];
  if (!a.s) {
    cudaStream_t s = nullptr;
    cudaEvent_t e[3] = {nullptr, nullptr, nullptr};
    bool ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess;
    for (int i = 0; i < 3 && ok; ++i) ok = cudaEventCreateWithFlags(&e[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      for (int i = 0; i < 3; ++i)
        if (e[i]) cudaEventDestroy(e[i]);
      if (s) cudaStreamDestroy(s);
      return nullptr;
    }
    a.s = s;
    a.mid = e[0];
    a.jq = e[1];
    a.jb = e[2];
  }
  return &a;
}

int run_batch(const info_esrf_problem* probs, int32_t count, const info_esrf_options* opt_in, void* ws,
              size_t ws_bytes, void* stream, info_esrf_stats* stats) {
  info_esrf_options o;
  int rc = check_options(opt_in, &o);
  if (rc) return rc;
  if (!ws || (reinterpret_cast<uintptr_t>(ws) % kAlign) != 0) return INFO_ESRF_ERR_WORKSPACE;
  const int sms = num_sms_current();
  static thread_local ProblemTable tab;   // large; keep it off the stack
  size_t need = 0;
  ProblemDev* dtab = nullptr;
  int32_t* counter = nullptr;
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  rc = build_table(probs, count, o, ws, tab, &need, &dtab, &counter, &scratch, &scratch_bytes, sms);
  if (rc) return rc;
  if (need > ws_bytes) return INFO_ESRF_ERR_WORKSPACE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaGetLastError();
  auto mark = [&](int i) {
    if (o.phase_events && o.phase_events[i]) cudaEventRecord(reinterpret_cast<cudaEvent_t>(o.phase_events[i]), st);
  };
  static thread_local double tile_mm_ms[kMaxProblems];
  static thread_local int tile_mm_n[kMaxProblems];
  for (int i = 0; i < count; ++i) {
    tile_mm_ms[i] = 0.0;
    tile_mm_n[i] = 0;
  }
  mark(0);
  launch_prepare(tab, dtab, st);
  launch_anomalies(tab, dtab, st);
  if (o.precision == INFO_ESRF_PRECISION_BF16) {
    // block-tile path: tile order and C blocks, quadrature, Ritz pairs over
    // the blocks, then each problem's PCG loop (host-driven) and the finish
    launch_tile_setup(tab, dtab, st);
    launch_quadrature(tab, dtab, st);
    if (o.learned_model) {
      // learned term on 2-D observation lattices: per-shift coefficients and
      // the lattice's stencil tables
      launch_learn_coef(tab, dtab, st);
      launch_tile_lattice(tab, dtab, st);
    }
    mark(1);
    launch_ritz(tab, dtab, st);
    mark(2);
    for (int i = 0; i < count; ++i) {
      const int r = run_tile_pcg(tab.p[i], dtab + i, st, stats ? &tile_mm_ms[i] : nullptr,
                                 stats ? &tile_mm_n[i] : nullptr);
      if (r != 0) return r;
    }
    mark(3);
    launch_tile_finish(tab, dtab, st);
  } else if (o.solver == INFO_ESRF_SOLVER_BLOCK) {
    // block CG: bands and quadrature, no Ritz stage, then each problem's
    // host-driven block iteration, then the usual finish from U
    launch_band_obs(tab, dtab, st);
    launch_band_state(tab, dtab, st);
    launch_quadrature(tab, dtab, st);
    mark(1);
    mark(2);
    for (int i = 0; i < count; ++i) {
      const int r = run_bcg(tab.p[i], dtab + i, st);
      if (r != 0) return r;
    }
    mark(3);
    launch_finish(tab, dtab, st);
  } else if (o.solver == INFO_ESRF_SOLVER_MULTISHIFT) {
    launch_band_obs(tab, dtab, st);
    // no Ritz stage and no learned coefficients: the quadrature and the
    // state-obs band run on the side stream while nothing else waits
    AuxStream* aux = aux_stream();
    if (aux) {
      cudaEventRecord(aux->mid, st);
      cudaStreamWaitEvent(aux->s, aux->mid, 0);
      launch_band_state(tab, dtab, aux->s);
      cudaEventRecord(aux->jb, aux->s);
    } else {
      launch_band_state(tab, dtab, st);
    }
    launch_quadrature(tab, dtab, st);
    mark(1);
    mark(2);
    if (launch_mscg(tab, dtab, tab.ms, sms, st) != 0) {
      if (aux) cudaStreamWaitEvent(st, aux->jb, 0);
      return INFO_ESRF_ERR_CUDA;
    }
    mark(3);
    if (aux) cudaStreamWaitEvent(st, aux->jb, 0);
    launch_finish(tab, dtab, st, false);
  } else {
    launch_band_obs(tab, dtab, st);
    // the quadrature and the state-obs band overlap the Ritz stage on a side
    // stream, which rejoins before the first use of each
    AuxStream* aux = aux_stream();
    // the learned coefficients need only the quadrature and the band's scalars
    if (aux) {
      cudaEventRecord(aux->mid, st);
      cudaStreamWaitEvent(aux->s, aux->mid, 0);
      launch_quadrature(tab, dtab, aux->s);
      launch_learn_coef(tab, dtab, aux->s);
      cudaEventRecord(aux->jq, aux->s);
      launch_band_state(tab, dtab, aux->s);
      cudaEventRecord(aux->jb, aux->s);
    } else {
      launch_quadrature(tab, dtab, st);
      launch_learn_coef(tab, dtab, st);
      launch_band_state(tab, dtab, st);
    }
    mark(1);
    launch_ritz(tab, dtab, st);
    if (aux) cudaStreamWaitEvent(st, aux->jq, 0);
    mark(2);
    if (launch_pcg(tab, dtab, counter, scratch, scratch_bytes, sms, st) != 0) {
      if (aux) cudaStreamWaitEvent(st, aux->jb, 0);
      return INFO_ESRF_ERR_WORKSPACE;
    }
    mark(3);
    if (aux) cudaStreamWaitEvent(st, aux->jb, 0);
    launch_finish(tab, dtab, st);
  }
  if (o.system_iters && count == 1)
    cudaMemcpyAsync(o.system_iters, tab.p[0].iters, (size_t)tab.p[0].nsys * sizeof(int32_t),
                    cudaMemcpyDeviceToDevice, st);
  mark(4);
  if (cudaGetLastError() != cudaSuccess) return INFO_ESRF_ERR_CUDA;
  if (!stats) return INFO_ESRF_OK;
  if (cudaStreamSynchronize(st) != cudaSuccess) return INFO_ESRF_ERR_CUDA;
  int worst = INFO_ESRF_OK;
  for (int i = 0; i < count; ++i) {
    const ProblemDev& pr = tab.p[i];
    info_esrf_stats& s = stats[i];
    memset(&s, 0, sizeof(s));
    int32_t status[4];
    double scal[8];
    const size_t nsys = (size_t)pr.nsys;
    std::vector<int32_t> it(nsys);
    std::vector<double> rr(nsys);
    if (cudaMemcpy(status, pr.status, sizeof(status), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(scal, pr.scal, sizeof(scal), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(it.data(), pr.iters, nsys * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(rr.data(), pr.relres, nsys * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
      return INFO_ESRF_ERR_CUDA;
    // count live systems: perturbation lanes < N per group and the mean lane
    int64_t live = 0, sum_it = 0;
    int32_t it_max = 0, unconv = 0;
    double rmax = 0.0;
    for (size_t sidx = 0; sidx < nsys; ++sidx) {
      ++live;
      sum_it += it[sidx];
      it_max = std::max(it_max, it[sidx]);
      rmax = std::max(rmax, rr[sidx]);
      if (o.fixed_iters <= 0 && !(rr[sidx] <= pr.tol)) ++unconv;
    }
    s.device_flags = status[0];
    s.solver_path = o.precision == INFO_ESRF_PRECISION_BF16 ? 3
                    : o.solver == INFO_ESRF_SOLVER_BLOCK ? 4
                    : (status[1] & 2) ? 2 : (status[1] & 1);
    s.iters_max = it_max;
    s.n_systems = (int32_t)live;
    s.iters_mean = live ? (double)sum_it / (double)live : 0.0;
    s.n_unconverged = unconv;
    s.max_rel_resid = rmax;
    s.ell_used = scal[2];
    s.gershgorin = scal[0];
    s.learned = !pr.learned_model ? 0 : (s.solver_path == 1 ? 1 : -1);
    if (pr.learned_model && s.solver_path == 3) {   // applied where the observations form a 2-D lattice
      int32_t lat_ok = 0;
      if (cudaMemcpy(&lat_ok, pr.lat_info, sizeof(lat_ok), cudaMemcpyDeviceToHost) != cudaSuccess)
        return INFO_ESRF_ERR_CUDA;
      s.learned = lat_ok == 1 ? 1 : -1;
    }
    if (o.precision == INFO_ESRF_PRECISION_BF16) {
      int32_t nblocks = 0;
      if (cudaMemcpy(&nblocks, pr.rowptr + pr.nrt, sizeof(nblocks), cudaMemcpyDeviceToHost) != cudaSuccess)
        return INFO_ESRF_ERR_CUDA;
      s.matvec_ms = tile_mm_ms[i];
      s.matvec_launches = tile_mm_n[i];
      s.tile_blocks = nblocks;
      s.c_nnz = scal[3];
    }
    s.status = status_to_code(status[0]);
    if (s.status < 0 && (worst >= 0 || s.status < worst)) worst = s.status;
    else if (worst == INFO_ESRF_OK && s.status > 0) worst = s.status;
  }
  return worst;
}

info_esrf_problem one_problem(const info_esrf_grid* grid, int64_t N, const double* X, int64_t d,
                              const int64_t* obs, const double* y, const double* R, int32_t Q, double tol,
                              double* mu_a, double* A_a) {
  info_esrf_problem P;
  memset(&P, 0, sizeof(P));
  if (grid) P.grid = *grid;
  P.N = N;
  P.d = d;
  P.Q = Q;
  P.tol = tol;
  P.X = X;
  P.obs_idx = obs;
  P.y = y;
  P.R_diag = R;
  P.mu_a = mu_a;
  P.A_a = A_a;
  return P;
}

}  // namespace

extern "C" {

void info_esrf_default_options(info_esrf_options* opt) {
  if (!opt) return;
  memset(opt, 0, sizeof(*opt));
  opt->precision = INFO_ESRF_PRECISION_FP64;
  opt->ritz_rank = 10;
  opt->oversample = 10;
  opt->power_iters = 1;
  opt->max_iter = 1000;
  opt->fixed_iters = 0;
  opt->rule = INFO_ESRF_RULE_ELLIPTIC;
  opt->cluster_size = 0;
  opt->ell = 0.0;
  opt->seed = 0x1234abcdULL;
  opt->max_neighbors = 0;
  opt->learned_model = nullptr;
  opt->learned_max_shift = 0.0;
  opt->system_iters = nullptr;
  opt->phase_events = nullptr;
}

const char* info_esrf_error_string(int code) {
  switch (code) {
    case INFO_ESRF_OK: return "ok";
    case INFO_ESRF_NOT_CONVERGED: return "some PCG system reached the iteration cap";
    case INFO_ESRF_ERR_INVALID_ARG: return "invalid argument";
    case INFO_ESRF_ERR_BAD_OBS_INDEX: return "observation index out of range or not strictly increasing";
    case INFO_ESRF_ERR_NONPOSITIVE_R: return "observation-error variance not positive and finite";
    case INFO_ESRF_ERR_WORKSPACE: return "workspace too small or not 256-byte aligned";
    case INFO_ESRF_ERR_CUDA: return "CUDA runtime error";
    case INFO_ESRF_ERR_NONFINITE: return "non-finite value in the ensemble";
    case INFO_ESRF_ERR_BAND_OVERFLOW: return "more neighbours than the band capacity";
    case INFO_ESRF_ERR_BREAKDOWN: return "PCG breakdown";
    case INFO_ESRF_ERR_UNSUPPORTED: return "size beyond a documented limit";
    case INFO_ESRF_ERR_TIMEOUT: return "a bounded device wait expired";
    default: return "unknown status";
  }
}

int info_esrf_version(void) { return 10000; }

int64_t info_esrf_launch_count(void) { return (int64_t)g_launches.load(std::memory_order_relaxed); }

int info_esrf_neighbor_counts(const info_esrf_grid* grid, int64_t d, const int64_t* obs_idx_dev,
                              int64_t* counts_dev, void* stream, int64_t* max_oo, int64_t* max_xo) {
  GridDev g;
  int rc = make_grid(grid, &g);
  if (rc) return rc;
  if (d < 1 || !obs_idx_dev || !counts_dev || !max_oo || !max_xo) return INFO_ESRF_ERR_INVALID_ARG;
  const int64_t n = g.ext[0] * g.ext[1] * g.ext[2];
  if (d > n) return INFO_ESRF_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaGetLastError();
  launch_count_neighbours(g, obs_idx_dev, d, n, counts_dev, st);
  int64_t host[2] = {0, 0};
  if (cudaMemcpyAsync(host, counts_dev, sizeof(host), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return INFO_ESRF_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return INFO_ESRF_ERR_CUDA;
  *max_oo = host[0];
  *max_xo = host[1];
  return 0;
}

size_t info_esrf_batched_workspace_size(const info_esrf_problem* probs, int32_t count,
                                        const info_esrf_options* opt) {
  info_esrf_options o;
  if (check_options(opt, &o)) return 0;
  static thread_local ProblemTable tab;
  size_t need = 0;
  if (build_table(probs, count, o, nullptr, tab, &need, nullptr, nullptr, nullptr, nullptr, num_sms_current()))
    return 0;
  return need;
}

size_t info_esrf_workspace_size(const info_esrf_grid* grid, int64_t N, int64_t d, int32_t Q,
                                const info_esrf_options* opt) {
  // both updates: dummy non-null pointers mark mu_a and A_a as requested
  static double dummy;
  static int64_t idummy;
  info_esrf_problem P = one_problem(grid, N, &dummy, d, &idummy, &dummy, &dummy, Q, 1.0, &dummy, &dummy);
  return info_esrf_batched_workspace_size(&P, 1, opt);
}

int info_esrf_mean_update(const info_esrf_grid* grid, int64_t N, const double* X_dev, int64_t d,
                          const int64_t* obs_idx_dev, const double* y_dev, const double* R_diag_dev, double tol,
                          const info_esrf_options* opt, void* workspace, size_t ws_bytes, void* stream,
                          double* mu_a_dev, info_esrf_stats* stats) {
  if (!mu_a_dev) return INFO_ESRF_ERR_INVALID_ARG;
  info_esrf_problem P = one_problem(grid, N, X_dev, d, obs_idx_dev, y_dev, R_diag_dev, 0, tol, mu_a_dev, nullptr);
  return run_batch(&P, 1, opt, workspace, ws_bytes, stream, stats);
}

int info_esrf_perturbation_update(const info_esrf_grid* grid, int64_t N, const double* X_dev, int64_t d,
                                  const int64_t* obs_idx_dev, const double* R_diag_dev, int32_t Q, double tol,
                                  const info_esrf_options* opt, void* workspace, size_t ws_bytes, void* stream,
                                  double* A_a_dev, info_esrf_stats* stats) {
  if (!A_a_dev) return INFO_ESRF_ERR_INVALID_ARG;
  info_esrf_problem P = one_problem(grid, N, X_dev, d, obs_idx_dev, nullptr, R_diag_dev, Q, tol, nullptr, A_a_dev);
  return run_batch(&P, 1, opt, workspace, ws_bytes, stream, stats);
}

int info_esrf_analysis(const info_esrf_grid* grid, int64_t N, const double* X_dev, int64_t d,
                       const int64_t* obs_idx_dev, const double* y_dev, const double* R_diag_dev, int32_t Q,
                       double tol, const info_esrf_options* opt, void* workspace, size_t ws_bytes, void* stream,
                       double* mu_a_dev, double* A_a_dev, info_esrf_stats* stats) {
  if (!mu_a_dev || !A_a_dev) return INFO_ESRF_ERR_INVALID_ARG;
  info_esrf_problem P = one_problem(grid, N, X_dev, d, obs_idx_dev, y_dev, R_diag_dev, Q, tol, mu_a_dev, A_a_dev);
  return run_batch(&P, 1, opt, workspace, ws_bytes, stream, stats);
}

constexpr int kTuneReps = 5;   // timed calls per candidate

int info_esrf_autotune(const info_esrf_problem* probs, int32_t count, info_esrf_options* opt, void* workspace,
                       size_t ws_bytes, void* stream, double* best_ms) {
  if (!probs || !opt || count < 1) return INFO_ESRF_ERR_INVALID_ARG;
  info_esrf_options base;
  int rc = check_options(opt, &base);
  if (rc) return rc;
  base.phase_events = nullptr;
  base.system_iters = nullptr;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    return INFO_ESRF_ERR_CUDA;
  }
  std::vector<info_esrf_stats> stats((size_t)count);
  double best = -1.0;
  info_esrf_options best_o = base;
  int first_rc = 0;
  const int cs_list[3] = {0, 4, -1}, pi_list[2] = {0, 1}, os_list[3] = {2, 6, 10};
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 2; ++b)
      for (int c = 0; c < 3; ++c) {
        info_esrf_options o = base;
        o.cluster_size = cs_list[a];
        o.power_iters = pi_list[b];
        o.oversample = os_list[c];
        if (o.ritz_rank + o.oversample > kMaxRitz) continue;
        if (info_esrf_batched_workspace_size(probs, count, &o) > ws_bytes) continue;
        int r = run_batch(probs, count, &o, workspace, ws_bytes, stream, stats.data());
        if (r < 0) {
          if (!first_rc) first_rc = r;
          continue;
        }
        bool ok = true;
        for (int i = 0; i < count; ++i) ok &= stats[i].n_unconverged == 0 && stats[i].status == 0;
        if (!ok) continue;
        // the fastest of kTuneReps separately timed calls: candidates often differ
        // by about 1 %, which the minimum resolves and a mean of a few calls does not
        double per = -1.0;
        for (int rep = 0; rep < kTuneReps; ++rep) {
          cudaEventRecord(e0, st);
          run_batch(probs, count, &o, workspace, ws_bytes, stream, nullptr);
          cudaEventRecord(e1, st);
          if (cudaEventSynchronize(e1) != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return INFO_ESRF_ERR_CUDA;
          }
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (per < 0.0 || ms < per) per = ms;
        }
        if (best < 0.0 || per < best) {
          best = per;
          best_o = o;
        }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best < 0.0) return first_rc ? first_rc : INFO_ESRF_ERR_UNSUPPORTED;
  opt->cluster_size = best_o.cluster_size;
  opt->power_iters = best_o.power_iters;
  opt->oversample = best_o.oversample;
  if (best_ms) *best_ms = best;
  return INFO_ESRF_OK;
}

int info_esrf_analysis_batched(const info_esrf_problem* probs, int32_t count, const info_esrf_options* opt,
                               void* workspace, size_t ws_bytes, void* stream, info_esrf_stats* stats) {
  if (!probs) return INFO_ESRF_ERR_INVALID_ARG;
  return run_batch(probs, count, opt, workspace, ws_bytes, stream, stats);
}

// ---------------------------------------------------------------------------
// Stage entry points (info_esrf_stages.h)
// ---------------------------------------------------------------------------

int info_esrf_philox_normals(uint64_t seed, int64_t count, double* out_dev, void* stream) {
  if (count < 0 || (count > 0 && !out_dev)) return INFO_ESRF_ERR_INVALID_ARG;
  cudaGetLastError();
  launch_philox(seed, count, out_dev, reinterpret_cast<cudaStream_t>(stream));
  return cudaGetLastError() == cudaSuccess ? 0 : INFO_ESRF_ERR_CUDA;
}

int info_esrf_quadrature_nodes(int32_t Q, double ell, int32_t rule, double* s_dev, double* p_dev, void* stream) {
  if (Q < 1 || !s_dev || !p_dev || (rule != 0 && rule != 1) || (rule == 0 && !(ell > 0.0)))
    return INFO_ESRF_ERR_INVALID_ARG;
  cudaGetLastError();
  launch_quadrature_nodes(Q, ell, rule, s_dev, p_dev, reinterpret_cast<cudaStream_t>(stream));
  return cudaGetLastError() == cudaSuccess ? 0 : INFO_ESRF_ERR_CUDA;
}

static int prepare_one(const info_esrf_grid* grid, int64_t N, const double* X_dev, int64_t d,
                       const int64_t* obs_idx_dev, const double* R_diag_dev, int32_t Q,
                       const info_esrf_options* opt_in, void* ws, size_t ws_bytes, void* stream, bool run,
                       ProblemDev** dpr, ProblemDev* hpr, double tol = 1.0) {
  info_esrf_options o;
  int rc = check_options(opt_in, &o);
  if (rc) return rc;
  if (!ws || (reinterpret_cast<uintptr_t>(ws) % kAlign) != 0) return INFO_ESRF_ERR_WORKSPACE;
  static double dummy;
  info_esrf_problem P = one_problem(grid, N, X_dev, d, obs_idx_dev, nullptr, R_diag_dev, Q, tol, nullptr, &dummy);
  static thread_local ProblemTable tab;
  size_t need = 0;
  ProblemDev* dtab = nullptr;
  rc = build_table(&P, 1, o, ws, tab, &need, &dtab, nullptr, nullptr, nullptr, num_sms_current());
  if (rc) return rc;
  if (need > ws_bytes) return INFO_ESRF_ERR_WORKSPACE;
  *dpr = dtab;
  *hpr = tab.p[0];
  if (!run) return 0;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaGetLastError();
  launch_prepare(tab, dtab, st);
  launch_anomalies(tab, dtab, st);
  launch_bands(tab, dtab, st);
  launch_quadrature(tab, dtab, st);
  launch_ritz(tab, dtab, st);
  launch_learn_coef(tab, dtab, st);
  return cudaGetLastError() == cudaSuccess ? 0 : INFO_ESRF_ERR_CUDA;
}

int info_esrf_prepare(const info_esrf_grid* grid, int64_t N, const double* X_dev, int64_t d,
                      const int64_t* obs_idx_dev, const double* R_diag_dev, int32_t Q,
                      const info_esrf_options* opt, void* workspace, size_t ws_bytes, void* stream) {
  ProblemDev* dpr;
  ProblemDev hpr;
  return prepare_one(grid, N, X_dev, d, obs_idx_dev, R_diag_dev, Q, opt, workspace, ws_bytes, stream, true, &dpr,
                     &hpr);
}

int info_esrf_prepared_obs_matvec(const info_esrf_grid* grid, int64_t N, int64_t d, int32_t Q,
                                  const info_esrf_options* opt, void* workspace, size_t ws_bytes, int32_t nvec,
                                  const double* P_dev, const double* sigma_dev, double* Y_dev, void* stream) {
  ProblemDev* dpr;
  ProblemDev hpr;
  static double dx;
  static int64_t di;
  int rc = prepare_one(grid, N, &dx, d, &di, &dx, Q, opt, workspace, ws_bytes, stream, false, &dpr, &hpr);
  if (rc) return rc;
  if (nvec < 0 || (nvec > 0 && (!P_dev || !sigma_dev || !Y_dev))) return INFO_ESRF_ERR_INVALID_ARG;
  cudaGetLastError();
  launch_obs_matvec(hpr, dpr, nvec, P_dev, sigma_dev, Y_dev, reinterpret_cast<cudaStream_t>(stream));
  return cudaGetLastError() == cudaSuccess ? 0 : INFO_ESRF_ERR_CUDA;
}

int info_esrf_prepared_lmp_apply(const info_esrf_grid* grid, int64_t N, int64_t d, int32_t Q,
                                 const info_esrf_options* opt, void* workspace, size_t ws_bytes, int32_t nvec,
                                 const double* R_dev, const double* sigma_dev, double* Z_dev, void* stream) {
  ProblemDev* dpr;
  ProblemDev hpr;
  static double dx;
  static int64_t di;
  int rc = prepare_one(grid, N, &dx, d, &di, &dx, Q, opt, workspace, ws_bytes, stream, false, &dpr, &hpr);
  if (rc) return rc;
  if (nvec < 0 || (nvec > 0 && (!R_dev || !sigma_dev || !Z_dev))) return INFO_ESRF_ERR_INVALID_ARG;
  cudaGetLastError();
  launch_lmp_apply(hpr, dpr, nvec, R_dev, sigma_dev, Z_dev, reinterpret_cast<cudaStream_t>(stream));
  return cudaGetLastError() == cudaSuccess ? 0 : INFO_ESRF_ERR_CUDA;
}

int info_esrf_prepared_export(const info_esrf_grid* grid, int64_t N, int64_t d, int32_t Q,
                              const info_esrf_options* opt, void* workspace, size_t ws_bytes, int32_t item,
                              void* dst_host, size_t dst_bytes, void* stream) {
  ProblemDev* dpr;
  ProblemDev hpr;
  static double dx;
  static int64_t di;
  int rc = prepare_one(grid, N, &dx, d, &di, &dx, Q, opt, workspace, ws_bytes, stream, false, &dpr, &hpr);
  if (rc) return rc;
  const size_t esz = hpr.precision == 0 ? 8 : 4;
  const void* src = nullptr;
  size_t bytes = 0;
  switch (item) {
    case INFO_ESRF_ITEM_SCALARS: src = hpr.scal; bytes = 8 * 8; break;
    case INFO_ESRF_ITEM_STATUS: src = hpr.status; bytes = 4 * 4; break;
    case INFO_ESRF_ITEM_QUAD_S: src = hpr.s; bytes = (size_t)hpr.Q * 8; break;
    case INFO_ESRF_ITEM_QUAD_P: src = hpr.p; bytes = (size_t)hpr.Q * 8; break;
    case INFO_ESRF_ITEM_THETA: src = hpr.theta; bytes = (size_t)hpr.kR * 8; break;
    case INFO_ESRF_ITEM_PHI: src = hpr.Phi; bytes = (size_t)hpr.d * hpr.kR * esz; break;
    case INFO_ESRF_ITEM_CPHI: src = hpr.CPhi; bytes = (size_t)hpr.d * hpr.kR * esz; break;
    case INFO_ESRF_ITEM_OO_VAL: src = hpr.oo_val; bytes = (size_t)hpr.max_oo * hpr.d * esz; break;
    case INFO_ESRF_ITEM_OO_COL: src = hpr.oo_col; bytes = (size_t)hpr.max_oo * hpr.d * 4; break;
    case INFO_ESRF_ITEM_OO_NNZ: src = hpr.oo_nnz; bytes = (size_t)hpr.d * 4; break;
    case INFO_ESRF_ITEM_XO_VAL: src = hpr.xo_val; bytes = (size_t)hpr.max_xo * hpr.n * esz; break;
    case INFO_ESRF_ITEM_XO_COL: src = hpr.xo_col; bytes = (size_t)hpr.max_xo * hpr.n * 4; break;
    case INFO_ESRF_ITEM_XO_NNZ: src = hpr.xo_nnz; bytes = (size_t)hpr.n * 4; break;
    case INFO_ESRF_ITEM_W: src = hpr.W; bytes = (size_t)hpr.d * hpr.N * esz; break;
    case INFO_ESRF_ITEM_MU: src = hpr.mu; bytes = (size_t)hpr.n * 8; break;
    default: return INFO_ESRF_ERR_INVALID_ARG;
  }
  if (!dst_host || dst_bytes < bytes) return INFO_ESRF_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (bytes && cudaMemcpyAsync(dst_host, src, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return INFO_ESRF_ERR_CUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? 0 : INFO_ESRF_ERR_CUDA;
}

int info_esrf_krylov_capture(const info_esrf_grid* grid, int64_t N, const double* X_dev, int64_t d,
                             const int64_t* obs_idx_dev, const double* R_diag_dev, int32_t Q,
                             const info_esrf_options* opt, void* workspace, size_t ws_bytes, int32_t nsel,
                             const int32_t* sel_dev, int32_t K, float* V_dev, float* Y_dev, float* Z_dev,
                             float* feat_dev, void* stream) {
  if (nsel < 1 || K < 1 || !sel_dev || !V_dev || !Y_dev || !Z_dev || !feat_dev) return INFO_ESRF_ERR_INVALID_ARG;
  info_esrf_options o;
  int rc = check_options(opt, &o);
  if (rc) return rc;
  if (o.precision != INFO_ESRF_PRECISION_FP32) return INFO_ESRF_ERR_UNSUPPORTED;
  ProblemDev* dpr;
  ProblemDev hpr;
  rc = prepare_one(grid, N, X_dev, d, obs_idx_dev, R_diag_dev, Q, opt, workspace, ws_bytes, stream, true, &dpr,
                   &hpr);
  if (rc) return rc;
  static thread_local ProblemTable tab;
  tab.count = 1;
  tab.p[0] = hpr;
  cudaGetLastError();
  rc = launch_krylov_capture(tab, dpr, nsel, sel_dev, K, V_dev, Y_dev, Z_dev, feat_dev,
                             reinterpret_cast<cudaStream_t>(stream));
  if (rc) return rc;
  return cudaGetLastError() == cudaSuccess ? 0 : INFO_ESRF_ERR_CUDA;
}

int info_esrf_krylov_capture_lattice(const info_esrf_grid* grid, int64_t N, const double* X_dev, int64_t d,
                                     const int64_t* obs_idx_dev, const double* R_diag_dev, int32_t Q,
                                     const info_esrf_options* opt, void* workspace, size_t ws_bytes, int32_t nsel,
                                     const int32_t* sel_dev, int32_t K, float* V_dev, float* Y_dev, float* Z_dev,
                                     float* feat_dev, int32_t* Lx, int32_t* Ly, void* stream) {
  if (nsel < 1 || K < 1 || !sel_dev || !V_dev || !Y_dev || !Z_dev || !feat_dev || !Lx || !Ly)
    return INFO_ESRF_ERR_INVALID_ARG;
  info_esrf_options o;
  int rc = check_options(opt, &o);
  if (rc) return rc;
  if (o.precision != INFO_ESRF_PRECISION_BF16) return INFO_ESRF_ERR_UNSUPPORTED;
  info_esrf_options o2 = o;
  o2.learned_model = nullptr;   // the paper's preconditioner
  ProblemDev* dpr;
  ProblemDev hpr;
  // a system stops recording once its residual is at 1e-6 of the right-hand side
  rc = prepare_one(grid, N, X_dev, d, obs_idx_dev, R_diag_dev, Q, &o2, workspace, ws_bytes, stream, false, &dpr,
                   &hpr, 1e-6);
  if (rc) return rc;
  static thread_local ProblemTable tab;
  tab.count = 1;
  tab.p[0] = hpr;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaGetLastError();
  launch_prepare(tab, dpr, st);
  launch_anomalies(tab, dpr, st);
  launch_tile_setup(tab, dpr, st);
  launch_quadrature(tab, dpr, st);
  launch_tile_lattice(tab, dpr, st);
  launch_ritz(tab, dpr, st);
  int32_t info[8] = {};
  if (cudaMemcpyAsync(info, hpr.lat_info, sizeof(info), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return INFO_ESRF_ERR_CUDA;
  if (info[0] != 1) return INFO_ESRF_ERR_UNSUPPORTED;   // the observations are not a 2-D lattice
  *Lx = info[1];
  *Ly = info[2];
  TileCapture cap;
  cap.nsel = nsel;
  cap.K = K;
  cap.sel = sel_dev;
  cap.V = V_dev;
  cap.Y = Y_dev;
  rc = run_tile_pcg_capture(hpr, dpr, cap, Z_dev, feat_dev, st);
  if (rc) return rc;
  return cudaGetLastError() == cudaSuccess ? 0 : INFO_ESRF_ERR_CUDA;
}

int info_esrf_model_save(const char* path, const float* theta_host, double max_shift) {
  if (!path || !theta_host) return INFO_ESRF_ERR_INVALID_ARG;
  FILE* f = fopen(path, "wb");
  if (!f) return INFO_ESRF_ERR_INVALID_ARG;
  const char tag[8] = {'I', 'E', 'S', 'R', 'F', 'N', 'N', '1'};
  const int32_t np = kLearnParams;
  const bool ok = fwrite(tag, 1, 8, f) == 8 && fwrite(&np, 4, 1, f) == 1 &&
                  fwrite(theta_host, sizeof(float), np, f) == (size_t)np && fwrite(&max_shift, 8, 1, f) == 1;
  return (fclose(f) == 0 && ok) ? 0 : INFO_ESRF_ERR_INVALID_ARG;
}

int info_esrf_model_load(const char* path, float* theta_host, double* max_shift) {
  if (!path || !theta_host || !max_shift) return INFO_ESRF_ERR_INVALID_ARG;
  FILE* f = fopen(path, "rb");
  if (!f) return INFO_ESRF_ERR_INVALID_ARG;
  char tag[8];
  int32_t np = 0;
  bool ok = fread(tag, 1, 8, f) == 8 && memcmp(tag, "IESRFNN1", 8) == 0 && fread(&np, 4, 1, f) == 1 &&
            np == kLearnParams && fread(theta_host, sizeof(float), np, f) == (size_t)np &&
            fread(max_shift, 8, 1, f) == 1;
  fclose(f);
  return ok ? 0 : INFO_ESRF_ERR_INVALID_ARG;
}

int info_esrf_prepared_band_capacity(const info_esrf_grid* grid, int64_t N, int64_t d, int32_t Q,
                                     const info_esrf_options* opt, int64_t* max_oo, int64_t* max_xo) {
  info_esrf_options o;
  int rc = check_options(opt, &o);
  if (rc) return rc;
  static double dx;
  static int64_t di;
  info_esrf_problem P = one_problem(grid, N, &dx, d, &di, nullptr, &dx, Q, 1.0, nullptr, &dx);
  static thread_local ProblemTable tab;
  size_t need = 0;
  rc = build_table(&P, 1, o, nullptr, tab, &need, nullptr, nullptr, nullptr, nullptr, 160);
  if (rc) return rc;
  if (max_oo) *max_oo = tab.p[0].max_oo;
  if (max_xo) *max_xo = tab.p[0].max_xo;
  return 0;
}

}  // extern "C"
