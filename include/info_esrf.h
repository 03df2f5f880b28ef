/*
 * info_esrf.h -- C ABI of a single-GPU (sm_103a) library for the InFo-ESRF
 * mean update and perturbation update (Armstrong & Grooms, "Data
 * Assimilation With An Integral-Form Ensemble Square-Root Filter").
 *
 * Operations
 *   Mean update (Sec. 3.2, Eq. info_esrf_mean_solve):
 *       mu_a = mu + Sxh (R + Shh)^-1 (y - H mu).
 *   Perturbation update (Sec. 3.2, Eq. info_esrf_perturbation_solve, App. D-E):
 *       z_a^(i) = z^(i) - Sxh sum_q p_q v_q^(i),  ((s_q + 1) R + Shh) v_q^(i) = w^(i),
 *   with (s_q, p_q) the elliptic (App. D, Eq. elliptic_quadrature_rule) or
 *   Gauss-Legendre (Eq. gaussian_quadrature_rule) rule, every system solved
 *   in the normalized form of Eq. normalized_linear_solve by PCG with the
 *   limited-memory preconditioner of App. E.
 *   Localized covariances (Sec. 2.3, Eq. localized_state_covar):
 *       Sxx = L o (Z Z^T),  Sxh = Sxx H^T,  Shh = H Sxx H^T,
 *   Z the normalized perturbations (Eq. normalized_perturbations), H the
 *   observation subsampling operator given by obs_idx, R diagonal, and L the
 *   Gaspari-Cohn localization of the grid distance.
 *
 * Conventions
 *   - Every array argument named *_dev is a DEVICE pointer; the caller owns it.
 *   - Ensembles are member-major: X[k * n + x] is member k at grid point x.
 *   - Outputs: mu_a [n] the analysis mean; A_a [N][n] the analysis anomalies
 *     sqrt(N - 1) z_a^(i), so the analysis ensemble is mu_a + A_a.
 *   - obs_idx [d]: strictly increasing flat grid indices in [0, n).
 *   - R_diag [d]: observation-error variances, > 0.
 *   - workspace: caller-allocated device memory of info_esrf_workspace_size()
 *     bytes, 256-byte aligned.  The library keeps no pointer after return
 *     and allocates nothing.
 *   - stream: a cudaStream_t passed as void*; NULL is the legacy stream.  All
 *     work is stream-ordered.  If stats is NULL the call returns as soon as
 *     the work is queued; otherwise it waits for the stream and fills stats,
 *     and device-detected input errors become the return code.
 *
 * Return codes: 0 success; > 0 warning (outputs written); < 0 error
 * (outputs unspecified, nothing freed or leaked).
 */
#ifndef INFO_ESRF_H
#define INFO_ESRF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define INFO_ESRF_OK 0
#define INFO_ESRF_NOT_CONVERGED 1          /* some system hit max_iter */
#define INFO_ESRF_ERR_INVALID_ARG (-1)     /* bad size, pointer or option */
#define INFO_ESRF_ERR_BAD_OBS_INDEX (-2)   /* obs_idx out of range or not increasing */
#define INFO_ESRF_ERR_NONPOSITIVE_R (-3)   /* R_diag <= 0 or not finite */
#define INFO_ESRF_ERR_WORKSPACE (-4)       /* workspace too small or misaligned */
#define INFO_ESRF_ERR_CUDA (-5)            /* a CUDA runtime call failed */
#define INFO_ESRF_ERR_NONFINITE (-6)       /* NaN or Inf in the ensemble */
#define INFO_ESRF_ERR_BAND_OVERFLOW (-7)   /* more neighbours than max_neighbors */
#define INFO_ESRF_ERR_BREAKDOWN (-8)       /* PCG breakdown (p^T C_q p <= 0) */
#define INFO_ESRF_ERR_UNSUPPORTED (-9)     /* size beyond a documented limit */
#define INFO_ESRF_ERR_TIMEOUT (-10)        /* a bounded device wait expired (no hang) */

#define INFO_ESRF_PRECISION_FP64 0         /* every vector and matrix in FP64 */
#define INFO_ESRF_PRECISION_FP32 1         /* FP32 bulk, FP64 scalars and quadrature sum */
/* BF16 tensor-core matvec (block-tile path): C formed in FP32 and kept as
 * two BF16 planes hi + lo (about 16 significant bits), search directions in
 * BF16, products on the tensor cores with FP32 accumulation; iterates,
 * residuals and the preconditioner in FP32; CG scalars, partial-sum merges
 * and the quadrature sum in FP64.  Any grid (1-D, 2-D, layered), subsampling
 * observations only, N <= 128, solver PCG.  The call synchronizes its stream
 * once per PCG iteration (convergence is tested on the host), so it cannot be
 * captured in a CUDA graph. */
#define INFO_ESRF_PRECISION_BF16 2

#define INFO_ESRF_RULE_ELLIPTIC 0          /* App. D, Eq. elliptic_quadrature_rule */
#define INFO_ESRF_RULE_GAUSS_LEGENDRE 1    /* App. D, Eq. gaussian_quadrature_rule */

#define INFO_ESRF_SOLVER_PCG 0             /* one PCG run per (node, member) system (Sec. 3.3, App. E) */
#define INFO_ESRF_SOLVER_MULTISHIFT 1      /* one CG run per member for all Q shifts (Sec. 3.3, item 1) */
/* Block CG across members (Sec. 3.3, second alternative; O'Leary's block CG):
 * for every node the N members' systems share one block Krylov space and are
 * solved together, X_0 = 0, R_0 = P_0 = B, alpha = (P^T C_q P)^-1 (R^T R),
 * beta = (R^T R)^-1 (R'^T R'), without a preconditioner (the mean system is
 * a block of one column); a block stops when every column meets tol (or
 * after fixed_iters).  The members' right-hand sides sum to zero, so the
 * block runs on N - 1 columns and the last member's solution is minus the sum
 * of the others; Gram pivots at rounding level count as zero.  FP64 or FP32 bulk (s x s algebra
 * and Gram sums in FP64), N <= 64.  The call synchronizes its stream once per
 * iteration (convergence is tested on the host). */
#define INFO_ESRF_SOLVER_BLOCK 2

/* Regular grid.  Flat index = (z * shape[1] + y) * shape[0] + x.  Axes of
 * extent 1 are ignored.  The Gaspari-Cohn argument is
 * r = sqrt(sum_axes (dist_axis / half_width[axis])^2), L = GC(r), zero for
 * r >= 2 (support 2 * half_width).  On periodic axes dist is the chordal
 * distance (n / pi) sin(pi |i - j| / n) if chordal != 0 (Sec. 4.1, Sec. 5.2),
 * otherwise the minimum-image distance; on other axes |i - j|. */
typedef struct {
  int64_t shape[3];
  int32_t periodic[3];
  int32_t chordal;
  double half_width[3];
} info_esrf_grid;

typedef struct {
  int32_t precision;      /* INFO_ESRF_PRECISION_*; default FP64 */
  int32_t ritz_rank;      /* k_R Ritz vectors in the preconditioner (App. E); 0 = none; <= 24; default 10 */
  int32_t oversample;     /* extra test vectors of the randomized eigensolver; default 10; k_R + oversample <= 32 */
  int32_t power_iters;    /* power iterations of the range finder; default 1 */
  int32_t max_iter;       /* PCG iteration cap; default 1000 */
  int32_t fixed_iters;    /* > 0: run exactly this many PCG iterations (paper's experiments) */
  int32_t rule;           /* INFO_ESRF_RULE_*; default elliptic */
  int32_t cluster_size;   /* CTAs per cluster of the FP32 cluster-resident PCG kernel (one-dimensional grids):
                             2, 4 or 8 (halved while a CTA would own fewer than 32 rows), one launch per
                             eligible problem; 0 = 8 for a single problem, and that kernel off in a batch
                             of several; -1 = off (the general PCG kernel solves every system) */
  double ell;             /* spectrum bound of App. D; <= 0: power of ten above a Gershgorin bound of C */
  uint64_t seed;          /* Philox key of the randomized eigensolver's test matrix */
  int64_t max_neighbors;  /* band capacity per row; <= 0: bound from the geometry */
  /* Learned preconditioner correction (not in the paper), or NULL: device
   * array of info_esrf_learn_nparams() floats, the parameters of the network
   * described in info_esrf_stages.h.  Each shifted system is then
   * preconditioned by M_q = a_q P_q^-1 + S_q^T S_q (symmetric positive
   * definite), a_q and the stencil S_q produced by the network from the
   * shift and the spectrum statistics of C.  Used by the cluster-resident
   * FP32 solver for 1-D networks (S_q a circulant over the observation
   * index), and by the BF16 path where the observations fill a periodic 2-D
   * lattice (S_q a symmetric 5 x 5 lattice stencil, M_q = a_q P_q^-1 + S_q S_q;
   * the workspace then holds one more vector per system).  A system that
   * breaks down or reaches max_iter with it is solved again with P_q^-1
   * alone.  Convergence is always tested on the unpreconditioned residual
   * ||b - C_q u||.  Other solvers and geometries do not apply it and report
   * so in info_esrf_stats.learned. */
  const float* learned_model;
  double learned_max_shift;  /* > 0: the learned term is used only for shifts sigma = s_q + 1 <= this */
  /* NULL, or a device int32 array receiving each system's PCG iteration
   * count (single-problem calls): with the mean update, entry 0 is the mean
   * system and 1 + q * N + i the perturbation systems; without it, q * N + i. */
  int32_t* system_iters;
  /* NULL, or 5 cudaEvent_t handles (as void*) recorded on the call's stream
   * at the phase boundaries: start; after the setup of a1-a3 (anomalies, W,
   * bands, quadrature); after the Ritz pairs (a4); after the persistent PCG
   * (a5-a8); after the accumulation and state update (a9-a11). */
  void* const* phase_events;
  /* INFO_ESRF_SOLVER_*; default PCG.  MULTISHIFT solves all Q shifted systems
   * of a member with one unpreconditioned CG run on C + sigma_0 I, sigma_0 the
   * smallest shift, using the shift invariance of Krylov subspaces (Sec. 3.3,
   * first alternative; the systems are exact shifts of C in normalized form,
   * App. E).  The mean system is a chain with the single shift 1.  Each shift
   * stops at ||r_q|| <= tol ||b||; max_iter and fixed_iters count iterations
   * of the run.  ritz_rank, oversample, power_iters and learned_model are then
   * not used (no Ritz stage), and cluster_size 2, 4 or 8 sets the CTAs per
   * cluster of the multi-shift kernel (0 or -1: chosen from d).  Every CTA
   * keeps a full copy of each chain's direction next to its own rows, so one
   * chain needs about 1.5 d elements of shared memory per CTA (8 CTAs per
   * cluster): d above about 35,000 (FP32) or 18,000 (FP64) returns
   * INFO_ESRF_ERR_UNSUPPORTED. */
  int32_t solver;
  int32_t reserved_;
  /* BF16 path: stored 128 x 64 blocks of C (tile_capacity) and of the state
   * update (state_tile_capacity) to reserve in the workspace; <= 0: an
   * estimate from the geometry and the mean observation density (1.3 x the
   * count for evenly spread observations).  More blocks than reserved make
   * the call return INFO_ESRF_ERR_BAND_OVERFLOW. */
  int64_t tile_capacity;
  int64_t state_tile_capacity;
} info_esrf_options;

typedef struct {
  int32_t status;         /* return code of the call */
  int32_t device_flags;   /* raw device status bits */
  int32_t iters_max;      /* max PCG iterations over systems */
  int32_t n_systems;      /* systems solved (Q * N perturbation + mean) */
  double iters_mean;
  int32_t n_unconverged;
  int32_t solver_path;    /* 1: cluster-resident band kernel (1-D networks), 0: general kernel,
                             2: multi-shift CG, 3: BF16 block-tile path (tensor cores), 4: block CG */
  double max_rel_resid;   /* max recurrence ||r|| / ||b|| at exit */
  double ell_used;
  double gershgorin;      /* max_a sum_b |C(a, b)| */
  /* Learned correction of options.learned_model: 0 no model was given; 1 the
   * solver that ran applies it (systems with shift <= learned_max_shift);
   * -1 a model was given but the solver that ran does not apply it (the
   * analysis is still correct, preconditioned by P_q^-1 alone). */
  int32_t learned;
  int32_t pad_;
  /* BF16 path (solver_path 3), zero otherwise: device time of the
   * tensor-core matvec launches, summed from CUDA events recorded on the
   * call's stream around each launch; their count; the stored 128 x 64 blocks
   * of C; and the nonzeros of C (entries inside the Gaspari-Cohn support,
   * counted while forming the blocks). */
  double matvec_ms;
  int64_t tile_blocks;
  double c_nnz;
  int32_t matvec_launches;
  int32_t pad2_;
} info_esrf_stats;

/* One problem of a batched call: inputs and outputs are device pointers.
 * mu_a or A_a may be NULL to skip that update (y may then be NULL too). */
typedef struct {
  info_esrf_grid grid;
  int64_t N;              /* members, >= 2 */
  int64_t d;              /* observations, >= 1 */
  int32_t Q;              /* quadrature nodes, >= 1 */
  int32_t pad_;
  double tol;             /* PCG relative residual tolerance */
  const double* X;        /* [N][n] */
  const int64_t* obs_idx; /* [d] */
  const double* y;        /* [d] */
  const double* R_diag;   /* [d] */
  double* mu_a;           /* [n] or NULL */
  double* A_a;            /* [N][n] or NULL */
  int64_t max_oo;         /* band capacities; <= 0: from the options / geometry */
  int64_t max_xo;
  /* General linear observation operator, or NULL (subsampling at obs_idx).
   * The paper's experiments observe weighted sums of the state (Sec. 4.1,
   * Sec. 5.1); with h linearized and model-space localization (Sec. 2.3) the
   * covariances are Sxh = (L o Z Z^T) H^T [n][d] and Shh = H Sxh [d][d].  H is
   * given in CSR form as device arrays, one row per observation: H_rowptr [d + 1]
   * (H_rowptr[0] = 0, non-decreasing, H_rowptr[d] = H_nnz), H_col [H_nnz] state
   * indices in [0, n), H_val [H_nnz] weights.  obs_idx is then not read, and y
   * (if given) is an observation of H x.  Both covariances are formed densely,
   * so n d <= 2^28 (INFO_ESRF_ERR_UNSUPPORTED above); the PCG runs in the
   * general kernel.  A malformed H (row pointers or columns out of range)
   * makes the call return INFO_ESRF_ERR_BAD_OBS_INDEX; no entry outside the
   * arrays is read. */
  const int64_t* H_rowptr;
  const int64_t* H_col;
  const double* H_val;
  int64_t H_nnz;
} info_esrf_problem;

/* Fills *opt with the defaults listed above. */
void info_esrf_default_options(info_esrf_options* opt);

/* Human-readable text of a return code (static storage). */
const char* info_esrf_error_string(int code);

int info_esrf_version(void);

/* Exact band capacities for one observation pattern: the largest number of
 * observations inside the Gaspari-Cohn support of any observation (*max_oo)
 * and of any grid point (*max_xo).  counts_dev is a caller-owned device
 * buffer of two int64 values used as the kernel's output.  Runs on the
 * device and synchronizes the stream.  Use the results as problem.max_oo /
 * max_xo (or options.max_neighbors) to shrink the workspace below the
 * geometric bound, which assumes every grid point in the support box is
 * observed. */
int info_esrf_neighbor_counts(const info_esrf_grid* grid, int64_t d, const int64_t* obs_idx_dev,
                              int64_t* counts_dev, void* stream, int64_t* max_oo, int64_t* max_xo);

/* Workspace bytes for one problem (both updates) and for a batch. */
size_t info_esrf_workspace_size(const info_esrf_grid* grid, int64_t N, int64_t d, int32_t Q,
                                const info_esrf_options* opt);
size_t info_esrf_batched_workspace_size(const info_esrf_problem* probs, int32_t count,
                                        const info_esrf_options* opt);

/* Mean update alone (Sec. 3.2, Eq. info_esrf_mean_solve).  Writes mu_a_dev [n]. */
int info_esrf_mean_update(const info_esrf_grid* grid, int64_t N, const double* X_dev, int64_t d,
                          const int64_t* obs_idx_dev, const double* y_dev, const double* R_diag_dev,
                          double tol, const info_esrf_options* opt, void* workspace, size_t ws_bytes,
                          void* stream, double* mu_a_dev, info_esrf_stats* stats);

/* Perturbation update alone (Sec. 3.2, App. D-E).  Writes A_a_dev [N][n]. */
int info_esrf_perturbation_update(const info_esrf_grid* grid, int64_t N, const double* X_dev, int64_t d,
                                  const int64_t* obs_idx_dev, const double* R_diag_dev, int32_t Q,
                                  double tol, const info_esrf_options* opt, void* workspace,
                                  size_t ws_bytes, void* stream, double* A_a_dev, info_esrf_stats* stats);

/* Both updates of one analysis sharing one setup (the mean system rides in
 * the same persistent PCG launch).  Writes mu_a_dev [n] and A_a_dev [N][n]. */
int info_esrf_analysis(const info_esrf_grid* grid, int64_t N, const double* X_dev, int64_t d,
                       const int64_t* obs_idx_dev, const double* y_dev, const double* R_diag_dev,
                       int32_t Q, double tol, const info_esrf_options* opt, void* workspace,
                       size_t ws_bytes, void* stream, double* mu_a_dev, double* A_a_dev,
                       info_esrf_stats* stats);

/* Many independent problems of uneven n, N, d and Q in one pass: every stage
 * is one launch over all problems and the PCG is one persistent launch over
 * all of their systems.  count <= 64.  stats, if not NULL, has count entries. */
int info_esrf_analysis_batched(const info_esrf_problem* probs, int32_t count,
                               const info_esrf_options* opt, void* workspace, size_t ws_bytes,
                               void* stream, info_esrf_stats* stats);

/* Autotuner (not in the paper): times the analysis of probs[0..count) with
 * each candidate setting of the launch and eigensolver parameters that do not
 * change the converged answer -- cluster_size (0, 4 or -1), power_iters (0 or 1)
 * and oversample (2, 6 or 10) -- starting from *opt, and writes the fastest into
 * *opt (other fields untouched).  A candidate whose warm-up run leaves a
 * system unconverged, fails, or needs more workspace than ws_bytes is skipped.
 * Each candidate runs once untimed and then five times, each call timed on
 * its own (CUDA events on stream), and is ranked by its fastest call; the
 * problems' outputs are overwritten and the stream is synchronized.  best_ms
 * (host, may be NULL) receives the winner's fastest time per call.  Returns 0, or the first error of the base setting. */
int info_esrf_autotune(const info_esrf_problem* probs, int32_t count, info_esrf_options* opt, void* workspace,
                       size_t ws_bytes, void* stream, double* best_ms);

/* Allocation-free variant of info_esrf_analysis.  The paper has no
 * counterpart: this is a deployment convenience of this library.
 *
 * For callers that may not allocate device memory at all (a plug-in inside
 * an application that owns every device byte through its own pool, or a
 * real-time loop that cannot take cudaMalloc's implicit synchronization) and
 * so cannot hand in a workspace.  The workspace comes from a 32 MiB array
 * compiled into the library; every GPU that loads the library holds it until
 * the process exits.  Problems whose info_esrf_workspace_size() exceeds
 * 32 MiB are rejected with INFO_ESRF_ERR_UNSUPPORTED (set
 * options.max_neighbors, e.g. from info_esrf_neighbor_counts, to shrink the
 * bands).  The call allocates nothing and never calls cudaMalloc/cudaFree.
 *
 * Each call looks up the array's device address in the calling thread's
 * current CUDA context (the primary context of the current device, or a
 * driver context the caller made current); every context holds its own copy
 * of the array, and a context re-created after cudaDeviceReset gets a fresh
 * address.  A call made during stream capture cannot query the runtime and
 * reuses the address found by the last uncaptured call in the same context,
 * so make one uncaptured call in each context before any capture (a captured
 * first call returns INFO_ESRF_ERR_CUDA).  All calls in one context share the
 * one array, so calls whose GPU work overlaps (other streams, other threads)
 * race and corrupt each other: serialize them.  Every scratch word a call
 * reads is written earlier in the same call, so leftovers of the previous
 * call are harmless.  The call is asynchronous and returns no statistics;
 * device-detected input errors are not reported (use info_esrf_analysis
 * with stats to diagnose).  Arguments, outputs and the return codes of
 * invalid or unsupported arguments are those of info_esrf_analysis. */
int info_esrf_analysis_noalloc(const info_esrf_grid* grid, int64_t N, const double* X_dev, int64_t d,
                               const int64_t* obs_idx_dev, const double* y_dev, const double* R_diag_dev,
                               int32_t Q, double tol, const info_esrf_options* opt, void* stream,
                               double* mu_a_dev, double* A_a_dev);

#ifdef __cplusplus
}
#endif

#endif /* INFO_ESRF_H */
