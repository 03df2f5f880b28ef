/*
 * info_esrf_stages.h -- stage-level entry points of the InFo-ESRF library,
 * for testing each step of the analysis on its own and for callers that
 * reuse one prepared operator.  Same conventions as info_esrf.h: *_dev are
 * device pointers owned by the caller; stream is a cudaStream_t as void*.
 *
 * A "prepared" workspace is one on which info_esrf_prepare() ran with the
 * same (grid, N, d, Q, options); the other calls below recompute its layout
 * from those arguments and read it.
 */
#ifndef INFO_ESRF_STAGES_H
#define INFO_ESRF_STAGES_H

#include <stddef.h>
#include <stdint.h>

#include "info_esrf.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Items readable with info_esrf_prepared_export (host destination). */
#define INFO_ESRF_ITEM_SCALARS 0   /* double[8]: Gershgorin bound, min_a C(a,a), ell, 0... */
#define INFO_ESRF_ITEM_STATUS 1    /* int32[4]: device status bits */
#define INFO_ESRF_ITEM_QUAD_S 2    /* double[Q] nodes s_q */
#define INFO_ESRF_ITEM_QUAD_P 3    /* double[Q] weights p_q */
#define INFO_ESRF_ITEM_THETA 4     /* double[k_R] Ritz values of C */
#define INFO_ESRF_ITEM_PHI 5       /* T[d][k_R] Ritz vectors (T = FP64 or FP32 by precision) */
#define INFO_ESRF_ITEM_CPHI 6      /* T[d][k_R] C Phi */
#define INFO_ESRF_ITEM_OO_VAL 7    /* T[max_oo][d] band of C, entry e of row a at e*d + a */
#define INFO_ESRF_ITEM_OO_COL 8    /* int32[max_oo][d] column (obs index) of each entry */
#define INFO_ESRF_ITEM_OO_NNZ 9    /* int32[d] entries per row */
#define INFO_ESRF_ITEM_XO_VAL 10   /* T[max_xo][n] band of Sxh, entry e of row x at e*n + x */
#define INFO_ESRF_ITEM_XO_COL 11   /* int32[max_xo][n] */
#define INFO_ESRF_ITEM_XO_NNZ 12   /* int32[n] */
#define INFO_ESRF_ITEM_W 13        /* T[d][N] observed normalized anomalies W = H Z (Eq. normalized_perturbations) */
#define INFO_ESRF_ITEM_MU 14       /* double[n] ensemble mean */

/* Standard normals from Philox4x32-10 (Salmon et al., SC'11) with Box-Muller:
 * element e uses counter (e/2, 0, 0, 0) and key (seed lo, seed hi); the test
 * matrix of the randomized eigensolver (App. E) is element (a, j) = e = j*d + a. */
int info_esrf_philox_normals(uint64_t seed, int64_t count, double* out_dev, void* stream);

/* Quadrature nodes s_q and weights p_q, q = 1..Q (App. D): the elliptic rule
 * (Eq. elliptic_quadrature_rule) for spectrum bound ell > 0, or Gauss-Legendre
 * (Eq. gaussian_quadrature_rule, ell ignored). */
int info_esrf_quadrature_nodes(int32_t Q, double ell, int32_t rule, double* s_dev, double* p_dev,
                               void* stream);

/* Runs the setup of one analysis into the workspace: anomalies and W = H Z
 * (Eq. normalized_perturbations), the bands of C = R^-1/2 Shh R^-1/2 and of
 * Sxh (Sec. 2.3), the quadrature (App. D) and the Ritz pairs (App. E). */
int info_esrf_prepare(const info_esrf_grid* grid, int64_t N, const double* X_dev, int64_t d,
                      const int64_t* obs_idx_dev, const double* R_diag_dev, int32_t Q,
                      const info_esrf_options* opt, void* workspace, size_t ws_bytes, void* stream);

/* Y_v = sigma_v P_v + C P_v for nvec vectors P [nvec][d] (FP64 in and out; the
 * product runs in the workspace's precision).  The localized-covariance
 * matvec of every PCG iteration (App. E, Eq. normalized_linear_solve). */
int info_esrf_prepared_obs_matvec(const info_esrf_grid* grid, int64_t N, int64_t d, int32_t Q,
                                  const info_esrf_options* opt, void* workspace, size_t ws_bytes,
                                  int32_t nvec, const double* P_dev, const double* sigma_dev,
                                  double* Y_dev, void* stream);

/* Z_v = P^-1 R_v with the limited-memory preconditioner of App. E for the
 * shifted matrix sigma_v I + C (theta = Ritz values + sigma_v,
 * beta = sigma_v + min_a C(a, a)), R and Z [nvec][d] in FP64. */
int info_esrf_prepared_lmp_apply(const info_esrf_grid* grid, int64_t N, int64_t d, int32_t Q,
                                 const info_esrf_options* opt, void* workspace, size_t ws_bytes,
                                 int32_t nvec, const double* R_dev, const double* sigma_dev,
                                 double* Z_dev, void* stream);

/* Copies one prepared array (INFO_ESRF_ITEM_*) to host memory; synchronizes. */
int info_esrf_prepared_export(const info_esrf_grid* grid, int64_t N, int64_t d, int32_t Q,
                              const info_esrf_options* opt, void* workspace, size_t ws_bytes,
                              int32_t item, void* dst_host, size_t dst_bytes, void* stream);

/* Number of CUDA kernels this library has launched in this process so far
 * (host-side counter; used to report launches per analysis). */
int64_t info_esrf_launch_count(void);

/* Sustained FMA throughput of this GPU: every SM runs independent FMA chains
 * for about iters steps per thread in FP32 (precision 1) or FP64 (precision 0).
 * Writes the achieved FLOP/s (2 per FMA) and the kernel time in ms; synchronizes. */
int info_esrf_fma_probe(int32_t precision, int64_t iters, double* flops_per_s, double* ms, void* stream);

/* Per-phase clock counts of the cluster-resident 1-D band PCG kernel (the
 * kernel of solver_path 1; App. E, one PCG iteration per round), for a
 * separate build of the library compiled with -DINFO_ESRF_PHASE_CLOCKS (the
 * default build returns INFO_ESRF_ERR_UNSUPPORTED).  Thread 0 of every CTA
 * sums clock64() deltas per phase over the launches since the last reset:
 * out[0..9] the cycles of the ten phases of a round (0 band matvec, 1 p^T y
 * push and cluster barrier 1, 2 alpha and right-hand-side prefetch wait,
 * 3 residual update and its dot products, 4 warp reductions and learned term, 5 reductions push
 * and cluster barrier 2, 6 CG and preconditioner scalars, 7 direction update,
 * 8 queue, halo push and cluster barrier 3, 9 refills), out[10] rounds,
 * out[11] set-up cycles, out[12] CTAs, each summed over CTAs; n values are
 * written (at most 13).  reset != 0 zeroes the counters afterwards.
 * Synchronizes the device. */
int info_esrf_band_phase_clocks(int64_t* out, int32_t n, int32_t reset);

/* Per-stage clock counts of the fused randomized eigensolver kernel (a4 of
 * the FP32 path, App. E and Halko, Martinsson & Tropp Alg. 5.3), same build
 * and contract as info_esrf_band_phase_clocks: thread 0 of cluster rank 0
 * sums clock64() deltas over the launches since the last reset: out[0] test
 * matrix, out[1] band products of the range finder, out[2] first and out[3]
 * second CholeskyQR pass, out[4] C Q, out[5] Q^T C Q partials, out[6]
 * Rayleigh-Ritz (merge, one-sided Jacobi, ordering), out[7] broadcast of the
 * Ritz coefficients, out[8] Ritz vectors, out[9] Gram matrices; out[10]
 * launches.  n values are written (at most 11). */
int info_esrf_ritz_phase_clocks(int64_t* out, int32_t n, int32_t reset);

/* One bounded wait on a shared-memory mbarrier, the wait every tensor-core
 * kernel of the BF16 path uses for its copies and MMAs (those give up after
 * about 2^32 cycles and report INFO_ESRF_ERR_TIMEOUT).  Thread 0 of one block
 * initializes a barrier expecting one arrival, arrives on it first when
 * `arrive` != 0, then waits for it at most `limit_cycles` SM cycles
 * (1 .. 2^32); *status_dev (device, one int32) becomes 0 when the wait
 * succeeded and the timeout status bit (128) when it ran out.  With arrive = 0
 * nothing ever arrives, so the call shows the bounded wait ending and the
 * context staying usable, without a fault or a hang.  Asynchronous on
 * `stream`; INFO_ESRF_ERR_INVALID_ARG for a null status or a limit out of
 * range. */
int info_esrf_wait_probe(int64_t limit_cycles, int32_t arrive, int32_t* status_dev, void* stream);

/* Band capacities the workspace layout uses for these arguments. */
int info_esrf_prepared_band_capacity(const info_esrf_grid* grid, int64_t N, int64_t d, int32_t Q,
                                     const info_esrf_options* opt, int64_t* max_oo, int64_t* max_xo);

/* ------------------------------------------------------------------------
 * Learned preconditioner correction.  Not in the paper: the paper's
 * preconditioner is the limited-memory one of App. E.  Each shifted system
 * may instead use M_q = a_q P_q^-1 + S_q^T S_q (a_q > 0; S_q a circulant
 * stencil over the observation index, (S r)_a = sum_{t=-h..h} w[t+h]
 * r_{(a+t) mod d}, h = info_esrf_learn_halfwidth()), symmetric positive
 * definite by construction.  a_q = exp(out_0) / sigma and w_q = out_1.. /
 * sqrt(sigma) (relative to C_q^-1 ~ I / sigma), out from a network applied to
 *   phi = (log(sigma)/5, (log(sigma)/5)^2, log(mean_a C(a,a))/5, log(b)/10),
 * sigma = s_q + 1, b the Gershgorin bound of C:
 *   h1 = tanh(W1 phi + b1), h2 = tanh(W2 h1 + b2), out = W3 h2 + b3,
 * parameters packed as one float vector W1[32][4], b1[32], W2[32][32],
 * b2[32], W3[18][32], b3[18] (info_esrf_learn_nparams() values).
 * Training minimizes L = mean_s ||a_s z_s + S_s^T S_s y_s - v_s||^2 / ||v_s||^2
 * over Krylov samples (v, y = C_q v, z = P_q^-1 y, phi) from
 * info_esrf_krylov_capture.  Sample arrays are [S][d] float, phi [S][4].
 * ------------------------------------------------------------------------ */
int32_t info_esrf_learn_nparams(void);
int32_t info_esrf_learn_halfwidth(void);

/* coef[s] = (a_s, w_s[2h+1]) for nshift feature rows (inference). */
int info_esrf_learn_coefficients(const float* theta_dev, int32_t nshift, const float* feat_dev, float* coef_dev,
                                 void* stream);

/* Scratch bytes for info_esrf_learn_loss_grad / _train with nsamp samples. */
size_t info_esrf_learn_scratch_size(int32_t nsamp);

/* grad = dL/dtheta and *loss_dev = L (device double, may be NULL), by the
 * hand-written forward and backward kernels; d <= 8192. */
int info_esrf_learn_loss_grad(const float* theta_dev, int32_t nsamp, int64_t d, const float* feat_dev,
                              const float* V_dev, const float* Y_dev, const float* Z_dev, float* grad_dev,
                              double* loss_dev, void* scratch_dev, size_t scratch_bytes, void* stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) at step number `step` >= 1;
 * m_dev and v_dev are the moment buffers (zero before the first step). */
int info_esrf_learn_adam_step(float* theta_dev, float* m_dev, float* v_dev, const float* grad_dev, int32_t step,
                              float lr, void* stream);

/* `steps` Adam steps starting at step number first_step, stream-ordered;
 * loss_hist_dev (device, `steps` doubles) receives L before each step. */
int info_esrf_learn_train(float* theta_dev, float* m_dev, float* v_dev, int32_t first_step, int32_t steps, float lr,
                          int32_t nsamp, int64_t d, const float* feat_dev, const float* V_dev, const float* Y_dev,
                          const float* Z_dev, float* grad_dev, double* loss_hist_dev, void* scratch_dev,
                          size_t scratch_bytes, void* stream);

/* Krylov samples of the method's own PCG (paper preconditioner, FP32 vectors):
 * prepares one analysis into the workspace (as info_esrf_prepare) and, for
 * each of the nsel systems sel_dev[] (number q * N + i: shift sigma = s_q + 1),
 * runs K iterations of that PCG from a random right-hand side (Philox keyed by
 * options.seed and the system, drawn again whenever ||r|| <= 1e-6 ||b||),
 * recording v = p/||p||, y = C_q v, z = P_q^-1 y and phi.
 * Outputs [nsel * K][d] and [nsel * K][4], float; d <= 10240. */
int info_esrf_krylov_capture(const info_esrf_grid* grid, int64_t N, const double* X_dev, int64_t d,
                             const int64_t* obs_idx_dev, const double* R_diag_dev, int32_t Q,
                             const info_esrf_options* opt, void* workspace, size_t ws_bytes, int32_t nsel,
                             const int32_t* sel_dev, int32_t K, float* V_dev, float* Y_dev, float* Z_dev,
                             float* feat_dev, void* stream);

/* Two-dimensional lattice form (BF16 path, precision INFO_ESRF_PRECISION_BF16):
 * where the observations are exactly the points (x0 + i sx, y0 + j sy),
 * i < Lx, j < Ly, of the two axes of extent > 1 of the grid, both periodic
 * (Lx sx and Ly sy the extents), the correction is M_q = a_q P_q^-1 + S_q S_q
 * with S_q the symmetric stencil over the lattice offsets (dx, dy),
 * dx^2 + dy^2 <= 8 (the 5 x 5 square), whose tap for squared length
 * 0, 1, 2, 4, 5, 8 is w_q[0..5] (the first six stencil outputs of the same
 * network).  Vectors of the lattice form are in lattice order, index i + Lx j.
 * The loss is the same with S S in place of S^T S. */

/* Scratch bytes for info_esrf_learn_loss_grad_lattice / _train_lattice with
 * nsamp samples of d = Lx Ly values. */
size_t info_esrf_learn_lattice_scratch_size(int32_t nsamp, int64_t d);

/* grad = dL/dtheta and *loss_dev = L of the lattice form (device, hand-written
 * forward and backward kernels); samples [nsamp][Lx Ly] float in lattice
 * order, feat [nsamp][4]; samples with v = 0 contribute nothing. */
int info_esrf_learn_loss_grad_lattice(const float* theta_dev, int32_t nsamp, int32_t Lx, int32_t Ly,
                                      const float* feat_dev, const float* V_dev, const float* Y_dev,
                                      const float* Z_dev, float* grad_dev, double* loss_dev, void* scratch_dev,
                                      size_t scratch_bytes, void* stream);

/* `steps` Adam steps on the lattice-form loss (as info_esrf_learn_train). */
int info_esrf_learn_train_lattice(float* theta_dev, float* m_dev, float* v_dev, int32_t first_step, int32_t steps,
                                  float lr, int32_t nsamp, int32_t Lx, int32_t Ly, const float* feat_dev,
                                  const float* V_dev, const float* Y_dev, const float* Z_dev, float* grad_dev,
                                  double* loss_hist_dev, void* scratch_dev, size_t scratch_bytes, void* stream);

/* Krylov samples of the BF16 path for the lattice form (options.precision
 * must be INFO_ESRF_PRECISION_BF16; the model in the options is ignored:
 * the paper's preconditioner runs): prepares one analysis into the
 * workspace and runs K iterations of the BF16 PCG from the systems' own
 * right-hand sides, recording for each of the nsel systems sel_dev[]
 * (number q * N + i) and iteration v = p / ||p||, y = (sigma p + C p) / ||p||
 * (p the BF16 direction the matvec used), z = P_q^-1 y and phi; all zero for
 * a system that stopped (residual at 1e-6 of its right-hand side) before that
 * iteration.  Outputs [nsel * K][d] and
 * [nsel * K][4] float in lattice order, *Lx and *Ly the lattice shape.
 * INFO_ESRF_ERR_UNSUPPORTED when the observations are not a 2-D lattice. */
int info_esrf_krylov_capture_lattice(const info_esrf_grid* grid, int64_t N, const double* X_dev, int64_t d,
                                     const int64_t* obs_idx_dev, const double* R_diag_dev, int32_t Q,
                                     const info_esrf_options* opt, void* workspace, size_t ws_bytes, int32_t nsel,
                                     const int32_t* sel_dev, int32_t K, float* V_dev, float* Y_dev, float* Z_dev,
                                     float* feat_dev, int32_t* Lx, int32_t* Ly, void* stream);

/* Versioned binary model file: 8-byte tag "IESRFNN1", int32 parameter count,
 * parameters (float), then the shift cut-off (double, see
 * options.learned_max_shift); little-endian.  Host arrays. */
int info_esrf_model_save(const char* path, const float* theta_host, double max_shift);
int info_esrf_model_load(const char* path, float* theta_host, double* max_shift);

/* Block-sparse BF16 matvec of the BF16 path (App. E: the localized-covariance
 * product of every PCG iteration, y_j = sigma_j p_j + C p_j for J systems at
 * once; C is shared by every system, Sec. 2.3), on the fifth-generation tensor
 * cores.  C (d_pad = 128 n_row_tiles rows and columns) is given as n_tiles
 * stored 128 x 64 blocks: row tile t owns blocks rowptr[t] .. rowptr[t+1]-1
 * (rowptr [n_row_tiles + 1], int32, rowptr[0] = 0, rowptr[n_row_tiles] =
 * n_tiles, every row tile at least one block), block b covering columns
 * 64 colblk[b] .. 64 colblk[b] + 63 (colblk [n_tiles], < d_pad / 64).  Each
 * block is two BF16 planes (uint16 bit patterns, row-major [n_tiles][128][64]):
 * C = C_hi + C_lo.  P [J][d_pad] BF16 directions, sigma [J] FP32 shifts.
 * Outputs: Y [J][d_pad] FP32 = sigma P + (C_hi + C_lo) P (products exact,
 * FP32 accumulation) and, if pty_dev is not NULL, pty [n_row_tiles][J] FP32,
 * the dot product of P_j and Y_j over each row tile's 128 rows.  status_dev
 * (may be NULL) receives bit 7 if a bounded device wait expired.  Every
 * pointer 16-byte aligned.  Asynchronous; allocates nothing. */
int info_esrf_bf16_tile_matvec(int32_t n_row_tiles, const int32_t* rowptr_dev, const int32_t* colblk_dev,
                               int64_t n_tiles, const uint16_t* C_hi_dev, const uint16_t* C_lo_dev, int32_t J,
                               const uint16_t* P_dev, const float* sigma_dev, float* Y_dev, float* pty_dev,
                               int32_t* status_dev, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* INFO_ESRF_STAGES_H */
