// Internal layout shared by the host API and the kernels (not part of the ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace infoesrf {

constexpr int kMaxProblems = 64;      // problems per batched call
constexpr int kMaxRitz = 32;          // k_R + oversampling
constexpr int kMaxK = 24;             // Ritz vectors used by the preconditioner
constexpr int kLearnH = 8;            // half-width of the learned stencil
constexpr int kLearnTaps = 2 * kLearnH + 1;
constexpr int kLearnOut = 1 + kLearnTaps;  // log a and the taps
constexpr int kLearnT = 4 * kLearnH + 1;   // taps of S^T S
constexpr int kLearnParams = 1810;    // network parameters (see learn.cu)
constexpr int kLatPts = 25;           // points of the 2-D lattice stencil (dx^2 + dy^2 <= 8, the 5 x 5 square)
constexpr int kLatBins = 6;           // its taps: one per squared length 0, 1, 2, 4, 5, 8
// Point n of the lattice stencil: dx = n % 5 - 2, dy = n / 5 - 2; its tap is
// the rank of dx^2 + dy^2 among 0, 1, 2, 4, 5, 8.
__host__ __device__ inline int lat_dx(int n) { return n % 5 - 2; }
__host__ __device__ inline int lat_dy(int n) { return n / 5 - 2; }
__host__ __device__ inline int lat_bin(int n) {
  const int dx = lat_dx(n), dy = lat_dy(n), r2 = dx * dx + dy * dy;
  return r2 < 3 ? r2 : (r2 == 4 ? 3 : (r2 == 5 ? 4 : 5));
}
constexpr int kThreads = 256;         // CTA size of the persistent PCG kernel

// Status bits written by kernels (ws status word 0).
enum : int32_t {
  kStatBadObs = 1 << 0,        // obs index out of range or not strictly increasing
  kStatBadR = 1 << 1,          // R <= 0 or not finite
  kStatNonFinite = 1 << 2,     // non-finite ensemble value
  kStatBandOverflow = 1 << 3,  // more neighbours than the band capacity
  kStatBreakdown = 1 << 4,     // PCG breakdown (p^T A p <= 0 or NaN)
  kStatNotConverged = 1 << 5,  // iteration cap reached
  kStatEigFail = 1 << 6,       // randomized eigensolver lost rank
  kStatTimeout = 1 << 7,       // a bounded device wait expired
  kStatTileOverflow = 1 << 8,  // more C blocks than the tile capacity
};

// BF16 block-tile path: C stored in 128 x 64 blocks (row tile x column block)
// of tile-ordered observations.
constexpr int kTileM = 128;
constexpr int kTileK = 64;

struct TileMmArgs {
  const int32_t* rowptr;        // [nrt + 1] first block of each row tile
  const int32_t* colblk;        // [tiles] column block of each stored block
  const __nv_bfloat16* P;       // [J][d_pad] directions
  const float* sigma;           // [J] shifts (NULL: zero)
  const int32_t* active;        // [ceil(J / 16)] nonzero: the unit of 16 systems has an unconverged one (or NULL: all)
  float* Y;                     // [J][d_pad] sigma p + C p
  float* pty;                   // partial p^T y per row tile (or NULL): [nrt][J], or [J][nrt] if pty_by_system
  int32_t* status;              // status bits (kStatTimeout), or NULL
  int64_t d_pad;
  int32_t J, nrt, nchunks, pty_by_system;
  int32_t units;                // number of nonzero flags in `active` (ignored when it is NULL)
  int32_t* ulist;               // [ceil(J / 16)] scratch: the ordered list of those units
};
constexpr int kTileUnit = 16;   // systems per unit of the tile matvec (one 16-row TMA box of P)
int launch_tile_mm(TileMmArgs a, const void* chi, const void* clo, int64_t ntiles, cudaStream_t st);
constexpr int kStK = 128;           // member slots of the tensor-core state update (N <= 128)
constexpr int kTileDotRows = 512;   // rows per partial dot product of the BF16 PCG
// Dot values per system of the BF16 PCG: r^T r, f = Phi^T r, g = (C Phi)^T r,
// then u^T u of the learned term.
__host__ __device__ inline int tile_dot_values(int k) { return 2 * k + 2; }
constexpr int kBcgMaxS = 64;        // block CG: largest block (members per node)
struct ProblemDev;
int run_bcg(const ProblemDev& p, const ProblemDev* dp, cudaStream_t st);
struct ProblemDev;
struct ProblemTable;
int64_t tile_max_members();
// Set-up (tile order, block patterns, C blocks), the Ritz-stage matvec, the
// per-problem PCG loop (synchronizes the stream once per iteration) and the
// finish (quadrature sum and state update) of the BF16 path.
void launch_tile_setup(const ProblemTable& tab, const ProblemDev* dtab, cudaStream_t st);
void launch_tile_ritz_matvec(const ProblemTable& tab, const ProblemDev* dtab, int src, cudaStream_t st);
// mm_ms / mm_count (host, may be NULL): summed device time and count of the
// tensor-core matvec launches, from CUDA events on st around each launch.
int run_tile_pcg(const ProblemDev& p, const ProblemDev* dp, cudaStream_t st, double* mm_ms, int* mm_count);
void launch_tile_finish(const ProblemTable& tab, const ProblemDev* dtab, cudaStream_t st);
// The state update on the tensor cores (tile_state.cu): 0 when launched for
// every BF16 problem; otherwise the caller runs the CUDA-core kernel.
int launch_tile_state_mma(const ProblemTable& tab, const ProblemDev* dtab, cudaStream_t st);
// The C blocks of the set-up on the tensor cores (tile_form.cu), same contract.
int launch_tile_form_mma(const ProblemTable& tab, const ProblemDev* dtab, cudaStream_t st);
// Lattice of the observations of each BF16 problem with a learned model (or
// for a capture): detection and the stencil tables (tile_learn.cu).
void launch_tile_lattice(const ProblemTable& tab, const ProblemDev* dtab, cudaStream_t st);
// Krylov samples of the BF16 path (paper preconditioner): directions and
// their images of the selected systems at iterations 1..K, in lattice order.
struct TileCapture {
  int32_t nsel, K;
  const int32_t* sel;   // [nsel] systems q * N + i
  float* V;             // [nsel * K][d]
  float* Y;
};
int run_tile_pcg_capture(const ProblemDev& p, const ProblemDev* dp, const TileCapture& cap, float* Z, float* feat,
                         cudaStream_t st);
// u = S r for the listed learned systems, with partial sums of u^T u
// (tile_learn.cu); stages of the BF16 PCG loop.
void launch_tile_learn_u(const ProblemDev& p, const ProblemDev* dp, const int32_t* list, int64_t count, int nsub,
                         cudaStream_t st);
void launch_tile_capture_record(const ProblemDev& p, const ProblemDev* dp, const TileCapture& cap, int it,
                                cudaStream_t st);
void launch_tile_capture_finish(const ProblemDev& p, const ProblemDev* dp, const TileCapture& cap, float* Z,
                                float* feat, cudaStream_t st);

struct GridDev {
  int64_t ext[3];
  int64_t reach[3];      // candidate half-window per axis (grid units)
  int32_t whole[3];      // 1: scan the whole axis
  int32_t periodic[3];
  int32_t chordal;
  int32_t pad_;
  double inv_c[3];       // 1 / half-width
};

// Everything one problem needs on the device.  Pointers into the caller's
// buffers and into the workspace; sizes; offsets into the global group space.
struct ProblemDev {
  GridDev grid;
  int64_t n, N, d;
  int32_t Q, kR, l, do_mean, do_pert, rule, precision, fixed_iters;
  int32_t max_iter, power_iters, pad0_, pad_;
  double tol, ell_fixed, sqrt_nm1;
  uint64_t seed;
  int64_t max_oo, max_xo;      // ELL capacities (obs-obs, state-obs)
  // inputs (caller-owned, device)
  const double* X;      // [N][n]
  const int64_t* obs;   // [d] (subsampling; NULL with a general H)
  const int64_t* H_rowptr;   // general observation operator (CSR, [d + 1]), or NULL
  const int64_t* H_col;      // [H_nnz]
  const double* H_val;       // [H_nnz]
  int64_t H_nnz;
  const double* y;      // [d] (mean update only)
  const double* R;      // [d]
  // outputs (caller-owned, device)
  double* mu_a;         // [n]
  double* A_a;          // [N][n]
  // workspace
  double* mu;           // [n]
  double* d2tab;        // [ext0 + ext1 + ext2] (axis distance / half-width)^2 by index offset
  void* Zt;             // [n][N] T normalized anomalies, state-major
  void* W;              // [d][N] T observed anomalies W = H Z
  double* rinv;         // [d] R^-1/2
  double* bmean;        // [d] R^-1/2 (y - H mu)
  double* scal;         // [8] 0 gershgorin bound, 1 min diag C, 2 ell, 3 nonzeros of C (BF16 path), 4 sum of diag C
  int32_t* status;      // [4]
  double* s;            // [Q] quadrature nodes
  double* p;            // [Q] quadrature weights
  void* oo_val;         // [max_oo][d] T: C(a, b) (ELL, transposed)
  int32_t* oo_col;      // [max_oo][d]
  int32_t* oo_nnz;      // [d]
  void* xo_val;         // [max_xo][n] T: Sxh(x, b) (ELL, transposed)
  int32_t* xo_col;      // [max_xo][n]
  int32_t* xo_nnz;      // [n]
  // randomized eigensolver
  void* Om;             // [d][l] T test matrix / range basis
  void* Yb;             // [d][l] T image of the basis under C
  double* Gm;           // [l][l] Gram / projected matrix
  double* Rm;           // [l][l] Cholesky factor / eigenvectors
  double* ev;           // [l] eigenvalues (descending)
  void* Phi;            // [d][kR] T Ritz vectors
  void* CPhi;           // [d][kR] T C Phi
  double* theta;        // [kR] Ritz values of C
  double* gram;         // [3][kR][kR]: Phi^T Phi, A^T Phi, A^T A with A = C Phi
  // learned correction a_q P_q^-1 + S_q^T S_q (optional)
  const float* learned_model;   // network parameters, NULL: none
  double learned_max_shift;     // > 0: learned term only for sigma <= this
  float* learn_coef;            // [Q + 1][kLearnOut]: a_q, taps (slot Q: mean system)
  float* learn_T;               // [Q + 1][kLearnT]: taps of T_q = S_q^T S_q, offsets -2h..2h
  // batched PCG
  // Systems are numbered hardest first: sid 0 is the mean system (shift 1)
  // when requested, then the perturbation systems node-major,
  // sid = mean_sys + q * N + i (s_q increases with q).
  int32_t JT, groups_per_q, num_groups, group_base;
  int32_t nsys, mean_sys;   // number of systems; 1 if sid 0 is the mean system else 0
  int32_t sys_base, pad2_;  // first sid of this problem in a batch-wide numbering
  void* U;              // [nsys][d] T solutions u of C_q u = b
  int32_t* iters;       // [nsys]
  double* relres;       // [nsys] final ||r|| / ||b|| (recurrence)
  double* Vbar;         // [d][N + 1] FP64 R^-1/2 sum_q p_q u_q (last column: mean)
  void* VbarT;          // [d][N + 1] T copy for the state apply
  // BF16 block-tile path (precision 2).  Observations are numbered in tile
  // order: position a' of original observation a is the rank of the Morton
  // code of its grid point.  C is stored in 128 x 64 blocks (kTileM x kTileK)
  // of tile-ordered rows and columns; the state update runs over state tiles
  // of 128 consecutive grid points against the same 64-column blocks.
  int32_t nrt, nblk;            // row tiles (d_pad / 128), column blocks (d_pad / 64)
  int32_t nst, nsort;           // state tiles (ceil(n / 128)); sort length (power of two >= d)
  int64_t d_pad, tile_cap, st_cap;
  uint64_t* skey;               // [nsort] Morton keys (sort scratch)
  int32_t* sidx;                // [nsort] original observation of each key
  int32_t* tpos_src;            // [d_pad] original observation at tile position (-1: padding)
  int32_t* obs_tpos;            // [d] tile position of each original observation
  int32_t* tbox;                // [nblk][6] bounding box of each column block (lo, hi per axis)
  int32_t* tcount;              // [nrt + nst] blocks per row tile / state tile
  int32_t* rowptr;              // [nrt + 1] first stored block of each row tile
  int32_t* colblk;              // [tile_cap] column block of each stored block
  int32_t* st_rowptr;           // [nst + 1]
  int32_t* st_colblk;           // [st_cap]
  __nv_bfloat16* Chi;           // [tile_cap][128][64] bf16(C)
  __nv_bfloat16* Clo;           // [tile_cap][128][64] bf16(C - Chi)
  float* Wp;                    // [d_pad][N] W in tile order (0 at padding)
  float* rinvp;                 // [d_pad] R^-1/2 in tile order (0 at padding)
  // BF16 PCG state: systems j = sid (mean first, then q * N + i), J = nsys
  __nv_bfloat16* Pdir;          // [J][d_pad] search directions (bf16, as used)
  float* Yv;                    // [J][d_pad] sigma p + C p
  float* Xv;                    // [J][d_pad] iterates
  float* Rv;                    // [J][d_pad] residuals
  float* pty;                   // [J][nrt] p^T y per row tile
  double* dots;                 // [J][2 kR + 1][nsub] partial r^T r, Phi^T r, (C Phi)^T r per row block
  double* dsum;                 // [J][2 kR + 1] their sums
  double* sysd;                 // [J][8] per-system scalars (see tile_pcg.cu)
  float* lcoef;                 // [J][2 kR] LMP coefficients of the current direction update
  float* sigmaf;                // [J] shift per system (FP32)
  int32_t* active;              // [J] 1 while the system runs
  int32_t* unit_active;         // [ceil(J / 16)] 1 while a unit of 16 systems has a running system
  int32_t* unit_list;           // [ceil(J / 16)] the tile matvec's ordered list of those units
  int32_t* nactive;             // [2] running systems; copy of status[0] for the host
  int32_t* alist;               // [J] the running systems (unordered), rebuilt every iteration
  // learned correction on the BF16 path, for observations on every point of a
  // periodic 2-D lattice (the stencil S over lattice offsets, see tile_learn.cu)
  int32_t* lat_info;            // [16] device: ok, Lx, Ly, x0, y0, sx, sy, retries, learned systems
  int32_t* lat_tpos;            // [d] tile position of lattice point i + Lx j
  int32_t* lat_nbr;             // [d_pad][kLatPts] tile positions of the stencil points of each row
  float* learn_u;               // [J][d_pad] u = S r of the current residual (learned systems)
  int32_t* learn_on;            // [J] 1: the system applies the learned term; 2: retry without it
  // state update on the tensor cores (tile_state.cu): BF16 hi and lo planes
  // of the operands in tile order, made by the finish
  __nv_bfloat16* st_W;          // [3][d_pad][kStK] W in three planes, members padded to kStK
  __nv_bfloat16* st_V;          // [2][st_NV][d_pad] Vbar^T of the members, padded to st_NV columns
  float* st_vm;                 // [d_pad] the mean column of Vbar
  int4* st_xyz;                 // [d_pad] grid coordinates of each tile position (w = -1: padding)
  int32_t st_NV, pad4_;
  // block CG (solver 2): blocks = the mean system (one column) and one block of
  // N columns per node; vectors [nsys][d] of the bulk type, X is U
  int32_t bcg_nblocks, pad3_;
  void* bcg_R;                  // residuals
  void* bcg_P;                  // directions
  void* bcg_Q;                  // C_q P
  double* bcg_G1;               // [nblocks][kBcgMaxS][kBcgMaxS] P^T Q
  double* bcg_G2;               // R^T R of the new residual
  double* bcg_RR;               // R^T R of the current residual
  double* bcg_alpha;            // block step
  double* bcg_beta;             // block direction update
  double* bcg_bn2;              // [nsys] ||b_i||^2
  int32_t* bcg_state;           // [nblocks] 0 running, 1 stopped, 2 breakdown
  int32_t* bcg_running;         // [1] running blocks after the last iteration
};

// Launch plan of the multi-shift CG kernel (host side): CTAs per cluster,
// observation rows per CTA (a multiple of 4), length of each full copy of p,
// shift slots per chain (a multiple of 4), band slots of C per row, element
// size, and for every chain-group size LC = 1..4 whether the CTA's slice of C
// and the shifted directions fit in shared memory (else they are read from
// the band in L2, or kept in the CTA's scratch slice) with the resulting
// dynamic size; LCmax is the largest LC that fits at all.
struct MsPlan {
  int CS, Rc, dall, Qs, cap, esz, LCmax;
  int c_smem[5], ps_smem[5];
  size_t dyn[5];
  size_t scratch_bytes;
};

struct ProblemTable {
  int32_t count;
  int32_t total_groups;
  int32_t total_sys;
  int32_t cluster_size;         // options.cluster_size (0: chosen from d)
  ProblemDev p[kMaxProblems];
  // host-only (never uploaded): the solver and the multi-shift plan
  int32_t solver;
  MsPlan ms;
  void* ms_scratch;
};

// Launchers (one per stage).  All are stream-ordered and never synchronize.
void launch_prepare(const ProblemTable& tab, ProblemDev* dtab, cudaStream_t st);
void launch_anomalies(const ProblemTable& tab, const ProblemDev* dtab, cudaStream_t st);
void launch_bands(const ProblemTable& tab, const ProblemDev* dtab, cudaStream_t st);
void launch_band_obs(const ProblemTable& tab, const ProblemDev* dtab, cudaStream_t st);
void launch_band_state(const ProblemTable& tab, const ProblemDev* dtab, cudaStream_t st);
void launch_quadrature(const ProblemTable& tab, const ProblemDev* dtab, cudaStream_t st);
void launch_ritz(const ProblemTable& tab, const ProblemDev* dtab, cudaStream_t st);
int launch_ritz_cluster(const ProblemTable& tab, const ProblemDev* dtab, cudaStream_t st);
bool ritz_cluster_fits(int64_t d, int l);
int launch_pcg(const ProblemTable& tab, const ProblemDev* dtab, int32_t* counter, void* scratch,
               size_t scratch_bytes, int num_sms, cudaStream_t st);
// accumulate = false: vbar was written by the solver (multi-shift CG)
void launch_finish(const ProblemTable& tab, const ProblemDev* dtab, cudaStream_t st, bool accumulate = true);
void launch_count_neighbours(const GridDev& g, const int64_t* obs, int64_t d, int64_t n,
                             int64_t* out2, cudaStream_t st);
void launch_philox(uint64_t seed, int64_t count, double* out, cudaStream_t st);
void launch_quadrature_nodes(int32_t Q, double ell, int32_t rule, double* s, double* p, cudaStream_t st);
void launch_obs_matvec(const ProblemDev& pr, const ProblemDev* dpr, int32_t nvec, const double* P,
                       const double* sigma, double* Y, cudaStream_t st);
void launch_lmp_apply(const ProblemDev& pr, const ProblemDev* dpr, int32_t nvec, const double* Rv,
                      const double* sigma, double* Z, cudaStream_t st);

// Host-side count of kernel launches issued by this library.
void note_launches(int n);

// Learned correction: per-shift coefficients, Krylov capture.
void launch_learn_coef(const ProblemTable& tab, const ProblemDev* dtab, cudaStream_t st);
int launch_krylov_capture(const ProblemTable& tab, const ProblemDev* dtab, int nsel, const int32_t* sel, int K,
                          float* V, float* Y, float* Z, float* feat, cudaStream_t st);

// Cluster-resident PCG for 1-D observation networks (FP32), one launch per
// problem: p is the host copy, dp the device copy of the same problem.
bool band1d_eligible(const ProblemDev& p);
int band1d_cluster_size(const ProblemDev& p, int requested);
int launch_pcg_band1d(const ProblemDev& p, const ProblemDev* dp, int CS, int32_t* queue, int32_t* fallback,
                      int num_sms, cudaStream_t st);

// Multi-shift CG (one Krylov run per member for all shifts): plan and launch.
// mscg_plan returns -1 when one chain's full p does not fit a CTA.
int mscg_plan(const ProblemTable& tab, int num_sms, int requested_cs, MsPlan* out);
int launch_mscg(const ProblemTable& tab, const ProblemDev* dtab, const MsPlan& pl, int num_sms, cudaStream_t st);

// Work counters of the PCG stage: [0] group queue of the general kernel,
// [1 + i] system queue of the band kernel for problem i, [1 + kMaxProblems + i]
// its fall-back flag.
constexpr int kCounterInts = 256;
static_assert(1 + 2 * kMaxProblems <= kCounterInts, "PCG counter area");

// PCG vector scratch per CTA when vectors do not fit in shared memory.
size_t pcg_scratch_bytes(const ProblemTable& tab, int num_sms);
int pcg_jt(int precision);

}  // namespace infoesrf
