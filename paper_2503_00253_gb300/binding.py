"""Thin Python binding of the C ABI (include/info_esrf.h, include/info_esrf_stages.h).

Argument marshalling only: ctypes structures that mirror the C structs, and
functions with the C names that take torch tensors, pass their device
pointers and the current CUDA stream, and return the outputs.  Every step of
the analysis runs inside ``libinfo_esrf.so``; if the library is missing the
import fails, there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import torch

from . import build as _build

c_int32, c_int64, c_double, c_uint64, c_void_p = (ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                                                  ctypes.c_uint64, ctypes.c_void_p)

OK = 0
NOT_CONVERGED = 1
ERR_INVALID_ARG = -1
ERR_BAD_OBS_INDEX = -2
ERR_NONPOSITIVE_R = -3
ERR_WORKSPACE = -4
ERR_CUDA = -5
ERR_NONFINITE = -6
ERR_BAND_OVERFLOW = -7
ERR_BREAKDOWN = -8
ERR_UNSUPPORTED = -9
ERR_TIMEOUT = -10

PRECISION_FP64 = 0
PRECISION_FP32 = 1
PRECISION_BF16 = 2
RULE_ELLIPTIC = 0
RULE_GAUSS_LEGENDRE = 1
SOLVER_PCG = 0
SOLVER_MULTISHIFT = 1
SOLVER_BLOCK = 2

ITEM = dict(scalars=0, status=1, quad_s=2, quad_p=3, theta=4, phi=5, cphi=6, oo_val=7, oo_col=8,
            oo_nnz=9, xo_val=10, xo_col=11, xo_nnz=12, W=13, mu=14)


class Grid(ctypes.Structure):
    _fields_ = [("shape", c_int64 * 3), ("periodic", c_int32 * 3), ("chordal", c_int32),
                ("half_width", c_double * 3)]


class Options(ctypes.Structure):
    _fields_ = [("precision", c_int32), ("ritz_rank", c_int32), ("oversample", c_int32),
                ("power_iters", c_int32), ("max_iter", c_int32), ("fixed_iters", c_int32),
                ("rule", c_int32), ("cluster_size", c_int32), ("ell", c_double), ("seed", c_uint64),
                ("max_neighbors", c_int64), ("learned_model", c_void_p), ("learned_max_shift", c_double),
                ("system_iters", c_void_p), ("phase_events", ctypes.POINTER(c_void_p)),
                ("solver", c_int32), ("reserved_", c_int32), ("tile_capacity", c_int64),
                ("state_tile_capacity", c_int64)]


class Stats(ctypes.Structure):
    _fields_ = [("status", c_int32), ("device_flags", c_int32), ("iters_max", c_int32),
                ("n_systems", c_int32), ("iters_mean", c_double), ("n_unconverged", c_int32),
                ("solver_path", c_int32), ("max_rel_resid", c_double), ("ell_used", c_double),
                ("gershgorin", c_double), ("learned", c_int32), ("pad_", c_int32), ("matvec_ms", c_double),
                ("tile_blocks", c_int64), ("c_nnz", c_double), ("matvec_launches", c_int32), ("pad2_", c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("pad")}


class ProblemC(ctypes.Structure):
    _fields_ = [("grid", Grid), ("N", c_int64), ("d", c_int64), ("Q", c_int32), ("pad_", c_int32),
                ("tol", c_double), ("X", c_void_p), ("obs_idx", c_void_p), ("y", c_void_p),
                ("R_diag", c_void_p), ("mu_a", c_void_p), ("A_a", c_void_p), ("max_oo", c_int64),
                ("max_xo", c_int64), ("H_rowptr", c_void_p), ("H_col", c_void_p), ("H_val", c_void_p),
                ("H_nnz", c_int64)]


_LIB = None


def library() -> ctypes.CDLL:
    """Loads libinfo_esrf.so (building it first if sources are newer); with
    INFO_ESRF_PHASE_CLOCKS=1 in the environment, the instrumented build
    libinfo_esrf_phase.so instead."""
    global _LIB
    if _LIB is not None:
        return _LIB
    phase = os.environ.get("INFO_ESRF_PHASE_CLOCKS") == "1"
    path = _build.library_path(phase)
    if not _build.up_to_date(phase):
        path = _build.build(phase_clocks=phase)
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing; run build() first")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    sig = {
        "info_esrf_default_options": (None, [P(Options)]),
        "info_esrf_error_string": (ctypes.c_char_p, [c_int32]),
        "info_esrf_version": (c_int32, []),
        "info_esrf_neighbor_counts": (c_int32, [P(Grid), c_int64, c_void_p, c_void_p, c_void_p,
                                                P(c_int64), P(c_int64)]),
        "info_esrf_workspace_size": (ctypes.c_size_t, [P(Grid), c_int64, c_int64, c_int32, P(Options)]),
        "info_esrf_batched_workspace_size": (ctypes.c_size_t, [P(ProblemC), c_int32, P(Options)]),
        "info_esrf_mean_update": (c_int32, [P(Grid), c_int64, c_void_p, c_int64, c_void_p, c_void_p,
                                            c_void_p, c_double, P(Options), c_void_p, ctypes.c_size_t,
                                            c_void_p, c_void_p, P(Stats)]),
        "info_esrf_perturbation_update": (c_int32, [P(Grid), c_int64, c_void_p, c_int64, c_void_p,
                                                    c_void_p, c_int32, c_double, P(Options), c_void_p,
                                                    ctypes.c_size_t, c_void_p, c_void_p, P(Stats)]),
        "info_esrf_analysis": (c_int32, [P(Grid), c_int64, c_void_p, c_int64, c_void_p, c_void_p,
                                         c_void_p, c_int32, c_double, P(Options), c_void_p,
                                         ctypes.c_size_t, c_void_p, c_void_p, c_void_p, P(Stats)]),
        "info_esrf_analysis_batched": (c_int32, [P(ProblemC), c_int32, P(Options), c_void_p,
                                                 ctypes.c_size_t, c_void_p, P(Stats)]),
        "info_esrf_philox_normals": (c_int32, [c_uint64, c_int64, c_void_p, c_void_p]),
        "info_esrf_quadrature_nodes": (c_int32, [c_int32, c_double, c_int32, c_void_p, c_void_p,
                                                 c_void_p]),
        "info_esrf_prepare": (c_int32, [P(Grid), c_int64, c_void_p, c_int64, c_void_p, c_void_p,
                                        c_int32, P(Options), c_void_p, ctypes.c_size_t, c_void_p]),
        "info_esrf_prepared_obs_matvec": (c_int32, [P(Grid), c_int64, c_int64, c_int32, P(Options),
                                                    c_void_p, ctypes.c_size_t, c_int32, c_void_p,
                                                    c_void_p, c_void_p, c_void_p]),
        "info_esrf_prepared_lmp_apply": (c_int32, [P(Grid), c_int64, c_int64, c_int32, P(Options),
                                                   c_void_p, ctypes.c_size_t, c_int32, c_void_p,
                                                   c_void_p, c_void_p, c_void_p]),
        "info_esrf_prepared_export": (c_int32, [P(Grid), c_int64, c_int64, c_int32, P(Options),
                                                c_void_p, ctypes.c_size_t, c_int32, c_void_p,
                                                ctypes.c_size_t, c_void_p]),
        "info_esrf_launch_count": (c_int64, []),
        "info_esrf_learn_nparams": (c_int32, []),
        "info_esrf_learn_halfwidth": (c_int32, []),
        "info_esrf_learn_coefficients": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p]),
        "info_esrf_learn_scratch_size": (ctypes.c_size_t, [c_int32]),
        "info_esrf_learn_loss_grad": (c_int32, [c_void_p, c_int32, c_int64, c_void_p, c_void_p, c_void_p,
                                                c_void_p, c_void_p, c_void_p, c_void_p, ctypes.c_size_t,
                                                c_void_p]),
        "info_esrf_learn_adam_step": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_int32,
                                                ctypes.c_float, c_void_p]),
        "info_esrf_learn_train": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_int32, ctypes.c_float,
                                            c_int32, c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                            c_void_p, c_void_p, ctypes.c_size_t, c_void_p]),
        "info_esrf_krylov_capture": (c_int32, [P(Grid), c_int64, c_void_p, c_int64, c_void_p, c_void_p,
                                               c_int32, P(Options), c_void_p, ctypes.c_size_t, c_int32,
                                               c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_void_p,
                                               c_void_p]),
        "info_esrf_autotune": (c_int32, [P(ProblemC), c_int32, P(Options), c_void_p, ctypes.c_size_t, c_void_p,
                                          P(c_double)]),
        "info_esrf_model_save": (c_int32, [ctypes.c_char_p, c_void_p, c_double]),
        "info_esrf_model_load": (c_int32, [ctypes.c_char_p, c_void_p, P(c_double)]),
        "info_esrf_fma_probe": (c_int32, [c_int32, c_int64, P(c_double), P(c_double), c_void_p]),
        "info_esrf_prepared_band_capacity": (c_int32, [P(Grid), c_int64, c_int64, c_int32, P(Options),
                                                       P(c_int64), P(c_int64)]),
        "info_esrf_band_phase_clocks": (c_int32, [P(c_int64), c_int32, c_int32]),
        "info_esrf_ritz_phase_clocks": (c_int32, [P(c_int64), c_int32, c_int32]),
        "info_esrf_wait_probe": (c_int32, [c_int64, c_int32, c_void_p, c_void_p]),
        "info_esrf_learn_lattice_scratch_size": (ctypes.c_size_t, [c_int32, c_int64]),
        "info_esrf_learn_loss_grad_lattice": (c_int32, [c_void_p, c_int32, c_int32, c_int32, c_void_p, c_void_p,
                                                        c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                                        ctypes.c_size_t, c_void_p]),
        "info_esrf_learn_train_lattice": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_int32, ctypes.c_float,
                                                    c_int32, c_int32, c_int32, c_void_p, c_void_p, c_void_p,
                                                    c_void_p, c_void_p, c_void_p, c_void_p, ctypes.c_size_t,
                                                    c_void_p]),
        "info_esrf_krylov_capture_lattice": (c_int32, [P(Grid), c_int64, c_void_p, c_int64, c_void_p, c_void_p,
                                                       c_int32, P(Options), c_void_p, ctypes.c_size_t, c_int32,
                                                       c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_void_p,
                                                       P(c_int32), P(c_int32), c_void_p]),
        "info_esrf_bf16_tile_matvec": (c_int32, [c_int32, c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_int32,
                                                 c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


class InfoEsrfError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = library().info_esrf_error_string(code).decode()
        super().__init__(f"{where}: {msg} (code {code})")
        self.code = code


def _check(code: int, where: str, allow_warning: bool = True) -> int:
    if code < 0 or (code > 0 and not allow_warning):
        raise InfoEsrfError(code, where)
    return code


# ---------------------------------------------------------------------------
# Marshalling helpers
# ---------------------------------------------------------------------------

def make_grid(grid) -> Grid:
    """Converts any object with shape / periodic / half_width / chordal attributes."""
    g = Grid()
    shape = list(grid.shape) + [1] * (3 - len(grid.shape))
    per = list(grid.periodic) + [False] * (3 - len(grid.periodic))
    hw = list(grid.half_width) + [1.0] * (3 - len(grid.half_width))
    for i in range(3):
        g.shape[i] = int(shape[i])
        g.periodic[i] = 1 if per[i] else 0
        g.half_width[i] = float(hw[i])
    g.chordal = 1 if getattr(grid, "chordal", True) else 0
    return g


def make_options(precision: int = PRECISION_FP64, ritz_rank: int = 10, oversample: int = 10,
                 power_iters: int = 1, max_iter: int = 1000, fixed_iters: int = 0,
                 rule: int = RULE_ELLIPTIC, ell: float = 0.0, seed: int = 0x1234ABCD,
                 max_neighbors: int = 0, learned_model: Optional[torch.Tensor] = None,
                 learned_max_shift: float = 0.0, system_iters: Optional[torch.Tensor] = None,
                 cluster_size: int = 0, solver: int = SOLVER_PCG, tile_capacity: int = 0,
                 state_tile_capacity: int = 0) -> Options:
    o = Options()
    library().info_esrf_default_options(ctypes.byref(o))
    o.precision, o.ritz_rank, o.oversample, o.power_iters = precision, ritz_rank, oversample, power_iters
    o.max_iter, o.fixed_iters, o.rule, o.ell, o.seed = max_iter, fixed_iters, rule, ell, seed
    o.max_neighbors = max_neighbors
    o.cluster_size = cluster_size
    o.solver = solver
    o.tile_capacity, o.state_tile_capacity = tile_capacity, state_tile_capacity
    if system_iters is not None:
        _need(system_iters, torch.int32, "system_iters")
        o.system_iters = system_iters.data_ptr()
        o._iters_keep = system_iters
    if learned_model is not None:
        _need(learned_model, torch.float32, "learned_model")
        o.learned_model = learned_model.data_ptr()
        o.learned_max_shift = float(learned_max_shift)
        o._model_keep = learned_model
    return o


def _need(t: torch.Tensor, dtype, name: str):
    if not isinstance(t, torch.Tensor) or t.dtype != dtype or not t.is_cuda or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous CUDA tensor of {dtype}")


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def set_phase_events(options: Options, events) -> None:
    """Records the 5 torch.cuda.Event objects at the library's phase boundaries (None: off)."""
    if events is None:
        options.phase_events = None
        return
    arr = (c_void_p * 5)(*[e.cuda_event for e in events])
    options._phase_keep = arr
    options.phase_events = ctypes.cast(arr, ctypes.POINTER(c_void_p))


def launch_count() -> int:
    return int(library().info_esrf_launch_count())


BAND_PHASES = ("band matvec", "p^T y push + cluster barrier 1", "alpha, RHS prefetch wait",
               "residual update, Phi^T r, A^T r", "warp reductions, learned term (r halo push, barrier 2a, T r)",
               "reductions push + cluster barrier 2", "decisions (CG scalars, LMP algebra)",
               "direction update z, p", "queue, halo push, cluster barrier 3", "refills, RHS prefetch issue")


def band_phase_clocks(reset: bool = True) -> dict:
    """Per-round phase cycles of the 1-D band PCG kernel since the last reset
    (instrumented build only: INFO_ESRF_PHASE_CLOCKS=1), averaged over CTAs."""
    out = (c_int64 * 13)()
    _check(library().info_esrf_band_phase_clocks(out, 13, 1 if reset else 0), "info_esrf_band_phase_clocks")
    v = list(out)
    rounds, ctas = v[10], max(v[12], 1)
    per_round = {name: v[i] / max(rounds, 1) for i, name in enumerate(BAND_PHASES)}
    return {"cycles_per_round": per_round, "rounds_per_cta": rounds / ctas, "setup_cycles_per_cta": v[11] / ctas,
            "ctas": v[12], "total_per_round": sum(v[:10]) / max(rounds, 1)}


RITZ_PHASES = ("test matrix", "range-finder band products", "CholeskyQR pass 1", "CholeskyQR pass 2", "C Q",
               "Q^T C Q partials", "Rayleigh-Ritz (merge, Jacobi, ordering)", "Ritz coefficient broadcast",
               "Ritz vectors", "Gram matrices")


def ritz_phase_clocks(reset: bool = True) -> dict:
    """Per-stage cycles of the fused eigensolver kernel since the last reset
    (instrumented build only: INFO_ESRF_PHASE_CLOCKS=1), averaged over launches."""
    out = (c_int64 * 11)()
    _check(library().info_esrf_ritz_phase_clocks(out, 11, 1 if reset else 0), "info_esrf_ritz_phase_clocks")
    v = list(out)
    n = max(v[10], 1)
    return {"cycles_per_launch": {name: v[i] / n for i, name in enumerate(RITZ_PHASES)}, "launches": v[10],
            "total_per_launch": sum(v[:10]) / n}


def wait_probe(limit_cycles: int, arrive: bool, status: torch.Tensor, stream=None) -> None:
    """One bounded mbarrier wait on the device (status: int32 CUDA tensor, one element)."""
    _need(status, torch.int32, "status")
    _check(library().info_esrf_wait_probe(int(limit_cycles), 1 if arrive else 0, status.data_ptr(), _stream(stream)),
           "info_esrf_wait_probe")


def fma_probe(precision: int, iters: int, stream=None):
    f, ms = c_double(), c_double()
    _check(library().info_esrf_fma_probe(precision, iters, ctypes.byref(f), ctypes.byref(ms), _stream(stream)),
           "info_esrf_fma_probe")
    return f.value, ms.value


def workspace(nbytes: int, device=None) -> torch.Tensor:
    """Device workspace (256-byte aligned; torch allocations are)."""
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device or "cuda")


def neighbor_counts(grid, obs_idx: torch.Tensor, stream=None):
    _need(obs_idx, torch.int64, "obs_idx")
    g = make_grid(grid)
    buf = torch.zeros(2, dtype=torch.int64, device=obs_idx.device)
    a, b = c_int64(), c_int64()
    _check(library().info_esrf_neighbor_counts(ctypes.byref(g), obs_idx.numel(), obs_idx.data_ptr(),
                                               buf.data_ptr(), _stream(stream), ctypes.byref(a),
                                               ctypes.byref(b)), "info_esrf_neighbor_counts")
    return int(a.value), int(b.value)


def workspace_size(grid, N: int, d: int, Q: int, options: Options) -> int:
    g = make_grid(grid)
    return int(library().info_esrf_workspace_size(ctypes.byref(g), N, d, Q, ctypes.byref(options)))


# ---------------------------------------------------------------------------
# Entry points with the C names
# ---------------------------------------------------------------------------

def info_esrf_analysis(grid, X: torch.Tensor, obs_idx: torch.Tensor, y: torch.Tensor, R: torch.Tensor,
                       Q: int, tol: float, options: Optional[Options] = None, ws: Optional[torch.Tensor] = None,
                       mu_a: Optional[torch.Tensor] = None, A_a: Optional[torch.Tensor] = None,
                       stats: bool = True, stream=None, allow_warning: bool = True):
    """Mean and perturbation update of one analysis.  Returns (mu_a, A_a, stats or None)."""
    for t, name, dt in ((X, "X", torch.float64), (obs_idx, "obs_idx", torch.int64),
                        (y, "y", torch.float64), (R, "R", torch.float64)):
        _need(t, dt, name)
    N, n = X.shape
    d = obs_idx.numel()
    o = options if options is not None else make_options()
    g = make_grid(grid)
    need = library().info_esrf_workspace_size(ctypes.byref(g), N, d, Q, ctypes.byref(o))
    if ws is None:
        ws = workspace(need, X.device)
    if mu_a is None:
        mu_a = torch.empty(n, dtype=torch.float64, device=X.device)
    if A_a is None:
        A_a = torch.empty((N, n), dtype=torch.float64, device=X.device)
    st = Stats()
    code = library().info_esrf_analysis(ctypes.byref(g), N, X.data_ptr(), d, obs_idx.data_ptr(), y.data_ptr(),
                                        R.data_ptr(), Q, tol, ctypes.byref(o), ws.data_ptr(), ws.numel(),
                                        _stream(stream), mu_a.data_ptr(), A_a.data_ptr(),
                                        ctypes.byref(st) if stats else None)
    _check(code, "info_esrf_analysis", allow_warning)
    return mu_a, A_a, (st.as_dict() if stats else None)


def info_esrf_mean_update(grid, X, obs_idx, y, R, tol, options=None, ws=None, mu_a=None, stats=True,
                          stream=None):
    for t, name, dt in ((X, "X", torch.float64), (obs_idx, "obs_idx", torch.int64),
                        (y, "y", torch.float64), (R, "R", torch.float64)):
        _need(t, dt, name)
    N, n = X.shape
    d = obs_idx.numel()
    o = options if options is not None else make_options()
    g = make_grid(grid)
    if ws is None:
        ws = workspace(library().info_esrf_workspace_size(ctypes.byref(g), N, d, 1, ctypes.byref(o)), X.device)
    if mu_a is None:
        mu_a = torch.empty(n, dtype=torch.float64, device=X.device)
    st = Stats()
    code = library().info_esrf_mean_update(ctypes.byref(g), N, X.data_ptr(), d, obs_idx.data_ptr(), y.data_ptr(),
                                           R.data_ptr(), tol, ctypes.byref(o), ws.data_ptr(), ws.numel(),
                                           _stream(stream), mu_a.data_ptr(), ctypes.byref(st) if stats else None)
    _check(code, "info_esrf_mean_update")
    return mu_a, (st.as_dict() if stats else None)


def info_esrf_perturbation_update(grid, X, obs_idx, R, Q, tol, options=None, ws=None, A_a=None, stats=True,
                                  stream=None):
    for t, name, dt in ((X, "X", torch.float64), (obs_idx, "obs_idx", torch.int64), (R, "R", torch.float64)):
        _need(t, dt, name)
    N, n = X.shape
    d = obs_idx.numel()
    o = options if options is not None else make_options()
    g = make_grid(grid)
    if ws is None:
        ws = workspace(library().info_esrf_workspace_size(ctypes.byref(g), N, d, Q, ctypes.byref(o)), X.device)
    if A_a is None:
        A_a = torch.empty((N, n), dtype=torch.float64, device=X.device)
    st = Stats()
    code = library().info_esrf_perturbation_update(ctypes.byref(g), N, X.data_ptr(), d, obs_idx.data_ptr(),
                                                   R.data_ptr(), Q, tol, ctypes.byref(o), ws.data_ptr(),
                                                   ws.numel(), _stream(stream), A_a.data_ptr(),
                                                   ctypes.byref(st) if stats else None)
    _check(code, "info_esrf_perturbation_update")
    return A_a, (st.as_dict() if stats else None)


def _fill_problem(c: "ProblemC", p: dict, X: torch.Tensor, mu_a: torch.Tensor, A_a: torch.Tensor) -> None:
    """One problem of a batched call.  Observations are either indices (``obs_idx``)
    or a general linear operator ``H`` = (rowptr int64 [d + 1], col int64 [nnz],
    val float64 [nnz]), device tensors in CSR form."""
    N = X.shape[0]
    c.grid = make_grid(p["grid"])
    H = p.get("H")
    if H is not None:
        rowptr, col, val = H
        _need(rowptr, torch.int64, "H rowptr")
        _need(col, torch.int64, "H col")
        _need(val, torch.float64, "H val")
        d = rowptr.numel() - 1
        c.H_rowptr, c.H_col, c.H_val, c.H_nnz = rowptr.data_ptr(), col.data_ptr(), val.data_ptr(), col.numel()
        c.obs_idx = None
    else:
        d = p["obs_idx"].numel()
        c.obs_idx = p["obs_idx"].data_ptr()
        c.H_rowptr, c.H_col, c.H_val, c.H_nnz = None, None, None, 0
    c.N, c.d, c.Q, c.tol = N, d, int(p["Q"]), float(p["tol"])
    c.X, c.y, c.R_diag = X.data_ptr(), p["y"].data_ptr(), p["R"].data_ptr()
    c.mu_a, c.A_a = mu_a.data_ptr(), A_a.data_ptr()
    c.max_oo, c.max_xo = int(p.get("max_oo", 0)), int(p.get("max_xo", 0))


def info_esrf_analysis_batched(problems: Sequence[dict], options: Optional[Options] = None,
                               ws: Optional[torch.Tensor] = None, stats: bool = True, stream=None):
    """problems: dicts with grid, X, obs_idx (or H, see _fill_problem), y, R, Q, tol and optional
    mu_a, A_a, max_oo, max_xo."""
    arr = (ProblemC * len(problems))()
    keep = []
    for i, p in enumerate(problems):
        X = p["X"]
        _need(X, torch.float64, "X")
        N, n = X.shape
        mu_a = p.get("mu_a")
        A_a = p.get("A_a")
        if mu_a is None:
            mu_a = torch.empty(n, dtype=torch.float64, device=X.device)
        if A_a is None:
            A_a = torch.empty((N, n), dtype=torch.float64, device=X.device)
        keep.append((mu_a, A_a))
        _fill_problem(arr[i], p, X, mu_a, A_a)
    o = options if options is not None else make_options()
    need = library().info_esrf_batched_workspace_size(arr, len(problems), ctypes.byref(o))
    if need == 0:
        raise InfoEsrfError(ERR_INVALID_ARG, "info_esrf_batched_workspace_size")
    if ws is None or ws.numel() < need:
        ws = workspace(need)
    st = (Stats * len(problems))()
    code = library().info_esrf_analysis_batched(arr, len(problems), ctypes.byref(o), ws.data_ptr(), ws.numel(),
                                                _stream(stream), st if stats else None)
    _check(code, "info_esrf_analysis_batched")
    return keep, ([s.as_dict() for s in st] if stats else None)


def autotune(problems: Sequence[dict], options: Options, ws: Optional[torch.Tensor] = None, stream=None):
    """Times the candidate settings on these problems (overwriting their outputs) and writes the fastest
    cluster_size, power_iters and oversample into `options`.  Returns the best time per call (ms)."""
    arr = (ProblemC * len(problems))()
    keep = []
    for i, p in enumerate(problems):
        X = p["X"]
        _need(X, torch.float64, "X")
        N, n = X.shape
        mu_a = p.get("mu_a")
        A_a = p.get("A_a")
        if mu_a is None:
            mu_a = torch.empty(n, dtype=torch.float64, device=X.device)
        if A_a is None:
            A_a = torch.empty((N, n), dtype=torch.float64, device=X.device)
        keep.append((mu_a, A_a))
        _fill_problem(arr[i], p, X, mu_a, A_a)
    need = library().info_esrf_batched_workspace_size(arr, len(problems), ctypes.byref(options))
    if ws is None or ws.numel() < need:
        ws = workspace(need)
    best = c_double(0.0)
    _check(library().info_esrf_autotune(arr, len(problems), ctypes.byref(options), ws.data_ptr(), ws.numel(),
                                        _stream(stream), ctypes.byref(best)), "info_esrf_autotune")
    return best.value


def info_esrf_bf16_tile_matvec(rowptr: torch.Tensor, colblk: torch.Tensor, C_hi: torch.Tensor, C_lo: torch.Tensor,
                               P: torch.Tensor, sigma: torch.Tensor, want_pty: bool = True, stream=None):
    """Y = sigma P + (C_hi + C_lo) P for the block-sparse BF16 C (tensor-core stage entry).
    rowptr int32 [nrt + 1], colblk int32 [tiles], C_hi / C_lo bfloat16 [tiles][128][64],
    P bfloat16 [J][128 nrt], sigma float32 [J].  Returns (Y float32 [J][d_pad], pty float32 [nrt][J], status)."""
    _need(rowptr, torch.int32, "rowptr")
    _need(colblk, torch.int32, "colblk")
    for t, name in ((C_hi, "C_hi"), (C_lo, "C_lo"), (P, "P")):
        _need(t, torch.bfloat16, name)
    _need(sigma, torch.float32, "sigma")
    nrt = rowptr.numel() - 1
    J, d_pad = P.shape
    Y = torch.empty((J, d_pad), dtype=torch.float32, device=P.device)
    pty = torch.empty((nrt, J), dtype=torch.float32, device=P.device) if want_pty else None
    status = torch.zeros(1, dtype=torch.int32, device=P.device)
    _check(library().info_esrf_bf16_tile_matvec(nrt, rowptr.data_ptr(), colblk.data_ptr(), colblk.numel(),
                                                C_hi.data_ptr(), C_lo.data_ptr(), J, P.data_ptr(), sigma.data_ptr(),
                                                Y.data_ptr(), pty.data_ptr() if want_pty else None,
                                                status.data_ptr(), _stream(stream)), "info_esrf_bf16_tile_matvec")
    return Y, pty, status


def info_esrf_philox_normals(seed: int, count: int, device="cuda", stream=None) -> torch.Tensor:
    out = torch.empty(max(count, 1), dtype=torch.float64, device=device)
    _check(library().info_esrf_philox_normals(seed, count, out.data_ptr(), _stream(stream)),
           "info_esrf_philox_normals")
    return out[:count]


def info_esrf_quadrature_nodes(Q: int, ell: float, rule: int = RULE_ELLIPTIC, device="cuda", stream=None):
    s = torch.empty(Q, dtype=torch.float64, device=device)
    p = torch.empty(Q, dtype=torch.float64, device=device)
    _check(library().info_esrf_quadrature_nodes(Q, ell, rule, s.data_ptr(), p.data_ptr(), _stream(stream)),
           "info_esrf_quadrature_nodes")
    return s, p


# ---------------------------------------------------------------------------
# Learned preconditioner correction
# ---------------------------------------------------------------------------

def learn_nparams() -> int:
    return int(library().info_esrf_learn_nparams())


def krylov_capture(grid, X, obs_idx, R, Q, sel, K, options: Optional[Options] = None, stream=None):
    """Krylov samples (V, Y, Z, feat) of the method's own PCG for systems `sel`."""
    o = options if options is not None else make_options(precision=PRECISION_FP32)
    g = make_grid(grid)
    N, n = X.shape
    d = obs_idx.numel()
    need = library().info_esrf_workspace_size(ctypes.byref(g), N, d, Q, ctypes.byref(o))
    ws = workspace(need, X.device)
    sel_t = torch.as_tensor(sel, dtype=torch.int32, device=X.device)
    S = sel_t.numel() * K
    V = torch.empty((S, d), dtype=torch.float32, device=X.device)
    Y = torch.empty_like(V)
    Z = torch.empty_like(V)
    feat = torch.empty((S, 4), dtype=torch.float32, device=X.device)
    _check(library().info_esrf_krylov_capture(ctypes.byref(g), N, X.data_ptr(), d, obs_idx.data_ptr(), R.data_ptr(),
                                              Q, ctypes.byref(o), ws.data_ptr(), ws.numel(), sel_t.numel(),
                                              sel_t.data_ptr(), K, V.data_ptr(), Y.data_ptr(), Z.data_ptr(),
                                              feat.data_ptr(), _stream(stream)), "info_esrf_krylov_capture")
    return V, Y, Z, feat


def krylov_capture_lattice(grid, X, obs_idx, R, Q, sel, K, options: Optional[Options] = None, stream=None):
    """Krylov samples (V, Y, Z, feat) of the BF16 path in lattice order, and the lattice shape (Lx, Ly)."""
    o = options if options is not None else make_options(precision=PRECISION_BF16)
    g = make_grid(grid)
    N, n = X.shape
    d = obs_idx.numel()
    need = library().info_esrf_workspace_size(ctypes.byref(g), N, d, Q, ctypes.byref(o))
    ws = workspace(need, X.device)
    sel_t = torch.as_tensor(sel, dtype=torch.int32, device=X.device)
    S = sel_t.numel() * K
    V = torch.empty((S, d), dtype=torch.float32, device=X.device)
    Y = torch.empty_like(V)
    Z = torch.empty_like(V)
    feat = torch.empty((S, 4), dtype=torch.float32, device=X.device)
    lx, ly = c_int32(), c_int32()
    _check(library().info_esrf_krylov_capture_lattice(
        ctypes.byref(g), N, X.data_ptr(), d, obs_idx.data_ptr(), R.data_ptr(), Q, ctypes.byref(o), ws.data_ptr(),
        ws.numel(), sel_t.numel(), sel_t.data_ptr(), K, V.data_ptr(), Y.data_ptr(), Z.data_ptr(), feat.data_ptr(),
        ctypes.byref(lx), ctypes.byref(ly), _stream(stream)), "info_esrf_krylov_capture_lattice")
    return V, Y, Z, feat, int(lx.value), int(ly.value)


def learn_loss_grad_lattice(theta, feat, V, Y, Z, Lx, Ly, stream=None):
    S, d = V.shape
    scratch = workspace(library().info_esrf_learn_lattice_scratch_size(S, d), V.device)
    grad = torch.empty_like(theta)
    loss = torch.zeros(1, dtype=torch.float64, device=V.device)
    _check(library().info_esrf_learn_loss_grad_lattice(theta.data_ptr(), S, Lx, Ly, feat.data_ptr(), V.data_ptr(),
                                                       Y.data_ptr(), Z.data_ptr(), grad.data_ptr(), loss.data_ptr(),
                                                       scratch.data_ptr(), scratch.numel(), _stream(stream)),
           "info_esrf_learn_loss_grad_lattice")
    return float(loss.item()), grad


def learn_train_lattice(theta, feat, V, Y, Z, Lx, Ly, steps, lr=1e-2, state=None, stream=None):
    """Adam training of the lattice form in place on theta.  Returns (loss history, state)."""
    S, d = V.shape
    if state is None:
        state = dict(m=torch.zeros_like(theta), v=torch.zeros_like(theta), step=1)
    scratch = workspace(library().info_esrf_learn_lattice_scratch_size(S, d), V.device)
    grad = torch.empty_like(theta)
    hist = torch.zeros(steps, dtype=torch.float64, device=V.device)
    _check(library().info_esrf_learn_train_lattice(theta.data_ptr(), state["m"].data_ptr(), state["v"].data_ptr(),
                                                   state["step"], steps, lr, S, Lx, Ly, feat.data_ptr(),
                                                   V.data_ptr(), Y.data_ptr(), Z.data_ptr(), grad.data_ptr(),
                                                   hist.data_ptr(), scratch.data_ptr(), scratch.numel(),
                                                   _stream(stream)), "info_esrf_learn_train_lattice")
    state["step"] += steps
    return hist, state


def learn_loss_grad(theta, feat, V, Y, Z, stream=None):
    S, d = V.shape
    scratch = workspace(library().info_esrf_learn_scratch_size(S), V.device)
    grad = torch.empty_like(theta)
    loss = torch.zeros(1, dtype=torch.float64, device=V.device)
    _check(library().info_esrf_learn_loss_grad(theta.data_ptr(), S, d, feat.data_ptr(), V.data_ptr(), Y.data_ptr(),
                                               Z.data_ptr(), grad.data_ptr(), loss.data_ptr(), scratch.data_ptr(),
                                               scratch.numel(), _stream(stream)), "info_esrf_learn_loss_grad")
    return float(loss.item()), grad


def learn_train(theta, feat, V, Y, Z, steps, lr=1e-2, state=None, stream=None):
    """Adam training in place on theta (device float).  Returns (loss history, state)."""
    S, d = V.shape
    if state is None:
        state = dict(m=torch.zeros_like(theta), v=torch.zeros_like(theta), step=1)
    scratch = workspace(library().info_esrf_learn_scratch_size(S), V.device)
    grad = torch.empty_like(theta)
    hist = torch.zeros(steps, dtype=torch.float64, device=V.device)
    _check(library().info_esrf_learn_train(theta.data_ptr(), state["m"].data_ptr(), state["v"].data_ptr(),
                                           state["step"], steps, lr, S, d, feat.data_ptr(), V.data_ptr(),
                                           Y.data_ptr(), Z.data_ptr(), grad.data_ptr(), hist.data_ptr(),
                                           scratch.data_ptr(), scratch.numel(), _stream(stream)),
           "info_esrf_learn_train")
    state["step"] += steps
    return hist, state


def learn_coefficients(theta, feat, stream=None):
    nshift = feat.shape[0]
    coef = torch.empty((nshift, 2 * int(library().info_esrf_learn_halfwidth()) + 2), dtype=torch.float32,
                       device=feat.device)
    _check(library().info_esrf_learn_coefficients(theta.data_ptr(), nshift, feat.data_ptr(), coef.data_ptr(),
                                                  _stream(stream)), "info_esrf_learn_coefficients")
    return coef


def model_save(path: str, theta_host, max_shift: float = 0.0) -> None:
    import numpy as np
    arr = np.ascontiguousarray(np.asarray(theta_host, dtype=np.float32))
    _check(library().info_esrf_model_save(path.encode(), arr.ctypes.data, float(max_shift)),
           "info_esrf_model_save")


def model_load(path: str):
    """Returns (parameters as a float32 NumPy array, shift cut-off)."""
    import numpy as np
    arr = np.zeros(learn_nparams(), dtype=np.float32)
    ms = c_double()
    _check(library().info_esrf_model_load(path.encode(), arr.ctypes.data, ctypes.byref(ms)), "info_esrf_model_load")
    return arr, float(ms.value)


class Prepared:
    """A workspace on which info_esrf_prepare ran, with its stage-level calls."""

    def __init__(self, grid, X, obs_idx, R, Q, options: Optional[Options] = None, stream=None):
        _need(X, torch.float64, "X")
        _need(obs_idx, torch.int64, "obs_idx")
        _need(R, torch.float64, "R")
        self.g = make_grid(grid)
        self.N, self.n = X.shape
        self.d = obs_idx.numel()
        self.Q = Q
        self.o = options if options is not None else make_options()
        self.precision = self.o.precision
        lib = library()
        need = lib.info_esrf_workspace_size(ctypes.byref(self.g), self.N, self.d, Q, ctypes.byref(self.o))
        self.ws = workspace(need, X.device)
        self.stream = stream
        _check(lib.info_esrf_prepare(ctypes.byref(self.g), self.N, X.data_ptr(), self.d, obs_idx.data_ptr(),
                                     R.data_ptr(), Q, ctypes.byref(self.o), self.ws.data_ptr(), self.ws.numel(),
                                     _stream(stream)), "info_esrf_prepare")

    def _args(self):
        return (ctypes.byref(self.g), self.N, self.d, self.Q, ctypes.byref(self.o), self.ws.data_ptr(),
                self.ws.numel())

    def obs_matvec(self, P: torch.Tensor, sigma: torch.Tensor) -> torch.Tensor:
        _need(P, torch.float64, "P")
        _need(sigma, torch.float64, "sigma")
        Y = torch.empty_like(P)
        _check(library().info_esrf_prepared_obs_matvec(*self._args(), P.shape[0], P.data_ptr(), sigma.data_ptr(),
                                                       Y.data_ptr(), _stream(self.stream)),
               "info_esrf_prepared_obs_matvec")
        return Y

    def lmp_apply(self, Rv: torch.Tensor, sigma: torch.Tensor) -> torch.Tensor:
        _need(Rv, torch.float64, "R")
        _need(sigma, torch.float64, "sigma")
        Z = torch.empty_like(Rv)
        _check(library().info_esrf_prepared_lmp_apply(*self._args(), Rv.shape[0], Rv.data_ptr(), sigma.data_ptr(),
                                                      Z.data_ptr(), _stream(self.stream)),
               "info_esrf_prepared_lmp_apply")
        return Z

    def capacity(self):
        a, b = c_int64(), c_int64()
        _check(library().info_esrf_prepared_band_capacity(ctypes.byref(self.g), self.N, self.d, self.Q,
                                                          ctypes.byref(self.o), ctypes.byref(a), ctypes.byref(b)),
               "info_esrf_prepared_band_capacity")
        return int(a.value), int(b.value)

    def export(self, item: str):
        """Copies one prepared array to a host torch tensor."""
        import numpy as np
        esz = 8 if self.precision == 0 else 4
        fdt = np.float64 if esz == 8 else np.float32
        mo, mx = self.capacity()
        kR = min(self.o.ritz_rank, self.d)
        shapes = dict(scalars=(8, np.float64), status=(4, np.int32), quad_s=(self.Q, np.float64),
                      quad_p=(self.Q, np.float64), theta=(kR, np.float64), phi=(self.d * kR, fdt),
                      cphi=(self.d * kR, fdt), oo_val=(mo * self.d, fdt), oo_col=(mo * self.d, np.int32),
                      oo_nnz=(self.d, np.int32), xo_val=(mx * self.n, fdt), xo_col=(mx * self.n, np.int32),
                      xo_nnz=(self.n, np.int32), W=(self.d * self.N, fdt), mu=(self.n, np.float64))
        count, dt = shapes[item]
        out = np.zeros(max(count, 1), dtype=dt)
        _check(library().info_esrf_prepared_export(*self._args(), ITEM[item], out.ctypes.data, out.nbytes,
                                                   _stream(self.stream)), "info_esrf_prepared_export")
        return out[:count]
