"""The allocation-free analysis entry point agrees with the regular one.

Callers that cannot allocate device memory use info_esrf_analysis_noalloc,
whose workspace is a fixed array inside the library.  This test calls it
through the C ABI twice in a row (the second call reuses the array the first
one left behind) and compares both results with info_esrf_analysis run on a
workspace allocated by the caller, at the FP64 parity tolerance of the other
tests.  It also checks that a problem too large for the fixed array is
rejected.  The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest
import torch

from parity_checks import increment_error, mean_error
from oracle import filter as F
from paper_2503_00253_gb300 import workloads

pytestmark = pytest.mark.gpu


def _noalloc_fn(B):
    fn = B.library().info_esrf_analysis_noalloc
    P = ctypes.POINTER
    fn.restype = ctypes.c_int32
    fn.argtypes = [P(B.Grid), ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_void_p, ctypes.c_int32, ctypes.c_double, P(B.Options), ctypes.c_void_p,
                   ctypes.c_void_p, ctypes.c_void_p]
    return fn


def test_noalloc_matches_regular_entry_point_twice():
    from paper_2503_00253_gb300 import binding as B
    fn = _noalloc_fn(B)
    runs = [(workloads.config1(), 0, 1e-12), (workloads.gaussian_problem_1d(
        "na", n=700, N=13, length_scale=5.0, obs_stride=3, r2=0.4, half_width=8.0, Q=6, tol=1e-12, seed=21), 0, 1e-12)]
    for pr, prec, tol in runs:
        X, obs, y, R = (torch.tensor(a, device="cuda") for a in (pr.X, pr.obs_idx, pr.y, pr.R))
        opts = B.make_options(precision=prec)
        mu_ref, A_ref, st = B.info_esrf_analysis(pr.grid, X, obs, y, R, pr.Q, tol, opts)
        torch.cuda.synchronize()
        assert st["status"] == 0
        g = B.make_grid(pr.grid)
        Af = pr.X - pr.X.mean(0)
        for call in range(2):
            mu_a = torch.full_like(mu_ref, float("nan"))
            A_a = torch.full_like(A_ref, float("nan"))
            rc = fn(ctypes.byref(g), pr.N, X.data_ptr(), pr.d, obs.data_ptr(), y.data_ptr(), R.data_ptr(), pr.Q,
                    tol, ctypes.byref(opts), torch.cuda.current_stream().cuda_stream, mu_a.data_ptr(),
                    A_a.data_ptr())
            torch.cuda.synchronize()
            assert rc == 0, (call, rc)
            err_A = increment_error(A_a.cpu().numpy(), A_ref.cpu().numpy(), Af)
            mu0 = pr.X.mean(0)
            err_mu = mean_error(mu_a, mu_ref, mu0)
            assert err_A <= 1e-10 and err_mu <= 1e-10, (call, err_A, err_mu)


def _call(fn, B, pr, X, obs, y, R, tol, opts, mu_a, A_a):
    g = B.make_grid(pr.grid)
    return fn(ctypes.byref(g), pr.N, X.data_ptr(), pr.d, obs.data_ptr(), y.data_ptr(), R.data_ptr(), pr.Q, tol,
              ctypes.byref(opts), torch.cuda.current_stream().cuda_stream, mu_a.data_ptr(), A_a.data_ptr())


@pytest.mark.parametrize("solver,precision,tol,bound", [(1, 0, 1e-12, 1e-10), (1, 1, 1e-6, 1e-4),
                                                         (0, 1, 1e-6, 1e-4)])
def test_noalloc_other_solvers_and_precisions_after_a_pcg_call(solver, precision, tol, bound):
    """The array keeps whatever the previous call left (here an FP64 PCG analysis of another problem):
    multi-shift CG (solver 1) and the FP32 paths carve it differently, and two calls in a row must
    still agree with the regular entry point on a caller-allocated workspace, at the FP64 (1e-10) or
    FP32 (1e-4) parity tolerance.  The FP32 PCG case runs the cluster-resident band kernel."""
    from paper_2503_00253_gb300 import binding as B
    fn = _noalloc_fn(B)
    first = workloads.config1()
    X1, obs1, y1, R1 = (torch.tensor(a, device="cuda") for a in (first.X, first.obs_idx, first.y, first.R))
    m1 = torch.empty(first.n, dtype=torch.float64, device="cuda")
    a1 = torch.empty((first.N, first.n), dtype=torch.float64, device="cuda")
    assert _call(fn, B, first, X1, obs1, y1, R1, 1e-12, B.make_options(precision=0), m1, a1) == 0
    pr = workloads.gaussian_problem_1d("na2", n=2048, N=10, length_scale=16.0, obs_stride=4, r2=0.3,
                                       half_width=24.0, Q=12, tol=tol, seed=22)
    X, obs, y, R = (torch.tensor(a, device="cuda") for a in (pr.X, pr.obs_idx, pr.y, pr.R))
    max_oo, max_xo = B.neighbor_counts(pr.grid, obs)
    opts = B.make_options(precision=precision, solver=solver, max_neighbors=max(max_oo, max_xo))
    mu_ref, A_ref, st = B.info_esrf_analysis(pr.grid, X, obs, y, R, pr.Q, tol, opts)
    torch.cuda.synchronize()
    assert st["status"] == 0 and st["solver_path"] == (2 if solver == 1 else 1), st
    Af = pr.X - pr.X.mean(0)
    for call in range(2):
        mu_a = torch.full_like(mu_ref, float("nan"))
        A_a = torch.full_like(A_ref, float("nan"))
        rc = _call(fn, B, pr, X, obs, y, R, tol, opts, mu_a, A_a)
        torch.cuda.synchronize()
        assert rc == 0, (call, rc)
        err_A = increment_error(A_a.cpu().numpy(), A_ref.cpu().numpy(), Af)
        err_mu = mean_error(mu_a, mu_ref, pr.X.mean(0))
        assert err_A <= bound and err_mu <= bound, (call, err_A, err_mu)


def test_noalloc_returns_the_regular_entry_points_error_codes():
    """Invalid or unsupported arguments give the same code as info_esrf_analysis."""
    from paper_2503_00253_gb300 import binding as B
    fn = _noalloc_fn(B)
    pr = workloads.config1()
    X, obs, y, R = (torch.tensor(a, device="cuda") for a in (pr.X, pr.obs_idx, pr.y, pr.R))
    mu_a = torch.empty(pr.n, dtype=torch.float64, device="cuda")
    A_a = torch.empty((pr.N, pr.n), dtype=torch.float64, device="cuda")
    for opts, code in ((B.make_options(ritz_rank=40), B.ERR_UNSUPPORTED),
                       (B.make_options(precision=7), B.ERR_INVALID_ARG),
                       (B.make_options(cluster_size=3), B.ERR_INVALID_ARG)):
        assert _call(fn, B, pr, X, obs, y, R, 1e-12, opts, mu_a, A_a) == code
        with pytest.raises(B.InfoEsrfError) as e:
            B.info_esrf_analysis(pr.grid, X, obs, y, R, pr.Q, 1e-12, opts)
        assert e.value.code == code


def test_noalloc_rejects_problems_beyond_its_array():
    from paper_2503_00253_gb300 import binding as B
    fn = _noalloc_fn(B)
    pr = workloads.config2()
    X, obs, y, R = (torch.tensor(a, device="cuda") for a in (pr.X, pr.obs_idx, pr.y, pr.R))
    opts = B.make_options(precision=0)          # geometric band bound: far above 32 MiB
    g = B.make_grid(pr.grid)
    assert B.library().info_esrf_workspace_size(ctypes.byref(g), pr.N, pr.d, pr.Q, ctypes.byref(opts)) > 32 << 20
    mu_a = torch.empty(pr.n, dtype=torch.float64, device="cuda")
    A_a = torch.empty((pr.N, pr.n), dtype=torch.float64, device="cuda")
    rc = fn(ctypes.byref(g), pr.N, X.data_ptr(), pr.d, obs.data_ptr(), y.data_ptr(), R.data_ptr(), pr.Q, 1e-8,
            ctypes.byref(opts), torch.cuda.current_stream().cuda_stream, mu_a.data_ptr(), A_a.data_ptr())
    assert rc == B.ERR_UNSUPPORTED
