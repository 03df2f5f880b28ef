"""GPU parity of the multi-shift CG solver (Sec. 3.3, shift invariance of Krylov
subspaces) against the FP64 oracle, through the C ABI.

The multi-shift path solves the same shifted systems as the PCG path, so its
results are held to the same bounds against the same-node exact result:
FP64 <= 1e-10 (tolerance 1e-12), FP32 <= 1e-4 (tolerance 1e-6), as
||A_gpu - A_ref||_F / ||A_ref - A_f||_F and the same for the mean.  In
fixed-iteration mode it is compared with the oracle's own multi-shift run.
"""
import ctypes
import math

import numpy as np
import pytest
import torch

from parity_checks import increment_error, mean_error
from oracle import filter as F
from oracle import pcg, quadrature
from paper_2503_00253_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2503_00253_gb300 import binding
    binding.library()
    return binding


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda")


def ms_opts(B, precision, **kw):
    return B.make_options(precision=precision, solver=B.SOLVER_MULTISHIFT, **kw)


def run(B, pr, precision, tol, **kw):
    mu_a, A_a, st = B.info_esrf_analysis(pr.grid, dev(pr.X), dev(pr.obs_idx), dev(pr.y), dev(pr.R), pr.Q, tol,
                                         ms_opts(B, precision, **kw))
    torch.cuda.synchronize()
    return mu_a.cpu().numpy(), A_a.cpu().numpy(), st


def errors(pr, mu_a, A_a):
    A_ref = F.perturbation_update(pr.X, pr.obs_idx, pr.R, pr.grid, pr.Q)
    mu_ref = F.mean_update(pr.X, pr.obs_idx, pr.y, pr.R, pr.grid)
    ea = increment_error(A_a, A_ref, pr.X - pr.X.mean(0))
    em = mean_error(mu_a, mu_ref, pr.X.mean(0))
    return ea, em


def test_multishift_config1_fp64(B):
    pr = workloads.config1()
    mu_a, A_a, st = run(B, pr, 0, 1e-12)
    assert st["status"] == 0 and st["solver_path"] == 2, st
    assert st["n_systems"] == pr.Q * pr.N + 1 and st["n_unconverged"] == 0
    ea, em = errors(pr, mu_a, A_a)
    assert ea <= 1e-10 and em <= 1e-10, (ea, em)


def test_multishift_config2_fp64_and_fp32(B):
    """n = 8192, N = 40, d = 1024, Q = 32: 41 chains in clusters of 8 CTAs."""
    pr = workloads.config2()
    A_ref = F.perturbation_update(pr.X, pr.obs_idx, pr.R, pr.grid, pr.Q)
    mu_ref = F.mean_update(pr.X, pr.obs_idx, pr.y, pr.R, pr.grid)
    for precision, tol, bound in ((0, 1e-12, 1e-10), (1, 1e-6, 1e-4)):
        mu_a, A_a, st = run(B, pr, precision, tol)
        ea = increment_error(A_a, A_ref, pr.X - pr.X.mean(0))
        em = mean_error(mu_a, mu_ref, pr.X.mean(0))
        assert st["status"] == 0 and st["solver_path"] == 2, st
        assert ea <= bound and em <= bound, (precision, ea, em)


SMALL = [
    ("1d", lambda: workloads.gaussian_problem_1d("s", n=300, N=11, length_scale=6.0, obs_stride=3, r2=0.4,
                                                 half_width=9.0, Q=5, tol=1e-12, seed=1, obs_offset=1)),
    ("layered", lambda: workloads.random_obs_problem(workloads.Grid((40, 1, 6), (True, False, False),
                                                                    (5.0, 1.0, 1.5)), N=10, d=70, r2=0.8,
                                                     Q=6, tol=1e-12, seed=3)),
    ("2d", lambda: workloads.random_obs_problem(workloads.Grid((24, 20, 1), (True, True, False),
                                                               (3.0, 2.5, 1.0)), N=7, d=90, r2=0.5, Q=5,
                                                tol=1e-12, seed=4)),
]


@pytest.mark.parametrize("name,make", SMALL)
@pytest.mark.parametrize("precision,tol,bound", [(0, 1e-12, 1e-10), (1, 1e-6, 1e-4)])
def test_multishift_small_grids(B, name, make, precision, tol, bound):
    pr = make()
    mu_a, A_a, st = run(B, pr, precision, tol)
    assert st["status"] == 0 and st["solver_path"] == 2, st
    ea, em = errors(pr, mu_a, A_a)
    assert ea <= bound and em <= bound, (name, ea, em)


@pytest.mark.parametrize("iters", [2, 10])
def test_multishift_fixed_iterations_match_oracle(B, iters):
    """Exactly k iterations of the run (the paper's experiments use 2 and 10):
    the same shifted iterates as the oracle's multi-shift CG."""
    pr = workloads.gaussian_problem_1d("fixms", n=600, N=8, length_scale=6.0, obs_stride=2, r2=0.4,
                                       half_width=10.0, Q=5, tol=1e-12, seed=11)
    mu, Z = F.anomalies(pr.X)
    W, Sxh, Shh = F.localized_covariances(Z, pr.obs_idx, pr.grid)
    C = F.normalized_obs_covariance(Shh, pr.R)
    s, p = quadrature.elliptic_rule(pr.Q, F.choose_ell(Shh, pr.R))
    vbar, it = pcg.solve_normalized_multishift(C, s, p, W, pr.R, fixed_iters=iters)
    A_ref = math.sqrt(pr.N - 1) * (Z - Sxh @ vbar).T
    sys_it = torch.zeros(pr.Q * pr.N, dtype=torch.int32, device="cuda")
    A_a, st = B.info_esrf_perturbation_update(pr.grid, dev(pr.X), dev(pr.obs_idx), dev(pr.R), pr.Q, 1e-12,
                                              ms_opts(B, 0, fixed_iters=iters, system_iters=sys_it))
    torch.cuda.synchronize()
    err = increment_error(A_a.cpu().numpy(), A_ref, pr.X - pr.X.mean(0))
    assert err < 1e-9, (iters, err)
    assert st["iters_max"] == iters
    # system q * N + i carries shift q of member i
    assert np.array_equal(sys_it.cpu().numpy().reshape(pr.Q, pr.N), it)


@pytest.mark.parametrize("cluster_size,precision,Q", [(2, 0, 48), (4, 1, 32), (8, 1, 48)])
def test_multishift_cluster_sizes_and_scratch_directions(B, cluster_size, precision, Q):
    """Explicit cluster sizes; at 2 CTAs per cluster in FP64 with 48 shifts the
    shifted directions (48 x 512 rows x 8 B per chain) exceed shared memory and
    live in the CTA's scratch slice instead."""
    pr = workloads.gaussian_problem_1d("cs", n=8192, N=12, length_scale=64.0, obs_stride=8, r2=0.25,
                                       half_width=256.0, Q=Q, tol=1e-12, seed=21)
    tol, bound = (1e-12, 1e-10) if precision == 0 else (1e-6, 1e-4)
    mu_a, A_a, st = run(B, pr, precision, tol, cluster_size=cluster_size)
    assert st["status"] == 0 and st["solver_path"] == 2, st
    ea, em = errors(pr, mu_a, A_a)
    assert ea <= bound and em <= bound, (cluster_size, ea, em)


def test_multishift_batched_uneven(B):
    probs = workloads.uneven_batch(count=5, seed=12, tol=1e-12, n_min=200, n_max=1500)
    dicts = [dict(grid=p.grid, X=dev(p.X), obs_idx=dev(p.obs_idx), y=dev(p.y), R=dev(p.R), Q=p.Q, tol=1e-12)
             for p in probs]
    outs, stats = B.info_esrf_analysis_batched(dicts, ms_opts(B, 0))
    torch.cuda.synchronize()
    for p, (mu_a, A_a), st in zip(probs, outs, stats):
        assert st["status"] == 0 and st["solver_path"] == 2 and st["n_systems"] == p.Q * p.N + 1, st
        ea, em = errors(p, mu_a.cpu().numpy(), A_a.cpu().numpy())
        assert ea <= 1e-10 and em <= 1e-10, (p.name, ea, em)


def test_multishift_mean_and_perturbation_calls_alone(B):
    pr = workloads.gaussian_problem_1d("sepms", n=500, N=12, length_scale=5.0, obs_stride=4, r2=0.5,
                                       half_width=8.0, Q=6, tol=1e-12, seed=10)
    X, obs, y, R = dev(pr.X), dev(pr.obs_idx), dev(pr.y), dev(pr.R)
    mu_a, st = B.info_esrf_mean_update(pr.grid, X, obs, y, R, 1e-12, ms_opts(B, 0))
    A_a, st2 = B.info_esrf_perturbation_update(pr.grid, X, obs, R, pr.Q, 1e-12, ms_opts(B, 0))
    torch.cuda.synchronize()
    ea, em = errors(pr, mu_a.cpu().numpy(), A_a.cpu().numpy())
    assert st["n_systems"] == 1 and st2["n_systems"] == pr.Q * pr.N
    assert st["solver_path"] == 2 and st2["solver_path"] == 2
    assert ea <= 1e-10 and em <= 1e-10, (ea, em)


@pytest.mark.parametrize("precision,tol,bound", [(0, 1e-12, 1e-10), (1, 1e-6, 1e-4)])
def test_multishift_general_observation_operator(B, precision, tol, bound):
    """Weighted-sum observations (dense C): 100 Gaussian channels on a circle of 2000 points."""
    pr = workloads.gaussian_problem_1d("chanms", n=2000, N=20, length_scale=10.0, obs_stride=20, r2=0.5,
                                       half_width=20.0, Q=16, tol=tol, seed=91)
    Hd, (rowptr, col, val) = workloads.gaussian_channel_operator(pr.n, 100, 10.0)
    R = np.full(100, 0.5)
    y = Hd @ pr.truth + np.sqrt(R) * np.random.default_rng(92).standard_normal(100)
    d = dict(grid=pr.grid, X=dev(pr.X), H=(dev(rowptr), dev(col), dev(val)), y=dev(y), R=dev(R), Q=pr.Q, tol=tol)
    outs, stats = B.info_esrf_analysis_batched([d], ms_opts(B, precision))
    torch.cuda.synchronize()
    (mu_a, A_a), st = outs[0], stats[0]
    assert st["status"] == 0 and st["solver_path"] == 2, st
    A_ref = F.perturbation_update_H(pr.X, Hd, R, pr.grid, pr.Q)
    mu_ref = F.mean_update_H(pr.X, Hd, y, R, pr.grid)
    ea = increment_error(A_a.cpu().numpy(), A_ref, pr.X - pr.X.mean(0))
    em = mean_error(mu_a, mu_ref, pr.X.mean(0))
    assert ea <= bound and em <= bound, (ea, em)


def test_multishift_iteration_cap_reports_not_converged(B):
    pr = workloads.gaussian_problem_1d("capms", n=400, N=5, length_scale=6.0, obs_stride=2, r2=0.1,
                                       half_width=10.0, Q=4, tol=1e-14, seed=14)
    mu_a, A_a, st = B.info_esrf_analysis(pr.grid, dev(pr.X), dev(pr.obs_idx), dev(pr.y), dev(pr.R), pr.Q, 1e-14,
                                         ms_opts(B, 0, max_iter=2))
    assert st["status"] == B.NOT_CONVERGED and st["n_unconverged"] > 0 and st["iters_max"] == 2
    assert np.all(np.isfinite(A_a.cpu().numpy()))


def test_multishift_replays_as_cuda_graph(B):
    """The multi-shift analysis captures into a CUDA graph and replays bit for bit."""
    pr = workloads.gaussian_problem_1d("gms", n=2048, N=16, length_scale=16.0, obs_stride=4, r2=0.5,
                                       half_width=40.0, Q=8, tol=1e-6, seed=43)
    X, obs, y, R = dev(pr.X), dev(pr.obs_idx), dev(pr.y), dev(pr.R)
    opts = ms_opts(B, B.PRECISION_FP32)
    g = B.make_grid(pr.grid)
    need = B.library().info_esrf_workspace_size(ctypes.byref(g), pr.N, pr.d, pr.Q, ctypes.byref(opts))
    ws = B.workspace(need, X.device)
    mu1 = torch.empty(pr.n, dtype=torch.float64, device="cuda")
    A1 = torch.empty((pr.N, pr.n), dtype=torch.float64, device="cuda")
    B.info_esrf_analysis(pr.grid, X, obs, y, R, pr.Q, 1e-6, opts, ws=ws, mu_a=mu1, A_a=A1, stats=False)
    torch.cuda.synchronize()
    ref_mu, ref_A = mu1.clone(), A1.clone()
    mu1.zero_()
    A1.zero_()
    cap = torch.cuda.Stream()
    cap.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=cap):
        B.info_esrf_analysis(pr.grid, X, obs, y, R, pr.Q, 1e-6, opts, ws=ws, mu_a=mu1, A_a=A1, stats=False,
                             stream=cap)
    torch.cuda.current_stream().wait_stream(cap)
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(mu1, ref_mu) and torch.equal(A1, ref_A)


@pytest.mark.parametrize("N,Q,stride", [(2, 1, 5), (3, 2, 7), (9, 3, 1), (17, 5, 4)])
def test_multishift_ragged_and_degenerate_sizes(B, N, Q, stride):
    """Two members, one node, every point observed (d = n = 331, rows not a multiple of 4 per CTA)."""
    pr = workloads.gaussian_problem_1d("g", n=331, N=N, length_scale=5.0, obs_stride=stride, r2=0.7,
                                       half_width=6.0, Q=Q, tol=1e-12, seed=N * 10 + Q)
    for precision, bound, tol in ((0, 1e-10, 1e-12), (1, 1e-4, 1e-6)):
        mu_a, A_a, st = run(B, pr, precision, tol)
        assert st["status"] == 0 and st["solver_path"] == 2, st
        ea, em = errors(pr, mu_a, A_a)
        assert ea <= bound and em <= bound, (precision, ea, em)


def test_multishift_single_observation(B):
    pr = workloads.gaussian_problem_1d("one", n=50, N=6, length_scale=4.0, obs_stride=50, r2=0.2,
                                       half_width=5.0, Q=4, tol=1e-12, seed=9)
    assert pr.d == 1
    mu_a, A_a, st = run(B, pr, 0, 1e-12)
    assert st["status"] == 0, st
    ea, em = errors(pr, mu_a, A_a)
    assert ea <= 1e-10 and em <= 1e-10, (ea, em)
