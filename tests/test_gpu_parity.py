"""GPU parity: every stage of the CUDA path against the FP64 oracle, through the C ABI.

Tolerances: FP64 path <= 1e-10 relative error of the analysis increment
(PCG tolerance 1e-12); FP32 bulk path <= 1e-4 (PCG tolerance 1e-6).  The
error of an analysis is the larger of the Frobenius ratio
||A_gpu - A_ref||_F / ||A_ref - A_f||_F and the per-member element-wise ratio
max_x |A_gpu - A_ref| / max_x |A_ref - A_f| (tests/parity_checks.py).
"""
import math
import types

import numpy as np
import pytest
import torch

from parity_checks import increment_error, mean_error
from oracle import filter as F
from oracle import localization, pcg, philox, quadrature
from paper_2503_00253_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2503_00253_gb300 import binding
    binding.library()
    return binding


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda")


def run_analysis(B, pr, precision=0, tol=None, **kw):
    opts = B.make_options(precision=precision, **kw)
    tol = pr.tol if tol is None else tol
    mu_a, A_a, st = B.info_esrf_analysis(pr.grid, dev(pr.X), dev(pr.obs_idx), dev(pr.y), dev(pr.R),
                                         pr.Q, tol, opts)
    torch.cuda.synchronize()
    return mu_a.cpu().numpy(), A_a.cpu().numpy(), st


def errors(pr, mu_a, A_a, ell=None, rule="elliptic"):
    A_ref = F.perturbation_update(pr.X, pr.obs_idx, pr.R, pr.grid, pr.Q, ell=ell, rule=rule)
    mu_ref = F.mean_update(pr.X, pr.obs_idx, pr.y, pr.R, pr.grid)
    Af = pr.X - pr.X.mean(0)
    mu0 = pr.X.mean(0)
    ea = increment_error(A_a, A_ref, Af)
    em = mean_error(mu_a, mu_ref, mu0)
    return ea, em


# ---------------------------------------------------------------------------
# a2 quadrature, Philox
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("Q,ell", [(1, 10.0), (7, 100.0), (16, 100.0), (32, 1000.0), (48, 1e4), (24, 1e6),
                                   (32, 1e8), (48, 1e10)])
def test_quadrature_nodes_match_oracle(B, Q, ell):
    if ell > 1e4:
        pytest.importorskip("mpmath")   # the oracle's extended-precision elliptic functions
    s, p = B.info_esrf_quadrature_nodes(Q, ell)
    s_ref, p_ref = quadrature.elliptic_rule(Q, ell)
    assert np.max(np.abs(s.cpu().numpy() / s_ref - 1)) < 1e-11
    assert np.max(np.abs(p.cpu().numpy() / p_ref - 1)) < 1e-11


@pytest.mark.parametrize("Q", [1, 2, 5, 16, 33])
def test_gauss_legendre_nodes_match_oracle(B, Q):
    s, p = B.info_esrf_quadrature_nodes(Q, 1.0, B.RULE_GAUSS_LEGENDRE)
    s_ref, p_ref = quadrature.gauss_legendre_rule(Q)
    order = np.argsort(s.cpu().numpy())
    assert np.max(np.abs(s.cpu().numpy()[order] / s_ref - 1)) < 1e-10
    assert np.max(np.abs(p.cpu().numpy()[order] / p_ref - 1)) < 1e-10


def test_philox_normals_match_oracle(B):
    for seed, count in ((0, 5), (123456789, 1001), (2**40 + 7, 4096)):
        g = B.info_esrf_philox_normals(seed, count).cpu().numpy()
        ref = philox.normals(count, seed)
        assert np.max(np.abs(g - ref)) < 1e-12


# ---------------------------------------------------------------------------
# a1/a5: anomalies, bands of C and Sxh, matvec
# ---------------------------------------------------------------------------

def _dense_from_ell(val, col, nnz, rows, cols, cap):
    M = np.zeros((rows, cols))
    for a in range(rows):
        for e in range(nnz[a]):
            M[a, col[e * rows + a]] += val[e * rows + a]
    return M


SMALL_GRIDS = [
    ("1d", lambda: workloads.gaussian_problem_1d("s", n=300, N=11, length_scale=6.0, obs_stride=3, r2=0.4,
                                                 half_width=9.0, Q=5, tol=1e-12, seed=1, obs_offset=1)),
    ("1d_minimage", lambda: workloads.gaussian_problem_1d("s", n=256, N=9, length_scale=6.0, obs_stride=2,
                                                          r2=0.4, half_width=7.5, Q=4, tol=1e-12, seed=2,
                                                          chordal=False)),
    ("layered", lambda: workloads.random_obs_problem(workloads.Grid((40, 1, 6), (True, False, False),
                                                                    (5.0, 1.0, 1.5)), N=10, d=70, r2=0.8,
                                                     Q=6, tol=1e-12, seed=3)),
    ("2d", lambda: workloads.random_obs_problem(workloads.Grid((24, 20, 1), (True, True, False),
                                                               (3.0, 2.5, 1.0)), N=7, d=90, r2=0.5, Q=5,
                                                tol=1e-12, seed=4)),
]


@pytest.mark.parametrize("name,make", SMALL_GRIDS)
@pytest.mark.parametrize("precision", [0, 1])
def test_prepared_bands_match_oracle(B, name, make, precision):
    pr = make()
    opts = B.make_options(precision=precision, ritz_rank=4, oversample=4)
    P = B.Prepared(pr.grid, dev(pr.X), dev(pr.obs_idx), dev(pr.R), pr.Q, opts)
    torch.cuda.synchronize()
    mo, mx = P.capacity()
    mu, Z = F.anomalies(pr.X)
    W, Sxh, Shh = F.localized_covariances(Z, pr.obs_idx, pr.grid)
    C = F.normalized_obs_covariance(Shh, pr.R)
    tol = 1e-13 if precision == 0 else 2e-6
    assert np.max(np.abs(P.export("mu") - mu)) < 1e-13 * np.max(np.abs(mu) + 1)
    assert np.max(np.abs(P.export("W").reshape(pr.d, pr.N) - W)) < tol * np.max(np.abs(W))
    Cg = _dense_from_ell(P.export("oo_val"), P.export("oo_col"), P.export("oo_nnz"), pr.d, pr.d, mo)
    assert np.max(np.abs(Cg - C)) < tol * np.max(np.abs(C))
    # the band holds exactly the pairs inside the GC support
    L_oo = localization.localization_matrix(pr.grid, pr.obs_idx, pr.obs_idx)
    assert np.array_equal(P.export("oo_nnz"), (L_oo > 0).sum(1))
    Sg = _dense_from_ell(P.export("xo_val"), P.export("xo_col"), P.export("xo_nnz"), pr.n, pr.d, mx)
    assert np.max(np.abs(Sg - Sxh)) < tol * np.max(np.abs(Sxh))
    sc = P.export("scalars")
    assert abs(sc[0] / quadrature.gershgorin_bound(C) - 1) < (1e-12 if precision == 0 else 1e-5)
    assert abs(sc[1] / np.min(np.diag(C)) - 1) < (1e-12 if precision == 0 else 1e-5)
    assert int(P.export("status")[0]) == 0


@pytest.mark.parametrize("precision", [0, 1])
def test_obs_matvec_matches_oracle(B, precision):
    pr = workloads.gaussian_problem_1d("m", n=2000, N=13, length_scale=8.0, obs_stride=3, r2=0.3,
                                       half_width=20.0, Q=3, tol=1e-12, seed=5)
    opts = B.make_options(precision=precision, ritz_rank=0)
    P = B.Prepared(pr.grid, dev(pr.X), dev(pr.obs_idx), dev(pr.R), pr.Q, opts)
    mu, Z = F.anomalies(pr.X)
    W, Sxh, Shh = F.localized_covariances(Z, pr.obs_idx, pr.grid)
    C = F.normalized_obs_covariance(Shh, pr.R)
    rng = np.random.default_rng(0)
    V = rng.standard_normal((5, pr.d))
    sig = np.array([1.0, 2.5, 1e3, 1.0 + 1e-9, 17.0])
    Y = P.obs_matvec(dev(V), dev(sig)).cpu().numpy()
    ref = sig[:, None] * V + V @ C.T
    tol = 1e-13 if precision == 0 else 3e-6
    assert np.max(np.abs(Y - ref)) < tol * np.max(np.abs(ref))


# ---------------------------------------------------------------------------
# a4/a7: Ritz pairs and the limited-memory preconditioner
# ---------------------------------------------------------------------------

def test_ritz_pairs_and_lmp_match_oracle(B):
    pr = workloads.gaussian_problem_1d("r", n=1200, N=15, length_scale=6.0, obs_stride=2, r2=0.3,
                                       half_width=12.0, Q=4, tol=1e-12, seed=6)
    k, os_, seed = 8, 8, 987654321
    opts = B.make_options(precision=0, ritz_rank=k, oversample=os_, seed=seed)
    P = B.Prepared(pr.grid, dev(pr.X), dev(pr.obs_idx), dev(pr.R), pr.Q, opts)
    mu, Z = F.anomalies(pr.X)
    W, Sxh, Shh = F.localized_covariances(Z, pr.obs_idx, pr.grid)
    C = F.normalized_obs_covariance(Shh, pr.R)
    Om = philox.test_matrix(pr.d, k + os_, seed)
    Phi_ref, th_ref = pcg.randomized_ritz(C, k, Om, power_iters=1)
    th = P.export("theta")
    assert np.max(np.abs(th - th_ref) / th_ref[0]) < 1e-10
    Phi = P.export("phi").reshape(pr.d, k)
    overlap = np.abs(Phi.T @ Phi_ref)
    assert np.max(np.abs(overlap - np.eye(k))) < 1e-7
    # LMP applied to random vectors for three shifts, against the oracle's own Ritz pairs
    rng = np.random.default_rng(1)
    Rv = rng.standard_normal((3, pr.d))
    sig = np.array([1.0, 3.7, 250.0])
    Zg = P.lmp_apply(dev(Rv), dev(sig)).cpu().numpy()
    cmin = np.min(np.diag(C))
    for v in range(3):
        Chat_Phi = C @ Phi_ref + sig[v] * Phi_ref
        z = pcg.lmp_apply(Rv[v], Chat_Phi, Phi_ref, th_ref + sig[v], sig[v] + cmin)
        assert np.max(np.abs(Zg[v] - z)) < 1e-8 * np.max(np.abs(z))


def test_ritz_pairs_fp32_match_oracle(B):
    """Mixed path: FP32 basis with FP64 Cholesky, one-warp FP32 Jacobi."""
    pr = workloads.gaussian_problem_1d("r32", n=1600, N=20, length_scale=8.0, obs_stride=2, r2=0.3,
                                       half_width=16.0, Q=4, tol=1e-6, seed=7)
    k, os_, seed = 10, 10, 12345
    opts = B.make_options(precision=1, ritz_rank=k, oversample=os_, seed=seed)
    P = B.Prepared(pr.grid, dev(pr.X), dev(pr.obs_idx), dev(pr.R), pr.Q, opts)
    mu, Z = F.anomalies(pr.X)
    W, Sxh, Shh = F.localized_covariances(Z, pr.obs_idx, pr.grid)
    C = F.normalized_obs_covariance(Shh, pr.R)
    Om = philox.test_matrix(pr.d, k + os_, seed)
    Phi_ref, th_ref = pcg.randomized_ritz(C, k, Om, power_iters=1)
    th = P.export("theta")
    assert np.all(np.diff(th) <= 0)
    assert np.max(np.abs(th - th_ref) / th_ref[0]) < 1e-4
    Phi = P.export("phi").reshape(pr.d, k).astype(np.float64)
    CPhi = P.export("cphi").reshape(pr.d, k).astype(np.float64)
    assert np.max(np.abs(Phi.T @ Phi - np.eye(k))) < 1e-4
    assert np.max(np.abs(CPhi - C @ Phi)) < 1e-5 * np.max(np.abs(CPhi))
    # Rayleigh quotients of the returned vectors are the returned values
    rq = np.einsum("ai,ai->i", Phi, C @ Phi)
    assert np.max(np.abs(rq - th) / th[0]) < 1e-4
    # leading Ritz vectors agree with the oracle's where the gap is large
    gap = np.abs(np.diff(th_ref)) / th_ref[0]
    for i in range(k - 1):
        if gap[i] > 1e-2 and (i == 0 or gap[i - 1] > 1e-2):
            assert abs(Phi[:, i] @ Phi_ref[:, i]) > 1 - 1e-3


# ---------------------------------------------------------------------------
# end to end
# ---------------------------------------------------------------------------

def test_config1_fp64_parity(B):
    pr = workloads.config1()
    mu_a, A_a, st = run_analysis(B, pr, precision=0)
    ea, em = errors(pr, mu_a, A_a)
    assert st["status"] == 0 and st["n_unconverged"] == 0
    assert st["n_systems"] == pr.Q * pr.N + 1
    assert ea <= 1e-10 and em <= 1e-10, (ea, em)
    # zero-mean analysis perturbations (Theorem 3)
    assert np.max(np.abs(A_a.sum(0))) < 1e-10 * np.max(np.abs(A_a))


@pytest.mark.parametrize("name,make", SMALL_GRIDS)
@pytest.mark.parametrize("precision,tol,bound", [(0, 1e-12, 1e-10), (1, 1e-6, 1e-4)])
def test_small_problems_parity(B, name, make, precision, tol, bound):
    pr = make()
    mu_a, A_a, st = run_analysis(B, pr, precision=precision, tol=tol, ritz_rank=5, oversample=5)
    ea, em = errors(pr, mu_a, A_a)
    assert st["status"] == 0, st
    assert ea <= bound and em <= bound, (ea, em)


@pytest.mark.parametrize("kw", [dict(ritz_rank=0), dict(ritz_rank=24, oversample=8), dict(rule=1),
                                dict(ell=1e5), dict(power_iters=0)])
def test_option_variants_parity(B, kw):
    pr = workloads.gaussian_problem_1d("v", n=900, N=10, length_scale=5.0, obs_stride=3, r2=0.5,
                                       half_width=10.0, Q=9, tol=1e-12, seed=8)
    mu_a, A_a, st = run_analysis(B, pr, precision=0, **kw)
    rule = "gauss_legendre" if kw.get("rule") == 1 else "elliptic"
    ea, em = errors(pr, mu_a, A_a, ell=kw.get("ell"), rule=rule)
    assert st["status"] == 0, st
    assert ea <= 1e-10 and em <= 1e-10, (ea, em)


@pytest.mark.parametrize("N,Q,stride", [(2, 1, 5), (3, 2, 7), (9, 3, 1), (17, 5, 4)])
def test_ragged_and_degenerate_sizes(B, N, Q, stride):
    pr = workloads.gaussian_problem_1d("g", n=331, N=N, length_scale=5.0, obs_stride=stride, r2=0.7,
                                       half_width=6.0, Q=Q, tol=1e-12, seed=N * 10 + Q)
    for precision, bound, tol in ((0, 1e-10, 1e-12), (1, 1e-4, 1e-6)):
        mu_a, A_a, st = run_analysis(B, pr, precision=precision, tol=tol, ritz_rank=3, oversample=3)
        ea, em = errors(pr, mu_a, A_a)
        assert st["status"] == 0, st
        assert ea <= bound and em <= bound, (precision, ea, em)


def test_single_observation(B):
    pr = workloads.gaussian_problem_1d("one", n=50, N=6, length_scale=4.0, obs_stride=50, r2=0.2,
                                       half_width=5.0, Q=4, tol=1e-12, seed=9)
    assert pr.d == 1
    mu_a, A_a, st = run_analysis(B, pr, precision=0, ritz_rank=2)
    ea, em = errors(pr, mu_a, A_a)
    assert ea <= 1e-10 and em <= 1e-10


def test_fp32_band_kernel_falls_back_when_band_degenerate(B):
    """One observation: its band is not a proper sub-range, so the general kernel solves."""
    pr = workloads.gaussian_problem_1d("one32", n=64, N=9, length_scale=4.0, obs_stride=64, r2=0.2,
                                       half_width=5.0, Q=5, tol=1e-6, seed=19)
    mu_a, A_a, st = run_analysis(B, pr, precision=1, ritz_rank=1)
    ea, em = errors(pr, mu_a, A_a)
    assert st["solver_path"] == 0 and st["status"] == 0
    assert ea <= 1e-4 and em <= 1e-4


@pytest.mark.parametrize("n,stride,hw,N", [(4096, 4, 40.0, 40), (3001, 3, 25.0, 33), (1500, 2, 60.0, 20)])
def test_fp32_band_kernel_sizes(B, n, stride, hw, N):
    """Cluster-resident kernel over several slice/cluster shapes, ragged last slice included."""
    pr = workloads.gaussian_problem_1d("bk", n=n, N=N, length_scale=hw / 3, obs_stride=stride, r2=0.3,
                                       half_width=hw, Q=7, tol=1e-6, seed=n + N)
    mu_a, A_a, st = run_analysis(B, pr, precision=1, ritz_rank=6, oversample=6)
    ea, em = errors(pr, mu_a, A_a)
    assert st["status"] == 0, st
    assert st["solver_path"] == 1
    assert ea <= 1e-4 and em <= 1e-4, (ea, em)


def test_fp32_band_kernel_with_widely_varying_R(B):
    """Observation-error variances spread over four orders of magnitude, so that
    neighbouring rows of C differ in size by up to 10^4: the cluster kernel's
    FP16 tensor-core matvec (C split into scaled FP16 pairs) must still meet the
    mixed-precision bound."""
    import dataclasses
    pr = workloads.gaussian_problem_1d("rvar", n=4096, N=24, length_scale=24.0, obs_stride=4, r2=0.5,
                                       half_width=60.0, Q=12, tol=1e-6, seed=77)
    rng = np.random.default_rng(78)
    R = 0.5 * 10.0 ** rng.uniform(-2.0, 2.0, pr.d)
    y = pr.truth[pr.obs_idx] + np.sqrt(R) * rng.standard_normal(pr.d)
    pr = dataclasses.replace(pr, R=R, y=y)
    mu_a, A_a, st = run_analysis(B, pr, precision=1, ritz_rank=8)
    ea, em = errors(pr, mu_a, A_a)
    assert st["status"] == 0 and st["solver_path"] == 1, st
    assert ea <= 1e-4 and em <= 1e-4, (ea, em)


def test_mean_and_perturbation_calls_alone(B):
    pr = workloads.gaussian_problem_1d("sep", n=500, N=12, length_scale=5.0, obs_stride=4, r2=0.5,
                                       half_width=8.0, Q=6, tol=1e-12, seed=10)
    X, obs, y, R = dev(pr.X), dev(pr.obs_idx), dev(pr.y), dev(pr.R)
    mu_a, st = B.info_esrf_mean_update(pr.grid, X, obs, y, R, 1e-12)
    A_a, st2 = B.info_esrf_perturbation_update(pr.grid, X, obs, R, pr.Q, 1e-12)
    torch.cuda.synchronize()
    ea, em = errors(pr, mu_a.cpu().numpy(), A_a.cpu().numpy())
    assert st["n_systems"] == 1 and st2["n_systems"] == pr.Q * pr.N
    assert ea <= 1e-10 and em <= 1e-10


def test_fixed_iterations_match_oracle_pcg(B):
    """Paper-style fixed iteration counts (2 and 10): same iterates as the oracle's PCG + LMP."""
    pr = workloads.gaussian_problem_1d("fix", n=600, N=8, length_scale=6.0, obs_stride=2, r2=0.4,
                                       half_width=10.0, Q=5, tol=1e-12, seed=11)
    k, os_, seed = 6, 6, 4242
    mu, Z = F.anomalies(pr.X)
    W, Sxh, Shh = F.localized_covariances(Z, pr.obs_idx, pr.grid)
    C = F.normalized_obs_covariance(Shh, pr.R)
    s, p = quadrature.elliptic_rule(pr.Q, F.choose_ell(Shh, pr.R))
    Om = philox.test_matrix(pr.d, k + os_, seed)
    for iters in (2, 10):
        vbar, _ = pcg.solve_normalized(C, s, p, W, pr.R, k=k, Omega=Om, fixed_iters=iters)
        A_ref = math.sqrt(pr.N - 1) * (Z - Sxh @ vbar).T
        opts = B.make_options(precision=0, ritz_rank=k, oversample=os_, seed=seed, fixed_iters=iters)
        A_a, st = B.info_esrf_perturbation_update(pr.grid, dev(pr.X), dev(pr.obs_idx), dev(pr.R), pr.Q, 1e-12,
                                                  opts)
        Af = pr.X - pr.X.mean(0)
        err = increment_error(A_a.cpu().numpy(), A_ref, Af)
        assert err < 1e-9, (iters, err)
        assert st["iters_max"] == iters


def test_config2_parity_fp64_and_fp32(B):
    pr = workloads.config2()
    A_ref = F.perturbation_update(pr.X, pr.obs_idx, pr.R, pr.grid, pr.Q)
    mu_ref = F.mean_update(pr.X, pr.obs_idx, pr.y, pr.R, pr.grid)
    Af = pr.X - pr.X.mean(0)
    mu0 = pr.X.mean(0)
    for precision, tol, bound in ((0, 1e-12, 1e-10), (1, 1e-6, 1e-4)):
        mu_a, A_a, st = run_analysis(B, pr, precision=precision, tol=tol)
        ea = increment_error(A_a, A_ref, Af)
        em = mean_error(mu_a, mu_ref, mu0)
        assert st["status"] == 0, st
        assert st["n_systems"] == 1281
        # the FP32 path on this 1-D network runs on the cluster-resident band kernel
        assert st["solver_path"] == (1 if precision == 1 else 0)
        assert ea <= bound and em <= bound, (precision, ea, em)


def test_batched_uneven_parity(B):
    probs = workloads.uneven_batch(count=5, seed=12, tol=1e-12, n_min=200, n_max=1500)
    dicts = [dict(grid=p.grid, X=dev(p.X), obs_idx=dev(p.obs_idx), y=dev(p.y), R=dev(p.R), Q=p.Q, tol=1e-12)
             for p in probs]
    outs, stats = B.info_esrf_analysis_batched(dicts, B.make_options(precision=0))
    torch.cuda.synchronize()
    for p, (mu_a, A_a), st in zip(probs, outs, stats):
        ea, em = errors(p, mu_a.cpu().numpy(), A_a.cpu().numpy())
        assert st["status"] == 0 and st["n_systems"] == p.Q * p.N + 1
        assert ea <= 1e-10 and em <= 1e-10, (p.name, ea, em)


# ---------------------------------------------------------------------------
# failure handling (host-visible status; nothing faults)
# ---------------------------------------------------------------------------

def test_invalid_inputs_return_codes(B):
    pr = workloads.gaussian_problem_1d("bad", n=200, N=6, length_scale=4.0, obs_stride=4, r2=0.5,
                                       half_width=5.0, Q=3, tol=1e-10, seed=13)
    def call(obs=None, R=None, X=None):
        with pytest.raises(B.InfoEsrfError) as ei:
            B.info_esrf_analysis(pr.grid, dev(pr.X if X is None else X), dev(pr.obs_idx if obs is None else obs),
                                 dev(pr.y), dev(pr.R if R is None else R), pr.Q, pr.tol)
        return ei.value.code
    bad_obs = pr.obs_idx.copy(); bad_obs[3] = 10**6
    assert call(obs=bad_obs) == B.ERR_BAD_OBS_INDEX
    unsorted = pr.obs_idx.copy(); unsorted[[1, 2]] = unsorted[[2, 1]]
    assert call(obs=unsorted) == B.ERR_BAD_OBS_INDEX
    badR = pr.R.copy(); badR[0] = 0.0
    assert call(R=badR) == B.ERR_NONPOSITIVE_R
    badX = pr.X.copy(); badX[1, 5] = np.nan
    assert call(X=badX) == B.ERR_NONFINITE


def test_iteration_cap_reports_not_converged(B):
    pr = workloads.gaussian_problem_1d("cap", n=400, N=5, length_scale=6.0, obs_stride=2, r2=0.1,
                                       half_width=10.0, Q=4, tol=1e-14, seed=14)
    opts = B.make_options(precision=0, ritz_rank=0, max_iter=2)
    mu_a, A_a, st = B.info_esrf_analysis(pr.grid, dev(pr.X), dev(pr.obs_idx), dev(pr.y), dev(pr.R), pr.Q,
                                         1e-14, opts)
    assert st["status"] == B.NOT_CONVERGED and st["n_unconverged"] > 0 and st["iters_max"] == 2
    assert np.all(np.isfinite(A_a.cpu().numpy()))


def test_analysis_replays_as_cuda_graph(B):
    """The analysis call captures into a CUDA graph (side stream included) and
    its replay reproduces the direct call bit for bit."""
    pr = workloads.gaussian_problem_1d("g", n=2048, N=16, length_scale=16.0, obs_stride=4, r2=0.5,
                                       half_width=40.0, Q=8, tol=1e-6, seed=43)
    X, obs, y, R = dev(pr.X), dev(pr.obs_idx), dev(pr.y), dev(pr.R)
    opts = B.make_options(precision=B.PRECISION_FP32)
    import ctypes
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


def test_batched_equals_single_calls_bit_for_bit(B):
    """FP64 batched launch sequence (uneven n, N, d, Q in one persistent PCG launch) gives the
    same bits as one call per problem: every system's arithmetic is independent of the others."""
    probs = workloads.uneven_batch(count=6, seed=21, tol=1e-10, n_min=300, n_max=3000)
    dicts = [dict(grid=p.grid, X=dev(p.X), obs_idx=dev(p.obs_idx), y=dev(p.y), R=dev(p.R), Q=p.Q, tol=1e-10)
             for p in probs]
    opts = B.make_options(precision=0)
    outs, stats = B.info_esrf_analysis_batched(dicts, opts)
    torch.cuda.synchronize()
    for p, dct, (mu_b, A_b), st in zip(probs, dicts, outs, stats):
        mu_s, A_s, st_s = B.info_esrf_analysis(p.grid, dct["X"], dct["obs_idx"], dct["y"], dct["R"], p.Q, 1e-10,
                                               opts)
        torch.cuda.synchronize()
        assert torch.equal(mu_b, mu_s) and torch.equal(A_b, A_s), p.name
        assert st["iters_max"] == st_s["iters_max"]


def test_batched_fp32_mixes_band_and_general_kernels(B):
    """FP32 batch with cluster_size 8: three 1-D problems go to the cluster-resident
    band kernel (one launch each), one 1-D problem with a single observation falls back on
    the device, and a 2-D problem is solved by the general kernel.  Every problem
    meets the mixed-precision bound against the oracle, reports the path that
    solved it, and equals its single call bit for bit."""
    probs = workloads.uneven_batch(count=3, seed=31, tol=1e-6, n_min=1000, n_max=3000)
    probs.append(workloads.gaussian_problem_1d("one32", n=64, N=9, length_scale=4.0, obs_stride=64, r2=0.2,
                                               half_width=5.0, Q=5, tol=1e-6, seed=19))
    probs.append(workloads.random_obs_problem(workloads.Grid((24, 20, 1), (True, True, False), (3.0, 2.5, 1.0)),
                                              N=7, d=90, r2=0.5, Q=5, tol=1e-6, seed=4))
    expect_path = [1, 1, 1, 0, 0]
    dicts = [dict(grid=p.grid, X=dev(p.X), obs_idx=dev(p.obs_idx), y=dev(p.y), R=dev(p.R), Q=p.Q, tol=1e-6)
             for p in probs]
    opts = B.make_options(precision=B.PRECISION_FP32, ritz_rank=8, cluster_size=8)
    outs, stats = B.info_esrf_analysis_batched(dicts, opts)
    torch.cuda.synchronize()
    for p, dct, (mu_b, A_b), st, path in zip(probs, dicts, outs, stats, expect_path):
        assert st["status"] == 0 and st["solver_path"] == path, (p.name, st)
        ea, em = errors(p, mu_b.cpu().numpy(), A_b.cpu().numpy())
        assert ea <= 1e-4 and em <= 1e-4, (p.name, ea, em)
        mu_s, A_s, st_s = B.info_esrf_analysis(p.grid, dct["X"], dct["obs_idx"], dct["y"], dct["R"], p.Q, 1e-6,
                                               opts)
        torch.cuda.synchronize()
        assert st_s["solver_path"] == path
        assert torch.equal(mu_b, mu_s) and torch.equal(A_b, A_s), p.name
    # cluster_size -1 turns the band kernel off, and 0 leaves it off in a batch:
    # the general kernel solves every problem
    for cs in (-1, 0):
        outs, stats = B.info_esrf_analysis_batched(dicts, B.make_options(precision=B.PRECISION_FP32, ritz_rank=8,
                                                                         cluster_size=cs))
        torch.cuda.synchronize()
        for p, (mu_b, A_b), st in zip(probs, outs, stats):
            assert st["status"] == 0 and st["solver_path"] == 0, (cs, p.name, st)
            ea, em = errors(p, mu_b.cpu().numpy(), A_b.cpu().numpy())
            assert ea <= 1e-4 and em <= 1e-4, (cs, p.name, ea, em)


def _l96(nx, nz, N, spinup, seed, c_x, c_z):
    return workloads.layered_l96_problem(nx=nx, nz=nz, N=N, spinup=spinup, seed=seed, Q=24, c_x=c_x, c_z=c_z)


def test_layered_l96_full_size_parity(B):
    """Layered Lorenz-96 analysis at full size: 8 layers x 960 longitudes, N=40, 25% random
    observations (d=1920), anisotropic Gaspari-Cohn (60 horizontally, 2 layers vertically), Q=24,
    in FP32, in BF16 (tensor-core block-tile path: BF16 matvec with FP32 accumulation) and in FP64."""
    pr = workloads.layered_l96_problem()
    A_ref = F.perturbation_update(pr.X, pr.obs_idx, pr.R, pr.grid, pr.Q)
    mu_ref = F.mean_update(pr.X, pr.obs_idx, pr.y, pr.R, pr.grid)
    Af = pr.X - pr.X.mean(0)
    mu0 = pr.X.mean(0)
    for prec, tol, bound in ((1, 1e-6, 1e-4), (2, 1e-6, 1e-4), (0, 1e-12, 1e-10)):
        mu_a, A_a, st = B.info_esrf_analysis(pr.grid, dev(pr.X), dev(pr.obs_idx), dev(pr.y), dev(pr.R), pr.Q, tol,
                                             B.make_options(precision=prec))
        torch.cuda.synchronize()
        assert st["status"] == 0 and st["n_unconverged"] == 0
        ea = increment_error(A_a.cpu().numpy(), A_ref, Af)
        em = mean_error(mu_a, mu_ref, mu0)
        assert ea <= bound and em <= bound, (prec, ea, em)


@pytest.mark.parametrize("precision", [1, 2])
def test_layered_l96_cycling_tracks_truth(B, precision):
    """Cycled assimilation on a reduced layered Lorenz-96 (4 layers x 240, N=20, 25% observed,
    localization 12 horizontally and 1 layer vertically, relaxation to prior spread 0.5), starting
    from a climatological ensemble: every cycle converges, the first matches the oracle, and the
    analysis error falls well below the climatological spread (the oracle run of the same set-up
    reaches about 1.05 after 40 cycles, from 2.9)."""
    nx, nz, N, cycles, dt, steps = 240, 4, 20, 40, 0.01, 5
    pr = _l96(nx, nz, N, spinup=500, seed=31, c_x=12.0, c_z=1.0)
    rng = np.random.default_rng(7)
    X = pr.X.reshape(N, nz, nx).copy()
    truth = pr.truth.reshape(nz, nx).copy()
    obs = pr.obs_idx
    rmse_f, rmse_a = [], []
    opts = B.make_options(precision=precision)
    for c in range(cycles):
        if c > 0:
            X = workloads.ll96_rk4(X, dt, steps)
            truth = workloads.ll96_rk4(truth[None], dt, steps)[0]
        Xf = X.reshape(N, -1)
        y = truth.reshape(-1)[obs] + np.sqrt(pr.R) * rng.standard_normal(obs.size)
        mu_a, A_a, st = B.info_esrf_analysis(pr.grid, dev(Xf), dev(obs), dev(y), dev(pr.R), pr.Q, 1e-6, opts)
        torch.cuda.synchronize()
        assert st["status"] == 0 and st["n_unconverged"] == 0
        mu_a, A_a = mu_a.cpu().numpy(), A_a.cpu().numpy()
        if c == 0:
            A_ref = F.perturbation_update(Xf, obs, pr.R, pr.grid, pr.Q)
            mu_ref = F.mean_update(Xf, obs, y, pr.R, pr.grid)
            assert increment_error(A_a, A_ref, Xf - Xf.mean(0)) <= 1e-4
            assert mean_error(mu_a, mu_ref, Xf.mean(0)) <= 1e-4
        sf = Xf.std(0, ddof=1).mean()
        sa = A_a.std(0, ddof=1).mean()
        A_a = A_a * (1.0 + 0.5 * (sf - sa) / max(sa, 1e-12))
        rmse_f.append(np.sqrt(np.mean((Xf.mean(0) - truth.reshape(-1)) ** 2)))
        rmse_a.append(np.sqrt(np.mean((mu_a - truth.reshape(-1)) ** 2)))
        X = (mu_a[None, :] + A_a).reshape(N, nz, nx)
    clim = pr.truth.std()
    assert np.mean(rmse_a[30:]) < 0.45 * clim, (rmse_a, clim)
    assert np.mean(rmse_a[30:]) < 0.6 * np.mean(rmse_a[:5])
    assert np.mean(rmse_a) < np.mean(rmse_f)


def test_autotune_picks_a_converging_setting_and_keeps_parity(B):
    """The native autotuner times cluster size, power iterations and oversampling on the caller's
    problem and returns one of its candidates; the tuned analysis still matches the oracle."""
    pr = workloads.gaussian_problem_1d("tune", n=4096, N=16, length_scale=32.0, obs_stride=4, r2=0.25,
                                       half_width=128.0, Q=12, tol=1e-6, seed=51)
    probs = [dict(grid=pr.grid, X=dev(pr.X), obs_idx=dev(pr.obs_idx), y=dev(pr.y), R=dev(pr.R), Q=pr.Q, tol=1e-6)]
    opts = B.make_options(precision=1)
    best = B.autotune(probs, opts)
    assert best > 0.0
    assert opts.cluster_size in (0, 4, -1) and opts.power_iters in (0, 1) and opts.oversample in (2, 6, 10)
    mu_a, A_a, st = B.info_esrf_analysis(pr.grid, probs[0]["X"], probs[0]["obs_idx"], probs[0]["y"], probs[0]["R"],
                                         pr.Q, 1e-6, opts)
    torch.cuda.synchronize()
    assert st["status"] == 0 and st["n_unconverged"] == 0
    ea, em = errors(pr, mu_a.cpu().numpy(), A_a.cpu().numpy())
    assert ea <= 1e-4 and em <= 1e-4


# ---------------------------------------------------------------------------
# General linear observation operators (the paper's weighted sums)
# ---------------------------------------------------------------------------

def _h_dict(pr, H, y, R, tol):
    _, (rowptr, col, val) = H
    return dict(grid=pr.grid, X=dev(pr.X), H=(dev(rowptr), dev(col), dev(val)), y=dev(y), R=dev(R), Q=pr.Q,
                tol=tol)


def _h_errors(pr, Hd, y, R, mu_a, A_a):
    A_ref = F.perturbation_update_H(pr.X, Hd, R, pr.grid, pr.Q)
    mu_ref = F.mean_update_H(pr.X, Hd, y, R, pr.grid)
    Af = pr.X - pr.X.mean(0)
    ea = increment_error(A_a, A_ref, Af)
    em = mean_error(mu_a, mu_ref, pr.X.mean(0))
    return ea, em


@pytest.mark.parametrize("precision,tol,bound", [(0, 1e-12, 1e-10), (1, 1e-6, 1e-4)])
def test_general_H_gaussian_channels_parity(B, precision, tol, bound):
    """The single-cycle experiment's operator shape (Sec. 4.1): n = 2000 on a circle,
    d = 100 Gaussian-weighted channel sums of bandwidth 10, N = 20."""
    pr = workloads.gaussian_problem_1d("chan", n=2000, N=20, length_scale=10.0, obs_stride=20, r2=0.5,
                                       half_width=20.0, Q=16, tol=tol, seed=91)
    H = workloads.gaussian_channel_operator(pr.n, 100, 10.0)
    rng = np.random.default_rng(92)
    R = np.full(100, 0.5)
    y = H[0] @ pr.truth + np.sqrt(R) * rng.standard_normal(100)
    outs, stats = B.info_esrf_analysis_batched([_h_dict(pr, H, y, R, tol)], B.make_options(precision=precision))
    torch.cuda.synchronize()
    (mu_a, A_a), st = outs[0], stats[0]
    assert st["status"] == 0 and st["solver_path"] == 0, st
    ea, em = _h_errors(pr, H[0], y, R, mu_a.cpu().numpy(), A_a.cpu().numpy())
    assert ea <= bound and em <= bound, (ea, em)


@pytest.mark.parametrize("precision,tol,bound", [(0, 1e-12, 1e-10), (1, 1e-6, 1e-4)])
def test_general_H_column_sums_layered_parity(B, precision, tol, bound):
    """The layered experiment's operator shape (Sec. 5.1): 8 observed columns of a
    40 x 32 grid, 5 weighted vertical sums each, isotropic localization length 3."""
    grid = workloads.Grid((40, 1, 32), (True, False, False), (3.0, 1.0, 3.0))
    base = workloads.random_obs_problem(grid, N=24, d=10, r2=0.25, Q=8, tol=tol, seed=93)
    H = workloads.column_sum_operator((40, 1, 32), list(range(0, 40, 5)), 5, 6.0, 8.0)
    rng = np.random.default_rng(94)
    R = np.full(40, 0.25)
    y = H[0] @ base.truth + np.sqrt(R) * rng.standard_normal(40)
    outs, stats = B.info_esrf_analysis_batched([_h_dict(base, H, y, R, tol)], B.make_options(precision=precision))
    torch.cuda.synchronize()
    (mu_a, A_a), st = outs[0], stats[0]
    assert st["status"] == 0, st
    ea, em = _h_errors(base, H[0], y, R, mu_a.cpu().numpy(), A_a.cpu().numpy())
    assert ea <= bound and em <= bound, (ea, em)


def test_batch_mixes_index_and_general_H_problems(B):
    """An index-observed problem and a weighted-sum problem in one batched call:
    each meets the FP64 bound and equals its own single-problem call bit for bit."""
    p1 = workloads.gaussian_problem_1d("idx", n=600, N=12, length_scale=6.0, obs_stride=4, r2=0.4,
                                       half_width=10.0, Q=6, tol=1e-12, seed=95)
    p2 = workloads.gaussian_problem_1d("chan2", n=800, N=10, length_scale=8.0, obs_stride=16, r2=0.5,
                                       half_width=16.0, Q=8, tol=1e-12, seed=96)
    H = workloads.gaussian_channel_operator(p2.n, 40, 6.0)
    y2 = H[0] @ p2.truth + 0.3 * np.random.default_rng(97).standard_normal(40)
    R2 = np.full(40, 0.4)
    d1 = dict(grid=p1.grid, X=dev(p1.X), obs_idx=dev(p1.obs_idx), y=dev(p1.y), R=dev(p1.R), Q=p1.Q, tol=1e-12)
    d2 = _h_dict(p2, H, y2, R2, 1e-12)
    opts = B.make_options(precision=0)
    outs, stats = B.info_esrf_analysis_batched([d1, d2], opts)
    torch.cuda.synchronize()
    assert all(s["status"] == 0 for s in stats), stats
    ea, em = errors(p1, outs[0][0].cpu().numpy(), outs[0][1].cpu().numpy())
    assert ea <= 1e-10 and em <= 1e-10, (ea, em)
    ea, em = _h_errors(p2, H[0], y2, R2, outs[1][0].cpu().numpy(), outs[1][1].cpu().numpy())
    assert ea <= 1e-10 and em <= 1e-10, (ea, em)
    for dd, (mu_b, A_b) in ((d1, outs[0]), (d2, outs[1])):
        single, _ = B.info_esrf_analysis_batched([dd], opts)
        torch.cuda.synchronize()
        assert torch.equal(single[0][0], mu_b) and torch.equal(single[0][1], A_b)


def test_general_H_malformed_is_rejected(B):
    """A column index outside the state makes the call fail with the bad-observation
    code; nothing outside the arrays is read."""
    pr = workloads.gaussian_problem_1d("badH", n=300, N=8, length_scale=5.0, obs_stride=10, r2=0.5,
                                       half_width=8.0, Q=4, tol=1e-10, seed=98)
    Hd, (rowptr, col, val) = workloads.gaussian_channel_operator(pr.n, 12, 4.0)
    col = col.copy()
    col[5] = pr.n + 7
    y = Hd @ pr.truth
    R = np.full(12, 0.5)
    d = dict(grid=pr.grid, X=dev(pr.X), H=(dev(rowptr), dev(col), dev(val)), y=dev(y), R=dev(R), Q=pr.Q, tol=1e-10)
    with pytest.raises(B.InfoEsrfError) as ei:
        B.info_esrf_analysis_batched([d], B.make_options(precision=0))
    assert ei.value.code == B.ERR_BAD_OBS_INDEX
