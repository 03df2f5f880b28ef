"""GPU tests of the learned preconditioner correction (not in the paper).

Gradients of the hand-written backward kernels are checked against the FP64
oracle's finite differences; a trained network must reduce PCG iterations on
a held-out problem while the analysis stays within the FP32 parity bound.
"""
import numpy as np
import pytest
import torch

from parity_checks import increment_error, mean_error
from oracle import filter as F
from oracle import learned as LR
from oracle import pcg, philox, quadrature
from paper_2503_00253_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2503_00253_gb300 import binding
    binding.library()
    return binding


def dev(a, dtype=None):
    t = torch.tensor(np.ascontiguousarray(a), device="cuda")
    return t.to(dtype) if dtype is not None else t


def test_loss_and_gradient_match_oracle(B):
    rng = np.random.default_rng(0)
    d, S = 61, 5
    theta = LR.init_params(seed=1, scale=0.3).astype(np.float32)
    phi = LR.features(np.array([1.1, 3.0, 20.0, 300.0, 1.0]), 2.0, 140.0).astype(np.float32)
    V = rng.standard_normal((S, d)).astype(np.float32)
    Y = rng.standard_normal((S, d)).astype(np.float32)
    Z = rng.standard_normal((S, d)).astype(np.float32)
    loss, grad = B.learn_loss_grad(dev(theta), dev(phi), dev(V), dev(Y), dev(Z))
    args = (theta.astype(np.float64), phi.astype(np.float64), V.astype(np.float64), Y.astype(np.float64),
            Z.astype(np.float64))
    ref_loss = LR.loss(*args)
    ref_grad = LR.fd_gradient(*args)
    assert abs(loss - ref_loss) < 1e-4 * ref_loss
    g = grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - ref_grad) < 1e-3 * np.linalg.norm(ref_grad)


def test_coefficients_match_oracle_network(B):
    theta = LR.init_params(seed=2, scale=0.5).astype(np.float32)
    phi = LR.features(np.array([1.0, 2.0, 10.0, 1e3, 1e5]), 0.8, 40.0).astype(np.float32)
    coef = B.learn_coefficients(dev(theta), dev(phi)).cpu().numpy()
    la, w = LR.coefficients(theta.astype(np.float64), phi.astype(np.float64))
    assert np.max(np.abs(coef[:, 0] / np.exp(la) - 1)) < 1e-5
    assert np.max(np.abs(coef[:, 1:] - w)) < 1e-5 * max(1.0, np.max(np.abs(w)))


def test_krylov_capture_is_consistent_with_oracle_operators(B):
    pr = workloads.gaussian_problem_1d("cap", n=1200, N=10, length_scale=8.0, obs_stride=3, r2=0.3,
                                       half_width=20.0, Q=6, tol=1e-6, seed=31)
    k, os_, seed = 6, 6, 77
    opts = B.make_options(precision=B.PRECISION_FP32, ritz_rank=k, oversample=os_, seed=seed)
    sel = [0, 1, 3 * pr.N + 4]
    K = 4
    V, Y, Z, feat = B.krylov_capture(pr.grid, dev(pr.X), dev(pr.obs_idx), dev(pr.R), pr.Q, sel, K, opts)
    V, Y, Z, feat = (t.cpu().numpy().astype(np.float64) for t in (V, Y, Z, feat))
    mu, Zs = F.anomalies(pr.X)
    W, Sxh, Shh = F.localized_covariances(Zs, pr.obs_idx, pr.grid)
    C = F.normalized_obs_covariance(Shh, pr.R)
    s, p = quadrature.elliptic_rule(pr.Q, F.choose_ell(Shh, pr.R))
    Om = philox.test_matrix(pr.d, k + os_, seed)
    Phi, th = pcg.randomized_ritz(C, k, Om)
    cmin = np.min(np.diag(C))
    for si, sid in enumerate(sel):
        sigma = s[sid // pr.N] + 1.0
        Chat = sigma * np.eye(pr.d) + C
        for it in range(K):
            row = si * K + it
            assert abs(np.linalg.norm(V[row]) - 1.0) < 1e-5
            assert np.linalg.norm(Y[row] - Chat @ V[row]) < 1e-5 * np.linalg.norm(Y[row])
            z = pcg.lmp_apply(Y[row], Chat @ Phi, Phi, th + sigma, sigma + cmin)
            assert np.linalg.norm(Z[row] - z) < 1e-4 * np.linalg.norm(z)
            assert abs(feat[row, 0] - np.log(sigma) / 5) < 1e-6
    # consecutive search directions are C_q-conjugate (PCG)
    for si in range(len(sel)):
        for it in range(K - 1):
            a, b = si * K + it, si * K + it + 1
            assert abs(V[a] @ Y[b]) < 2e-3 * np.sqrt((V[a] @ Y[a]) * (V[b] @ Y[b]))


def _family(seed):
    return workloads.gaussian_problem_1d(f"fam{seed}", n=4096, N=24, length_scale=32.0, obs_stride=4, r2=0.25,
                                         half_width=128.0, Q=16, tol=1e-6, seed=seed)


def test_trained_network_reduces_iterations_and_keeps_parity(B):
    from paper_2503_00253_gb300 import learned
    train_set = [_family(s) for s in (101, 102, 103)]
    theta, max_shift, hist = learned.fit(train_set, K=12, members_per_q=3, steps=300)
    assert hist[-1] < 0.1 * hist[0], (hist[0], hist[-1])
    assert max_shift > 1.0
    pr = _family(104)                                   # held out
    X, obs, y, R = dev(pr.X), dev(pr.obs_idx), dev(pr.y), dev(pr.R)
    base = B.make_options(precision=B.PRECISION_FP32)
    withm = B.make_options(precision=B.PRECISION_FP32, learned_model=theta, learned_max_shift=max_shift)
    mu0, A0, st0 = B.info_esrf_analysis(pr.grid, X, obs, y, R, pr.Q, 1e-6, base)
    mu1, A1, st1 = B.info_esrf_analysis(pr.grid, X, obs, y, R, pr.Q, 1e-6, withm)
    torch.cuda.synchronize()
    assert st0["solver_path"] == 1 and st1["solver_path"] == 1
    assert st1["status"] == 0 and st1["n_unconverged"] == 0
    A_ref = F.perturbation_update(pr.X, pr.obs_idx, pr.R, pr.grid, pr.Q)
    mu_ref = F.mean_update(pr.X, pr.obs_idx, pr.y, pr.R, pr.grid)
    Af = pr.X - pr.X.mean(0)
    for mu_a, A_a in ((mu0, A0), (mu1, A1)):
        assert increment_error(A_a.cpu().numpy(), A_ref, Af) <= 1e-4
        assert mean_error(mu_a, mu_ref, pr.X.mean(0)) <= 1e-4
    print(f"iterations mean {st0['iters_mean']:.2f} -> {st1['iters_mean']:.2f}, "
          f"max {st0['iters_max']} -> {st1['iters_max']}; loss {hist[0]:.3f} -> {hist[-1]:.3f}; "
          f"shift cut-off {max_shift:.3g}")
    assert st1["iters_mean"] < 0.8 * st0["iters_mean"]
    assert st1["iters_max"] < st0["iters_max"]


def test_model_file_round_trip(B, tmp_path):
    theta = LR.init_params(seed=5).astype(np.float32)
    path = str(tmp_path / "model.bin")
    B.model_save(path, theta, 37.5)
    back, ms = B.model_load(path)
    assert np.array_equal(back, theta) and ms == 37.5


def test_bad_network_falls_back_to_paper_preconditioner(B):
    """A network whose stencil ruins the conditioning hits max_iter; the system is re-solved with P_q^-1 alone."""
    pr = workloads.gaussian_problem_1d("fb", n=2048, N=16, length_scale=16.0, obs_stride=4, r2=0.5,
                                       half_width=40.0, Q=8, tol=1e-6, seed=41)
    theta = np.zeros(LR.NPARAM, dtype=np.float32)
    off_b3 = LR.NPARAM - LR.NOUT
    theta[off_b3] = -12.0                                # a = e^-12 / sigma: P^-1 contributes nothing
    theta[off_b3 + 1:] = np.where(np.arange(LR.NTAP) % 2 == 0, 3.0, -3.0)   # high-pass stencil
    X, obs, y, R = dev(pr.X), dev(pr.obs_idx), dev(pr.y), dev(pr.R)
    opts = B.make_options(precision=B.PRECISION_FP32, max_iter=150, learned_model=dev(theta))
    mu_a, A_a, st = B.info_esrf_analysis(pr.grid, X, obs, y, R, pr.Q, 1e-6, opts)
    torch.cuda.synchronize()
    assert st["solver_path"] == 1
    assert st["status"] == 0 and st["n_unconverged"] == 0, st
    A_ref = F.perturbation_update(pr.X, pr.obs_idx, pr.R, pr.grid, pr.Q)
    assert increment_error(A_a.cpu().numpy(), A_ref, pr.X - pr.X.mean(0)) <= 1e-4


def test_headline_configuration_with_trained_network(B):
    """The configuration the benchmark reports, exactly: the 1-D Gaussian forecast n = 8192, N = 40,
    observations every 8th point (d = 1024), R = 0.25, Gaspari-Cohn half-width 256, Q = 32, FP32 bulk,
    tol 1e-6, Ritz rank 10, band capacities from the observation pattern, the network trained on seeds
    11-13 of the same workload (12 Krylov vectors, 3 members per node, 300 Adam steps) with its shift
    cut-off, and the autotuned eigensolver settings.  The analysis must match the FP64 oracle's
    same-node result (Sec. 3.2) within 1e-4, element-wise per member, and use fewer iterations than
    the paper's preconditioner alone."""
    from paper_2503_00253_gb300 import learned
    train_set = [workloads.config2(tol=1e-6, seed=s) for s in (11, 12, 13)]
    theta, cutoff, hist = learned.fit(train_set, K=12, members_per_q=3, steps=300)
    pr = workloads.config2()
    X, obs, y, R = dev(pr.X), dev(pr.obs_idx), dev(pr.y), dev(pr.R)
    max_oo, max_xo = B.neighbor_counts(pr.grid, obs)
    cap = max(max_oo, max_xo)
    opts = B.make_options(precision=B.PRECISION_FP32, ritz_rank=10, max_neighbors=cap, learned_model=theta,
                          learned_max_shift=cutoff)
    B.autotune([dict(grid=pr.grid, X=X, obs_idx=obs, y=y, R=R, Q=pr.Q, tol=1e-6, max_oo=max_oo,
                     max_xo=max_xo)], opts)
    mu_a, A_a, st = B.info_esrf_analysis(pr.grid, X, obs, y, R, pr.Q, 1e-6, opts)
    base = B.make_options(precision=B.PRECISION_FP32, ritz_rank=10, max_neighbors=cap,
                          oversample=int(opts.oversample), power_iters=int(opts.power_iters))
    base.cluster_size = opts.cluster_size
    _, _, st0 = B.info_esrf_analysis(pr.grid, X, obs, y, R, pr.Q, 1e-6, base)
    torch.cuda.synchronize()
    assert st["status"] == 0 and st["n_unconverged"] == 0 and st["n_systems"] == 1281, st
    assert st["learned"] == 1 and st0["learned"] == 0
    A_ref = F.perturbation_update(pr.X, pr.obs_idx, pr.R, pr.grid, pr.Q)
    mu_ref = F.mean_update(pr.X, pr.obs_idx, pr.y, pr.R, pr.grid)
    ea = increment_error(A_a, A_ref, pr.X - pr.X.mean(0))
    em = mean_error(mu_a, mu_ref, pr.X.mean(0))
    print(f"headline configuration: rel err {ea:.2e} (mean {em:.2e}); iterations mean "
          f"{st0['iters_mean']:.2f} -> {st['iters_mean']:.2f}")
    assert ea <= 1e-4 and em <= 1e-4, (ea, em)
    assert st["iters_mean"] < st0["iters_mean"]


def test_learned_flag_reports_when_the_term_is_not_applied(B):
    """Only the cluster-resident 1-D kernel applies the learned correction.  On a layered grid (general
    kernel), or with multi-shift CG, a given model is reported as not applied (stats learned = -1), and
    the analysis still matches the oracle."""
    theta = dev(LR.init_params(seed=3, scale=0.1).astype(np.float32))
    pr = workloads.layered_l96_problem(nx=120, nz=4, N=12, spinup=200, c_x=10.0, c_z=1.0, Q=8)
    X, obs, y, R = dev(pr.X), dev(pr.obs_idx), dev(pr.y), dev(pr.R)
    A_ref = F.perturbation_update(pr.X, pr.obs_idx, pr.R, pr.grid, pr.Q)
    for solver in (B.SOLVER_PCG, B.SOLVER_MULTISHIFT):
        opts = B.make_options(precision=B.PRECISION_FP32, learned_model=theta, solver=solver)
        mu_a, A_a, st = B.info_esrf_analysis(pr.grid, X, obs, y, R, pr.Q, 1e-6, opts)
        torch.cuda.synchronize()
        assert st["status"] == 0 and st["solver_path"] in (0, 2), st
        assert st["learned"] == -1, st
        assert increment_error(A_a, A_ref, pr.X - pr.X.mean(0)) <= 1e-4
    _, _, st = B.info_esrf_analysis(pr.grid, X, obs, y, R, pr.Q, 1e-6, B.make_options(precision=1))
    torch.cuda.synchronize()
    assert st["learned"] == 0
