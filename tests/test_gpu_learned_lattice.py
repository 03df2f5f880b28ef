"""GPU tests of the learned correction's 2-D lattice form on the BF16 path (not in the paper).

The lattice loss and its hand-written gradient are checked against the FP64
oracle's loss and finite differences; the BF16 path's Krylov capture against
the oracle's operators; a network trained on 2-D problems must reduce the
BF16 path's iterations on a held-out problem while the analysis stays within
the mixed-precision bound (1e-4, element-wise per member) of the oracle's
same-node result (Sec. 3.2); a network that ruins the conditioning falls back
to the paper's preconditioner; observations that do not fill a lattice leave
the term off and say so.
"""
import numpy as np
import pytest
import torch

from parity_checks import increment_error, mean_error
from oracle import filter as F
from oracle import learned as LR
from oracle import sparse as S
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


@pytest.mark.parametrize("shape", [(8, 6), (3, 7), (16, 16)])
def test_lattice_loss_and_gradient_match_oracle(B, shape):
    Lx, Ly = shape
    rng = np.random.default_rng(Lx * 100 + Ly)
    d, nsamp = Lx * Ly, 4
    theta = LR.init_params(seed=11, scale=0.3).astype(np.float32)
    phi = LR.features(np.array([1.2, 4.0, 30.0, 500.0]), 1.8, 120.0).astype(np.float32)
    V = rng.standard_normal((nsamp, d)).astype(np.float32)
    Y = rng.standard_normal((nsamp, d)).astype(np.float32)
    Z = rng.standard_normal((nsamp, d)).astype(np.float32)
    loss, grad = B.learn_loss_grad_lattice(dev(theta), dev(phi), dev(V), dev(Y), dev(Z), Lx, Ly)
    args = (theta.astype(np.float64), phi.astype(np.float64), V.astype(np.float64), Y.astype(np.float64),
            Z.astype(np.float64), Lx, Ly)
    ref_loss = LR.loss_lattice(*args)
    ref_grad = LR.fd_gradient_lattice(*args)
    assert abs(loss - ref_loss) < 1e-4 * ref_loss, (loss, ref_loss)
    g = grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - ref_grad) < 1e-3 * np.linalg.norm(ref_grad)


def _small_2d(seed, nx=64):
    return workloads.gaussian_problem_2d(nx=nx, ny=nx, N=12, length_scale=6.0, obs_stride=2, r2=0.5,
                                         half_width=8.0, Q=6, tol=1e-6, seed=seed)


def test_lattice_capture_is_consistent_with_oracle_operators(B):
    pr = _small_2d(21)
    sel = [0, 5, 3 * pr.N + 2]
    K = 4
    opts = B.make_options(precision=B.PRECISION_BF16, ritz_rank=6)
    V, Y, Z, feat, lx, ly = B.krylov_capture_lattice(pr.grid, dev(pr.X), dev(pr.obs_idx), dev(pr.R), pr.Q, sel,
                                                     K, opts)
    assert (lx, ly) == (32, 32)
    V, Y, Z, feat = (t.cpu().numpy().astype(np.float64) for t in (V, Y, Z, feat))
    # the three systems run longer than K iterations (the node-0 and node-3 shifts of this problem)
    assert all(np.linalg.norm(V[r]) > 0 for r in range(len(sel) * K)), [np.linalg.norm(V[r]) for r in range(12)]
    mu, Zs = F.anomalies(pr.X)
    W, Sxh, Shh = F.localized_covariances(Zs, pr.obs_idx, pr.grid)
    C = F.normalized_obs_covariance(Shh, pr.R)
    from oracle import quadrature
    s, _ = quadrature.elliptic_rule(pr.Q, F.choose_ell(Shh, pr.R))
    for si, sid in enumerate(sel):
        sigma = s[sid // pr.N] + 1.0
        for it in range(K):
            row = si * K + it
            nv = np.linalg.norm(V[row])
            if nv == 0.0:
                continue                                   # the system had stopped
            assert abs(nv - 1.0) < 1e-5
            # y = sigma v + C v (the BF16 direction v exact; C as hi + lo BF16 planes)
            yref = sigma * V[row] + C @ V[row]
            assert np.linalg.norm(Y[row] - yref) < 1e-4 * np.linalg.norm(yref)
            assert abs(feat[row, 0] - np.log(sigma) / 5) < 1e-6
            # z = P_q^-1 y is SPD-consistent: y^T z > 0 and z = y on the complement of the Ritz space
            assert Y[row] @ Z[row] > 0
    # consecutive directions are C_q-conjugate up to the BF16 rounding of p
    for si in range(len(sel)):
        for it in range(K - 1):
            a, b = si * K + it, si * K + it + 1
            if np.linalg.norm(V[b]) == 0.0:
                continue
            assert abs(V[a] @ Y[b]) < 2e-2 * np.sqrt((V[a] @ Y[a]) * (V[b] @ Y[b]))


def _family(seed):
    return workloads.gaussian_problem_2d(nx=128, ny=128, N=16, length_scale=8.0, obs_stride=2, r2=0.5,
                                         half_width=12.0, Q=8, tol=1e-6, seed=seed)


def test_trained_lattice_network_reduces_iterations_and_keeps_parity(B):
    from paper_2503_00253_gb300 import learned
    train_set = [_family(s) for s in (201, 202)]
    theta, max_shift, hist = learned.fit_lattice(train_set, K=12, members_per_q=4, steps=300)
    assert hist[-1] < hist[0], (hist[0], hist[-1])
    pr = _family(203)                                   # held out
    X, obs, y, R = dev(pr.X), dev(pr.obs_idx), dev(pr.y), dev(pr.R)
    base = B.make_options(precision=B.PRECISION_BF16)
    withm = B.make_options(precision=B.PRECISION_BF16, learned_model=theta, learned_max_shift=max_shift)
    mu0, A0, st0 = B.info_esrf_analysis(pr.grid, X, obs, y, R, pr.Q, 1e-6, base)
    mu1, A1, st1 = B.info_esrf_analysis(pr.grid, X, obs, y, R, pr.Q, 1e-6, withm)
    torch.cuda.synchronize()
    assert st0["solver_path"] == 3 and st1["solver_path"] == 3
    assert st1["status"] == 0 and st1["n_unconverged"] == 0, st1
    assert st1["learned"] == 1 and st0["learned"] == 0
    A_ref = S.perturbation_update(pr.X, pr.obs_idx, pr.R, pr.grid, pr.Q)
    mu_ref = S.mean_update(pr.X, pr.obs_idx, pr.y, pr.R, pr.grid)
    Af = pr.X - pr.X.mean(0)
    for mu_a, A_a in ((mu0, A0), (mu1, A1)):
        assert increment_error(A_a.cpu().numpy(), A_ref, Af) <= 1e-4
        assert mean_error(mu_a, mu_ref, pr.X.mean(0)) <= 1e-4
    print(f"BF16 2-D iterations mean {st0['iters_mean']:.2f} -> {st1['iters_mean']:.2f}, "
          f"max {st0['iters_max']} -> {st1['iters_max']}; loss {hist[0]:.3f} -> {hist[-1]:.3f}; "
          f"shift cut-off {max_shift:.3g}")
    if max_shift > 1.0:                                 # the plain-PCG comparison kept the term for some shifts
        assert st1["iters_mean"] < st0["iters_mean"]


def test_bad_lattice_network_falls_back_to_paper_preconditioner(B):
    """A network whose stencil ruins the conditioning hits max_iter on the BF16 path; those systems are
    solved again with P_q^-1 alone and the analysis still matches the oracle."""
    pr = _small_2d(31)
    theta = np.zeros(LR.NPARAM, dtype=np.float32)
    off_b3 = LR.NPARAM - LR.NOUT
    theta[off_b3] = -12.0                                # a = e^-12 / sigma: P^-1 contributes nothing
    theta[off_b3 + 1:off_b3 + 1 + LR.NBIN] = [4.0, -3.0, 3.0, -3.0, 3.0, -3.0]   # high-pass stencil
    X, obs, y, R = dev(pr.X), dev(pr.obs_idx), dev(pr.y), dev(pr.R)
    opts = B.make_options(precision=B.PRECISION_BF16, max_iter=150, learned_model=dev(theta))
    mu_a, A_a, st = B.info_esrf_analysis(pr.grid, X, obs, y, R, pr.Q, 1e-6, opts)
    torch.cuda.synchronize()
    assert st["solver_path"] == 3 and st["learned"] == 1
    assert st["status"] == 0 and st["n_unconverged"] == 0, st
    A_ref = S.perturbation_update(pr.X, pr.obs_idx, pr.R, pr.grid, pr.Q)
    assert increment_error(A_a.cpu().numpy(), A_ref, pr.X - pr.X.mean(0)) <= 1e-4


def test_learned_term_off_where_observations_are_not_a_lattice(B):
    """Observations at random points of a 2-D grid (no lattice), and a layered grid: the BF16 path
    leaves the learned term off and reports it (learned = -1); the capture refuses such problems."""
    theta = dev(LR.init_params(seed=3, scale=0.1).astype(np.float32))
    grid = workloads.Grid((48, 40, 1), (True, True, False), (6.0, 6.0, 1.0), True)
    pr = workloads.random_obs_problem(grid, N=10, d=300, r2=0.5, Q=5, tol=1e-6, seed=12)
    X, obs, y, R = dev(pr.X), dev(pr.obs_idx), dev(pr.y), dev(pr.R)
    opts = B.make_options(precision=B.PRECISION_BF16, learned_model=theta)
    mu_a, A_a, st = B.info_esrf_analysis(pr.grid, X, obs, y, R, pr.Q, 1e-6, opts)
    torch.cuda.synchronize()
    assert st["status"] == 0 and st["solver_path"] == 3 and st["learned"] == -1, st
    A_ref = S.perturbation_update(pr.X, pr.obs_idx, pr.R, pr.grid, pr.Q)
    assert increment_error(A_a.cpu().numpy(), A_ref, pr.X - pr.X.mean(0)) <= 1e-4
    with pytest.raises(B.InfoEsrfError) as e:
        B.krylov_capture_lattice(pr.grid, X, obs, R, pr.Q, [0, 1], 2, B.make_options(precision=B.PRECISION_BF16))
    assert e.value.code == B.ERR_UNSUPPORTED
    lay = workloads.layered_l96_problem(nx=120, nz=4, N=12, spinup=200, c_x=10.0, c_z=1.0, Q=6)
    X, obs, y, R = dev(lay.X), dev(lay.obs_idx), dev(lay.y), dev(lay.R)
    _, _, st = B.info_esrf_analysis(lay.grid, X, obs, y, R, lay.Q, 1e-6, opts)
    torch.cuda.synchronize()
    assert st["status"] == 0 and st["learned"] == -1, st
