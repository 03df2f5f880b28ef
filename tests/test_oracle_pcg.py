"""Pins of the oracle's PCG, limited-memory preconditioner and randomized Ritz pairs (App. E)."""
import numpy as np
import pytest

from oracle import filter as F
from oracle import pcg, philox, quadrature
from paper_2503_00253_gb300 import workloads


def _C(seed=0, n=120, N=10, stride=2, hw=8.0):
    pr = workloads.gaussian_problem_1d("t", n=n, N=N, length_scale=6.0, obs_stride=stride,
                                       r2=0.3, half_width=hw, Q=8, tol=1e-12, seed=seed)
    mu, Z = F.anomalies(pr.X)
    W, Sxh, Shh = F.localized_covariances(Z, pr.obs_idx, pr.grid)
    return pr, W, F.normalized_obs_covariance(Shh, pr.R)


def test_pcg_matches_dense_solve():
    pr, W, C = _C()
    A = 1.3 * np.eye(C.shape[0]) + C
    b = W[:, 0] / np.sqrt(pr.R)
    x, it = pcg.pcg(lambda v: A @ v, b, lambda r: r, tol=1e-13, max_iter=500)
    assert np.linalg.norm(x - np.linalg.solve(A, b)) < 1e-11 * np.linalg.norm(x)
    assert 0 < it < C.shape[0]


def test_lmp_maps_ritz_vectors_to_beta():
    """P^-1 C_q Phi = beta Phi whenever Phi^T C_q Phi = Theta (App. E, Tshimanga LMP)."""
    pr, W, C = _C(seed=1)
    d = C.shape[0]
    Om = philox.test_matrix(d, 18, seed=77)
    Phi, theta = pcg.randomized_ritz(C, 8, Om)
    sigma = 2.5
    Chat = sigma * np.eye(d) + C
    beta = sigma + np.min(np.diag(C))
    Pinv = pcg.lmp_matrix(Chat, Phi, theta + sigma, beta)
    assert np.max(np.abs(Pinv @ Chat @ Phi - beta * Phi)) < 1e-10
    assert np.max(np.abs(Phi.T @ Chat @ Phi - np.diag(theta + sigma))) < 1e-10
    # the vector form agrees with the dense operator
    r = np.sin(np.arange(d))
    z = pcg.lmp_apply(r, Chat @ Phi, Phi, theta + sigma, beta)
    assert np.max(np.abs(z - Pinv @ r)) < 1e-12 * np.max(np.abs(z))
    # symmetric positive definite
    assert np.max(np.abs(Pinv - Pinv.T)) < 1e-10
    assert np.linalg.eigvalsh(0.5 * (Pinv + Pinv.T)).min() > 0


def test_lmp_spectrum_with_exact_eigenpairs():
    """With exact eigenpairs, spec(P^-1 C_q) = {beta}^k u {remaining eigenvalues of C_q}."""
    pr, W, C = _C(seed=2, n=80)
    d = C.shape[0]
    lam, V = np.linalg.eigh(C)
    k = 5
    Phi, theta = V[:, -k:], lam[-k:]
    sigma = 1.0
    Chat = sigma * np.eye(d) + C
    beta = sigma + np.min(np.diag(C))
    ev = np.sort(np.linalg.eigvals(pcg.lmp_matrix(Chat, Phi, theta + sigma, beta) @ Chat).real)
    expect = np.sort(np.concatenate([np.full(k, beta), lam[:-k] + sigma]))
    assert np.max(np.abs(ev - expect)) < 1e-9 * expect.max()
    # beta lies inside [lambda_min, lambda_max] of C_q
    assert lam[0] + sigma <= beta <= lam[-1] + sigma


def test_randomized_ritz_approximates_top_eigenvalues():
    pr, W, C = _C(seed=3, n=400, stride=2)
    d = C.shape[0]
    Om = philox.test_matrix(d, 20, seed=5)
    Phi, theta = pcg.randomized_ritz(C, 10, Om)
    lam = np.sort(np.linalg.eigvalsh(C))[::-1][:10]
    assert np.all(np.abs(theta - lam) <= 0.05 * lam[0])
    assert np.all(theta <= lam + 1e-9 * lam[0])          # Ritz values interlace from below
    assert np.max(np.abs(Phi.T @ Phi - np.eye(10))) < 1e-12


def test_pcg_lmp_same_answer_fewer_iterations():
    pr, W, C = _C(seed=4, n=300)
    ell = quadrature.ell_rule(C)
    s, p = quadrature.elliptic_rule(6, ell)
    Shh = np.sqrt(pr.R)[:, None] * C * np.sqrt(pr.R)[None, :]
    ref = F.perturbation_solves(Shh, W, pr.R, s, p)
    Om = philox.test_matrix(C.shape[0], 20, seed=1)
    v0, it0 = pcg.solve_normalized(C, s, p, W, pr.R, k=0, tol=1e-12)
    v1, it1 = pcg.solve_normalized(C, s, p, W, pr.R, k=10, Omega=Om, tol=1e-12)
    for v in (v0, v1):
        assert np.max(np.abs(v - ref)) < 1e-9 * np.max(np.abs(ref))
    assert it1.sum() < it0.sum()


# ---------------------------------------------------------------------------
# Multi-shift CG (Sec. 3.3, shift invariance of Krylov subspaces)
# ---------------------------------------------------------------------------

def _krylov_galerkin(A, b, sigma, k):
    """Definition of the k-th CG iterate for A + sigma I: the Galerkin
    projection onto K_k(A, b) = span{b, A b, ..., A^(k-1) b} (the space does
    not depend on sigma), from an orthonormal basis built column by column."""
    V = np.zeros((b.shape[0], k))
    v = b / np.linalg.norm(b)
    for j in range(k):
        for _ in range(2):                       # Gram-Schmidt twice
            v = v - V[:, :j] @ (V[:, :j].T @ v)
        V[:, j] = v / np.linalg.norm(v)
        v = A @ V[:, j]
    M = V.T @ (A + sigma * np.eye(A.shape[0])) @ V
    return V @ np.linalg.solve(M, V.T @ b)


def test_multishift_iterates_are_galerkin_projections():
    """After k iterations every shifted iterate is the CG (Galerkin) iterate of
    its own system in K_k: this fixes zeta, alpha^(q) and beta^(q) at every step."""
    rng = np.random.default_rng(3)
    d = 14
    Qm, _ = np.linalg.qr(rng.standard_normal((d, d)))
    lam = np.geomspace(0.02, 30.0, d)
    A = (Qm * lam) @ Qm.T
    b = rng.standard_normal(d)
    shifts = np.array([0.7, 0.9, 2.5, 40.0, 900.0])
    for k in range(1, 9):
        X, it, _ = pcg.multishift_cg(lambda v: A @ v, b, shifts, fixed_iters=k)
        for q, sg in enumerate(shifts):
            ref = _krylov_galerkin(A, b, sg, k)
            assert np.linalg.norm(X[q] - ref) <= 1e-9 * np.linalg.norm(ref), (k, q)
        assert np.all(it[:3] == k)


def test_multishift_base_shift_is_plain_cg():
    """With one shift, the run is textbook CG on A + sigma I (Golub & Van Loan
    Alg. 11.5.1 without preconditioner), iterate for iterate."""
    pr, W, C = _C(seed=4)
    b = W[:, 1] / np.sqrt(pr.R)
    for k in (1, 3, 7):
        X, it, _ = pcg.multishift_cg(lambda v: C @ v, b, [1.7], fixed_iters=k)
        x, kk = pcg.pcg(lambda v: 1.7 * v + C @ v, b, lambda r: r, fixed_iters=k)
        assert kk == k and it[0] == k
        assert np.linalg.norm(X[0] - x) <= 1e-13 * np.linalg.norm(x)


def test_multishift_converges_to_dense_solves_for_every_shift():
    """Each shifted solution meets its tolerance against a dense solve, including
    the shifts that stopped early; larger shifts need fewer iterations."""
    pr, W, C = _C(seed=5)
    d = C.shape[0]
    s, _ = quadrature.elliptic_rule(16, 100.0)
    shifts = s + 1.0
    b = W[:, 2] / np.sqrt(pr.R)
    X, it, rel = pcg.multishift_cg(lambda v: C @ v, b, shifts, tol=1e-12)
    for q, sg in enumerate(shifts):
        A = C + sg * np.eye(d)
        assert np.linalg.norm(b - A @ X[q]) <= 5e-12 * np.linalg.norm(b), q
        assert rel[q] <= 1e-12
    assert np.all(np.diff(it) <= 0) and it[-1] < it[0]


def test_multishift_quadrature_sum_matches_exact_perturbation_solves():
    """vbar from one multi-shift run per member equals the same-node result of
    Sec. 3.2 (exact solves) to the CG tolerance."""
    pr, W, C = _C(seed=6)
    s, p = quadrature.elliptic_rule(12, quadrature.ell_rule(C))
    mu, Z = F.anomalies(pr.X)
    _, _, Shh = F.localized_covariances(Z, pr.obs_idx, pr.grid)
    ref = F.perturbation_solves(Shh, W, pr.R, s, p)
    vbar, iters = pcg.solve_normalized_multishift(C, s, p, W, pr.R, tol=1e-13)
    assert np.linalg.norm(vbar - ref) <= 1e-10 * np.linalg.norm(ref)
    assert iters.shape == (12, W.shape[1]) and iters.max() < C.shape[0]


def test_multishift_zero_rhs():
    X, it, rel = pcg.multishift_cg(lambda v: v, np.zeros(5), [1.0, 2.0], tol=1e-10)
    assert not X.any() and not it.any() and not rel.any()


# ---------------------------------------------------------------------------
# Block CG (Sec. 3.3, second alternative)
# ---------------------------------------------------------------------------

def _block_galerkin(A, B, k):
    """Definition of the k-th block CG iterate: the A-orthogonal (Galerkin)
    projection of every column onto span{B, A B, ..., A^(k-1) B}, from an
    orthonormal basis built block by block."""
    V = np.zeros((B.shape[0], 0))
    blk = B.copy()
    for _ in range(k):
        for _ in range(2):
            blk = blk - V @ (V.T @ blk)
        Qb, _ = np.linalg.qr(blk)
        V = np.hstack([V, Qb])
        blk = A @ Qb
    return V @ np.linalg.solve(V.T @ A @ V, V.T @ B)


def test_block_cg_iterates_are_block_galerkin_projections():
    rng = np.random.default_rng(7)
    d, s = 24, 3
    Qm, _ = np.linalg.qr(rng.standard_normal((d, d)))
    A = (Qm * np.geomspace(0.05, 40.0, d)) @ Qm.T
    B = rng.standard_normal((d, s))
    for k in range(1, 6):
        X, it = pcg.block_cg(lambda V: A @ V, B, fixed_iters=k)
        ref = _block_galerkin(A, B, k)
        assert it == k
        assert np.linalg.norm(X - ref) <= 1e-9 * np.linalg.norm(ref), k


def test_block_cg_single_column_is_plain_cg():
    pr, W, C = _C(seed=8)
    b = W[:, 0] / np.sqrt(pr.R)
    A = 1.4 * np.eye(C.shape[0]) + C
    for k in (1, 4, 9):
        X, it = pcg.block_cg(lambda V: A @ V, b[:, None], fixed_iters=k)
        x, kk = pcg.pcg(lambda v: A @ v, b, lambda r: r, fixed_iters=k)
        assert np.linalg.norm(X[:, 0] - x) <= 1e-12 * np.linalg.norm(x)


def test_block_cg_matches_dense_and_needs_fewer_iterations_than_cg():
    """Every member meets the tolerance against a dense solve, and the block
    run needs fewer iterations than the slowest single-member CG run."""
    pr, W, C = _C(seed=9)
    A = 1.2 * np.eye(C.shape[0]) + C
    B = W / np.sqrt(pr.R)[:, None]
    X, it = pcg.block_cg(lambda V: A @ V, B, tol=1e-10)
    assert np.linalg.norm(X - np.linalg.solve(A, B)) <= 1e-8 * np.linalg.norm(X)
    single = max(pcg.pcg(lambda v: A @ v, B[:, i], lambda r: r, tol=1e-10)[1] for i in range(B.shape[1]))
    assert it < single, (it, single)


def test_block_cg_quadrature_sum_matches_exact_perturbation_solves():
    pr, W, C = _C(seed=10)
    s, p = quadrature.elliptic_rule(8, quadrature.ell_rule(C))
    mu, Z = F.anomalies(pr.X)
    _, _, Shh = F.localized_covariances(Z, pr.obs_idx, pr.grid)
    ref = F.perturbation_solves(Shh, W, pr.R, s, p)
    vbar, iters = pcg.solve_normalized_block(C, s, p, W, pr.R, tol=1e-12)
    assert np.linalg.norm(vbar - ref) <= 1e-9 * np.linalg.norm(ref)
    assert iters.shape == (8,) and np.all(np.diff(iters) <= 0)
