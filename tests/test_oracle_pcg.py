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
