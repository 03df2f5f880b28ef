"""Pins of the oracle's mean/perturbation updates against closed forms and invariants."""
import math
import types

import numpy as np
import pytest
import scipy.linalg
from scipy import integrate

from oracle import filter as F
from oracle import localization, quadrature
from paper_2503_00253_gb300 import workloads


def _small(n=48, N=9, stride=3, hw=5.0, seed=0, r2=0.5):
    return workloads.gaussian_problem_1d("t", n=n, N=N, length_scale=4.0, obs_stride=stride,
                                         r2=r2, half_width=hw, Q=16, tol=1e-12, seed=seed)


def _symmetric_etkf(X, obs_idx, R):
    """Z_a = Z (I + W^T R^-1 W)^-1/2: the unlocalized square-root update (App. C algebra)."""
    N = X.shape[0]
    mu = X.mean(0)
    Z = (X - mu).T / math.sqrt(N - 1)
    W = Z[obs_idx]
    M = np.eye(N) + W.T @ (W / R[:, None])
    lam, V = np.linalg.eigh(M)
    T = V @ np.diag(lam ** -0.5) @ V.T
    return math.sqrt(N - 1) * (Z @ T).T


def test_unlocalized_limit_is_symmetric_etkf():
    pr = _small(N=7)
    n = pr.n
    R = pr.R * (1.0 + np.linspace(0, 1, pr.d))          # non-uniform R
    A = F.perturbation_update(pr.X, pr.obs_idx, R, pr.grid, Q=48, ell=1e4, L=np.ones((n, n)))
    A_ref = _symmetric_etkf(pr.X, pr.obs_idx, R)
    Af = pr.X - pr.X.mean(0)
    assert F.relative_increment_error(A, A_ref, Af) < 1e-10


def test_unlocalized_analysis_covariance_is_kalman():
    pr = _small(N=6)
    n = pr.n
    A = F.perturbation_update(pr.X, pr.obs_idx, pr.R, pr.grid, Q=48, ell=1e4, L=np.ones((n, n)))
    N = pr.N
    Za = A.T / math.sqrt(N - 1)
    mu, Z = F.anomalies(pr.X)
    W = Z[pr.obs_idx]
    S = Z @ Z.T
    Sa = S - Z @ W.T @ np.linalg.solve(np.diag(pr.R) + W @ W.T, W @ Z.T)
    assert np.max(np.abs(Za @ Za.T - Sa)) < 1e-10 * np.max(np.abs(S))


def test_localized_quadrature_converges_to_getkf():
    pr = _small()
    Af = pr.X - pr.X.mean(0)
    ref = F.getkf_update(pr.X, pr.obs_idx, pr.R, pr.grid)
    errs = []
    for Q in (2, 4, 8, 16, 32):
        A = F.perturbation_update(pr.X, pr.obs_idx, pr.R, pr.grid, Q=Q)
        errs.append(F.relative_increment_error(A, ref, Af))
    assert all(b < a for a, b in zip(errs[:3], errs[1:4]))
    assert errs[-1] < 1e-11


def test_dense_solve_matches_eigen_form():
    """Exact same-node result two ways: direct solves vs. eigendecomposition of C (App. C)."""
    pr = _small(seed=3)
    A, info = F.perturbation_update(pr.X, pr.obs_idx, pr.R, pr.grid, Q=16, return_info=True)
    rih = 1.0 / np.sqrt(pr.R)
    C = rih[:, None] * info["Shh"] * rih[None, :]
    lam, V = np.linalg.eigh(C)
    g = (info["p"][None, :] / (info["s"][None, :] + 1.0 + lam[:, None])).sum(1)
    vbar = rih[:, None] * (V @ (g[:, None] * (V.T @ (rih[:, None] * info["W"]))))
    Za = info["Z"] - info["Sxh"] @ vbar
    A2 = math.sqrt(pr.N - 1) * Za.T
    assert np.max(np.abs(A - A2)) < 1e-12 * np.max(np.abs(A))


def test_subsampled_covariances_match_full_matrix():
    """Sxh = Sxx H^T and Shh = H Sxx H^T with the full dense Sxx (Sec. 2.3)."""
    pr = _small(n=30, stride=4)
    mu, Z = F.anomalies(pr.X)
    L = localization.localization_matrix(pr.grid, np.arange(pr.n), np.arange(pr.n))
    Sxx = L * (Z @ Z.T)
    H = np.eye(pr.n)[pr.obs_idx]
    W, Sxh, Shh = F.localized_covariances(Z, pr.obs_idx, pr.grid)
    assert np.allclose(W, H @ Z, atol=0, rtol=0)
    assert np.max(np.abs(Sxh - Sxx @ H.T)) < 1e-14
    assert np.max(np.abs(Shh - H @ Sxx @ H.T)) < 1e-14
    # the un-normalized sample covariance is Z Z^T with Z scaled by sqrt(N-1) (Sec. 2.3)
    Xa = pr.X - pr.X.mean(0)
    assert np.max(np.abs(Z @ Z.T - Xa.T @ Xa / (pr.N - 1))) < 1e-13


def test_localized_adjustment_identity():
    """(I - G H) Sxx (I - G H)^T = Sxx - Sxh (R + Shh)^-1 Sxh^T (App. B, Eq. adjustment_integral_form)."""
    pr = _small(n=36, stride=3, seed=5)
    mu, Z = F.anomalies(pr.X)
    L = localization.localization_matrix(pr.grid, np.arange(pr.n), np.arange(pr.n))
    Sxx = L * (Z @ Z.T)
    H = np.eye(pr.n)[pr.obs_idx]
    W, Sxh, Shh = F.localized_covariances(Z, pr.obs_idx, pr.grid)
    s, p = quadrature.elliptic_rule(48, F.choose_ell(Shh, pr.R))
    # G = sum_q p_q K(s_q) with K(s) = Sxh ((s+1) R + Shh)^-1 (Eq. inflated_kalman_gain)
    G = sum(pq * np.linalg.solve(((sq + 1.0) * np.diag(pr.R) + Shh).T, Sxh.T).T
            for sq, pq in zip(s, p))
    Ax = np.eye(pr.n) - G @ H
    lhs = Ax @ Sxx @ Ax.T
    rhs = Sxx - Sxh @ np.linalg.solve(np.diag(pr.R) + Shh, Sxh.T)
    assert np.max(np.abs(lhs - rhs)) < 1e-10 * np.max(np.abs(Sxx))


def test_zero_mean_analysis_perturbations():
    pr = _small(seed=7)
    A = F.perturbation_update(pr.X, pr.obs_idx, pr.R, pr.grid, Q=8)
    assert np.max(np.abs(A.sum(0))) < 1e-12 * np.max(np.abs(A))


def test_scalar_case_closed_form():
    """n = d = 1: z_a = z - G w with G = s_xh / (R + s_hh + R sqrt(1 + s_hh / R))."""
    rng = np.random.default_rng(11)
    X = rng.standard_normal((15, 1)) * 3.0
    grid = types.SimpleNamespace(shape=(1, 1, 1), periodic=(False, False, False),
                                 half_width=(1.0, 1.0, 1.0), chordal=True)
    R = np.array([0.7])
    A = F.perturbation_update(X, np.array([0]), R, grid, Q=40, ell=1e4)
    mu, Z = F.anomalies(X)
    s2 = float(Z[0] @ Z[0])
    G = quadrature.scalar_gain(s2, s2, 0.7)
    ref = math.sqrt(14) * (Z[0] - G * Z[0])
    assert np.max(np.abs(A[:, 0] - ref)) < 1e-13 * np.max(np.abs(ref))


def test_theorem2_integral_brute_force():
    """Z_a = Z - int_0^inf p(s) K(s) W ds (Theorem 2) by adaptive quadrature, tiny case."""
    pr = _small(n=12, N=5, stride=4, hw=3.0, seed=2)
    mu, Z = F.anomalies(pr.X)
    W, Sxh, Shh = F.localized_covariances(Z, pr.obs_idx, pr.grid)
    Rm = np.diag(pr.R)

    def integrand(t):   # s = t^2, p(s) ds = 2 dt / (pi (t^2 + 1))
        s = t * t
        K = np.linalg.solve(((s + 1.0) * Rm + Shh).T, Sxh.T).T
        return (2.0 / (math.pi * (s + 1.0))) * (K @ W)

    val, _ = integrate.quad_vec(integrand, 0.0, np.inf, epsabs=1e-13, epsrel=1e-12)
    A_int = math.sqrt(pr.N - 1) * (Z - val).T
    A = F.getkf_update(pr.X, pr.obs_idx, pr.R, pr.grid)
    assert np.max(np.abs(A - A_int)) < 1e-9 * np.max(np.abs(A))


def test_mean_update_information_form():
    """mu_a from the gain form equals the information form (Sigma^-1 + H^T R^-1 H)^-1 (N > n)."""
    pr = _small(n=10, N=25, stride=2, hw=4.0, seed=4)
    mu, Z = F.anomalies(pr.X)
    L = localization.localization_matrix(pr.grid, np.arange(pr.n), np.arange(pr.n))
    Sxx = L * (Z @ Z.T)
    H = np.eye(pr.n)[pr.obs_idx]
    Rinv = np.diag(1.0 / pr.R)
    Sa = np.linalg.inv(np.linalg.inv(Sxx) + H.T @ Rinv @ H)
    mu_info = mu + Sa @ H.T @ Rinv @ (pr.y - H @ mu)
    mu_a = F.mean_update(pr.X, pr.obs_idx, pr.y, pr.R, pr.grid)
    assert np.max(np.abs(mu_a - mu_info)) < 1e-9 * np.max(np.abs(mu_info - mu))


def test_getkf_gain_matches_eigen_f2():
    """G = Sxh R^-1/2 Q f2(Lambda) Q^T R^-1/2 with f2(x) = 1/(1+x+sqrt(1+x)) (App. C)."""
    pr = _small(seed=9)
    mu, Z = F.anomalies(pr.X)
    W, Sxh, Shh = F.localized_covariances(Z, pr.obs_idx, pr.grid)
    G = F.getkf_gain(Sxh, Shh, pr.R)
    rih = 1.0 / np.sqrt(pr.R)
    lam, V = np.linalg.eigh(rih[:, None] * Shh * rih[None, :])
    f2 = 1.0 / (1.0 + lam + np.sqrt(1.0 + lam))
    G2 = Sxh @ (rih[:, None] * (V @ np.diag(f2) @ V.T) * rih[None, :])
    assert np.max(np.abs(G - G2)) < 1e-12 * np.max(np.abs(G))


# ---------------------------------------------------------------------------
# General linear observation operators (Sec. 2.3 with h linearized; the
# paper's experiments observe weighted sums, Sec. 4.1 and Sec. 5.1)
# ---------------------------------------------------------------------------

def test_general_H_selection_matches_subsampling():
    """H = rows of the identity at obs_idx gives the subsampling path's results."""
    pr = _small(n=60, N=8, stride=3, hw=6.0, seed=5)
    H = np.eye(pr.n)[pr.obs_idx]
    A = F.perturbation_update_H(pr.X, H, pr.R, pr.grid, Q=12)
    A_ref = F.perturbation_update(pr.X, pr.obs_idx, pr.R, pr.grid, Q=12)
    Af = pr.X - pr.X.mean(0)
    assert F.relative_increment_error(A, A_ref, Af) < 1e-12
    mu = F.mean_update_H(pr.X, H, pr.y, pr.R, pr.grid)
    mu_ref = F.mean_update(pr.X, pr.obs_idx, pr.y, pr.R, pr.grid)
    assert np.max(np.abs(mu - mu_ref)) < 1e-12 * np.max(np.abs(mu_ref))


def test_general_H_unlocalized_analysis_covariance_is_kalman():
    """Weighted-sum observations, no localization, many nodes: Z_a Z_a^T is the
    Kalman analysis covariance S - S H^T (R + H S H^T)^-1 H S with S = Z Z^T."""
    pr = _small(n=60, N=7, seed=6)
    H, _ = workloads.gaussian_channel_operator(pr.n, 12, 3.0)
    R = 0.3 * (1.0 + np.linspace(0, 1, 12))
    A = F.perturbation_update_H(pr.X, H, R, pr.grid, Q=48, ell=1e4, L=np.ones((pr.n, pr.n)))
    Za = A.T / math.sqrt(pr.N - 1)
    mu, Z = F.anomalies(pr.X)
    S = Z @ Z.T
    Sa = S - S @ H.T @ np.linalg.solve(np.diag(R) + H @ S @ H.T, H @ S)
    assert np.max(np.abs(Za @ Za.T - Sa)) < 1e-10 * np.max(np.abs(S))


def test_general_H_mean_update_information_form():
    """mu_a with a weighted-sum H equals (Sxx^-1 + H^T R^-1 H)^-1 applied as in the
    information form (N > n so that the localized Sxx is invertible)."""
    pr = _small(n=10, N=25, stride=2, hw=4.0, seed=7)
    H, _ = workloads.gaussian_channel_operator(pr.n, 4, 1.5)
    rng = np.random.default_rng(8)
    y = rng.standard_normal(4)
    R = np.full(4, 0.4)
    mu, Z = F.anomalies(pr.X)
    L = localization.localization_matrix(pr.grid, np.arange(pr.n), np.arange(pr.n))
    Sxx = L * (Z @ Z.T)
    Rinv = np.diag(1.0 / R)
    Sa = np.linalg.inv(np.linalg.inv(Sxx) + H.T @ Rinv @ H)
    mu_info = mu + Sa @ H.T @ Rinv @ (y - H @ mu)
    mu_a = F.mean_update_H(pr.X, H, y, R, pr.grid)
    assert np.max(np.abs(mu_a - mu_info)) < 1e-9 * np.max(np.abs(mu_info - mu))


def test_weighted_sum_operators_follow_the_paper_forms():
    """Channel weights peak at 1 on their centre and decay as the Gaussian of the
    chordal distance; column-sum weights have unit 2-norm per channel."""
    H, (rp, col, val) = workloads.gaussian_channel_operator(200, 10, 4.0)
    assert np.allclose(H[np.arange(10), (np.arange(10) * 200) // 10], 1.0)
    c = (200 / math.pi) * math.sin(math.pi * 3 / 200)
    assert abs(H[0, 3] - math.exp(-c * c / 32.0)) < 1e-15
    assert np.array_equal(np.diff(rp), (H != 0).sum(1))
    H2, _ = workloads.column_sum_operator((8, 1, 12), [1, 5], 3, 4.0, 2.0)
    assert np.allclose((H2 ** 2).sum(1), 1.0)
    assert np.all(H2.reshape(6, 12, 8)[:, :, [0, 2, 3, 4, 6, 7]] == 0.0)


# ---------------------------------------------------------------------------
# Error measures of the experiments (Sec. 4.3, Sec. 5.2)
# ---------------------------------------------------------------------------

def test_kalman_analysis_covariance_equals_information_form():
    rng = np.random.default_rng(21)
    n, d = 30, 8
    M = rng.standard_normal((n, n))
    Sxx = M @ M.T / n + 0.1 * np.eye(n)
    H = rng.standard_normal((d, n))
    R = rng.uniform(0.2, 2.0, d)
    Sa = F.kalman_analysis_covariance(Sxx, H, R)
    info = np.linalg.inv(np.linalg.inv(Sxx) + H.T @ np.diag(1.0 / R) @ H)
    assert np.max(np.abs(Sa - info)) <= 1e-10 * np.max(np.abs(info))


def test_variance_error_e2_closed_forms():
    """E^2 = 0 when the empirical variances are exact, and 1 when they are twice
    the reference (each term ((2 s - s) / s)^2 = 1)."""
    rng = np.random.default_rng(22)
    A = rng.standard_normal((12, 50))
    emp = (A ** 2).sum(0) / 11
    assert F.variance_error_e2(A, emp) <= 1e-28
    assert abs(F.variance_error_e2(A, emp / 2.0) - 1.0) <= 1e-12
    assert abs(F.variance_error_e2(A, emp * 2.0) - 0.25) <= 1e-12


def test_forecast_mse_and_ratio():
    truth = np.array([1.0, 2.0, 3.0, 4.0])
    mu = np.array([1.0, 0.0, 3.0, 6.0])
    assert F.forecast_mse(mu, truth) == 2.0
    Xf = np.array([[0.0, 0.0, 0.0, 0.0], [2.0, 2.0, 2.0, 2.0]])   # variance 2 per component
    assert F.mse_over_variance(mu, truth, Xf) == 1.0


def test_single_cycle_observation_error_matches_the_paper():
    """Sec. 4.1 (Eq. single_cycle_obserr_covar) prints r^2 ~ 36.3 as one tenth of the observable
    variance under Eq. single_cycle_covar and Eq. single_cycle_obsop: the generator's covariance
    and channels reproduce it."""
    tr = workloads.single_cycle_trial(0)
    assert abs(tr["r2"] - 36.3) < 0.05, tr["r2"]
    assert tr["H"].shape == (100, 2000) and tr["X"].shape == (20, 2000)
