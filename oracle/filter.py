"""InFo-ESRF mean and perturbation updates, dense FP64 (oracle; test infrastructure only).

Follows the paper's formulas literally, with dense matrices and direct solves:

* Eq. normalized_perturbations: z^(i) = (x^(i) - mu) / sqrt(N - 1); W = H Z with
  H the observation subsampling operator (rows of the identity at obs_idx), or,
  in the *_H functions, a general linear operator H [d][n] (the paper's
  experiments observe weighted sums, Sec. 4.1 and Sec. 5.1).
* Eq. localized_state_covar and Sec. 2.3: Sxx = L o (Z Z^T), Sxh = Sxx H^T,
  Shh = H Sxx H^T.
* Eq. info_esrf_mean_solve: mu_a = mu + Sxh (R + Shh)^-1 (y - H mu).
* Sec. 3.2, Eq. info_esrf_perturbation_solve:
  z_a^(i) = z^(i) - Sxh sum_q p_q v_q^(i),  ((s_q + 1) R + Shh) v_q^(i) = w^(i).
  Every system is solved exactly (LU), so this is the finite-Q result the
  method converges to when every PCG solve converges.
* Eq. modified_gain / Eq. getkf: the Q -> infinity limit
  G = Sxh (R + Shh + R (I + R^-1 Shh)^(1/2))^-1 (Prop. 4).

The library returns analysis anomalies A_a = sqrt(N - 1) Z_a with members
along the leading axis, [N][n], so the analysis ensemble is mu_a + A_a.

A dense localization matrix can replace Gaspari-Cohn through ``L`` (used by
tests for the unlocalized case L = all-ones).

Error measures of the experiments: the exact Kalman analysis covariance and
E^2 of Eq. diagonal_error_metric (Sec. 4.3), the forecast MSE and the MSE over
the forecast variance (Sec. 5.2).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg

from . import localization, quadrature


def anomalies(X: np.ndarray):
    """Ensemble mean and normalized perturbations Z [n][N] (Eq. normalized_perturbations)."""
    X = np.asarray(X, dtype=np.float64)
    N = X.shape[0]
    mu = X.mean(axis=0)
    Z = (X - mu[None, :]).T / math.sqrt(N - 1)
    return mu, Z


def localized_covariances(Z, obs_idx, grid, L=None):
    """W = H Z, Sxh = (L o Z Z^T) H^T [n][d], Shh = H (L o Z Z^T) H^T [d][d]."""
    n = Z.shape[0]
    obs_idx = np.asarray(obs_idx, dtype=np.int64)
    W = Z[obs_idx, :]
    if L is None:
        L_xo = localization.localization_matrix(grid, np.arange(n), obs_idx)
    else:
        L_xo = np.asarray(L, dtype=np.float64)[:, obs_idx]
    Sxh = L_xo * (Z @ W.T)
    Shh = L_xo[obs_idx, :] * (W @ W.T)
    return W, Sxh, Shh


def normalized_obs_covariance(Shh, R):
    """C = R^-1/2 Shh R^-1/2 (Sec. 3.1, definition before Theorem 3)."""
    rih = 1.0 / np.sqrt(np.asarray(R, dtype=np.float64))
    return rih[:, None] * Shh * rih[None, :]


def choose_ell(Shh, R, ell=None):
    if ell is not None and ell > 0:
        return float(ell)
    return quadrature.ell_rule(normalized_obs_covariance(Shh, R))


def mean_update(X, obs_idx, y, R, grid, L=None):
    """mu_a = mu + Sxh (R + Shh)^-1 (y - H mu)  (Eq. info_esrf_mean_solve)."""
    mu, Z = anomalies(X)
    W, Sxh, Shh = localized_covariances(Z, obs_idx, grid, L)
    innov = np.asarray(y, dtype=np.float64) - mu[np.asarray(obs_idx)]
    v = np.linalg.solve(np.diag(R) + Shh, innov)
    return mu + Sxh @ v


def perturbation_solves(Shh, W, R, s, p):
    """vbar^(i) = sum_q p_q ((s_q + 1) R + Shh)^-1 w^(i), for all members at once."""
    vbar = np.zeros_like(W)
    Rm = np.diag(np.asarray(R, dtype=np.float64))
    for sq, pq in zip(s, p):
        vbar += pq * np.linalg.solve((sq + 1.0) * Rm + Shh, W)
    return vbar


def localized_covariances_H(Z, H, grid, L=None):
    """The same covariances for a general linear observation operator H [d][n]
    (Sec. 2.3: h linearized, model-space localization): W = H Z,
    Sxh = (L o Z Z^T) H^T [n][d], Shh = H Sxh [d][d]."""
    n = Z.shape[0]
    H = np.asarray(H, dtype=np.float64)
    if L is None:
        Lxx = localization.localization_matrix(grid, np.arange(n), np.arange(n))
    else:
        Lxx = np.asarray(L, dtype=np.float64)
    Sxh = (Lxx * (Z @ Z.T)) @ H.T
    return H @ Z, Sxh, H @ Sxh


def mean_update_H(X, H, y, R, grid, L=None):
    """Eq. info_esrf_mean_solve with a general H: mu_a = mu + Sxh (R + Shh)^-1 (y - H mu)."""
    mu, Z = anomalies(X)
    W, Sxh, Shh = localized_covariances_H(Z, H, grid, L)
    innov = np.asarray(y, dtype=np.float64) - np.asarray(H, dtype=np.float64) @ mu
    return mu + Sxh @ np.linalg.solve(np.diag(R) + Shh, innov)


def _perturbation_from(Z, W, Sxh, Shh, R, Q, ell, rule):
    """z_a^(i) = z^(i) - Sxh sum_q p_q ((s_q + 1) R + Shh)^-1 w^(i) (Sec. 3.2), exact solves."""
    ell_used = choose_ell(Shh, R, ell)
    s, p = quadrature.quadrature(Q, ell_used, rule)
    vbar = perturbation_solves(Shh, W, R, s, p)
    N = Z.shape[1]
    return math.sqrt(N - 1) * (Z - Sxh @ vbar).T


def perturbation_update_H(X, H, R, grid, Q, ell=None, rule="elliptic", L=None):
    """Analysis anomalies A_a [N][n] of Sec. 3.2 for a general linear H [d][n]."""
    mu, Z = anomalies(X)
    W, Sxh, Shh = localized_covariances_H(Z, H, grid, L)
    return _perturbation_from(Z, W, Sxh, Shh, R, Q, ell, rule)


def perturbation_update(X, obs_idx, R, grid, Q, ell=None, rule="elliptic", L=None,
                        return_info=False):
    """Analysis anomalies A_a [N][n] of Sec. 3.2 with exact solves."""
    mu, Z = anomalies(X)
    W, Sxh, Shh = localized_covariances(Z, obs_idx, grid, L)
    ell_used = choose_ell(Shh, R, ell)
    s, p = quadrature.quadrature(Q, ell_used, rule)
    vbar = perturbation_solves(Shh, W, R, s, p)
    Za = Z - Sxh @ vbar
    N = Z.shape[1]
    A = math.sqrt(N - 1) * Za.T
    if return_info:
        return A, dict(ell=ell_used, s=s, p=p, vbar=vbar, W=W, Sxh=Sxh, Shh=Shh, mu=mu, Z=Z)
    return A


def analysis(X, obs_idx, y, R, grid, Q, ell=None, rule="elliptic", L=None):
    """(mu_a, A_a): mean update and perturbation update of one cycle."""
    return (mean_update(X, obs_idx, y, R, grid, L),
            perturbation_update(X, obs_idx, R, grid, Q, ell, rule, L))


def getkf_gain(Sxh, Shh, R):
    """Modified gain G = Sxh (R + Shh + R (I + R^-1 Shh)^(1/2))^-1 (Eq. modified_gain)."""
    Rm = np.diag(np.asarray(R, dtype=np.float64))
    Rinv = np.diag(1.0 / np.asarray(R, dtype=np.float64))
    root = scipy.linalg.sqrtm(np.eye(Shh.shape[0]) + Rinv @ Shh)
    root = np.real(root)
    M = Rm + Shh + Rm @ root
    return np.linalg.solve(M.T, Sxh.T).T


def getkf_update(X, obs_idx, R, grid, L=None):
    """Q -> infinity limit of the perturbation update: z_a = z - G w (Eq. getkf)."""
    mu, Z = anomalies(X)
    W, Sxh, Shh = localized_covariances(Z, obs_idx, grid, L)
    G = getkf_gain(Sxh, Shh, R)
    N = Z.shape[1]
    return math.sqrt(N - 1) * (Z - G @ W).T


def relative_increment_error(A_test, A_ref, A_forecast):
    """||(A_test - A_f) - (A_ref - A_f)||_F / ||A_ref - A_f||_F."""
    num = np.linalg.norm(np.asarray(A_test) - np.asarray(A_ref))
    den = np.linalg.norm(np.asarray(A_ref) - np.asarray(A_forecast))
    return float(num / den) if den > 0 else float(num)


# ---------------------------------------------------------------------------
# Error measures of the experiments (Sec. 4.3, Sec. 5.2)
# ---------------------------------------------------------------------------

def kalman_analysis_covariance(Sxx, H, R):
    """Exact analysis covariance of the Kalman filter, the reference of
    Eq. diagonal_error_metric: Sxx - Sxx H^T (H Sxx H^T + R)^-1 H Sxx."""
    Sxx = np.asarray(Sxx, dtype=np.float64)
    H = np.asarray(H, dtype=np.float64)
    SH = Sxx @ H.T
    return Sxx - SH @ np.linalg.solve(H @ SH + np.diag(np.asarray(R, dtype=np.float64)), SH.T)


def variance_error_e2(A_a, Sa_diag):
    """E^2 of Eq. diagonal_error_metric: the mean over state components of the squared relative
    error of the analysis ensemble's empirical variance (anomalies A_a [N][n], divisor N - 1)
    against the exact analysis variance Sa_diag [n]."""
    A_a = np.asarray(A_a, dtype=np.float64)
    emp = (A_a ** 2).sum(axis=0) / (A_a.shape[0] - 1)
    Sa = np.asarray(Sa_diag, dtype=np.float64)
    return float(np.mean(((emp - Sa) / Sa) ** 2))


def forecast_mse(mu_f, truth):
    """Squared forecast error per component, ||mu_f - x||^2 / n (Sec. 5.2)."""
    e = np.asarray(mu_f, dtype=np.float64) - np.asarray(truth, dtype=np.float64)
    return float(e @ e) / e.size


def mse_over_variance(mu_f, truth, X_f):
    """Forecast MSE over the forecast ensemble variance averaged over components (Sec. 5.2;
    near 1 for a calibrated filter).  The printed formula omits the 1/n of the MSE; this is the
    ratio of the two per-component quantities."""
    var = float(np.mean(np.var(np.asarray(X_f, dtype=np.float64), axis=0, ddof=1)))
    return forecast_mse(mu_f, truth) / var
