"""Error measures of the paper's experiments, on the device (torch, FP64).

* Sec. 4.3, Eq. diagonal_error_metric: E^2 = mean_i ((S~_a(i,i) - S_a(i,i)) / S_a(i,i))^2,
  S~_a the empirical covariance of the analysis ensemble, S_a the exact analysis
  covariance of the Kalman filter, S_a = Sxx - Sxx H^T (H Sxx H^T + R)^-1 H Sxx.
* Sec. 5.2: forecast MSE ||mu_f - x||^2 / n, and its ratio to the forecast
  ensemble variance averaged over components (near 1 for a calibrated filter).

These evaluate results; they are not part of the analysis path.
"""
from __future__ import annotations

import torch


def kalman_analysis_variance(Sxx: torch.Tensor, H: torch.Tensor, R: torch.Tensor) -> torch.Tensor:
    """diag of S_a = Sxx - Sxx H^T (H Sxx H^T + R)^-1 H Sxx, through a Cholesky factor of
    H Sxx H^T + R (R given as its diagonal)."""
    SH = Sxx @ H.T                                   # [n][d]
    M = H @ SH + torch.diag(R)
    Lc = torch.linalg.cholesky(M)
    V = torch.linalg.solve_triangular(Lc, SH.T, upper=False)   # L^-1 H Sxx, [d][n]
    return torch.diagonal(Sxx) - (V * V).sum(dim=0)


def variance_error_e2(A_a: torch.Tensor, Sa_diag: torch.Tensor) -> float:
    """E^2 of the analysis anomalies A_a [N][n] (divisor N - 1) against the exact variances."""
    emp = (A_a * A_a).sum(dim=0) / (A_a.shape[0] - 1)
    return float((((emp - Sa_diag) / Sa_diag) ** 2).mean())


def forecast_mse(mu_f: torch.Tensor, truth: torch.Tensor) -> float:
    e = mu_f - truth
    return float((e * e).sum()) / e.numel()


def mse_over_variance(mu_f: torch.Tensor, truth: torch.Tensor, X_f: torch.Tensor) -> float:
    """Forecast MSE over the forecast ensemble variance averaged over components."""
    return forecast_mse(mu_f, truth) / float(X_f.var(dim=0, unbiased=True).mean())
