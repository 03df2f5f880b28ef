"""The device metrics module (torch) against the oracle's error measures, on CPU
tensors: E^2 of Eq. diagonal_error_metric, the exact Kalman analysis variance,
the forecast MSE and the MSE over variance (Sec. 5.2), and relaxation to prior
spread."""
import numpy as np
import torch

from oracle import filter as F
from paper_2503_00253_gb300 import experiments, metrics


def _case(seed=31, n=40, d=9, N=12):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((n, n))
    Sxx = M @ M.T / n + 0.2 * np.eye(n)
    H = rng.standard_normal((d, n))
    R = rng.uniform(0.3, 2.0, d)
    A = rng.standard_normal((N, n))
    return Sxx, H, R, A, rng


def test_kalman_analysis_variance_matches_oracle():
    Sxx, H, R, _, _ = _case()
    Sa = metrics.kalman_analysis_variance(torch.tensor(Sxx), torch.tensor(H), torch.tensor(R)).numpy()
    ref = np.diag(F.kalman_analysis_covariance(Sxx, H, R))
    assert np.max(np.abs(Sa - ref) / ref) <= 1e-11


def test_e2_mse_and_ratio_match_oracle():
    Sxx, H, R, A, rng = _case()
    Sa = np.diag(F.kalman_analysis_covariance(Sxx, H, R))
    assert abs(metrics.variance_error_e2(torch.tensor(A), torch.tensor(Sa)) - F.variance_error_e2(A, Sa)) <= 1e-12
    mu, x = rng.standard_normal(40), rng.standard_normal(40)
    X = rng.standard_normal((12, 40))
    assert abs(metrics.forecast_mse(torch.tensor(mu), torch.tensor(x)) - F.forecast_mse(mu, x)) <= 1e-14
    assert abs(metrics.mse_over_variance(torch.tensor(mu), torch.tensor(x), torch.tensor(X))
               - F.mse_over_variance(mu, x, X)) <= 1e-12


def test_rtps_spread_per_component():
    rng = np.random.default_rng(32)
    Af = torch.tensor(rng.standard_normal((15, 7)) * 3.0)
    Aa = torch.tensor(rng.standard_normal((15, 7)))
    for alpha in (0.0, 0.01, 0.5, 1.0):
        out = experiments.rtps(Af, Aa, alpha)
        assert torch.allclose(out.std(0), alpha * Af.std(0) + (1 - alpha) * Aa.std(0), rtol=1e-12)
