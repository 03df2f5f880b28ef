"""The single-cycle experiment (Sec. 4) through the library.

Each trial draws N = 20 forecast members and a truth from the Gaussian forecast
covariance of Sec. 4.1, observes 100 Gaussian-weighted channel sums, runs one
analysis with a fixed number of PCG iterations (the paper uses 2), and scores
the analysis ensemble with E^2 against the exact Kalman analysis variances.
The library localizes with Gaspari-Cohn; the paper's Gaussian taper of length
12 is replaced by the Gaspari-Cohn function of matching half-width
(workloads.single_cycle_trial).
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import binding as B
from . import metrics, workloads


def single_cycle_e2(trials: int = 10, Q: int = 8, ritz_rank: int = 10, iters: int = 2,
                    precision: int = B.PRECISION_FP64, solver: int = B.SOLVER_PCG, seed: int = 1000,
                    device: str = "cuda") -> dict:
    """Mean E^2 over ``trials`` analyses, and the device time per analysis (ms)."""
    Sxx = workloads.single_cycle_covariance()
    Sxx_t = torch.tensor(Sxx, device=device)
    e2, ms = [], []
    Sa, r2 = None, None
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for t in range(trials):
        tr = workloads.single_cycle_trial(t, Q=Q, Sxx=Sxx, seed=seed, r2=r2)
        r2 = tr["r2"]
        rowptr, col, val = tr["csr"]
        H = torch.tensor(tr["H"], device=device)
        R = torch.tensor(tr["R"], device=device)
        if Sa is None:   # the covariance model, H and R are the same in every trial
            Sa = metrics.kalman_analysis_variance(Sxx_t, H, R)
        prob = dict(grid=tr["grid"], X=torch.tensor(tr["X"], device=device),
                    H=(torch.tensor(rowptr, device=device), torch.tensor(col, device=device),
                       torch.tensor(val, device=device)),
                    y=torch.tensor(tr["y"], device=device), R=R, Q=Q, tol=tr["tol"])
        opts = B.make_options(precision=precision, ritz_rank=ritz_rank, fixed_iters=iters, solver=solver)
        ev0.record()
        outs, _ = B.info_esrf_analysis_batched([prob], opts, stats=False)
        ev1.record()
        ev1.synchronize()
        ms.append(ev0.elapsed_time(ev1))
        e2.append(metrics.variance_error_e2(outs[0][1], Sa))
    return dict(trials=trials, Q=Q, ritz_rank=ritz_rank, iters=iters, e2_mean=float(np.mean(e2)),
                e2_std=float(np.std(e2)), ms_median=float(np.median(ms)))


def rtps(A_f: torch.Tensor, A_a: torch.Tensor, alpha: float) -> torch.Tensor:
    """Relaxation to prior spread (Whitaker & Hamill 2012; Sec. 5.2 uses alpha = 0.01): each state
    component's analysis anomalies are scaled so that its spread becomes
    alpha sigma_f + (1 - alpha) sigma_a."""
    sf = A_f.std(dim=0, unbiased=True)
    sa = A_a.std(dim=0, unbiased=True)
    scale = 1.0 + alpha * (sf - sa) / torch.clamp(sa, min=1e-300)
    return A_a * scale[None, :]


def cycled_l96(cycles: int = 200, burn_in: int = 50, Q: int = 24, ritz_rank: int = 10, iters: int = 10,
               precision: int = B.PRECISION_FP32, solver: int = B.SOLVER_PCG, alpha: float = 0.01,
               nx: int = 960, nz: int = 8, N: int = 40, spinup: int = 2000, dt: float = 0.01,
               steps_per_cycle: int = 5, seed: int = 3, device: str = "cuda") -> dict:
    """Cycled assimilation on the layered Lorenz-96 model (Sec. 5): N members and the truth from
    perturbed spin-ups, 25% random point observations every 5 RK4 steps of 0.01 (Delta t = 0.05),
    analyses with a fixed number of Krylov iterations, relaxation to prior spread.  Returns the
    averages over the cycles after burn_in of the forecast MSE and of the forecast MSE over the
    forecast variance (Sec. 5.2), and the median device time of one analysis (ms)."""
    pr = workloads.layered_l96_problem(nx=nx, nz=nz, N=N, spinup=spinup, dt=dt, Q=Q, seed=seed)
    n = nx * nz
    rng = np.random.default_rng(seed + 1)
    X = pr.X.reshape(N, nz, nx).copy()
    truth = pr.truth.reshape(nz, nx).copy()
    obs = torch.tensor(pr.obs_idx, device=device)
    R = torch.tensor(pr.R, device=device)
    opts = B.make_options(precision=precision, ritz_rank=ritz_rank, fixed_iters=iters, solver=solver)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    mse, ratio, ms = [], [], []
    for c in range(cycles):
        if c > 0:
            X = workloads.ll96_rk4(X, dt, steps_per_cycle)
            truth = workloads.ll96_rk4(truth[None], dt, steps_per_cycle)[0]
        Xf = torch.tensor(X.reshape(N, n), device=device)
        xt = torch.tensor(truth.reshape(n), device=device)
        if c >= burn_in:
            mu_f = Xf.mean(dim=0)
            mse.append(metrics.forecast_mse(mu_f, xt))
            ratio.append(metrics.mse_over_variance(mu_f, xt, Xf))
        y = xt[obs] + torch.sqrt(R) * torch.tensor(rng.standard_normal(obs.numel()), device=device)
        ev0.record()
        mu_a, A_a, _ = B.info_esrf_analysis(pr.grid, Xf, obs, y, R, Q, pr.tol, opts, stats=False)
        ev1.record()
        ev1.synchronize()
        ms.append(ev0.elapsed_time(ev1))
        A_a = rtps(Xf - Xf.mean(dim=0), A_a, alpha)
        X = (mu_a[None, :] + A_a).cpu().numpy().reshape(N, nz, nx)
    return dict(cycles=cycles, burn_in=burn_in, Q=Q, ritz_rank=ritz_rank, iters=iters, alpha=alpha,
                forecast_mse=float(np.mean(mse)) if mse else None,
                mse_over_variance=float(np.mean(ratio)) if ratio else None,
                analysis_ms_median=float(np.median(ms)),
                climatological_variance=float(np.var(pr.truth)))
