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
