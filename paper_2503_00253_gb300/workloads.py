"""Seeded synthetic inputs shaped like the paper's experiments.

This module only draws inputs: forecast ensembles, truths, observation
patterns and observation values.  It holds none of the filter's arithmetic
(no localization, no quadrature, no solves), so that both the CUDA path and
the FP64 oracle can take their inputs from here without sharing any of the
method.

Forecast ensembles follow Sec. 4.1 (Eq. single_cycle_covar): independent
draws from N(0, Sigma) with Sigma(i,j) = variance * exp(-c(i,j)^2 / (2 nu^2))
+ eta * delta_ij and c the chordal distance on a circle of circumference n.
That covariance is circulant (block-circulant with circulant blocks in 2-D,
where it is the product of two 1-D chordal kernels), so draws are exact via
the FFT: x = F^-1 diag(sqrt(lambda)) F xi with xi white noise.  The truth is
one more independent draw (Sec. 4.3).  The layered Lorenz-96 model is
Eq. ll96_ode of Sec. 5.1, integrated with classical RK4.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np


@dataclasses.dataclass
class Grid:
    """Regular grid; flat index = (z * ny + y) * nx + x.

    ``half_width`` is the Gaspari-Cohn half-width c per axis (support 2c) in
    grid units; axes of extent 1 are ignored.  ``chordal`` selects the chordal
    distance (n/pi) sin(pi |i-j| / n) on periodic axes (the paper's choice,
    Sec. 4.1 and Sec. 5.2); otherwise the minimum-image distance is used.
    """

    shape: Sequence[int]                 # (nx, ny, nz)
    periodic: Sequence[bool] = (True, True, False)
    half_width: Sequence[float] = (1.0, 1.0, 1.0)
    chordal: bool = True

    @property
    def n(self) -> int:
        return int(np.prod(self.shape))

    def coords(self, idx: np.ndarray) -> np.ndarray:
        nx, ny, nz = (int(s) for s in self.shape)
        idx = np.asarray(idx, dtype=np.int64)
        x = idx % nx
        y = (idx // nx) % ny
        z = idx // (nx * ny)
        return np.stack([x, y, z], axis=-1)


@dataclasses.dataclass
class Problem:
    """One data-assimilation problem: ensemble, observations and settings."""

    name: str
    grid: Grid
    X: np.ndarray            # [N][n] forecast ensemble, float64
    truth: np.ndarray        # [n]
    obs_idx: np.ndarray      # [d] sorted unique int64
    y: np.ndarray            # [d] observed values
    R: np.ndarray            # [d] observation-error variances (diagonal of R)
    Q: int                   # quadrature size
    tol: float               # PCG relative tolerance
    ell: float = 0.0         # <= 0: estimated from the data
    ritz_rank: int = 10

    @property
    def N(self) -> int:
        return self.X.shape[0]

    @property
    def n(self) -> int:
        return self.X.shape[1]

    @property
    def d(self) -> int:
        return self.obs_idx.shape[0]


def _chordal(delta: np.ndarray, n: int) -> np.ndarray:
    return (n / math.pi) * np.sin(math.pi * np.abs(delta) / n)


def gaussian_ensemble_1d(n: int, members: int, length_scale: float, variance: float,
                         nugget: float, rng: np.random.Generator) -> np.ndarray:
    """``members`` exact draws [members][n] from the chordal Gaussian covariance."""
    lag = np.arange(n)
    row = variance * np.exp(-_chordal(lag, n) ** 2 / (2.0 * length_scale ** 2))
    row[0] += nugget
    lam = np.clip(np.fft.fft(row).real, 0.0, None)
    xi = rng.standard_normal((members, n))
    return np.fft.ifft(np.sqrt(lam)[None, :] * np.fft.fft(xi, axis=1), axis=1).real


def gaussian_ensemble_2d(nx: int, ny: int, members: int, length_scale: float,
                         variance: float, nugget: float,
                         rng: np.random.Generator) -> np.ndarray:
    """Exact draws [members][ny*nx] (row-major, x fastest) on a 2-D torus."""
    cx = _chordal(np.arange(nx), nx)
    cy = _chordal(np.arange(ny), ny)
    row = variance * np.exp(-(cy[:, None] ** 2 + cx[None, :] ** 2) / (2.0 * length_scale ** 2))
    row[0, 0] += nugget
    lam = np.clip(np.fft.fft2(row).real, 0.0, None)
    out = np.empty((members, ny * nx))
    for k in range(members):  # one member at a time keeps memory bounded
        xi = rng.standard_normal((ny, nx))
        out[k] = np.fft.ifft2(np.sqrt(lam) * np.fft.fft2(xi)).real.reshape(-1)
    return out


def _observe(truth: np.ndarray, obs_idx: np.ndarray, r2: float,
             rng: np.random.Generator):
    R = np.full(obs_idx.shape[0], float(r2))
    y = truth[obs_idx] + math.sqrt(r2) * rng.standard_normal(obs_idx.shape[0])
    return y, R


def gaussian_problem_1d(name: str, n: int, N: int, length_scale: float, obs_stride: int,
                        r2: float, half_width: float, Q: int, tol: float, seed: int,
                        variance: float = 1.0, nugget: float = 1e-4,
                        obs_offset: int = 0, ritz_rank: int = 10,
                        chordal: bool = True) -> Problem:
    rng = np.random.default_rng(seed)
    draws = gaussian_ensemble_1d(n, N + 1, length_scale, variance, nugget, rng)
    X, truth = draws[:N].copy(), draws[N].copy()
    obs_idx = np.arange(obs_offset % obs_stride, n, obs_stride, dtype=np.int64)
    y, R = _observe(truth, obs_idx, r2, rng)
    grid = Grid((n, 1, 1), (True, False, False), (half_width, 1.0, 1.0), chordal)
    return Problem(name, grid, X, truth, obs_idx, y, R, Q, tol, ritz_rank=ritz_rank)


def config1() -> Problem:
    """n=240, N=20, every 4th point observed (d=60), R=0.5, GC c=20, Q=16, tol 1e-12."""
    return gaussian_problem_1d("gauss1d_n240_N20_d60_Q16", n=240, N=20, length_scale=10.0,
                               obs_stride=4, r2=0.5, half_width=20.0, Q=16, tol=1e-12,
                               seed=0)


def config2(tol: float = 1e-12, seed: int = 2) -> Problem:
    """n=8192, N=40, stride 8 (d=1024), R=0.25, GC c=256, Q=32 (1280 shifted systems)."""
    return gaussian_problem_1d("gauss1d_n8192_N40_d1024_Q32", n=8192, N=40, length_scale=64.0,
                               obs_stride=8, r2=0.25, half_width=256.0, Q=32, tol=tol,
                               seed=seed)


# ---------------------------------------------------------------------------
# Layered Lorenz-96 (Sec. 5.1, Eq. ll96_ode)
# ---------------------------------------------------------------------------

def ll96_tendency(X: np.ndarray, F: float, gamma: float) -> np.ndarray:
    """dX/dt for states X[..., nz, nx] (layer-major, longitude periodic)."""
    P = np.concatenate([X[..., -2:], X, X[..., :1]], axis=-1)   # periodic halo: 2 left, 1 right
    xm2, xm1, xp1 = P[..., :-3], P[..., 1:-2], P[..., 3:]
    dX = xm1 * (xp1 - xm2) - X + F
    coup = np.zeros_like(X)
    coup[..., 1:, :] += gamma * (X[..., :-1, :] - X[..., 1:, :])
    coup[..., :-1, :] += gamma * (X[..., 1:, :] - X[..., :-1, :])
    return dX + coup


def ll96_rk4(X: np.ndarray, dt: float, steps: int, F: float = 8.0,
             gamma: float = 1.0) -> np.ndarray:
    X = X.copy()
    for _ in range(steps):
        k1 = ll96_tendency(X, F, gamma)
        k2 = ll96_tendency(X + 0.5 * dt * k1, F, gamma)
        k3 = ll96_tendency(X + 0.5 * dt * k2, F, gamma)
        k4 = ll96_tendency(X + dt * k3, F, gamma)
        X += (dt / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
    return X


def layered_l96_problem(nx: int = 960, nz: int = 8, N: int = 40, spinup: int = 2000,
                        dt: float = 0.01, obs_fraction: float = 0.25, r2: float = 1.0,
                        c_x: float = 60.0, c_z: float = 2.0, Q: int = 24,
                        tol: float = 1e-6, seed: int = 3, obs_seed: int = 1,
                        F: float = 8.0) -> Problem:
    """Ensemble and truth from N+1 perturbed spin-ups; 25% random point observations."""
    rng = np.random.default_rng(seed)
    X0 = F + rng.standard_normal((N + 1, nz, nx))
    Xs = ll96_rk4(X0, dt, spinup, F=F)
    n = nx * nz
    X = Xs[:N].reshape(N, n).copy()
    truth = Xs[N].reshape(n).copy()
    orng = np.random.default_rng(obs_seed)
    d = int(round(obs_fraction * n))
    obs_idx = np.sort(orng.choice(n, size=d, replace=False)).astype(np.int64)
    y, R = _observe(truth, obs_idx, r2, orng)
    grid = Grid((nx, 1, nz), (True, False, False), (c_x, 1.0, c_z), True)
    return Problem(f"ll96_{nz}x{nx}_N{N}_d{d}_Q{Q}", grid, X, truth, obs_idx, y, R, Q, tol)


def uneven_batch(count: int = 64, seed: int = 4, tol: float = 1e-6,
                 n_min: int = 1024, n_max: int = 65536) -> List[Problem]:
    """Batched uneven workload: n log-uniform, N in {20,40,80}, stride 4..16, Q 16..48."""
    rng = np.random.default_rng(seed)
    probs = []
    for p in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        N = int(rng.choice([20, 40, 80]))
        stride = int(rng.integers(4, 17))
        Q = int(rng.integers(16, 49))
        probs.append(gaussian_problem_1d(f"uneven{p}_n{n}_N{N}_s{stride}_Q{Q}", n=n, N=N,
                                         length_scale=16.0, obs_stride=stride, r2=0.5,
                                         half_width=64.0, Q=Q, tol=tol,
                                         seed=int(rng.integers(1 << 31))))
    return probs


def gaussian_problem_2d(nx: int = 1024, ny: int = 1024, N: int = 80, length_scale: float = 32.0,
                        obs_stride: int = 2, r2: float = 0.5, half_width: float = 96.0,
                        Q: int = 32, tol: float = 1e-4, seed: int = 5) -> Problem:
    """2-D periodic Gaussian forecast, observations every ``obs_stride`` cells per axis."""
    rng = np.random.default_rng(seed)
    draws = gaussian_ensemble_2d(nx, ny, N + 1, length_scale, 1.0, 1e-4, rng)
    X, truth = draws[:N].copy(), draws[N].copy()
    ox, oy = np.meshgrid(np.arange(0, nx, obs_stride), np.arange(0, ny, obs_stride))
    obs_idx = np.sort((oy * nx + ox).reshape(-1)).astype(np.int64)
    y, R = _observe(truth, obs_idx, r2, rng)
    grid = Grid((nx, ny, 1), (True, True, False), (half_width, half_width, 1.0), True)
    return Problem(f"gauss2d_{nx}x{ny}_N{N}_Q{Q}", grid, X, truth, obs_idx, y, R, Q, tol)


def config5(tol: float = 1e-6, seed: int = 5) -> Problem:
    """2-D periodic 1024 x 1024 (n = 1,048,576), N = 80, length scale 32 cells, observations every
    2nd cell per axis (d = 262,144), R = 0.5, GC half-width 96 cells, Q = 32 (2560 shifted systems)."""
    return gaussian_problem_2d(nx=1024, ny=1024, N=80, length_scale=32.0, obs_stride=2, r2=0.5,
                               half_width=96.0, Q=32, tol=tol, seed=seed)


def random_obs_problem(grid: Grid, N: int, d: int, r2: float, Q: int, tol: float,
                       seed: int, length_scale: float = 4.0) -> Problem:
    """Small problem with random observation positions and random R (for edge cases)."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = (int(s) for s in grid.shape)
    n = nx * ny * nz
    if ny == 1 and nz == 1:
        draws = gaussian_ensemble_1d(n, N + 1, length_scale, 1.0, 1e-4, rng)
    else:
        draws = rng.standard_normal((N + 1, n))
        # smooth along x so neighbouring points correlate
        draws = np.cumsum(draws.reshape(N + 1, nz * ny, nx), axis=-1).reshape(N + 1, n) / math.sqrt(nx)
    X, truth = draws[:N].copy(), draws[N].copy()
    obs_idx = np.sort(rng.choice(n, size=d, replace=False)).astype(np.int64)
    R = r2 * (0.5 + rng.random(d))
    y = truth[obs_idx] + np.sqrt(R) * rng.standard_normal(d)
    return Problem(f"random_{n}_{d}", grid, X, truth, obs_idx, y, R, Q, tol)


def gaussian_channel_operator(n: int, d: int, bandwidth: float, cutoff: float = 1e-10):
    """Weighted-sum observations in the form of the single-cycle experiment
    (Sec. 4.1): row i weights state j by exp(-c(j, centre_i)^2 / (2 b^2)), with
    c the chordal distance on the circle of circumference n and centres evenly
    spaced (n / d apart).  Weights below ``cutoff`` are dropped.  Returns the
    dense matrix [d][n] and its CSR arrays (rowptr, col, val)."""
    j = np.arange(n)
    centres = (np.arange(d) * n) // d
    delta = np.abs(j[None, :] - centres[:, None])
    c = _chordal(delta, n)
    H = np.exp(-(c ** 2) / (2.0 * bandwidth ** 2))
    H[H < cutoff] = 0.0
    return H, _csr(H)


def column_sum_operator(grid_shape, columns, channels: int, spacing: float, bandwidth: float):
    """Vertical weighted sums in the form of the layered experiment (Sec. 5.1):
    for each observed column x and channel r, sum_z X[z][x] f_r(z) with
    f_r(z) proportional to exp(-(z - spacing r)^2 / (2 b^2)) and sum_z f_r(z)^2 = 1
    (z and r counted from 1).  ``grid_shape`` is (nx, 1, nz); flat index z nx + x.
    Returns the dense matrix [len(columns) channels][n] and its CSR arrays."""
    nx, _, nz = (int(v) for v in grid_shape)
    n = nx * nz
    z = np.arange(1, nz + 1)
    rows = []
    for x in columns:
        for r in range(1, channels + 1):
            f = np.exp(-((z - spacing * r) ** 2) / (2.0 * bandwidth ** 2))
            f /= math.sqrt(float((f ** 2).sum()))
            row = np.zeros(n)
            row[(z - 1) * nx + int(x)] = f
            rows.append(row)
    H = np.array(rows)
    return H, _csr(H)


def _csr(H: np.ndarray):
    rowptr = np.zeros(H.shape[0] + 1, dtype=np.int64)
    cols, vals = [], []
    for i in range(H.shape[0]):
        nz = np.nonzero(H[i])[0]
        cols.append(nz)
        vals.append(H[i, nz])
        rowptr[i + 1] = rowptr[i] + nz.size
    return rowptr, np.concatenate(cols).astype(np.int64), np.concatenate(vals).astype(np.float64)


def general_obs_problem(name: str, grid: Grid, X: np.ndarray, truth: np.ndarray, H: np.ndarray, r2: float,
                        Q: int, tol: float, seed: int):
    """Observations y = H truth + noise with variance r2 for a dense H [d][n]."""
    rng = np.random.default_rng(seed)
    d = H.shape[0]
    R = np.full(d, float(r2))
    y = H @ truth + math.sqrt(r2) * rng.standard_normal(d)
    return dict(name=name, grid=grid, X=X, truth=truth, H=H, y=y, R=R, Q=Q, tol=tol)


# ---------------------------------------------------------------------------
# Single-cycle experiment (Sec. 4.1)
# ---------------------------------------------------------------------------

def single_cycle_covariance(n: int = 2000, nu: float = 10.0, eta: float = 1e-4) -> np.ndarray:
    """Forecast covariance of Eq. single_cycle_covar: eta delta_ij + exp(-c(i,j)^2 / (2 nu^2)),
    with c the chordal distance on the circle of circumference n (dense [n][n])."""
    idx = np.arange(n)
    c = _chordal(idx[:, None] - idx[None, :], n)
    return np.exp(-(c ** 2) / (2.0 * nu ** 2)) + eta * np.eye(n)


def single_cycle_trial(trial: int, N: int = 20, n: int = 2000, nu: float = 10.0, eta: float = 1e-4,
                       d: int = 100, bandwidth: float = 10.0, loc_length: float = 12.0, Q: int = 8,
                       tol: float = 1e-12, Sxx: np.ndarray = None, seed: int = 1000, r2: float = None):
    """One trial of the single-cycle experiment (Sec. 4.1): N forecast members and a truth (draw N + 1)
    from N(0, Sxx), d Gaussian-channel observations (Eq. single_cycle_obsop) with R = r^2 I, r^2 one
    tenth of the mean observable variance diag(H Sxx H^T) (Eq. single_cycle_obserr_covar).  The
    paper's localization is a Gaussian taper of length L; the library localizes with Gaspari-Cohn, so
    the grid carries the half-width sqrt(10/3) L of the matching Gaspari-Cohn function."""
    rng = np.random.default_rng(seed + trial)
    draws = gaussian_ensemble_1d(n, N + 1, nu, 1.0, eta, rng)
    X, truth = draws[:N].copy(), draws[N].copy()
    H, csr = gaussian_channel_operator(n, d, bandwidth)
    if r2 is None:   # the same in every trial: pass it in to skip the contraction
        if Sxx is None:
            Sxx = single_cycle_covariance(n, nu, eta)
        r2 = 0.1 * float(np.mean(np.einsum("ij,jk,ik->i", H, Sxx, H)))
    R = np.full(d, r2)
    y = H @ truth + math.sqrt(r2) * rng.standard_normal(d)
    grid = Grid((n, 1, 1), (True, False, False), (math.sqrt(10.0 / 3.0) * loc_length, 1.0, 1.0), True)
    return dict(name=f"single_cycle_{trial}", grid=grid, X=X, truth=truth, H=H, csr=csr, y=y, R=R, Q=Q,
                tol=tol, r2=r2)
