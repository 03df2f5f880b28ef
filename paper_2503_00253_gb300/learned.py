"""Training recipe for the learned preconditioner correction (not in the paper).

The correction M_q = a_q P_q^-1 + S_q^T S_q and its network are described in
include/info_esrf_stages.h.  This module only orchestrates library calls:
Krylov samples are captured from the method's own PCG runs on training
problems (info_esrf_krylov_capture), and the network is trained by the
library's forward, backward and Adam kernels (info_esrf_learn_train).  The
2-D lattice form (BF16 path) uses info_esrf_krylov_capture_lattice and
info_esrf_learn_train_lattice the same way (fit_lattice).
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B

NIN, HID, NOUT = 4, 32, 18


def init_params(seed: int = 0, scale: float = 0.1, device="cuda") -> torch.Tensor:
    """Small random weights with a zero output bias: the starting preconditioner
    is close to the paper's P_q^-1 (a = 1, stencil near zero)."""
    rng = np.random.default_rng(seed)
    shapes = [(HID, NIN), (HID,), (HID, HID), (HID,), (NOUT, HID), (NOUT,)]
    parts = [scale * rng.standard_normal(s) for s in shapes]
    parts[-1] = np.zeros(NOUT)
    theta = np.concatenate([p.reshape(-1) for p in parts]).astype(np.float32)
    assert theta.size == B.learn_nparams()
    return torch.tensor(theta, device=device)


def select_systems(N: int, Q: int, members_per_q: int, seed: int = 0):
    """`members_per_q` perturbation systems (number q * N + i) at every quadrature node."""
    rng = np.random.default_rng(seed)
    sel = []
    for q in range(Q):
        for i in rng.choice(N, size=min(members_per_q, N), replace=False):
            sel.append(q * N + int(i))
    return sel


def capture(problems, K: int = 10, members_per_q: int = 2, ritz_rank: int = 10, device="cuda"):
    """Krylov samples (V, Y, Z, feat) from each problem, concatenated."""
    parts = []
    for idx, pr in enumerate(problems):
        opts = B.make_options(precision=B.PRECISION_FP32, ritz_rank=ritz_rank)
        X = torch.tensor(pr.X, device=device)
        obs = torch.tensor(pr.obs_idx, device=device)
        R = torch.tensor(pr.R, device=device)
        sel = select_systems(pr.N, pr.Q, members_per_q, seed=idx)
        parts.append(B.krylov_capture(pr.grid, X, obs, R, pr.Q, sel, K, opts))
    return tuple(torch.cat([p[i] for p in parts], 0) for i in range(4))


def train(V, Y, Z, feat, steps: int = 400, lr: float = 3e-3, seed: int = 0):
    """Trains a fresh network on the samples; returns (theta, loss history)."""
    theta = init_params(seed, device=V.device)
    hist, _ = B.learn_train(theta, feat, V, Y, Z, steps, lr)
    return theta, hist.cpu().numpy()


def system_iterations(pr, options, device="cuda"):
    """Per-system PCG iterations of one analysis (mean system first), and its stats."""
    X = torch.tensor(pr.X, device=device)
    obs = torch.tensor(pr.obs_idx, device=device)
    y = torch.tensor(pr.y, device=device)
    R = torch.tensor(pr.R, device=device)
    it = torch.zeros(1 + pr.Q * pr.N, dtype=torch.int32, device=device)
    options.system_iters = it.data_ptr()
    options._iters_keep = it
    _, _, st = B.info_esrf_analysis(pr.grid, X, obs, y, R, pr.Q, pr.tol, options)
    return it.cpu().numpy(), st


def choose_max_shift(theta, problems, ritz_rank: int = 10):
    """Plain PCG as the reference: the shift cut-off that minimizes the total number
    of iterations over the problems, comparing every quadrature node's systems
    with and without the learned term.  Returns sigma*; when the term never
    helps, 0.5 (below every shift sigma = s_q + 1 >= 1, so the term is off)."""
    shifts = None
    gain = None
    for pr in problems:
        base = B.make_options(precision=B.PRECISION_FP32, ritz_rank=ritz_rank)
        withm = B.make_options(precision=B.PRECISION_FP32, ritz_rank=ritz_rank, learned_model=theta)
        it0, st = system_iterations(pr, base)
        it1, _ = system_iterations(pr, withm)
        s, _ = B.info_esrf_quadrature_nodes(pr.Q, st["ell_used"])
        sig = s.cpu().numpy() + 1.0
        g = np.array([it1[1 + q * pr.N:1 + (q + 1) * pr.N].sum() - it0[1 + q * pr.N:1 + (q + 1) * pr.N].sum()
                      for q in range(pr.Q)], dtype=np.float64)
        g[0] += it1[0] - it0[0]                      # the mean system has the shift of node 0 (about 1)
        shifts = sig if shifts is None else shifts
        gain = g if gain is None else gain + g
    # total change when the learned term is used for nodes 0..c (prefix sums)
    best_c, best = -1, 0.0
    acc = 0.0
    for c in range(len(gain)):
        acc += gain[c]
        if acc < best:
            best, best_c = acc, c
    return 0.5 if best_c < 0 else float(shifts[best_c]) * (1.0 + 1e-9)


def fit(train_problems, K: int = 12, members_per_q: int = 3, steps: int = 300, lr: float = 3e-3, seed: int = 0):
    """Capture, train and choose the shift cut-off: returns (theta, max_shift, loss history)."""
    V, Y, Z, feat = capture(train_problems, K=K, members_per_q=members_per_q)
    theta, hist = train(V, Y, Z, feat, steps=steps, lr=lr, seed=seed)
    return theta, choose_max_shift(theta, train_problems), hist


def capture_lattice(problems, K: int = 12, members_per_q: int = 3, ritz_rank: int = 10, device="cuda"):
    """Krylov samples (V, Y, Z, feat) of the BF16 path from each 2-D problem, and the common lattice shape."""
    parts, shape = [], None
    for idx, pr in enumerate(problems):
        opts = B.make_options(precision=B.PRECISION_BF16, ritz_rank=ritz_rank)
        X = torch.tensor(pr.X, device=device)
        obs = torch.tensor(pr.obs_idx, device=device)
        R = torch.tensor(pr.R, device=device)
        sel = select_systems(pr.N, pr.Q, members_per_q, seed=idx)
        V, Y, Z, feat, lx, ly = B.krylov_capture_lattice(pr.grid, X, obs, R, pr.Q, sel, K, opts)
        if shape is not None and shape != (lx, ly):
            raise ValueError("training problems on different lattices")
        shape = (lx, ly)
        parts.append((V, Y, Z, feat))
    return tuple(torch.cat([p[i] for p in parts], 0) for i in range(4)) + shape


def system_iterations_bf16(pr, theta=None, max_shift: float = 0.0, ritz_rank: int = 10, device="cuda"):
    """Per-system iterations of one BF16 analysis, with the lattice-form model or without."""
    o = B.make_options(precision=B.PRECISION_BF16, ritz_rank=ritz_rank, learned_model=theta,
                       learned_max_shift=max_shift)
    return system_iterations(pr, o, device=device)


def choose_max_shift_bf16(theta, problems, ritz_rank: int = 10):
    """As choose_max_shift, on the BF16 path (the lattice form)."""
    shifts, gain = None, None
    for pr in problems:
        it0, st = system_iterations_bf16(pr, None, 0.0, ritz_rank)
        it1, _ = system_iterations_bf16(pr, theta, 0.0, ritz_rank)
        s, _ = B.info_esrf_quadrature_nodes(pr.Q, st["ell_used"])
        sig = s.cpu().numpy() + 1.0
        g = np.array([it1[1 + q * pr.N:1 + (q + 1) * pr.N].sum() - it0[1 + q * pr.N:1 + (q + 1) * pr.N].sum()
                      for q in range(pr.Q)], dtype=np.float64)
        g[0] += it1[0] - it0[0]
        shifts = sig if shifts is None else shifts
        gain = g if gain is None else gain + g
    best_c, best, acc = -1, 0.0, 0.0
    for c in range(len(gain)):
        acc += gain[c]
        if acc < best:
            best, best_c = acc, c
    return 0.5 if best_c < 0 else float(shifts[best_c]) * (1.0 + 1e-9)


def fit_lattice(train_problems, K: int = 12, members_per_q: int = 3, steps: int = 300, lr: float = 3e-3,
                seed: int = 0):
    """Capture, train and choose the shift cut-off of the 2-D lattice form on BF16 problems: returns (theta,
    max_shift, loss history)."""
    V, Y, Z, feat, lx, ly = capture_lattice(train_problems, K=K, members_per_q=members_per_q)
    theta = init_params(seed, device=V.device)
    hist, _ = B.learn_train_lattice(theta, feat, V, Y, Z, lx, ly, steps, lr)
    return theta, choose_max_shift_bf16(theta, train_problems), hist.cpu().numpy()

