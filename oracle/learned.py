"""Learned preconditioner correction: forward, loss and gradients (oracle; tests only).

Not in the paper: the paper preconditions every shifted system with the
limited-memory preconditioner P_q^-1 of App. E.  The library adds a learned
correction and keeps the result symmetric positive definite by construction:

    M_q = a_q P_q^-1 + S_q^T S_q,

a_q > 0 a scale and S_q a circulant stencil over the observation index with
taps w_q[delta], delta = -h..h, (S r)_a = sum_delta w[delta] r_{(a + delta) mod d}.
A small network maps per-shift features to out = (out_0, out_1..2h+1), and
a_q = exp(out_0) / sigma, w_q = out_1.. / sqrt(sigma): the correction is
expressed relative to C_q^-1 ~ I / sigma, so every shift's loss is O(1) (CG
does not see a common scale of M).

    features phi = (log(sigma)/5, (log(sigma)/5)^2, log(mean_a C(a,a))/5, log(b)/10),
    sigma = s_q + 1, b the Gershgorin bound of C;
    h1 = tanh(W1 phi + b1), h2 = tanh(W2 h1 + b2), out = W3 h2 + b3 (out[0] = log a, out[1:] = w).

Parameters are one flat float vector: W1 [32][4], b1 [32], W2 [32][32],
b2 [32], W3 [18][32], b3 [18] (row-major), 1810 values; h = 8.

Training minimizes, over Krylov vectors v with images y = C_q v and
z = P_q^-1 y taken from the method's own runs,
    L = (1/S) sum_s ||a_s z_s + S_s^T S_s y_s - v_s||^2 / ||v_s||^2.

Two-dimensional lattice form (observations on every point of a periodic
Lx x Ly lattice, vectors indexed a = i + Lx j in lattice order): S is the
stencil over the lattice offsets (dx, dy) with dx^2 + dy^2 <= 8 (the 5 x 5
square), with one tap per squared length (LAT_BINS = 0, 1, 2, 4, 5, 8), so S
is symmetric and S^T S = S S.  The network is the same; w_q holds the bin taps
in its first len(LAT_BINS) entries, the rest unused.  Same loss with S S.

Parity pins: the 1-D stencil against the explicit circulant matrix; the lattice
stencil against a brute-force double loop and against its Fourier symbol
(eigenvalues sum_offsets w cos(2 pi (k dx / Lx + l dy / Ly))); M SPD by
construction; the loss against the base preconditioner at a zero network; the
finite-difference gradients against autograd of an independent PyTorch
restatement (tests/test_oracle_learned.py).
"""
from __future__ import annotations

import numpy as np

H = 8
NTAP = 2 * H + 1
HID = 32
NIN = 4
NOUT = 1 + NTAP
SHAPES = [("W1", (HID, NIN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)),
          ("W3", (NOUT, HID)), ("b3", (NOUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    out, off = {}, 0
    for name, shape in SHAPES:
        size = int(np.prod(shape))
        out[name] = np.asarray(theta[off:off + size], dtype=np.float64).reshape(shape)
        off += size
    return out


def features(sigma, mean_diag, gersh):
    ls = np.log(np.asarray(sigma, dtype=np.float64)) / 5.0
    return np.stack([ls, ls * ls, np.full_like(ls, np.log(mean_diag) / 5.0),
                     np.full_like(ls, np.log(gersh) / 10.0)], axis=-1)


def network(theta, phi):
    """Raw outputs (out_0, out_1..) for each feature row phi [S][4]."""
    p = unpack(theta)
    h1 = np.tanh(phi @ p["W1"].T + p["b1"])
    h2 = np.tanh(h1 @ p["W2"].T + p["b2"])
    out = h2 @ p["W3"].T + p["b3"]
    return out[:, 0], out[:, 1:]


def coefficients(theta, phi):
    """(log a_q, w_q) with a = exp(out_0) / sigma, w = out / sqrt(sigma), sigma = exp(5 phi_0)."""
    o0, ow = network(theta, phi)
    sigma = np.exp(5.0 * np.asarray(phi)[:, 0])
    return o0 - np.log(sigma), ow / np.sqrt(sigma)[:, None]


def stencil(w, r):
    """(S r)_a = sum_delta w[delta + h] r[(a + delta) mod d]."""
    return sum(w[j] * np.roll(r, -(j - H)) for j in range(NTAP))


def stencil_t(w, u):
    """(S^T u)_a = sum_delta w[delta + h] u[(a - delta) mod d]."""
    return sum(w[j] * np.roll(u, j - H) for j in range(NTAP))


def apply_correction(log_a, w, z, r):
    """a z + S^T S r (z = P^-1 r computed by the caller)."""
    return np.exp(log_a) * z + stencil_t(w, stencil(w, r))


def sample_losses(theta, phi, V, Y, Z):
    """Per-sample ||a z + S^T S y - v||^2 / ||v||^2 for samples [S][d]."""
    la, w = coefficients(theta, phi)
    out = np.empty(V.shape[0])
    for s in range(V.shape[0]):
        e = apply_correction(la[s], w[s], Z[s], Y[s]) - V[s]
        out[s] = float(e @ e) / float(V[s] @ V[s])
    return out


def loss(theta, phi, V, Y, Z):
    return float(np.mean(sample_losses(theta, phi, V, Y, Z)))


def fd_gradient(theta, phi, V, Y, Z, eps=1e-6):
    """Central finite differences of the loss in float64 (the check, not a kernel)."""
    g = np.zeros(NPARAM)
    th = np.asarray(theta, dtype=np.float64).copy()
    for i in range(NPARAM):
        old = th[i]
        th[i] = old + eps
        lp = loss(th, phi, V, Y, Z)
        th[i] = old - eps
        lm = loss(th, phi, V, Y, Z)
        th[i] = old
        g[i] = (lp - lm) / (2 * eps)
    return g


def init_params(seed=0, scale=0.1):
    """Small random weights; output bias starts at log a = 0 and a centred delta stencil."""
    rng = np.random.default_rng(seed)
    p = {name: scale * rng.standard_normal(shape) for name, shape in SHAPES}
    p["b3"] = np.zeros(NOUT)
    return np.concatenate([p[name].reshape(-1) for name, _ in SHAPES])


# ---- two-dimensional lattice form ----
H2_LAT = 8
LAT_BINS = (0, 1, 2, 4, 5, 8)
NBIN = len(LAT_BINS)


def lattice_offsets():
    """(dx, dy, bin) for every offset of the stencil, bin = LAT_BINS.index(dx^2 + dy^2)."""
    out = []
    for dy in range(-2, 3):
        for dx in range(-2, 3):
            r2 = dx * dx + dy * dy
            if r2 <= H2_LAT:
                out.append((dx, dy, LAT_BINS.index(r2)))
    return out


def stencil_lattice(wb, r, Lx, Ly):
    """(S r)_(i, j) = sum_offsets wb[bin] r_((i + dx) mod Lx, (j + dy) mod Ly), r in lattice order."""
    R = np.asarray(r, dtype=np.float64).reshape(Ly, Lx)
    out = np.zeros_like(R)
    for dx, dy, b in lattice_offsets():
        out += wb[b] * np.roll(np.roll(R, -dy, axis=0), -dx, axis=1)
    return out.reshape(-1)


def apply_correction_lattice(log_a, wb, z, r, Lx, Ly):
    """a z + S S r (S symmetric; z = P^-1 r computed by the caller)."""
    return np.exp(log_a) * z + stencil_lattice(wb, stencil_lattice(wb, r, Lx, Ly), Lx, Ly)


def sample_losses_lattice(theta, phi, V, Y, Z, Lx, Ly):
    la, w = coefficients(theta, phi)
    out = np.empty(V.shape[0])
    for s in range(V.shape[0]):
        e = apply_correction_lattice(la[s], w[s, :NBIN], Z[s], Y[s], Lx, Ly) - V[s]
        out[s] = float(e @ e) / float(V[s] @ V[s])
    return out


def loss_lattice(theta, phi, V, Y, Z, Lx, Ly):
    return float(np.mean(sample_losses_lattice(theta, phi, V, Y, Z, Lx, Ly)))


def fd_gradient_lattice(theta, phi, V, Y, Z, Lx, Ly, eps=1e-6):
    """Central finite differences of the lattice-form loss in float64."""
    g = np.zeros(NPARAM)
    th = np.asarray(theta, dtype=np.float64).copy()
    for i in range(NPARAM):
        old = th[i]
        th[i] = old + eps
        lp = loss_lattice(th, phi, V, Y, Z, Lx, Ly)
        th[i] = old - eps
        lm = loss_lattice(th, phi, V, Y, Z, Lx, Ly)
        th[i] = old
        g[i] = (lp - lm) / (2 * eps)
    return g

