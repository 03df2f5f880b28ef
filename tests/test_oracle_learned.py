"""Pins of the oracle for the learned preconditioner correction (not in the paper)."""
import numpy as np
import pytest
import torch

from oracle import learned as LR


def _circulant(w, d):
    """Dense S with (S r)_a = sum_t w[t + h] r[(a + t) mod d]."""
    S = np.zeros((d, d))
    for a in range(d):
        for j, wt in enumerate(w):
            S[a, (a + j - LR.H) % d] += wt
    return S


def test_stencil_and_transpose_are_the_circulant_matrix():
    rng = np.random.default_rng(0)
    d = 37
    w = rng.standard_normal(LR.NTAP)
    r = rng.standard_normal(d)
    S = _circulant(w, d)
    assert np.max(np.abs(LR.stencil(w, r) - S @ r)) < 1e-13
    assert np.max(np.abs(LR.stencil_t(w, r) - S.T @ r)) < 1e-13


def test_correction_is_spd():
    rng = np.random.default_rng(1)
    d = 29
    w = rng.standard_normal(LR.NTAP)
    B = rng.standard_normal((d, d))
    Pinv = B @ B.T + 0.5 * np.eye(d)          # any SPD base preconditioner
    M = np.exp(-0.7) * Pinv + _circulant(w, d).T @ _circulant(w, d)
    assert np.allclose(M, M.T)
    assert np.linalg.eigvalsh(M).min() > 0


def test_zero_network_reduces_to_base_preconditioner():
    theta = np.zeros(LR.NPARAM)
    phi = LR.features(np.array([1.0, 1.0]), 2.0, 150.0)
    la, w = LR.coefficients(theta, phi)
    assert np.all(np.abs(la) < 1e-15) and np.all(w == 0)     # sigma = 1: a = 1, no stencil
    rng = np.random.default_rng(2)
    d = 20
    A = rng.standard_normal((d, d))
    Chat = A @ A.T + np.eye(d)
    V = rng.standard_normal((2, d))
    Y = V @ Chat.T
    Z = Y.copy()                               # base preconditioner = identity
    ref = [np.linalg.norm(Chat @ v - v) ** 2 / np.linalg.norm(v) ** 2 for v in V]
    assert abs(LR.loss(theta, phi, V, Y, Z) - np.mean(ref)) < 1e-12


def _torch_loss(theta, phi, V, Y, Z):
    """Independent restatement with PyTorch CPU ops (circulant as an explicit matrix)."""
    offs, p = 0, {}
    for name, shape in LR.SHAPES:
        size = int(np.prod(shape))
        p[name] = theta[offs:offs + size].reshape(shape)
        offs += size
    ph = torch.tensor(phi)
    h1 = torch.tanh(ph @ p["W1"].T + p["b1"])
    h2 = torch.tanh(h1 @ p["W2"].T + p["b2"])
    out = h2 @ p["W3"].T + p["b3"]
    sigma = torch.exp(5.0 * ph[:, 0])
    d = V.shape[1]
    idx = torch.arange(d)
    total = 0.0
    for s in range(V.shape[0]):
        w = out[s, 1:] / torch.sqrt(sigma[s])
        S = torch.zeros((d, d), dtype=torch.float64)
        for j in range(LR.NTAP):
            S = S.index_put((idx, (idx + j - LR.H) % d), w[j], accumulate=True)
        y, z, v = (torch.tensor(a[s]) for a in (Y, Z, V))
        e = torch.exp(out[s, 0]) / sigma[s] * z + S.T @ (S @ y) - v
        total = total + (e @ e) / (v @ v)
    return total / V.shape[0]


def test_fd_gradient_matches_autograd():
    rng = np.random.default_rng(3)
    d, nsamp = 23, 3
    theta = LR.init_params(seed=4, scale=0.3)
    phi = LR.features(np.array([1.3, 4.0, 60.0]), 1.7, 90.0)
    V = rng.standard_normal((nsamp, d))
    Y = rng.standard_normal((nsamp, d))
    Z = rng.standard_normal((nsamp, d))
    th = torch.tensor(theta, requires_grad=True)
    lt = _torch_loss(th, phi, V, Y, Z)
    lt.backward()
    assert abs(float(lt) - LR.loss(theta, phi, V, Y, Z)) < 1e-12 * max(1.0, float(lt))
    g_fd = LR.fd_gradient(theta, phi, V, Y, Z)
    g_ad = th.grad.numpy()
    assert np.max(np.abs(g_fd - g_ad)) < 1e-6 * max(1.0, np.max(np.abs(g_ad)))


# ---- two-dimensional lattice form ----

def _lattice_brute(wb, r, Lx, Ly):
    """Brute force: explicit loops over lattice points and the 5 x 5 offsets."""
    out = np.zeros(Lx * Ly)
    for j in range(Ly):
        for i in range(Lx):
            acc = 0.0
            for dy in range(-2, 3):
                for dx in range(-2, 3):
                    r2 = dx * dx + dy * dy
                    if r2 <= 8:
                        acc += wb[[0, 1, 2, 4, 5, 8].index(r2)] * r[((i + dx) % Lx) + Lx * ((j + dy) % Ly)]
            out[i + Lx * j] = acc
    return out


def test_lattice_offsets_are_the_5x5_square():
    offs = LR.lattice_offsets()
    assert len(offs) == 25 and len({(dx, dy) for dx, dy, _ in offs}) == 25
    counts = np.bincount([b for _, _, b in offs], minlength=LR.NBIN)
    assert list(counts) == [1, 4, 4, 4, 8, 4]      # squared lengths 0, 1, 2, 4, 5, 8


def test_lattice_stencil_matches_brute_force_and_is_symmetric():
    rng = np.random.default_rng(5)
    for Lx, Ly in ((7, 5), (6, 9), (8, 1)):
        wb = rng.standard_normal(LR.NBIN)
        r = rng.standard_normal(Lx * Ly)
        assert np.max(np.abs(LR.stencil_lattice(wb, r, Lx, Ly) - _lattice_brute(wb, r, Lx, Ly))) < 1e-13
        S = np.stack([LR.stencil_lattice(wb, e, Lx, Ly) for e in np.eye(Lx * Ly)], axis=1)
        assert np.max(np.abs(S - S.T)) < 1e-13


def test_lattice_stencil_eigenvalues_are_its_fourier_symbol():
    rng = np.random.default_rng(6)
    Lx, Ly = 9, 7
    wb = rng.standard_normal(LR.NBIN)
    S = np.stack([LR.stencil_lattice(wb, e, Lx, Ly) for e in np.eye(Lx * Ly)], axis=1)
    sym = [sum(wb[b] * np.cos(2 * np.pi * (k * dx / Lx + l * dy / Ly)) for dx, dy, b in LR.lattice_offsets())
           for l in range(Ly) for k in range(Lx)]
    assert np.max(np.abs(np.sort(np.linalg.eigvalsh(S)) - np.sort(sym))) < 1e-12
    # a plane wave is an eigenvector
    jj, ii = np.meshgrid(np.arange(Ly), np.arange(Lx), indexing="ij")
    wave = np.cos(2 * np.pi * (2 * ii / Lx + 3 * jj / Ly)).reshape(-1)
    lam = sum(wb[b] * np.cos(2 * np.pi * (2 * dx / Lx + 3 * dy / Ly)) for dx, dy, b in LR.lattice_offsets())
    assert np.max(np.abs(LR.stencil_lattice(wb, wave, Lx, Ly) - lam * wave)) < 1e-12


def test_lattice_correction_is_spd():
    rng = np.random.default_rng(7)
    Lx, Ly = 6, 5
    d = Lx * Ly
    wb = rng.standard_normal(LR.NBIN)
    B = rng.standard_normal((d, d))
    Pinv = B @ B.T + 0.5 * np.eye(d)
    M = np.stack([LR.apply_correction_lattice(-0.4, wb, Pinv @ e, e, Lx, Ly) for e in np.eye(d)], axis=1)
    assert np.max(np.abs(M - M.T)) < 1e-10 * np.max(np.abs(M))
    assert np.linalg.eigvalsh(M).min() > 0


def _torch_loss_lattice(theta, phi, V, Y, Z, Lx, Ly):
    """Independent restatement: the lattice stencil as an explicit matrix built by index arithmetic."""
    offs, p = 0, {}
    for name, shape in LR.SHAPES:
        size = int(np.prod(shape))
        p[name] = theta[offs:offs + size].reshape(shape)
        offs += size
    ph = torch.tensor(phi)
    h1 = torch.tanh(ph @ p["W1"].T + p["b1"])
    h2 = torch.tanh(h1 @ p["W2"].T + p["b2"])
    out = h2 @ p["W3"].T + p["b3"]
    sigma = torch.exp(5.0 * ph[:, 0])
    d = Lx * Ly
    ii = torch.arange(d) % Lx
    jj = torch.arange(d) // Lx
    bins = {0: 0, 1: 1, 2: 2, 4: 3, 5: 4, 8: 5}
    total = 0.0
    for s in range(V.shape[0]):
        w = out[s, 1:] / torch.sqrt(sigma[s])
        S = torch.zeros((d, d), dtype=torch.float64)
        for dy in range(-2, 3):
            for dx in range(-2, 3):
                if dx * dx + dy * dy <= 8:
                    col = (ii + dx) % Lx + Lx * ((jj + dy) % Ly)
                    S = S.index_put((torch.arange(d), col), w[bins[dx * dx + dy * dy]], accumulate=True)
        y, z, v = (torch.tensor(a[s]) for a in (Y, Z, V))
        e = torch.exp(out[s, 0]) / sigma[s] * z + S @ (S @ y) - v
        total = total + (e @ e) / (v @ v)
    return total / V.shape[0]


def test_lattice_fd_gradient_matches_autograd():
    rng = np.random.default_rng(8)
    Lx, Ly, nsamp = 6, 5, 3
    d = Lx * Ly
    theta = LR.init_params(seed=9, scale=0.3)
    phi = LR.features(np.array([1.2, 3.0, 40.0]), 1.9, 70.0)
    V = rng.standard_normal((nsamp, d))
    Y = rng.standard_normal((nsamp, d))
    Z = rng.standard_normal((nsamp, d))
    th = torch.tensor(theta, requires_grad=True)
    lt = _torch_loss_lattice(th, phi, V, Y, Z, Lx, Ly)
    lt.backward()
    assert abs(float(lt) - LR.loss_lattice(theta, phi, V, Y, Z, Lx, Ly)) < 1e-12 * max(1.0, float(lt))
    g_fd = LR.fd_gradient_lattice(theta, phi, V, Y, Z, Lx, Ly)
    g_ad = th.grad.numpy()
    assert np.max(np.abs(g_fd - g_ad)) < 1e-6 * max(1.0, np.max(np.abs(g_ad)))

