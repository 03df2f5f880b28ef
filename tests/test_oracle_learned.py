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
