"""PCG, the limited-memory preconditioner and randomized Ritz pairs (oracle; tests only).

App. E: each perturbation system is solved in normalized form
C_q u = R^-1/2 w with C_q = (s_q + 1) I + C and C = R^-1/2 Shh R^-1/2, then
v = R^-1/2 u (Eq. normalized_linear_solve), by PCG (Golub & Van Loan
Alg. 11.5.1) with the limited-memory preconditioner

    P_q^-1 = (I - Phi T^-1 Phi^T C_q)(I - C_q Phi T^-1 Phi^T) + beta_q Phi T^-1 Phi^T,

T = diag(theta_q).  The Ritz pairs come from a randomized symmetric
eigendecomposition (Halko, Martinsson, Tropp Alg. 5.3) of C, computed once
and shifted to every q: Phi_q = Phi, theta_q = theta(C) + s_q + 1.
beta_q = min_a C_q(a, a) = s_q + 1 + min_a C(a, a).

Readings (the paper does not fix them): Gaussian test matrix with
``oversample`` = 10 extra columns and ``power_iters`` = 1 power iteration
on the range finder; x0 = 0; stop when ||r||_2 <= tol ||b||_2 or after
``max_iter`` iterations; ``fixed_iters`` runs exactly that many iterations
(the paper's experiments use 2 and 10).
"""
from __future__ import annotations

import numpy as np


def pcg(A_mv, b, Minv, tol=1e-12, max_iter=1000, fixed_iters=None):
    """Preconditioned CG (Golub & Van Loan Alg. 11.5.1), x0 = 0.  Returns (x, iters)."""
    x = np.zeros_like(b)
    r = b.copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0
    k = 0
    limit = fixed_iters if fixed_iters is not None else max_iter
    rho = None
    p = None
    while k < limit:
        if fixed_iters is None and np.linalg.norm(r) <= tol * bnorm:
            break
        z = Minv(r)
        k += 1
        if k == 1:
            p = z.copy()
            rho = float(r @ z)
        else:
            rho_new = float(r @ z)
            beta = rho_new / rho
            p = z + beta * p
            rho = rho_new
        Ap = A_mv(p)
        alpha = rho / float(p @ Ap)
        x = x + alpha * p
        r = r - alpha * Ap
    return x, k


def randomized_ritz(C, k, Omega, power_iters=1):
    """k largest Ritz pairs (Phi [d][k], theta [k]) of symmetric C (Halko Alg. 5.3)."""
    Y = C @ Omega
    for _ in range(power_iters):
        Qm, _ = np.linalg.qr(Y)
        Y = C @ Qm
    Qm, _ = np.linalg.qr(Y)
    B = Qm.T @ (C @ Qm)
    B = 0.5 * (B + B.T)
    lam, V = np.linalg.eigh(B)
    order = np.argsort(lam)[::-1][:k]
    return Qm @ V[:, order], lam[order]


def lmp_apply(r, Chat_Phi, Phi, theta_q, beta_q):
    """z = P_q^-1 r with C_q Phi given explicitly (App. E)."""
    t = (Phi.T @ r) / theta_q
    u = r - Chat_Phi @ t
    return u - Phi @ ((Chat_Phi.T @ u) / theta_q) + beta_q * (Phi @ t)


def lmp_matrix(Chat, Phi, theta_q, beta_q):
    """Dense P_q^-1 (tiny sizes only)."""
    d = Chat.shape[0]
    I = np.eye(d)
    T = np.diag(1.0 / theta_q)
    return (I - Phi @ T @ Phi.T @ Chat) @ (I - Chat @ Phi @ T @ Phi.T) + beta_q * Phi @ T @ Phi.T


def solve_normalized(C, s, p, W, R, k=10, Omega=None, tol=1e-12, max_iter=1000,
                     fixed_iters=None, power_iters=1):
    """vbar^(i) = R^-1/2 sum_q p_q u_q^(i) with every C_q u = R^-1/2 w solved by PCG.

    Returns (vbar [d][N], iterations [Q][N]).
    """
    d, N = W.shape
    rih = 1.0 / np.sqrt(np.asarray(R, dtype=np.float64))
    B = rih[:, None] * W
    use_lmp = k > 0 and Omega is not None
    if use_lmp:
        Phi, theta = randomized_ritz(C, k, Omega, power_iters)
        CPhi = C @ Phi
    cmin = float(np.min(np.diag(C))) if d else 0.0
    ubar = np.zeros_like(W)
    iters = np.zeros((len(s), N), dtype=np.int64)
    for qi, (sq, pq) in enumerate(zip(s, p)):
        sigma = sq + 1.0
        A_mv = (lambda v, sigma=sigma: sigma * v + C @ v)
        if use_lmp:
            Chat_Phi = CPhi + sigma * Phi
            theta_q = theta + sigma
            beta_q = sigma + cmin
            Minv = (lambda r, a=Chat_Phi, t=theta_q, b=beta_q: lmp_apply(r, a, Phi, t, b))
        else:
            Minv = (lambda r: r)
        for i in range(N):
            u, it = pcg(A_mv, B[:, i], Minv, tol, max_iter, fixed_iters)
            ubar[:, i] += pq * u
            iters[qi, i] = it
    return rih[:, None] * ubar, iters
