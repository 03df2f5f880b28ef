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

Multi-shift CG (Sec. 3.3, first alternative to per-system PCG; shift
invariance of Krylov subspaces): in normalized form every C_q is the same C
shifted by sigma_q = s_q + 1, so K_k(C + sigma I, b) does not depend on sigma.
One CG run on the base system (C + sigma_0 I) u = b, sigma_0 = min_q sigma_q,
yields every shifted iterate: the shifted residuals stay collinear with the
base residual, r_k^(q) = zeta_k^(q) r_k, and zeta, alpha^(q), beta^(q) follow
from matching the three-term residual recurrences of CG for the two systems
(Frommer & Glassner 1998; Jegerlehner 1996).  It runs without a
preconditioner, as the paper notes.

Block CG (Sec. 3.3, second alternative): for one node, the N members'
systems share the block Krylov space span{B, C_q B, ...}; O'Leary's block CG
gives each member the C_q-norm-optimal iterate in it, with dense s x s solves
per iteration.

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


def multishift_cg(A_mv, b, shifts, tol=1e-12, max_iter=1000, fixed_iters=None):
    """Solves (A + shifts[q] I) x_q = b for every q from one CG run (Sec. 3.3).

    The base system is A + sigma_0 I with sigma_0 = min(shifts); shift q is
    sigma_0 + delta_q.  With beta_{-1} = 0, alpha_{-1} = 1 and
    zeta_{-1} = zeta_0 = 1, iteration k of base CG (alpha_k, beta_k) gives

        zeta_{k+1} = zeta_k zeta_{k-1} alpha_{k-1} /
                     (alpha_k beta_{k-1} (zeta_{k-1} - zeta_k) + zeta_{k-1} alpha_{k-1} (1 + delta alpha_k)),
        alpha_k^(q) = alpha_k zeta_{k+1} / zeta_k,   beta_k^(q) = beta_k (zeta_{k+1} / zeta_k)^2,
        x^(q) += alpha_k^(q) p^(q),   p^(q) <- zeta_{k+1} r_{k+1} + beta_k^(q) p^(q).

    Shift q stops being updated once its residual |zeta^(q)| ||r|| is at most
    tol ||b|| (with fixed_iters: 1e-30 ||b||, so that zeta never underflows);
    the run ends when every shift has stopped, at max_iter, or after
    fixed_iters iterations.  Returns (X [Q][d], iters [Q], relres [Q]).
    """
    shifts = np.asarray(shifts, dtype=np.float64)
    nq = shifts.shape[0]
    d = b.shape[0]
    X = np.zeros((nq, d))
    iters = np.zeros(nq, dtype=np.int64)
    relres = np.zeros(nq)
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0 or nq == 0:
        return X, iters, relres
    sigma0 = float(shifts.min())
    delta = shifts - sigma0
    stop = (1e-30 if fixed_iters is not None else tol) * bnorm
    limit = fixed_iters if fixed_iters is not None else max_iter
    r = b.copy()
    p = b.copy()
    rr = float(r @ r)
    P = np.tile(b, (nq, 1))
    zeta = np.ones(nq)
    zeta_prev = np.ones(nq)
    alpha_prev, beta_prev = 1.0, 0.0
    active = np.full(nq, True)
    relres[:] = 1.0
    k = 0
    while k < limit and active.any():
        Ap = A_mv(p) + sigma0 * p
        alpha = rr / float(p @ Ap)
        r = r - alpha * Ap
        rr_new = float(r @ r)
        beta = rr_new / rr
        for q in np.nonzero(active)[0]:
            z0, zm = zeta[q], zeta_prev[q]
            z1 = z0 * zm * alpha_prev / (alpha * beta_prev * (zm - z0) + zm * alpha_prev * (1.0 + delta[q] * alpha))
            ratio = z1 / z0
            X[q] += alpha * ratio * P[q]
            P[q] = z1 * r + beta * ratio * ratio * P[q]
            zeta_prev[q], zeta[q] = z0, z1
            iters[q] = k + 1
            relres[q] = abs(z1) * np.sqrt(rr_new) / bnorm
            if abs(z1) * np.sqrt(rr_new) <= stop:
                active[q] = False
        p = r + beta * p
        rr = rr_new
        alpha_prev, beta_prev = alpha, beta
        k += 1
    return X, iters, relres


def solve_normalized_multishift(C, s, p, W, R, tol=1e-12, max_iter=1000, fixed_iters=None):
    """vbar^(i) = R^-1/2 sum_q p_q u_q^(i) with all Q shifts of member i solved
    by one multi-shift CG run on C (no preconditioner).  Returns (vbar [d][N],
    iterations [Q][N])."""
    d, N = W.shape
    rih = 1.0 / np.sqrt(np.asarray(R, dtype=np.float64))
    B = rih[:, None] * W
    shifts = np.asarray(s, dtype=np.float64) + 1.0
    ubar = np.zeros_like(W)
    iters = np.zeros((len(s), N), dtype=np.int64)
    for i in range(N):
        U, it, _ = multishift_cg(lambda v: C @ v, B[:, i], shifts, tol, max_iter, fixed_iters)
        ubar[:, i] = np.asarray(p) @ U
        iters[:, i] = it
    return rih[:, None] * ubar, iters


def block_cg(A_mv, B, tol=1e-12, max_iter=1000, fixed_iters=None):
    """Block CG (O'Leary 1980) for A X = B with X, B in R^{d x s} (Sec. 3.3, the
    second alternative: the s members' systems of one shift share a block
    Krylov space, span{B, A B, ..., A^{k-1} B}, and each column's iterate is the
    A-norm-optimal approximation within it).

    X_0 = 0, R_0 = B, P_0 = R_0; with Q = A P,
        alpha = (P^T Q)^-1 (R^T R),  X += P alpha,  R' = R - Q alpha,
        beta = (R^T R)^-1 (R'^T R'),  P <- R' + P beta.
    Stops when every column has ||r_i|| <= tol ||b_i||, at max_iter, or after
    fixed_iters iterations.  The s x s solves are dense (no deflation: the
    block must stay of full rank, which holds while no column has converged
    exactly).  Returns (X, iterations)."""
    B = np.asarray(B, dtype=np.float64)
    X = np.zeros_like(B)
    R = B.copy()
    bn = np.linalg.norm(B, axis=0)
    if not np.any(bn > 0):
        return X, 0
    P = R.copy()
    RR = R.T @ R
    limit = fixed_iters if fixed_iters is not None else max_iter
    k = 0
    while k < limit:
        if fixed_iters is None and np.all(np.linalg.norm(R, axis=0) <= tol * bn):
            break
        Q = A_mv(P)
        alpha = np.linalg.solve(P.T @ Q, RR)
        X = X + P @ alpha
        R = R - Q @ alpha
        RR_new = R.T @ R
        beta = np.linalg.solve(RR, RR_new)
        P = R + P @ beta
        RR = RR_new
        k += 1
    return X, k


def solve_normalized_block(C, s, p, W, R, tol=1e-12, max_iter=1000, fixed_iters=None):
    """vbar = R^-1/2 sum_q p_q U_q with, for every node q, all members' systems
    ((s_q + 1) I + C) U_q = R^-1/2 W solved together by block CG.  Returns
    (vbar [d][N], iterations [Q])."""
    rih = 1.0 / np.sqrt(np.asarray(R, dtype=np.float64))
    B = rih[:, None] * W
    ubar = np.zeros_like(W)
    iters = np.zeros(len(s), dtype=np.int64)
    for qi, (sq, pq) in enumerate(zip(s, p)):
        sigma = sq + 1.0
        U, it = block_cg(lambda V, sigma=sigma: sigma * V + C @ V, B, tol, max_iter, fixed_iters)
        ubar += pq * U
        iters[qi] = it
    return rih[:, None] * ubar, iters
