"""Same-node InFo-ESRF result with sparse matrices (oracle; test infrastructure only).

The dense oracle (``filter``) forms n x n matrices, which stops at a few
thousand grid points.  This module computes the same definitions for large
grids:

* Z, W, mu as in Eq. normalized_perturbations (``filter.anomalies``).
* The localized covariances of Sec. 2.3 / Eq. localized_state_covar, kept
  only at the pairs (a, b) with GC(r_ab) > 0.  Gaspari-Cohn is exactly zero
  for r >= 2, so the dropped entries are exact zeros, not an approximation.
  Pairs are enumerated from a box of grid offsets per axis wide enough for
  the axis distance alone to stay below 2 c (chordal distance <= min-image
  distance, so the box is taken in min-image offsets and then filtered by the
  true distance), and GC and the distances come from ``localization``.
* C = R^-1/2 Shh R^-1/2 (Sec. 3.1), ell by the rule of ``quadrature.ell_rule``
  (Gershgorin bound of C), the nodes and weights of App. D.
* Every normalized shifted system ((s_q + 1) I + C) u = R^-1/2 w of
  Eq. normalized_linear_solve (App. E) is solved exactly by a sparse LU
  factorisation (SuperLU), one per node for all members at once, and
  v_bar = R^-1/2 sum_q p_q u_q (Sec. 3.2, Eq. info_esrf_perturbation_solve).
* z_a = z - Sxh v_bar, A_a = sqrt(N - 1) Z_a^T; mu_a = mu + Sxh (R + Shh)^-1 (y - H mu)
  (Eq. info_esrf_mean_solve), also by sparse LU.

Only subsampling observation operators (obs_idx) are covered.  Pinned against
the dense oracle on small grids (tests/test_oracle_sparse.py).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import localization, quadrature
from .filter import anomalies


def _axis_reach(grid, ax):
    """Largest min-image offset on axis ax whose axis distance alone can be < 2 c (0 for unused axes)."""
    extent = int(grid.shape[ax])
    if extent <= 1:
        return 0
    lim = 2.0 * float(grid.half_width[ax])
    periodic = bool(grid.periodic[ax])
    half = extent // 2 if periodic else extent - 1
    reach = 0
    for off in range(1, half + 1):
        dist = float(localization.axis_distance(0, off, extent, periodic, bool(grid.chordal)))
        if dist < lim:
            reach = off
    return reach


def support_pairs(grid, idx_rows, idx_cols, chunk=1 << 22):
    """(i, j, L) for every pair of flat indices idx_rows[i], idx_cols[j] with GC(r) > 0."""
    nx, ny, nz = (int(s) for s in grid.shape)
    n = nx * ny * nz
    where = np.full(n, -1, dtype=np.int64)
    where[np.asarray(idx_cols, dtype=np.int64)] = np.arange(len(idx_cols))
    ranges = []
    for ax in range(3):
        r, e = _axis_reach(grid, ax), int(grid.shape[ax])
        if grid.periodic[ax] and e > 1:
            # offsets distinct modulo the extent (a support wider than the axis wraps once)
            ranges.append(np.arange(-min(r, (e - 1) // 2), min(r, e // 2) + 1))
        else:
            ranges.append(np.arange(-r, r + 1))
    offs = np.stack(np.meshgrid(*ranges, indexing="ij"), -1).reshape(-1, 3)
    rows = np.asarray(idx_rows, dtype=np.int64)
    rc = localization.coords(grid, rows)
    ext = np.array([nx, ny, nz])
    per = np.array([bool(grid.periodic[a]) for a in range(3)])
    I, J, V = [], [], []
    step = max(1, chunk // max(1, len(offs)))
    for s0 in range(0, len(rows), step):
        c = rc[s0:s0 + step][:, None, :] + offs[None, :, :]            # [rows, offs, 3]
        ok = np.ones(c.shape[:2], dtype=bool)
        for a in range(3):
            if per[a]:
                c[..., a] %= ext[a]
            else:
                ok &= (c[..., a] >= 0) & (c[..., a] < ext[a])
        c = np.where(ok[..., None], c, 0)
        flat = (c[..., 2] * ny + c[..., 1]) * nx + c[..., 0]
        j = np.where(ok, where[flat], -1)
        ii, oo = np.nonzero(j >= 0)
        jj = j[ii, oo]
        gi = s0 + ii
        L = _pair_gc(grid, rows[gi], np.asarray(idx_cols, dtype=np.int64)[jj])
        keep = L > 0.0
        I.append(gi[keep])
        J.append(jj[keep])
        V.append(L[keep])
    return np.concatenate(I), np.concatenate(J), np.concatenate(V)


def _pair_gc(grid, a, b):
    """GC(r(a_k, b_k)) for paired index arrays (the diagonal of localization_matrix)."""
    ca = localization.coords(grid, a)
    cb = localization.coords(grid, b)
    r2 = np.zeros(len(a))
    for ax in range(3):
        extent = int(grid.shape[ax])
        if extent <= 1:
            continue
        dist = localization.axis_distance(ca[:, ax], cb[:, ax], extent, bool(grid.periodic[ax]),
                                          bool(grid.chordal))
        r2 += (dist / float(grid.half_width[ax])) ** 2
    return localization.gaspari_cohn(np.sqrt(r2))


def localized_covariances(Z, obs_idx, grid):
    """W = H Z, Sxh = (L o Z Z^T) H^T (sparse n x d), C = R-free Shh (sparse d x d)."""
    n, N = Z.shape
    obs_idx = np.asarray(obs_idx, dtype=np.int64)
    d = obs_idx.size
    W = Z[obs_idx, :]
    i, j, L = support_pairs(grid, obs_idx, obs_idx)
    Shh = sp.csr_matrix((L * np.einsum("kn,kn->k", W[i], W[j]), (i, j)), shape=(d, d))
    i, j, L = support_pairs(grid, np.arange(n), obs_idx)
    Sxh = sp.csr_matrix((L * np.einsum("kn,kn->k", Z[i], W[j]), (i, j)), shape=(n, d))
    return W, Sxh, Shh


def _normalized(Shh, R):
    rih = 1.0 / np.sqrt(np.asarray(R, dtype=np.float64))
    return sp.diags(rih) @ Shh @ sp.diags(rih), rih


def ell_rule(Shh, R):
    """quadrature.ell_rule on the Gershgorin bound of the sparse C."""
    C, _ = _normalized(Shh, R)
    b = max(float(np.max(np.asarray(abs(C).sum(axis=1)).ravel())), 1.0)
    return float(10.0 ** (math.floor(math.log10(b)) + 1))


def perturbation_update(X, obs_idx, R, grid, Q, ell=None, rule="elliptic"):
    """Analysis anomalies A_a [N][n] of Sec. 3.2 with exact (sparse LU) solves per node."""
    mu, Z = anomalies(X)
    W, Sxh, Shh = localized_covariances(Z, obs_idx, grid)
    C, rih = _normalized(Shh, R)
    ell_used = float(ell) if ell is not None and ell > 0 else ell_rule(Shh, R)
    s, p = quadrature.quadrature(Q, ell_used, rule)
    B = rih[:, None] * W
    I = sp.identity(C.shape[0], format="csc")
    vbar = np.zeros_like(W)
    for sq, pq in zip(s, p):
        lu = spla.splu(((sq + 1.0) * I + C).tocsc())
        vbar += pq * lu.solve(B)
    vbar *= rih[:, None]
    N = Z.shape[1]
    return math.sqrt(N - 1) * (Z - Sxh @ vbar).T


def mean_update(X, obs_idx, y, R, grid):
    """mu_a = mu + Sxh (R + Shh)^-1 (y - H mu) (Eq. info_esrf_mean_solve), normalized and solved by sparse LU."""
    mu, Z = anomalies(X)
    W, Sxh, Shh = localized_covariances(Z, obs_idx, grid)
    C, rih = _normalized(Shh, R)
    innov = np.asarray(y, dtype=np.float64) - mu[np.asarray(obs_idx, dtype=np.int64)]
    lu = spla.splu((sp.identity(C.shape[0], format="csc") + C).tocsc())
    return mu + Sxh @ (rih * lu.solve(rih * innov))
