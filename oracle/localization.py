"""Gaspari-Cohn localization on regular grids (oracle; test infrastructure only).

Model-space localization multiplies the ensemble covariance elementwise by L
(Sec. 2.3, Eq. localized_state_covar).  The paper builds L from the
Gaspari-Cohn function of a scaled distance (Fig. 1 caption; Sec. 5.2 uses
G_2(dist / L) supported on [-2, 2]).  The GC formula itself is not printed in
the paper; it is the fifth-order piecewise rational function of Gaspari &
Cohn (1999), Eq. 4.10, with half-width c: L = GC(dist / c), GC(0) = 1 and
GC(z) = 0 for z >= 2.

Distances: on periodic axes the chordal distance c(i,j) = (n/pi) sin(pi|i-j|/n)
(Sec. 4.1, Eq. single_cycle_covar; Sec. 5.2) unless the grid asks for the
minimum-image distance; on non-periodic axes |i - j|.  Several axes combine as
r = sqrt(sum_a (dist_a / c_a)^2) (Sec. 5.2 with one c per axis).
"""
from __future__ import annotations

import numpy as np


def gaspari_cohn(z):
    """GC(z) for z = distance / half-width (Gaspari & Cohn 1999, Eq. 4.10)."""
    z = np.abs(np.asarray(z, dtype=np.float64))
    out = np.zeros_like(z)
    inner = z <= 1.0
    outer = (z > 1.0) & (z < 2.0)
    a = z[inner]
    out[inner] = -0.25 * a**5 + 0.5 * a**4 + 0.625 * a**3 - (5.0 / 3.0) * a**2 + 1.0
    b = z[outer]
    out[outer] = (b**5 / 12.0 - 0.5 * b**4 + 0.625 * b**3 + (5.0 / 3.0) * b**2
                  - 5.0 * b + 4.0 - (2.0 / 3.0) / b)
    return out


def coords(grid, idx):
    nx, ny, nz = (int(s) for s in grid.shape)
    idx = np.asarray(idx, dtype=np.int64)
    return np.stack([idx % nx, (idx // nx) % ny, idx // (nx * ny)], axis=-1)


def axis_distance(a, b, extent, periodic, chordal):
    delta = np.abs(np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64))
    if periodic:
        if chordal:
            return (extent / np.pi) * np.sin(np.pi * delta / extent)
        return np.minimum(delta, extent - delta)
    return delta


def scaled_distance(grid, idx_a, idx_b):
    """Dense matrix of r(a, b) = sqrt(sum_axes (dist / c)^2)."""
    ca = coords(grid, idx_a)
    cb = coords(grid, idx_b)
    r2 = np.zeros((ca.shape[0], cb.shape[0]))
    for ax in range(3):
        extent = int(grid.shape[ax])
        if extent <= 1:
            continue
        dist = axis_distance(ca[:, ax][:, None], cb[:, ax][None, :], extent,
                             bool(grid.periodic[ax]), bool(grid.chordal))
        r2 += (dist / float(grid.half_width[ax])) ** 2
    return np.sqrt(r2)


def localization_matrix(grid, idx_a, idx_b):
    """Dense L(a, b) = GC(r(a, b)) between two index sets."""
    return gaspari_cohn(scaled_distance(grid, idx_a, idx_b))
