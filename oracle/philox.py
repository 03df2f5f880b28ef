"""Philox4x32-10 and Box-Muller normals (oracle side; test infrastructure only).

The randomized eigensolver of App. E (Halko et al. Alg. 5.3 with a Gaussian
test matrix) draws random numbers.  Both the CUDA path and this oracle draw
them from one counter-based generator written independently from its
published definition: Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11).

Round: (hi0, lo0) = mulhilo(0xD2511F53, x0), (hi1, lo1) = mulhilo(0xCD9E8D57, x2),
x <- (hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0); between rounds the key is
bumped by (0x9E3779B9, 0xBB67AE85).

Element e of a test matrix uses counter (t_lo, t_hi, 0, 0) with t = e // 2 and
key (seed_lo, seed_hi); u1 = (x0 + 1/2) 2^-32, u2 = (x1 + 1/2) 2^-32 and the
pair (sqrt(-2 ln u1) cos(2 pi u2), sqrt(-2 ln u1) sin(2 pi u2)) gives elements
2t and 2t + 1.
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(counter, key):
    """Vectorised Philox4x32-10.  counter: uint32 array [..., 4]; key: uint32 [2]."""
    x = [np.asarray(counter[..., i], dtype=np.uint64) for i in range(4)]
    k0 = np.uint64(int(key[0]) & 0xFFFFFFFF)
    k1 = np.uint64(int(key[1]) & 0xFFFFFFFF)
    for rnd in range(10):
        p0 = M0 * x[0]
        p1 = M1 * x[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        x = [(hi1 ^ x[1] ^ k0) & MASK, lo1, (hi0 ^ x[3] ^ k1) & MASK, lo0]
        if rnd < 9:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
    return np.stack([xi.astype(np.uint32) for xi in x], axis=-1)


def normals(count: int, seed: int) -> np.ndarray:
    """``count`` standard normals, element e from pair t = e // 2 (see module doc)."""
    pairs = (count + 1) // 2
    t = np.arange(pairs, dtype=np.uint64)
    ctr = np.zeros((pairs, 4), dtype=np.uint32)
    ctr[:, 0] = (t & MASK).astype(np.uint32)
    ctr[:, 1] = (t >> np.uint64(32)).astype(np.uint32)
    key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    out = philox4x32_10(ctr, key)
    u1 = (out[:, 0].astype(np.float64) + 0.5) * 2.0**-32
    u2 = (out[:, 1].astype(np.float64) + 0.5) * 2.0**-32
    rad = np.sqrt(-2.0 * np.log(u1))
    g = np.empty(2 * pairs)
    g[0::2] = rad * np.cos(2.0 * np.pi * u2)
    g[1::2] = rad * np.sin(2.0 * np.pi * u2)
    return g[:count]


def test_matrix(d: int, l: int, seed: int) -> np.ndarray:
    """Gaussian test matrix Omega [d][l]; element (a, j) is flat index e = j * d + a."""
    return normals(d * l, seed).reshape(l, d).T.copy()
