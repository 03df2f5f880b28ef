"""Pins of the oracle's Gaspari-Cohn localization (Sec. 2.3, Sec. 5.2)."""
import math
import types

import numpy as np
import pytest

from oracle import localization


def _grid(shape, periodic, hw, chordal=True):
    return types.SimpleNamespace(shape=shape, periodic=periodic, half_width=hw, chordal=chordal)


def test_gc_values_and_support():
    gc = localization.gaspari_cohn
    assert gc(0.0) == 1.0
    assert abs(gc(1.0) - 5.0 / 24.0) < 1e-15        # both branches meet at 5/24
    assert gc(2.0) == 0.0 and gc(2.5) == 0.0
    eps = 1e-7
    for z in (1.0, 2.0):                              # C^1 at the knots
        left = (gc(z - eps) - gc(z - 2 * eps)) / eps
        right = (gc(z + 2 * eps) - gc(z + eps)) / eps
        assert abs(left - right) < 1e-5
        assert abs(gc(z - eps) - gc(z + eps)) < 1e-6
    z = np.linspace(0, 2, 401)
    assert np.all(np.diff(gc(z)) <= 1e-15)            # monotone decreasing


@pytest.mark.parametrize("chordal", [True, False])
def test_localization_psd_1d(chordal):
    g = _grid((64, 1, 1), (True, False, False), (6.0, 1.0, 1.0), chordal)
    L = localization.localization_matrix(g, np.arange(64), np.arange(64))
    assert np.allclose(L, L.T)
    assert np.allclose(np.diag(L), 1.0)
    assert np.linalg.eigvalsh(L).min() > -1e-10


def test_localization_layered_anisotropic():
    g = _grid((40, 1, 6), (True, False, False), (5.0, 1.0, 1.5), True)
    idx = np.arange(240)
    L = localization.localization_matrix(g, idx, idx)
    assert np.allclose(L, L.T)
    # vertical axis is not periodic: bottom and top layers at the same column decouple
    assert L[0, 5 * 40] == 0.0
    # one layer up, same column: r = 1 / 1.5
    assert abs(L[0, 40] - localization.gaspari_cohn(1.0 / 1.5)) < 1e-15
    # chordal horizontal distance wraps around
    d = (40 / math.pi) * math.sin(math.pi * 39 / 40)
    assert abs(L[0, 39] - localization.gaspari_cohn(d / 5.0)) < 1e-15
    assert np.linalg.eigvalsh(L).min() > -1e-10
