"""Pins of the oracle's quadrature rules (App. D) against closed forms."""
import math
import os

import numpy as np
import pytest
from scipy import integrate

from oracle import quadrature

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _f2(c):
    # int p(s) / (s + 1 + c) ds = 1 / (1 + c + sqrt(1 + c))  (App. C, partial fractions)
    return 1.0 / (1.0 + c + np.sqrt(1.0 + c))


def _read_pairs(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


@pytest.mark.parametrize("ell", [10.0, 100.0, 1000.0])
@pytest.mark.parametrize("Q", [16, 24, 32])
def test_elliptic_rule_inverse_sqrt_identity(ell, Q):
    """sum_q r_q / (s_q + c + 1) -> (c + 1)^-1/2 for c in [0, ell] (Eq. generic_invsqrt_integral)."""
    s, p = quadrature.elliptic_rule(Q, ell)
    r = p * (s + 1.0)
    c = np.concatenate([[0.0], np.logspace(-4, math.log10(ell), 200)])
    approx = (r[None, :] / (s[None, :] + c[:, None] + 1.0)).sum(1)
    err = np.max(np.abs(approx * np.sqrt(c + 1.0) - 1.0))
    bound = {10.0: 1e-12, 100.0: 1e-11, 1000.0: 1e-9}[ell] if Q >= 16 else 1e-6
    assert err < bound
    # weights integrate the density: sum p_q = 1 (c = 0 in Theorem 3)
    assert abs(p.sum() - 1.0) < bound
    assert np.all(s > 0) and np.all(p > 0)


def test_elliptic_rule_is_hale_higham_trefethen_rate():
    """Q = O(log(1/eps) log(ell)): at fixed Q the error grows slowly with ell (App. D)."""
    errs = []
    for ell in [10.0, 100.0, 1000.0, 10000.0]:
        s, p = quadrature.elliptic_rule(12, ell)
        c = np.logspace(-3, math.log10(ell), 200)
        approx = (p[None, :] / (s[None, :] + 1.0 + c[:, None])).sum(1)
        errs.append(np.max(np.abs(approx / _f2(c) - 1.0)))
    assert errs[0] < errs[1] < errs[2] < errs[3] < 1e-3
    # doubling Q at ell = 1000 squares the error (exponential convergence)
    e = []
    for Q in (8, 16):
        s, p = quadrature.elliptic_rule(Q, 1000.0)
        c = np.logspace(-3, 3, 200)
        e.append(np.max(np.abs((p[None, :] / (s[None, :] + 1.0 + c[:, None])).sum(1) / _f2(c) - 1.0)))
    assert e[1] < 10 * e[0] ** 2


def test_scalar_modified_gain_appD():
    """App. D scalar test: sum_q p_q s_xh / (1 + s_q + s_hh) -> s_xh / (1 + s_hh + sqrt(1 + s_hh))."""
    g = _read_pairs("scalar_gain_appD.txt")
    sxh, shh = g["sigma_xh"], g["sigma_hh"]
    G = sxh / (1.0 + shh + math.sqrt(1.0 + shh))
    assert abs(G - quadrature.scalar_gain(sxh, shh)) < 1e-15
    errs_e, errs_g = [], []
    for Q in (2, 4, 8, 16):
        s, p = quadrature.elliptic_rule(Q, 100.0)
        errs_e.append(abs((p * sxh / (1.0 + s + shh)).sum() - G) / G)
        s, p = quadrature.gauss_legendre_rule(Q)
        errs_g.append(abs((p * sxh / (1.0 + s + shh)).sum() - G) / G)
    assert errs_e[-1] < 1e-13
    # the elliptic rule converges much faster than Gauss-Legendre (App. D)
    for a, b in zip(errs_e[1:], errs_g[1:]):
        assert a < b


def test_gauss_legendre_rule_limit():
    s, p = quadrature.gauss_legendre_rule(64)
    assert abs(p.sum() - 1.0) < 1e-14
    c = np.array([0.0, 0.5, 3.0, 10.0])
    approx = (p[None, :] / (s[None, :] + 1.0 + c[:, None])).sum(1)
    assert np.max(np.abs(approx / _f2(c) - 1.0)) < 1e-6


@pytest.mark.parametrize("lam", [0.0, 0.3, 7.0, 120.0])
def test_theorem2_density_brute_force(lam):
    """int_0^inf p(s) / (s + 1 + lam) ds with p(s) = [pi sqrt(s) (s+1)]^-1 equals f2(lam) (Thm 2, Prop 4)."""
    f = lambda t: 2.0 / (math.pi * (t * t + 1.0) * (t * t + 1.0 + lam))  # s = t^2
    val, _ = integrate.quad(f, 0.0, np.inf, epsabs=1e-14, epsrel=1e-13)
    assert abs(val - _f2(lam)) < 1e-12


def test_ell_rule_powers_of_ten():
    C = np.array([[3.0, -1.0], [-1.0, 2.0]])
    assert quadrature.gershgorin_bound(C) == 4.0
    assert quadrature.ell_rule(C) == 10.0
    assert quadrature.ell_rule(np.array([[10.0]])) == 100.0     # strictly above b
    assert quadrature.ell_rule(np.array([[99.0, 2.0], [2.0, 1.0]])) == 1000.0
    assert quadrature.ell_rule(np.zeros((3, 3))) == 10.0
    lam_max = np.linalg.eigvalsh(C)[-1]
    assert quadrature.ell_rule(C) > lam_max


@pytest.mark.parametrize("Q,ell,bound", [(24, 1e6, 1e-11), (32, 1e8, 1e-11), (48, 1e10, 1e-12)])
def test_elliptic_rule_at_large_ell_meets_the_identity(Q, ell, bound):
    """Above ell = 1e4 the oracle evaluates the elliptic functions in extended precision; the rule must still
    satisfy sum_q r_q / (s_q + c + 1) = (c + 1)^-1/2 over c in [0, ell] (Eq. generic_invsqrt_integral)."""
    pytest.importorskip("mpmath")
    s, p = quadrature.elliptic_rule(Q, ell)
    r = p * (s + 1.0)
    c = np.concatenate([[0.0], np.logspace(-4, math.log10(ell), 300)])
    err = np.max(np.abs((r[None, :] / (s[None, :] + c[:, None] + 1.0)).sum(1) * np.sqrt(c + 1.0) - 1.0))
    assert err < bound
    assert np.all(np.diff(s) > 0) and np.all(p > 0)


def test_extended_precision_rule_agrees_with_scipy_where_both_are_accurate():
    pytest.importorskip("mpmath")
    for Q, ell in ((16, 100.0), (32, 1e4)):
        s1, p1 = quadrature._elliptic_rule_mp(Q, ell)
        s2, p2 = quadrature.elliptic_rule(Q, ell)
        assert np.max(np.abs(s1 / s2 - 1)) < 1e-12 and np.max(np.abs(p1 / p2 - 1)) < 1e-12
