"""Quadrature rules for the integral-form update (oracle; test infrastructure only).

Theorem 3 lets any (I, r_t, s_t) with int r_t / (s_t + c + 1) dt = (c+1)^-1/2
for c in a neighbourhood of spec(C) u {0} define the update; the weights are
p_t = r_t / (s_t + 1).  App. D gives two discretisations.

Elliptic rule (App. D, Eq. elliptic_quadrature_rule).  As printed, the
interval is (0, K(g)) with g = sqrt(1 - (1+ell)^-1) and the nodes are
|sn(i t_q K(g) | g)|^2.  Read literally (modulus g for the imaginary-argument
functions) the integrand has a pole inside (0, K(g)) and the rule diverges.
Reading taken here: the imaginary-argument functions carry the complementary
modulus g' = (1+ell)^-1/2, which is the Hale-Higham-Trefethen setting the
paper cites (their k^2 = m/M with spectrum [1, 1+ell]).  Jacobi's imaginary
transformation then gives real-argument functions of modulus g on the
paper's interval (0, K(g)):

    |sn(iu | g')|^2 = sc(u | g)^2,  cn(iu | g') = nc(u | g),  dn(iu | g') = dc(u | g)

    s_q = sc(t_q K | g)^2
    r_q = (2 / (pi Q)) K nc(t_q K | g) dc(t_q K | g)
    p_q = r_q / (s_q + 1)                  with t_q = (q - 1/2) / Q,  K = K(g).

This reading reproduces the convergence the paper states
(Q = O(log(1/eps) log ell)); the alternative reading (interval (0, K(g'))
with modulus g') is exact as Q -> infinity too but converges far more slowly
for large ell.  SciPy's ellipj/ellipk take the parameter m = g^2.

Gauss-Legendre rule (Eq. gaussian_quadrature_rule): I = (0, 1),
s_q = tan^2(pi lambda_q / 2), p_q = v_q / 2 with (lambda_q, v_q) the
Gauss-Legendre nodes mapped to (0, 1) and weights on (-1, 1).

Choice of ell (App. D asks for a rough order-of-magnitude estimate above
lambda_max(C), fixed in advance).  Rule used when the caller gives none:
b = max_a sum_b |C_ab| (a Gershgorin bound, so b >= lambda_max(C)) and
ell = 10^(floor(log10(max(b, 1))) + 1), a power of ten strictly above b.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import ellipj, ellipk


def _elliptic_rule_mp(Q: int, ell: float, digits: int = 40):
    """The same rule with the elliptic functions evaluated by mpmath at `digits`
    significant digits and the parameter m = ell / (1 + ell) formed exactly.
    For large ell, m is within 1/ell of 1 and SciPy's double-precision
    ellipk / ellipj lose digits (K off by about 3e-12 at ell = 1e6, 2e-10 at
    1e8)."""
    import mpmath
    with mpmath.workdps(digits):
        L = mpmath.mpf(ell)
        m = L / (1 + L)
        K = mpmath.ellipk(m)
        s = np.empty(Q)
        p = np.empty(Q)
        for q in range(1, Q + 1):
            u = (q - mpmath.mpf(1) / 2) / Q * K
            sn, cn, dn = (mpmath.ellipfun(f, u, m=m) for f in ("sn", "cn", "dn"))
            sq = (sn / cn) ** 2
            rq = 2 / (mpmath.pi * Q) * K / cn * (dn / cn)
            s[q - 1] = float(sq)
            p[q - 1] = float(rq / (sq + 1))
    return s, p


def elliptic_rule(Q: int, ell: float):
    """(s_q, p_q), q = 1..Q, of the elliptic rule (App. D) for spectrum bound ell.
    Above ell = 1e4 the elliptic functions are evaluated in extended precision
    (_elliptic_rule_mp); below, SciPy's are accurate to rounding."""
    if Q < 1 or not ell > 0:
        raise ValueError("need Q >= 1 and ell > 0")
    if ell > 1e4:
        return _elliptic_rule_mp(Q, ell)
    g2 = 1.0 - 1.0 / (1.0 + ell)           # parameter m = g^2, g as printed in App. D
    K = ellipk(g2)
    t = (np.arange(1, Q + 1) - 0.5) / Q
    sn, cn, dn, _ = ellipj(t * K, g2)
    s = (sn / cn) ** 2                      # |sn(i t K | g')|^2 = sc(t K | g)^2
    r = (2.0 / (math.pi * Q)) * K * (1.0 / cn) * (dn / cn)   # K nc dc
    p = r / (s + 1.0)
    return s, p


def gauss_legendre_rule(Q: int):
    """(s_q, p_q) of the Gauss-Legendre rule on the trigonometric form (App. D)."""
    x, v = np.polynomial.legendre.leggauss(Q)
    lam = 0.5 * (x + 1.0)
    s = np.tan(0.5 * math.pi * lam) ** 2
    p = 0.5 * v
    return s, p


def quadrature(Q: int, ell: float, rule: str = "elliptic"):
    if rule == "elliptic":
        return elliptic_rule(Q, ell)
    if rule == "gauss_legendre":
        return gauss_legendre_rule(Q)
    raise ValueError(rule)


def gershgorin_bound(C: np.ndarray) -> float:
    return float(np.max(np.sum(np.abs(C), axis=1))) if C.size else 0.0


def ell_rule(C: np.ndarray) -> float:
    """Power of ten strictly above the Gershgorin bound of C (at least 10)."""
    b = max(gershgorin_bound(C), 1.0)
    return float(10.0 ** (math.floor(math.log10(b)) + 1))


def scalar_gain(sigma_xh: float, sigma_hh: float, r: float = 1.0) -> float:
    """Scalar modified gain G = s_xh / (r + s_hh + r sqrt(1 + s_hh / r)) (Eq. modified_gain)."""
    return sigma_xh / (r + sigma_hh + r * math.sqrt(1.0 + sigma_hh / r))
