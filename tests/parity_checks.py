"""Error measures of the end-to-end parity tests (not the method's arithmetic).

Every GPU analysis is compared with the oracle's same-node result (Sec. 3.2,
exact solves per quadrature node) through its increment, the part of the
output the update produces: dA = A_a - A_f for the perturbations and
dmu = mu_a - mu_f for the mean.  Two measures are taken and the larger is
returned, so one bound in a test covers both:

- the Frobenius ratio ||dA_gpu - dA_ref||_F / ||dA_ref||_F over all members;
- an element-wise bound per member i,
      max_x |dA_gpu[i, x] - dA_ref[i, x]| / max_x |dA_ref[i, x]|,
  maximised over members, so that a single wrong state point (or a single
  wrong member) fails the test even when it is lost in the norm.

Since dA_gpu - dA_ref = A_gpu - A_ref, no forecast subtraction enters the
numerators.
"""
from __future__ import annotations

import numpy as np


def _np(a):
    if hasattr(a, "detach"):
        a = a.detach().cpu().numpy()
    return np.asarray(a, dtype=np.float64)


def increment_error(A_gpu, A_ref, A_f) -> float:
    """max(Frobenius ratio, per-member element-wise ratio) of the perturbation increment."""
    A_gpu, A_ref, A_f = _np(A_gpu), _np(A_ref), _np(A_f)
    diff = A_gpu - A_ref
    inc = A_ref - A_f
    frob = float(np.linalg.norm(diff) / np.linalg.norm(inc))
    scale = np.abs(inc).max(axis=1)
    elem = float(np.max(np.abs(diff).max(axis=1) / scale))
    return max(frob, elem)


def mean_error(mu_gpu, mu_ref, mu_f) -> float:
    """max(2-norm ratio, element-wise ratio) of the mean increment."""
    mu_gpu, mu_ref, mu_f = _np(mu_gpu), _np(mu_ref), _np(mu_f)
    diff = mu_gpu - mu_ref
    inc = mu_ref - mu_f
    return max(float(np.linalg.norm(diff) / np.linalg.norm(inc)),
               float(np.abs(diff).max() / np.abs(inc).max()))
