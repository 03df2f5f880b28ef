"""Pins of the sparse same-node oracle (oracle/sparse.py) against the dense one.

The dense oracle is itself pinned by closed forms (test_oracle_filter.py); the
sparse form must give the same analysis on every geometry it covers: 1-D
periodic (chordal and minimum-image), 2-D periodic, layered (periodic x,
non-periodic z with its own half-width), ragged sizes, and a support that
wraps the whole axis.  Its pair enumeration is also checked directly against
the dense localization matrix.
"""
import numpy as np
import pytest

from oracle import filter as F
from oracle import localization
from oracle import sparse as S
from paper_2503_00253_gb300 import workloads


def _grid(shape, periodic, hw, chordal=True):
    return workloads.Grid(shape, periodic, hw, chordal)


GRIDS = [
    ("1d_chordal", _grid((301, 1, 1), (True, False, False), (9.0, 1.0, 1.0))),
    ("1d_min_image", _grid((256, 1, 1), (True, False, False), (11.0, 1.0, 1.0), chordal=False)),
    ("1d_whole_axis", _grid((40, 1, 1), (True, False, False), (15.0, 1.0, 1.0))),
    ("2d", _grid((24, 18, 1), (True, True, False), (3.0, 2.5, 1.0))),
    ("layered", _grid((30, 1, 5), (True, False, False), (4.0, 1.0, 1.3))),
]


@pytest.mark.parametrize("name,grid", GRIDS)
def test_support_pairs_equal_the_dense_localization(name, grid):
    rng = np.random.default_rng(3)
    n = int(np.prod(grid.shape))
    rows = np.sort(rng.choice(n, size=min(n, 97), replace=False))
    cols = np.sort(rng.choice(n, size=min(n, 83), replace=False))
    i, j, L = S.support_pairs(grid, rows, cols)
    dense = np.zeros((rows.size, cols.size))
    dense[i, j] = L
    assert np.array_equal(dense, localization.localization_matrix(grid, rows, cols))
    # no pair is listed twice
    assert len(set(zip(i.tolist(), j.tolist()))) == i.size


@pytest.mark.parametrize("name,grid", GRIDS)
def test_sparse_analysis_equals_dense(name, grid):
    rng = np.random.default_rng(11)
    n = int(np.prod(grid.shape))
    N, Q = 9, 7
    X = np.cumsum(rng.standard_normal((N, n)), axis=1) / np.sqrt(n) + rng.standard_normal((N, n))
    obs = np.sort(rng.choice(n, size=max(1, n // 3), replace=False)).astype(np.int64)
    R = rng.uniform(0.2, 2.0, obs.size)
    y = rng.standard_normal(obs.size)
    A_d = F.perturbation_update(X, obs, R, grid, Q)
    A_s = S.perturbation_update(X, obs, R, grid, Q)
    Af = X - X.mean(0)
    assert F.relative_increment_error(A_s, A_d, Af) < 1e-12
    mu_d = F.mean_update(X, obs, y, R, grid)
    mu_s = S.mean_update(X, obs, y, R, grid)
    assert np.max(np.abs(mu_s - mu_d)) < 1e-12 * np.max(np.abs(mu_d - X.mean(0)))
    # the same ell rule on the same C
    _, Z = F.anomalies(X)
    _, _, Shh = F.localized_covariances(Z, obs, grid)
    assert S.ell_rule(S.localized_covariances(Z, obs, grid)[2], R) == F.choose_ell(Shh, R)


def test_sparse_analysis_equals_dense_on_a_1d_gaussian_forecast():
    pr = workloads.gaussian_problem_1d("sp", n=1500, N=16, length_scale=12.0, obs_stride=4, r2=0.3,
                                       half_width=30.0, Q=12, tol=1e-12, seed=5)
    A_d = F.perturbation_update(pr.X, pr.obs_idx, pr.R, pr.grid, pr.Q)
    A_s = S.perturbation_update(pr.X, pr.obs_idx, pr.R, pr.grid, pr.Q)
    assert F.relative_increment_error(A_s, A_d, pr.X - pr.X.mean(0)) < 1e-12
