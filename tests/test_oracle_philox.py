"""Pin of the oracle's Philox4x32-10 against published known-answer vectors."""
import os

import numpy as np

from oracle import philox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append([int(v, 16) for v in line.split()])
    assert len(rows) == 3
    for row in rows:
        out = philox.philox4x32_10(np.array([row[:4]], dtype=np.uint32), row[4:6])
        assert [int(v) for v in out[0]] == row[6:10]


def test_normals_moments_and_layout():
    g = philox.normals(200001, seed=12345)
    assert abs(g.mean()) < 0.01 and abs(g.std() - 1.0) < 0.01
    Om = philox.test_matrix(7, 3, seed=9)
    flat = philox.normals(21, seed=9)
    assert Om[4, 2] == flat[2 * 7 + 4]
