"""Pins against values the paper prints (fixtures under tests/golden/, each
file states its source)."""
import os

import numpy as np

from oracle import fem

HERE = os.path.dirname(os.path.abspath(__file__))


def _table(name):
    rows = []
    for line in open(os.path.join(HERE, "golden", name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append([int(v) for v in line.split()])
    return np.array(rows)


def test_table1_dof_counts():
    """Table 1: velocity and vertex-pressure counts equal the Q2 / Q1 lattice
    sizes of the oracle's grid; the P2-P1* frame adds 2n^2 centroids, the
    Q2-Q1* frame on quadrilaterals adds n^2 element constants."""
    for lev, nvel, np1, npstar in _table("table1_dofs.txt"):
        n = 2 ** lev
        g = fem.Grid(n)
        assert g.nu == nvel
        assert g.n1 == np1
        assert npstar == np1 + 2 * n * n
        assert g.np_ == np1 + n * n
