"""Host-side logic of the CUDA library that runs without a GPU.

The exact lattice domain table (mf_domain_table) must reproduce, vertex by
vertex, the oracle's decision "x(y) lies in the closed box", for vertices deep
inside, outside and on the boundary of the box."""
import math

import numpy as np
import pytest

import oracle
from paper_2406_04795_gb300 import mf
from paper_2406_04795_gb300 import workloads as W


def _dom(lo, hi, off):
    d = mf.mf_domain()
    for i in range(len(lo)):
        d.lo[i], d.hi[i], d.offset[i] = float(lo[i]), float(hi[i]), float(off[i])
    return d


@pytest.mark.parametrize("d,lam,box", [(2, 0.1, 1.0), (3, 0.1, math.pi), (4, 0.3, 1.3),
                                       (5, 0.05, math.pi), (6, 0.2, 2.0)])
def test_domain_table_matches_oracle_box_test(d, lam, box):
    rng = np.random.default_rng(d)
    lo = -box * np.ones(d) + rng.uniform(-0.05, 0.05, d)
    hi = box * np.ones(d) + rng.uniform(-0.05, 0.05, d)
    off = W.lattice_offset(d, lam)
    smin, tab = mf.mf_domain_table(d, lam, _dom(lo, hi, off))
    cinv = oracle.lattice_c(d) * math.sqrt(d + 1)
    # candidate vertices: located points around the box faces, and random ones
    pts = rng.uniform(lo - 3 * lam, hi + 3 * lam, size=(4000, d))
    k = rng.integers(0, d, size=4000)
    side = rng.integers(0, 2, size=4000)
    pts[np.arange(4000), k] = np.where(side, hi[k], lo[k]) + rng.normal(scale=lam, size=4000)
    ys = []
    for p in pts:
        y, _ = oracle.locate(d, lam, off, p)
        ys.append(y)
        ys.append(tuple(v + int(rng.integers(-1, 2)) for v in y))
    ys = np.array(ys, dtype=np.int32)
    X = oracle.vertex_x(d, lam, off, ys)
    inside = np.all((X >= lo) & (X <= hi), axis=1)
    n_in = n_edge = 0
    for y, want in zip(ys, inside):
        s = int(y.sum())
        row = s - smin
        got = 0 <= row < tab.shape[0] and all(tab[row, i, 0] <= y[i] <= tab[row, i, 1]
                                               for i in range(d))
        assert got == bool(want), (y, want)
        n_in += bool(want)
    assert 0 < n_in < len(ys)
    del n_edge, cinv
