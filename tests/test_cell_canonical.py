"""The cell enumeration's canonical-pair rule, checked on the host against
the oracle (Sec. IV-C).

The GPU writes a cell (an n-simplex that contains a traced edge) only from
its canonical pair: the first pair of in-domain vertices of opposite sign in
the cell's vertex order z, z + e(pi_0), ...  The rule relies on every such
pair being a traced edge: within a cell, the pairs of opposite sign are
connected through crossing triangles whose vertices are all in the domain,
and the search follows those.  This test enumerates the n-cofaces of the
oracle's traced edges (oracle.edge_ncofaces), applies the rule, and checks
that every oracle cell comes out exactly once."""
import numpy as np
import pytest

import oracle
from paper_2406_04795_gb300 import workloads as W


def _canonical(signs):
    """First (i, j), i < j, with both in the domain and opposite signs;
    signs[k] is None (outside) or f >= 0."""
    n = len(signs)
    for i in range(n):
        if signs[i] is None:
            continue
        for j in range(i + 1, n):
            if signs[j] is not None and signs[j] != signs[i]:
                return i, j
    return None


@pytest.mark.parametrize("d,n_sv,seed,lam", [(3, 30, 5, 0.3), (4, 24, 9, 0.45)])
def test_each_cell_written_once_by_its_canonical_pair(d, n_sv, seed, lam):
    w = W.random_small(d, n_sv, seed, lam, n_seeds=2)
    r = oracle.trace(w.sv, w.alpha, w.gamma, w.b, w.lam, w.offset, w.lo, w.hi, w.seeds,
                     roots=False, cells=True)
    E = r["edge_y"].shape[0]
    assert E > 50
    allp = (1 << (d + 1)) - 1
    cache = {}

    def sign(v):
        key = tuple(int(a) for a in v)
        if key not in cache:
            x = oracle.vertex_x(d, w.lam, w.offset, np.array(v))
            inside = bool(np.all((x >= w.lo) & (x <= w.hi)))
            cache[key] = (oracle.f(w.sv, w.alpha, w.gamma, w.b, x)[0] >= 0) if inside else None
        return cache[key]

    written = []
    for y, m in zip(r["edge_y"], r["edge_mask"].astype(np.int64)):
        ends = {tuple(int(a) for a in y), tuple(int(a) + ((int(m) >> k) & 1)
                                                for k, a in enumerate(y))}
        for cy, cparts in oracle.edge_ncofaces(d, y, (int(m), allp ^ int(m))):
            z, parts = oracle.canonicalize(d, cy, cparts)
            verts = [tuple(int(a) for a in v) for v in oracle.simplex_vertices(d, z, parts)]
            pair = _canonical([sign(v) for v in verts])
            assert pair is not None  # the edge itself is such a pair
            if {verts[pair[0]], verts[pair[1]]} == ends:
                perm = tuple(int(p).bit_length() - 1 for p in parts[:d])
                written.append((tuple(int(a) for a in z), perm))
    ref = {(tuple(int(a) for a in cy), tuple(int(a) for a in cp))
           for cy, cp in zip(r["cell_y"], r["cell_perm"])}
    assert len(written) == len(set(written))
    assert set(written) == ref


@pytest.mark.parametrize("d,n_sv,seed,lam", [(3, 30, 5, 0.3), (4, 24, 9, 0.45), (5, 20, 3, 0.6)])
def test_canonical_pair_conditions(d, n_sv, seed, lam):
    """The enumeration writes exactly the cofaces where (y, y + e(S)) is the
    canonical pair, and it reaches them through two conditions on the
    cell's vertex order (y at position a, y + e(S) at a + |S|):
      A: every vertex before y is outside the domain;
      B: every vertex strictly between them is outside or has y's sign.
    Checked here against the canonical rule itself on the oracle's traced
    edges and all their n-cofaces."""
    w = W.random_small(d, n_sv, seed, lam, n_seeds=2)
    r = oracle.trace(w.sv, w.alpha, w.gamma, w.b, w.lam, w.offset, w.lo, w.hi, w.seeds,
                     roots=False, cells=False)
    assert r["edge_y"].shape[0] > 30
    allp = (1 << (d + 1)) - 1
    cache = {}

    def sign(v):
        if v not in cache:
            x = oracle.vertex_x(d, w.lam, w.offset, np.array(v))
            inside = bool(np.all((x >= w.lo) & (x <= w.hi)))
            cache[v] = (oracle.f(w.sv, w.alpha, w.gamma, w.b, x)[0] >= 0) if inside else None
        return cache[v]

    seen_true = seen_false = 0
    for y, m in zip(r["edge_y"][:60], r["edge_mask"][:60].astype(np.int64)):
        y0 = tuple(int(a) for a in y)
        y1 = tuple(int(a) + ((int(m) >> k) & 1) for k, a in enumerate(y))
        n1 = bin(int(m)).count("1")
        for cy, cparts in oracle.edge_ncofaces(d, y, (int(m), allp ^ int(m))):
            z, parts = oracle.canonicalize(d, cy, cparts)
            verts = [tuple(int(a) for a in v) for v in oracle.simplex_vertices(d, z, parts)]
            sg = [sign(v) for v in verts]
            a, b = verts.index(y0), verts.index(y1)
            assert b - a == n1
            cond = all(sg[i] is None for i in range(a)) and \
                all(sg[i] is None or sg[i] == sg[a] for i in range(a + 1, b))
            pair = _canonical(sg)
            assert (pair == (a, b)) == cond
            seen_true += cond
            seen_false += not cond
    assert seen_true > 0 and seen_false > 0
