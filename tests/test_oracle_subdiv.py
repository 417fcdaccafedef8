"""Pins of the oracle's batch triangulation (Sec. V-B, Figs. 5-6, Eqs. bc and
local), CPU only.

- The local template: its vertices are exactly the lattice points of scale
  lam inside the reference n-simplex of scale k lam, found by barycentric
  coordinates of their C-space coordinates (not by Eq. local); there are
  C(k+d, d) of them, k^d Kuhn simplices of scale lam fill it, and its edges
  are exactly the vertex pairs (y, y + e(M)) inside it.  Fig. 5's first local
  edge belongs to it.
- The batch-triangulated set equals its definition computed by brute force:
  every crossing edge of scale lam in the box whose two vertices lie in a
  crossing n-simplex of the coarse trace (barycentric coordinates in C-space).
- The paper's claim that the result matches the fine triangulation: on the
  sphere at k = 3 it equals the direct trace at lam exactly, and otherwise it
  is a subset of it here (it misses fine crossings inside coarse simplices
  whose vertices all share a sign); roots equal the direct trace's."""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2406_04795_gb300 import workloads as W
from tests import _brute as B


def _kset(r):
    return {(tuple(int(v) for v in y), int(m)) for y, m in zip(r["edge_y"], r["edge_mask"])}


def _bary(P, x):
    return B.barycentric(P, x)


@pytest.mark.parametrize("d,k", [(2, 1), (2, 2), (2, 4), (3, 2), (3, 3), (4, 2), (5, 2)])
def test_template_is_the_fine_lattice_inside_the_coarse_simplex(d, k):
    lam, o = 0.1, np.zeros(d)
    v, e = oracle.subdiv_template(d, k)
    assert len(v) == math.comb(k + d, d)
    # reference coarse simplex z = 0, pi = identity: vertices k * (e_0 + ... + e_{j-1})
    Vc = np.array([[k if i < j else 0 for i in range(d)] for j in range(d + 1)], dtype=np.int32)
    Xc = oracle.vertex_x(d, lam, o, Vc)
    inside = set()
    for y in itertools.product(range(0, k + 1), repeat=d):
        x = oracle.vertex_x(d, lam, o, np.array([y], np.int32))[0]
        if np.all(_bary(Xc, x) >= -1e-9):
            inside.add(tuple(y))
    # local v' -> y = sum_j v'_j e_j (identity permutation)
    got = {tuple(int(a) for a in m) for m in v}
    assert got == inside
    # edges: all pairs (y, y + e(M)) with both ends inside
    want = {(y, M) for y in inside for M in range(1, 1 << d)
            if tuple(y[i] + ((M >> i) & 1) for i in range(d)) in inside}
    have = {(tuple(int(a) for a in v[i]), int(M)) for i, M in e}
    assert have == want
    # k^d Kuhn simplices of scale lam lie inside
    n_kuhn = 0
    for z in itertools.product(range(0, k), repeat=d):
        for pi in itertools.permutations(range(d)):
            if all(tuple(p) in inside for p in B.kuhn_vertices(z, pi)):
                n_kuhn += 1
    assert n_kuhn == k ** d
    if k == 2 and d in (2, 3):  # Fig. 5: the first local edge v' = 0, p = {{0}, {1..n}}
        assert (tuple([0] * d), 1) in have


@pytest.mark.parametrize("d,lam,k,n_sv,seed", [(2, 0.06, 2, 12, 2), (3, 0.12, 2, 10, 3),
                                               (3, 0.1, 3, 10, 4)])
def test_subdiv_equals_brute_force_definition(d, lam, k, n_sv, seed):
    w = W.random_small(d, n_sv, seed, lam, gamma=1.5, n_seeds=4, box=1.2)
    s = oracle.subdiv(w.sv, w.alpha, w.gamma, w.b, w.lam, k, w.offset, w.lo, w.hi, w.seeds)
    co = oracle.trace(w.sv, w.alpha, w.gamma, w.b, k * w.lam, w.offset, w.lo, w.hi, w.seeds,
                      roots=False, cells=True)
    assert s["n_coarse_cells"] == len(co["cell_y"]) > 10
    c = oracle.lattice_c(d)

    def fv(X):
        return oracle.f(w.sv, w.alpha, w.gamma, w.b, X)

    cross = B.brute_crossing_edges(d, w.lam, c, w.offset, w.lo, w.hi, fv)
    # coarse cells in C-space
    cells = []
    for z, perm in zip(co["cell_y"], co["cell_perm"]):
        parts = tuple(1 << int(p) for p in perm) + (1 << d,)
        Vc = np.array(oracle.simplex_vertices(d, z, parts), np.int32)
        cells.append(oracle.vertex_x(d, k * w.lam, w.offset, Vc))
    # barycentric coordinates of both vertices of every crossing edge in
    # every coarse cell (one linear solve per cell)
    keys = sorted(cross)
    ya = np.array([y for y, _ in keys], np.int32)
    yb = ya + np.array([[(m >> i) & 1 for i in range(d)] for _, m in keys], np.int32)
    Xa = oracle.vertex_x(d, w.lam, w.offset, ya)
    Xb = oracle.vertex_x(d, w.lam, w.offset, yb)
    ok = np.zeros(len(keys), bool)
    for Xc in cells:
        A = np.vstack([Xc.T, np.ones(d + 1)])
        Ai = np.linalg.inv(A)
        wa = Ai @ np.vstack([Xa.T, np.ones(len(keys))])
        wb = Ai @ np.vstack([Xb.T, np.ones(len(keys))])
        ok |= np.all(wa >= -1e-9, axis=0) & np.all(wb >= -1e-9, axis=0)
    want = {k for k, o in zip(keys, ok) if o}
    assert _kset(s) == want and len(want) > 50


def test_subdiv_matches_fine_trace_on_the_sphere():
    w = W.sphere_workload(3, r=1.0, gamma=1.0, lam=0.1)
    direct = oracle.trace(w.sv, w.alpha, w.gamma, w.b, w.lam, w.offset, w.lo, w.hi, w.seeds,
                          cells=False)
    s3 = oracle.subdiv(w.sv, w.alpha, w.gamma, w.b, w.lam, 3, w.offset, w.lo, w.hi, w.seeds)
    assert _kset(s3) == _kset(direct) and len(s3["edge_t"]) > 5000
    # roots: the same bisection on the same edges
    dm = {k: i for i, k in enumerate(zip(map(tuple, direct["edge_y"].tolist()),
                                         direct["edge_mask"].tolist()))}
    idx = [dm[k] for k in zip(map(tuple, s3["edge_y"].tolist()), s3["edge_mask"].tolist())]
    assert np.array_equal(s3["edge_t"], direct["edge_t"][idx])
    assert np.max(np.abs(np.linalg.norm(s3["edge_pt"], axis=1) - 1.0)) < 1e-12
    s2 = oracle.subdiv(w.sv, w.alpha, w.gamma, w.b, w.lam, 2, w.offset, w.lo, w.hi, w.seeds)
    assert _kset(s2) <= _kset(direct)
    assert len(_kset(direct) - _kset(s2)) < 0.01 * len(direct["edge_t"])
