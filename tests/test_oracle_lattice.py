"""Pins of the oracle's lattice and permutahedral queries (CPU only).

Worked examples printed in the paper (Fig. 2, Fig. 5), closed forms of the
Ã_d realisation, and brute force over Kuhn simplices.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from tests import _brute as B

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _parse_golden(name):
    rows = []
    with open(os.path.join(GOLD, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            v, p, verts = [s.strip() for s in line.split(";")]
            y = [int(t) for t in v.split(",")]
            parts = [[int(t) for t in grp.split(",")] for grp in p.split("|")]
            vs = [tuple(int(t) for t in w.split(",")) for w in verts.split()]
            rows.append((y, parts, vs))
    return rows


def test_fig2_triangles_of_the_unit_square():
    rows = _parse_golden("fig2_permutahedral_2d.txt")
    assert len(rows) == 2
    for y, parts, verts in rows:
        got = oracle.simplex_vertices(2, y, oracle.parts_from_sets(parts))
        assert [tuple(r) for r in got] == verts


def test_fig5_first_local_edge():
    for y, parts, verts in _parse_golden("fig5_first_local_edge.txt"):
        d = len(y)
        got = oracle.simplex_vertices(d, y, oracle.parts_from_sets(parts))
        assert [tuple(r) for r in got] == verts


@pytest.mark.parametrize("d", [2, 3, 4, 5, 6, 7, 8])
def test_lattice_steps_form_a_regular_simplex(d):
    # the d+1 steps e_0..e_{d-1}, e_d = -1 map to vectors of equal length
    # lam^2 d/(d+1) with pairwise inner products -lam^2/(d+1)
    lam = 0.37
    o = np.zeros(d)
    x0 = oracle.vertex_x(d, lam, o, np.zeros(d, np.int32))[0]
    steps = []
    for i in range(d):
        y = np.zeros(d, np.int32)
        y[i] = 1
        steps.append(oracle.vertex_x(d, lam, o, y)[0] - x0)
    steps.append(oracle.vertex_x(d, lam, o, -np.ones(d, np.int32))[0] - x0)
    G = np.array(steps) @ np.array(steps).T
    expect = lam * lam * (np.eye(d + 1) * (d / (d + 1) + 1 / (d + 1)) - 1 / (d + 1))
    np.testing.assert_allclose(G, expect, atol=1e-14)


@pytest.mark.parametrize("d", [2, 3, 4, 5, 6])
def test_edge_lengths_closed_form(d):
    rng = np.random.default_rng(d)
    lam = 0.05 * (1 + d)
    o = rng.uniform(-0.1, 0.1, d)
    for _ in range(50):
        y = rng.integers(-20, 20, size=d).astype(np.int32)
        S = int(rng.integers(1, 1 << d))
        vs = oracle.simplex_vertices(d, y, (S, ((2 << d) - 1) & ~S))
        xs = oracle.vertex_x(d, lam, o, vs)
        k = bin(S).count("1")
        assert np.sum((xs[1] - xs[0]) ** 2) == pytest.approx(lam * lam * k * (d + 1 - k) / (d + 1),
                                                            rel=1e-12)


@pytest.mark.parametrize("d", [2, 3, 4, 5])
def test_d2_equilateral_d3_disphenoid_equal_volumes(d):
    lam = 1.0
    o = np.zeros(d)
    vol = []
    for pi in itertools.permutations(range(d)):
        parts = tuple(1 << p for p in pi) + (1 << d,)
        vs = oracle.simplex_vertices(d, np.zeros(d, np.int32), parts)
        xs = oracle.vertex_x(d, lam, o, vs)
        vol.append(abs(np.linalg.det(xs[1:] - xs[0])) / math.factorial(d))
        lens = sorted(np.linalg.norm(xs[i] - xs[j]) for i in range(d + 1) for j in range(i))
        if d == 2:
            np.testing.assert_allclose(lens, [math.sqrt(2 / 3)] * 3, rtol=1e-12)
        if d == 3:  # Sommerville tetrahedron: four edges sqrt(3)/2, two edges 1
            np.testing.assert_allclose(lens, [math.sqrt(3) / 2] * 4 + [1.0, 1.0], rtol=1e-12)
    # det(L) = 1/sqrt(d+1): every n-simplex has volume 1/(d! sqrt(d+1))
    np.testing.assert_allclose(vol, 1.0 / (math.factorial(d) * math.sqrt(d + 1)), rtol=1e-10)


@pytest.mark.parametrize("d", [2, 3, 4, 5, 6])
def test_locate_barycentric_nonnegative(d):
    rng = np.random.default_rng(10 + d)
    lam = 0.1
    o = rng.uniform(-0.05, 0.05, d)
    for _ in range(200):
        x = rng.uniform(-3, 3, d)
        y, parts = oracle.locate(d, lam, o, x)
        assert len(parts) == d + 1 and parts[-1] == 1 << d
        assert sorted(parts) == sorted(1 << i for i in range(d + 1))
        vs = oracle.simplex_vertices(d, y, parts)
        bc = B.barycentric(oracle.vertex_x(d, lam, o, vs), x)
        assert bc.min() >= -1e-12, bc


def test_locate_ties_give_a_containing_simplex():
    d = 3
    lam = 1.0
    o = np.zeros(d)
    # points on lattice vertices and on shared faces
    for y in ([0, 0, 0], [1, 2, 3], [-1, 0, 2]):
        x = oracle.vertex_x(d, lam, o, np.array(y, np.int32))[0]
        for p in (x, x + 0.5 * (oracle.vertex_x(d, lam, o, np.array(y, np.int32) + 1)[0] - x)):
            yy, parts = oracle.locate(d, lam, o, p)
            vs = oracle.simplex_vertices(d, yy, parts)
            bc = B.barycentric(oracle.vertex_x(d, lam, o, vs), p)
            assert bc.min() >= -1e-12


def _vset(d, y, parts):
    return frozenset(tuple(r) for r in oracle.simplex_vertices(d, y, parts))


@pytest.mark.parametrize("d", [2, 3, 4, 5])
def test_cofaces_equal_brute_force(d):
    rng = np.random.default_rng(20 + d)
    all_ = (2 << d) - 1
    for S in range(1, 1 << d):
        y = tuple(int(v) for v in rng.integers(-5, 5, size=d))
        edge = (y, (S, all_ & ~S))
        tris = oracle.edge_cofaces(d, *edge)
        a, b = [tuple(r) for r in oracle.simplex_vertices(d, *edge)]
        got = {_vset(d, *t) for t in tris}
        assert len(got) == len(tris)  # no duplicates
        assert got == B.triangles_containing_edge(a, b)
        k1, k2 = bin(S).count("1"), d + 1 - bin(S).count("1")
        assert len(tris) == (2 ** k1 - 2) + (2 ** k2 - 2)  # Sec. IV-A count
        for t in tris:
            assert t[1][-1] >> d & 1  # canonical: d in the last part
            es = oracle.triangle_edges(d, *t)
            assert len(es) == 3
            assert (y, edge[1]) in [(tuple(e[0]), e[1]) for e in es]  # face round trip


@pytest.mark.parametrize("d", [2, 3, 4, 5])
def test_ncofaces_equal_brute_force(d):
    rng = np.random.default_rng(30 + d)
    all_ = (2 << d) - 1
    for S in range(1, 1 << d):
        y = tuple(int(v) for v in rng.integers(-5, 5, size=d))
        cells = oracle.edge_ncofaces(d, y, (S, all_ & ~S))
        a, b = [tuple(r) for r in oracle.simplex_vertices(d, y, (S, all_ & ~S))]
        got = {_vset(d, *c) for c in cells}
        assert len(got) == len(cells)
        assert got == B.nsimplices_containing_edge(a, b)
        k1 = bin(S).count("1")
        assert len(cells) == math.factorial(k1) * math.factorial(d + 1 - k1)  # Sec. IV-C count


@pytest.mark.parametrize("d", [2, 3, 4, 5, 6])
def test_nsimplex_edges_are_all_vertex_pairs(d):
    rng = np.random.default_rng(40 + d)
    for _ in range(20):
        pi = rng.permutation(d)
        y = rng.integers(-4, 4, size=d)
        parts = tuple(1 << int(p) for p in pi) + (1 << d,)
        vs = [tuple(r) for r in oracle.simplex_vertices(d, y, parts)]
        es = oracle.nsimplex_edges(d, y, parts)
        assert len(es) == (d + 1) * d // 2  # erratum of Sec. IV-A's n(n-1)/2
        pairs = {_vset(d, *e) for e in es}
        assert pairs == {frozenset((vs[i], vs[j])) for i in range(d + 1) for j in range(i)}


def test_canonical_rotation_keeps_the_vertex_set():
    d = 4
    rng = np.random.default_rng(5)
    for _ in range(100):
        k = int(rng.integers(1, d + 1))
        labels = rng.integers(0, k + 1, size=d + 1)
        labels[:k + 1] = np.arange(k + 1)
        rng.shuffle(labels)
        parts = tuple(int(sum(1 << i for i in range(d + 1) if labels[i] == g)) for g in range(k + 1))
        y = rng.integers(-3, 3, size=d)
        cy, cp = oracle.canonicalize(d, y, parts)
        assert cp[-1] >> d & 1
        assert _vset(d, cy, cp) == _vset(d, y, parts)
