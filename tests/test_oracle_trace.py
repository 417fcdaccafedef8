"""Pins of the oracle's manifold tracing, roots and cells (CPU only)."""
import math

import numpy as np
import pytest

import oracle
from paper_2406_04795_gb300 import workloads as W
from tests import _brute as B


def _trace(w, roots=True, cells=True):
    return oracle.trace(w.sv, w.alpha, w.gamma, w.b, w.lam, w.offset, w.lo, w.hi, w.seeds,
                        roots=roots, cells=cells)


def _edge_set(r):
    return {(tuple(int(v) for v in y), int(m)) for y, m in zip(r["edge_y"], r["edge_mask"])}


@pytest.mark.parametrize("d,lam,n_sv,seed", [(2, 0.12, 6, 1), (3, 0.25, 8, 2), (3, 0.3, 5, 3),
                                             (4, 0.45, 6, 4)])
def test_traced_set_equals_brute_force_components(d, lam, n_sv, seed):
    w = W.random_small(d, n_sv, seed, lam, gamma=1.5, n_seeds=3, box=1.2)
    r = _trace(w, roots=False, cells=False)
    c = oracle.lattice_c(d)

    def fv(X):
        return oracle.f(w.sv, w.alpha, w.gamma, w.b, X)

    traced, level = B.brute_trace(d, w.lam, c, w.offset, w.lo, w.hi, fv, w.seeds)
    got = _edge_set(r)
    assert len(got) == len(r["edge_mask"])
    assert got == traced
    # BFS levels are graph distances from the seed edges
    lev = {(tuple(int(v) for v in y), int(m)): int(L)
           for y, m, L in zip(r["edge_y"], r["edge_mask"], r["edge_level"])}
    assert lev == level
    assert r["levels"] == (max(level.values()) + 1 if level else 0)
    # the counters the GPU is compared with bit-exactly, from the same
    # enumeration: vertices evaluated, boundary pairs, near-zero vertices
    nv, nb, nz = B.brute_counts(d, w.lam, c, w.offset, w.lo, w.hi, fv, w.seeds, traced)
    assert (r["n_vertices"], r["n_boundary"], r["n_near_zero"]) == (nv, nb, nz)
    assert nb > 0 or d == 2


def test_lattice_x_matches_numpy_operation_order():
    d, lam = 5, 0.05
    o = W.lattice_offset(d, lam)
    rng = np.random.default_rng(0)
    Y = rng.integers(-200, 200, size=(100, d)).astype(np.int32)
    a = oracle.vertex_x(d, lam, o, Y)
    b = B.lattice_x(d, lam, oracle.lattice_c(d), o, Y)
    assert np.array_equal(a, b)


def test_sphere_d3_roots_euler_and_closed_mesh():
    # one-SV RBF: zero set is exactly |q| = r
    r0 = 1.0
    w = W.sphere_workload(3, r=r0, gamma=1.0, lam=0.2)
    res = _trace(w)
    E = len(res["edge_t"])
    assert E > 100 and res["n_dead_seeds"] == 0 and res["n_boundary"] == 0
    # roots: t solves |x1 + t (x2 - x1)|^2 = r^2 (closed form)
    d = 3
    ys = res["edge_y"]
    x1 = oracle.vertex_x(d, w.lam, w.offset, ys)
    y2 = ys.copy()
    for k in range(d):
        y2[:, k] += (res["edge_mask"] >> k) & 1
    x2 = oracle.vertex_x(d, w.lam, w.offset, y2)
    D = x2 - x1
    a = np.sum(D * D, 1)
    bq = 2 * np.sum(x1 * D, 1)
    cq = np.sum(x1 * x1, 1) - r0 * r0
    disc = np.sqrt(bq * bq - 4 * a * cq)
    t1 = (-bq - disc) / (2 * a)
    t2 = (-bq + disc) / (2 * a)
    t = np.where((t1 >= 0) & (t1 <= 1), t1, t2)
    assert np.max(np.abs(t - res["edge_t"])) < 1e-12
    assert np.max(np.abs(np.linalg.norm(res["edge_pt"], axis=1) - r0)) < 1e-12
    # Euler characteristic of the PL sphere: V - E + F = 2 with V = crossing
    # edges, E = crossing triangles, F = crossing tetrahedra
    T = res["n_crossing_triangles"]
    C = len(res["cell_y"])
    assert E - T + C == 2
    # closed mesh: every crossing triangle lies in exactly two crossing tets;
    # a tet with k crossing edges has k crossing faces, so sum_k = 2 T
    per_cell = np.diff(res["cell_off"])
    assert set(per_cell.tolist()) <= {3, 4}
    assert int(per_cell.sum()) == 2 * T


def test_sphere_d4_and_d5_points_on_sphere():
    for d, lam in ((4, 0.3), (5, 0.45)):
        w = W.sphere_workload(d, r=1.0, gamma=0.7, lam=lam)
        res = _trace(w, cells=False)
        assert len(res["edge_t"]) > 50
        assert np.max(np.abs(np.linalg.norm(res["edge_pt"], axis=1) - 1.0)) < 1e-12


@pytest.mark.parametrize("d", [2, 3, 4])
def test_plane_roots_and_full_crossing_set(d):
    w = W.plane_workload(d, lam=0.25 if d < 4 else 0.4)
    res = _trace(w, cells=False)
    s1, s2 = w.sv
    nrm = s2 - s1
    cst = 0.5 * (s2 @ s2 - s1 @ s1)
    ys = res["edge_y"]
    x1 = oracle.vertex_x(d, w.lam, w.offset, ys)
    y2 = ys.copy()
    for k in range(d):
        y2[:, k] += (res["edge_mask"] >> k) & 1
    x2 = oracle.vertex_x(d, w.lam, w.offset, y2)
    t = (cst - x1 @ nrm) / ((x2 - x1) @ nrm)
    assert np.max(np.abs(t - res["edge_t"])) < 1e-12
    # a hyperplane's crossing edges inside the box are one connected set
    def fv(X):
        return oracle.f(w.sv, w.alpha, w.gamma, w.b, X)
    traced, _ = B.brute_trace(d, w.lam, oracle.lattice_c(d), w.offset, w.lo, w.hi, fv, w.seeds)
    assert _edge_set(res) == traced


def test_crossing_triangles_have_two_crossing_edges():
    w = W.random_small(3, 8, 11, 0.2, gamma=1.5, n_seeds=2, box=1.2)
    res = _trace(w, roots=False, cells=False)
    d = 3
    all_ = (2 << d) - 1
    checked = 0
    for y, m in list(zip(res["edge_y"], res["edge_mask"]))[:200]:
        for ty, tp in oracle.edge_cofaces(d, tuple(int(v) for v in y), (int(m), all_ & ~int(m))):
            vs = oracle.simplex_vertices(d, ty, tp)
            X = oracle.vertex_x(d, w.lam, w.offset, vs)
            if np.any(X < w.lo) or np.any(X > w.hi):
                continue
            s = oracle.f(w.sv, w.alpha, w.gamma, w.b, X) >= 0
            assert int(s[0] != s[1]) + int(s[1] != s[2]) + int(s[0] != s[2]) == 2
            checked += 1
    assert checked > 100


def test_cells_contain_their_generating_edges_and_csr_is_consistent():
    w = W.random_small(3, 8, 12, 0.25, gamma=1.5, n_seeds=2, box=1.2)
    res = _trace(w)
    d = 3
    es = _edge_set(res)
    edges = [(tuple(int(v) for v in y), int(m)) for y, m in zip(res["edge_y"], res["edge_mask"])]
    all_ = (2 << d) - 1
    cells = set()
    for y, m in edges:
        for cy, cp in oracle.edge_ncofaces(d, y, (m, all_ & ~m)):
            cells.add((tuple(cy), cp))
    got = {(tuple(int(v) for v in cy), tuple(1 << int(p) for p in pp) + (1 << d,))
           for cy, pp in zip(res["cell_y"], res["cell_perm"])}
    assert got == cells
    off, idx = res["cell_off"], res["cell_idx"]
    for c, (cy, pp) in enumerate(zip(res["cell_y"], res["cell_perm"])):
        parts = tuple(1 << int(p) for p in pp) + (1 << d,)
        want = [(tuple(int(v) for v in e[0]), e[1][0]) for e in oracle.nsimplex_edges(d, cy, parts)]
        want = [e for e in want if e in es]
        have = [edges[i] for i in idx[off[c]:off[c + 1]]]
        assert have == want


def test_d3_config_counts_are_stable():
    w = W.config_d3()
    res = _trace(w)
    assert res["n_dead_seeds"] == 0
    assert len(res["edge_t"]) > 1000
    assert res["edge_multiroot"].sum() == 0
    # f changes sign across every traced edge
    assert np.all((res["edge_f"][:, 0] >= 0) != (res["edge_f"][:, 1] >= 0))


def test_empty_seed_list():
    w = W.config_d3()
    res = oracle.trace(w.sv, w.alpha, w.gamma, w.b, w.lam, w.offset, w.lo, w.hi,
                       np.zeros((0, 3)), roots=True, cells=True)
    assert len(res["edge_t"]) == 0 and res["levels"] == 0
