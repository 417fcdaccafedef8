"""Brute-force references for the oracle pins (test-only, numpy).

Independent of the oracle's permutahedral queries: simplices here are Kuhn
simplices given by a base vertex z and a permutation (vertices z, z + e_pi0,
..., z + 1), and the traced set is recomputed by enumerating every lattice
vertex, edge and triangle of a box and running union-find over shared
triangles.
"""
from __future__ import annotations

import itertools
import math
from collections import deque

import numpy as np


def kuhn_vertices(z, pi):
    v = list(z)
    out = [tuple(v)]
    for i in pi:
        v[i] += 1
        out.append(tuple(v))
    return out


def kuhn_simplices_with_vertex(y):
    """Every Kuhn n-simplex that has y as a vertex: base z in y - {0,1}^d."""
    d = len(y)
    for off in itertools.product((0, -1), repeat=d):
        z = tuple(y[i] + off[i] for i in range(d))
        for pi in itertools.permutations(range(d)):
            vs = kuhn_vertices(z, pi)
            if tuple(y) in vs:
                yield z, pi, vs


def triangles_containing_edge(a, b):
    """Vertex sets of all 2-simplices of the triangulation holding edge {a,b}."""
    out = set()
    for _, _, vs in kuhn_simplices_with_vertex(a):
        if tuple(b) in vs:
            for w in vs:
                if w != tuple(a) and w != tuple(b):
                    out.add(frozenset((tuple(a), tuple(b), w)))
    return out


def nsimplices_containing_edge(a, b):
    out = set()
    for _, _, vs in kuhn_simplices_with_vertex(a):
        if tuple(b) in vs:
            out.add(frozenset(vs))
    return out


def lattice_x(d, lam, c, o, Y):
    """x = lam * (y - c * sum(y)) + o with numpy's per-operation rounding."""
    Y = np.asarray(Y, dtype=np.int64)
    s = Y.sum(axis=1).astype(np.float64)
    cs = c * s
    u = Y.astype(np.float64) - cs[:, None]
    return lam * u + np.asarray(o)[None, :]


def barycentric(P, x):
    """Barycentric coordinates of x in the simplex with vertex rows P."""
    d = P.shape[1]
    A = np.vstack([P.T, np.ones(d + 1)])
    rhs = np.concatenate([x, [1.0]])
    return np.linalg.solve(A, rhs)


def brute_trace(d, lam, c, o, lo, hi, fvals_fn, seeds):
    """Traced set by exhaustive enumeration of a box of the lattice.

    Returns (edges: set of (y, mask), levels: dict edge -> BFS distance from
    the seed edges).  brute_counts derives the evaluation counters from it."""
    cinv = c * math.sqrt(d + 1)
    s_lo = float(np.sum(np.asarray(lo) - o))
    s_hi = float(np.sum(np.asarray(hi) - o))
    ymin = [int(math.floor(((lo[i] - o[i]) + cinv * s_lo) / lam)) - 2 for i in range(d)]
    ymax = [int(math.ceil(((hi[i] - o[i]) + cinv * s_hi) / lam)) + 2 for i in range(d)]
    axes = [np.arange(ymin[i], ymax[i] + 1) for i in range(d)]
    grid = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, d)
    X = lattice_x(d, lam, c, o, grid)
    inb = np.all((X >= np.asarray(lo)[None]) & (X <= np.asarray(hi)[None]), axis=1)
    Yin = grid[inb]
    fin = fvals_fn(X[inb])
    index = {tuple(y): i for i, y in enumerate(Yin.tolist())}
    sign = fin >= 0.0

    def vid(y):
        return index.get(tuple(y))

    masks = range(1, 1 << d)

    def e(mask):
        return np.array([(mask >> i) & 1 for i in range(d)], dtype=np.int64)

    # crossing edges, keyed (y, mask)
    crossing = {}
    for mask in masks:
        em = e(mask)
        for i, y in enumerate(Yin.tolist()):
            j = vid(np.asarray(y) + em)
            if j is not None and sign[i] != sign[j]:
                crossing[(tuple(y), mask)] = (i, j)
    # union-find over triangles (y, (A, B, rest)) with all vertices in the box
    parent = {k: k for k in crossing}
    adj = {k: set() for k in crossing}

    def find(k):
        while parent[k] != k:
            parent[k] = parent[parent[k]]
            k = parent[k]
        return k

    full = (1 << d) - 1
    for A in masks:
        for B in masks:
            if A & B:
                continue
            eA, eB = e(A), e(B)
            for y in Yin.tolist():
                y = np.asarray(y)
                v1 = y + eA
                v2 = v1 + eB
                if vid(v1) is None or vid(v2) is None:
                    continue
                tri_edges = [(tuple(y), A), (tuple(y), A | B), (tuple(v1), B)]
                cr = [t for t in tri_edges if t in crossing]
                assert len(cr) in (0, 2), "binary signs give 0 or 2 crossing edges"
                if cr:
                    a, b = cr
                    parent[find(a)] = find(b)
                    adj[a].add(b)
                    adj[b].add(a)
    del full
    # seed edges: crossing in-box edges of the Kuhn simplex holding each seed
    seed_edges = set()
    for x in np.atleast_2d(seeds):
        yp = (np.asarray(x) - o + cinv * np.sum(np.asarray(x) - o)) / lam
        base = np.floor(yp).astype(np.int64)
        found = None
        for off in itertools.product((-1, 0, 1), repeat=d):
            z = base + np.asarray(off)
            for pi in itertools.permutations(range(d)):
                vs = np.array(kuhn_vertices(z, pi))
                bc = barycentric(lattice_x(d, lam, c, o, vs), np.asarray(x))
                if np.all(bc >= -1e-12):
                    found = vs
                    break
            if found is not None:
                break
        assert found is not None
        for i in range(d + 1):
            for j in range(i + 1, d + 1):
                a, b = found[i], found[j]
                diff = b - a
                # canonical: second vertex = first + e(mask) with mask >= 0 entries
                if np.all(diff >= 0):
                    key = (tuple(a), int(sum(1 << k for k in range(d) if diff[k])))
                else:
                    key = (tuple(b), int(sum(1 << k for k in range(d) if -diff[k])))
                if key in crossing:
                    seed_edges.add(key)
    roots = {find(k) for k in seed_edges}
    traced = {k for k in crossing if find(k) in roots}
    # BFS distances from the seed edges over shared triangles
    level = {k: 0 for k in seed_edges}
    q = deque(seed_edges)
    while q:
        k = q.popleft()
        for n in adj[k]:
            if n not in level:
                level[n] = level[k] + 1
                q.append(n)
    return traced, level


def brute_counts(d, lam, c, o, lo, hi, fvals_fn, seeds, traced):
    """The tracing counters derived from the traced set by Kuhn-simplex
    enumeration, independently of the oracle's permutahedral queries.

    f is evaluated at (i) the in-box vertices of each seed's n-simplex that
    belong to an in-box edge of it (at least two in-box vertices), and (ii)
    the vertices of every 2-simplex containing a traced edge whose three
    vertices are all in the box.  A (traced edge, 2-simplex) pair whose third
    vertex leaves the box is a boundary pair.  Returns (n_vertices,
    n_boundary, n_near_zero)."""
    cinv = c * math.sqrt(d + 1)
    lo, hi, o = np.asarray(lo), np.asarray(hi), np.asarray(o)

    def inbox(v):
        x = lattice_x(d, lam, c, o, np.asarray([v]))[0]
        return bool(np.all(x >= lo) and np.all(x <= hi))

    evaluated = set()
    for x in np.atleast_2d(seeds):
        yp = (np.asarray(x) - o + cinv * np.sum(np.asarray(x) - o)) / lam
        base = np.floor(yp).astype(np.int64)
        found = None
        for off in itertools.product((-1, 0, 1), repeat=d):
            z = base + np.asarray(off)
            for pi in itertools.permutations(range(d)):
                vs = np.array(kuhn_vertices(z, pi))
                bc = barycentric(lattice_x(d, lam, c, o, vs), np.asarray(x))
                if np.all(bc >= -1e-12):
                    found = vs
                    break
            if found is not None:
                break
        assert found is not None
        ins = [tuple(int(t) for t in v) for v in found if inbox(v)]
        if len(ins) >= 2:
            evaluated.update(ins)
    boundary = 0
    for (y, mask) in traced:
        a = tuple(y)
        b = tuple(y[i] + ((mask >> i) & 1) for i in range(d))
        for tri in triangles_containing_edge(a, b):
            (w,) = tuple(tri - {a, b})
            if inbox(w):
                evaluated.update((a, b, w))
            else:
                boundary += 1
    if evaluated:
        V = np.array(sorted(evaluated), dtype=np.int64)
        fv = fvals_fn(lattice_x(d, lam, c, o, V))
        near = int(np.sum(np.abs(fv) < 1e-12))
    else:
        near = 0
    return len(evaluated), boundary, near


def brute_crossing_edges(d, lam, c, o, lo, hi, fvals_fn):
    """Every lattice edge (y, mask) with both vertices in the box and a sign
    change of f (binary signs), by enumerating a box of the lattice."""
    cinv = c * math.sqrt(d + 1)
    s_lo = float(np.sum(np.asarray(lo) - o))
    s_hi = float(np.sum(np.asarray(hi) - o))
    ymin = [int(math.floor(((lo[i] - o[i]) + cinv * s_lo) / lam)) - 2 for i in range(d)]
    ymax = [int(math.ceil(((hi[i] - o[i]) + cinv * s_hi) / lam)) + 2 for i in range(d)]
    axes = [np.arange(ymin[i], ymax[i] + 1) for i in range(d)]
    grid = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, d)
    X = lattice_x(d, lam, c, o, grid)
    inb = np.all((X >= np.asarray(lo)[None]) & (X <= np.asarray(hi)[None]), axis=1)
    Yin = grid[inb]
    sign = fvals_fn(X[inb]) >= 0.0
    index = {tuple(y): i for i, y in enumerate(Yin.tolist())}
    out = set()
    for mask in range(1, 1 << d):
        em = np.array([(mask >> i) & 1 for i in range(d)], dtype=np.int64)
        for i, y in enumerate(Yin.tolist()):
            j = index.get(tuple(np.asarray(y) + em))
            if j is not None and sign[i] != sign[j]:
                out.add((tuple(y), mask))
    return out
