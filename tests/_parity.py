"""Helpers for the GPU-vs-oracle parity tests (test-only)."""
from __future__ import annotations

import numpy as np

import oracle

NEAR_ZERO = 1e-12


def keys(ys, masks):
    return [(tuple(int(v) for v in y), int(m)) for y, m in zip(np.asarray(ys), np.asarray(masks))]


def cell_keys(ys, perms):
    return [(tuple(int(v) for v in y), tuple(int(p) for p in pp))
            for y, pp in zip(np.asarray(ys), np.asarray(perms))]


def gpu_trace(ctx, w, precision=0, **kw):
    r = ctx.trace(w.sv, w.alpha, w.gamma, w.b, w.lam, w.offset, w.lo, w.hi, w.seeds,
                  precision=precision, **kw)
    out = {}
    for k, v in r.items():
        if k == "_buffers":
            continue
        out[k] = v.cpu().numpy() if hasattr(v, "cpu") else v
    out["edge_mask"] = out["edge_mask"].astype(np.uint32)
    return out


def oracle_trace(w, roots=True, cells=True):
    return oracle.trace(w.sv, w.alpha, w.gamma, w.b, w.lam, w.offset, w.lo, w.hi, w.seeds,
                        roots=roots, cells=cells)


def near_zero_edge(w, key):
    """True if one vertex of the edge has |f| < 1e-12 (oracle arithmetic)."""
    d = w.d
    y = np.array(key[0], np.int32)
    y2 = y.copy()
    for k in range(d):
        y2[k] += (key[1] >> k) & 1
    X = oracle.vertex_x(d, w.lam, w.offset, np.stack([y, y2]))
    f = oracle.f(w.sv, w.alpha, w.gamma, w.b, X)
    return bool(np.any(np.abs(f) < NEAR_ZERO))


def compare_traces(w, g, o, t_tol=1e-9, f_tol=1e-12, check_f=True, check_cells=True,
                   check_t=True):
    """Element-by-element comparison of a GPU trace with the oracle's."""
    gk = keys(g["edge_y"], g["edge_mask"])
    ok = keys(o["edge_y"], o["edge_mask"])
    assert len(set(gk)) == len(gk), "duplicate edges in the GPU output"
    sg, so = set(gk), set(ok)
    diff = sg ^ so
    assert all(near_zero_edge(w, k) for k in diff), "edge sets differ: %d edges" % len(diff)
    report = dict(n_edges=len(gk), n_diff=len(diff), n_near_zero=int(o["n_near_zero"]))
    if not diff:
        assert g["n_vertices"] == o["n_vertices"]
        assert g["n_boundary"] == o["n_boundary"]
        assert g["levels"] == o["levels"]
    assert g["n_dead_seeds"] == o["n_dead_seeds"]
    gi = {k: i for i, k in enumerate(gk)}
    common = [k for k in ok if k in gi]
    omap = {k: i for i, k in enumerate(ok)}
    oi = np.array([omap[k] for k in common], dtype=np.int64)
    gidx = np.array([gi[k] for k in common], dtype=np.int64)
    if check_f and len(common):
        assert np.max(np.abs(g["edge_f"][gidx] - o["edge_f"][oi])) <= f_tol
    if check_t and len(common) and g["edge_t"].shape[0]:
        mr = o["edge_multiroot"][oi] == 0
        dt = np.abs(g["edge_t"][gidx] - o["edge_t"][oi])[mr]
        report["max_dt"] = float(dt.max()) if dt.size else 0.0
        assert report["max_dt"] <= t_tol, report
        dp = np.abs(g["points"][gidx] - o["edge_pt"][oi])[mr]
        assert (dp.max() if dp.size else 0.0) <= t_tol
    if check_cells and "cell_y" in o:
        gc = cell_keys(g["cell_y"], g["cell_perm"])
        oc = cell_keys(o["cell_y"], o["cell_perm"])
        assert len(set(gc)) == len(gc)
        if not diff:
            assert set(gc) == set(oc)
            gcell = {k: i for i, k in enumerate(gc)}
            for c, k in enumerate(oc):
                j = gcell[k]
                have = {gk[i] for i in g["cell_idx"][g["cell_off"][j]:g["cell_off"][j + 1]]}
                want = {ok[i] for i in o["cell_idx"][o["cell_off"][c]:o["cell_off"][c + 1]]}
                assert have == want
        report["n_cells"] = len(gc)
    return report
