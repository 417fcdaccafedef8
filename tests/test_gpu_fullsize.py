"""Parity at the full size of the d=5 FP64 workload (2048 support vectors,
lambda = 0.05, 16 seeds: ~7.4e7 traced edges, ~6.1e8 cells), in the launch
configuration the benchmark times (autotuned).  The oracle cannot trace this
in a test's time, so the checks are on sampled outputs it computes one by
one, plus properties that hold at any size:
  - traced edges are unique and lie in the domain;
  - sampled edges: end values, sign change and root against the oracle;
  - sampled edges: every crossing 2-coface inside the domain leads to an edge
    that is traced (the traced set is closed under the BFS step, Sec. IV-A);
  - sampled cells: the CSR row is exactly the cell's in-domain vertex pairs
    of opposite sign (Sec. IV-C);
  - sampled points: certification verdicts and margins against the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2406_04795_gb300 import workloads as W
from paper_2406_04795_gb300.api import Context
from paper_2406_04795_gb300.pipeline import Proof

pytestmark = pytest.mark.gpu

NEAR_ZERO = 1e-12
OFF, RAD = 512, 1024  # key packing: y + OFF in [0, RAD) per axis


def _keys(y, mask, d):
    """int64 edge keys (torch, on the tensors' device)."""
    y = y.to(torch.int64) + OFF
    assert int(y.min()) >= 0 and int(y.max()) < RAD
    k = torch.zeros(y.shape[0], dtype=torch.int64, device=y.device)
    for i in range(d):
        k = k * RAD + y[:, i]
    return k * (1 << d) + mask.to(torch.int64)


def _key1(y, mask, d):
    k = 0
    for i in range(d):
        k = k * RAD + int(y[i]) + OFF
    return k * (1 << d) + int(mask)


@pytest.fixture(scope="module")
def full():
    w = W.config_d5()
    ctx = Context(0, 0)
    p = Proof(ctx, w)
    p.step()
    sz = p.sizing
    ctx.autotune(w, precision=p.precision, batch_cap=w.batch_cap, max_edges=sz["max_edges"],
                 max_vertices=sz["max_vertices"], max_cells=sz["max_cells"],
                 recheck_band=w.recheck_band)
    r, v, m, cv = p.step()
    E = r["n_edges"]
    keys = _keys(r["edge_y"], r["edge_mask"], w.d)
    sorted_keys, _ = torch.sort(keys)
    yield dict(w=w, r=r, v=v, m=m, cv=cv, E=E, keys=keys, sorted_keys=sorted_keys,
               rng=np.random.default_rng(2024))
    del r, v, m, cv, keys, sorted_keys
    p.outputs = None
    ctx.close()


def _in_domain(w, ys):
    x = oracle.vertex_x(w.d, w.lam, w.offset, ys)
    return np.all((x >= w.lo) & (x <= w.hi), axis=1)


def test_fullsize_edges_unique_and_in_domain(full):
    w, r, E = full["w"], full["r"], full["E"]
    assert E > 50_000_000
    assert torch.unique(full["sorted_keys"]).numel() == E
    idx = full["rng"].choice(E, 4000, replace=False)
    y = r["edge_y"][idx].cpu().numpy()
    m = r["edge_mask"][idx].cpu().numpy().astype(np.int64)
    y2 = y + ((m[:, None] >> np.arange(w.d)) & 1)
    assert _in_domain(w, y).all() and _in_domain(w, y2).all()


def test_fullsize_sampled_edges_against_oracle(full):
    w, r, E = full["w"], full["r"], full["E"]
    idx = np.sort(full["rng"].choice(E, 1500, replace=False))
    y = r["edge_y"][idx].cpu().numpy()
    m = r["edge_mask"][idx].cpu().numpy().astype(np.uint32)
    f_gpu = r["edge_f"][idx].cpu().numpy()
    t_gpu = r["edge_t"][idx].cpu().numpy()
    pt_gpu = r["points"][idx].cpu().numpy()
    f2, t, pt, multi = oracle.edge_roots(w.sv, w.alpha, w.gamma, w.b, w.lam, w.offset, y, m)
    assert np.max(np.abs(f_gpu - f2)) <= 1e-12
    sure = np.all(np.abs(f2) >= NEAR_ZERO, axis=1)
    assert np.all((f2[sure, 0] >= 0) != (f2[sure, 1] >= 0))
    ok = sure & (multi == 0)
    assert ok.sum() > 1400
    assert np.max(np.abs(t_gpu[ok] - t[ok])) <= 1e-9
    assert np.max(np.abs(pt_gpu[ok] - pt[ok])) <= 1e-8


def test_fullsize_bfs_closure_sampled(full):
    """For sampled traced edges, each crossing triangle (2-coface) with all
    vertices in the domain has its other crossing edge in the traced set."""
    w, r, E = full["w"], full["r"], full["E"]
    d = w.d
    allp = (1 << (d + 1)) - 1
    idx = full["rng"].choice(E, 250, replace=False)
    ys = r["edge_y"][idx].cpu().numpy()
    ms = r["edge_mask"][idx].cpu().numpy().astype(np.int64)
    fcache = {}

    def sign(v):
        key = tuple(int(a) for a in v)
        if key not in fcache:
            x = oracle.vertex_x(d, w.lam, w.offset, np.array(v))
            inside = bool(np.all((x >= w.lo) & (x <= w.hi)))
            fcache[key] = (inside, oracle.f(w.sv, w.alpha, w.gamma, w.b, x)[0] if inside else 0.0)
        return fcache[key]

    wanted = []
    for y, m in zip(ys, ms):
        for ty, tparts in oracle.edge_cofaces(d, y, (int(m), allp ^ int(m))):
            verts = oracle.simplex_vertices(d, ty, tparts)
            info = [sign(v) for v in verts]
            if not all(i for i, _ in info):
                continue  # a vertex outside the domain: the BFS does not follow it
            if any(abs(fv) < NEAR_ZERO for _, fv in info):
                continue  # sign of a near-zero vertex is not pinned
            for ey, eparts in oracle.triangle_edges(d, ty, tparts):
                a, b = oracle.simplex_vertices(d, ey, eparts)
                sa, sb = sign(a)[1] >= 0, sign(b)[1] >= 0
                if sa != sb:
                    wanted.append(_key1(ey, eparts[0], d))
    assert len(wanted) > 1000
    q = torch.tensor(wanted, dtype=torch.int64, device=full["sorted_keys"].device)
    pos = torch.searchsorted(full["sorted_keys"], q).clamp(max=E - 1)
    assert bool(torch.all(full["sorted_keys"][pos] == q))


def test_fullsize_cells_csr_sampled(full):
    w, r = full["w"], full["r"]
    d = w.d
    nc = r["n_cells"]
    assert nc > 100_000_000
    idx = full["rng"].choice(nc, 300, replace=False)
    cy = r["cell_y"][idx].cpu().numpy()
    cp = r["cell_perm"][idx].cpu().numpy()
    off = r["cell_off"]
    lo_hi = torch.stack([off[idx], off[idx + 1]], 1).cpu().numpy()
    checked = 0
    for z, perm, (a, b) in zip(cy, cp, lo_hi):
        parts = tuple(1 << int(p) for p in perm) + (1 << d,)
        verts = oracle.simplex_vertices(d, z, parts)
        x = oracle.vertex_x(d, w.lam, w.offset, verts)
        inside = np.all((x >= w.lo) & (x <= w.hi), axis=1)
        fv = oracle.f(w.sv, w.alpha, w.gamma, w.b, x)
        if np.any(inside & (np.abs(fv) < NEAR_ZERO)):
            continue
        expect = set()
        for i in range(d + 1):
            for j in range(i + 1, d + 1):
                if inside[i] and inside[j] and (fv[i] >= 0) != (fv[j] >= 0):
                    mask = sum(1 << int(p) for p in perm[i:j])
                    expect.add(_key1(verts[i], mask, d))
        rows = r["cell_idx"][int(a):int(b)]
        got = set(full["keys"][rows].cpu().numpy().tolist()) if b > a else set()
        assert got == expect
        checked += 1
    assert checked > 250


def test_fullsize_certify_sampled(full):
    w, r, E = full["w"], full["r"], full["E"]
    idx = np.sort(full["rng"].choice(E, 2000, replace=False))
    pts = r["points"][idx].cpu().numpy()
    vg = full["v"][idx].cpu().numpy()
    mg = full["m"][idx].cpu().numpy()
    vo, mo, _ = oracle.certify(w.dh, w.radius, w.obs_type, w.obs_pose, w.obs_dims, pts)
    sure = np.abs(mo) > 1e-12
    assert np.array_equal(vg[sure], vo[sure])
    assert np.max(np.abs(mg - mo)) <= 1e-9


def test_fullsize_cell_verdicts_sampled(full):
    """Sampled cells: the cell verdict is the AND of its points' verdicts,
    each point's verdict recomputed by the oracle (cells with a point whose
    |margin| <= 1e-12 are skipped: its verdict is not pinned)."""
    w, r = full["w"], full["r"]
    nc = r["n_cells"]
    idx = np.sort(full["rng"].choice(nc, 400, replace=False))
    off = r["cell_off"]
    lo_hi = torch.stack([off[idx], off[idx + 1]], 1).cpu().numpy()
    rows = [r["cell_idx"][int(a):int(b)].cpu().numpy() for a, b in lo_hi]
    allp = np.unique(np.concatenate([x for x in rows if x.size] or [np.zeros(0, np.int64)]))
    pts = r["points"][torch.as_tensor(allp, device=r["points"].device)].cpu().numpy()
    vo, mo, _ = oracle.certify(w.dh, w.radius, w.obs_type, w.obs_pose, w.obs_dims, pts)
    pos = {int(p): i for i, p in enumerate(allp)}
    cv = full["cv"][torch.as_tensor(idx, device=full["cv"].device)].cpu().numpy()
    checked = both = 0
    for c, row in enumerate(rows):
        if row.size == 0:
            continue
        k = np.array([pos[int(e)] for e in row])
        if np.any(np.abs(mo[k]) <= 1e-12):
            continue
        assert int(cv[c]) == int(np.all(vo[k] == 1)), c
        checked += 1
        both += int(cv[c])
    assert checked > 300 and 0 < both < checked
