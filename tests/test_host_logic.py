"""Host-side logic of the CUDA library that runs without a GPU.

The exact lattice domain table (mf_domain_table) must reproduce, vertex by
vertex, the oracle's decision "x(y) lies in the closed box", for vertices deep
inside, outside and on the boundary of the box."""
import math
import os

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


@pytest.mark.parametrize("d,lam,box", [(2, 0.1, 1.0), (3, 0.02, math.pi), (5, 0.05, math.pi),
                                       (6, 0.03, math.pi), (6, 0.02, math.pi), (8, 0.3, 2.0)])
def test_vertex_keys_unique_near_the_box(d, lam, box):
    """Every vertex within three lattice steps of a point of the box lies in
    the key packing, and distinct vertices get distinct keys."""
    rng = np.random.default_rng(100 + d)
    lo, hi = -box * np.ones(d), box * np.ones(d)
    off = W.lattice_offset(d, lam)
    dom = _dom(lo, hi, off)
    # box points: uniform, on faces and at corners
    pts = rng.uniform(lo, hi, size=(300, d))
    k = rng.integers(0, d, size=300)
    pts[np.arange(300), k] = np.where(rng.integers(0, 2, size=300), hi[k], lo[k])
    corners = np.where(rng.integers(0, 2, size=(100, d)), hi, lo)
    ys = []
    for p in np.concatenate([pts, corners]):
        y, _ = oracle.locate(d, lam, off, p)
        y = np.array(y, dtype=np.int64)
        for _ in range(40):
            ys.append(y + rng.integers(-3, 4, size=d))
        ys.append(y)
    ys = np.unique(np.array(ys), axis=0)
    keys, ok = mf.mf_vertex_keys(d, lam, dom, ys)
    assert ok.all()
    assert np.unique(keys).size == ys.shape[0]
    # far outside: reported as outside the packing
    _, ok_far = mf.mf_vertex_keys(d, lam, dom, ys[:5] + 10_000)
    assert not ok_far.any()


def test_vertex_keys_reject_too_fine_lattice():
    d = 6
    off = W.lattice_offset(d, 0.005)
    dom = _dom(-math.pi * np.ones(d), math.pi * np.ones(d), off)
    with pytest.raises(mf.MfError) as e:
        mf.mf_vertex_keys(d, 0.005, dom, np.zeros((1, d), np.int32))
    assert e.value.code == mf.MF_ERR_DOMAIN


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    from paper_2406_04795_gb300.scaling import reduce_timing
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    try:
        # each rank traces its own workload (seed + 10 rank) and reports its time
        w = bench.make_workload("d3", rank)
        res = reduce_timing(100.0 + rank, 1000 * (rank + 1), 2.0 * (rank + 1), 10 + rank, world,
                            "cpu")
        with open(os.path.join(out_dir, "r%d.txt" % rank), "w") as fh:
            fh.write("%r %r %r %r %r\n" % (res + (float(w.sv[0, 0]),)))
    finally:
        dist.destroy_process_group()


def test_weak_scaling_reduction_two_gloo_ranks(tmp_path):
    """The multi-GPU bench path on CPU: two gloo ranks get distinct workloads
    and agree on max time and summed units."""
    import socket
    import torch.multiprocessing as tmp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    tmp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    rows = [open(tmp_path / ("r%d.txt" % r)).read().split() for r in range(2)]
    for row in rows:
        ms, units, e2e, e2e_units = (float(v) for v in row[:4])
        assert (ms, units, e2e, e2e_units) == (101.0, 3000.0, 4.0, 21.0)
    assert rows[0][4] != rows[1][4]  # different seeds per rank


@pytest.mark.parametrize("d,lam", [(2, 0.3), (3, 0.1), (5, 0.05), (6, 0.04), (8, 0.2)])
def test_longest_edge_bound_for_vertex_lists(d, lam):
    """The per-vertex lists of the root screen assume every edge (y, y + e(M))
    is at most lam * max_k sqrt(k (1 - 2ck + c^2 k d)) long (|M| = k): check
    it against the oracle's lattice map for every mask, and that it is
    attained."""
    rng = np.random.default_rng(d)
    c = oracle.lattice_c(d)
    bound = lam * max(math.sqrt(k * (1 - 2 * c * k + c * c * k * d)) for k in range(1, d + 1))
    off = W.lattice_offset(d, lam)
    longest = 0.0
    for _ in range(20):
        y = rng.integers(-50, 50, size=d)
        x0 = oracle.vertex_x(d, lam, off, y[None, :])[0]
        for m in range(1, 1 << d):
            e = np.array([(m >> k) & 1 for k in range(d)])
            x1 = oracle.vertex_x(d, lam, off, (y + e)[None, :])[0]
            longest = max(longest, float(np.linalg.norm(x1 - x0)))
    assert longest <= bound * (1 + 1e-12)
    assert longest >= bound * (1 - 1e-9)
