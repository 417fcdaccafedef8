"""Batch triangulation on the GPU (mf_subdiv_begin / mf_subdiv_next) against
the oracle's (Sec. V-B): the same fine edge set exactly, f at the edge ends
within 1e-12 (FP64) or the recheck band (mixed), roots within 1e-9 (FP64) or
1e-6 (mixed); over several batches the union of the batches is the set and no
batch repeats an edge."""
import numpy as np
import pytest

import oracle
from paper_2406_04795_gb300 import mf
from paper_2406_04795_gb300 import workloads as W
from tests import _parity as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2406_04795_gb300.api import Context
    c = Context(0, 16 << 30)
    yield c
    c.close()


def _np(r):
    return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in r.items()}


def _check(w, g, o, f_tol, t_tol):
    gk = P.keys(g["edge_y"], g["edge_mask"].astype(np.uint32))
    ok = P.keys(o["edge_y"], o["edge_mask"])
    assert set(gk) == set(ok) and len(ok) > 100
    om = {k: i for i, k in enumerate(ok)}
    oi = np.array([om[k] for k in gk])
    assert np.max(np.abs(g["edge_f"] - o["edge_f"][oi])) <= f_tol
    mr = o["edge_multiroot"][oi] == 0
    assert np.max(np.abs(g["edge_t"] - o["edge_t"][oi])[mr]) <= t_tol
    assert np.max(np.abs(g["points"] - o["edge_pt"][oi])[mr]) <= t_tol


CASES = [("rand2", 2, 2), ("rand3", 3, 2), ("sphere3", 3, 3), ("rand4", 4, 2), ("d5", 5, 2)]


def _workload(name):
    if name == "rand2":
        return W.random_small(2, 12, 2, 0.06, gamma=1.5, n_seeds=4, box=1.2)
    if name == "rand3":
        return W.random_small(3, 10, 3, 0.08, gamma=1.5, n_seeds=4, box=1.2)
    if name == "sphere3":
        return W.sphere_workload(3, r=1.0, gamma=1.0, lam=0.1)
    if name == "rand4":
        return W.random_small(4, 16, 3, 0.2, gamma=1.5, n_seeds=4, box=1.3)
    return W.config_d5(lam=0.45)


@pytest.mark.parametrize("name,d,k", CASES)
def test_subdiv_one_batch_against_oracle(ctx, name, d, k):
    w = _workload(name)
    o = oracle.subdiv(w.sv, w.alpha, w.gamma, w.b, w.lam, k, w.offset, w.lo, w.hi, w.seeds)
    g = _np(ctx.subdiv(w, k, precision=mf.MF_FP64, max_edges=1 << 20))
    assert g["batches"] == 1 and g["n_coarse_cells"] == o["n_coarse_cells"]
    _check(w, g, o, 1e-12, 1e-9)
    if name == "sphere3":  # the paper's claim holds here: the direct fine trace
        t = P.oracle_trace(w, cells=False)
        assert set(P.keys(g["edge_y"], g["edge_mask"])) == set(P.keys(t["edge_y"], t["edge_mask"]))


@pytest.mark.parametrize("precision", [mf.MF_MIXED_BF16, mf.MF_MIXED_FP32])
def test_subdiv_mixed_against_oracle(ctx, precision):
    w = _workload("rand4")
    o = oracle.subdiv(w.sv, w.alpha, w.gamma, w.b, w.lam, 2, w.offset, w.lo, w.hi, w.seeds)
    g = _np(ctx.subdiv(w, 2, precision=precision, max_edges=1 << 20))
    _check(w, g, o, 1e-3, 1e-6)


def test_subdiv_batches_union(ctx):
    w = _workload("rand3")
    o = oracle.subdiv(w.sv, w.alpha, w.gamma, w.b, w.lam, 2, w.offset, w.lo, w.hi, w.seeds)
    seen = []

    def each(b):
        k = P.keys(b["edge_y"].cpu().numpy(), b["edge_mask"].cpu().numpy().astype(np.uint32))
        assert len(set(k)) == len(k)  # within a batch, every edge once
        seen.append(set(k))

    g = ctx.subdiv(w, 2, precision=mf.MF_FP64, cells_per_batch=37, max_edges=1 << 18,
                   each_batch=each)
    assert g["batches"] == len(seen) == -(-g["n_coarse_cells"] // 37) > 3
    union = set().union(*seen)
    assert union == set(P.keys(o["edge_y"], o["edge_mask"]))
    # edges on faces shared by two batches are reported by both
    assert sum(len(s) for s in seen) >= len(union)
