"""Batched multi-trace (mf_trace_batch): many uneven traces in one launch give
each trace exactly what it gets alone (mf_trace), and small ones match the
FP64 oracle."""
import numpy as np
import pytest

from paper_2406_04795_gb300 import mf
from paper_2406_04795_gb300 import workloads as W
from tests import _parity as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2406_04795_gb300.api import Context
    c = Context(0, 64 << 30)
    yield c
    c.close()


def _np(r):
    out = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in r.items() if k != "_buffers"}
    out["edge_mask"] = out["edge_mask"].astype(np.uint32)
    return out


def _same(a, b, t_tol=1e-9, f_tol=1e-12):
    ka = P.keys(a["edge_y"], a["edge_mask"])
    kb = P.keys(b["edge_y"], b["edge_mask"])
    assert len(ka) == len(kb) and set(ka) == set(kb)
    for k in ("n_vertices", "n_boundary", "n_dead_seeds", "levels", "n_cells", "n_cell_edges"):
        assert a[k] == b[k], k
    mb = {k: i for i, k in enumerate(kb)}
    order = np.array([mb[k] for k in ka], dtype=np.int64)
    if len(order):
        assert np.max(np.abs(a["edge_t"] - b["edge_t"][order])) <= t_tol
        assert np.max(np.abs(a["edge_f"] - b["edge_f"][order])) <= f_tol
    ca = P.cell_keys(a["cell_y"], a["cell_perm"])
    cb = P.cell_keys(b["cell_y"], b["cell_perm"])
    assert set(ca) == set(cb)
    cmap = {k: i for i, k in enumerate(cb)}
    for i, k in enumerate(ca):
        j = cmap[k]
        ha = {ka[x] for x in a["cell_idx"][a["cell_off"][i]:a["cell_off"][i + 1]]}
        hb = {kb[x] for x in b["cell_idx"][b["cell_off"][j]:b["cell_off"][j + 1]]}
        assert ha == hb


def test_batch_equals_each_trace_alone(ctx):
    ws = [W.config_d3(), W.random_small(2, 12, 2, 0.05, gamma=1.5, n_seeds=4, box=1.3),
          W.random_small(4, 16, 3, 0.3, gamma=1.5, n_seeds=4, box=1.3)]
    ws += W.config_batched(n_traces=5, lam_scale=3.0)
    precs = [mf.MF_FP64, mf.MF_MIXED_FP32, mf.MF_MIXED_BF16, mf.MF_FP64, mf.MF_MIXED_FP32,
             mf.MF_MIXED_BF16, mf.MF_MIXED_FP32, mf.MF_FP64]
    caps = [dict(max_edges=1 << 20, max_vertices=1 << 20, max_cells=1 << 23)] * len(ws)
    got = ctx.trace_batch(ws, precisions=precs, capacities=caps)
    for w, p, g in zip(ws, precs, got):
        alone = ctx.trace(w.sv, w.alpha, w.gamma, w.b, w.lam, w.offset, w.lo, w.hi, w.seeds,
                          precision=p, max_edges=1 << 20, max_vertices=1 << 20, max_cells=1 << 23)
        assert g["n_edges"] > 10
        # mixed precision: the batched and single-trace FP32 evaluators sum in
        # different orders, so unrechecked vertex values agree to the band
        # only, and roots (each within 1e-6 of the exact one) to 2e-6
        fp64 = p == mf.MF_FP64
        _same(_np(g), _np(alone), f_tol=1e-12 if fp64 else 1e-3, t_tol=1e-9 if fp64 else 2e-6)


def test_batch_small_traces_match_oracle(ctx):
    ws = [W.config_d3(), W.sphere_workload(3, r=1.0, gamma=1.0, lam=0.2),
          W.random_small(3, 20, 2, 0.15, gamma=1.5, n_seeds=4, box=1.3)]
    got = ctx.trace_batch(ws, capacities=[dict(max_edges=1 << 18)] * 3)
    for w, g in zip(ws, got):
        o = P.oracle_trace(w)
        rep = P.compare_traces(w, _np(g), o)
        assert rep["n_diff"] == 0


def test_batch_reports_small_buffers(ctx):
    from paper_2406_04795_gb300.api import Context  # noqa: F401
    w = W.config_d3()
    with pytest.raises(mf.MfError) as e:
        ctx.trace_batch([w, w], capacities=[dict(max_edges=1 << 18), dict(max_edges=100)])
    assert e.value.code in (mf.MF_ERR_MAXEDGES, mf.MF_ERR_CAPACITY)
