"""Mixed-precision paths against the FP64 oracle (not against another CUDA
path): the tensor-core evaluation with many support-vector chunks and
vertex tiles, the batched engine with FP32 SIMT and tensor-core slots, and
the proof server under queueing.

Tolerances: traced edge sets, cells and cell -> edge rows exact; f at the
edge ends within the recheck band 1e-3 (FP32 values of vertices the bound
decided) or 1e-12 (FP64 rechecks); roots within 1e-6 on the mixed paths and
1e-9 when FP64-exact roots are asked for or on FP64 slots."""
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


# d = 3: 400 vectors = 6 full chunks of 64 and a ragged one of 16, ~3300
# vertices = 26 tiles of 128 with a ragged last tile; d = 4: 333 vectors
# (5 chunks + 13), ~10^4 vertices
MULTI = [(3, 400, 0.12, 31), (4, 333, 0.25, 31)]


@pytest.mark.parametrize("d,n_sv,lam,seed", MULTI)
@pytest.mark.parametrize("exact", [False, True])
def test_bf16_multichunk_against_oracle(ctx, d, n_sv, lam, seed, exact):
    w = W.random_small(d, n_sv, seed, lam, gamma=1.5, n_seeds=4, box=1.3)
    o = P.oracle_trace(w)
    g = P.gpu_trace(ctx, w, mf.MF_MIXED_BF16, exact_roots=exact)
    assert g["n_vertices"] > 3 * 128 and n_sv > 5 * 64
    rep = P.compare_traces(w, g, o, f_tol=1e-3, t_tol=1e-9 if exact else 1e-6)
    assert rep["n_diff"] == 0
    # most vertices keep their tensor-core value: the MMA path decided them
    assert 0 < g["n_recheck"] < 0.5 * g["n_vertices"]
    ok = P.keys(o["edge_y"], o["edge_mask"])
    om = {k: i for i, k in enumerate(ok)}
    oi = np.array([om[k] for k in P.keys(g["edge_y"], g["edge_mask"])])
    df = np.abs(g["edge_f"] - o["edge_f"][oi])
    assert np.mean(df > 1e-12) > 0.3


def _small_set():
    return [W.random_small(3, 400, 31, 0.12, gamma=1.5, n_seeds=4, box=1.3),
            W.config_d3(),
            W.sphere_workload(3, r=1.0, gamma=1.0, lam=0.2),
            W.random_small(4, 333, 31, 0.3, gamma=1.5, n_seeds=4, box=1.3),
            W.random_small(2, 40, 5, 0.05, gamma=1.5, n_seeds=3, box=1.3)]


def test_batched_mixed_slots_against_oracle(ctx):
    ws = _small_set()
    precs = [mf.MF_MIXED_BF16, mf.MF_MIXED_FP32, mf.MF_MIXED_BF16, mf.MF_MIXED_FP32,
             mf.MF_MIXED_BF16]
    got = ctx.trace_batch(ws, precisions=precs,
                          capacities=[dict(max_edges=1 << 18, max_cells=1 << 21)] * len(ws))
    for w, p, g in zip(ws, precs, got):
        o = P.oracle_trace(w)
        rep = P.compare_traces(w, _np(g), o, f_tol=1e-3, t_tol=1e-6)
        assert rep["n_diff"] == 0 and rep["n_edges"] > 100, (w.name, p)
    # the same slots with FP64-exact roots
    got = ctx.trace_batch(ws[:2], precisions=precs[:2], exact_roots=True,
                          capacities=[dict(max_edges=1 << 18, max_cells=1 << 21)] * 2)
    for w, g in zip(ws[:2], got):
        assert P.compare_traces(w, _np(g), P.oracle_trace(w), f_tol=1e-3, t_tol=1e-9)["n_diff"] == 0


def test_served_requests_against_oracle(ctx):
    """Five requests through two slots (three queue), mixed FP32, BF16 and
    FP64, each result compared with the oracle."""
    ws = _small_set()
    precs = [mf.MF_MIXED_BF16, mf.MF_FP64, mf.MF_MIXED_FP32, mf.MF_MIXED_BF16, mf.MF_FP64]
    server = ctx.server(max_slots=2, hbm_bytes=8 << 30)
    ids = [server.submit(w, precision=p, max_edges=1 << 18, max_cells=1 << 21)
           for w, p in zip(ws, precs)]
    got, saw_queue, steps = {}, False, 0
    while len(got) < len(ids):
        running, queued = server.step()
        saw_queue = saw_queue or queued > 0
        for rid in server.done():
            assert server.status(rid)[0] == 2
            got[rid] = server.fetch(rid)
        steps += 1
        assert steps < 5000
    assert saw_queue
    server.close()
    for w, p, rid in zip(ws, precs, ids):
        o = P.oracle_trace(w)
        fp64 = p == mf.MF_FP64
        rep = P.compare_traces(w, _np(got[rid]), o, f_tol=1e-12 if fp64 else 1e-3,
                               t_tol=1e-9 if fp64 else 1e-6)
        assert rep["n_diff"] == 0 and rep["n_edges"] > 100, (w.name, p)
