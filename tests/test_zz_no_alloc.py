"""mf_trace_noalloc: the entry point for callers that cannot allocate device
memory (code under another framework's memory pool, real-time loops that
forbid allocation, processes whose device memory is reserved elsewhere).

It is called through the C ABI on the d=3 workload twice in a row, and each
result must match the allocating entry point mf_trace: the same edge set and
cells with the same cell -> edge lists, f at the edge ends within 1e-12, root
parameters within 1e-9.  A d=4 workload with more than one 32-vector block
(caller-order support vectors) runs the same way on both mixed precisions:
the tensor-core evaluation and its FP64 recheck queue, and the FP32 SIMT
evaluation; edge and cell sets exact, f at the edge ends within the recheck
band 1e-3 and roots within 2e-6 (each within 1e-6 of the exact root).
The file is named so that pytest collects it last.
"""
import numpy as np
import pytest
import torch

from paper_2406_04795_gb300 import mf
from paper_2406_04795_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _keys(y, m):
    return [(tuple(int(v) for v in a), int(b)) for a, b in zip(y, m)]


def _call_noalloc(ctx, w, bufs, precision=mf.MF_FP64, max_edges=0):
    rbf, keep = ctx.rbf(w.sv, w.alpha, w.gamma, w.b)
    dom = ctx.domain(w.lo, w.hi, w.offset)
    seeds = torch.as_tensor(w.seeds, dtype=torch.float64, device="cuda")
    opts = mf.mf_trace_opts(w.lam, 1 << 24, precision, 1e-3, 1e-12, max_edges, 0, 0,
                            mf.MF_WANT_ROOTS | mf.MF_WANT_CELLS)
    out = ctx._out_struct(bufs, w.d)
    rc = mf.mf_trace_noalloc(rbf, dom, opts, seeds.data_ptr(), seeds.shape[0], out,
                             torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert rc == mf.MF_OK, rc
    E, C, CE = out.n_edges, out.n_cells, out.n_cell_edges
    return dict(y=bufs["edge_y"][:E].cpu().numpy(), m=bufs["edge_mask"][:E].cpu().numpy(),
                f=bufs["edge_f"][:E].cpu().numpy(), t=bufs["edge_t"][:E].cpu().numpy(),
                cy=bufs["cell_y"][:C].cpu().numpy(), cp=bufs["cell_perm"][:C].cpu().numpy(),
                off=bufs["cell_off"][:C + 1].cpu().numpy(), idx=bufs["cell_idx"][:CE].cpu().numpy(),
                levels=out.levels, n_vertices=out.n_vertices)


@pytest.mark.parametrize("case", ["d3_fp64", "d4_bf16", "d4_fp32"])
def test_noalloc_matches_mf_trace_twice(case):
    from paper_2406_04795_gb300.api import Context
    if case == "d3_fp64":
        w, prec, f_tol, t_tol, me = W.config_d3(), mf.MF_FP64, 1e-12, 1e-9, 0
    else:
        w = W.random_small(4, 333, 31, 0.3, gamma=1.5, n_seeds=4, box=1.3)
        prec = mf.MF_MIXED_BF16 if case == "d4_bf16" else mf.MF_MIXED_FP32
        f_tol, t_tol, me = 1e-3, 2e-6, 1 << 16
    ctx = Context(0, 8 << 30)
    ref = ctx.trace(w.sv, w.alpha, w.gamma, w.b, w.lam, w.offset, w.lo, w.hi, w.seeds,
                    precision=prec)
    rk = _keys(ref["edge_y"].cpu().numpy(), ref["edge_mask"].cpu().numpy())
    rmap = {k: i for i, k in enumerate(rk)}
    rt = ref["edge_t"].cpu().numpy()
    rf = ref["edge_f"].cpu().numpy()
    rcells = {(tuple(c), tuple(p)): i for i, (c, p) in
              enumerate(zip(ref["cell_y"].cpu().numpy().tolist(), ref["cell_perm"].cpu().numpy().tolist()))}
    roff, ridx = ref["cell_off"].cpu().numpy(), ref["cell_idx"].cpu().numpy()
    bufs = ctx._alloc_outputs(w.d, ref["n_edges"] + 16, ref["n_cells"] + 16,
                              ref["n_cell_edges"] + 64)
    for call in range(2):
        r = _call_noalloc(ctx, w, bufs, prec, me)
        k = _keys(r["y"], r["m"])
        assert len(k) == len(rk) and set(k) == set(rk), "call %d: edge sets differ" % call
        order = np.array([rmap[x] for x in k])
        assert np.max(np.abs(r["f"] - rf[order])) <= f_tol
        assert np.max(np.abs(r["t"] - rt[order])) <= t_tol
        assert r["levels"] == ref["levels"] and r["n_vertices"] == ref["n_vertices"]
        cells = [(tuple(c), tuple(p)) for c, p in zip(r["cy"].tolist(), r["cp"].tolist())]
        assert set(cells) == set(rcells)
        for ci, key in enumerate(cells):
            j = rcells[key]
            have = {k[i] for i in r["idx"][r["off"][ci]:r["off"][ci + 1]]}
            want = {rk[i] for i in ridx[roff[j]:roff[j + 1]]}
            assert have == want
    ctx.close()
