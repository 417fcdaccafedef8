"""Sorted output (MF_SORT_OUTPUT): edges in increasing order of their edge
key, cells in increasing order of (vertex key of z, pi as base-8 digits),
the same sets and per-element values as the unsorted output, and the
cell -> edge rows carried over to the new orders."""
import numpy as np
import pytest

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


def _vkeys(w, y):
    import ctypes as C
    dom = mf.mf_domain()
    for i in range(w.d):
        dom.lo[i], dom.hi[i], dom.offset[i] = w.lo[i], w.hi[i], w.offset[i]
    y = np.ascontiguousarray(y, dtype=np.int32)
    keys = np.zeros(max(len(y), 1), dtype=np.uint64)
    rc = mf.load().mf_vertex_keys(w.d, float(w.lam), C.byref(dom), y.ctypes.data, len(y),
                                  keys.ctypes.data, None)
    assert rc == 0
    return keys[:len(y)]


@pytest.mark.parametrize("name", ["d3", "d5"])
def test_sorted_output(ctx, name):
    w = W.config_d3() if name == "d3" else W.config_d5(lam=0.3)
    a = P.gpu_trace(ctx, w)
    s = P.gpu_trace(ctx, w, sort=True)
    d = w.d
    ek = (_vkeys(w, s["edge_y"]).astype(object) * (1 << d) + s["edge_mask"].astype(object))
    assert all(ek[i] < ek[i + 1] for i in range(len(ek) - 1))
    ka, ks = P.keys(a["edge_y"], a["edge_mask"]), P.keys(s["edge_y"], s["edge_mask"])
    assert set(ka) == set(ks) and len(ks) > 1000
    am = {k: i for i, k in enumerate(ka)}
    o = np.array([am[k] for k in ks])
    for f in ("edge_f", "edge_t", "points"):  # the same computation: bit-identical
        assert np.array_equal(s[f], a[f][o])
    # cells: (vertex key, pi code) increasing
    code = np.zeros(len(s["cell_y"]), dtype=np.int64)
    for k in range(d):
        code = code * 8 + s["cell_perm"][:, k].astype(np.int64)
    ck = list(zip(_vkeys(w, s["cell_y"]).tolist(), code.tolist()))
    assert all(ck[i] < ck[i + 1] for i in range(len(ck) - 1))
    ca, cs = P.cell_keys(a["cell_y"], a["cell_perm"]), P.cell_keys(s["cell_y"], s["cell_perm"])
    assert set(ca) == set(cs)
    cam = {k: i for i, k in enumerate(ca)}
    for i, k in enumerate(cs[:20000]):
        j = cam[k]
        rs = [ks[e] for e in s["cell_idx"][s["cell_off"][i]:s["cell_off"][i + 1]]]
        ra = [ka[e] for e in a["cell_idx"][a["cell_off"][j]:a["cell_off"][j + 1]]]
        assert rs == ra  # same row, same order (vertex pairs in order)


def test_sorted_output_rejected_by_batches(ctx):
    w = W.config_d3()
    with pytest.raises(mf.MfError) as e:
        ctx.trace_batch([w], capacities=[dict(max_edges=1 << 18)], sort=True)
    assert e.value.code == mf.MF_ERR_INVALID
