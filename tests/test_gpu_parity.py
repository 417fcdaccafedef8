"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle,
element by element on seeded inputs."""
import math

import numpy as np
import pytest
import torch

import oracle
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


@pytest.mark.parametrize("d", [2, 3, 4, 5, 6, 7, 8])
def test_locate_bit_exact(ctx, d):
    rng = np.random.default_rng(100 + d)
    lam = 0.07
    o = rng.uniform(-0.03, 0.03, d)
    pts = rng.uniform(-3, 3, size=(3000, d))
    # points exactly on lattice vertices exercise the tie rule
    pts[:50] = oracle.vertex_x(d, lam, o, rng.integers(-30, 30, size=(50, d)).astype(np.int32))
    y, perm = ctx.locate(d, lam, o, pts)
    y, perm = y.cpu().numpy(), perm.cpu().numpy()
    for i in range(pts.shape[0]):
        oy, parts = oracle.locate(d, lam, o, pts[i])
        assert tuple(y[i]) == oy
        assert tuple(1 << int(p) for p in perm[i]) + (1 << d,) == parts


@pytest.mark.parametrize("d,n_sv,gamma", [(3, 64, 2.0), (5, 2048, 4.0), (6, 1000, 6.0)])
def test_eval_fp64_and_mixed(ctx, d, n_sv, gamma):
    rng = np.random.default_rng(d)
    sv = rng.uniform(-math.pi, math.pi, size=(n_sv, d))
    alpha = rng.normal(size=n_sv)
    b = 0.1
    q = rng.uniform(-math.pi, math.pi, size=(5000, d))
    k = min(200, n_sv)
    q[:k] = sv[:k] + rng.normal(scale=0.2, size=(k, d))
    fo = oracle.f(sv, alpha, gamma, b, q)
    f64 = ctx.eval(sv, alpha, gamma, b, q, precision=mf.MF_FP64).cpu().numpy()
    assert np.max(np.abs(f64 - fo)) <= 1e-12
    for prec in (mf.MF_MIXED_FP32,):
        fm = ctx.eval(sv, alpha, gamma, b, q, precision=prec, band=1e-3).cpu().numpy()
        assert np.max(np.abs(fm - fo)) <= 1e-3
        mask = np.abs(fo) >= 1e-12
        assert np.array_equal(fm[mask] >= 0, fo[mask] >= 0)
    # the BF16 tensor-core GEMM needs lattice vertices (small integer offsets
    # within a tile): arbitrary points are refused, never silently downgraded
    with pytest.raises(mf.MfError) as e:
        ctx.eval(sv, alpha, gamma, b, q, precision=mf.MF_MIXED_BF16)
    assert e.value.code == mf.MF_ERR_INVALID


@pytest.mark.parametrize("precision,exact", [(mf.MF_FP64, False), (mf.MF_MIXED_FP32, False),
                                             (mf.MF_MIXED_BF16, False), (mf.MF_MIXED_BF16, True)])
def test_d3_config_full_parity(ctx, precision, exact):
    """Roots: |dt| <= 1e-9 on the FP64 path (and on a mixed path asked for
    FP64-exact roots), <= 1e-6 on the mixed paths."""
    w = W.config_d3()
    g = P.gpu_trace(ctx, w, precision, exact_roots=exact)
    o = P.oracle_trace(w)
    t_tol = 1e-9 if precision == mf.MF_FP64 or exact else 1e-6
    rep = P.compare_traces(w, g, o, t_tol=t_tol, f_tol=1e-12 if precision == mf.MF_FP64 else 1e-3)
    assert rep["n_diff"] == 0 and rep["n_edges"] > 1000
    # certification of the traced points and cells
    vg, mg, cg = ctx.certify(w.dh, w.radius, w.obs_type, w.obs_pose, w.obs_dims, g["points"],
                             g["cell_off"], g["cell_idx"])
    vo, mo, co = oracle.certify(w.dh, w.radius, w.obs_type, w.obs_pose, w.obs_dims, g["points"],
                                g["cell_off"], g["cell_idx"])
    vg, mg, cg = vg.cpu().numpy(), mg.cpu().numpy(), cg.cpu().numpy()
    sure = np.abs(mo) > 1e-12
    assert np.array_equal(vg[sure], vo[sure])
    assert np.max(np.abs(mg - mo)) <= 1e-9
    if sure.all():
        assert np.array_equal(cg, co)


@pytest.mark.parametrize("cap", [1, 7, 100])
def test_result_independent_of_batch_cap(ctx, cap):
    w = W.random_small(3, 10, 21, 0.2, gamma=1.5, n_seeds=3, box=1.2)
    o = P.oracle_trace(w, roots=False, cells=True)
    g = P.gpu_trace(ctx, w, batch_cap=cap, roots=False)
    rep = P.compare_traces(w, g, o, check_t=False)
    assert rep["n_diff"] == 0


@pytest.mark.parametrize("d,lam,n_sv,seed", [(2, 0.05, 12, 2), (3, 0.15, 20, 2), (4, 0.3, 16, 3),
                                             (5, 0.5, 16, 4), (6, 0.7, 12, 5), (7, 0.9, 10, 6),
                                             (8, 1.1, 8, 7)])
@pytest.mark.parametrize("precision", [mf.MF_FP64, mf.MF_MIXED_FP32, mf.MF_MIXED_BF16])
def test_random_problems_parity(ctx, d, lam, n_sv, seed, precision):
    w = W.random_small(d, n_sv, seed, lam, gamma=1.5, n_seeds=4, box=1.3)
    o = P.oracle_trace(w, roots=True, cells=d <= 5)
    g = P.gpu_trace(ctx, w, precision, cells=d <= 5)
    rep = P.compare_traces(w, g, o, f_tol=1e-12 if precision == mf.MF_FP64 else 1e-3,
                           t_tol=1e-9 if precision == mf.MF_FP64 else 1e-6,
                           check_cells=d <= 5)
    assert rep["n_edges"] > 20


def test_sphere_closed_form_on_gpu(ctx):
    w = W.sphere_workload(4, r=1.0, gamma=0.8, lam=0.25)
    g = P.gpu_trace(ctx, w)
    assert g["n_edges"] > 500
    assert np.max(np.abs(np.linalg.norm(g["points"], axis=1) - 1.0)) < 1e-9
    # Euler characteristic in d = 3
    w3 = W.sphere_workload(3, r=1.0, gamma=1.0, lam=0.2)
    g3 = P.gpu_trace(ctx, w3)
    o3 = P.oracle_trace(w3)
    assert P.compare_traces(w3, g3, o3)["n_diff"] == 0
    assert g3["n_edges"] - o3["n_crossing_triangles"] + g3["n_cells"] == 2


def test_empty_and_dead_seeds(ctx):
    w = W.config_d3()
    w.seeds = np.zeros((0, 3))
    g = P.gpu_trace(ctx, w)
    assert g["n_edges"] == 0 and g["levels"] == 0
    w.seeds = np.array([[3.0, 3.0, 3.0], [100.0, 0.0, 0.0]])  # far from f = 0 / outside the box
    g = P.gpu_trace(ctx, w)
    o = P.oracle_trace(w)
    assert g["n_dead_seeds"] == o["n_dead_seeds"] == 2 and g["n_edges"] == 0


def test_error_codes(ctx):
    w = W.config_d3()
    with pytest.raises(mf.MfError) as e:
        P.gpu_trace(ctx, w, max_edges=100)
    assert e.value.code == mf.MF_ERR_MAXEDGES
    bad = W.config_d3()
    bad.lam = -1.0
    with pytest.raises(mf.MfError) as e:
        P.gpu_trace(ctx, bad)
    assert e.value.code == mf.MF_ERR_INVALID
    bad = W.config_d3()
    bad.alpha = bad.alpha.copy()
    bad.alpha[3] = np.nan
    with pytest.raises(mf.MfError) as e:
        P.gpu_trace(ctx, bad)
    assert e.value.code == mf.MF_ERR_INVALID
    # a context whose budget cannot hold the tables
    from paper_2406_04795_gb300.api import Context
    small = Context(0, 1 << 20)
    with pytest.raises(mf.MfError) as e:
        P.gpu_trace(small, w)
    assert e.value.code == mf.MF_ERR_OOM
    small.close()
    # the context stays usable after errors
    g = P.gpu_trace(ctx, w)
    assert g["n_edges"] > 1000


def test_two_call_capacity_pattern(ctx):
    w = W.config_d3()
    r = ctx.trace(w.sv, w.alpha, w.gamma, w.b, w.lam, w.offset, w.lo, w.hi, w.seeds)
    E = r["n_edges"]
    small = ctx._alloc_outputs(3, 10, 10, 10)
    out = ctx._out_struct(small, 3)
    rbf, keep = ctx.rbf(w.sv, w.alpha, w.gamma, w.b)
    dom = ctx.domain(w.lo, w.hi, w.offset)
    opts = mf.mf_trace_opts(w.lam, 1 << 24, 0, 1e-3, 1e-12, 1 << 22, 0, 0, 3)
    seeds = torch.as_tensor(w.seeds, device="cuda")
    rc = mf.mf_trace(ctx.h, rbf, dom, opts, seeds.data_ptr(), 1, out,
                     torch.cuda.current_stream().cuda_stream, check=False)
    assert rc == mf.MF_ERR_CAPACITY and out.n_edges == E
    big = ctx._alloc_outputs(3, out.n_edges, out.n_cells, out.n_cell_edges)
    out2 = ctx._out_struct(big, 3)
    mf.mf_trace_fetch(ctx.h, out2)
    assert out2.n_edges == E
    assert set(P.keys(big["edge_y"].cpu().numpy(), big["edge_mask"].cpu().numpy())) == \
        set(P.keys(r["edge_y"].cpu().numpy(), r["edge_mask"].cpu().numpy()))


@pytest.mark.parametrize("d,lam", [(5, 0.3), (6, 0.5)])
def test_tensor_core_eval_matches_fp64(ctx, d, lam):
    """The tcgen05 vertex evaluation (many 128-vertex tiles, many 64-vector
    chunks, ragged last tile) leaves every sign decision FP64-exact: the
    traced set, cells and roots equal the FP64 path's, and the FP32 values it
    keeps are within the band of the FP64 ones."""
    w = W.config_d5(lam=lam) if d == 5 else W.config_d6(lam=lam, n_sv=4096)
    a = P.gpu_trace(ctx, w, mf.MF_FP64)
    b = P.gpu_trace(ctx, w, mf.MF_MIXED_BF16, exact_roots=True)
    assert a["n_edges"] > 5000 and a["n_edges"] == b["n_edges"]
    ka = {k: i for i, k in enumerate(P.keys(a["edge_y"], a["edge_mask"]))}
    kb = P.keys(b["edge_y"], b["edge_mask"])
    assert set(kb) == set(ka)
    ia = np.array([ka[k] for k in kb])
    assert np.max(np.abs(a["edge_t"][ia] - b["edge_t"])) <= 1e-9
    assert np.max(np.abs(a["edge_f"][ia] - b["edge_f"])) <= 1e-3
    assert set(P.cell_keys(a["cell_y"], a["cell_perm"])) == set(P.cell_keys(b["cell_y"], b["cell_perm"]))
    assert 0 < b["n_recheck"] < b["n_vertices"]


@pytest.mark.parametrize("precision", [mf.MF_FP64, mf.MF_MIXED_BF16])
def test_autotune_choices_leave_results_unchanged(ctx, precision):
    """mf_autotune picks launch variants from its candidate sets, and traces
    under the tuned context equal those under the defaults element by
    element (sets, roots and cells do not depend on launch shapes)."""
    w = W.config_d5(lam=0.3)
    try:
        mf.mf_ctx_set_tune(ctx.h, None)
        base = P.gpu_trace(ctx, w, precision)
        t = ctx.autotune(w, precision=precision)
        assert t["roots_variant"] in (0, 1) and t["roots_blocks_per_sm"] in (2, 4, 8)
        assert t["eval_blocks_per_sm"] in (4, 8, 16) and t["tc_chunk"] in (64, 128)
        assert t["frontier_chunk"] in (0, 1 << 20, 1 << 18) and t["n_candidates"] >= 20
        assert t["roots_group"] in (1, 8, 16)
        assert t["ms_bfs"] > 0 and t["ms_roots"] > 0
        got = mf.mf_ctx_get_tune(ctx.h).as_dict()
        for k in ("roots_variant", "roots_blocks_per_sm", "eval_blocks_per_sm", "tc_chunk",
                  "frontier_chunk", "roots_group"):
            assert got[k] == t[k]
        tuned = P.gpu_trace(ctx, w, precision)
    finally:
        mf.mf_ctx_set_tune(ctx.h, None)
    ka = {k: i for i, k in enumerate(P.keys(base["edge_y"], base["edge_mask"]))}
    kb = P.keys(tuned["edge_y"], tuned["edge_mask"])
    assert set(kb) == set(ka)
    ia = np.array([ka[k] for k in kb])
    if precision == mf.MF_FP64:  # per-edge FP64 arithmetic: bit-identical
        assert np.array_equal(base["edge_t"][ia], tuned["edge_t"])
        assert np.array_equal(base["points"][ia], tuned["points"])
    else:  # mixed roots: each within 1e-6 of the exact root
        assert np.max(np.abs(base["edge_t"][ia] - tuned["edge_t"])) <= 2e-6
    assert set(P.cell_keys(base["cell_y"], base["cell_perm"])) == \
        set(P.cell_keys(tuned["cell_y"], tuned["cell_perm"]))


def test_set_tune_rejects_out_of_range(ctx):
    t = mf.mf_tune()
    t.roots_variant, t.roots_blocks_per_sm, t.eval_blocks_per_sm, t.roots_group = 0, 4, 8, 8
    t.tc_chunk = 96  # not a supported chunk width
    with pytest.raises(mf.MfError):
        mf.mf_ctx_set_tune(ctx.h, t)
    mf.mf_ctx_set_tune(ctx.h, None)


def test_group_screen_roots_bit_identical(ctx):
    """Edges sharing a group screen see the same candidates, in the same
    order, as a full per-edge screen: roots and points are bit-identical."""
    w = W.config_d5(lam=0.3)
    out = {}
    try:
        for g in (1, 16):
            t = mf.mf_ctx_get_tune(ctx.h)
            t.roots_group = g
            mf.mf_ctx_set_tune(ctx.h, t)
            out[g] = P.gpu_trace(ctx, w, mf.MF_FP64, cells=False)
    finally:
        mf.mf_ctx_set_tune(ctx.h, None)
    a, b = out[1], out[16]
    ka = {k: i for i, k in enumerate(P.keys(a["edge_y"], a["edge_mask"]))}
    ia = np.array([ka[k] for k in P.keys(b["edge_y"], b["edge_mask"])])
    assert np.array_equal(a["edge_t"][ia], b["edge_t"])
    assert np.array_equal(a["points"][ia], b["points"])


@pytest.mark.parametrize("cfg", ["d5", "d6"])
def test_certify_many_links_against_oracle(ctx, cfg):
    """Certification of 5- and 6-link arms (boxes; boxes and spheres) on
    random configurations: verdicts bit-exact away from |margin| < 1e-12,
    margins within 1e-9 of the oracle's."""
    w = W.config_d5() if cfg == "d5" else W.config_d6(n_sv=64)
    rng = np.random.default_rng(11)
    pts = rng.uniform(-np.pi, np.pi, size=(3000, w.d))
    vg, mg, _ = ctx.certify(w.dh, w.radius, w.obs_type, w.obs_pose, w.obs_dims, pts, None, None)
    vo, mo, _ = oracle.certify(w.dh, w.radius, w.obs_type, w.obs_pose, w.obs_dims, pts)
    vg, mg = vg.cpu().numpy(), mg.cpu().numpy()
    sure = np.abs(mo) > 1e-12
    assert np.array_equal(vg[sure], vo[sure])
    assert np.max(np.abs(mg - mo)) <= 1e-9
    assert 0 < vg.sum() < len(vg)
