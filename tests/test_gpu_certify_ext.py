"""Certification with link spheres (the paper's robot model), cylinder
obstacles (App. A) and the whole-cell certificate, on the GPU through
mf_certify_ex, against the FP64 oracle: verdicts bit-exact away from
|margin| < 1e-12, margins within 1e-9, the deciding element equal, the
whole-cell slack within 1e-9 and its verdict exact away from |slack| < 1e-9."""
import math

import numpy as np
import pytest

import oracle
from paper_2406_04795_gb300 import workloads as W
from tests import _parity as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2406_04795_gb300.api import Context
    c = Context(0, 16 << 30)
    yield c
    c.close()


def _rot(rng):
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def _scene(rng, reach, n_box=6, n_sph=4, n_cyl=6):
    types, poses, dims = [], [], []
    for typ, n in ((0, n_box), (1, n_sph), (2, n_cyl)):
        for _ in range(n):
            c = rng.uniform(-reach, reach, 3)
            R = _rot(rng) if typ != 1 else np.eye(3)
            types.append(typ)
            poses.append(np.concatenate([R.reshape(-1), c]))
            if typ == 0:
                dims.append(rng.uniform(0.1, 0.5, 3))
            elif typ == 1:
                dims.append([rng.uniform(0.05, 0.25), 0, 0])
            else:
                dims.append([rng.uniform(0.03, 0.2), rng.uniform(0.2, 0.9), 0])
    return np.array(types, np.int32), np.array(poses), np.array(dims)


def _robot(rng, n, spheres_per_link=3, radius=0.04):
    dh = np.zeros((n, 4))
    dh[:, 0] = rng.uniform(-1, 1, n)
    dh[:, 1] = rng.uniform(0, 0.2, n)
    dh[:, 2] = rng.uniform(0.2, 0.5, n)
    dh[:, 3] = rng.choice([-math.pi / 2, 0, math.pi / 2], n)
    link = np.repeat(np.arange(n), spheres_per_link).astype(np.int32)
    centre = np.stack([-rng.uniform(0, 1, link.shape[0]) * dh[link, 2],
                       rng.uniform(-0.03, 0.03, link.shape[0]),
                       rng.uniform(-0.03, 0.03, link.shape[0])], 1)
    rad = rng.uniform(0.03, 0.08, link.shape[0])
    return dh, np.full(n, radius), (link, centre, rad)


def _compare(g, o, cells=False):
    gv, gm, ge = (g[k].cpu().numpy() for k in ("verdict", "margin", "element"))
    sure = np.abs(o["margin"]) > 1e-12
    assert np.array_equal(gv[sure], o["verdict"][sure])
    assert np.max(np.abs(gm - o["margin"])) <= 1e-9
    assert np.mean(ge == o["element"]) >= 0.999
    if cells:
        gs = g["cell_slack"].cpu().numpy()
        gw = g["cell_whole"].cpu().numpy()
        assert np.array_equal(g["cell_verdict"].cpu().numpy(), o["cell_verdict"])
        assert np.max(np.abs(gs - o["cell_slack"])) <= 1e-9
        clear = np.abs(o["cell_slack"]) > 1e-9
        assert np.array_equal(gw[clear], o["cell_whole"][clear])
        return gw


@pytest.mark.parametrize("d,mode", [(5, "capsules+spheres"), (6, "spheres"), (6, "capsules")])
def test_elements_and_cylinders_against_oracle(ctx, d, mode):
    rng = np.random.default_rng(40 + d)
    dh, radius, spheres = _robot(rng, d)
    if mode == "spheres":
        radius = None
    if mode == "capsules":
        spheres = None
    types, pose, dims = _scene(rng, float(dh[:, 2].sum()) * 0.6)
    pts = rng.uniform(-math.pi, math.pi, size=(4000, d))
    g = ctx.certify_ex(dh, radius, types, pose, dims, pts, spheres=spheres)
    o = oracle.certify_ex(dh, radius, types, pose, dims, pts, spheres=spheres)
    _compare(g, o)
    v = o["verdict"]
    assert 0.05 < v.mean() < 0.95
    if spheres is not None:
        nc = 0 if radius is None else d
        assert np.any(o["element"] >= nc)  # spheres decide some points


def test_whole_cell_certificate_against_oracle(ctx):
    """Point clouds as cells (3-8 points, spreads 0.0005-0.01 rad) around
    random configurations of a 5-link arm (capsules of radius 0.06, spheres)
    among boxes, spheres and cylinders: about a quarter of the cells have
    every point in collision, and most of those are certified whole."""
    rng = np.random.default_rng(47)
    d = 5
    dh, radius, spheres = _robot(rng, d, radius=0.06)
    types, pose, dims = _scene(rng, float(dh[:, 2].sum()) * 0.9, 4, 2, 4)
    pts, off = [], [0]
    for _ in range(3000):
        m = int(rng.integers(3, 9))
        pts.append(rng.uniform(-math.pi, math.pi, d) +
                   rng.normal(scale=rng.choice([0.0005, 0.002, 0.01]), size=(m, d)))
        off.append(off[-1] + m)
    pts = np.concatenate(pts)
    off = np.array(off, np.int64)
    # the points stored in a shuffled order: the rows index them where they are
    perm = rng.permutation(pts.shape[0])
    pts = pts[perm]
    idx = np.argsort(perm).astype(np.int64)
    g = ctx.certify_ex(dh, radius, types, pose, dims, pts, off, idx, spheres=spheres)
    o = oracle.certify_ex(dh, radius, types, pose, dims, pts, off, idx, spheres=spheres)
    gw = _compare(g, o, cells=True)
    assert 50 < gw.sum() < gw.shape[0]
    assert np.all(gw <= g["cell_verdict"].cpu().numpy())
    # without the slack output the library decides cells in FP32 under its
    # error bound and recomputes the close ones in FP64: the same verdicts
    f = ctx.certify_ex(dh, radius, types, pose, dims, pts, off, idx, spheres=spheres, slack=False)
    fw = f["cell_whole"].cpu().numpy()
    clear = np.abs(o["cell_slack"]) > 1e-9
    assert np.array_equal(fw[clear], o["cell_whole"][clear])
    assert np.array_equal(fw, gw)


def test_traced_cells_whole_certificate(ctx):
    """The d=3 workload's traced points and cells: mf_certify_ex against the
    oracle on the same points and CSR, with a cylinder added to the scene."""
    w = W.config_d3()
    g = P.gpu_trace(ctx, w)
    types = np.concatenate([w.obs_type, [2]]).astype(np.int32)
    pose = np.concatenate([w.obs_pose, [np.concatenate([np.eye(3).reshape(-1), [1.2, 0.8, 0.0]])]])
    dims = np.concatenate([w.obs_dims, [[0.3, 0.5, 0.0]]])
    gc = ctx.certify_ex(w.dh, w.radius, types, pose, dims, g["points"], g["cell_off"],
                        g["cell_idx"])
    oc = oracle.certify_ex(w.dh, w.radius, types, pose, dims, g["points"], g["cell_off"],
                           g["cell_idx"])
    gw = _compare(gc, oc, cells=True)
    fc = ctx.certify_ex(w.dh, w.radius, types, pose, dims, g["points"], g["cell_off"],
                        g["cell_idx"], slack=False)
    assert np.array_equal(fc["cell_whole"].cpu().numpy(), gw)
