"""Pins of the oracle's certification (CPU only): forward kinematics against
closed forms, capsule/obstacle distances against App. A's sphere/box test and
against dense sampling."""
import math

import numpy as np
import pytest

import oracle


def _rot(rng):
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def _pose(R, t):
    return np.concatenate([R.reshape(-1), t])


def test_fk_planar_arm_closed_form():
    rng = np.random.default_rng(0)
    dh = np.zeros((3, 4))
    dh[:, 2] = 1.0
    for _ in range(50):
        q = rng.uniform(-math.pi, math.pi, 3)
        org = oracle.fk(dh, np.full(3, 0.05), q)
        cum = np.cumsum(q)
        expect = np.zeros((4, 3))
        expect[1:, 0] = np.cumsum(np.cos(cum))
        expect[1:, 1] = np.cumsum(np.sin(cum))
        np.testing.assert_allclose(org, expect, atol=1e-13)


def test_fk_dh_link_lengths_and_twist():
    rng = np.random.default_rng(1)
    for _ in range(20):
        n = 6
        dh = np.zeros((n, 4))
        dh[:, 0] = rng.uniform(-1, 1, n)
        dh[:, 1] = rng.uniform(0, 0.2, n)
        dh[:, 2] = rng.uniform(0.2, 0.5, n)
        dh[:, 3] = rng.choice([-math.pi / 2, 0, math.pi / 2], n)
        q = rng.uniform(-math.pi, math.pi, n)
        org = oracle.fk(dh, np.full(n, 0.04), q)
        lens = np.linalg.norm(np.diff(org, axis=0), axis=1)
        np.testing.assert_allclose(lens, np.hypot(dh[:, 1], dh[:, 2]), rtol=1e-12)
    # first link: origin moves d_0 along z then a_0 along the rotated x axis
    dh = np.array([[0.3, 0.1, 0.4, 0.7]])
    org = oracle.fk(dh, [0.05], [0.2])
    np.testing.assert_allclose(org[1], [0.4 * math.cos(0.5), 0.4 * math.sin(0.5), 0.1], atol=1e-14)


def _appendix_a_sphere_box_collides(p_world, r, R, t, l):
    """App. A, sphere vs box, written from the three steps of the appendix
    (the vertex-region sum reads (p_i - l_i/2)^2)."""
    p = np.abs(R.T @ (p_world - t))
    h = l / 2.0
    if np.any(p - h > r):  # outside the box padded by r
        return False
    out = p > h
    if out.sum() == 2:  # edge region
        j, k = np.nonzero(out)[0]
        if (p[j] - h[j]) ** 2 + (p[k] - h[k]) ** 2 > r * r:
            return False
    if out.sum() == 3:  # vertex region
        if np.sum((p - h) ** 2) > r * r:
            return False
    return True


def test_sphere_box_matches_appendix_a():
    rng = np.random.default_rng(2)
    n_col = n_free = 0
    for _ in range(4000):
        R = _rot(rng)
        t = rng.uniform(-1, 1, 3)
        l = rng.uniform(0.1, 1.0, 3)
        c = t + rng.uniform(-1.2, 1.2, 3)
        r = rng.uniform(0.01, 0.4)
        dist = oracle.segment_obstacle_dist(c, c, 0, _pose(R, t), l)
        ours = dist <= r
        if abs(dist - r) < 1e-9:
            continue
        assert ours == _appendix_a_sphere_box_collides(c, r, R, t, l)
        n_col += ours
        n_free += not ours
    assert n_col > 200 and n_free > 200


def _point_box(P, h):
    u = np.maximum(np.abs(P) - h, 0.0)
    return np.sqrt(np.sum(u * u, axis=-1))


@pytest.mark.parametrize("seed", [3, 4])
def test_capsule_box_distance_vs_dense_sampling(seed):
    rng = np.random.default_rng(seed)
    for _ in range(400):
        R = _rot(rng)
        t = rng.uniform(-1, 1, 3)
        l = rng.uniform(0.1, 1.0, 3)
        a = t + rng.uniform(-1.5, 1.5, 3)
        b = a + rng.uniform(-1, 1, 3)
        dist = oracle.segment_obstacle_dist(a, b, 0, _pose(R, t), l)
        ts = np.linspace(0, 1, 20001)[:, None]
        P = (a + ts * (b - a) - t) @ R
        samp = _point_box(P, l / 2).min()
        seglen = np.linalg.norm(b - a)
        assert dist <= samp + 1e-12
        assert samp - dist <= seglen / 20000 + 1e-12


def test_capsule_sphere_distance_vs_dense_sampling():
    rng = np.random.default_rng(5)
    for _ in range(400):
        t = rng.uniform(-1, 1, 3)
        rad = rng.uniform(0.05, 0.5)
        a = t + rng.uniform(-1.5, 1.5, 3)
        b = a + rng.uniform(-1, 1, 3)
        dist = oracle.segment_obstacle_dist(a, b, 1, _pose(np.eye(3), t), [rad, 0, 0])
        ts = np.linspace(0, 1, 20001)[:, None]
        samp = np.maximum(np.linalg.norm(a + ts * (b - a) - t, axis=1) - rad, 0).min()
        assert dist <= samp + 1e-12
        assert samp - dist <= np.linalg.norm(b - a) / 20000 + 1e-12


def test_segment_segment_distance_vs_grid():
    rng = np.random.default_rng(6)
    s = np.linspace(0, 1, 801)
    for k in range(100):
        p1, q1, p2 = rng.uniform(-1, 1, (3, 3))
        q2 = p2 + (q1 - p1) * 0.7 if k % 10 == 0 else rng.uniform(-1, 1, 3)  # some parallel
        dist = oracle.segseg_dist(p1, q1, p2, q2)
        A = p1 + s[:, None] * (q1 - p1)
        Bp = p2 + s[:, None] * (q2 - p2)
        grid = np.linalg.norm(A[:, None, :] - Bp[None, :, :], axis=2).min()
        assert dist <= grid + 1e-12
        assert grid - dist <= (np.linalg.norm(q1 - p1) + np.linalg.norm(q2 - p2)) / 800 + 1e-12


def test_certify_verdicts_margins_and_cells():
    dh = np.zeros((3, 4))
    dh[:, 2] = 1.0
    radius = np.full(3, 0.05)
    # one box straddling the first link when q1 = 0, far from it when q1 = pi/2
    types = np.array([0])
    pose = _pose(np.eye(3), np.array([0.5, 0.0, 0.0]))[None]
    dims = np.array([[0.2, 0.2, 0.2]])
    pts = np.array([[0.0, 0.3, 0.3], [math.pi / 2, math.pi / 2, 0.0], [0.0, 0.0, 0.0]])
    off = np.array([0, 2, 3])
    idx = np.array([0, 1, 2])
    v, m, cv = oracle.certify(dh, radius, types, pose, dims, pts, off, idx)
    assert v.tolist() == [1, 0, 1]
    assert m[0] == pytest.approx(0.05) and m[2] == pytest.approx(0.05)
    assert m[1] < 0
    assert cv.tolist() == [0, 1]
