"""The numerical claims behind the certification kernel, checked on the host
against the oracle's exact segment/box distance (App. A).

In the box frame the squared distance along the segment,
F(t) = sum_i max(0, |a_i + t dl_i| - h_i)^2, is convex and C^1, so for any t
in [0, 1]: min F >= F(t) - |F'(t)| (t or 1 - t).  The kernel uses this twice:
  - in FP32, after three clamped Newton steps, as a lower bound on every
    pair's distance (with a rounding allowance eta and the 1e-4 (1 + scale)
    slack);
  - in FP64, as the certificate that accepts a Newton minimiser as exact to
    2e-12 in the distance.
It also takes the squared distance at the FP32 Newton point, plus eta, as an
upper bound (the first certification pass's lower bound on a pair's
margin).  This test restates these steps in numpy (float32 / float64) and
checks them against the oracle on random segments and boxes."""
import math

import numpy as np

import oracle


def _local(a, b, R, t):
    return R.T @ (a - t), R.T @ (b - t)


def _newton_tangent(a, dl, h, t, steps, dtype):
    a, dl, h = (np.asarray(v, dtype) for v in (a, dl, h))
    t = dtype(t)
    F = G = dtype(0)
    for it in range(steps + 1):
        F = G = H = dtype(0)
        for i in range(3):
            p = dtype(t * dl[i] + a[i])
            q = dtype(abs(p) - h[i])
            if q > 0:
                F = dtype(F + q * q)
                G = dtype(G + math.copysign(q, p) * dl[i])
                H = dtype(H + dl[i] * dl[i])
        if it < steps and H > 0:
            t = dtype(min(max(t - G / H, 0), 1))
    room = dtype(2 * abs(G) * (t if G > 0 else 1 - t))
    return t, F, room


def test_fp32_tangent_bound_is_a_lower_bound():
    rng = np.random.default_rng(11)
    gaps = []
    for _ in range(3000):
        R, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        tt = rng.uniform(-1, 1, 3)
        h = rng.uniform(0.02, 0.4, 3)
        pa = rng.uniform(-1.5, 1.5, 3)
        pb = pa + rng.normal(scale=0.4, size=3)
        exact = oracle.segment_obstacle_dist(pa, pb, 0, np.concatenate([R.reshape(-1), tt]), 2 * h)
        a, b = _local(pa.astype(np.float32), pb.astype(np.float32), R.astype(np.float32),
                      tt.astype(np.float32))
        dl = b - a
        dd = float(dl @ dl)
        t0 = min(max(-float(a @ dl) / dd, 0.0), 1.0) if dd > 0 else 0.0
        _, F, room = _newton_tangent(a, dl, h, t0, 3, np.float32)
        scale = max(1.0, np.abs(pa).max(), np.abs(pb).max(), (np.abs(tt) + h).max())
        eta = 4e-5 * (1 + scale) ** 2
        lbF = F - room - eta
        lb = math.sqrt(lbF) if lbF > 0 else 0.0
        assert lb - 1e-4 * (1 + scale) <= exact
        gaps.append(exact - lb)
    assert np.median(gaps) < 1e-3  # tight enough to prune


def test_fp32_upper_bound_is_an_upper_bound():
    """The first certification pass also bounds each pair's distance from
    above: the squared distance at the FP32 Newton point plus the rounding
    allowance eta, then the same 1e-4 (1 + scale) slack.  radius minus that
    is the lower bound on the pair's margin that lets one or two exact
    evaluations settle a point; it must never exceed the exact margin."""
    rng = np.random.default_rng(14)
    gaps = []
    for _ in range(3000):
        R, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        tt = rng.uniform(-1, 1, 3)
        h = rng.uniform(0.02, 0.4, 3)
        pa = rng.uniform(-1.5, 1.5, 3)
        pb = pa + rng.normal(scale=0.4, size=3)
        exact = oracle.segment_obstacle_dist(pa, pb, 0, np.concatenate([R.reshape(-1), tt]), 2 * h)
        a, b = _local(pa.astype(np.float32), pb.astype(np.float32), R.astype(np.float32),
                      tt.astype(np.float32))
        dl = b - a
        dd = float(dl @ dl)
        t0 = min(max(-float(a @ dl) / dd, 0.0), 1.0) if dd > 0 else 0.0
        _, F, _ = _newton_tangent(a, dl, h, t0, 3, np.float32)
        scale = max(1.0, np.abs(pa).max(), np.abs(pb).max(), (np.abs(tt) + h).max())
        eta = 4e-5 * (1 + scale) ** 2
        ub = float(np.float32(math.sqrt(float(F) + eta)) * np.float32(1.000001))
        assert ub + 1e-4 * (1 + scale) >= exact
        gaps.append(ub - exact)
    assert np.median(gaps) < 1e-3  # tight enough to settle most points


def test_fp64_certificate_accepts_only_exact_minima():
    rng = np.random.default_rng(12)
    accepted = 0
    for _ in range(3000):
        R, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        tt = rng.uniform(-1, 1, 3)
        h = rng.uniform(0.02, 0.4, 3)
        pa = rng.uniform(-1.5, 1.5, 3)
        pb = pa + rng.normal(scale=0.4, size=3)
        exact = oracle.segment_obstacle_dist(pa, pb, 0, np.concatenate([R.reshape(-1), tt]), 2 * h)
        a, b = _local(pa, pb, R, tt)
        dl = b - a
        # start from a float32-accurate minimiser, as the kernel does
        t32, _, _ = _newton_tangent(a.astype(np.float32), dl.astype(np.float32),
                                    h.astype(np.float32), 0.5, 3, np.float32)
        _, F, room = _newton_tangent(a, dl, h, float(t32), 2, np.float64)
        D = math.sqrt(F)
        if room <= 2e-12 * D:
            accepted += 1
            assert abs(D - exact) <= 2e-12 + 1e-14 * (1 + exact)
    assert accepted > 2500  # the breakpoint fallback is rare


def test_table_driven_sincos_method():
    """The FP64 chain's sin/cos: x = k pi/64 + r with a two-part pi/64 (the
    first part has 25 significant bits), a 128-entry table of sin/cos(j pi/64)
    and Taylor polynomials on |r| <= pi/128 (Tang, 1991).  Restated here in
    float64; within a few ulps of libm for |x| <= 20."""
    p1 = float.fromhex("0x1.921fb5p-5")
    p2 = 4.966642116727561e-10
    assert abs((p1 + p2) - math.pi / 64) < 1e-17
    assert (p1 * 2 ** 29).is_integer()  # k * p1 exact for |k| < 2^28
    tab = [(math.sin(j * math.pi / 64), math.cos(j * math.pi / 64)) for j in range(128)]
    rng = np.random.default_rng(13)
    worst = 0.0
    for x in rng.uniform(-20, 20, 50000):
        kd = float(np.rint(x * 20.371832715762604))
        r = (x - kd * p1) - kd * p2
        s0, c0 = tab[int(kd) & 127]
        r2 = r * r
        sr = r * r2 * (r2 * (r2 * (-1 / 5040) + 1 / 120) - 1 / 6) + r
        cm = r2 * (r2 * (r2 * (r2 * (1 / 40320) - 1 / 720) + 1 / 24) - 0.5)
        s = s0 * cm + (c0 * sr + s0)
        c = c0 * cm + (-s0 * sr + c0)
        worst = max(worst, abs(s - math.sin(x)), abs(c - math.cos(x)))
    assert worst < 1e-15
