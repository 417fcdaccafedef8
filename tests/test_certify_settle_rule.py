"""The rule that settles a point of the certification with at most two exact
pair evaluations, restated on the host and checked against the oracle's full
search (App. A distances, the deciding element = the lowest index within
1e-9 of the maximum margin).

Per (element, obstacle) pair the first pass has an upper bound ub and a
lower bound lb on the pair's exact margin (radius - distance); pairs with a
point provably inside the obstacle have margin exactly the radius.  With
L = max(radius of those elements, lb of the two pairs with the largest ub),
a point is settled when the third-largest ub lies below L - 4e-6 (1 + |L|):
its margin is then the maximum over those elements and the (at most two)
pairs among the top two whose ub reaches that threshold.  Here the bounds are
the oracle's exact margins widened by random amounts up to the slack the
kernel allows, and every settled point must reproduce the oracle's margin
and deciding element."""
import numpy as np
import pytest

import oracle
from paper_2406_04795_gb300 import workloads as W

TIE = 1e-9


def _mixed_scene(w, rng):
    """The workload's boxes, every third turned into a sphere and every
    third (offset by one) into a cylinder (App. A's obstacle types)."""
    types = np.array(w.obs_type, dtype=np.int32).copy()
    dims = np.array(w.obs_dims, dtype=np.float64).copy()
    for k in range(len(types)):
        if k % 3 == 0:
            types[k] = 1  # sphere: radius in dims[0]
            dims[k] = [dims[k].min() / 2, 0.0, 0.0]
        elif k % 3 == 1:
            types[k] = 2  # cylinder: radius, height
            dims[k] = [dims[k][0] / 2, dims[k][2], 0.0]
    return types, dims


@pytest.mark.parametrize("scene", ["boxes", "boxes_spheres_cylinders"])
def test_settled_points_match_the_full_search(scene):
    w = W.config_d5(lam=0.6)
    rng = np.random.default_rng(21)
    if scene != "boxes":
        types, dims = _mixed_scene(w, rng)
        w.obs_type, w.obs_dims = types, dims
    NL = w.dh.shape[0]
    pts = rng.uniform(-np.pi, np.pi, size=(300, NL))
    o = oracle.certify_ex(w.dh, w.radius, w.obs_type, w.obs_pose, w.obs_dims, pts)
    settled = 0
    for p, q in enumerate(pts):
        org = oracle.fk(w.dh, w.radius, q)
        m = np.empty((NL, len(w.obs_type)))
        deep = np.zeros(NL, bool)
        for e in range(NL):
            for k in range(len(w.obs_type)):
                dist = oracle.segment_obstacle_dist(org[e], org[e + 1], int(w.obs_type[k]),
                                                    w.obs_pose[k], w.obs_dims[k])
                m[e, k] = w.radius[e] - dist
                if dist == 0.0:
                    deep[e] = True
        # bounds: exact margins widened by up to the kernel's slack
        ub = m + rng.uniform(0, 3e-4, m.shape)
        lb = m - rng.uniform(0, 3e-4, m.shape)
        pairs = [(ub[e, k], lb[e, k], e, k) for e in range(NL) for k in range(m.shape[1])
                 if not (deep[e] and m[e, k] == w.radius[e])]
        pairs.sort(key=lambda t: -t[0])
        best_in = max((w.radius[e] for e in range(NL) if deep[e]), default=-np.inf)
        if not pairs:
            continue
        ub3 = pairs[2][0] if len(pairs) > 2 else -np.inf
        L = max(best_in, pairs[0][1], pairs[1][1] if len(pairs) > 1 else -np.inf)
        thr = L - 4e-6 * (1 + abs(L))
        if not ub3 < thr:
            continue  # the full search decides this point
        settled += 1
        cand = [(m[e, k], e) for (u, _, e, k) in pairs[:2] if u >= thr]
        best = max([w.radius[e] for e in range(NL) if deep[e]] + [mc for mc, _ in cand])
        be = min([e for e in range(NL) if deep[e] and w.radius[e] >= best - TIE] +
                 [e for mc, e in cand if mc >= best - TIE])
        assert abs(best - o["margin"][p]) <= 1e-12
        if abs(best - o["margin"][p]) < 1e-12 and all(
                abs(x - (best - TIE)) > 1e-12 for x in m.max(axis=1)):
            assert be == o["element"][p]
    assert settled > 200  # the rule settles most points
