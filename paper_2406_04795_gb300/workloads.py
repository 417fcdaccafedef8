"""Seeded synthetic workloads for manifold tracing and certification.

This module only builds inputs: RBF decision-function parameters (support
vectors, weights, gamma, b), seeds, the lattice scale and offset, the C-space
box, and the robot/obstacle geometry.  It holds none of the tracing or
certification arithmetic, and both the CUDA path and the CPU oracle receive
exactly the arrays it returns.

The paper's scenes (Packbot, UR5, Schunk; Sec. VI) and its learned SVMs are not
available, so each workload is a stand-in with the paper's shapes: a d-DoF
serial arm with capsule links among box/sphere obstacles and an RBF-kernel SVM
decision function (Sec. IV-A) over [-pi, pi]^d.

Seeds stand in for the paper's manifold sampler (SLSQP minimising |M(q)|,
Sec. IV-A), which is not part of the traced path: they are placed by plain
numpy bisection between a point with f < 0 and one with f >= 0.  The traced
set depends only on the n-simplex each seed falls in.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BOX, SPHERE = 0, 1


@dataclasses.dataclass
class Workload:
    name: str
    d: int
    sv: np.ndarray          # [N, d] support vectors
    alpha: np.ndarray       # [N] dual weights (signed)
    gamma: float
    b: float
    lam: float              # lattice scale lambda_T
    offset: np.ndarray      # [d] lattice offset o
    lo: np.ndarray          # [d] C-space box
    hi: np.ndarray
    seeds: np.ndarray       # [S, d]
    dh: np.ndarray          # [d, 4] theta0, d, a, alpha (DH) per link
    radius: np.ndarray      # [d] capsule radius per link
    obs_type: np.ndarray    # [M] BOX / SPHERE
    obs_pose: np.ndarray    # [M, 12] R (row-major, local->world) then t
    obs_dims: np.ndarray    # [M, 3] box side lengths / sphere radius in [0]
    batch_cap: int = 1 << 24
    precision: str = "fp64"
    recheck_band: float = 1e-3
    meta: dict = dataclasses.field(default_factory=dict)


def lattice_offset(d: int, lam: float) -> np.ndarray:
    """A fixed, generic lattice offset so that seeds and constructed zeros do
    not sit on lattice vertices."""
    i = np.arange(d, dtype=np.float64)
    return lam * np.modf(i * 0.6180339887498949 + 0.5)[0] / 7.0


def _rbf_numpy(sv, alpha, gamma, b, q):
    # Used only to place seeds (stand-in for the out-of-scope manifold sampler).
    q = np.atleast_2d(q)
    d2 = ((q[:, None, :] - sv[None, :, :]) ** 2).sum(-1)
    return np.exp(-gamma * d2) @ alpha + b


def place_seeds(rng, sv, alpha, gamma, b, lo, hi, n_seeds, inner=None, step=0.05, max_steps=200):
    """Seeds on f = 0: march from an inner point (f < 0) along a random
    direction until f >= 0, then bisect 60 times."""
    d = sv.shape[1]
    if inner is None:
        cand = np.concatenate([sv, rng.uniform(lo, hi, size=(4096, d))])
        fc = _rbf_numpy(sv, alpha, gamma, b, cand)
        inner = cand[fc < 0]
    else:
        # the march stays within max_steps * step of the inner points: support
        # vectors farther than that plus sqrt(30 / gamma) add < e^-30 each
        reach = max_steps * step + math.sqrt(30.0 / gamma)
        dist = np.min(np.linalg.norm(sv[:, None, :] - inner[None, :, :], axis=2), axis=1)
        keep = dist <= reach
        sv, alpha = sv[keep], alpha[keep]
    if inner.shape[0] == 0:
        raise ValueError("no point with f < 0 to start from")
    seeds = []
    tries = 0
    while len(seeds) < n_seeds and tries < 100 * n_seeds:
        tries += 1
        a = inner[rng.integers(inner.shape[0])]
        u = rng.normal(size=d)
        u /= np.linalg.norm(u)
        fa = _rbf_numpy(sv, alpha, gamma, b, a)[0]
        if fa >= 0:
            continue
        bpt = None
        for k in range(1, max_steps + 1):
            p = a + k * step * u
            if np.any(p < lo) or np.any(p > hi):
                break
            if _rbf_numpy(sv, alpha, gamma, b, p)[0] >= 0:
                bpt = p
                break
        if bpt is None:
            continue
        x0, x1 = a.copy(), bpt.copy()
        for _ in range(60):
            m = 0.5 * (x0 + x1)
            if _rbf_numpy(sv, alpha, gamma, b, m)[0] >= 0:
                x1 = m
            else:
                x0 = m
        seeds.append(0.5 * (x0 + x1))
    if len(seeds) < n_seeds:
        raise ValueError("could not place %d seeds" % n_seeds)
    return np.array(seeds)


def _aabb_pose(center):
    pose = np.zeros(12)
    pose[[0, 4, 8]] = 1.0
    pose[9:12] = center
    return pose


def _ball(rng, n, radius):
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    r = radius * rng.uniform(size=(n, 1)) ** (1.0 / 3.0)
    return u * r


def _dh_arm(rng, d, radius):
    dh = np.zeros((d, 4))
    dh[:, 1] = rng.uniform(0.0, 0.2, size=d)
    dh[:, 2] = rng.uniform(0.2, 0.5, size=d)
    dh[:, 3] = rng.choice([-math.pi / 2, 0.0, math.pi / 2], size=d)
    return dh, np.full(d, radius)


def _svm_stand_in(rng, d, n_sv, p_neg, b):
    """Support vectors uniform in the C-space box; alpha = label * |N(0,1)|
    with a share p_neg of free-space (negative) labels; fixed bias b > 0, so
    the zero set is a family of closed shells around free-space vectors."""
    sv = rng.uniform(-math.pi, math.pi, size=(n_sv, d))
    lab = np.where(rng.uniform(size=n_sv) < p_neg, -1.0, 1.0)
    alpha = lab * np.abs(rng.normal(size=n_sv))
    return sv, alpha, float(b)


def config_d3(seed: int = 1000, lam: float = 0.1) -> Workload:
    """d=3 plain FP64: 64 SVs uniform in [-pi,pi]^3, alpha ~ N(0,1), gamma=2,
    b so that f(0) = 0, one seed at the origin (a zero of f by construction),
    lambda=0.1, planar 3-link arm (unit links, capsule r=0.05) among 4 random
    axis-aligned boxes."""
    rng = np.random.default_rng(seed)
    d = 3
    sv = rng.uniform(-math.pi, math.pi, size=(64, d))
    alpha = rng.normal(size=64)
    gamma = 2.0
    b = -float(np.sum(alpha * np.exp(-gamma * np.sum(sv * sv, axis=1))))
    dh = np.zeros((3, 4))
    dh[:, 2] = 1.0
    radius = np.full(3, 0.05)
    centers = np.zeros((4, 3))
    centers[:, :2] = rng.uniform(-2.5, 2.5, size=(4, 2))
    half = rng.uniform(0.1, 0.5, size=(4, 3))
    lo, hi = np.full(d, -math.pi), np.full(d, math.pi)
    return Workload("d3_fp64_64sv", d, sv, alpha, gamma, b, lam, lattice_offset(d, lam), lo, hi,
                    np.zeros((1, d)), dh, radius, np.zeros(4, np.int32),
                    np.stack([_aabb_pose(c) for c in centers]), 2.0 * half,
                    batch_cap=1 << 24, precision="fp64")


def config_d5(seed: int = 1001, lam: float = 0.05, n_sv: int = 2048, n_seeds: int = 16,
              b: float = 0.6, p_neg: float = 0.3) -> Workload:
    """d=5 plain FP64: 5-DoF DH arm (a in [0.2,0.5], d in [0,0.2], link twist
    in {-pi/2, 0, pi/2}, capsules r=0.04) among 12 random boxes; RBF with 2048
    SVs from seeded C-space samples, gamma=4; lambda=0.05; 16 seeds; batch cap
    2^24 edges."""
    rng = np.random.default_rng(seed)
    d = 5
    dh, radius = _dh_arm(rng, d, 0.04)
    reach = float(dh[:, 2].sum())
    centers = _ball(rng, 12, reach)
    half = rng.uniform(0.05, 0.3, size=(12, 3))
    sv, alpha, b = _svm_stand_in(rng, d, n_sv, p_neg, b)
    gamma = 4.0
    lo, hi = np.full(d, -math.pi), np.full(d, math.pi)
    seeds = place_seeds(rng, sv, alpha, gamma, b, lo, hi, n_seeds)
    return Workload("d5_fp64_%dsv" % n_sv, d, sv, alpha, gamma, b, lam, lattice_offset(d, lam),
                    lo, hi, seeds, dh, radius, np.zeros(12, np.int32),
                    np.stack([_aabb_pose(c) for c in centers]), 2.0 * half,
                    batch_cap=1 << 24, precision="fp64")


def config_d6(seed: int = 1002, lam: float = 0.04, n_sv: int = 8192, n_seeds: int = 64,
              b: float = 0.6, p_neg: float = 0.3) -> Workload:
    """d=6 mixed precision: 6-DoF arm among 10 boxes + 10 spheres; RBF with
    8192 SVs, gamma=6; distance GEMM in BF16 with FP32 accumulation, FP64
    recheck band |f| < 1e-3; lambda=0.04; 64 seeds."""
    rng = np.random.default_rng(seed)
    d = 6
    dh, radius = _dh_arm(rng, d, 0.04)
    reach = float(dh[:, 2].sum())
    cb = _ball(rng, 10, reach)
    cs = _ball(rng, 10, reach)
    half = rng.uniform(0.05, 0.3, size=(10, 3))
    rs = rng.uniform(0.05, 0.25, size=10)
    sv, alpha, b = _svm_stand_in(rng, d, n_sv, p_neg, b)
    gamma = 6.0
    lo, hi = np.full(d, -math.pi), np.full(d, math.pi)
    seeds = place_seeds(rng, sv, alpha, gamma, b, lo, hi, n_seeds)
    types = np.array([BOX] * 10 + [SPHERE] * 10, np.int32)
    poses = np.stack([_aabb_pose(c) for c in np.concatenate([cb, cs])])
    dims = np.concatenate([2.0 * half, np.stack([rs, np.zeros(10), np.zeros(10)], 1)])
    return Workload("d6_mixed_%dsv" % n_sv, d, sv, alpha, gamma, b, lam, lattice_offset(d, lam),
                    lo, hi, seeds, dh, radius, types, poses, dims,
                    batch_cap=1 << 24, precision="mixed", recheck_band=1e-3)


# shell radius in lattice units per dimension: bounds the traced set of a
# batched / served trace to about 1e5 - 3e6 edges
SHELL_LATTICE_RADIUS = {2: 12.0, 3: 10.0, 4: 8.0, 5: 5.0, 6: 3.0, 7: 2.5, 8: 2.0}


def shell_trace(rng, d: int, n_sv: int, lam: float, n_seeds: int, n_free: int = 1,
                b: float = 0.5, name: str = "shell") -> Workload:
    """One trace of the batched and served workloads: n_sv support vectors
    uniform in [-pi, pi]^d, obstacle-class weights alpha = +|N(0,1)|/2 and
    n_free free-space vectors with alpha = -2; gamma is chosen so that a free
    vector's shell 2 exp(-gamma r^2) = b has radius SHELL_LATTICE_RADIUS[d] *
    lambda; all seeds lie on the free vectors' shells."""
    sv = rng.uniform(-math.pi, math.pi, size=(n_sv, d))
    alpha0 = 0.5 * np.abs(rng.normal(size=n_sv))
    r_shell = min(SHELL_LATTICE_RADIUS.get(d, 2.0) * lam, 0.8)
    gamma = math.log(2.0 / b) / (r_shell * r_shell)
    lo, hi = np.full(d, -math.pi), np.full(d, math.pi)
    for attempt in range(32):
        # a free vector crowded by obstacle vectors may have f >= 0 at its
        # centre: draw other free vectors
        alpha = alpha0.copy()
        free = rng.choice(n_sv, size=n_free, replace=False)
        alpha[free] = -2.0
        try:
            seeds = place_seeds(rng, sv, alpha, gamma, b, lo, hi, n_seeds, inner=sv[free],
                                step=0.25 * r_shell, max_steps=16)
            break
        except ValueError:
            if attempt == 31:
                raise
    dh, radius = _dh_arm(rng, d, 0.04)
    reach = float(dh[:, 2].sum())
    centers = _ball(rng, 8, reach)
    half = rng.uniform(0.05, 0.3, size=(8, 3))
    return Workload(name, d, sv, alpha, gamma, b, lam, lattice_offset(d, lam), lo, hi, seeds, dh,
                    radius, np.zeros(8, np.int32), np.stack([_aabb_pose(c) for c in centers]),
                    2.0 * half, precision="mixed")


def shell_capacity(w) -> dict:
    """Table capacities for one shell trace: its shells hold a fixed number of
    lattice radii, so edges depend on d only (measured: d=4 ~1e5, d=5 ~5e5,
    d=6 ~1e6 per two shells); cells per edge grow with d."""
    me = {2: 1 << 16, 3: 1 << 17, 4: 1 << 19, 5: 1 << 21, 6: 1 << 22}.get(w.d, 1 << 22)
    cells_per_edge = {2: 2, 3: 3, 4: 8, 5: 12, 6: 32}.get(w.d, 40)
    return dict(max_edges=me, max_vertices=me, max_cells=me * cells_per_edge)


def config_batched(seed: int = 1003, n_traces: int = 64, lam_scale: float = 1.0):
    """Batched: 64 independent traces, d in {4,5,6}, 256-8192 support vectors
    log-uniform, lambda in [0.03, 0.1], 1-64 seeds each (lam_scale > 1 makes
    every lattice coarser for quick tests)."""
    rng = np.random.default_rng(seed)
    out = []
    for t in range(n_traces):
        d = int(rng.integers(4, 7))
        n_sv = int(round(math.exp(rng.uniform(math.log(256), math.log(8192)))))
        lam = float(rng.uniform(0.03, 0.1)) * lam_scale
        n_seeds = int(rng.integers(1, 65))
        out.append(shell_trace(rng, d, n_sv, lam, n_seeds, n_free=int(rng.integers(1, 3)),
                               name="batch%d_d%d_%dsv" % (t, d, n_sv)))
    return out


def served_requests(seed: int = 1005, n_requests: int = 2000, rate_hz: float = 50.0,
                    lam_scale: float = 1.0):
    """Served: a Poisson stream (exponential inter-arrival times, mean
    1/rate) of proof requests, d in {4,5,6}, 512-8192 support vectors
    log-uniform, lambda in [0.03, 0.08].  Returns (arrival_s, workloads)."""
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate_hz, size=n_requests))
    reqs = []
    for i in range(n_requests):
        d = int(rng.integers(4, 7))
        n_sv = int(round(math.exp(rng.uniform(math.log(512), math.log(8192)))))
        lam = float(rng.uniform(0.03, 0.08)) * lam_scale
        n_seeds = int(rng.integers(1, 17))
        reqs.append(shell_trace(rng, d, n_sv, lam, n_seeds, name="req%d_d%d_%dsv" % (i, d, n_sv)))
    return arrivals, reqs


def sphere_workload(d: int, r: float = 1.0, gamma: float = 1.0, lam: float = 0.2,
                    center=None) -> Workload:
    """One-SV RBF whose zero set is exactly the sphere |q - c| = r:
    f = -exp(-gamma |q - c|^2) + exp(-gamma r^2)."""
    c = np.zeros(d) if center is None else np.asarray(center, np.float64)
    sv = c[None, :].copy()
    alpha = np.array([-1.0])
    b = math.exp(-gamma * r * r)
    seed = c.copy()
    seed[0] += r
    lo, hi = np.full(d, -math.pi), np.full(d, math.pi)
    dh = np.zeros((d, 4))
    dh[:, 2] = 1.0
    return Workload("sphere_d%d" % d, d, sv, alpha, gamma, b, lam, lattice_offset(d, lam), lo, hi,
                    seed[None, :], dh, np.full(d, 0.05), np.zeros(0, np.int32),
                    np.zeros((0, 12)), np.zeros((0, 3)))


def plane_workload(d: int, lam: float = 0.2, gamma: float = 0.5, rng_seed: int = 7) -> Workload:
    """Two SVs with alpha = (+1, -1), b = 0: the zero set is the bisector
    hyperplane of the two support vectors."""
    rng = np.random.default_rng(rng_seed)
    s1 = rng.uniform(-1, 1, size=d)
    s2 = rng.uniform(-1, 1, size=d)
    sv = np.stack([s1, s2])
    alpha = np.array([1.0, -1.0])
    seed = 0.5 * (s1 + s2)
    lo, hi = np.full(d, -1.0), np.full(d, 1.0)
    dh = np.zeros((d, 4))
    dh[:, 2] = 1.0
    return Workload("plane_d%d" % d, d, sv, alpha, gamma, 0.0, lam, lattice_offset(d, lam), lo, hi,
                    seed[None, :], dh, np.full(d, 0.05), np.zeros(0, np.int32),
                    np.zeros((0, 12)), np.zeros((0, 3)))


def random_small(d: int, n_sv: int, seed: int, lam: float, gamma: float = 2.0, n_seeds: int = 4,
                 box: float = 1.5, b: float = 0.3, p_neg: float = 0.5) -> Workload:
    """Small random RBF problems for brute-force and parity tests."""
    rng = np.random.default_rng(seed)
    sv = rng.uniform(-box, box, size=(n_sv, d))
    lab = np.where(rng.uniform(size=n_sv) < p_neg, -1.0, 1.0)
    alpha = lab * (0.5 + np.abs(rng.normal(size=n_sv)))
    lo, hi = np.full(d, -box), np.full(d, box)
    seeds = place_seeds(rng, sv, alpha, gamma, b, lo, hi, n_seeds)
    dh, radius = _dh_arm(rng, d, 0.04)
    return Workload("rand_d%d_%d" % (d, seed), d, sv, alpha, gamma, b, lam,
                    lattice_offset(d, lam), lo, hi, seeds, dh, radius,
                    np.zeros(0, np.int32), np.zeros((0, 12)), np.zeros((0, 3)))
