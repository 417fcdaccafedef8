"""Plain FP64 CPU oracle for Coxeter-triangulation manifold tracing and capsule
certification (arXiv 2406.04795, Sec. II-B, IV, V-C and App. A).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library
(``paper_2406_04795_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``mf_oracle.c`` (plain C, ``-ffp-contract=off``); this
module only marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mf_oracle.c")
_LIB = os.path.join(_HERE, "libmf_oracle.so")
MAXD = 8


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, FP64, no contraction) next to its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def set_threads(n: int) -> int:
    """Host threads of the oracle's per-edge and per-point loops (n <= 0:
    all cores); returns the count in use.  Results do not depend on it."""
    return int(lib().or_set_threads(int(n)))


class Simplex(C.Structure):
    _fields_ = [("y", C.c_int32 * MAXD), ("k", C.c_int32), ("part", C.c_uint32 * (MAXD + 1))]


class Rbf(C.Structure):
    _fields_ = [("d", C.c_int32), ("n_sv", C.c_int64), ("sv", C.POINTER(C.c_double)),
                ("alpha", C.POINTER(C.c_double)), ("gamma", C.c_double), ("b", C.c_double)]


class TraceResult(C.Structure):
    _fields_ = [("d", C.c_int32), ("n_edges", C.c_int64),
                ("edge_y", C.POINTER(C.c_int32)), ("edge_mask", C.POINTER(C.c_uint32)),
                ("edge_level", C.POINTER(C.c_int32)), ("edge_f", C.POINTER(C.c_double)),
                ("edge_t", C.POINTER(C.c_double)), ("edge_pt", C.POINTER(C.c_double)),
                ("edge_multiroot", C.POINTER(C.c_uint8)),
                ("n_cells", C.c_int64), ("cell_y", C.POINTER(C.c_int32)),
                ("cell_perm", C.POINTER(C.c_uint8)), ("cell_off", C.POINTER(C.c_int64)),
                ("cell_idx", C.POINTER(C.c_int64)),
                ("n_vertices", C.c_int64), ("n_near_zero", C.c_int64), ("n_boundary", C.c_int64),
                ("n_dead_seeds", C.c_int64), ("levels", C.c_int64),
                ("n_crossing_triangles", C.c_int64)]


class Robot(C.Structure):
    _fields_ = [("n_links", C.c_int32), ("dh", C.POINTER(C.c_double)),
                ("radius", C.POINTER(C.c_double)), ("n_spheres", C.c_int32),
                ("sphere_link", C.POINTER(C.c_int32)), ("sphere_center", C.POINTER(C.c_double)),
                ("sphere_radius", C.POINTER(C.c_double))]


class Scene(C.Structure):
    _fields_ = [("n", C.c_int32), ("type", C.POINTER(C.c_int32)),
                ("pose", C.POINTER(C.c_double)), ("dims", C.POINTER(C.c_double))]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P = C.POINTER
        L.or_lattice_c.restype = C.c_double
        L.or_lattice_c.argtypes = [C.c_int]
        L.or_lattice_cinv.restype = C.c_double
        L.or_lattice_cinv.argtypes = [C.c_int]
        L.or_vertex_x.argtypes = [C.c_int, C.c_double, P(C.c_double), P(C.c_int32), P(C.c_double)]
        L.or_locate.argtypes = [C.c_int, C.c_double, P(C.c_double), P(C.c_double), P(Simplex)]
        L.or_simplex_vertices.argtypes = [C.c_int, P(Simplex), P(C.c_int32)]
        L.or_canonicalize.argtypes = [C.c_int, P(Simplex)]
        for name in ("or_triangle_edges", "or_nsimplex_edges", "or_edge_cofaces", "or_edge_ncofaces"):
            getattr(L, name).argtypes = [C.c_int, P(Simplex), P(Simplex)]
            getattr(L, name).restype = C.c_int
        L.or_f.restype = C.c_double
        L.or_f.argtypes = [P(Rbf), P(C.c_double)]
        L.or_f_batch.argtypes = [P(Rbf), P(C.c_double), C.c_int64, P(C.c_double)]
        L.or_trace.restype = C.c_int
        L.or_trace.argtypes = [P(Rbf), C.c_double, P(C.c_double), P(C.c_double), P(C.c_double),
                               P(C.c_double), C.c_int64, C.c_int, C.c_int, C.c_int64,
                               P(TraceResult)]
        L.or_trace_free.argtypes = [P(TraceResult)]
        L.or_edge_roots.argtypes = [P(Rbf), C.c_double, P(C.c_double), P(C.c_int32),
                                    P(C.c_uint32), C.c_int64, P(C.c_double), P(C.c_double),
                                    P(C.c_double), P(C.c_uint8)]
        L.or_fk.argtypes = [P(Robot), P(C.c_double), P(C.c_double)]
        L.or_segseg_dist.restype = C.c_double
        L.or_segseg_dist.argtypes = [P(C.c_double)] * 4
        L.or_segment_obstacle_dist.restype = C.c_double
        L.or_segment_obstacle_dist.argtypes = [P(C.c_double), P(C.c_double), C.c_int32,
                                               P(C.c_double), P(C.c_double)]
        L.or_certify.argtypes = [P(Robot), P(Scene), P(C.c_double), C.c_int64, C.c_int32,
                                 P(C.c_int64), P(C.c_int64), C.c_int64,
                                 P(C.c_uint8), P(C.c_double), P(C.c_uint8)]
        L.or_subdiv_template.restype = C.c_int
        L.or_subdiv_template.argtypes = [C.c_int, C.c_int, P(C.c_int32), P(C.c_int64),
                                         P(C.c_int32), P(C.c_int64)]
        L.or_subdiv.restype = C.c_int
        L.or_subdiv.argtypes = [P(Rbf), C.c_double, C.c_int, P(C.c_double), P(C.c_double),
                                P(C.c_double), P(C.c_double), C.c_int64, C.c_int,
                                P(TraceResult), P(C.c_int64)]
        L.or_fk_frames.argtypes = [P(Robot), P(C.c_double), P(C.c_double)]
        L.or_lipschitz.argtypes = [P(Robot), P(C.c_double)]
        L.or_certify_ex.argtypes = [P(Robot), P(Scene), P(C.c_double), C.c_int64, C.c_int32,
                                    P(C.c_int64), P(C.c_int64), C.c_int64, P(C.c_uint8),
                                    P(C.c_double), P(C.c_int32), P(C.c_uint8), P(C.c_uint8),
                                    P(C.c_double)]
        L.or_set_threads.restype = C.c_int
        L.or_set_threads.argtypes = [C.c_int]
        _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
# Simplices: (y, parts) with parts a tuple of bitmasks over {0..d}
# --------------------------------------------------------------------------
def _mk(d, y, parts):
    s = Simplex()
    for i in range(d):
        s.y[i] = int(y[i])
    s.k = len(parts) - 1
    for i, p in enumerate(parts):
        s.part[i] = int(p)
    return s


def _un(d, s):
    return tuple(int(s.y[i]) for i in range(d)), tuple(int(s.part[i]) for i in range(s.k + 1))


def parts_from_sets(sets):
    """Ordered partition given as a list of element lists -> tuple of masks."""
    return tuple(sum(1 << e for e in st) for st in sets)


def simplex_vertices(d, y, parts):
    s = _mk(d, y, parts)
    out = np.zeros((len(parts), d), dtype=np.int32)
    lib().or_simplex_vertices(d, C.byref(s), _p(out, C.c_int32))
    return out


def canonicalize(d, y, parts):
    s = _mk(d, y, parts)
    lib().or_canonicalize(d, C.byref(s))
    return _un(d, s)


def _query(name, d, y, parts, cap):
    s = _mk(d, y, parts)
    out = (Simplex * cap)()
    n = getattr(lib(), name)(d, C.byref(s), out)
    return [_un(d, out[i]) for i in range(n)]


def triangle_edges(d, y, parts):
    return _query("or_triangle_edges", d, y, parts, 3)


def nsimplex_edges(d, y, parts):
    return _query("or_nsimplex_edges", d, y, parts, (d + 1) * d // 2)


def edge_cofaces(d, y, parts):
    return _query("or_edge_cofaces", d, y, parts, 2 << d)


def edge_ncofaces(d, y, parts):
    import math
    return _query("or_edge_ncofaces", d, y, parts, math.factorial(d) * (d + 1))


def lattice_c(d):
    return lib().or_lattice_c(d)


def vertex_x(d, lam, o, y):
    y = np.ascontiguousarray(np.atleast_2d(y), dtype=np.int32)
    o = _f64(o)
    out = np.zeros((y.shape[0], d))
    for i in range(y.shape[0]):
        lib().or_vertex_x(d, lam, _p(o, C.c_double), _p(y[i], C.c_int32),
                          _p(out[i], C.c_double))
    return out


def locate(d, lam, o, x):
    s = Simplex()
    o = _f64(o)
    x = _f64(x)
    lib().or_locate(d, lam, _p(o, C.c_double), _p(x, C.c_double), C.byref(s))
    return _un(d, s)


# --------------------------------------------------------------------------
# RBF and tracing
# --------------------------------------------------------------------------
class _RbfHold:
    def __init__(self, sv, alpha, gamma, b):
        self.sv = _f64(sv)
        self.alpha = _f64(alpha)
        self.s = Rbf(self.sv.shape[1], self.sv.shape[0], _p(self.sv, C.c_double),
                     _p(self.alpha, C.c_double), float(gamma), float(b))


def f(sv, alpha, gamma, b, q):
    h = _RbfHold(sv, alpha, gamma, b)
    q = _f64(np.atleast_2d(q))
    out = np.zeros(q.shape[0])
    lib().or_f_batch(C.byref(h.s), _p(q, C.c_double), q.shape[0], _p(out, C.c_double))
    return out


def _arr(ptr, n, dtype):
    if n == 0:
        return np.zeros(0, dtype=dtype)
    return np.ctypeslib.as_array(ptr, shape=(n,)).astype(dtype, copy=True)


def trace(sv, alpha, gamma, b, lam, o, lo, hi, seeds, roots=True, cells=True, max_edges=0):
    """Trace from the seeds; returns a dict of numpy arrays and counters.
    max_edges > 0 stops the search once that many edges exist (bounded sample)."""
    h = _RbfHold(sv, alpha, gamma, b)
    d = h.sv.shape[1]
    o, lo, hi = _f64(o), _f64(lo), _f64(hi)
    seeds = _f64(np.atleast_2d(seeds)).reshape(-1, d)
    r = TraceResult()
    rc = lib().or_trace(C.byref(h.s), float(lam), _p(o, C.c_double), _p(lo, C.c_double),
                        _p(hi, C.c_double), _p(seeds, C.c_double), seeds.shape[0],
                        int(bool(roots)), int(bool(cells)), int(max_edges), C.byref(r))
    if rc != 0:
        raise RuntimeError("oracle trace failed")
    E, Cn = r.n_edges, r.n_cells
    out = dict(
        d=d,
        edge_y=_arr(r.edge_y, E * d, np.int32).reshape(E, d),
        edge_mask=_arr(r.edge_mask, E, np.uint32),
        edge_level=_arr(r.edge_level, E, np.int32),
        edge_f=_arr(r.edge_f, 2 * E, np.float64).reshape(E, 2),
        edge_t=_arr(r.edge_t, E, np.float64),
        edge_pt=_arr(r.edge_pt, E * d, np.float64).reshape(E, d),
        edge_multiroot=_arr(r.edge_multiroot, E, np.uint8),
        n_vertices=r.n_vertices, n_near_zero=r.n_near_zero, n_boundary=r.n_boundary,
        n_dead_seeds=r.n_dead_seeds, levels=r.levels,
        n_crossing_triangles=r.n_crossing_triangles,
    )
    if cells:
        off = _arr(r.cell_off, Cn + 1, np.int64)
        out.update(cell_y=_arr(r.cell_y, Cn * d, np.int32).reshape(Cn, d),
                   cell_perm=_arr(r.cell_perm, Cn * d, np.uint8).reshape(Cn, d),
                   cell_off=off, cell_idx=_arr(r.cell_idx, int(off[-1]) if Cn else 0, np.int64))
    lib().or_trace_free(C.byref(r))
    return out


def subdiv_template(d, k):
    """The local triangulation of the subdivided reference n-simplex
    (Sec. V-B): vertices [nv][d] (local coordinates v') and edges [ne] as
    (vertex index, local mask M')."""
    nv, ne = C.c_int64(), C.c_int64()
    lib().or_subdiv_template(d, k, None, C.byref(nv), None, C.byref(ne))
    v = np.zeros((max(nv.value, 1), d), np.int32)
    e = np.zeros((max(ne.value, 1), 2), np.int32)
    lib().or_subdiv_template(d, k, _p(v, C.c_int32), C.byref(nv), _p(e, C.c_int32), C.byref(ne))
    return v[:nv.value], e[:ne.value]


def subdiv(sv, alpha, gamma, b, lam, k, o, lo, hi, seeds, roots=True):
    """Batch triangulation (Sec. V-B): the crossing edges of the scale-lam
    local triangulations of the crossing n-simplices of the coarse trace at
    scale k * lam.  Returns the trace dict (no cells) and 'n_coarse_cells'."""
    h = _RbfHold(sv, alpha, gamma, b)
    d = h.sv.shape[1]
    o, lo, hi = _f64(o), _f64(lo), _f64(hi)
    seeds = _f64(np.atleast_2d(seeds)).reshape(-1, d)
    res = TraceResult()
    nco = C.c_int64()
    rc = lib().or_subdiv(C.byref(h.s), float(lam), int(k), _p(o, C.c_double), _p(lo, C.c_double),
                         _p(hi, C.c_double), _p(seeds, C.c_double), seeds.shape[0], int(roots),
                         C.byref(res), C.byref(nco))
    if rc:
        raise RuntimeError("or_subdiv failed")
    E = res.n_edges
    out = dict(
        d=d,
        edge_y=_arr(res.edge_y, E * d, np.int32).reshape(E, d),
        edge_mask=_arr(res.edge_mask, E, np.uint32),
        edge_f=_arr(res.edge_f, 2 * E, np.float64).reshape(E, 2),
        edge_t=_arr(res.edge_t, E, np.float64),
        edge_pt=_arr(res.edge_pt, E * d, np.float64).reshape(E, d),
        edge_multiroot=_arr(res.edge_multiroot, E, np.uint8),
        n_vertices=res.n_vertices, n_near_zero=res.n_near_zero, n_dead_seeds=res.n_dead_seeds,
        levels=res.levels, n_coarse_cells=int(nco.value))
    lib().or_trace_free(C.byref(res))
    return out


def edge_roots(sv, alpha, gamma, b, lam, o, edge_y, edge_mask):
    """f at both vertices, bisection root, point and multi-root flag of given edges."""
    h = _RbfHold(sv, alpha, gamma, b)
    d = h.sv.shape[1]
    ey = np.ascontiguousarray(edge_y, dtype=np.int32).reshape(-1, d)
    em = np.ascontiguousarray(edge_mask, dtype=np.uint32)
    n = ey.shape[0]
    o = _f64(o)
    f2 = np.zeros((n, 2))
    t = np.zeros(n)
    pt = np.zeros((n, d))
    mr = np.zeros(n, dtype=np.uint8)
    if n:
        lib().or_edge_roots(C.byref(h.s), float(lam), _p(o, C.c_double), _p(ey, C.c_int32),
                            _p(em, C.c_uint32), n, _p(f2, C.c_double), _p(t, C.c_double),
                            _p(pt, C.c_double), _p(mr, C.c_uint8))
    return f2, t, pt, mr


# --------------------------------------------------------------------------
# Certification
# --------------------------------------------------------------------------
class _RobotHold:
    """radius None: no link capsules; spheres = (link [n], centre [n][3] in
    frame T_{link+1}, radius [n]) or None."""

    def __init__(self, dh, radius, spheres=None):
        self.dh = _f64(dh).reshape(-1, 4)
        self.radius = None if radius is None else _f64(radius)
        rad = _p(self.radius, C.c_double) if self.radius is not None else None
        if spheres is None:
            self.sl = np.zeros(1, np.int32)
            self.sc = np.zeros(3)
            self.sr = np.zeros(1)
            ns = 0
        else:
            self.sl = np.ascontiguousarray(spheres[0], dtype=np.int32)
            self.sc = _f64(spheres[1]).reshape(-1, 3)
            self.sr = _f64(spheres[2])
            ns = self.sl.shape[0]
        self.s = Robot(self.dh.shape[0], _p(self.dh, C.c_double), rad, ns,
                       _p(self.sl, C.c_int32), _p(self.sc, C.c_double), _p(self.sr, C.c_double))


class _SceneHold:
    def __init__(self, types, pose, dims):
        self.type = np.ascontiguousarray(types, dtype=np.int32)
        self.pose = _f64(pose).reshape(-1, 12)
        self.dims = _f64(dims).reshape(-1, 3)
        self.s = Scene(self.type.shape[0], _p(self.type, C.c_int32), _p(self.pose, C.c_double),
                       _p(self.dims, C.c_double))


def fk(dh, radius, q):
    r = _RobotHold(dh, radius)
    q = _f64(q)
    out = np.zeros((r.dh.shape[0] + 1, 3))
    lib().or_fk(C.byref(r.s), _p(q, C.c_double), _p(out, C.c_double))
    return out


def segment_obstacle_dist(a, b, typ, pose, dims):
    a, b, pose, dims = _f64(a), _f64(b), _f64(pose), _f64(dims)
    return lib().or_segment_obstacle_dist(_p(a, C.c_double), _p(b, C.c_double), int(typ),
                                          _p(pose, C.c_double), _p(dims, C.c_double))


def segseg_dist(p1, q1, p2, q2):
    args = [_f64(v) for v in (p1, q1, p2, q2)]
    return lib().or_segseg_dist(*[_p(v, C.c_double) for v in args])


def fk_frames(dh, q):
    """Frames T_0 .. T_n of the chain, each 3x4 [R | t]."""
    r = _RobotHold(dh, np.zeros(len(np.atleast_1d(q))))
    q = _f64(q)
    out = np.zeros((r.dh.shape[0] + 1, 12))
    lib().or_fk_frames(C.byref(r.s), _p(q, C.c_double), _p(out, C.c_double))
    return out.reshape(-1, 3, 4)


def lipschitz(dh, radius, spheres=None):
    """Per robot element (capsules, then spheres) and joint: the bound on how
    far a point of the element moves per radian of that joint."""
    r = _RobotHold(dh, radius, spheres)
    ne = (r.dh.shape[0] if radius is not None else 0) + int(r.s.n_spheres)
    L = np.zeros((max(ne, 1), r.dh.shape[0]))
    lib().or_lipschitz(C.byref(r.s), _p(L, C.c_double))
    return L[:ne]


def certify_ex(dh, radius, types, pose, dims, points, cell_off=None, cell_idx=None,
               spheres=None):
    """Per point: verdict, margin, deciding element; per cell: the AND of its
    points' verdicts, the whole-cell (Lipschitz) verdict and its slack."""
    r = _RobotHold(dh, radius, spheres)
    s = _SceneHold(types, pose, dims)
    d = r.dh.shape[0]
    pts = _f64(points).reshape(-1, d)
    P = pts.shape[0]
    if cell_off is None:
        cell_off = np.zeros(1, dtype=np.int64)
        cell_idx = np.zeros(1, dtype=np.int64)
    cell_off = np.ascontiguousarray(cell_off, dtype=np.int64)
    cell_idx = np.ascontiguousarray(cell_idx if len(cell_idx) else np.zeros(1), dtype=np.int64)
    nc = cell_off.shape[0] - 1
    verdict = np.zeros(max(P, 1), dtype=np.uint8)
    margin = np.zeros(max(P, 1))
    elem = np.zeros(max(P, 1), dtype=np.int32)
    cv = np.zeros(max(nc, 1), dtype=np.uint8)
    whole = np.zeros(max(nc, 1), dtype=np.uint8)
    slack = np.zeros(max(nc, 1))
    lib().or_certify_ex(C.byref(r.s), C.byref(s.s), _p(pts, C.c_double), P, d,
                        _p(cell_off, C.c_int64), _p(cell_idx, C.c_int64), nc,
                        _p(verdict, C.c_uint8), _p(margin, C.c_double), _p(elem, C.c_int32),
                        _p(cv, C.c_uint8), _p(whole, C.c_uint8), _p(slack, C.c_double))
    return dict(verdict=verdict[:P], margin=margin[:P], element=elem[:P], cell_verdict=cv[:nc],
                cell_whole=whole[:nc], cell_slack=slack[:nc])


def certify(dh, radius, types, pose, dims, points, cell_off=None, cell_idx=None):
    r = _RobotHold(dh, radius)
    s = _SceneHold(types, pose, dims)
    d = r.dh.shape[0]
    pts = _f64(points).reshape(-1, d)
    P = pts.shape[0]
    if cell_off is None:
        cell_off = np.zeros(1, dtype=np.int64)
        cell_idx = np.zeros(1, dtype=np.int64)
    cell_off = np.ascontiguousarray(cell_off, dtype=np.int64)
    cell_idx = np.ascontiguousarray(cell_idx if len(cell_idx) else np.zeros(1), dtype=np.int64)
    nc = cell_off.shape[0] - 1
    verdict = np.zeros(max(P, 1), dtype=np.uint8)
    margin = np.zeros(max(P, 1))
    cv = np.zeros(max(nc, 1), dtype=np.uint8)
    lib().or_certify(C.byref(r.s), C.byref(s.s), _p(pts, C.c_double), P, d,
                     _p(cell_off, C.c_int64), _p(cell_idx, C.c_int64), nc,
                     _p(verdict, C.c_uint8), _p(margin, C.c_double), _p(cv, C.c_uint8))
    return verdict[:P], margin[:P], cv[:nc]
