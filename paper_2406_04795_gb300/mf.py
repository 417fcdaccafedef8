"""ctypes binding of libmf.so (include/mf.h), same names as the C ABI.

Argument marshalling only: every step of the traced path runs in the CUDA
library.  Loading fails loudly when the library is missing; there is no CPU
fallback.  Device buffers are passed as raw pointers (e.g. torch CUDA tensors'
``data_ptr()``); streams as ``torch.cuda.Stream.cuda_stream`` integers.
"""
from __future__ import annotations

import ctypes as C
import os

MF_MAXD = 8
MF_OK = 0
MF_ERR_INVALID = -1
MF_ERR_DOMAIN = -2
MF_ERR_OOM = -3
MF_ERR_CAPACITY = -4
MF_ERR_MAXEDGES = -5
MF_ERR_TIMEOUT = -6
MF_ERR_CUDA = -7
MF_ERR_DEVICE = -8

MF_FP64 = 0
MF_MIXED_BF16 = 1
MF_MIXED_FP32 = 2

MF_WANT_ROOTS = 1
MF_WANT_CELLS = 2
MF_ROOTS_FP64_EXACT = 4
MF_SORT_OUTPUT = 8

MF_BOX = 0
MF_SPHERE = 1
MF_CYLINDER = 2
MF_MAX_SPHERES = 64

EXPORTS = ("mf_ctx_create", "mf_ctx_destroy", "mf_last_error", "mf_ctx_bytes", "mf_locate",
           "mf_eval", "mf_trace", "mf_trace_fetch", "mf_certify", "mf_ctx_set_profiling",
           "mf_ctx_get_stats", "mf_trace_noalloc", "mf_trace_batch", "mf_domain_table",
           "mf_server_create", "mf_server_destroy", "mf_server_submit", "mf_server_step",
           "mf_server_status", "mf_server_fetch", "mf_server_done", "mf_autotune", "mf_ctx_set_tune",
           "mf_ctx_get_tune", "mf_vertex_keys", "mf_probe_rates", "mf_diag_exp",
           "mf_certify_ex", "mf_subdiv_begin", "mf_subdiv_next",
           "mf_server_wait")

MF_PHASES = 12
PHASE_NAMES = ("prepare", "seeds", "expand_vertices", "eval", "expand_edges", "roots", "cells",
               "csr", "copy", "certify_points", "certify_cells", "other")

_ERRNAMES = {v: k for k, v in globals().items() if k.startswith("MF_ERR_") or k == "MF_OK"}


class mf_rbf(C.Structure):
    _fields_ = [("d", C.c_int32), ("n_sv", C.c_int64), ("sv", C.c_void_p), ("alpha", C.c_void_p),
                ("gamma", C.c_double), ("b", C.c_double)]


class mf_domain(C.Structure):
    _fields_ = [("lo", C.c_double * MF_MAXD), ("hi", C.c_double * MF_MAXD),
                ("offset", C.c_double * MF_MAXD)]


class mf_trace_opts(C.Structure):
    _fields_ = [("lambda_", C.c_double), ("batch_cap_edges", C.c_int64), ("precision", C.c_int32),
                ("recheck_band", C.c_double), ("root_tol", C.c_double), ("max_edges", C.c_int64),
                ("max_vertices", C.c_int64), ("max_cells", C.c_int64), ("flags", C.c_uint32)]


class mf_trace_out(C.Structure):
    _fields_ = [("cap_edges", C.c_int64), ("edge_y", C.c_void_p), ("edge_mask", C.c_void_p),
                ("edge_f", C.c_void_p), ("edge_t", C.c_void_p), ("points", C.c_void_p),
                ("cap_cells", C.c_int64), ("cell_y", C.c_void_p), ("cell_perm", C.c_void_p),
                ("cell_edge_off", C.c_void_p), ("cap_cell_edges", C.c_int64),
                ("cell_edge_idx", C.c_void_p),
                ("n_edges", C.c_int64), ("n_cells", C.c_int64), ("n_cell_edges", C.c_int64),
                ("n_vertices", C.c_int64), ("n_near_zero", C.c_int64), ("n_recheck", C.c_int64),
                ("n_boundary", C.c_int64), ("n_dead_seeds", C.c_int64), ("levels", C.c_int64),
                ("root_evals", C.c_int64)]


class mf_robot(C.Structure):
    _fields_ = [("n_links", C.c_int32), ("dh", C.c_void_p), ("radius", C.c_void_p),
                ("n_spheres", C.c_int32), ("sphere_link", C.c_void_p),
                ("sphere_center", C.c_void_p), ("sphere_radius", C.c_void_p)]


class mf_certify_out(C.Structure):
    _fields_ = [("point_verdict", C.c_void_p), ("margin", C.c_void_p), ("element", C.c_void_p),
                ("cell_verdict", C.c_void_p), ("cell_whole", C.c_void_p),
                ("cell_slack", C.c_void_p)]


class mf_scene(C.Structure):
    _fields_ = [("n", C.c_int32), ("type", C.c_void_p), ("pose", C.c_void_p), ("dims", C.c_void_p)]


class mf_stats(C.Structure):
    _fields_ = [("ms", C.c_double * MF_PHASES), ("launches", C.c_int64 * MF_PHASES),
                ("units", C.c_int64 * MF_PHASES), ("terms", C.c_int64 * MF_PHASES),
                ("terms_weak", C.c_int64 * MF_PHASES)]


class mf_rates(C.Structure):
    _fields_ = [("fp64_fma_per_s", C.c_double), ("fp32_fma_per_s", C.c_double),
                ("ex2_per_s", C.c_double), ("exp_neg_per_s", C.c_double),
                ("sm_count", C.c_int32), ("sm_clock_mhz", C.c_double)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class mf_tune(C.Structure):
    _fields_ = [("roots_variant", C.c_int32), ("roots_blocks_per_sm", C.c_int32),
                ("eval_blocks_per_sm", C.c_int32), ("tc_chunk", C.c_int32),
                ("frontier_chunk", C.c_int64), ("ms_bfs", C.c_double), ("ms_roots", C.c_double),
                ("ms_eval", C.c_double), ("n_candidates", C.c_int32), ("roots_group", C.c_int32)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


_lib = None


def lib_path() -> str:
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "libmf.so")


def load(build_if_missing: bool = True):
    """Loads libmf.so (building it in-tree if absent).  Raises if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if build_if_missing:
        from . import build as _build
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError("libmf.so is missing: build it with paper_2406_04795_gb300.build")
    L = C.CDLL(path)
    P, V = C.POINTER, C.c_void_p
    L.mf_ctx_create.restype = C.c_int
    L.mf_ctx_create.argtypes = [C.c_int, C.c_size_t, P(V)]
    L.mf_ctx_destroy.restype = None
    L.mf_ctx_destroy.argtypes = [V]
    L.mf_last_error.restype = C.c_char_p
    L.mf_last_error.argtypes = [V]
    L.mf_ctx_bytes.restype = C.c_size_t
    L.mf_ctx_bytes.argtypes = [V]
    L.mf_locate.restype = C.c_int
    L.mf_locate.argtypes = [V, C.c_int32, C.c_double, P(C.c_double), V, C.c_int64, V, V, V]
    L.mf_eval.restype = C.c_int
    L.mf_eval.argtypes = [V, P(mf_rbf), V, C.c_int64, C.c_int32, C.c_double, V, V]
    L.mf_trace.restype = C.c_int
    L.mf_trace.argtypes = [V, P(mf_rbf), P(mf_domain), P(mf_trace_opts), V, C.c_int64,
                           P(mf_trace_out), V]
    L.mf_trace_fetch.restype = C.c_int
    L.mf_trace_fetch.argtypes = [V, P(mf_trace_out), V]
    L.mf_certify.restype = C.c_int
    L.mf_certify.argtypes = [V, P(mf_robot), P(mf_scene), V, C.c_int64, C.c_int32, V, V,
                             C.c_int64, V, V, V, V]
    L.mf_ctx_set_profiling.restype = C.c_int
    L.mf_ctx_set_profiling.argtypes = [V, C.c_int]
    L.mf_ctx_get_stats.restype = C.c_int
    L.mf_ctx_get_stats.argtypes = [V, P(mf_stats)]
    L.mf_autotune.restype = C.c_int
    L.mf_autotune.argtypes = [V, P(mf_rbf), P(mf_domain), P(mf_trace_opts), V, C.c_int64,
                              P(mf_tune), V]
    L.mf_ctx_set_tune.restype = C.c_int
    L.mf_ctx_set_tune.argtypes = [V, P(mf_tune)]
    L.mf_ctx_get_tune.restype = C.c_int
    L.mf_ctx_get_tune.argtypes = [V, P(mf_tune)]
    L.mf_server_create.restype = C.c_int
    L.mf_server_create.argtypes = [V, C.c_int32, C.c_size_t, P(V)]
    L.mf_server_destroy.restype = None
    L.mf_server_destroy.argtypes = [V]
    L.mf_server_submit.restype = C.c_int
    L.mf_server_submit.argtypes = [V, P(mf_rbf), P(mf_domain), P(mf_trace_opts), V, C.c_int64,
                                   P(C.c_int64)]
    L.mf_server_step.restype = C.c_int
    L.mf_server_step.argtypes = [V, V, P(C.c_int32), P(C.c_int32)]
    L.mf_server_status.restype = C.c_int
    L.mf_server_status.argtypes = [V, C.c_int64, P(C.c_int32), P(C.c_double), P(C.c_double),
                                   P(C.c_double)]
    L.mf_server_done.restype = C.c_int
    L.mf_server_done.argtypes = [V, P(C.c_int64), C.c_int32, P(C.c_int32)]
    L.mf_server_fetch.restype = C.c_int
    L.mf_server_fetch.argtypes = [V, C.c_int64, P(mf_trace_out), V]
    L.mf_domain_table.restype = C.c_int
    L.mf_domain_table.argtypes = [C.c_int32, C.c_double, P(mf_domain), P(C.c_int32), P(C.c_int32),
                                  V, C.c_int64]
    L.mf_vertex_keys.restype = C.c_int
    L.mf_vertex_keys.argtypes = [C.c_int32, C.c_double, P(mf_domain), V, C.c_int64, V, V]
    L.mf_trace_batch.restype = C.c_int
    L.mf_trace_batch.argtypes = [V, C.c_int32, P(mf_rbf), P(mf_domain), P(mf_trace_opts),
                                 P(C.c_void_p), P(C.c_int64), P(mf_trace_out), V]
    L.mf_trace_noalloc.restype = C.c_int
    L.mf_trace_noalloc.argtypes = [P(mf_rbf), P(mf_domain), P(mf_trace_opts), V, C.c_int64,
                                   P(mf_trace_out), V]
    L.mf_server_wait.restype = C.c_int
    L.mf_server_wait.argtypes = [V, C.c_int64, C.c_double, V, P(C.c_int32)]
    L.mf_subdiv_begin.restype = C.c_int
    L.mf_subdiv_begin.argtypes = [V, P(mf_rbf), P(mf_domain), P(mf_trace_opts), C.c_int32, V,
                                  C.c_int64, C.c_int64, P(C.c_int64), V]
    L.mf_subdiv_next.restype = C.c_int
    L.mf_subdiv_next.argtypes = [V, P(mf_trace_out), P(C.c_int64), V]
    L.mf_certify_ex.restype = C.c_int
    L.mf_certify_ex.argtypes = [V, P(mf_robot), P(mf_scene), V, C.c_int64, C.c_int32, V, V,
                                C.c_int64, P(mf_certify_out), V]
    L.mf_probe_rates.restype = C.c_int
    L.mf_probe_rates.argtypes = [V, P(mf_rates), V]
    L.mf_diag_exp.restype = C.c_int
    L.mf_diag_exp.argtypes = [V, V, C.c_int64, V, V, V]
    _lib = L
    return L


class MfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (_ERRNAMES.get(code, "MF_ERR"), code, msg))
        self.code = code


def _check(ctx, rc):
    if rc != MF_OK:
        msg = load().mf_last_error(ctx).decode() if ctx else ""
        raise MfError(rc, msg)
    return rc


# ---------------------------------------------------------------------------
# Same-name wrappers (raw pointers in, return code checked)
# ---------------------------------------------------------------------------
def mf_ctx_create(device: int = 0, hbm_budget_bytes: int = 0):
    h = C.c_void_p()
    rc = load().mf_ctx_create(device, hbm_budget_bytes, C.byref(h))
    if rc != MF_OK:
        raise MfError(rc, "mf_ctx_create failed")
    return h


def mf_ctx_destroy(ctx):
    load().mf_ctx_destroy(ctx)


def mf_last_error(ctx) -> str:
    return load().mf_last_error(ctx).decode()


def mf_ctx_bytes(ctx) -> int:
    return load().mf_ctx_bytes(ctx)


def mf_locate(ctx, d, lam, offset, points_ptr, n, y_ptr, perm_ptr, stream=0):
    off = (C.c_double * MF_MAXD)(*[float(v) for v in offset])
    return _check(ctx, load().mf_locate(ctx, d, lam, off, points_ptr, n, y_ptr, perm_ptr, stream))


def mf_eval(ctx, rbf: mf_rbf, q_ptr, n, precision, band, f_ptr, stream=0):
    return _check(ctx, load().mf_eval(ctx, C.byref(rbf), q_ptr, n, precision, band, f_ptr, stream))


def mf_trace(ctx, rbf: mf_rbf, dom: mf_domain, opts: mf_trace_opts, seeds_ptr, n_seeds,
             out: mf_trace_out, stream=0, check=True):
    rc = load().mf_trace(ctx, C.byref(rbf), C.byref(dom), C.byref(opts), seeds_ptr, n_seeds,
                         C.byref(out), stream)
    return _check(ctx, rc) if check else rc


def mf_trace_fetch(ctx, out: mf_trace_out, stream=0):
    return _check(ctx, load().mf_trace_fetch(ctx, C.byref(out), stream))


def mf_server_create(ctx, max_slots, hbm_bytes):
    h = C.c_void_p()
    _check(ctx, load().mf_server_create(ctx, max_slots, hbm_bytes, C.byref(h)))
    return h


def mf_server_destroy(server):
    load().mf_server_destroy(server)


def mf_server_submit(ctx, server, rbf, dom, opts, seeds_ptr, n_seeds):
    rid = C.c_int64()
    _check(ctx, load().mf_server_submit(server, C.byref(rbf), C.byref(dom), C.byref(opts),
                                        seeds_ptr, n_seeds, C.byref(rid)))
    return rid.value


def mf_server_step(ctx, server, stream=0):
    nr, nq = C.c_int32(), C.c_int32()
    _check(ctx, load().mf_server_step(server, stream, C.byref(nr), C.byref(nq)))
    return nr.value, nq.value


def mf_server_status(ctx, server, rid):
    st = C.c_int32()
    t = [C.c_double(), C.c_double(), C.c_double()]
    _check(ctx, load().mf_server_status(server, rid, C.byref(st), *[C.byref(x) for x in t]))
    return st.value, t[0].value, t[1].value, t[2].value


def mf_server_done(ctx, server, cap=4096):
    ids = (C.c_int64 * cap)()
    n = C.c_int32()
    _check(ctx, load().mf_server_done(server, ids, cap, C.byref(n)))
    return [ids[i] for i in range(n.value)]


def mf_server_fetch(ctx, server, rid, out: mf_trace_out, stream=0, check=True):
    rc = load().mf_server_fetch(server, rid, C.byref(out), stream)
    return _check(ctx, rc) if check else rc


def mf_domain_table(d, lam, dom: mf_domain):
    """(smin, table[span][d][2]) of the exact lattice domain test (host only)."""
    import numpy as np
    smin, span = C.c_int32(), C.c_int32()
    rc = load().mf_domain_table(d, lam, C.byref(dom), C.byref(smin), C.byref(span), None, 0)
    if rc != MF_OK:
        raise MfError(rc, "mf_domain_table")
    tab = np.zeros((span.value, d, 2), dtype=np.int32)
    rc = load().mf_domain_table(d, lam, C.byref(dom), C.byref(smin), C.byref(span),
                                tab.ctypes.data_as(C.c_void_p), tab.size)
    if rc != MF_OK:
        raise MfError(rc, "mf_domain_table")
    return smin.value, tab


def mf_vertex_keys(d, lam, dom: mf_domain, y):
    """(keys uint64[n], in_range bool[n]) of lattice vertices y [n][d] under
    the tracing tables' key packing (host only)."""
    import numpy as np
    y = np.ascontiguousarray(y, dtype=np.int32).reshape(-1, d)
    keys = np.zeros(y.shape[0], dtype=np.uint64)
    ok = np.zeros(y.shape[0], dtype=np.uint8)
    rc = load().mf_vertex_keys(d, lam, C.byref(dom), y.ctypes.data_as(C.c_void_p), y.shape[0],
                               keys.ctypes.data_as(C.c_void_p), ok.ctypes.data_as(C.c_void_p))
    if rc != MF_OK:
        raise MfError(rc, "mf_vertex_keys")
    return keys, ok.astype(bool)


def mf_trace_batch(ctx, rbfs, doms, opts, seed_ptrs, n_seeds, outs, stream=0, check=True):
    """rbfs / doms / opts / outs: ctypes arrays of the structs; seed_ptrs: a
    ctypes array of device pointers; n_seeds: a ctypes int64 array."""
    rc = load().mf_trace_batch(ctx, len(rbfs), rbfs, doms, opts, seed_ptrs, n_seeds, outs, stream)
    return _check(ctx, rc) if check else rc


def mf_trace_noalloc(rbf: mf_rbf, dom: mf_domain, opts: mf_trace_opts, seeds_ptr, n_seeds,
                     out: mf_trace_out, stream=0) -> int:
    """The allocation-free trace (for callers that cannot allocate device
    memory); returns the MF_* code (there is no context to hold a message)."""
    return load().mf_trace_noalloc(C.byref(rbf), C.byref(dom), C.byref(opts), seeds_ptr, n_seeds,
                                   C.byref(out), stream)


def mf_ctx_set_profiling(ctx, enable: bool):
    return _check(ctx, load().mf_ctx_set_profiling(ctx, 1 if enable else 0))


def mf_ctx_get_stats(ctx) -> dict:
    s = mf_stats()
    _check(ctx, load().mf_ctx_get_stats(ctx, C.byref(s)))
    return {name: dict(ms=s.ms[i], launches=s.launches[i], units=s.units[i], terms=s.terms[i],
                       terms_weak=s.terms_weak[i])
            for i, name in enumerate(PHASE_NAMES)}


def mf_autotune(ctx, rbf: mf_rbf, dom: mf_domain, opts: mf_trace_opts, seeds_ptr, n_seeds,
                stream=0) -> mf_tune:
    t = mf_tune()
    _check(ctx, load().mf_autotune(ctx, C.byref(rbf), C.byref(dom), C.byref(opts), seeds_ptr,
                                   n_seeds, C.byref(t), stream))
    return t


def mf_server_wait(ctx, server, rid, timeout_ms, stream=0, check=True):
    """Returns (rc, state); raises on errors other than MF_ERR_TIMEOUT unless check=False."""
    st = C.c_int32()
    rc = load().mf_server_wait(server, rid, float(timeout_ms), stream, C.byref(st))
    if check and rc not in (MF_OK, MF_ERR_TIMEOUT):
        _check(ctx, rc)
    return rc, st.value


def mf_subdiv_begin(ctx, rbf: mf_rbf, dom: mf_domain, opts: mf_trace_opts, k, seeds_ptr, n_seeds,
                    cells_per_batch, stream=0) -> int:
    n = C.c_int64()
    _check(ctx, load().mf_subdiv_begin(ctx, C.byref(rbf), C.byref(dom), C.byref(opts), k,
                                       seeds_ptr, n_seeds, cells_per_batch, C.byref(n), stream))
    return n.value


def mf_subdiv_next(ctx, out: mf_trace_out, stream=0) -> int:
    left = C.c_int64()
    _check(ctx, load().mf_subdiv_next(ctx, C.byref(out), C.byref(left), stream))
    return left.value


def mf_certify_ex(ctx, robot: mf_robot, scene: mf_scene, points_ptr, n_points, d, off_ptr,
                  idx_ptr, n_cells, out: mf_certify_out, stream=0):
    return _check(ctx, load().mf_certify_ex(ctx, C.byref(robot), C.byref(scene), points_ptr,
                                            n_points, d, off_ptr, idx_ptr, n_cells, C.byref(out),
                                            stream))


def mf_probe_rates(ctx, stream=0) -> mf_rates:
    r = mf_rates()
    _check(ctx, load().mf_probe_rates(ctx, C.byref(r), stream))
    return r


def mf_diag_exp(ctx, x_ptr, n, y_table_ptr, y_lib_ptr, stream=0):
    return _check(ctx, load().mf_diag_exp(ctx, x_ptr, n, y_table_ptr, y_lib_ptr, stream))


def mf_ctx_set_tune(ctx, t):
    return _check(ctx, load().mf_ctx_set_tune(ctx, C.byref(t) if t is not None else None))


def mf_ctx_get_tune(ctx) -> mf_tune:
    t = mf_tune()
    _check(ctx, load().mf_ctx_get_tune(ctx, C.byref(t)))
    return t


def mf_certify(ctx, robot: mf_robot, scene: mf_scene, points_ptr, n_points, d, off_ptr, idx_ptr,
               n_cells, verdict_ptr, margin_ptr, cell_verdict_ptr, stream=0):
    return _check(ctx, load().mf_certify(ctx, C.byref(robot), C.byref(scene), points_ptr, n_points,
                                         d, off_ptr, idx_ptr, n_cells, verdict_ptr, margin_ptr,
                                         cell_verdict_ptr, stream))
