"""Torch-facing convenience layer over the C ABI (argument marshalling only).

``Context`` owns one library context (its resident hash tables and lists) and
turns numpy / torch inputs into device buffers for ``mf_trace``, ``mf_certify``,
``mf_eval`` and ``mf_locate``.  Every computation runs in libmf.so.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import mf


def _dev(x, dtype, device):
    if isinstance(x, torch.Tensor):
        return x.to(device=device, dtype=dtype).contiguous()
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device=device)


def _stream_handle(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


class Context:
    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        if not torch.cuda.is_available():
            raise RuntimeError("the GB300 library needs a CUDA device; there is no CPU path")
        self.device = torch.device("cuda", device)
        torch.cuda.set_device(self.device)
        self.h = mf.mf_ctx_create(device, hbm_budget_bytes)

    def close(self):
        if self.h:
            mf.mf_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------
    def rbf(self, sv, alpha, gamma, b):
        sv_t = _dev(sv, torch.float64, self.device)
        al_t = _dev(alpha, torch.float64, self.device)
        r = mf.mf_rbf(sv_t.shape[1], sv_t.shape[0], sv_t.data_ptr(), al_t.data_ptr(), float(gamma),
                      float(b))
        return r, (sv_t, al_t)

    @staticmethod
    def domain(lo, hi, offset):
        dom = mf.mf_domain()
        for i, v in enumerate(lo):
            dom.lo[i] = float(v)
        for i, v in enumerate(hi):
            dom.hi[i] = float(v)
        for i, v in enumerate(offset):
            dom.offset[i] = float(v)
        return dom

    def locate(self, d, lam, offset, points, stream=None):
        pts = _dev(points, torch.float64, self.device).reshape(-1, d)
        n = pts.shape[0]
        y = torch.empty((n, d), dtype=torch.int32, device=self.device)
        perm = torch.empty((n, d), dtype=torch.uint8, device=self.device)
        mf.mf_locate(self.h, d, float(lam), list(offset), pts.data_ptr(), n, y.data_ptr(),
                     perm.data_ptr(), _stream_handle(stream))
        return y, perm

    def eval(self, sv, alpha, gamma, b, points, precision=mf.MF_FP64, band=1e-3, stream=None):
        r, keep = self.rbf(sv, alpha, gamma, b)
        pts = _dev(points, torch.float64, self.device).reshape(-1, r.d)
        out = torch.empty(pts.shape[0], dtype=torch.float64, device=self.device)
        mf.mf_eval(self.h, r, pts.data_ptr(), pts.shape[0], precision, band, out.data_ptr(),
                   _stream_handle(stream))
        return out

    def trace(self, sv, alpha, gamma, b, lam, offset, lo, hi, seeds, precision=mf.MF_FP64,
              roots=True, cells=True, batch_cap=1 << 24, max_edges=1 << 22, max_vertices=0,
              max_cells=0, recheck_band=1e-3, root_tol=1e-12, stream=None, outputs=None,
              exact_roots=False, sort=False):
        """Traces the zero set; returns a dict of device tensors and counters.

        ``outputs`` may hold preallocated output tensors (as returned by an
        earlier call) to avoid allocations in timed loops.  ``exact_roots``
        gives a mixed precision the FP64 path's root accuracy
        (MF_ROOTS_FP64_EXACT)."""
        r, keep = self.rbf(sv, alpha, gamma, b)
        d = r.d
        dom = self.domain(lo, hi, offset)
        seeds_t = _dev(seeds, torch.float64, self.device).reshape(-1, d)
        opts = mf.mf_trace_opts(float(lam), int(batch_cap), int(precision), float(recheck_band),
                                float(root_tol), int(max_edges), int(max_vertices), int(max_cells),
                                (mf.MF_WANT_ROOTS if roots else 0) | (mf.MF_WANT_CELLS if cells else 0)
                                | (mf.MF_ROOTS_FP64_EXACT if exact_roots else 0)
                                | (mf.MF_SORT_OUTPUT if sort else 0))
        st = _stream_handle(stream)
        res = outputs if outputs is not None else {}
        out = self._out_struct(res, d)
        rc = mf.mf_trace(self.h, r, dom, opts, seeds_t.data_ptr(), seeds_t.shape[0], out, st,
                         check=False)
        if rc == mf.MF_ERR_CAPACITY or (rc == mf.MF_OK and not res):
            res = self._alloc_outputs(d, out.n_edges, out.n_cells, out.n_cell_edges)
            out = self._out_struct(res, d)
            mf.mf_trace_fetch(self.h, out, st)
        elif rc != mf.MF_OK:
            mf._check(self.h, rc)
        E, Cn, CE = out.n_edges, out.n_cells, out.n_cell_edges
        result = dict(
            edge_y=res["edge_y"][:E], edge_mask=res["edge_mask"][:E], edge_f=res["edge_f"][:E],
            edge_t=res["edge_t"][:E], points=res["points"][:E],
            cell_y=res["cell_y"][:Cn], cell_perm=res["cell_perm"][:Cn],
            cell_off=res["cell_off"][:Cn + 1], cell_idx=res["cell_idx"][:CE],
            n_edges=E, n_cells=Cn, n_cell_edges=CE, n_vertices=out.n_vertices,
            n_near_zero=out.n_near_zero, n_recheck=out.n_recheck, n_boundary=out.n_boundary,
            n_dead_seeds=out.n_dead_seeds, levels=out.levels, root_evals=out.root_evals,
            _buffers=res)
        return result

    def subdiv(self, w, k, precision=mf.MF_FP64, cells_per_batch=0, max_edges=1 << 22,
               max_vertices=0, max_cells=0, roots=True, exact_roots=False, recheck_band=1e-3,
               root_tol=1e-12, stream=None, each_batch=None):
        """Batch triangulation (mf_subdiv_begin / next) of workload w at its
        lambda with coarse factor k.  max_* size the coarse trace and each
        batch's fine tables.  Returns the batches' edges concatenated (an
        edge on a face shared by two batches appears in both) and counters;
        each_batch(batch_dict) is called per batch when given."""
        r, keep = self.rbf(w.sv, w.alpha, w.gamma, w.b)
        d = r.d
        dom = self.domain(w.lo, w.hi, w.offset)
        sd = _dev(w.seeds, torch.float64, self.device).reshape(-1, d)
        flags = (mf.MF_WANT_ROOTS if roots else 0) | (mf.MF_ROOTS_FP64_EXACT if exact_roots else 0)
        opts = mf.mf_trace_opts(float(w.lam), 1 << 24, int(precision), float(recheck_band),
                                float(root_tol), int(max_edges), int(max_vertices), int(max_cells),
                                flags)
        st = _stream_handle(stream)
        n_coarse = mf.mf_subdiv_begin(self.h, r, dom, opts, int(k), sd.data_ptr(), sd.shape[0],
                                      int(cells_per_batch), st)
        res = self._alloc_outputs(d, int(max_edges), 1, 1)
        out = self._out_struct(res, d)
        parts, counts = [], dict(n_vertices=0, n_recheck=0, n_near_zero=0, root_evals=0, batches=0)
        left = n_coarse
        while left > 0:
            left = mf.mf_subdiv_next(self.h, out, st)
            E = out.n_edges
            b = {k2: res[k2][:E].clone() for k2 in ("edge_y", "edge_mask", "edge_f", "edge_t",
                                                    "points")}
            b["n_edges"] = E
            if each_batch is not None:
                each_batch(b)
            parts.append(b)
            for k2 in ("n_vertices", "n_recheck", "n_near_zero", "root_evals"):
                counts[k2] += getattr(out, k2)
            counts["batches"] += 1
        cat = {k2: (torch.cat([p[k2] for p in parts]) if parts else res[k2][:0])
               for k2 in ("edge_y", "edge_mask", "edge_f", "edge_t", "points")}
        cat.update(counts, n_edges=int(sum(p["n_edges"] for p in parts)), n_coarse_cells=n_coarse,
                   levels=out.levels, n_dead_seeds=out.n_dead_seeds)
        return cat

    def autotune(self, w, precision=mf.MF_FP64, batch_cap=1 << 24, max_edges=1 << 22,
                 max_vertices=0, max_cells=0, recheck_band=1e-3, root_tol=1e-12, stream=None):
        """Times launch variants on a trace of workload w and keeps the
        fastest for later traces on this context (mf_autotune)."""
        r, keep = self.rbf(w.sv, w.alpha, w.gamma, w.b)
        dom = self.domain(w.lo, w.hi, w.offset)
        sd = _dev(w.seeds, torch.float64, self.device).reshape(-1, r.d)
        opts = mf.mf_trace_opts(float(w.lam), int(batch_cap), int(precision), float(recheck_band),
                                float(root_tol), int(max_edges), int(max_vertices), int(max_cells),
                                0)
        return mf.mf_autotune(self.h, r, dom, opts, sd.data_ptr(), sd.shape[0],
                              _stream_handle(stream)).as_dict()

    def trace_batch(self, workloads, precisions=None, roots=True, cells=True, capacities=None,
                    batch_cap=1 << 24, recheck_band=1e-3, root_tol=1e-12, stream=None,
                    exact_roots=False, sort=False):
        """Traces many workloads in one batched call (mf_trace_batch).

        workloads: objects with sv, alpha, gamma, b, lam, offset, lo, hi, seeds.
        capacities: per-trace dicts (max_edges, max_vertices, max_cells); the
        output buffers are allocated at those capacities."""
        n = len(workloads)
        precisions = precisions or [mf.MF_FP64] * n
        capacities = capacities or [dict(max_edges=1 << 18)] * n
        rbfs = (mf.mf_rbf * n)()
        doms = (mf.mf_domain * n)()
        opts = (mf.mf_trace_opts * n)()
        outs = (mf.mf_trace_out * n)()
        seeds = (C.c_void_p * n)()
        nseeds = (C.c_int64 * n)()
        keep, bufs = [], []
        flags = (mf.MF_WANT_ROOTS if roots else 0) | (mf.MF_WANT_CELLS if cells else 0) | \
            (mf.MF_ROOTS_FP64_EXACT if exact_roots else 0) | (mf.MF_SORT_OUTPUT if sort else 0)
        for t, w in enumerate(workloads):
            r, k = self.rbf(w.sv, w.alpha, w.gamma, w.b)
            keep.append(k)
            rbfs[t] = r
            doms[t] = self.domain(w.lo, w.hi, w.offset)
            cap = capacities[t]
            me = int(cap.get("max_edges", 1 << 18))
            mv = int(cap.get("max_vertices", me))
            mc = int(cap.get("max_cells", 2 * me))
            opts[t] = mf.mf_trace_opts(float(w.lam), int(batch_cap), int(precisions[t]),
                                       float(recheck_band), float(root_tol), me, mv, mc, flags)
            sd = _dev(w.seeds, torch.float64, self.device).reshape(-1, r.d)
            keep.append(sd)
            seeds[t] = sd.data_ptr() if sd.numel() else None
            nseeds[t] = sd.shape[0]
            ce = mc * (r.d + 1) * r.d // 2
            b = self._alloc_outputs(r.d, me, mc, ce)
            bufs.append(b)
            outs[t] = self._out_struct(b, r.d)
        mf.mf_trace_batch(self.h, rbfs, doms, opts, seeds, nseeds, outs, _stream_handle(stream))
        results = []
        for t in range(n):
            o, b = outs[t], bufs[t]
            E, Cn, CE = o.n_edges, o.n_cells, o.n_cell_edges
            results.append(dict(
                edge_y=b["edge_y"][:E], edge_mask=b["edge_mask"][:E], edge_f=b["edge_f"][:E],
                edge_t=b["edge_t"][:E], points=b["points"][:E], cell_y=b["cell_y"][:Cn],
                cell_perm=b["cell_perm"][:Cn], cell_off=b["cell_off"][:Cn + 1],
                cell_idx=b["cell_idx"][:CE], n_edges=E, n_cells=Cn, n_cell_edges=CE,
                n_vertices=o.n_vertices, n_near_zero=o.n_near_zero, n_recheck=o.n_recheck,
                n_boundary=o.n_boundary, n_dead_seeds=o.n_dead_seeds, levels=o.levels,
                root_evals=o.root_evals))
        return results

    def server(self, max_slots=64, hbm_bytes=16 << 30):
        return Server(self, max_slots, hbm_bytes)

    def _alloc_outputs(self, d, E, Cn, CE):
        E, Cn, CE = max(int(E), 1), max(int(Cn), 1), max(int(CE), 1)
        dev = self.device
        return dict(edge_y=torch.empty((E, d), dtype=torch.int32, device=dev),
                    edge_mask=torch.empty(E, dtype=torch.int32, device=dev),
                    edge_f=torch.empty((E, 2), dtype=torch.float64, device=dev),
                    edge_t=torch.empty(E, dtype=torch.float64, device=dev),
                    points=torch.empty((E, d), dtype=torch.float64, device=dev),
                    cell_y=torch.empty((Cn, d), dtype=torch.int32, device=dev),
                    cell_perm=torch.empty((Cn, d), dtype=torch.uint8, device=dev),
                    cell_off=torch.empty(Cn + 1, dtype=torch.int64, device=dev),
                    cell_idx=torch.empty(CE, dtype=torch.int64, device=dev))

    @staticmethod
    def _out_struct(res, d):
        o = mf.mf_trace_out()
        if res:
            o.cap_edges = res["edge_y"].shape[0]
            o.edge_y = res["edge_y"].data_ptr()
            o.edge_mask = res["edge_mask"].data_ptr()
            o.edge_f = res["edge_f"].data_ptr()
            o.edge_t = res["edge_t"].data_ptr()
            o.points = res["points"].data_ptr()
            o.cap_cells = res["cell_y"].shape[0]
            o.cell_y = res["cell_y"].data_ptr()
            o.cell_perm = res["cell_perm"].data_ptr()
            o.cell_edge_off = res["cell_off"].data_ptr()
            o.cap_cell_edges = res["cell_idx"].shape[0]
            o.cell_edge_idx = res["cell_idx"].data_ptr()
        else:
            # ask for everything with zero capacity: the call reports the sizes
            o.cap_edges = 0
            o.edge_y = C.c_void_p(1).value
            o.cap_cells = 0
            o.cell_y = C.c_void_p(1).value
            o.cap_cell_edges = 0
            o.cell_edge_idx = C.c_void_p(1).value
        return o

    def certify(self, dh, radius, types, pose, dims, points, cell_off=None, cell_idx=None,
                stream=None):
        """Point verdicts, margins and per-cell AND of the point verdicts
        (mf_certify)."""
        r = self.certify_ex(dh, radius, types, pose, dims, points, cell_off, cell_idx,
                            whole=False, stream=stream)
        return r["verdict"], r["margin"], r["cell_verdict"]

    def certify_ex(self, dh, radius, types, pose, dims, points, cell_off=None, cell_idx=None,
                   spheres=None, whole=True, slack=True, stream=None):
        """mf_certify_ex: radius None = no link capsules; spheres = (link [n],
        centre [n][3] in frame T_{link+1}, radius [n]) or None.  Returns device
        tensors verdict, margin, element and, with cells, cell_verdict and
        (whole=True) cell_whole and (slack=True) cell_slack; without the
        slack the library decides most cells in FP32 under an error bound."""
        dev = self.device
        dh_t = _dev(dh, torch.float64, dev).reshape(-1, 4)
        rad_t = None if radius is None else _dev(radius, torch.float64, dev)
        ty_t = _dev(types, torch.int32, dev)
        po_t = _dev(pose, torch.float64, dev).reshape(-1, 12)
        di_t = _dev(dims, torch.float64, dev).reshape(-1, 3)
        d = dh_t.shape[0]
        pts = _dev(points, torch.float64, dev).reshape(-1, d)
        P = pts.shape[0]
        res = dict(verdict=torch.empty(max(P, 1), dtype=torch.uint8, device=dev),
                   margin=torch.empty(max(P, 1), dtype=torch.float64, device=dev),
                   element=torch.empty(max(P, 1), dtype=torch.int16, device=dev))
        if spheres is not None:
            sl = _dev(spheres[0], torch.int32, dev)
            sc = _dev(spheres[1], torch.float64, dev).reshape(-1, 3)
            sr = _dev(spheres[2], torch.float64, dev)
            sph = (int(sl.shape[0]), sl.data_ptr(), sc.data_ptr(), sr.data_ptr())
        else:
            sph = (0, None, None, None)
        robot = mf.mf_robot(d, dh_t.data_ptr(), rad_t.data_ptr() if rad_t is not None else None,
                            *sph)
        scene = mf.mf_scene(ty_t.shape[0], ty_t.data_ptr(), po_t.data_ptr(), di_t.data_ptr())
        out = mf.mf_certify_out(res["verdict"].data_ptr(), res["margin"].data_ptr(),
                                res["element"].data_ptr(), None, None, None)
        nc, offp, idxp = 0, None, None
        if cell_off is not None and cell_off.shape[0] > 1:
            off_t = _dev(cell_off, torch.int64, dev)
            idx_t = _dev(cell_idx, torch.int64, dev)
            nc = off_t.shape[0] - 1
            offp, idxp = off_t.data_ptr(), idx_t.data_ptr() if idx_t.numel() else None
            res["cell_verdict"] = torch.empty(nc, dtype=torch.uint8, device=dev)
            out.cell_verdict = res["cell_verdict"].data_ptr()
            if whole:
                res["cell_whole"] = torch.empty(nc, dtype=torch.uint8, device=dev)
                out.cell_whole = res["cell_whole"].data_ptr()
                if slack:
                    res["cell_slack"] = torch.empty(nc, dtype=torch.float64, device=dev)
                    out.cell_slack = res["cell_slack"].data_ptr()
        else:
            res["cell_verdict"] = torch.empty(0, dtype=torch.uint8, device=dev)
        mf.mf_certify_ex(self.h, robot, scene, pts.data_ptr(), P, d, offp, idxp, nc, out,
                         _stream_handle(stream))
        for k in ("verdict", "margin", "element"):
            res[k] = res[k][:P]
        return res


class Server:
    """Continuous-batching proof server (mf_server_*): submit requests at any
    time, call step() to admit, advance and finish traces, fetch() results."""

    def __init__(self, ctx: Context, max_slots=64, hbm_bytes=16 << 30):
        self.ctx = ctx
        self.h = mf.mf_server_create(ctx.h, max_slots, hbm_bytes)
        self._keep = {}

    def close(self):
        if self.h:
            mf.mf_server_destroy(self.h)
            self.h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, w, precision=mf.MF_MIXED_FP32, roots=True, cells=True, max_edges=1 << 20,
               max_vertices=0, max_cells=0, batch_cap=1 << 24, recheck_band=1e-3, root_tol=1e-12,
               exact_roots=False):
        r, keep = self.ctx.rbf(w.sv, w.alpha, w.gamma, w.b)
        dom = self.ctx.domain(w.lo, w.hi, w.offset)
        sd = _dev(w.seeds, torch.float64, self.ctx.device).reshape(-1, r.d)
        opts = mf.mf_trace_opts(float(w.lam), int(batch_cap), int(precision), float(recheck_band),
                                float(root_tol), int(max_edges), int(max_vertices), int(max_cells),
                                (mf.MF_WANT_ROOTS if roots else 0) | (mf.MF_WANT_CELLS if cells else 0)
                                | (mf.MF_ROOTS_FP64_EXACT if exact_roots else 0))
        rid = mf.mf_server_submit(self.ctx.h, self.h, r, dom, opts, sd.data_ptr(), sd.shape[0])
        self._keep[rid] = (keep, sd, r.d, max_edges, max_cells or 2 * max_edges)
        return rid

    def step(self, stream=None):
        return mf.mf_server_step(self.ctx.h, self.h, _stream_handle(stream))

    def status(self, rid):
        return mf.mf_server_status(self.ctx.h, self.h, rid)

    def wait(self, rid, timeout_ms, stream=None):
        """Steps the server until request rid is done or failed (returns its
        state), or until timeout_ms passes (returns None)."""
        rc, state = mf.mf_server_wait(self.ctx.h, self.h, rid, timeout_ms, _stream_handle(stream))
        return None if rc == mf.MF_ERR_TIMEOUT else state

    def done(self):
        """Ids of the requests that finished or failed since the last call."""
        return mf.mf_server_done(self.ctx.h, self.h)

    def fetch(self, rid, stream=None):
        keep, sd, d, me, mc = self._keep[rid]
        # two-call pattern: the counts first (capacity error, request kept),
        # then buffers of exactly that size
        probe = mf.mf_trace_out()
        state = self.status(rid)[0]
        rc = mf.mf_server_fetch(self.ctx.h, self.h, rid, probe, _stream_handle(stream), check=False)
        if rc not in (mf.MF_OK, mf.MF_ERR_CAPACITY):
            if state < 0:  # a failed request is forgotten by the server
                self._keep.pop(rid, None)
            mf._check(self.ctx.h, rc)
        bufs = self.ctx._alloc_outputs(d, probe.n_edges, probe.n_cells, probe.n_cell_edges)
        out = probe  # an empty result fits zero capacities and is already fetched
        if rc == mf.MF_ERR_CAPACITY:
            out = self.ctx._out_struct(bufs, d)
            mf.mf_server_fetch(self.ctx.h, self.h, rid, out, _stream_handle(stream))
        del self._keep[rid]
        E, Cn, CE = out.n_edges, out.n_cells, out.n_cell_edges
        return dict(edge_y=bufs["edge_y"][:E], edge_mask=bufs["edge_mask"][:E],
                    edge_f=bufs["edge_f"][:E], edge_t=bufs["edge_t"][:E], points=bufs["points"][:E],
                    cell_y=bufs["cell_y"][:Cn], cell_perm=bufs["cell_perm"][:Cn],
                    cell_off=bufs["cell_off"][:Cn + 1], cell_idx=bufs["cell_idx"][:CE],
                    n_edges=E, n_cells=Cn, n_cell_edges=CE, n_vertices=out.n_vertices,
                    n_near_zero=out.n_near_zero, n_recheck=out.n_recheck,
                    n_boundary=out.n_boundary, n_dead_seeds=out.n_dead_seeds, levels=out.levels,
                    root_evals=out.root_evals)
