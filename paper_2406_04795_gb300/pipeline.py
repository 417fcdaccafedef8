"""One proof = one pass of the traced path on one workload: ``mf_trace`` (locate
seeds, breadth-first tracing, roots, cells and their CSR) followed by
``mf_certify_ex`` (forward kinematics and capsule/obstacle checks of every
intersection point, AND over each cell, and the whole-cell certificate of each
cell's manifold piece).  Inputs stay resident on the device;
outputs are preallocated after the first call so that repeated steps allocate
nothing."""
from __future__ import annotations

import numpy as np
import torch

from . import mf
from .api import Context

# Capacities of the resident tables per workload family (edges, vertices,
# cells).  Measured ratios on these workloads: vertices/edges ~ 0.2-0.5,
# cells/edges ~ 1.5 (d=3) to ~10 (d=5), cell edges/cell ~ 3-6.
SIZING = {
    3: dict(max_edges=1 << 20, max_vertices=1 << 20, max_cells=1 << 22),
    4: dict(max_edges=1 << 22, max_vertices=1 << 22, max_cells=1 << 25),
    5: dict(max_edges=100_000_000, max_vertices=40_000_000, max_cells=1_000_000_000),
    # d=6 measured at lambda=0.2: 2.56e6 edges, 3.9e5 vertices, 7.1e7 cells; at
    # lambda=0.04 the same power law gives ~8e9 edges, beyond one GPU's HBM
    6: dict(max_edges=4_000_000, max_vertices=1_000_000, max_cells=120_000_000),
}


LAMBDA_REF = {3: 0.1, 4: 0.08, 5: 0.05, 6: 0.2}


def sizing_for(w) -> dict:
    """Table capacities for a workload: the family's sizing scaled by
    (lambda_ref / lambda)^(d-1) (traced sets grow as lambda^-(d-1))."""
    base = SIZING.get(w.d, SIZING[6])
    f = (LAMBDA_REF.get(w.d, 0.04) / w.lam) ** (w.d - 1)
    if abs(f - 1.0) > 1e-9:
        f *= 1.6  # the power law is only approximate away from the reference lambda
    f = min(max(f, 1e-3), 64.0)
    return {k: int(max(v * f, 1 << 16)) for k, v in base.items()}


def precision_of(w) -> int:
    """fp64: FP64 throughout; mixed: distance GEMM on the tensor cores (BF16
    split operands, FP32 accumulation) with FP64 recheck; mixed_fp32: FP32
    SIMT distances with FP64 recheck."""
    return {"fp64": mf.MF_FP64, "mixed_fp32": mf.MF_MIXED_FP32}.get(w.precision, mf.MF_MIXED_BF16)


class Proof:
    """Device-resident inputs and reusable outputs for one workload."""

    def __init__(self, ctx: Context, w, precision=None, sizing=None):
        self.ctx, self.w = ctx, w
        dev = ctx.device
        self.precision = precision_of(w) if precision is None else precision
        self.sizing = dict(sizing_for(w) if sizing is None else sizing)
        t = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
        self.sv, self.alpha, self.seeds = t(w.sv), t(w.alpha), t(w.seeds)
        self.dh, self.radius = t(w.dh), t(w.radius)
        self.otype, self.opose, self.odims = t(w.obs_type, torch.int32), t(w.obs_pose), t(w.obs_dims)
        self.outputs = None
        self.last = None
        self.whole = None

    def step(self, stream=None):
        w = self.w
        for attempt in range(6):
            try:
                r = self.ctx.trace(self.sv, self.alpha, w.gamma, w.b, w.lam, w.offset, w.lo, w.hi,
                                   self.seeds, precision=self.precision, roots=True, cells=True,
                                   batch_cap=w.batch_cap, recheck_band=w.recheck_band,
                                   outputs=self.outputs, stream=stream, **self.sizing)
                break
            except mf.MfError as e:
                # capacities are estimates away from the reference lambda: grow
                # them (on the first, untimed steps) and trace again
                if e.code != mf.MF_ERR_MAXEDGES or attempt == 5:
                    raise
                self.sizing = {k: int(v * 2) for k, v in self.sizing.items()}
                self.outputs = None
        self.outputs = r["_buffers"]
        # points (verdicts, margins), the AND over each cell's points, and the
        # whole-cell (Lipschitz) certificate of each cell's manifold piece
        c = self.ctx.certify_ex(self.dh, self.radius, self.otype, self.opose, self.odims,
                                r["points"], r["cell_off"], r["cell_idx"], whole=True,
                                slack=False, stream=stream)
        v, m, cv = c["verdict"], c["margin"], c["cell_verdict"]
        self.whole = c.get("cell_whole")
        self.last = (r, v, m, cv)
        return r, v, m, cv


def host_inputs(w):
    """Pinned host copies of a workload's inputs (for end-to-end timing)."""
    pin = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt).pin_memory()
    return dict(sv=pin(w.sv), alpha=pin(w.alpha), seeds=pin(w.seeds), dh=pin(w.dh),
                radius=pin(w.radius), otype=pin(w.obs_type, torch.int32), opose=pin(w.obs_pose),
                odims=pin(w.obs_dims))
