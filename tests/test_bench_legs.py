"""Host logic of the benchmark's CPU-baseline leg: cells whose points are
all in collision are sampled from a traced proof (here the FP64 oracle's own
trace and certification of the d=5 workload at a coarse lambda), and the
dense-sampling check runs the oracle on convex combinations of each cell's
points."""
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import oracle  # noqa: E402
from paper_2406_04795_gb300 import workloads as W  # noqa: E402


def test_dense_sampling_leg_on_colliding_cells():
    w = W.config_d5(lam=0.6)
    o = oracle.trace(w.sv, w.alpha, w.gamma, w.b, w.lam, w.offset, w.lo, w.hi, w.seeds)
    v, m, cv = oracle.certify(w.dh, w.radius, w.obs_type, w.obs_pose, w.obs_dims, o["edge_pt"],
                              o["cell_off"], o["cell_idx"])
    assert cv.sum() > 0, "the workload should have cells in collision"
    r = {"points": torch.as_tensor(o["edge_pt"]), "cell_off": torch.as_tensor(o["cell_off"]),
         "cell_idx": torch.as_tensor(o["cell_idx"])}
    whole = torch.zeros(len(cv), dtype=torch.uint8)
    k = bench.sample_cells(w, r, torch.as_tensor(cv.astype(np.uint8)), whole, n_cells=20)
    assert 0 < len(k["cells"]) <= 20
    for P in k["cells"]:
        vv, _, _ = oracle.certify(w.dh, w.radius, w.obs_type, w.obs_pose, w.obs_dims, P)
        assert vv.all()  # a sampled cell's points are all in collision
    out = bench.oracle_checks({"main": k})
    rec = out["main_cells_dense_sampling"]
    assert rec["cells_sampled"] == len(k["cells"]) and rec["samples_per_cell"] == 200
    assert 0 <= rec["point_only_false_certify"] <= rec["cells_sampled"]
    assert rec["whole_certified_with_free_sample"] == 0
