"""Benchmark: traced simplices per second (and ms per proof) of the manifold
tracing + certification path on GB300.

A step is one proof: mf_trace (seeds, BFS, roots, cells, CSR) + mf_certify on
one synthetic workload (default: d=5, 2048 support vectors, gamma=4,
lambda=0.05, 16 seeds, batch cap 2^24, FP64 path).  Inputs are resident in HBM
for the device-timed value; the e2e figure copies the inputs from pinned host
memory and reads the point verdicts back every step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                  [--config d5|d3|d6] [--precision auto|fp64|mixed|mixed_fp32]

Under torchrun each rank traces its own independent workload (seed + rank):
weak scaling, no collective on the data path.  `--impl reference` times the
FP64 CPU oracle (the only other arm this method has) on a bounded sample.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2406_04795_gb300 import workloads as W  # noqa: E402

# FP64 flops of one table-driven exp: k (1 FMA), k - shift (1 add), r (2 FMA),
# r^2 (1 mul), degree-5 polynomial (4 FMA), table product (1 FMA), 2^m (1 mul);
# an FMA counts 2 flops
FP64_EXP_FLOPS = 19


# FP32-pipe operations of one double-float strong term of the root step
# (k_roots_terms): per coordinate 3 TwoSums, 3 adds and a fast TwoSum for
# u = x - s, a TwoProduct, an FMA and a fast TwoSum for u^2, a double-float
# add into r2 (47); then z = gamma r2, the reduction, the polynomial, the
# table product, the scaling, alpha e and the sum (68)
def df_term_ops(d):
    return 47 * d + 68


# FP32-pipe operations of one FP32 term (Halley step or weak term): per
# coordinate a hi and a lo difference, their sum, r2 and the projection
# FMAs (5); then the exponent, ex2, alpha e and the accumulations (8)
def f32_term_ops(d):
    return 5 * d + 8


# DRAM bytes per traced edge of the root phase's kernels from their ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum of k_roots_prep,
# k_roots_f64 (warp and redo launches), k_roots_x, k_roots_terms and
# k_roots_finish on the lambda = 0.15 case of the d=5 workload, divided by
# its 880,448 edges: 1229.8 MB); None once a kernel has changed since the
# capture
ROOTS_DRAM_BYTES_PER_EDGE = 1396.8


def make_workload(cfg: str, rank: int, lam=None):
    kw = {} if lam is None else {"lam": lam}
    if cfg == "d3":
        return W.config_d3(seed=1000 + 10 * rank, **kw)
    if cfg == "d6":
        return W.config_d6(seed=1002 + 10 * rank, **kw)
    return W.config_d5(seed=1001 + 10 * rank, **kw)


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.rows, self.proc = index, [], None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) < 9:
                continue
            for k, n in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


def roofline(stats, w, rates, E, ms_proof, n_proofs, root_traffic=True):
    """Roofline of the dominant phase against the measured peaks: the FP64
    pipe (mf_probe_rates FP64 FMA probe) for the FP64 vertex evaluation and
    certification, the FP32 pipe (FP32 FMA probe, one operation per
    instruction) for the root solve, whose strong terms are double-float
    and whose Halley steps and weak terms are FP32, the MUFU ex2 probe for
    the tensor-core evaluation, the STREAM copy for the table phases.  Work
    is counted in kept terms: the screened sum keeps only the terms that can
    exceed 3e-10 (1e-8 in the root step), so the dense N x (vertices + root
    evaluations) count of an unscreened sum does not apply.  Also the whole
    proof's per-edge time against its bound max(FP64 flops / FP64 peak,
    FP32 operations / FP32 rate, ex2 / ex2 rate, bytes / HBM)."""
    peaks, src = measured_peaks()
    dom = max(stats, key=lambda k: stats[k]["ms"])
    s = stats[dom]
    ms_per_launch = s["ms"] / max(s["launches"], 1)
    d = w.d
    fp64_peak = 2.0 * rates["fp64_fma_per_s"] / 1e12  # TFLOP/s, measured
    f32_peak = rates["fp32_fma_per_s"] / 1e12         # T FP32 instructions/s, measured
    ex2_peak = rates["ex2_per_s"] / 1e12             # T ex2/s, measured
    phase_ms = {k: round(v["ms"], 3) for k, v in stats.items() if v["ms"] > 0}
    per_eval = 3 * d + 3 + FP64_EXP_FLOPS
    # proof level (per traced edge): FP64 flops of the vertex evaluation's
    # strong terms, FP32 operations of the root solve (double-float strong
    # terms; FP32 Halley and weak terms) and of the evaluation's weak terms,
    # ex2 of all FP32 terms, and the algorithmic bytes of the table phases
    f64 = stats["eval"]["terms"] * per_eval
    f32 = (stats["roots"]["terms"] * df_term_ops(d) +
           (stats["roots"]["terms_weak"] + stats["eval"]["terms_weak"]) * f32_term_ops(d))
    ex2 = stats["roots"]["terms_weak"] + stats["eval"]["terms_weak"]
    k = d // 2
    by = (stats["expand_vertices"]["units"] * ((4 * d + 4) + 32 * 2 ** d) +
          stats["expand_edges"]["units"] * ((4 * d + 20) + 64 * 2 ** d) +
          stats["roots"]["units"] * (40 + 8 * d + 8 + 8 * d) +
          stats["cells"]["units"] * ((4 * d + 4) + 32 * (2 ** k + 2 ** (d - k + 1))) +
          stats["csr"]["units"] * ((5 * d) + (32 + 8) * (d + 1)))
    steps = max(n_proofs, 1)
    t_f64 = f64 / steps / (fp64_peak * 1e12)
    t_f32 = f32 / steps / (f32_peak * 1e12)
    t_ex2 = ex2 / steps / (ex2_peak * 1e12)
    t_hbm = by / steps / (peaks["hbm_gbs"] * 1e9)
    t_bound = max(t_f64, t_f32, t_ex2, t_hbm)
    proof = {"ns_per_edge": ms_proof * 1e6 / max(E, 1), "bound_ns_per_edge": t_bound * 1e9 / max(E, 1),
             "frac": t_bound / (ms_proof * 1e-3), "bound_by": ["fp64", "fp32", "ex2", "hbm"][
                 [t_f64, t_f32, t_ex2, t_hbm].index(t_bound)],
             "fp64_ms": t_f64 * 1e3, "fp32_ms": t_f32 * 1e3, "ex2_ms": t_ex2 * 1e3,
             "hbm_ms": t_hbm * 1e3}
    base = {"phase_ms": phase_ms, "proof": proof,
            "measured_rates": {k: v for k, v in rates.items()}}
    if dom == "eval" and w.precision not in ("fp64", "mixed_fp32"):
        # tensor-core evaluation: the distance GEMM runs on tcgen05, every term
        # then takes one MUFU ex2, which binds
        ex = s["terms_weak"] / max(s["launches"], 1)
        ach = ex / (ms_per_launch * 1e-3) / 1e12
        return dict(base, kernel="k_eval_tc", bound="alu", achieved=ach, peak=ex2_peak,
                    unit="T ex2/s", frac=ach / ex2_peak, traffic=None,
                    peak_source="measured: mf_probe_rates ex2.approx probe",
                    work="%d RBF terms (vertex x support vector), one ex2 each" % s["terms_weak"])
    if dom == "roots":
        # the root phase's arithmetic runs on the FP32 pipe: double-float
        # strong terms (k_roots_terms) and FP32 Halley / weak terms (the warp
        # kernel); the few full FP64 re-evaluations are counted as strong terms
        ops = (s["terms"] * df_term_ops(d) + s["terms_weak"] * f32_term_ops(d)) / max(s["launches"], 1)
        ach = ops / (ms_per_launch * 1e-3) / 1e12
        # DRAM bytes per edge from the ncu capture of the root kernels
        # (profiles/), scaled by the edges one launch processes
        # (taken on the FP64 path: none for the other precision)
        traffic = ROOTS_DRAM_BYTES_PER_EDGE * s["units"] / max(s["launches"], 1) \
            if ROOTS_DRAM_BYTES_PER_EDGE and root_traffic else None
        return dict(base, kernel="roots phase: k_roots_prep, k_roots_f64 (warp screen and FP32 "
                    "Halley steps), k_roots_x, k_roots_terms (double-float sums), k_roots_finish",
                    bound="alu", achieved=ach, peak=f32_peak, unit="T FP32 ops/s",
                    frac=ach / f32_peak, traffic=traffic,
                    peak_source="measured: mf_probe_rates FP32 FMA probe (one operation per "
                    "instruction)",
                    work="%d strong terms x %d FP32 ops (double-float) + %d FP32 terms x %d ops" % (
                        s["terms"], df_term_ops(d), s["terms_weak"], f32_term_ops(d)))
    if dom == "eval":
        flops = s["terms"] * per_eval / max(s["launches"], 1)
        ach = flops / (ms_per_launch * 1e-3) / 1e12
        return dict(base, kernel="k_eval_vertices_f64", bound="alu", achieved=ach, peak=fp64_peak,
                    unit="TFLOP/s", frac=ach / fp64_peak, traffic=None,
                    peak_source="measured: mf_probe_rates FP64 FMA probe (2 flops per FMA)",
                    work="%d kept FP64 terms x %d flops (and %d FP32 weak terms, not counted)" % (
                        s["terms"], per_eval, s["terms_weak"]))
    if dom == "certify_points":
        n_obs = int(w.obs_type.shape[0])
        flops = s["units"] * d * (60 + n_obs * 150) / max(s["launches"], 1)
        ach = flops / (ms_per_launch * 1e-3) / 1e12
        return dict(base, kernel="k_certify_points", bound="alu", achieved=ach, peak=fp64_peak,
                    unit="TFLOP/s", frac=ach / fp64_peak, traffic=None,
                    peak_source="measured: mf_probe_rates FP64 FMA probe")
    # table phases: algorithmic bytes = one 32-byte sector per hash probe / record touched
    per_unit = {"expand_vertices": (4 * d + 4) + 32 * (2 ** d),
                "expand_edges": (4 * d + 20) + 64 * (2 ** d),
                "cells": (4 * d + 4) + 32 * (2 ** k + 2 ** (d - k + 1)),
                "csr": (5 * d) + (32 + 8) * (d + 1)}.get(dom, 64)
    byl = s["units"] * per_unit / max(s["launches"], 1)
    ach = byl / (ms_per_launch * 1e-3) / 1e9
    return dict(base, kernel=dom, bound="hbm", achieved=ach, peak=peaks["hbm_gbs"], unit="GB/s",
                frac=ach / peaks["hbm_gbs"], traffic=None, peak_source=src)


def _oracle_rate(w, threads, budget_s):
    import oracle
    oracle.build()
    used = oracle.set_threads(threads)
    n = 200
    while True:
        t0 = time.perf_counter()
        r = oracle.trace(w.sv, w.alpha, w.gamma, w.b, w.lam, w.offset, w.lo, w.hi, w.seeds,
                         roots=True, cells=True, max_edges=n)
        oracle.certify(w.dh, w.radius, w.obs_type, w.obs_pose, w.obs_dims, r["edge_pt"],
                       r["cell_off"], r["cell_idx"])
        dt = time.perf_counter() - t0
        E = len(r["edge_t"])
        if dt > budget_s / 4 or E < n:
            return E / dt, E, dt, used
        n *= 4


def cpu_baseline(w, E_proof=None, budget_s=15.0):
    """The FP64 oracle on a bounded sample of the same workload: trace (with
    roots and cells) until max_edges edges exist, then certify those points;
    on all host cores (its per-edge root and certification loops are OpenMP)
    and on one.  The per-edge cost is dominated by the bisection roots
    (50 + 17 f evaluations per edge), which cost the same on every edge, so
    the BFS prefix is a fair sample of the proof's per-edge cost."""
    import oracle
    rate, E, dt, cores = _oracle_rate(w, 0, budget_s)
    rate1, E1, dt1, _ = _oracle_rate(w, 1, budget_s / 2)
    oracle.set_threads(0)
    out = {"value": rate, "unit": "simplices/s", "cores": cores, "kind": "oracle",
           "sample": "first %d edges of the BFS (+ roots, cells, certify) in %.1f s on %d threads;"
                     " %d edges in %.1f s on 1 thread" % (E, dt, cores, E1, dt1),
           "value_1core": rate1, "host_cores": os.cpu_count()}
    if E_proof:
        out["ms_per_proof_est"] = 1e3 * E_proof / rate
        out["ms_per_proof_est_1core"] = 1e3 * E_proof / rate1
    return out


def run_served(ctx, arrivals, reqs, precision, max_slots=64, hbm_bytes=200 << 30):
    """Requests arriving at the given times (seconds) through the
    continuous-batching server: p50 / p99 latency (arrival -> results
    fetched), simplices/s over the wall time, failed requests."""
    import torch
    from paper_2406_04795_gb300 import mf
    n_requests = len(reqs)
    free, _ = torch.cuda.mem_get_info()
    hbm_bytes = int(min(hbm_bytes, 0.8 * free))  # inside the context's budget (0.9 x free)
    server = ctx.server(max_slots=max_slots, hbm_bytes=hbm_bytes)
    lat, edges, nxt, failed, codes = [], 0, 0, 0, {}
    live = {}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    while nxt < n_requests or live:
        now = time.perf_counter() - t0
        if now > 600.0:
            raise RuntimeError("served run exceeded 600 s")
        while nxt < n_requests and arrivals[nxt] <= now:
            w = reqs[nxt]
            rid = server.submit(w, precision=precision, **W.shell_capacity(w))
            live[rid] = arrivals[nxt]
            nxt += 1
        if not live:
            time.sleep(max(0.0, arrivals[nxt] - (time.perf_counter() - t0)))
            continue
        server.step()
        for rid in server.done():
            state = server.status(rid)[0]
            if state == 2:
                edges += server.fetch(rid)["n_edges"]
            else:
                failed += 1
                codes[str(state)] = codes.get(str(state), 0) + 1
                try:
                    server.fetch(rid)
                except mf.MfError:
                    pass
            lat.append(time.perf_counter() - t0 - live.pop(rid))
    wall = time.perf_counter() - t0
    server.close()
    lat_ms = np.array(lat) * 1e3
    return {"requests": n_requests, "failed": failed, "failed_codes": codes, "slots": max_slots,
            "arena_gib": round(hbm_bytes / 2**30, 1),
            "p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
            "simplices_per_s": edges / wall, "simplices": edges, "wall_s": wall}


def tune_on(ctx, ws, caps=None):
    """Untimed: the autotuner on the largest of the workloads ws (mixed
    precision; caps: their capacities, else the shell capacities), so that
    the context's launch choices (tensor-core chunk width, root group screen)
    serve the batched engine and the server."""
    from paper_2406_04795_gb300 import mf
    i = max(range(len(ws)), key=lambda i: ws[i].sv.shape[0] / ws[i].lam ** ws[i].d)
    c = caps[i] if caps else W.shell_capacity(ws[i])
    try:
        return ctx.autotune(ws[i], precision=mf.MF_MIXED_BF16, **c)
    except Exception as e:  # a tuning failure leaves the defaults
        return {"error": str(e)[:200]}


def served_lines(ctx, n_requests, rate_hz, seed=1005):
    """The served workload at its arrival rate on the mixed path (distance
    GEMM on the tensor cores, FP64 recheck), and the same requests all at once
    on the mixed and on the FP64 path (capacity)."""
    from paper_2406_04795_gb300 import mf
    arrivals, reqs = W.served_requests(seed=seed, n_requests=n_requests, rate_hz=rate_hz)
    tune = tune_on(ctx, reqs)
    out = run_served(ctx, arrivals, reqs, mf.MF_MIXED_BF16)
    out["tune"] = tune
    out.update({"rate_hz": rate_hz, "precision": "mixed_bf16",
                "workload": "Poisson arrivals; d in {4,5,6}, 512-8192 SVs, lambda in [0.03,0.08], "
                            "1-16 seeds"})
    burst = np.zeros(len(reqs))
    cap = {}
    for name, prec in (("mixed_bf16", mf.MF_MIXED_BF16), ("fp64", mf.MF_FP64)):
        r = run_served(ctx, burst, reqs, prec)
        cap[name] = {"simplices_per_s": r["simplices_per_s"], "wall_s": r["wall_s"],
                     "p50_ms": r["p50_ms"], "failed": r["failed"]}
    out["saturated"] = cap
    return out


def _proof_ms(ctx, w, reps=2, stats=None):
    """Device-timed ms per proof of workload w (after one untimed proof);
    with a dict in stats, the library's per-phase counters of the timed
    proofs are put there (profiling on, as in the main line)."""
    import torch
    from paper_2406_04795_gb300 import mf
    from paper_2406_04795_gb300.pipeline import Proof
    p = Proof(ctx, w)
    p.step()
    torch.cuda.synchronize()
    if stats is not None:
        mf.mf_ctx_set_profiling(ctx.h, True)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        r, v, m, cv = p.step()
    e1.record(stream)
    torch.cuda.synchronize()
    if stats is not None:
        stats.update(mf.mf_ctx_get_stats(ctx.h))
        mf.mf_ctx_set_profiling(ctx.h, False)
    return e0.elapsed_time(e1) / reps, p, r


def eval_tc_roofline(stats, rates):
    """The tensor-core evaluation of a mixed proof against the MUFU ex2
    roofline: every RBF term (vertex x support vector) takes one ex2 after
    its distance comes out of the BF16 MMA."""
    s = stats["eval"]
    ex2_peak = rates["ex2_per_s"] / 1e12
    ms = s["ms"] / max(s["launches"], 1)
    ex = s["terms_weak"] / max(s["launches"], 1)
    ach = ex / (ms * 1e-3) / 1e12 if ms > 0 else 0.0
    return {"kernel": "k_eval_tc (+ FP64 recheck)", "bound": "alu", "achieved": ach,
            "peak": ex2_peak, "unit": "T ex2/s", "frac": ach / ex2_peak,
            "peak_source": "measured: mf_probe_rates ex2.approx probe",
            "phase_ms": s["ms"], "terms": s["terms_weak"]}


def config_lines(ctx, d6_lam=0.15):
    """The other workload configurations, each one line (untimed by the main
    metric): d=3 FP64; d=6 mixed BF16 at the finest lambda traced here.  The
    proofs' sampled edges are kept for the oracle comparison of the CPU
    baseline leg."""
    out, keep = {}, {}
    w3 = W.config_d3()
    ms, p, r = _proof_ms(ctx, w3, reps=5)
    out["d3_fp64"] = {"workload": w3.name, "lambda": w3.lam, "n_sv": int(w3.sv.shape[0]),
                      "ms_per_proof": ms, "simplices_per_s": r["n_edges"] / (ms * 1e-3),
                      "edges_per_proof": r["n_edges"], "cells_per_proof": r["n_cells"],
                      "cells_points_in_collision": int(p.last[3].sum().item()),
                      "cells_whole_certified": int(p.whole.sum().item())}
    keep["d3"] = sample_cells(w3, r, p.last[3], p.whole)
    del p, r
    w6 = W.config_d6(lam=d6_lam)
    ms, p, r = _proof_ms(ctx, w6)
    E = r["n_edges"]
    rng = np.random.default_rng(6)
    idx = np.sort(rng.choice(E, min(E, 400), replace=False))
    keep["d6"] = dict(w=w6, y=r["edge_y"][idx].cpu().numpy(),
                      m=r["edge_mask"][idx].cpu().numpy().astype(np.uint32),
                      t=r["edge_t"][idx].cpu().numpy(), f=r["edge_f"][idx].cpu().numpy(),
                      pt=r["points"][idx].cpu().numpy())
    out["d6_mixed_bf16"] = {
        "workload": w6.name, "lambda": w6.lam, "lambda_config": 0.04, "n_sv": int(w6.sv.shape[0]),
        "ms_per_proof": ms, "simplices_per_s": E / (ms * 1e-3), "edges_per_proof": E,
        "cells_per_proof": r["n_cells"], "vertices_per_proof": r["n_vertices"],
        "rechecked_vertices": r["n_recheck"],
        "note": "lambda 0.04 gives ~8e9 edges (lambda^-5 law), beyond one GPU's memory; its "
                "sampled error against the FP64 oracle is in cpu_baseline.d6_error_vs_oracle"}
    del p, r
    return out, keep


def sample_cells(w, r, cv, whole, n_cells=300, seed=7):
    """Up to n_cells random cells of a proof whose points are all in
    collision, with their points and whole-cell verdicts (host copies), for
    the dense-sampling check of the CPU-baseline leg."""
    import torch
    cells = torch.nonzero(cv).flatten()
    if cells.numel() == 0:
        return dict(w=w, cells=[], whole=np.zeros(0, bool))
    # distinct random positions (drawn on the host, few of them)
    rng = np.random.default_rng(seed)
    k = min(n_cells, cells.numel())
    if cells.numel() <= 4 * k:
        pos = rng.choice(cells.numel(), size=k, replace=False)
    else:
        pos = np.unique(rng.integers(0, cells.numel(), size=2 * k))
        rng.shuffle(pos)
        pos = pos[:k]
    pick = cells[torch.as_tensor(pos, dtype=torch.int64, device=cells.device)]
    lo = r["cell_off"][pick].cpu().tolist()
    hi = r["cell_off"][pick + 1].cpu().tolist()
    out = []
    for a, b in zip(lo, hi):
        idx = r["cell_idx"][a:b]
        out.append(r["points"][idx].cpu().numpy())
    wh = whole[pick].cpu().numpy().astype(bool) if whole is not None else np.zeros(len(out), bool)
    return dict(w=w, cells=out, whole=wh)


def oracle_checks(keep):
    """CPU-baseline leg: the FP64 oracle on the samples the GPU lines kept:
    the d=6 mixed proof's sampled roots and end values (error vs the oracle),
    and cells whose points are all in collision (from the main proof, and the
    d=3 proof's when it has any): the point-only verdict's false-certify rate
    against dense sampling of each cell's piece (convex combinations of its
    points), and that no whole-cell certified cell has a free sample."""
    import oracle
    oracle.set_threads(0)
    out = {}
    if "d6" in keep:
        k = keep["d6"]
        w6 = k["w"]
        f2, t, pt, multi = oracle.edge_roots(w6.sv, w6.alpha, w6.gamma, w6.b, w6.lam, w6.offset,
                                             k["y"], k["m"])
        ok = (multi == 0) & np.all(np.abs(f2) >= 1e-12, axis=1)
        out["d6_error_vs_oracle"] = {
            "sampled_edges": int(ok.sum()), "max_dt": float(np.abs(k["t"] - t)[ok].max()),
            "max_dpoint": float(np.abs(k["pt"] - pt)[ok].max()),
            "max_df_edge_ends": float(np.abs(k["f"] - f2).max()),
            "sign_mismatches": int(np.sum((f2 >= 0) != (k["f"] >= 0)))}
    for name in ("main", "d3"):
        if name not in keep:
            continue
        k = keep[name]
        w = k["w"]
        rng = np.random.default_rng(7)
        false_pt = false_whole = 0
        for P, wh in zip(k["cells"], k["whole"]):
            S = rng.dirichlet(np.ones(P.shape[0]), size=200) @ P
            v, _, _ = oracle.certify(w.dh, w.radius, w.obs_type, w.obs_pose, w.obs_dims, S)
            free = not v.all()
            false_pt += free
            false_whole += free and bool(wh)
        n = len(k["cells"])
        out["%s_cells_dense_sampling" % name] = {
            "workload": w.name, "cells_sampled": n, "samples_per_cell": 200,
            "cells_whole_certified": int(np.sum(k["whole"])),
            "point_only_false_certify": int(false_pt),
            "point_only_false_certify_rate": float(false_pt) / max(n, 1),
            "whole_certified_with_free_sample": int(false_whole)}
    return out


def batched_line(ctx, n_traces=64, seed=1003):
    """64 independent traces (d in {4,5,6}, 256-8192 SVs, lambda in
    [0.03, 0.1]) in one mf_trace_batch call, on the mixed (tensor-core) and
    FP64 paths, against the same traces one mf_trace call at a time.
    Capacities come from one untimed mf_trace of each trace (x1.25)."""
    import torch
    from paper_2406_04795_gb300 import mf
    ws = W.config_batched(seed=seed, n_traces=n_traces)
    caps, E_tot = [], 0
    for w in ws:
        r = ctx.trace(w.sv, w.alpha, w.gamma, w.b, w.lam, w.offset, w.lo, w.hi, w.seeds,
                      precision=mf.MF_FP64, **W.shell_capacity(w))
        caps.append(dict(max_edges=int(r["n_edges"] * 1.25) + 4096,
                         max_vertices=int(r["n_vertices"] * 1.25) + 4096,
                         max_cells=int(r["n_cells"] * 1.25) + 4096))
        E_tot += r["n_edges"]
        del r
    torch.cuda.empty_cache()
    tuned = tune_on(ctx, ws, caps)
    out = {"traces": n_traces, "edges": E_tot, "autotune": tuned,
           "workload": "d in {4,5,6}, 256-8192 SVs log-uniform, lambda in [0.03, 0.1], 1-64 seeds"}
    for name, prec in (("mixed_bf16", mf.MF_MIXED_BF16), ("fp64", mf.MF_FP64)):
        ctx.trace_batch(ws, precisions=[prec] * n_traces, capacities=caps)  # untimed
        torch.cuda.synchronize()
        mf.mf_ctx_set_profiling(ctx.h, True)  # per-phase CUDA events of the batch
        t0 = time.perf_counter()
        got = ctx.trace_batch(ws, precisions=[prec] * n_traces, capacities=caps)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        # (the batch records its whole search graph under expand_vertices)
        phases = {("bfs_graph" if k == "expand_vertices" else k): round(v["ms"], 3)
                  for k, v in mf.mf_ctx_get_stats(ctx.h).items() if v["ms"] > 0}
        mf.mf_ctx_set_profiling(ctx.h, False)
        E = sum(g["n_edges"] for g in got)
        del got
        t0 = time.perf_counter()
        for w, c in zip(ws, caps):
            r = ctx.trace(w.sv, w.alpha, w.gamma, w.b, w.lam, w.offset, w.lo, w.hi, w.seeds,
                          precision=prec, **c)
            del r
        torch.cuda.synchronize()
        dt1 = time.perf_counter() - t0
        out[name] = {"simplices_per_s": E / dt, "ms": dt * 1e3,
                     "one_at_a_time_simplices_per_s": E / dt1, "one_at_a_time_ms": dt1 * 1e3,
                     "phase_ms": phases}
    out["tune"] = mf.mf_ctx_get_tune(ctx.h).as_dict()
    torch.cuda.empty_cache()
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = make_workload(args.config, 0, args.lam)
    for _ in range(args.warmup):
        pass
    vals = []
    t_all = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(w, budget_s=8.0))
    dt = time.perf_counter() - t_all
    v = statistics.median([x["value"] for x in vals])
    line = {"impl": "reference", "metric": "traced simplices/s", "value": v, "unit": "simplices/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "lambda": w.lam, "n_sv": int(w.sv.shape[0]),
                       "seeds": int(w.seeds.shape[0]), "precision": "fp64"},
            "cpu_baseline": dict(vals[-1], value=v),
            "e2e": {"value": v, "unit": "simplices/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_gb300(args):
    import torch
    import torch.distributed as dist
    from paper_2406_04795_gb300 import mf
    from paper_2406_04795_gb300.api import Context
    from paper_2406_04795_gb300.pipeline import Proof, host_inputs
    from paper_2406_04795_gb300.scaling import reduce_timing

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    w = make_workload(args.config, rank, args.lam)
    if args.precision == "fp64":
        w.precision = "fp64"
    elif args.precision in ("mixed", "mixed_fp32"):
        w.precision = args.precision
    ctx = Context(local, 0)
    proof = Proof(ctx, w)
    stream = torch.cuda.current_stream()
    tune = None
    if args.tune_json:
        # fixed launch choices (reproduces a tuned configuration, e.g. under ncu)
        t = mf.mf_ctx_get_tune(ctx.h)
        for k, v in json.loads(args.tune_json).items():
            setattr(t, k, int(v))
        mf.mf_ctx_set_tune(ctx.h, t)
        tune = mf.mf_ctx_get_tune(ctx.h).as_dict()
    elif not args.no_autotune:
        # untimed: launch variants and BFS chunk picked on this workload (one
        # proof first, so that its capacities have grown to fit)
        proof.step()
        sz = proof.sizing
        tune = ctx.autotune(w, precision=proof.precision, batch_cap=w.batch_cap,
                            max_edges=sz["max_edges"], max_vertices=sz["max_vertices"],
                            max_cells=sz["max_cells"], recheck_band=w.recheck_band)

    def barrier():
        if world > 1:
            dist.barrier()

    # measured roofline denominators (FP64 FMA, FP32 FMA, ex2, table exp)
    rates = mf.mf_probe_rates(ctx.h).as_dict()

    for _ in range(max(args.warmup, 0)):
        proof.step()
    torch.cuda.synchronize()
    mf.mf_ctx_set_profiling(ctx.h, True)
    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    edges = 0
    for _ in range(args.steps):
        r, v, m, cv = proof.step()
        edges += r["n_edges"]
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1) / max(args.steps, 1)
    stats = mf.mf_ctx_get_stats(ctx.h)
    mf.mf_ctx_set_profiling(ctx.h, False)
    E = r["n_edges"]
    launches = sum(s["launches"] for s in stats.values())

    # end to end: pinned host inputs copied in, verdicts read back, every step
    hin = host_inputs(w)
    verdict_host = torch.empty(E, dtype=torch.uint8).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in hin.values())
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_edges = 0
    for _ in range(args.steps):
        for name, t in hin.items():
            getattr(proof, name).copy_(t, non_blocking=True)
        r, v, m, cv = proof.step()
        n = r["n_edges"]
        if verdict_host.numel() < n:
            verdict_host = torch.empty(n, dtype=torch.uint8).pin_memory()
        verdict_host[:n].copy_(v, non_blocking=True)
        torch.cuda.synchronize()
        e2e_edges += n
    e2e_s = time.perf_counter() - t0
    barrier()

    ms_max, edges_all, e2e_max, e2e_edges_all = reduce_timing(ms, edges, e2e_s, e2e_edges, world,
                                                              "cuda")
    if rank == 0:
        value = edges_all / args.steps / (ms_max * 1e-3)
        line = {
            "metric": "traced simplices/s", "value": value, "unit": "simplices/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp64": "f64", "mixed_fp32": "f32+f64"}.get(w.precision, "bf16+f32+f64"),
            "data": "synthetic",
            "config": {"workload": w.name, "d": w.d, "lambda": w.lam,
                       "n_sv": int(w.sv.shape[0]), "gamma": w.gamma,
                       "seeds": int(w.seeds.shape[0]), "batch_cap": w.batch_cap,
                       "precision": w.precision, "edges_per_proof": E,
                       "cells_per_proof": r["n_cells"], "vertices_per_proof": r["n_vertices"],
                       "bfs_levels": r["levels"], "ms_per_proof": ms_max,
                       "cells_points_in_collision": int(cv.sum().item()) if r["n_cells"] else 0,
                       "cells_whole_certified": int(proof.whole.sum().item())
                       if r["n_cells"] and proof.whole is not None else 0,
                       "autotune": tune,
                       "l2": "inputs larger than L2 (resident hash tables and lists are GBs)"},
            "e2e": {"value": e2e_edges_all / args.steps / (e2e_max / args.steps),
                    "unit": "simplices/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": E,
                    "note": "inputs (support vectors, seeds, robot, scene) copied in and the "
                            "per-point verdicts read back every step; the traced set stays "
                            "resident on the device, as the paper returns only C_free points"},
            "gpu_launches": launches,
            "clocks": clocks,
            "roofline": roofline(stats, w, rates, E, ms_max, args.steps),
        }
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(w, E_proof=E)
        if world == 1 and not args.no_extras:
            # the same proof on the other precision (mixed: distance GEMM on
            # the tensor cores, FP64 recheck, roots to 1e-6)
            wm = make_workload(args.config, rank, args.lam)
            wm.precision = "mixed" if w.precision == "fp64" else "fp64"
            st_m = {}
            msm, pm, rm = _proof_ms(ctx, wm, stats=st_m)
            line["other_precision"] = {"precision": wm.precision, "ms_per_proof": msm,
                                       "value": rm["n_edges"] / (msm * 1e-3),
                                       "edges_per_proof": rm["n_edges"],
                                       "rechecked_vertices": rm["n_recheck"],
                                       "roofline": roofline(st_m, wm, rates, rm["n_edges"], msm, 2,
                                                            root_traffic=False)}
            if wm.precision == "mixed":
                line["other_precision"]["eval_roofline"] = eval_tc_roofline(st_m, rates)
            del pm, rm
            # the server gets a context of its own: the proofs' resident tables
            # and outputs are released first, so that its arena can hold many
            # requests
            keep_main = sample_cells(w, r, cv, proof.whole)
            del proof, r, v, m, cv
            ctx.close()
            torch.cuda.empty_cache()
            ctx = Context(local, 0)
            line["configs"], keep = config_lines(ctx)
            keep["main"] = keep_main
            if "cpu_baseline" in line:
                line["cpu_baseline"].update(oracle_checks(keep))
            ctx.close()
            torch.cuda.empty_cache()
            ctx = Context(local, 0)
            line["batched"] = batched_line(ctx)
            ctx.close()
            torch.cuda.empty_cache()
            ctx = Context(local, 0)
            line["served"] = served_lines(ctx, args.served_requests, args.served_rate)
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--config", default="d5", choices=["d3", "d5", "d6"])
    ap.add_argument("--precision", default="auto", choices=["auto", "fp64", "mixed", "mixed_fp32"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    ap.add_argument("--tune-json", default="",
                    help="fixed launch choices instead of autotuning, e.g. '{\"roots_variant\": 1}'")
    ap.add_argument("--lam", type=float, default=None,
                    help="override the lattice scale (small profiling cases)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other-precision proof and the served run")
    ap.add_argument("--served-requests", type=int, default=2000)
    ap.add_argument("--served-rate", type=float, default=50.0)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gb300(args)


if __name__ == "__main__":
    main()
