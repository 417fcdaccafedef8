"""The benchmark's roofline arithmetic on synthetic phase counters: the
dominant phase is chosen by time, achieved = the phase's counted work per
launch over its time per launch, frac = achieved / peak, and the proof-level
bound is the largest of its four per-resource times."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2406_04795_gb300 import mf  # noqa: E402
from paper_2406_04795_gb300 import workloads as W  # noqa: E402


def _stats(**over):
    st = {k: dict(ms=0.0, launches=0, units=0, terms=0, terms_weak=0) for k in mf.PHASE_NAMES}
    for k, v in over.items():
        st[k].update(v)
    return st


RATES = {"fp64_fma_per_s": 5e11, "fp32_fma_per_s": 4e13, "ex2_per_s": 1e13,
         "exp_neg_per_s": 4e10, "sm_count": 152, "sm_clock_mhz": 2070.0}


def test_roots_dominant_roofline():
    w = W.config_d5()
    st = _stats(roots=dict(ms=600.0, launches=2, units=1000, terms=10 ** 9, terms_weak=4 * 10 ** 9),
                eval=dict(ms=100.0, launches=2, units=100, terms=10 ** 8, terms_weak=10 ** 9),
                cells=dict(ms=50.0, launches=2, units=1000))
    r = bench.roofline(st, w, RATES, E=1000, ms_proof=900.0, n_proofs=2)
    d = w.d
    ops = (10 ** 9 * bench.df_term_ops(d) + 4 * 10 ** 9 * bench.f32_term_ops(d)) / 2
    assert r["bound"] == "alu" and r["unit"] == "T FP32 ops/s"
    assert r["achieved"] == pytest.approx(ops / 0.3 / 1e12)
    assert r["peak"] == pytest.approx(40.0)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    p = r["proof"]
    assert p["ns_per_edge"] == pytest.approx(900.0 * 1e6 / 1000)
    assert p["frac"] == pytest.approx(max(p["fp64_ms"], p["fp32_ms"], p["ex2_ms"], p["hbm_ms"])
                                      / 900.0)
    assert p["bound_by"] in ("fp64", "fp32", "ex2", "hbm")


def test_table_phase_roofline_uses_hbm():
    w = W.config_d5()
    st = _stats(cells=dict(ms=500.0, launches=1, units=10 ** 6),
                roots=dict(ms=10.0, launches=1, units=10))
    r = bench.roofline(st, w, RATES, E=10 ** 6, ms_proof=600.0, n_proofs=1)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["kernel"] == "cells"
    k = w.d // 2
    per = (4 * w.d + 4) + 32 * (2 ** k + 2 ** (w.d - k + 1))
    assert r["achieved"] == pytest.approx(10 ** 6 * per / 0.5 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
