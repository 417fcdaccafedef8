"""Proof server (continuous batching): requests that arrive while others are
running are admitted as slots and memory free up, and each result is the
same in the mix as alone (mf_trace)."""
import numpy as np
import pytest

from paper_2406_04795_gb300 import mf
from paper_2406_04795_gb300 import workloads as W
from tests.test_gpu_batch import _np, _same

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2406_04795_gb300.api import Context
    c = Context(0, 64 << 30)
    yield c
    c.close()


def test_server_results_equal_alone_under_queueing(ctx):
    ws = W.config_batched(n_traces=5, lam_scale=3.0) + [W.config_d3()]
    ws += W.config_batched(seed=77, n_traces=3, lam_scale=3.5)
    precs = [(mf.MF_MIXED_FP32, mf.MF_FP64, mf.MF_MIXED_BF16)[i % 3] for i in range(len(ws))]
    server = ctx.server(max_slots=3, hbm_bytes=24 << 30)
    ids, got, saw_queue, steps = [], {}, False, 0
    pending = list(range(len(ws)))
    while pending or len(got) < len(ids):
        # four requests at once (one more than the slots), then two every
        # other step while earlier ones run
        if pending and steps % 2 == 0:
            for _ in range(4 if steps == 0 else 2):
                if pending:
                    k = pending.pop(0)
                    ids.append(server.submit(ws[k], precision=precs[k], **W.shell_capacity(ws[k])))
        running, queued = server.step()
        assert running <= 3
        saw_queue = saw_queue or queued > 0
        for rid in server.done():  # each finished request is reported once
            assert rid in ids and rid not in got
            state, t_sub, t_adm, t_done = server.status(rid)
            assert state == 2, "request %d failed: %d" % (rid, state)
            assert t_sub <= t_adm <= t_done
            got[rid] = server.fetch(rid)
        steps += 1
        assert steps < 20000
    assert saw_queue, "the slot limit should have queued requests"
    for k, rid in enumerate(ids):
        w = ws[k]
        alone = ctx.trace(w.sv, w.alpha, w.gamma, w.b, w.lam, w.offset, w.lo, w.hi, w.seeds,
                          precision=precs[k], **W.shell_capacity(w))
        assert got[rid]["n_edges"] > 10
        fp64 = precs[k] == mf.MF_FP64
        _same(_np(got[rid]), _np(alone), f_tol=1e-12 if fp64 else 1e-3,
              t_tol=1e-9 if fp64 else 2e-6)
    server.close()


def test_server_fetch_before_done_and_oversized(ctx):
    server = ctx.server(max_slots=2, hbm_bytes=2 << 30)
    w = W.config_d3()
    rid = server.submit(w, precision=mf.MF_FP64, max_edges=1 << 18)
    with pytest.raises(mf.MfError):
        server.fetch(rid)
    big = server.submit(w, precision=mf.MF_FP64, max_edges=1 << 28)  # cannot fit the budget
    for _ in range(1000):
        running, queued = server.step()
        if server.status(rid)[0] == 2 and server.status(big)[0] != 0:
            break
    assert server.status(big)[0] == mf.MF_ERR_OOM
    with pytest.raises(mf.MfError):
        server.fetch(big)
    assert server.fetch(rid)["n_edges"] > 1000
    server.close()


def test_server_wait_is_bounded(ctx):
    """mf_server_wait returns MF_ERR_TIMEOUT (the request still running) when
    the limit is too short, and the request's final state once it is done."""
    server = ctx.server(max_slots=2, hbm_bytes=4 << 30)
    w = W.config_d3()
    rid = server.submit(w, precision=mf.MF_FP64, max_edges=1 << 18)
    assert server.wait(rid, 0.0) is None  # no time at all: not done yet
    assert server.status(rid)[0] in (0, 1)
    state = server.wait(rid, 60_000.0)
    assert state == 2
    assert list(server.done()) == [rid]
    assert server.fetch(rid)["n_edges"] > 1000
    server.close()
