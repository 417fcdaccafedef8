"""The measured roofline denominators and the FP64 exp of the RBF terms.

mf_probe_rates: the probe rates are positive and ordered as the hardware
orders the pipes (FP32 FMA above FP64 FMA; the table-driven FP64 exp, about
a dozen FP64-pipe instructions, below the FP64 FMA rate).

mf_diag_exp: the table-driven FP64 exp (Tang's method) against CUDA's exp()
over [-708, 0], the argument range of the RBF terms.  Measured on the host
in units in the last place of the library value; the kernels' FP64 parity
budget (1e-12 on f) needs far less than the bound asserted here."""
import math

import numpy as np
import pytest
import torch

from paper_2406_04795_gb300 import mf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2406_04795_gb300.api import Context
    c = Context(0, 1 << 30)
    yield c
    c.close()


def test_probe_rates_are_ordered(ctx):
    r = mf.mf_probe_rates(ctx.h).as_dict()
    for k in ("fp64_fma_per_s", "fp32_fma_per_s", "ex2_per_s", "exp_neg_per_s"):
        assert r[k] > 0
    assert r["fp32_fma_per_s"] > 8 * r["fp64_fma_per_s"]
    assert r["exp_neg_per_s"] < r["fp64_fma_per_s"]
    assert r["sm_count"] > 0


def _ulp(a):
    return np.spacing(np.abs(a))


def test_table_exp_against_cuda_exp(ctx):
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.uniform(-708.0, 0.0, 200_000), rng.uniform(-1.0, 0.0, 50_000),
                        -np.arange(0, 708, 0.5), [0.0, -1e-300, -708.0]])
    # arguments at the reduction boundaries k ln2/64 and just beside them
    k = np.arange(0, 708 * 64 / math.log(2), 7.0)
    b = -k * math.log(2) / 64
    x = np.concatenate([x, b, np.nextafter(b, 1.0), np.nextafter(b, -1.0)])
    x = x[(x >= -708.0) & (x <= 0.0)]
    xd = torch.as_tensor(x, device="cuda")
    yt = torch.empty_like(xd)
    yl = torch.empty_like(xd)
    mf.mf_diag_exp(ctx.h, xd.data_ptr(), xd.numel(), yt.data_ptr(), yl.data_ptr(),
                   torch.cuda.current_stream().cuda_stream)
    yt, yl = yt.cpu().numpy(), yl.cpu().numpy()
    err = np.abs(yt - yl) / _ulp(yl)
    assert np.all(np.isfinite(yt)) and np.all(yt > 0)
    assert float(err.max()) <= 4.0, float(err.max())
    # relative error against numpy's exp (an independent libm)
    rel = np.abs(yt - np.exp(x)) / np.exp(x)
    assert float(rel.max()) <= 1e-15
