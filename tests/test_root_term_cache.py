"""The root solve's term cache: with u = x1 - s from FP32 hi/lo differences,
A = |u|^2 and Bp = u . dir (dir rounded to FP32), an evaluation at t takes
proj = Bp + t |dir|^2 and r2 = A + t (Bp + proj) in FP32.  The kernel bounds
the exponent's error of such a term by (d + 8) 2^-24 gamma (r + 2 |dir|)^2
(r the distance from the support vector to x(t)); this test restates the
FP32 operations on the host (float32 rounding after each FMA, the products
exact in float64) and checks gamma |r2~ - r2| against that bound on random
vertices, directions and support vectors at the workloads' scales."""
import numpy as np

F32 = np.float32


def _fma(a, b, c):
    return F32(np.float64(a) * np.float64(b) + np.float64(c))


def _split(v):
    hi = np.float32(v)
    return hi, np.float32(v - np.float64(hi))


def test_cached_r2_error_within_bound():
    rng = np.random.default_rng(31)
    u24 = 2.0 ** -24
    worst = 0.0
    for _ in range(20000):
        d = int(rng.integers(2, 9))
        gamma = float(rng.uniform(1.0, 12.0))
        lam = float(rng.uniform(0.02, 0.2))
        x1 = rng.uniform(-np.pi, np.pi, d)
        dirv = rng.normal(size=d)
        dirv *= lam / np.linalg.norm(dirv)
        s = x1 + rng.normal(size=d) * rng.uniform(0.001, 3.5) / np.sqrt(d)
        t = float(np.float32(rng.uniform(0, 1)))
        dir32 = dirv.astype(np.float32)
        A = F32(0)
        Bp = F32(0)
        dd = F32(0)
        for k in range(d):
            xh, xl = _split(x1[k])
            sh, sl = _split(s[k])
            u = F32(F32(xh - sh) + F32(xl - sl))
            A = _fma(u, u, A)
            Bp = _fma(u, dir32[k], Bp)
            dd = _fma(dir32[k], dir32[k], dd)
        proj = _fma(t, dd, Bp)
        r2c = _fma(t, F32(proj + Bp), A)
        x = x1 + t * dirv
        r = float(np.linalg.norm(x - s))
        err = gamma * abs(float(r2c) - r * r)
        bound = (d + 8) * u24 * gamma * (r + 2 * np.linalg.norm(dirv)) ** 2
        assert err <= bound, (err, bound)
        worst = max(worst, err / bound)
    assert worst > 0.0
