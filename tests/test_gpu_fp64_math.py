"""The FP64 elementary functions of the fused FP64 kernels (cg_fp64.cuh)
against the CUDA math library and IEEE division on the GPU.

exp2 (table-driven, Tang 1989) within 1 ulp of CUDA's exp2, the same
special values (overflow, underflow, subnormal results, NaN); the
reciprocal within 1 ulp of the correctly rounded quotient; log (table
driven, Tang 1990) within 3 ulp of CUDA's log (the two are within 1.9 and
1 ulp of the exact value), next to 1 as well; the running-product sum of
logs within its error bound of an exact sum of correctly rounded logs;
exp2 of an exact product (the product folded into the reduction) within 1
ulp of the correctly rounded 2^(a b), with no error from rounding a b.
"""
import ctypes
import math
import os
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def helper(tmp_path_factory):
    import torch
    assert torch.cuda.is_available()
    so = str(tmp_path_factory.mktemp("fp64") / "libfp64check.so")
    src = os.path.join(HERE, "cuda", "fp64_math_check.cu")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-Xcompiler",
                    "-fPIC", "-shared", "-cudart", "shared", "-o", so, src], check=True)
    L = ctypes.CDLL(so)
    L.fp64_check.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    L.fp64_logprod.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    L.fp64_exp2_prod.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    return L, torch


def _ulps(a, b):
    """|a - b| in units in the last place, through the ordered integer images
    of the doubles (negative doubles mapped below zero)."""
    def line(v):
        i = np.ascontiguousarray(v, dtype=np.float64).view(np.int64)
        return np.where(i < 0, -(i & 0x7fffffffffffffff), i)
    return np.abs(line(a) - line(b))


def _run(helper, y, p):
    L, torch = helper
    n = len(y)
    yd = torch.tensor(y, device="cuda")
    pd = torch.tensor(p, device="cuda")
    out = torch.empty(n * 6, dtype=torch.float64, device="cuda")
    assert L.fp64_check(ctypes.c_void_p(yd.data_ptr()), ctypes.c_void_p(pd.data_ptr()), n,
                        ctypes.c_void_p(out.data_ptr())) == 0
    return out.cpu().numpy().reshape(n, 6)


def test_exp2_reciprocal_log_against_cuda(helper):
    rng = np.random.default_rng(2203)
    n = 1 << 18
    y = np.concatenate([rng.uniform(-1080, 1030, n // 4), rng.uniform(-20, 20, n // 4),
                        rng.uniform(-1e-3, 1e-3, n // 4), -rng.uniform(0, 40, n // 4)])
    # positive values over the whole normal range, random fractions, plus values next to 1
    p = np.ldexp(1.0 + rng.random(n), rng.integers(-1021, 1021, n))
    p[: n // 8] = 1.0 + rng.uniform(-1e-2, 1e-2, n // 8)
    o = _run(helper, y, p)
    fin = np.isfinite(o[:, 1]) & (o[:, 1] > 0)
    assert np.array_equal(np.isnan(o[:, 0]), np.isnan(o[:, 1]))
    assert np.array_equal(o[~fin, 0], o[~fin, 1])                 # 0 and inf where CUDA gives them
    assert _ulps(o[fin, 0], o[fin, 1]).max() <= 1                  # exp2
    assert _ulps(o[:, 2], o[:, 3]).max() <= 1                      # reciprocal vs correctly rounded
    nz = o[:, 5] != 0.0
    assert np.all(o[~nz, 4] == 0.0)                                # log 1 = 0 exactly
    assert _ulps(o[nz, 4], o[nz, 5]).max() <= 3                    # log, p = 1 +- 1e-2 included


def test_exp2_special_values(helper):
    y = np.array([0.0, -0.0, 1.0, -1.0, 1023.5, 1024.0, 1024.5, -1022.0, -1021.99995, -1074.0, -1074.5,
                  -1075.0, -1100.0, -1e300, 1e300, np.inf, -np.inf, np.nan, 2.0 ** -13, -(2.0 ** -13)])
    p = np.ones_like(y)
    o = _run(helper, y, p)
    e = o[:, 1]
    assert np.array_equal(np.isnan(o[:, 0]), np.isnan(e))
    ok = ~np.isnan(e)
    assert np.all((o[ok, 0] == e[ok]) | (_ulps(o[ok, 0], e[ok]) <= 1))
    assert o[0, 0] == 1.0 and o[1, 0] == 1.0 and o[2, 0] == 2.0 and o[3, 0] == 0.5
    assert o[5, 0] == np.inf and o[11, 0] == 0.0 and o[10, 0] == 5e-324 and o[16, 0] == 0.0


def test_reciprocal_and_log_outside_the_fast_range(helper):
    p = np.array([0.0, -0.0, -2.0, 5e-324, 1e-310, 2.0 ** 1022, 1e308, np.inf, np.nan, 1.0])
    o = _run(helper, np.zeros_like(p), p)
    for k in range(len(p)):
        for a, b in ((o[k, 2], o[k, 3]), (o[k, 4], o[k, 5])):
            assert (np.isnan(a) and np.isnan(b)) or a == b or abs(a - b) <= 2 * np.spacing(abs(b))


def test_running_product_sum_of_logs(helper):
    L, torch = helper
    rng = np.random.default_rng(7)
    groups = 4096
    p = np.ldexp(1.0 + rng.random(groups * 64), rng.integers(-60, 40, groups * 64))
    pd = torch.tensor(p, device="cuda")
    out = torch.empty(groups, dtype=torch.float64, device="cuda")
    assert L.fp64_logprod(ctypes.c_void_p(pd.data_ptr()), groups, ctypes.c_void_p(out.data_ptr())) == 0
    got = out.cpu().numpy()
    lg = np.log(p).reshape(groups, 64)                         # each within 1 ulp
    ref = np.array([math.fsum(r) for r in lg])                 # exact sums of those
    # 64 products at 2^-53 each, the logs' own ulps, the final rounding
    bound = 64 * 2.0 ** -53 + np.abs(lg).sum(1) * 2.0 ** -52 + 2 * np.spacing(np.abs(ref))
    assert np.all(np.abs(got - ref) <= bound)


def _exp2_prod(helper, a, b):
    L, torch = helper
    ad, bd = torch.tensor(a, device="cuda"), torch.tensor(b, device="cuda")
    out = torch.empty(2 * len(a), dtype=torch.float64, device="cuda")
    assert L.fp64_exp2_prod(ctypes.c_void_p(ad.data_ptr()), ctypes.c_void_p(bd.data_ptr()), len(a),
                            ctypes.c_void_p(out.data_ptr())) == 0
    return out.cpu().numpy().reshape(-1, 2)


def test_exp2_of_an_exact_product(helper):
    """2^(a b) from the exact product: against 2^(a b) to 40 digits (the
    product exact in rationals), within 1 ulp, over exponents of -1000 to
    1000 and the narrow-peak form a = c2 d, b = d; CUDA's exp2 of the
    rounded product is off by up to |a b| 2^-53 ln 2 relative in comparison."""
    import decimal
    from fractions import Fraction
    rng = np.random.default_rng(11)
    n = 3000
    d = rng.uniform(-3.0, 3.0, n)
    c2 = -rng.uniform(0.5, 110.0, n)
    a = np.concatenate([c2 * d, rng.uniform(-40.0, 40.0, n)])
    b = np.concatenate([d, rng.uniform(-25.0, 25.0, n)])
    o = _exp2_prod(helper, a, b)
    ctx = decimal.Context(prec=40)
    ln2 = ctx.ln(decimal.Decimal(2))
    ref = np.empty(len(a))
    for i in range(len(a)):
        q = Fraction(float(a[i])) * Fraction(float(b[i]))
        y = ctx.divide(decimal.Decimal(q.numerator), decimal.Decimal(q.denominator))
        ref[i] = float(ctx.exp(ctx.multiply(y, ln2)))
    ok = np.abs(a * b) < 1000
    assert ok.sum() > 5000
    assert _ulps(o[ok, 0], ref[ok]).max() <= 1
    # the rounded product costs CUDA's exp2 more than that for large exponents
    assert _ulps(o[ok, 1], ref[ok]).max() > 1


def test_exp2_of_a_product_outside_the_fast_range(helper):
    """|a b| >= 1022, infinities and NaN: the same values as exp2 of the
    rounded product (overflow to infinity, subnormal results, zero), also
    through the integer early exit for |a| |b| >= 2^11."""
    a = np.array([1024.0, 2.0, -1075.0, -1.0, 1e300, -1e300, np.inf, np.nan, 0.0, 1022.0, -1021.9999, 3.0,
                  -3000.0, 50.0, 2000.0, -1.5, -np.inf, 1e-310, -2048.0, 1023.9, -1100.0, -33.0, 4.9e-324])
    b = np.array([1.0, 511.25, 1.0, 1074.5, 1e10, 1e10, 1.0, 1.0, np.inf, 1.0, 1.0, -340.7,
                  1.0, -50.0, 2.0, 1400.0, 2.0, 1e300, 1.0, -1.0, 1.0, 33.0, 1.7e308])
    o = _exp2_prod(helper, a, b)
    for k in range(len(a)):
        x, e = o[k, 0], o[k, 1]
        assert (np.isnan(x) and np.isnan(e)) or x == e or _ulps(np.array([x]), np.array([e]))[0] <= 1, (a[k], b[k], x, e)
