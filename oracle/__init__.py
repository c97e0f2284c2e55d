"""CPU oracle for the fit-objective gradients -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The CUDA
product path (``paper_2203_06139_gb300``) never imports it and shares no code
with it.

The arithmetic lives in ``cg_oracle.c``: a scalar tape-based reverse-mode AD
(Sec. 1-2 of the paper: reverse accumulation recorded on a tape, the
"tracing" approach) over the fit objectives of the histogram-fitting use case
(Sec. 4, Fig. 3).  This module compiles it with gcc (``-ffp-contract=off``)
and calls it through ctypes.  ctypes releases the GIL during the call, so
``many()`` evaluates independent parameter points on several host threads.

``cg_closed.c`` holds hand-written closed-form gradients (and a central
finite-difference gradient) of the mixture NLL and the 1-D chi2, parallel
with OpenMP: the CPU baselines timed beside the GPU kernels, and a second,
independent statement of the derivatives that the tape must reproduce.
"""
import ctypes
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cg_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libcg_oracle.so")

# objective codes of the oracle (its own numbering)
CHI2, POISSON, POISSON_BC = 0, 1, 2
OK, INVALID, DOMAIN = 0, 1, 2

_CLOSED_SRC = os.path.join(_HERE, "cg_closed.c")
_CLOSED_LIB = os.path.join(_HERE, "libcg_closed.so")

_lib = None
_closed = None


def _gcc(src, out, extra=()):
    stale = not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src)
    if stale:
        tmp = "%s.%d.tmp" % (out, os.getpid())
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", *extra,
                               "-shared", "-o", tmp, src, "-lm"])
        os.replace(tmp, out)
    return out


def build(force=False):
    """Compile cg_oracle.c into libcg_oracle.so next to it (plain gcc, no FMA
    contraction), and the closed-form CPU gradients cg_closed.c (OpenMP)."""
    if force:
        for f in (_LIB_PATH, _CLOSED_LIB):
            if os.path.exists(f):
                os.utime(f, (0, 0))
    _gcc(_CLOSED_SRC, _CLOSED_LIB, ("-fopenmp",))
    return _gcc(_SRC, _LIB_PATH)


def _load():
    global _lib
    if _lib is not None:
        return _lib
    # CG_ORACLE_LIB: load a library built elsewhere (the mutation tests build
    # copies of cg_oracle.c with planted mistakes and point this at them)
    override = os.environ.get("CG_ORACLE_LIB")
    lib = ctypes.CDLL(override if override else build())
    dp = ctypes.POINTER(ctypes.c_double)
    i64, c_int, c_d = ctypes.c_int64, ctypes.c_int, ctypes.c_double
    lib.orc_binned1d.argtypes = [c_int, c_int, c_int, c_int, i64, c_d, c_d, dp, dp, dp, dp, dp, dp]
    lib.orc_binned1d_gn.argtypes = [c_int, c_int, c_int, c_int, i64, c_d, c_d, dp, dp, dp, dp]
    lib.orc_binned1d_gnmat.argtypes = [c_int, c_int, c_int, c_int, i64, c_d, c_d, dp, dp, dp, dp]
    lib.orc_gauss_poly_eval.argtypes = [c_int, c_int, c_int, c_d, c_d, i64, dp, dp, dp]
    lib.orc_unbinned_mix.argtypes = [i64, dp, dp, c_d, c_d, dp, dp, dp, dp]
    lib.orc_binned2d.argtypes = [c_int, i64, i64, c_d, c_d, c_d, c_d, dp, dp, dp, dp, dp]
    lib.orc_listing1_gauss.argtypes = [c_d, c_d, c_d, dp, dp, dp]
    ip = ctypes.POINTER(ctypes.c_int32)
    lib.orc_expr.argtypes = [c_int, ip, ip, ip, ip, dp, c_int, c_int, ctypes.POINTER(dp), i64, dp, dp, dp, dp]
    lib.orc_expr.restype = c_int
    for f in (lib.orc_binned1d, lib.orc_binned1d_gn, lib.orc_binned1d_gnmat, lib.orc_gauss_poly_eval,
              lib.orc_unbinned_mix, lib.orc_binned2d, lib.orc_listing1_gauss):
        f.restype = c_int
    _lib = lib
    return lib


def _p(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


class Result:
    """Objective value, gradient, per-component scale S_k = sum_i |dT_i/dtheta_k|, status."""

    def __init__(self, value, grad, scale, rc):
        self.value, self.grad, self.scale, self.rc = value, grad, scale, rc

    def __repr__(self):
        return "Result(value=%r, grad=%r, rc=%d)" % (self.value, self.grad, self.rc)


def num_params_gauss_poly(K, D):
    return 3 * K + D + 1


def binned1d(K, D, poly_mode, obj, y, lo, hi, theta, centres=None):
    """1-D binned objective of K Gaussian peaks + degree-D polynomial (see cg_oracle.c)."""
    lib = _load()
    y = _f64(y)
    theta = _f64(theta)
    centres = _f64(centres)
    P = 3 * K + D + 1
    assert theta.shape == (P,)
    g = np.zeros(P)
    s = np.zeros(P)
    v = ctypes.c_double(0.0)
    rc = lib.orc_binned1d(K, D, poly_mode, obj, y.size, lo, hi, _p(centres), _p(y), _p(theta),
                          ctypes.byref(v), _p(g), _p(s))
    return Result(v.value, g, s, rc)


def binned1d_gn(K, D, poly_mode, obj, y, lo, hi, theta, centres=None):
    """Gauss-Newton diagonal sum_i h_i (df_i/dtheta_k)^2 of a 1-D binned objective."""
    lib = _load()
    y = _f64(y)
    theta = _f64(theta)
    centres = _f64(centres)
    gn = np.zeros(3 * K + D + 1)
    rc = lib.orc_binned1d_gn(K, D, poly_mode, obj, y.size, lo, hi, _p(centres), _p(y), _p(theta),
                             _p(gn))
    assert rc == OK
    return gn


def binned1d_gnmat(K, D, poly_mode, obj, y, lo, hi, theta, centres=None):
    """Gauss-Newton matrix sum_i h_i (df_i/dtheta_a)(df_i/dtheta_b) [P, P]."""
    lib = _load()
    y = _f64(y)
    theta = _f64(theta)
    centres = _f64(centres)
    P = 3 * K + D + 1
    gn = np.zeros((P, P))
    rc = lib.orc_binned1d_gnmat(K, D, poly_mode, obj, y.size, lo, hi, _p(centres), _p(y), _p(theta), _p(gn))
    assert rc == OK
    return gn


def gauss_poly_eval(K, D, poly_mode, lo, hi, x, theta):
    """Model value f(x) of the 1-D family at points x."""
    lib = _load()
    x = _f64(x)
    theta = _f64(theta)
    out = np.zeros(x.size)
    rc = lib.orc_gauss_poly_eval(K, D, poly_mode, lo, hi, x.size, _p(x), _p(theta), _p(out))
    assert rc == OK
    return out


def unbinned_mix(x, lo, hi, theta, weights=None):
    """Unbinned NLL of the Gaussian + exponential mixture, theta = (frac, mu, s, lambda)."""
    lib = _load()
    x = _f64(x)
    theta = _f64(theta)
    weights = _f64(weights)
    g = np.zeros(4)
    s = np.zeros(4)
    v = ctypes.c_double(0.0)
    rc = lib.orc_unbinned_mix(x.size, _p(x), _p(weights), lo, hi, _p(theta), ctypes.byref(v),
                              _p(g), _p(s))
    return Result(v.value, g, s, rc)


def binned2d(K, counts, lx, hx, ly, hy, theta):
    """2-D binned Poisson NLL of K rotated Gaussians + constant; counts has shape (ny, nx)."""
    lib = _load()
    counts = _f64(counts)
    ny, nx = counts.shape
    theta = _f64(theta)
    P = 6 * K + 1
    g = np.zeros(P)
    s = np.zeros(P)
    v = ctypes.c_double(0.0)
    rc = lib.orc_binned2d(K, nx, ny, lx, hx, ly, hy, _p(counts), _p(theta), ctypes.byref(v),
                          _p(g), _p(s))
    return Result(v.value, g, s, rc)


def listing1_gauss(x, p, sigma):
    """The Gaussian of Listing 1 and its derivatives with respect to x and p."""
    lib = _load()
    v, dx, dp = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    rc = lib.orc_listing1_gauss(x, p, sigma, ctypes.byref(v), ctypes.byref(dx), ctypes.byref(dp))
    assert rc == OK
    return v.value, dx.value, dp.value


def _load_closed():
    global _closed
    if _closed is not None:
        return _closed
    build()
    lib = ctypes.CDLL(_CLOSED_LIB)
    dp = ctypes.POINTER(ctypes.c_double)
    i64, c_int, c_d = ctypes.c_int64, ctypes.c_int, ctypes.c_double
    lib.clf_mix.argtypes = [i64, dp, c_d, c_d, dp, dp, dp, c_int]
    lib.clf_mix_fd.argtypes = [i64, dp, c_d, c_d, dp, dp, c_int]
    lib.clf_gauss_poly_chi2.argtypes = [c_int, c_int, c_int, i64, c_d, c_d, dp, dp, dp, dp, c_int]
    for f in (lib.clf_mix, lib.clf_mix_fd, lib.clf_gauss_poly_chi2):
        f.restype = c_int
    _closed = lib
    return lib


def closed_mix(x, lo, hi, theta, grad=True, threads=0):
    """Mixture NLL and its hand-written gradient (cg_closed.c, OpenMP; threads 0 = all)."""
    lib = _load_closed()
    x, theta = _f64(x), _f64(theta)
    g = np.zeros(4) if grad else None
    v = ctypes.c_double(0.0)
    rc = lib.clf_mix(x.size, _p(x), lo, hi, _p(theta), ctypes.byref(v), _p(g), threads)
    assert rc == 0
    return v.value, g


def closed_mix_fd(x, lo, hi, theta, threads=0):
    """Central-difference gradient of the mixture NLL from 8 value-only evaluations."""
    lib = _load_closed()
    x, theta = _f64(x), _f64(theta)
    g = np.zeros(4)
    assert lib.clf_mix_fd(x.size, _p(x), lo, hi, _p(theta), _p(g), threads) == 0
    return g


def closed_gauss_poly_chi2(K, D, poly_mode, y, lo, hi, theta, grad=True, threads=0):
    """chi2 of K Gaussians + degree-D polynomial and its hand-written gradient."""
    lib = _load_closed()
    y, theta = _f64(y), _f64(theta)
    g = np.zeros(3 * K + D + 1) if grad else None
    v = ctypes.c_double(0.0)
    rc = lib.clf_gauss_poly_chi2(K, D, poly_mode, y.size, lo, hi, _p(y), _p(theta), ctypes.byref(v), _p(g),
                                 threads)
    assert rc == 0
    return v.value, g


def expr(nodes, n_params, inputs, theta, n=None):
    """Objective and gradient of an expression program (nodes: rows of
    (op, a, b, i, c), topological order, last = per-element term; the
    operations are listed at orc_expr in cg_oracle.c)."""
    lib = _load()
    nodes = list(nodes)
    op = np.ascontiguousarray([r[0] for r in nodes], dtype=np.int32)
    na = np.ascontiguousarray([r[1] for r in nodes], dtype=np.int32)
    nb = np.ascontiguousarray([r[2] for r in nodes], dtype=np.int32)
    ni = np.ascontiguousarray([r[3] for r in nodes], dtype=np.int32)
    nc = np.ascontiguousarray([r[4] for r in nodes], dtype=np.float64)
    ins = [_f64(x) for x in inputs]
    if n is None:
        n = ins[0].size if ins else 0
    dp = ctypes.POINTER(ctypes.c_double)
    arr = (dp * max(1, len(ins)))(*[_p(x) for x in ins])
    ip = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    theta = _f64(theta)
    g = np.zeros(max(n_params, 1))
    s = np.zeros(max(n_params, 1))
    v = ctypes.c_double(0.0)
    rc = lib.orc_expr(len(nodes), ip(op), ip(na), ip(nb), ip(ni), _p(nc), n_params, len(ins), arr, n, _p(theta),
                      ctypes.byref(v), _p(g), _p(s))
    return Result(v.value, g[:n_params], s[:n_params], rc)


def many(fn, thetas, threads=None, **kw):
    """Evaluate fn(theta=t, **kw) for every row of thetas on a pool of host threads."""
    thetas = np.asarray(thetas, dtype=np.float64)
    threads = threads or os.cpu_count() or 1
    with ThreadPoolExecutor(max_workers=threads) as ex:
        return list(ex.map(lambda t: fn(theta=t, **kw), list(thetas)))
