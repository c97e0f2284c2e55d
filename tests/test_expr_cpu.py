"""Expression programs on the CPU: the node-list serialisation, the host-side
validation of cg_expr_compile, and the oracle's expression interpreter pinned
against its own hand-built models and against central differences."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2203_06139_gb300 import synth
from paper_2203_06139_gb300 import expr as E


def chi2_gauss_linear(lo, hi, n):
    """chi2 term of A exp(-(x-mu)^2/(2 s^2)) + c0 + c1 x, x from the element index."""
    x = lo + (E.index() + 0.5) * ((hi - lo) / n)
    y = E.inp(0)
    A, mu, s, c0, c1 = (E.param(k) for k in range(5))
    f = A * E.exp(-(x - mu) ** 2 / (2.0 * s ** 2)) + c0 + c1 * x
    return (y - f) ** 2 / E.maximum(y, 1.0)


def mixture_nll(lo, hi):
    """-log p(x) of the Gaussian + exponential mixture, each component
    normalised on [lo, hi] (erfc for the Gaussian's integral)."""
    x = E.inp(0)
    f, mu, s, lam = (E.param(k) for k in range(4))
    phi = lambda z: 0.5 * E.erfc(-z / np.sqrt(2.0))
    ZG = phi((hi - mu) / s) - phi((lo - mu) / s)
    ZE = E.exp(-lam * lo) - E.exp(-lam * hi)
    G = E.exp(-(x - mu) ** 2 / (2.0 * s ** 2)) / (s * np.sqrt(2.0 * np.pi) * ZG)
    Ex = lam * E.exp(-lam * x) / ZE
    return -E.log(f * G + (1.0 - f) * Ex)


def test_node_list_of_a_small_expression():
    """(p0 * x + p0)^2, with p0 shared: operands first, shared nodes once."""
    p0, x = E.param(0), E.inp(0)
    nl = E.nodes((p0 * x + p0) ** 2)
    assert nl == [(E.PARAM, -1, -1, 0, 0.0), (E.INPUT, -1, -1, 0, 0.0), (E.MUL, 0, 1, 0, 0.0),
                  (E.ADD, 2, 0, 0, 0.0), (E.POWI, 3, -1, 2, 0.0)]


def test_oracle_expression_chi2_equals_its_hand_built_tape():
    p = synth.c1_histogram()
    th = synth.c1_theta_points(3)
    nl = E.nodes(chi2_gauss_linear(0.0, 10.0, 10000))
    for t in th:
        r = oracle.expr(nl, 5, [p["y"]], t)
        ref = oracle.binned1d(1, 1, 0, oracle.CHI2, p["y"], 0.0, 10.0, t)
        assert r.rc == oracle.OK
        assert abs(r.value - ref.value) <= 1e-13 * abs(ref.value)
        assert np.max(np.abs(r.grad - ref.grad) / np.maximum(np.abs(ref.grad), 1e-6 * ref.scale)) <= 1e-12


def test_oracle_expression_mixture_equals_its_hand_built_tape():
    x = synth.c2_events(20000)
    nl = E.nodes(mixture_nll(0.0, 10.0))
    for t in synth.c2_theta_points(3):
        r = oracle.expr(nl, 4, [x], t)
        ref = oracle.unbinned_mix(x, 0.0, 10.0, t)
        assert abs(r.value - ref.value) <= 1e-13 * abs(ref.value)
        assert np.max(np.abs(r.grad - ref.grad) / np.maximum(np.abs(ref.grad), 1e-6 * ref.scale)) <= 1e-12


def _odd_expression():
    """sqrt, negative power, max, division and the index together."""
    a, b, c = E.param(0), E.param(1), E.param(2)
    u, w = E.inp(0), E.inp(1)
    i = E.index()
    return E.sqrt(a * a + u * u) * (b + 0.01 * i) ** -2 + E.maximum(c * w, 0.5 * u) / (1.0 + c * c)


def test_oracle_expression_matches_central_differences():
    rng = np.random.default_rng(5)
    u, w = rng.uniform(0.5, 2.0, 500), rng.uniform(-1.0, 1.0, 500)
    nl = E.nodes(_odd_expression())
    t = np.array([0.7, 1.3, 0.4])
    r = oracle.expr(nl, 3, [u, w], t)
    assert r.rc == oracle.OK
    for k in range(3):
        h = 1e-6 * max(abs(t[k]), 1e-3)
        tp, tm = t.copy(), t.copy()
        tp[k] += h
        tm[k] -= h
        fd = (oracle.expr(nl, 3, [u, w], tp).value - oracle.expr(nl, 3, [u, w], tm).value) / (2 * h)
        assert abs(fd - r.grad[k]) <= 1e-6 * max(abs(r.grad[k]), 1e-3 * r.scale[k])


def _compile_rc(nl, n_params, n_inputs):
    lib = E._lib()
    arr = (E._Node * len(nl))(*[E._Node(*r) for r in nl])
    h = ctypes.c_void_p()
    return lib.cg_expr_compile(arr, len(nl), n_params, n_inputs, 0, ctypes.byref(h))


def test_compile_rejects_malformed_programs_on_the_host():
    from paper_2203_06139_gb300 import cg
    p0 = (E.PARAM, -1, -1, 0, 0.0)
    x = (E.INPUT, -1, -1, 0, 0.0)
    assert _compile_rc([p0, x, (E.MUL, 0, 3, 0, 0.0), (E.ADD, 0, 1, 0, 0.0)], 1, 1) == cg.ERR_INVALID_ARG  # forward ref
    assert _compile_rc([p0, (E.EXP, 0, -1, 0, 0.0)], 1, 0) == cg.ERR_INVALID_ARG       # no element dependence
    assert _compile_rc([(E.PARAM, -1, -1, 3, 0.0), x, (E.MUL, 0, 1, 0, 0.0)], 2, 1) == cg.ERR_INVALID_ARG
    assert _compile_rc([p0, (E.INPUT, -1, -1, 5, 0.0), (E.MUL, 0, 1, 0, 0.0)], 1, 1) == cg.ERR_INVALID_ARG
    assert _compile_rc([p0, x, (E.POWI, 1, -1, 40, 0.0)], 1, 1) == cg.ERR_INVALID_ARG
    assert _compile_rc([p0, x, (99, 0, 1, 0, 0.0)], 1, 1) == cg.ERR_INVALID_ARG


def test_generated_source_hoists_the_parameter_only_part():
    """The CUDA source written for the mixture: deterministic; the divisions
    by per-point values (2 s^2, the Gaussian's normalisation, Z_E) are products
    with reciprocals taken once per point, so the element loop takes a
    reciprocal only where the adjoint of the log needs 1/p, and its
    exponentials, logarithm and reciprocal are the table-driven FP64
    functions of cg_fp64.cuh (CUDA's stay in the per-point prologue)."""
    src = E.generated_source(mixture_nll(0.0, 10.0), 4, 1)
    assert src == E.generated_source(mixture_nll(0.0, 10.0), 4, 1)
    assert "extern \"C\" __global__ void __launch_bounds__(256) cgx_tiles" in src
    assert "cgx_finalize" in src
    assert '#include "cg_fp64.cuh"' in src and "__shared__ cg::Fp64Tab tab;" in src
    loop = src[src.index("for (i64 e = e0"):src.index("for (int k = 0; k < NACC; ++k) {\n      const double w")]
    assert loop.count(" / ") == 0 and loop.count("cg::frcp_any(") == 1 and loop.count(" * r") >= 3
    assert loop.count("cg::fexp(") == 2 and loop.count("cg::flog(") == 1
    assert "exp(" not in loop.replace("cg::fexp(", "") and "log(" not in loop.replace("cg::flog(", "")
    assert "#define NACC 9" in src


def test_value_only_source_has_no_reverse_sweep():
    full = E.generated_source(mixture_nll(0.0, 10.0), 4, 1)
    vo = E.generated_source(mixture_nll(0.0, 10.0), 4, 1, value_only=True)
    assert "#define NACC 1" in vo and " g" not in vo.split("cgx_finalize")[0].split("acc[0] +=")[1]
    assert "grad[" in full and "grad[" not in vo



def test_accumulator_limit_on_the_host():
    """Up to 127 frontier adjoints (+ the value) per thread: the 32-peak
    program (99 accumulators), 126 and 127 frontier nodes (127 and 128
    accumulators) get their source; 128 frontier nodes are refused by the
    host-side validation (no handle, no source)."""
    import pytest
    from paper_2203_06139_gb300 import cg
    K, n = 32, 100
    x = (E.index() + 0.5) * (1.0 / n)
    f = E.param(3 * K) + E.param(3 * K + 1) * x
    for k in range(K):
        f = f + E.param(3 * k) * E.exp(-(x - E.param(3 * k + 1)) ** 2 / (2.0 * E.param(3 * k + 2) ** 2))
    src = E.generated_source((E.inp(0) - f) ** 2, 3 * K + 2, 1)
    assert "#define NACC 99" in src
    def two_per_param(m):   # p_k and p_k^2 both multiply the element: 2m frontier nodes
        e = E.const(0.0)
        for k in range(m):
            e = e + E.param(k) * E.inp(0) + (E.param(k) * E.param(k)) * E.index()
        return e
    assert "#define NACC 127" in E.generated_source(two_per_param(63), 63, 1)
    # the boundary itself: 127 frontier nodes (NACC 128) are accepted, 128 refused
    odd = two_per_param(63) + E.param(63) * E.inp(0)
    assert "#define NACC 128" in E.generated_source(odd, 64, 1)
    with pytest.raises(cg.CgError):
        E.generated_source(odd + E.param(64) * E.inp(0), 65, 1)
    with pytest.raises(cg.CgError):
        E.generated_source(two_per_param(64), 64, 1)
