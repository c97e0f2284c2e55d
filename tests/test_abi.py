"""The C ABI library loads on the host and exports every entry point that
include/*.h declares; host-side argument checks run without a GPU."""
import ctypes
import glob
import os
import re

import pytest

import __graft_entry__
from tests.conftest import ROOT


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(cg_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    from paper_2203_06139_gb300 import cg
    return cg.lib()


def test_header_declares_the_four_calls():
    names = declared_functions()
    for n in ("cg_objective", "cg_gradient", "cg_batch_gradient", "cg_fit_step"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_side_validation_without_gpu(lib):
    from paper_2203_06139_gb300 import cg
    p = cg._Problem()
    p.model, p.objective, p.precision = cg.MODEL_GAUSS_POLY, cg.OBJ_CHI2, cg.PREC_FP64
    p.n_peaks, p.poly_degree, p.poly_mode = 1, 1, 0
    p.n_bins[0] = 10000
    p.lo[0], p.hi[0] = 0.0, 10.0
    p.data = 256  # never dereferenced by the host checks
    assert lib.cg_num_params(ctypes.byref(p)) == 5
    assert lib.cg_workspace_size(ctypes.byref(p), 100) > 0
    bad = cg._Problem()
    bad.model = 7
    assert lib.cg_num_params(ctypes.byref(bad)) == -1
    assert lib.cg_workspace_size(ctypes.byref(bad), 1) == 0
    assert lib.cg_gradient(None, None, None, None, None, 0, None) == cg.ERR_INVALID_ARG
    p2 = cg._Problem.from_buffer_copy(p)
    p2.n_peaks = 5
    assert lib.cg_num_params(ctypes.byref(p2)) == -1
    # workspace too small / misaligned is refused before any launch
    assert lib.cg_gradient(ctypes.byref(p), ctypes.c_void_p(256), ctypes.c_void_p(512), ctypes.c_void_p(768),
                           ctypes.c_void_p(1024), 16, None) == cg.ERR_WORKSPACE
    assert lib.cg_gradient(ctypes.byref(p), ctypes.c_void_p(256), ctypes.c_void_p(512), ctypes.c_void_p(768),
                           ctypes.c_void_p(1025), 1 << 30, None) == cg.ERR_WORKSPACE
    assert lib.cg_status_string(cg.ERR_DOMAIN).startswith(b"domain")
    # the bounded-wait check refuses a missing status word before any launch
    assert lib.cg_check_wait_timeout(None, None) == cg.ERR_INVALID_ARG


def test_df64_tables_match_their_generator():
    """The committed lookup tables of the double-float exp/log are exactly what
    the generator writes (exactly rounded float pairs from 60-digit values)."""
    pytest.importorskip("mpmath")
    import importlib.util
    path = os.path.join(ROOT, "paper_2203_06139_gb300", "gen_df64_tables.py")
    spec = importlib.util.spec_from_file_location("gen_df64_tables", path)
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    with open(gen.OUT) as f:
        assert f.read() == gen.render()
    t = gen.tables()
    # spot values: 2^(1/64), log(F_0) = log(1 + 1/128), 1/F_63 = 1/(1 + 127/128)
    import math
    for (hi, lo), ref in ((t["exp2j"][1], 2 ** (1 / 64)), (t["logF"][0], math.log1p(1 / 128)),
                          (t["invF"][63], 128 / 255)):
        assert abs(float(hi) + float(lo) - ref) <= 2.0 ** -48 * abs(ref)   # what a float pair holds


def test_fp64_tables_match_their_generator():
    """The committed tables of the FP64 exp2 and log are exactly what the
    generator writes: every entry the double nearest 2^(j/4096), log(F_t) or
    1/F_t, F_t = 1 + t/128 (t = 0..53) and (1 + (t-1)/128)/2 (t = 54..129),
    checked here against Python's own correctly rounded arithmetic where it
    has it."""
    pytest.importorskip("mpmath")
    import importlib.util
    import math
    path = os.path.join(ROOT, "paper_2203_06139_gb300", "gen_fp64_tables.py")
    spec = importlib.util.spec_from_file_location("gen_fp64_tables", path)
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    with open(gen.OUT) as f:
        assert f.read() == gen.render()
    t = gen.table()
    logF, invF = gen.log_tables()
    assert len(t) == 4096 and len(logF) == len(invF) == 130
    assert t[0] == 1.0 and t[2048] == math.sqrt(2.0)          # sqrt is correctly rounded
    assert abs(t[1024] - 2 ** 0.25) <= 2 ** -52
    F = [1.0 + k / 128.0 for k in range(54)] + [(1.0 + k / 128.0) / 2.0 for k in range(53, 129)]   # exact
    assert F[0] == 1.0 and F[129] == 1.0 and F[53] == 2 * F[54] < math.sqrt(2.0)   # j = 53 in both binades
    for k in (0, 1, 53, 54, 77, 128, 129):
        assert invF[k] == 1.0 / F[k]                           # IEEE division is correctly rounded
        assert logF[k] == 0.0 if F[k] == 1.0 else abs(logF[k] - math.log(F[k])) <= 2 ** -52 * abs(math.log(F[k]))
    assert all(1.0 <= v < 2.0 for v in t) and all(t[i] < t[i + 1] for i in range(4095))


def test_lm_plan_sizes_and_refusals_without_gpu(lib):
    """The Levenberg-Marquardt workspace: tiles of at most 16384 bins per
    histogram (one for an empty one), rows of N + 1 + R(R+1)/2 doubles; FP64
    batches, decreasing offsets and missing plans' inputs are refused on the
    host."""
    from paper_2203_06139_gb300 import cg
    b = cg._Batch()
    b.tmpl.model, b.tmpl.objective, b.tmpl.precision = cg.MODEL_GAUSS_POLY, cg.OBJ_CHI2, cg.PREC_DF64
    b.tmpl.n_peaks, b.tmpl.poly_degree = 1, 2
    b.tmpl.data = 256
    b.n_hist, b.offsets, b.lo, b.hi = 3, 512, 768, 1024
    offs = (ctypes.c_int64 * 4)(0, 16384, 16385, 16385)   # 1 + 1 + 1 (empty) tiles
    offs2 = (ctypes.c_int64 * 4)(0, 40000, 40001, 40001)  # 3 + 1 + 1 tiles
    n1 = lib.cg_fit_lm_workspace_size(ctypes.byref(b), offs)
    n2 = lib.cg_fit_lm_workspace_size(ctypes.byref(b), offs2)
    row = (1 + 3 + 4) + 1 + 7 * 8 // 2
    assert n1 > 0 and n2 - n1 == 2 * row * 8
    assert lib.cg_fit_lm_workspace_size(ctypes.byref(b), (ctypes.c_int64 * 4)(0, 5, 3, 9)) == 0
    b64 = cg._Batch.from_buffer_copy(b)
    b64.tmpl.precision = cg.PREC_FP64
    assert lib.cg_fit_lm_workspace_size(ctypes.byref(b64), offs) == 0
    assert lib.cg_fit_lm_plan(ctypes.byref(b64), offs, ctypes.c_void_p(4096), 1 << 20, None) == cg.ERR_UNSUPPORTED
    assert lib.cg_fit_lm_plan(ctypes.byref(b), offs, ctypes.c_void_p(4096), 16, None) == cg.ERR_WORKSPACE
    assert lib.cg_fit_lm_step(ctypes.byref(b), ctypes.c_void_p(4096), 1, 1e-9, ctypes.c_void_p(4097), 1 << 20,
                              None) == cg.ERR_WORKSPACE


def test_fit_plan_refusals_without_gpu(lib):
    """cg_fit_plan checks its map and the host offsets before touching the
    device: CTA sizes outside 64..512 or not multiples of 32, cluster sizes
    other than 1/2/4/8, warp_max_bins > cta_max_bins and decreasing offsets
    are invalid arguments; FP64/df64 only; a too-small workspace is refused."""
    from paper_2203_06139_gb300 import cg
    b = cg._Batch()
    b.tmpl.model, b.tmpl.objective, b.tmpl.precision = cg.MODEL_GAUSS_POLY, cg.OBJ_CHI2, cg.PREC_DF64
    b.tmpl.n_peaks, b.tmpl.poly_degree = 1, 2
    b.tmpl.data = 256
    b.n_hist, b.offsets, b.lo, b.hi = 3, 512, 768, 1024
    n = lib.cg_fit_workspace_size(ctypes.byref(b))
    assert n > 0
    offs = (ctypes.c_int64 * 4)(0, 100, 300, 600)
    ws = ctypes.c_void_p(4096)
    good = dict(warp_max_bins=128, cta_max_bins=4096, cta_threads=256, cluster_size=2)
    for bad in (dict(cta_threads=48), dict(cta_threads=1024), dict(cta_threads=100), dict(cluster_size=3),
                dict(warp_max_bins=5000)):
        m = cg._TileMap()
        for k, v in dict(good, **bad).items():
            setattr(m, k, v)
        assert lib.cg_fit_plan(ctypes.byref(b), offs, ctypes.byref(m), ws, n, None) == cg.ERR_INVALID_ARG, bad
    m = cg._TileMap()
    for k, v in good.items():
        setattr(m, k, v)
    assert lib.cg_fit_plan(ctypes.byref(b), (ctypes.c_int64 * 4)(0, 100, 50, 600), ctypes.byref(m), ws, n,
                           None) == cg.ERR_INVALID_ARG
    assert lib.cg_fit_plan(ctypes.byref(b), offs, ctypes.byref(m), ws, n - 1, None) == cg.ERR_WORKSPACE
    assert lib.cg_fit_plan(ctypes.byref(b), offs, ctypes.byref(m), ctypes.c_void_p(4097), n, None) == cg.ERR_WORKSPACE


def test_python_binding_has_the_c_names():
    from paper_2203_06139_gb300 import cg, fit
    for n in ("cg_objective", "cg_gradient", "cg_batch_gradient"):
        assert callable(getattr(cg, n))
    for n in ("cg_fit_step", "cg_fit_lm_step", "cg_batch_gn"):
        assert callable(getattr(fit, n))


def test_the_package_never_reaches_the_oracle():
    """The product package imports neither the oracle nor the build entry
    point on any path (the oracle is test infrastructure); checked on every
    module's import statements and on a fresh interpreter's module table
    after importing every module of the package."""
    import ast
    import subprocess
    import sys
    pkg = os.path.join(ROOT, "paper_2203_06139_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if not f.endswith(".py"):
                continue
            tree = ast.parse(open(os.path.join(dirpath, f)).read())
            for node in ast.walk(tree):
                names = []
                if isinstance(node, ast.Import):
                    names = [a.name for a in node.names]
                elif isinstance(node, ast.ImportFrom):
                    names = [node.module or ""]
                for n in names:
                    assert not n.startswith("oracle") and n != "__graft_entry__", (f, n)
    code = ("import sys; sys.path.insert(0, %r)\n" % ROOT +
            "import importlib, pkgutil, paper_2203_06139_gb300 as p\n"
            "import os\n"
            "for m in pkgutil.iter_modules(p.__path__):\n"
            "    if os.path.exists(os.path.join(p.__path__[0], m.name + '.py')):\n"
            "        importlib.import_module('paper_2203_06139_gb300.' + m.name)\n"
            "bad = [k for k in sys.modules if k == 'oracle' or k.startswith('oracle.') or k == '__graft_entry__']\n"
            "print(','.join(bad))\n")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == "", r.stdout
