"""Fitting drivers over libcg: many histograms in one persistent launch
(captured in a CUDA graph), the plain per-histogram path, and the autotuner
that picks the warp / CTA / cluster mapping.

Marshalling only: every evaluation, line search and BFGS update runs in the
CUDA kernels of libcg (cg_fit_plan / cg_fit_init / cg_fit_step, the
Levenberg-Marquardt cg_fit_lm_* calls and the cg_fit_single_* calls).
"""
import ctypes
import json
import os
import time

import numpy as np
import torch

from . import cg

STATE_DOUBLES = cg.FIT_STATE_DOUBLES
STATE_BYTES = cg.FIT_STATE_BYTES
_TH, _GR, _H, _H0 = 0, 12, 24, 168
_F, _EDM, _FDATA = 180, 181, 182


class States:
    """View of a device array of cg_fit_state records."""

    def __init__(self, raw, P):
        self.raw = raw            # uint8 [H, STATE_BYTES]
        self.P = P
        self.d = raw.view(torch.float64).view(raw.shape[0], STATE_BYTES // 8)

    def _ints(self):
        return self.raw[:, STATE_DOUBLES * 8:STATE_DOUBLES * 8 + 16].contiguous().view(torch.int32)

    @property
    def theta(self):
        return self.d[:, _TH:_TH + self.P]

    @property
    def grad(self):
        return self.d[:, _GR:_GR + self.P]

    @property
    def f(self):
        return self.d[:, _F]

    @property
    def edm(self):
        return self.d[:, _EDM]

    @property
    def fdata(self):
        return self.d[:, _FDATA]

    @property
    def iters(self):
        return self._ints()[:, 0]

    @property
    def n_eval(self):
        return self._ints()[:, 1]

    @property
    def status(self):
        return self._ints()[:, 2]

    def clone(self):
        return States(self.raw.clone(), self.P)


class TileMap:
    def __init__(self, warp_max_bins=2048, cta_max_bins=32768, cta_threads=256, cluster_size=4):
        self.warp_max_bins, self.cta_max_bins = int(warp_max_bins), int(cta_max_bins)
        self.cta_threads, self.cluster_size = int(cta_threads), int(cluster_size)

    def c(self):
        m = cg._TileMap()
        m.warp_max_bins, m.cta_max_bins = self.warp_max_bins, self.cta_max_bins
        m.cta_threads, m.cluster_size = self.cta_threads, self.cluster_size
        return m

    def as_dict(self):
        return dict(warp_max_bins=self.warp_max_bins, cta_max_bins=self.cta_max_bins,
                    cta_threads=self.cta_threads, cluster_size=self.cluster_size)

    def __repr__(self):
        return "TileMap(%s)" % self.as_dict()


class HistBatch:
    """Many 1-D histograms of one model/objective, concatenated (a cg_batch)."""

    def __init__(self, y, offsets, lo, hi, n_peaks, poly_degree, objective, poly_mode=0,
                 precision=cg.PREC_FP64, device="cuda"):
        self.offsets_host = np.ascontiguousarray(offsets, dtype=np.int64)
        self.y = y if isinstance(y, torch.Tensor) else torch.tensor(np.asarray(y, np.float64), device=device)
        self.offsets = torch.tensor(self.offsets_host, device=self.y.device)
        self.lo = torch.as_tensor(np.asarray(lo, np.float64), device=self.y.device)
        self.hi = torch.as_tensor(np.asarray(hi, np.float64), device=self.y.device)
        self.H = len(self.offsets_host) - 1
        self.K, self.D = n_peaks, poly_degree
        self.P = 3 * n_peaks + poly_degree + 1
        self.pb = cg.Problem(cg.MODEL_GAUSS_POLY, objective, self.y, n_peaks=n_peaks, poly_degree=poly_degree,
                             poly_mode=poly_mode, n_bins=(self.y.numel(), 1), lo=(0.0, 0.0), hi=(1.0, 0.0),
                             precision=precision)
        b = cg._Batch()
        b.tmpl = self.pb.c
        b.n_hist = self.H
        b.offsets = self.offsets.data_ptr()
        b.lo = self.lo.data_ptr()
        b.hi = self.hi.data_ptr()
        self.c = b

    @property
    def sizes(self):
        return np.diff(self.offsets_host)

    def gradient(self, thetas, values=None, grads=None):
        """Value and gradient of every histogram at its own parameters thetas [H, P]."""
        thetas = cg._dev_f64(thetas, "thetas")
        if values is None:
            values = torch.empty(self.H, dtype=torch.float64, device=self.y.device)
        if grads is None:
            grads = torch.empty((self.H, self.P), dtype=torch.float64, device=self.y.device)
        n = cg.lib().cg_batch_workspace_size(ctypes.byref(self.c))
        ws = torch.empty(max(n, 256), dtype=torch.uint8, device=self.y.device)
        cg._check(cg.lib().cg_batch_gradient(ctypes.byref(self.c), cg._ptr(thetas), cg._ptr(values), cg._ptr(grads),
                                             cg._ptr(ws), ws.numel(), cg._stream()), "cg_batch_gradient")
        return values, grads

    def objective(self, thetas, values=None):
        """Value of every histogram at its own parameters (no adjoint sweep)."""
        thetas = cg._dev_f64(thetas, "thetas")
        if values is None:
            values = torch.empty(self.H, dtype=torch.float64, device=self.y.device)
        n = cg.lib().cg_batch_workspace_size(ctypes.byref(self.c))
        ws = torch.empty(max(n, 256), dtype=torch.uint8, device=self.y.device)
        cg._check(cg.lib().cg_batch_gradient(ctypes.byref(self.c), cg._ptr(thetas), cg._ptr(values), None,
                                             cg._ptr(ws), ws.numel(), cg._stream()), "cg_batch_gradient")
        return values


    def gauss_newton(self, thetas, values=None, grads=None, gn=None):
        """Value, gradient and Gauss-Newton matrix [H, P, P] of every histogram
        (df64 batches)."""
        thetas = cg._dev_f64(thetas, "thetas")
        dev = self.y.device
        if values is None:
            values = torch.empty(self.H, dtype=torch.float64, device=dev)
        if grads is None:
            grads = torch.empty((self.H, self.P), dtype=torch.float64, device=dev)
        if gn is None:
            gn = torch.empty((self.H, self.P, self.P), dtype=torch.float64, device=dev)
        ws = torch.empty(256, dtype=torch.uint8, device=dev)
        cg._check(cg.lib().cg_batch_gn(ctypes.byref(self.c), cg._ptr(thetas), cg._ptr(values), cg._ptr(grads),
                                       cg._ptr(gn), cg._ptr(ws), ws.numel(), cg._stream()), "cg_batch_gn")
        return values, grads, gn


class LMFitter:
    """Levenberg-Marquardt fits of every histogram of a df64 HistBatch: each
    step evaluates value, gradient and Gauss-Newton matrix at the trial points
    (tiles of at most 16384 bins) and runs the damping / Cholesky control
    (cg_fit_lm_plan / cg_fit_lm_init / cg_fit_lm_step).  States as for
    BatchFitter; hinv holds the GN matrix, h0[0] the damping."""

    def __init__(self, batch):
        self.b = batch
        offs = (ctypes.c_int64 * len(batch.offsets_host))(*batch.offsets_host.tolist())
        n = cg.lib().cg_fit_lm_workspace_size(ctypes.byref(batch.c), offs)
        if n == 0:
            raise cg.CgError(cg.ERR_UNSUPPORTED, "batch not supported by the Levenberg-Marquardt fitter "
                                                 "(df64 Gaussian + polynomial batches only)")
        self.ws = torch.empty(n, dtype=torch.uint8, device=batch.y.device)
        cg._check(cg.lib().cg_fit_lm_plan(ctypes.byref(batch.c), offs, cg._ptr(self.ws), self.ws.numel(),
                                          cg._stream()), "cg_fit_lm_plan")
        self.states = None
        self.graph = None

    def _init_into(self, theta0, tol, stream=None):
        cg._check(cg.lib().cg_fit_lm_init(ctypes.byref(self.b.c), cg._ptr(theta0), cg._ptr(self.states.raw),
                                          float(tol), cg._ptr(self.ws), self.ws.numel(), cg._stream(stream)),
                  "cg_fit_lm_init")

    def init(self, theta0, tol=1e-9):
        theta0 = cg._dev_f64(theta0, "theta0")
        if self.states is None:
            raw = torch.zeros((self.b.H, STATE_BYTES), dtype=torch.uint8, device=self.b.y.device)
            self.states = States(raw, self.b.P)
        self._init_into(theta0, tol)
        return self.states

    def _step_into(self, n_steps, tol, stream=None):
        cg._check(cg.lib().cg_fit_lm_step(ctypes.byref(self.b.c), cg._ptr(self.states.raw), int(n_steps), float(tol),
                                          cg._ptr(self.ws), self.ws.numel(), cg._stream(stream)), "cg_fit_lm_step")

    def step(self, n_steps=30, tol=1e-9):
        self._step_into(n_steps, tol)
        return self.states

    def capture(self, theta0, n_steps=30, tol=1e-9):
        """Capture init + n_steps steps into a CUDA graph (theta0 is kept)."""
        self._theta0 = cg._dev_f64(theta0, "theta0")
        if self.states is None:
            self.init(self._theta0, tol)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            g.capture_begin()
            self._init_into(self._theta0, tol, s)
            self._step_into(n_steps, tol, s)
            g.capture_end()
        torch.cuda.current_stream().wait_stream(s)
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()
        return self.states


class BatchFitter:
    """BFGS fits of every histogram of a HistBatch in one persistent launch."""

    def __init__(self, batch, tile_map=None):
        self.b = batch
        self.map = tile_map or TileMap()
        n = cg.lib().cg_fit_workspace_size(ctypes.byref(batch.c))
        if n == 0:
            raise cg.CgError(cg.ERR_UNSUPPORTED, "batch not supported by the fitter")
        self.ws = torch.empty(n, dtype=torch.uint8, device=batch.y.device)
        self.mc = self.map.c()
        offs = (ctypes.c_int64 * len(batch.offsets_host))(*batch.offsets_host.tolist())
        cg._check(cg.lib().cg_fit_plan(ctypes.byref(batch.c), offs, ctypes.byref(self.mc), cg._ptr(self.ws),
                                       self.ws.numel(), cg._stream()), "cg_fit_plan")
        self.states = None
        self.graph = None

    def _init_into(self, theta0, stream=None):
        cg._check(cg.lib().cg_fit_init(ctypes.byref(self.b.c), ctypes.byref(self.mc), cg._ptr(theta0),
                                       cg._ptr(self.states.raw), cg._ptr(self.ws), self.ws.numel(),
                                       cg._stream(stream)), "cg_fit_init")

    def init(self, theta0):
        """(Re)initialise every fit state at theta0 [H, P]; the state buffer is reused."""
        theta0 = cg._dev_f64(theta0, "theta0")
        if self.states is None:
            raw = torch.zeros((self.b.H, STATE_BYTES), dtype=torch.uint8, device=self.b.y.device)
            self.states = States(raw, self.b.P)
        self._init_into(theta0)
        return self.states

    def _step_into(self, st, n_steps, tol, stream=None):
        cg._check(cg.lib().cg_fit_step(ctypes.byref(self.b.c), ctypes.byref(self.mc), cg._ptr(st.raw), int(n_steps),
                                       float(tol), cg._ptr(self.ws), self.ws.numel(), cg._stream(stream)),
                  "cg_fit_step")

    def step(self, n_steps=50, tol=1e-9, states=None):
        st = states or self.states
        self._step_into(st, n_steps, tol)
        return st

    def capture(self, n_steps=50, tol=1e-9, theta0=None):
        """Capture the fit into a CUDA graph: cg_fit_step (counter reset + persistent
        kernel), preceded by cg_fit_init from theta0 when given (theta0 is kept)."""
        if theta0 is not None:
            self._theta0 = cg._dev_f64(theta0, "theta0")
            if self.states is None:
                self.init(self._theta0)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            g.capture_begin()
            if theta0 is not None:
                self._init_into(self._theta0, s)
            self._step_into(self.states, n_steps, tol, s)
            g.capture_end()
        torch.cuda.current_stream().wait_stream(s)
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()
        return self.states


class SingleFitter:
    """The plain per-histogram path: every trial point is a full-GPU gradient launch."""

    def __init__(self, problem):
        self.pb = problem
        n = cg.lib().cg_fit_single_workspace_size(ctypes.byref(problem.c))
        if n == 0:
            raise cg.CgError(cg.ERR_UNSUPPORTED, "problem not supported by the fitter")
        self.ws = torch.empty(n, dtype=torch.uint8, device=problem.data.device)
        self.states = None

    def init(self, theta0):
        theta0 = cg._dev_f64(theta0, "theta0")
        raw = torch.zeros((1, STATE_BYTES), dtype=torch.uint8, device=self.pb.data.device)
        cg._check(cg.lib().cg_fit_single_init(ctypes.byref(self.pb.c), cg._ptr(theta0), cg._ptr(raw),
                                              cg._ptr(self.ws), self.ws.numel(), cg._stream()), "cg_fit_single_init")
        self.states = States(raw, self.pb.n_params)
        return self.states

    def step(self, n_evals, tol=1e-9):
        cg._check(cg.lib().cg_fit_single_step(ctypes.byref(self.pb.c), cg._ptr(self.states.raw), int(n_evals),
                                              float(tol), cg._ptr(self.ws), self.ws.numel(), cg._stream()),
                  "cg_fit_single_step")
        return self.states

    def fit(self, theta0, max_iter=50, tol=1e-9, evals_per_sync=8):
        """Run to convergence (or max_iter iterations), checking the status every few evaluations."""
        st = self.init(theta0)
        while True:
            self.step(evals_per_sync, tol)
            status = int(st.status[0])
            if status != cg.FIT_RUNNING or int(st.iters[0]) >= max_iter:
                return st


# ----------------------------------------------------------------------------
# Autotuner: the mapping of histograms onto warps / CTAs / clusters
# ----------------------------------------------------------------------------
DEFAULT_CANDIDATES = [
    TileMap(w, c, t, k)
    for (w, c, t, k) in [(2048, 1 << 30, 256, 1), (512, 1 << 30, 256, 1), (2048, 32767, 256, 2), (2048, 16383, 256, 2),
                         (2048, 32767, 256, 4), (1024, 16384, 256, 4), (4096, 65536, 256, 1), (512, 4096, 128, 8)]
]


def _size_signature(sizes):
    edges = [0, 128, 512, 2048, 8192, 32768, 131072, 1 << 62]
    hist = np.histogram(sizes, bins=edges)[0]
    return "H%d:" % len(sizes) + ",".join(str(int(h)) for h in hist)


def _cache_path():
    return os.environ.get("CG_AUTOTUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "cg_autotune.json"))


# Version of the selection rule (pick_map) in the cache key: entries chosen
# by an earlier rule are not reused.
_PICK_RULE = "pick2"


def _autotune_key(batch, n_steps):
    c = batch.pb.c
    return "%s|%s|K%dD%dP%d|obj%d|prec%d|pm%d|S%d|%s" % (
        torch.cuda.get_device_name(), _size_signature(batch.sizes), batch.K, batch.D, batch.P, c.objective,
        c.precision, c.poly_mode, n_steps, _PICK_RULE)


def pick_map(timings, tie=0.02):
    """The map to use from (ms, map dict) pairs: among the maps within
    `tie` of the fastest (timing noise), the one with the smallest clusters,
    then the largest CTAs.  Smaller clusters synchronise less per
    evaluation, which sets the pace once only a few long fits are left: on
    the 4096-histogram workload a map with clusters of 8 x 128 threads tied
    with clusters of 2 x 256 over 50 iterations (50.9 against 51.1 ms) but
    took 2.0 s instead of 0.14 s to bring every fit to convergence."""
    if not timings:
        raise cg.CgError(cg.ERR_UNSUPPORTED, "no tile map could be planned for this batch")
    fastest = min(t for t, _ in timings)
    near = [(m["cluster_size"], -m["cta_threads"], t, i) for i, (t, m) in enumerate(timings)
            if t <= fastest * (1.0 + tie)]
    return timings[min(near)[3]][1]


def autotune(batch, theta0, candidates=None, n_steps=5, tol=1e-9, use_cache=True):
    """Time n_steps BFGS iterations of the whole batch under each candidate map
    and return (best_map, timings).  Time the iteration count the fit will
    run: the largest histograms set the tail of a long fit, which a few
    iterations do not show.  Results are cached per (GPU, size signature,
    model, objective, precision, n_steps) in a JSON file: a chi2 and a
    Poisson batch of the same shape, or an FP64 and a double-float batch,
    differ in per-bin cost and keep separate entries."""
    key = _autotune_key(batch, n_steps)
    path = _cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            cache = json.load(open(path))
        except (OSError, ValueError):
            cache = {}
        if key in cache:
            return TileMap(**cache[key]["map"]), cache[key]["timings"]
    timings = []
    for m in candidates or DEFAULT_CANDIDATES:
        try:
            f = BatchFitter(batch, m)
        except cg.CgError:
            continue
        f.init(theta0)
        st0 = f.states.clone()
        f.step(n_steps, tol)   # warm-up
        f.states = st0.clone()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        f.step(n_steps, tol)
        e1.record()
        torch.cuda.synchronize()
        timings.append((e0.elapsed_time(e1), m.as_dict()))
    timings.sort(key=lambda t: t[0])
    best = TileMap(**pick_map(timings))
    if use_cache:
        cache[key] = {"map": best.as_dict(), "timings": timings, "when": time.time()}
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            json.dump(cache, open(path, "w"), indent=1)
        except OSError:
            pass
    return best, timings


# The fitting calls of include/cg.h under their C names.
def cg_fit_step(fitter, n_steps=50, tol=1e-9):
    """cg_fit_step on a BatchFitter's batch, plan and states."""
    return fitter.step(n_steps, tol)


def cg_fit_lm_step(fitter, n_steps=30, tol=1e-9):
    """cg_fit_lm_step on an LMFitter's batch, plan and states."""
    return fitter.step(n_steps, tol)


def cg_batch_gn(batch, thetas):
    """cg_batch_gn: value, gradient and Gauss-Newton matrix of every histogram."""
    return batch.gauss_newton(thetas)
