"""Thin Python binding of libcg (include/cg.h): argument marshalling only.

Every number is computed by the CUDA kernels of libcg.so; this module only
builds the C structs, allocates device workspaces with PyTorch, and passes
pointers and the current CUDA stream.  There is no CPU fallback: without the
built library (or without a GPU) every call raises CgError.
"""
import ctypes
import os

import torch

from . import _build

# ---- enums, mirroring include/cg.h -----------------------------------------
OK, ERR_INVALID_ARG, ERR_DOMAIN, ERR_CUDA, ERR_TIMEOUT, ERR_NOT_CONVERGED, ERR_UNSUPPORTED, ERR_WORKSPACE = range(8)
MODEL_GAUSS_POLY, MODEL_MIX_GAUSS_EXP, MODEL_ROTGAUSS2D = 0, 1, 2
OBJ_CHI2, OBJ_POISSON, OBJ_POISSON_BC, OBJ_UNBINNED_NLL = 0, 1, 2, 3
PREC_FP64, PREC_DF64 = 0, 1
FIT_RUNNING, FIT_CONVERGED, FIT_MAX_ITER, FIT_LINESEARCH_FAILED, FIT_DOMAIN = range(5)
FIT_MAX_PARAMS = 12


class CgError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        msg = _status_string(code) if _lib is not None else "status %d" % code
        super().__init__("%s%s (cg_status %d)" % (what + ": " if what else "", msg, code))


class _Problem(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("objective", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("n_peaks", ctypes.c_int32), ("poly_degree", ctypes.c_int32), ("poly_mode", ctypes.c_int32),
                ("n_bins", ctypes.c_int64 * 2), ("lo", ctypes.c_double * 2), ("hi", ctypes.c_double * 2),
                ("centres", ctypes.c_void_p), ("data", ctypes.c_void_p), ("weights", ctypes.c_void_p),
                ("n_events", ctypes.c_int64)]


class _Batch(ctypes.Structure):
    _fields_ = [("tmpl", _Problem), ("n_hist", ctypes.c_int64), ("offsets", ctypes.c_void_p),
                ("lo", ctypes.c_void_p), ("hi", ctypes.c_void_p)]


class _TileMap(ctypes.Structure):
    _fields_ = [("warp_max_bins", ctypes.c_int32), ("cta_max_bins", ctypes.c_int32),
                ("cta_threads", ctypes.c_int32), ("cluster_size", ctypes.c_int32)]


# cg_fit_state as a flat record: 12 + 12 + 144 + 12 doubles, f, edm, fdata, 4 int32
FIT_STATE_DOUBLES = FIT_MAX_PARAMS * 3 + FIT_MAX_PARAMS * FIT_MAX_PARAMS + 3
FIT_STATE_BYTES = FIT_STATE_DOUBLES * 8 + 16

_lib = None
_vp, _sz, _i64, _dp = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int64, ctypes.c_void_p


def lib():
    """Load libcg.so (built in-tree by __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        raise CgError(ERR_CUDA, "libcg.so is not built (run __graft_entry__.build())")
    L = ctypes.CDLL(_build.LIB)
    P, B = ctypes.POINTER(_Problem), ctypes.POINTER(_Batch)
    sig = {
        "cg_num_params": (ctypes.c_int, [P]),
        "cg_workspace_size": (_sz, [P, _i64]),
        "cg_objective": (ctypes.c_int, [P, _dp, _dp, _vp, _sz, _vp]),
        "cg_gradient": (ctypes.c_int, [P, _dp, _dp, _dp, _vp, _sz, _vp]),
        "cg_batch_workspace_size": (_sz, [B]),
        "cg_batch_gradient": (ctypes.c_int, [B, _dp, _dp, _dp, _vp, _sz, _vp]),
        "cg_get_status": (ctypes.c_int, [_vp, _vp]),
        "cg_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "cg_set_profile_events": (None, [_vp, _vp]),
        "cg_rebin_normalize": (ctypes.c_int, [_vp, _i64, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp]),
        "cg_heuristic_start": (ctypes.c_int, [_vp, _i64, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                              ctypes.c_double, ctypes.c_int, _vp, _vp]),
        "cg_refine_start": (ctypes.c_int, [_vp, _i64, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                           _vp, _vp, ctypes.c_int, ctypes.c_double, _vp]),
        "cg_mse_loss": (ctypes.c_int, [_vp, _vp, _i64, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp]),
        "cg_colsum": (ctypes.c_int, [_vp, _i64, ctypes.c_int, _vp, _vp]),
        "cg_adamw": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                    ctypes.c_float, ctypes.c_float, ctypes.c_int, _vp, _vp]),
        "cg_to_bf16": (ctypes.c_int, [_vp, _i64, _vp, _vp]),
        "cg_select_start": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i64, ctypes.c_int, _vp, _vp, _vp]),
        "cg_decode_start": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp, _i64, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_double, ctypes.c_double, _vp, _vp]),
        "cg_gemm_bf16": (ctypes.c_int, [_vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp, ctypes.c_int, _vp, _vp,
                                        _vp, ctypes.c_int, _vp, _vp]),
        "cg_check_wait_timeout": (ctypes.c_int, [_vp, _vp]),
        "cg_fit_workspace_size": (_sz, [B]),
        "cg_fit_plan": (ctypes.c_int, [B, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(_TileMap), _vp, _sz, _vp]),
        "cg_fit_init": (ctypes.c_int, [B, ctypes.POINTER(_TileMap), _dp, _vp, _vp, _sz, _vp]),
        "cg_fit_step": (ctypes.c_int, [B, ctypes.POINTER(_TileMap), _vp, ctypes.c_int, ctypes.c_double, _vp, _sz,
                                       _vp]),
        "cg_batch_gn": (ctypes.c_int, [B, _dp, _dp, _dp, _dp, _vp, _sz, _vp]),
        "cg_fit_lm_workspace_size": (_sz, [B, ctypes.POINTER(ctypes.c_int64)]),
        "cg_fit_lm_plan": (ctypes.c_int, [B, ctypes.POINTER(ctypes.c_int64), _vp, _sz, _vp]),
        "cg_fit_lm_init": (ctypes.c_int, [B, _dp, _vp, ctypes.c_double, _vp, _sz, _vp]),
        "cg_fit_lm_step": (ctypes.c_int, [B, _vp, ctypes.c_int, ctypes.c_double, _vp, _sz, _vp]),
        "cg_fit_single_workspace_size": (_sz, [P]),
        "cg_fit_single_init": (ctypes.c_int, [P, _dp, _vp, _vp, _sz, _vp]),
        "cg_fit_single_step": (ctypes.c_int, [P, _vp, ctypes.c_int, ctypes.c_double, _vp, _sz, _vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _status_string(code):
    return lib().cg_status_string(int(code)).decode()


def _check(code, what):
    if code != OK:
        raise CgError(code, what)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev_f64(t, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
        raise CgError(ERR_INVALID_ARG, "%s must be a float64 CUDA tensor" % name)
    if not t.is_contiguous():
        raise CgError(ERR_INVALID_ARG, "%s must be contiguous" % name)
    return t


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class Problem:
    """A cg_problem plus references keeping its device tensors alive."""

    def __init__(self, model, objective, data, *, n_peaks=0, poly_degree=-1, poly_mode=0,
                 n_bins=(0, 0), lo=(0.0, 0.0), hi=(0.0, 0.0), centres=None, weights=None,
                 n_events=0, precision=PREC_FP64):
        self.data = _dev_f64(data, "data")
        self.centres = None if centres is None else _dev_f64(centres, "centres")
        self.weights = None if weights is None else _dev_f64(weights, "weights")
        s = _Problem()
        s.model, s.objective, s.precision = model, objective, precision
        s.n_peaks, s.poly_degree, s.poly_mode = n_peaks, poly_degree, poly_mode
        s.n_bins[0], s.n_bins[1] = int(n_bins[0]), int(n_bins[1])
        s.lo[0], s.lo[1] = float(lo[0]), float(lo[1])
        s.hi[0], s.hi[1] = float(hi[0]), float(hi[1])
        s.centres = None if self.centres is None else self.centres.data_ptr()
        s.data = self.data.data_ptr()
        s.weights = None if self.weights is None else self.weights.data_ptr()
        s.n_events = int(n_events)
        self.c = s
        self._ws = {}

    # ---- constructors for the three model families ----
    @staticmethod
    def gauss_poly(y, lo, hi, n_peaks, poly_degree, objective=OBJ_CHI2, poly_mode=0, centres=None,
                   precision=PREC_FP64):
        return Problem(MODEL_GAUSS_POLY, objective, y, n_peaks=n_peaks, poly_degree=poly_degree,
                       poly_mode=poly_mode, n_bins=(y.numel(), 1), lo=(lo, 0.0), hi=(hi, 0.0),
                       centres=centres, precision=precision)

    @staticmethod
    def mixture(x, lo, hi, weights=None, precision=PREC_FP64):
        return Problem(MODEL_MIX_GAUSS_EXP, OBJ_UNBINNED_NLL, x, n_events=x.numel(), lo=(lo, 0.0),
                       hi=(hi, 0.0), weights=weights, precision=precision)

    @staticmethod
    def rotgauss2d(counts, n_peaks, lo=(0.0, 0.0), hi=(1.0, 1.0), precision=PREC_FP64):
        ny, nx = counts.shape
        return Problem(MODEL_ROTGAUSS2D, OBJ_POISSON, counts, n_peaks=n_peaks, n_bins=(nx, ny),
                       lo=lo, hi=hi, precision=precision)

    @property
    def n_params(self):
        P = lib().cg_num_params(ctypes.byref(self.c))
        if P < 0:
            raise CgError(ERR_INVALID_ARG, "invalid problem")
        return P

    def workspace(self, n_theta=1):
        ws = self._ws.get(n_theta)
        if ws is None:
            n = lib().cg_workspace_size(ctypes.byref(self.c), n_theta)
            if n == 0:
                raise CgError(ERR_INVALID_ARG, "invalid problem")
            ws = torch.empty(n, dtype=torch.uint8, device=self.data.device)
            self._ws[n_theta] = ws
        return ws

    def status(self, n_theta=1, stream=None):
        """Device status of the last call on this problem's workspace (synchronises)."""
        return lib().cg_get_status(_ptr(self.workspace(n_theta)), _stream(stream))


def objective(pb, theta, value=None, stream=None):
    theta = _dev_f64(theta, "theta")
    if value is None:
        value = torch.empty((), dtype=torch.float64, device=theta.device)
    ws = pb.workspace(1)
    _check(lib().cg_objective(ctypes.byref(pb.c), _ptr(theta), _ptr(value), _ptr(ws), ws.numel(),
                              _stream(stream)), "cg_objective")
    return value


def gradient(pb, theta, value=None, grad=None, stream=None):
    """Objective value (0-d tensor) and gradient [P] at theta [P]."""
    theta = _dev_f64(theta, "theta")
    if value is None:
        value = torch.empty((), dtype=torch.float64, device=theta.device)
    if grad is None:
        grad = torch.empty(pb.n_params, dtype=torch.float64, device=theta.device)
    ws = pb.workspace(1)
    _check(lib().cg_gradient(ctypes.byref(pb.c), _ptr(theta), _ptr(value), _ptr(grad), _ptr(ws), ws.numel(),
                             _stream(stream)), "cg_gradient")
    return value, grad


def point_batch(pb, n_points):
    """A cg_batch of n_points parameter points on one problem (offsets = NULL)."""
    b = _Batch()
    b.tmpl = pb.c
    b.n_hist = int(n_points)
    b.offsets = b.lo = b.hi = None
    return b


def batch_gradient(pb, thetas, values=None, grads=None, stream=None):
    """Values [H] and gradients [H, P] at H parameter points thetas [H, P] on one problem."""
    thetas = _dev_f64(thetas, "thetas")
    H = thetas.shape[0]
    if values is None:
        values = torch.empty(H, dtype=torch.float64, device=thetas.device)
    if grads is None:
        grads = torch.empty((H, pb.n_params), dtype=torch.float64, device=thetas.device)
    b = point_batch(pb, H)
    ws = pb.workspace(H)
    _check(lib().cg_batch_gradient(ctypes.byref(b), _ptr(thetas), _ptr(values), _ptr(grads), _ptr(ws),
                                   ws.numel(), _stream(stream)), "cg_batch_gradient")
    return values, grads


def set_profile_events(start=None, stop=None):
    """Record torch.cuda.Event start/stop around every dominant-kernel launch (None, None: off)."""
    if start is None or stop is None:
        lib().cg_set_profile_events(None, None)
    else:
        lib().cg_set_profile_events(ctypes.c_void_p(start.cuda_event), ctypes.c_void_p(stop.cuda_event))


EPI_F32, EPI_BIAS_F32, EPI_BIAS_GELU, EPI_GELU_GRAD = 0, 1, 2, 3


def gemm_bf16(A, B, M, N, K, transA=0, transB=0, Cf=None, Cb=None, bias=None, aux_in=None, aux_out=None,
              epilogue=EPI_F32, err=None, stream=None):
    """C[M, N] = sum_k A[m, k] B[n, k] on the tensor cores (BF16 in, FP32 accumulate).
    A is [M, K] (transA = 0) or [K, M] (transA = 1); B is [N, K] (transB = 0) or [K, N]."""
    for t in (A, B):
        if t.dtype != torch.bfloat16 or not t.is_cuda or not t.is_contiguous():
            raise CgError(ERR_INVALID_ARG, "gemm operands must be contiguous bf16 CUDA tensors")
    lda = A.shape[1]
    ldb = B.shape[1]
    ldc = N
    _check(lib().cg_gemm_bf16(_ptr(A), _ptr(B), M, N, K, lda, ldb, transA, transB, _ptr(Cf), _ptr(Cb), ldc,
                              _ptr(bias), _ptr(aux_in), _ptr(aux_out), epilogue, _ptr(err), _stream(stream)),
           "cg_gemm_bf16")


def check_wait_timeout(err, stream=None):
    """Run the kernels' bounded wait on a barrier that nothing completes
    (cg_check_wait_timeout): bit 0 of err (int32 CUDA tensor) is set once the
    wait gives up, after about a second."""
    if err.dtype != torch.int32 or not err.is_cuda:
        raise CgError(ERR_INVALID_ARG, "err must be an int32 CUDA tensor")
    _check(lib().cg_check_wait_timeout(_ptr(err), _stream(stream)), "cg_check_wait_timeout")


def batch_objective(pb, thetas, values=None, stream=None):
    """Objective values [H] at H parameter points (no gradient; value-only kernels where available)."""
    thetas = _dev_f64(thetas, "thetas")
    H = thetas.shape[0]
    if values is None:
        values = torch.empty(H, dtype=torch.float64, device=thetas.device)
    b = point_batch(pb, H)
    ws = pb.workspace(H)
    _check(lib().cg_batch_gradient(ctypes.byref(b), _ptr(thetas), _ptr(values), None, _ptr(ws), ws.numel(),
                                   _stream(stream)), "cg_batch_gradient (values)")
    return values


# The calls of include/cg.h under their C names (the fitting calls are in fit.py).
cg_objective = objective
cg_gradient = gradient
cg_batch_gradient = batch_gradient
cg_check_wait_timeout = check_wait_timeout
