"""Expression programs: the per-element term of an objective written as an
expression of parameters and element inputs, differentiated by source
transformation in libcg.

The paper's tool turns the source of a C++ function into the source of its
reverse-mode derivative (Sec. 2-3, Listings 1-2).  Here the function is an
expression built with the operators below; ``compile`` hands its node list
to ``cg_expr_compile``, which writes the CUDA source of one fused kernel
(forward values and reverse sweep of every element, summed per tile in a
fixed order) and a finalize kernel, compiles it with NVRTC for this GPU and
loads it.  This module only builds and marshals the node list.

Example (chi2 of a Gaussian on a linear background; x = bin centre, y = count)::

    x, y = inp(0), inp(1)
    A, mu, s, c0, c1 = (param(k) for k in range(5))
    f = A * exp(-(x - mu) ** 2 / (2.0 * s ** 2)) + c0 + c1 * x
    prog = compile((y - f) ** 2 / maximum(y, 1.0), n_params=5, n_inputs=2)
    value, grad = prog.gradient([xs, ys], thetas)
"""
import ctypes

import torch

from . import cg

CONST, PARAM, INPUT, INDEX, ADD, SUB, MUL, DIV, NEG, EXP, LOG, SQRT, ERFC, POWI, MAX = range(15)
VALUE_ONLY = 1   # compile flag: the objective only
_UNARY = {NEG, EXP, LOG, SQRT, ERFC, POWI}
_BINARY = {ADD, SUB, MUL, DIV, MAX}


class Expr:
    """A node of an expression DAG (shared subexpressions stay shared)."""

    __slots__ = ("op", "a", "b", "i", "c")

    def __init__(self, op, a=None, b=None, i=0, c=0.0):
        self.op, self.a, self.b, self.i, self.c = op, a, b, int(i), float(c)

    def __add__(self, o): return Expr(ADD, self, _wrap(o))
    def __radd__(self, o): return Expr(ADD, _wrap(o), self)
    def __sub__(self, o): return Expr(SUB, self, _wrap(o))
    def __rsub__(self, o): return Expr(SUB, _wrap(o), self)
    def __mul__(self, o): return Expr(MUL, self, _wrap(o))
    def __rmul__(self, o): return Expr(MUL, _wrap(o), self)
    def __truediv__(self, o): return Expr(DIV, self, _wrap(o))
    def __rtruediv__(self, o): return Expr(DIV, _wrap(o), self)
    def __neg__(self): return Expr(NEG, self)

    def __pow__(self, k):
        if int(k) != k or abs(int(k)) > 16:
            raise ValueError("only integer powers in [-16, 16]")
        return Expr(POWI, self, i=int(k))


def _wrap(x):
    return x if isinstance(x, Expr) else Expr(CONST, c=float(x))


def param(i):
    """theta[i]"""
    return Expr(PARAM, i=i)


def inp(i):
    """Input array i at the element."""
    return Expr(INPUT, i=i)


def index():
    """The element index (as a double)."""
    return Expr(INDEX)


def const(c):
    return Expr(CONST, c=c)


def exp(e): return Expr(EXP, _wrap(e))
def log(e): return Expr(LOG, _wrap(e))
def sqrt(e): return Expr(SQRT, _wrap(e))
def erfc(e): return Expr(ERFC, _wrap(e))
def maximum(a, b): return Expr(MAX, _wrap(a), _wrap(b))


def nodes(root):
    """The node list of an expression, topological order (operands first,
    each shared subexpression once), the root last: rows (op, a, b, i, c)."""
    order, index_of = [], {}
    stack = [(root, False)]
    while stack:
        e, expanded = stack.pop()
        if id(e) in index_of:
            continue
        kids = [k for k in (e.a, e.b) if k is not None]
        if not expanded and any(id(k) not in index_of for k in kids):
            stack.append((e, True))
            for k in reversed(kids):
                if id(k) not in index_of:
                    stack.append((k, False))
            continue
        index_of[id(e)] = len(order)
        order.append(e)
    return [(e.op, index_of[id(e.a)] if e.a is not None else -1, index_of[id(e.b)] if e.b is not None else -1,
             e.i, e.c) for e in order]


class _Node(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("a", ctypes.c_int32), ("b", ctypes.c_int32), ("i", ctypes.c_int32),
                ("c", ctypes.c_double)]


_declared = False


def _lib():
    global _declared
    lib = cg.lib()
    if not _declared:
        vp, i64, c_int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        lib.cg_expr_compile.argtypes = [ctypes.POINTER(_Node), c_int, c_int, c_int, c_int, ctypes.POINTER(vp)]
        lib.cg_expr_compile.restype = c_int
        lib.cg_expr_source.argtypes = [vp]
        lib.cg_expr_source.restype = ctypes.c_char_p
        lib.cg_expr_log.argtypes = [vp]
        lib.cg_expr_log.restype = ctypes.c_char_p
        lib.cg_expr_num_acc.argtypes = [vp]
        lib.cg_expr_num_acc.restype = c_int
        lib.cg_expr_workspace_size.argtypes = [vp, i64, i64]
        lib.cg_expr_workspace_size.restype = ctypes.c_size_t
        lib.cg_expr_gradient.argtypes = [vp, ctypes.POINTER(vp), i64, vp, i64, vp, vp, vp, ctypes.c_size_t, vp]
        lib.cg_expr_gradient.restype = c_int
        lib.cg_expr_free.argtypes = [vp]
        lib.cg_expr_free.restype = None
        _declared = True
    return lib


class Program:
    """Compiled expression program: objective = sum over the elements of the
    root expression, gradient with respect to theta[0 .. n_params)."""

    def __init__(self, root, n_params, n_inputs, value_only=False):
        lib = _lib()
        self.node_list = nodes(_wrap(root))
        arr = (_Node * len(self.node_list))(*[_Node(*r) for r in self.node_list])
        h = ctypes.c_void_p()
        rc = lib.cg_expr_compile(arr, len(self.node_list), n_params, n_inputs, VALUE_ONLY if value_only else 0,
                                 ctypes.byref(h))
        self._h = h
        self.n_params, self.n_inputs, self.value_only = n_params, n_inputs, value_only
        if rc != cg.OK:
            log = lib.cg_expr_log(h).decode() if h.value else ""
            raise cg.CgError(rc, "cg_expr_compile: %s" % (log or "invalid or unsupported program"))
        self._ws = {}

    @property
    def source(self):
        return _lib().cg_expr_source(self._h).decode()

    @property
    def num_acc(self):
        return _lib().cg_expr_num_acc(self._h)

    def _call(self, inputs, thetas, values, grads, stream):
        if len(inputs) != self.n_inputs:
            raise cg.CgError(cg.ERR_INVALID_ARG, "expected %d input arrays" % self.n_inputs)
        ins = [cg._dev_f64(t, "input") for t in inputs]
        thetas = cg._dev_f64(thetas, "thetas")
        n = ins[0].numel() if ins else 0
        if any(t.numel() != n for t in ins):
            raise cg.CgError(cg.ERR_INVALID_ARG, "inputs of different lengths")
        H = thetas.shape[0]
        key = (n, H)
        ws = self._ws.get(key)
        if ws is None:
            nb = _lib().cg_expr_workspace_size(self._h, n, H)
            ws = torch.empty(max(nb, 256), dtype=torch.uint8, device=thetas.device)
            self._ws[key] = ws
        ptrs = (ctypes.c_void_p * max(1, len(ins)))(*[t.data_ptr() for t in ins])
        rc = _lib().cg_expr_gradient(self._h, ptrs, n, thetas.data_ptr(), H, values.data_ptr(),
                                     grads.data_ptr() if grads is not None else None, ws.data_ptr(), ws.numel(),
                                     cg._stream(stream))
        cg._check(rc, "cg_expr_gradient")

    def gradient(self, inputs, thetas, values=None, grads=None, stream=None):
        """Values [H] and gradients [H, P] at the H rows of thetas."""
        if self.value_only:
            raise cg.CgError(cg.ERR_INVALID_ARG, "a value-only program has no gradient")
        H = thetas.shape[0]
        if values is None:
            values = torch.empty(H, dtype=torch.float64, device=thetas.device)
        if grads is None:
            grads = torch.empty((H, self.n_params), dtype=torch.float64, device=thetas.device)
        self._call(inputs, thetas, values, grads, stream)
        return values, grads

    def objective(self, inputs, thetas, values=None, stream=None):
        """Values only (the finalize kernel skips the reverse sweep)."""
        if values is None:
            values = torch.empty(thetas.shape[0], dtype=torch.float64, device=thetas.device)
        self._call(inputs, thetas, values, None, stream)
        return values

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                _lib().cg_expr_free(h)
            except Exception:
                pass


def compile(root, n_params, n_inputs, value_only=False):
    return Program(root, n_params, n_inputs, value_only)


def generated_source(root, n_params, n_inputs, value_only=False):
    """The CUDA source libcg generates for an expression (also where it cannot
    compile or run it, e.g. on a machine without a GPU)."""
    lib = _lib()
    nl = nodes(_wrap(root))
    arr = (_Node * len(nl))(*[_Node(*r) for r in nl])
    h = ctypes.c_void_p()
    rc = lib.cg_expr_compile(arr, len(nl), n_params, n_inputs, VALUE_ONLY if value_only else 0, ctypes.byref(h))
    if not h.value:
        raise cg.CgError(rc, "cg_expr_compile rejected the program")
    try:
        return lib.cg_expr_source(h).decode()
    finally:
        lib.cg_expr_free(h)
