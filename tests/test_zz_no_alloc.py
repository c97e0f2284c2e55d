"""The allocation-free mixture gradient entry point, through the C ABI.

cg_mixture_gradient_noalloc is for callers that cannot allocate device
memory or hand over a workspace (code under another framework's allocator,
plug-ins whose host owns all device buffers, real-time loops).  Its only
scratch is a static array inside libcg.  This file is named so that pytest
collects it last; it passes alone in a fresh process and after the rest.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2203_06139_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def env():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2203_06139_gb300 import cg
    L = cg.lib()
    f = L.cg_mixture_gradient_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.POINTER(cg._Problem), ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p]
    return cg, f, torch.device("cuda:0")


def _noalloc(cg, f, pb, thetas):
    H = thetas.shape[0]
    v = torch.empty(H, dtype=torch.float64, device=thetas.device)
    g = torch.empty((H, 4), dtype=torch.float64, device=thetas.device)
    rc = f(ctypes.byref(pb.c), ctypes.c_void_p(thetas.data_ptr()), H, ctypes.c_void_p(v.data_ptr()),
           ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == cg.OK
    return v, g


def _close(v, g, v_ref, g_ref):
    v, g, v_ref, g_ref = (t.cpu().numpy() for t in (v, g, v_ref, g_ref))
    assert np.all(np.abs(v - v_ref) <= TOL * np.abs(v_ref))
    assert np.all(np.abs(g - g_ref) <= TOL * np.maximum(np.abs(g_ref), 1e-300))


def test_noalloc_matches_batch_gradient_twice(env):
    cg, f, dev = env
    x = torch.tensor(synth.c2_events(300001), device=dev)
    pb = cg.Problem.mixture(x, 0.0, 10.0)
    th_all = synth.c2_theta_points(14)
    for th_np in (th_all[:7], th_all[7:]):  # two calls in a row, different points
        th = torch.tensor(th_np, device=dev)
        v_ref, g_ref = cg.batch_gradient(pb, th)
        v, g = _noalloc(cg, f, pb, th)
        torch.cuda.synchronize()
        _close(v, g, v_ref, g_ref)


def test_noalloc_leaves_free_device_memory_unchanged(env):
    """After a first call (which takes the scratch array's device address),
    further calls allocate nothing: the device's free memory, read through
    cudaMemGetInfo, is the same before and after them."""
    cg, f, dev = env
    x = torch.tensor(synth.c2_events(200003), device=dev)
    pb = cg.Problem.mixture(x, 0.0, 10.0)
    th = torch.tensor(synth.c2_theta_points(5), device=dev)
    v = torch.empty(5, dtype=torch.float64, device=dev)
    g = torch.empty((5, 4), dtype=torch.float64, device=dev)
    args = (ctypes.byref(pb.c), ctypes.c_void_p(th.data_ptr()), 5, ctypes.c_void_p(v.data_ptr()),
            ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert f(*args) == cg.OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(4):
        assert f(*args) == cg.OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_weighted_and_limits(env):
    cg, f, dev = env
    x = torch.tensor(synth.c2_events(20001), device=dev)
    w = torch.tensor(np.random.default_rng(2).uniform(0.5, 1.5, 20001), device=dev)
    pb = cg.Problem.mixture(x, 0.0, 10.0, weights=w)
    th = torch.tensor(synth.c2_theta_points(3), device=dev)
    v_ref, g_ref = cg.batch_gradient(pb, th)
    for _ in range(2):
        v, g = _noalloc(cg, f, pb, th)
        torch.cuda.synchronize()
        _close(v, g, v_ref, g_ref)
    # more points than the static scratch holds: refused before any launch
    big = torch.zeros((4097, 4), dtype=torch.float64, device=dev)
    out = torch.empty(4097 * 4, dtype=torch.float64, device=dev)
    rc = f(ctypes.byref(pb.c), ctypes.c_void_p(big.data_ptr()), 4097, ctypes.c_void_p(out.data_ptr()),
           ctypes.c_void_p(out.data_ptr()), None)
    assert rc == cg.ERR_INVALID_ARG
