"""Error metric of the parity tests.

Per component k: e_k = |g_k - ref_k| / max(|ref_k|, floor * S_k), where
S_k = sum_i |dT_i/dtheta_k| is returned by the oracle.  The floor keeps the
metric defined for components whose total cancels to (near) zero.
"""
import numpy as np


def rel_err(g, ref, scale, floor=1e-6):
    g = np.asarray(g, np.float64)
    ref = np.asarray(ref, np.float64)
    scale = np.asarray(scale, np.float64)
    den = np.maximum(np.abs(ref), floor * scale)
    den = np.where(den > 0, den, 1.0)
    return np.abs(g - ref) / den


def max_rel_err(g, ref, scale, floor=1e-6):
    return float(np.max(rel_err(g, ref, scale, floor)))


def value_rel_err(v, ref):
    return abs(v - ref) / max(abs(ref), 1e-300)
