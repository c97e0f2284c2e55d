"""Write cg_df64_tables.inc: the lookup tables of the double-float exp and log.

    exp2j[j] = 2^(j/64)            j = 0..63   (Tang's table-driven exp)
    logF[j]  = log(F_j)            F_j = 1 + (2j + 1)/128
    invF[j]  = 1/F_j

Each value is stored as a pair of floats (hi, lo): hi = value rounded to
float, lo = (value - hi) rounded to float, from 60-digit mpmath values, so the
pair carries the value to about 2^-48 relative.  Run from anywhere:
``python gen_df64_tables.py`` (rewrites csrc/cg_df64_tables.inc beside this script); the
CPU test suite checks the committed file against this script's output.
"""
import os

import mpmath
import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "csrc", "cg_df64_tables.inc")


def _pair(v):
    hi = np.float32(float(v))
    lo = np.float32(float(v - mpmath.mpf(float(hi))))
    return hi, lo


def _lit(x):
    x = float(x)
    if x == 0.0:
        return "0.0f"
    return "%sf" % float.hex(x)


def tables():
    mpmath.mp.dps = 60
    out = {}
    out["exp2j"] = [_pair(mpmath.power(2, mpmath.mpf(j) / 64)) for j in range(64)]
    F = [1 + mpmath.mpf(2 * j + 1) / 128 for j in range(64)]
    out["logF"] = [_pair(mpmath.log(f)) for f in F]
    out["invF"] = [_pair(1 / f) for f in F]
    return out


def render():
    t = tables()
    lines = ["// Generated by gen_df64_tables.py -- do not edit.",
             "// (hi, lo) float pairs: 2^(j/64), log(F_j), 1/F_j with F_j = 1 + (2j+1)/128."]
    for name in ("exp2j", "logF", "invF"):
        lines.append("static __device__ const float2 g_df_%s[64] = {" % name)
        for hi, lo in t[name]:
            lines.append("    {%s, %s}," % (_lit(hi), _lit(lo)))
        lines.append("};")
    return "\n".join(lines) + "\n"


if __name__ == "__main__":
    with open(OUT, "w") as f:
        f.write(render())
    print("wrote", OUT)
