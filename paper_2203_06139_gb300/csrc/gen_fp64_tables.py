"""Write cg_fp64_tables.inc: the lookup tables of the FP64 exp2 and log of cg_fp64.cuh.

    exp2t[j] = 2^(j/4096)   j = 0..4095   (Tang's table-driven exponential, in base 2)
    logF[j]  = log(F_j)     F_j = 1 + (2j + 1)/256, j = 0..127 (Tang's table-driven logarithm)
    invF[j]  = 1/F_j

Each entry is the double nearest to the exact value, from 60-digit mpmath
values (mpmath's conversion to float rounds to nearest); F_j itself is exact
in binary and is formed in the kernel.  Run from anywhere:
``python gen_fp64_tables.py`` (rewrites the file next to this script); the
CPU test suite checks the committed file against this script's output.
"""
import os

import mpmath

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "cg_fp64_tables.inc")
BITS = 12
N = 1 << BITS
LOG_BITS = 7
NL = 1 << LOG_BITS


def table():
    mpmath.mp.dps = 60
    return [float(mpmath.power(2, mpmath.mpf(j) / N)) for j in range(N)]


def log_tables():
    mpmath.mp.dps = 60
    F = [1 + mpmath.mpf(2 * j + 1) / (2 * NL) for j in range(NL)]
    return [float(mpmath.log(f)) for f in F], [float(1 / f) for f in F]


def _rows(name, vals):
    out = ["static __device__ __align__(16) const double %s[%d] = {" % (name, len(vals))]
    for i in range(0, len(vals), 4):
        out.append("    " + " ".join("%s," % float.hex(v) for v in vals[i:i + 4]))
    out.append("};")
    return out


def render():
    t = table()
    logF, invF = log_tables()
    lines = ["// Generated by gen_fp64_tables.py -- do not edit.",
             "// 2^(j/%d), j = 0..%d; log(F_j) and 1/F_j with F_j = 1 + (2j+1)/%d, j = 0..%d;" % (N, N - 1, 2 * NL,
                                                                                             NL - 1),
             "// each rounded to the nearest double."]
    lines += _rows("g_exp2_tab", t)
    lines += _rows("g_log_tab", logF)
    lines += _rows("g_invf_tab", invF)
    return "\n".join(lines) + "\n"


if __name__ == "__main__":
    with open(OUT, "w") as f:
        f.write(render())
    print("wrote", OUT)
