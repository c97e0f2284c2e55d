"""Write cg_fp64_tables.inc: the lookup tables of the FP64 exp2 and log of cg_fp64.cuh.

    exp2t[j] = 2^(j/4096)   j = 0..4095   (Tang's table-driven exponential, in base 2)
    logF[t]  = log(F_t), invF[t] = 1/F_t, t = 0..129 (Tang's table-driven logarithm):
               F_t = 1 + t/128 for t = 0..53 (breakpoints in [1, sqrt 2)),
               F_t = (1 + (t - 1)/128)/2 for t = 54..129 (breakpoints in [sqrt 2 / 2, 1]).

Each entry is the double nearest to the exact value, from 60-digit mpmath
values (mpmath's conversion to float rounds to nearest); F_t itself is exact
in binary and is formed in the kernel from the argument's bits.  Run from anywhere:
``python gen_fp64_tables.py`` (rewrites csrc/cg_fp64_tables.inc beside this script); the
CPU test suite checks the committed file against this script's output.
"""
import os

import mpmath

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "csrc", "cg_fp64_tables.inc")
BITS = 12
N = 1 << BITS
NL = 130


def table():
    mpmath.mp.dps = 60
    return [float(mpmath.power(2, mpmath.mpf(j) / N)) for j in range(N)]


def breakpoints():
    """F_t: 1 + j/128 for j = 0..53, then (1 + j/128)/2 for j = 53..128."""
    return ([1 + mpmath.mpf(j) / 128 for j in range(54)] +
            [(1 + mpmath.mpf(j) / 128) / 2 for j in range(53, 129)])


def log_tables():
    mpmath.mp.dps = 60
    F = breakpoints()
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
             "// 2^(j/%d), j = 0..%d; log(F_t) and 1/F_t with F_t = 1 + t/128 (t = 0..53) and" % (N, N - 1),
             "// (1 + (t-1)/128)/2 (t = 54..129); each rounded to the nearest double."]
    lines += _rows("g_exp2_tab", t)
    lines += _rows("g_log_tab", logF)
    lines += _rows("g_invf_tab", invF)
    return "\n".join(lines) + "\n"


if __name__ == "__main__":
    with open(OUT, "w") as f:
        f.write(render())
    print("wrote", OUT)
