"""Writes sample_tables.h: the tables of the sampler's table-driven sincospi and log
(kernels_sample.cu, Box-Muller draws).  Run once, from this directory:

    python gen_sample_tables.py > sample_tables.h

Values are computed at 50 significant digits (sympy) and rounded to the nearest double:
  sinpi(k/256), cospi(k/256), k = 0..511                  (angle addition for sincospi(t), t in [0, 2))
  r_j = the double nearest 1/c_j, c_j = 0.75 + j/128      (j = 0..96: m in [0.75, 1.5))
  -log(r_j) as a double-double (hi + lo), of the double r_j itself
  ln 2 as hi + lo with hi on 42 significant bits (e * hi exact for |e| < 2^11)
"""
import sympy as sp

DIG = 50


def dbl(x):
    return float(sp.Float(x, DIG))


def hexf(x):
    return float.hex(x) if x != 0 else "0.0"


def main():
    out = ["// sample_tables.h -- generated by gen_sample_tables.py (do not edit): tables of the",
           "// sampler's table-driven sincospi and log, exact values rounded to the nearest double.",
           "#pragma once", ""]
    out.append("// kSinCosPi[2k], kSinCosPi[2k + 1] = sinpi(k / 256), cospi(k / 256), k = 0..511")
    out.append("__device__ const double kSinCosPi[1024] = {")
    vals = []
    for k in range(512):
        a = sp.pi * sp.Rational(k, 256)
        vals += [dbl(sp.sin(a).evalf(DIG)), dbl(sp.cos(a).evalf(DIG))]
    for i in range(0, len(vals), 4):
        out.append("    " + ", ".join(hexf(v) for v in vals[i:i + 4]) + ",")
    out.append("};")
    out.append("")
    out.append("// kLogTab[3j], [3j + 1], [3j + 2] = r_j, hi and lo of -log(r_j); r_j = the double")
    out.append("// nearest 1 / c_j, c_j = 0.75 + j / 128, j = 0..96 (r_32 = 1, -log r_32 = 0)")
    out.append("__device__ const double kLogTab[291] = {")
    for j in range(97):
        c = sp.Rational(3, 4) + sp.Rational(j, 128)
        r = dbl((1 / c).evalf(DIG))
        L = -sp.log(sp.Rational(r)).evalf(DIG)   # the log of the double r itself
        hi = dbl(L)
        lo = dbl((L - sp.Rational(hi)).evalf(DIG))
        out.append(f"    {hexf(r)}, {hexf(hi)}, {hexf(lo)},")
    out.append("};")
    ln2 = sp.log(2).evalf(DIG)
    hi = sp.floor(ln2 * 2 ** 42) / sp.Integer(2) ** 42
    lo = dbl((ln2 - hi).evalf(DIG))
    out.append("")
    out.append(f"constexpr double kLn2Hi = {hexf(float(hi))};   // 42 significant bits")
    out.append(f"constexpr double kLn2Lo = {hexf(lo)};")
    out.append(f"constexpr double kPi = {hexf(dbl(sp.pi.evalf(DIG)))};")
    print("\n".join(out))


if __name__ == "__main__":
    main()
