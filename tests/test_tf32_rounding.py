"""The TF32 splits of the tensor-core tile passes (kernels_brick_tc.cu), emulated
on FP32 bit patterns and checked against their definitions computed exactly:

  tf32_rna(x)   x rounded to the nearest value with 10 mantissa bits, ties away
                from zero ((bits + 0x1000) & 0xFFFFE000);
  tf32_rest(x)  x - trunc(x) (exact in FP32: the part the MMA's truncation of x
                drops), rounded the same way.  The rest has at most 13
                significant bits, of which TF32 keeps 11: truncated (the MMA's
                own reading) trunc(x) + rest is x to within 2^-21 |x|, always
                low in magnitude; rounded, to within 2^-22 |x|, and the exact
                ties that rounding away from zero meets leave a smaller mean
                error of the other sign.
CPU."""
import random
import struct
from fractions import Fraction

import numpy as np


def f2u(x):
    return struct.unpack("<I", struct.pack("<f", x))[0]


def u2f(u):
    return struct.unpack("<f", struct.pack("<I", u & 0xFFFFFFFF))[0]


def rna_bits(x):
    return u2f((f2u(x) + 0x1000) & 0xFFFFE000)


def trunc_bits(x):
    return u2f(f2u(x) & 0xFFFFE000)


def rest_bits(x):
    r = np.float32(x) - np.float32(trunc_bits(x))   # exact in FP32
    return rna_bits(float(r))


def rna_exact(x):
    """nearest multiple of 2^(e-10) for |x| in [2^e, 2^(e+1)), ties away from zero"""
    if x == 0:
        return 0.0
    m, e = np.frexp(abs(x))                 # |x| = m 2^e, m in [0.5, 1)
    q = Fraction(abs(x)) / Fraction(2) ** (int(e) - 11)   # units of 2^(e-11): 10 mantissa bits after the leading one
    n = int(q)
    if q - n >= Fraction(1, 2):
        n += 1
    v = float(Fraction(n) * Fraction(2) ** (int(e) - 11))
    return v if x > 0 else -v


def samples(count, seed):
    rnd = random.Random(seed)
    out = []
    for _ in range(count):
        u = rnd.getrandbits(23) | ((rnd.randrange(100, 150)) << 23) | (rnd.getrandbits(1) << 31)
        out.append(u2f(u))
    # ties and values just around them
    for base in (1.0, -1.0, 0.75, 3.0e-3, -7.5):
        b = f2u(base) & 0xFFFFE000
        for d in (0x0FFF, 0x1000, 0x1001, 0x1FFF):
            out.append(u2f(b | d if base > 0 else (b | d) | 0x80000000))
    return out


def test_rna_is_round_to_nearest_ties_away():
    for x in samples(20000, 1):
        assert rna_bits(x) == rna_exact(x), (x, rna_bits(x), rna_exact(x))


def test_rest_completes_the_truncated_part():
    errs, errs_trunc = [], []
    for x in samples(20000, 2):
        if x == 0:
            continue
        hi, lo = trunc_bits(x), rest_bits(x)
        assert f2u(lo) & 0x1FFF == 0                 # the low part is itself a TF32 value
        err = Fraction(hi) + Fraction(lo) - Fraction(x)
        assert abs(err) <= Fraction(abs(x)) * Fraction(1, 2 ** 22), x
        errs.append(float(err / Fraction(x)))
        r = float(np.float32(x) - np.float32(hi))
        errs_trunc.append(float((Fraction(hi) + Fraction(trunc_bits(r)) - Fraction(x)) / Fraction(x)))
    errs, errs_trunc = np.array(errs), np.array(errs_trunc)
    assert 0 < errs.mean() <= 2.0 ** -24                   # ties away from zero: under half an FP32 ulp
    assert errs_trunc.max() <= 0 and errs_trunc.min() >= -(2.0 ** -21)
    assert errs_trunc.mean() < -2 * errs.mean()            # truncating the rest: a larger bias towards zero
