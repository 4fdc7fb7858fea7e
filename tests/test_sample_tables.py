"""The tables and steps of the sampler's table-driven log and sincospi
(kernels_sample.cu: log_tab, sincospi_tab; tables in sample_tables.h, written by
gen_sample_tables.py), emulated in host doubles over the inputs the Box-Muller
draws produce (u = n 2^-53) and compared with the C library's log, sin and cos.
CPU."""
import math
import os
import random
import re
from fractions import Fraction

import pytest

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_2205_09900_gb300", "csrc", "sample_tables.h")


def _array(text, name):
    body = re.search(name + r"\[\d+\] = \{(.*?)\};", text, re.S).group(1)
    return [float.fromhex(t) if t.strip() != "0.0" else 0.0 for t in body.replace("\n", " ").split(",") if t.strip()]


def _const(text, name):
    return float.fromhex(re.search(r"constexpr double " + name + r" = ([^;]+);", text).group(1))


@pytest.fixture(scope="module")
def tabs():
    text = open(HDR).read()
    return (_array(text, "kSinCosPi"), _array(text, "kLogTab"), _const(text, "kLn2Hi"), _const(text, "kLn2Lo"),
            _const(text, "kPi"))


def fma(a, b, c):
    """a * b + c rounded once, as the device's fma"""
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def log_tab(u, tabs):
    _, lt, ln2h, ln2l, _ = tabs
    m, e = math.frexp(u)          # u = m 2^e, m in [0.5, 1)
    m, e = 2 * m, e - 1           # m in [1, 2)
    if m >= 1.5:
        m, e = m / 2, e + 1
    j = int(round((m - 0.75) * 128))
    r, lh, ll = lt[3 * j], lt[3 * j + 1], lt[3 * j + 2]
    y = fma(m, r, -1.0)
    p = fma(y, -1 / 9, 1 / 8)
    for c in (-1 / 7, 1 / 6, -1 / 5, 1 / 4, -1 / 3, 0.5, -1.0):
        p = fma(y, p, c)
    p = -(y * p)
    return fma(e, ln2h, lh) + (fma(e, ln2l, ll) + p)


def sincospi_tab(t, tabs):
    sc, _, _, _, pi = tabs
    k = int(t * 256.0)
    r = t - k / 256.0
    x = r * pi
    x2 = x * x
    sx = x * (1 + x2 * (-1 / 6 + x2 * (1 / 120 + x2 * (-1 / 5040))))
    cx = 1 + x2 * (-0.5 + x2 * (1 / 24 + x2 * (-1 / 720 + x2 / 40320)))
    sk, ck = sc[2 * k], sc[2 * k + 1]
    return fma(sk, cx, ck * sx), fma(ck, cx, -(sk * sx))


def test_tables_are_the_stated_values(tabs):
    sc, lt, ln2h, ln2l, pi = tabs
    assert len(sc) == 1024 and len(lt) == 291
    for k in range(0, 512, 7):   # libm's reference carries the rounding of pi * k / 256 (~4e-16)
        assert abs(sc[2 * k] - math.sin(math.pi * k / 256)) <= 1e-15
        assert abs(sc[2 * k + 1] - math.cos(math.pi * k / 256)) <= 1e-15
    for j in range(97):
        c = 0.75 + j / 128
        assert abs(lt[3 * j] * c - 1) <= 2 ** -52
        assert abs(lt[3 * j + 1] + math.log(lt[3 * j])) <= 1e-16
    assert lt[3 * 32: 3 * 32 + 3] == [1.0, 0.0, 0.0]
    assert ln2h + ln2l == math.log(2) and math.frexp(ln2h)[0] * 2 ** 42 == int(math.frexp(ln2h)[0] * 2 ** 42)


def test_log_tab_against_libm(tabs):
    rnd = random.Random(5)
    us = [(rnd.getrandbits(53) + 1) * 2.0 ** -53 for _ in range(20000)]
    us += [1.0, 1 - 2 ** -53, 1 - 2 ** -40, 1 - 2 ** -9, 0.75, 0.75 - 2 ** -53, 0.5, 2 ** -53, 2 ** -52, 1 / 3]
    us += [0.75 + j / 128 + d for j in range(97) for d in (-2 ** -9, 2 ** -9) if 0.5 <= 0.75 + j / 128 + d < 1.0]
    worst = 0.0
    for u in us:
        ref = math.log(u)
        got = log_tab(u, tabs)
        err = abs(got - ref) / max(abs(ref), 2 ** -1022)
        worst = max(worst, err)
    assert worst <= 4 * 2 ** -53, worst


def test_sincospi_tab_against_libm(tabs):
    rnd = random.Random(6)
    ts = [2 * rnd.getrandbits(53) * 2.0 ** -53 for _ in range(20000)] + [0.0, 0.5, 1.0, 1.5, 2 - 2 ** -52]
    worst = 0.0
    for t in ts:
        s, c = sincospi_tab(t, tabs)
        worst = max(worst, abs(s - math.sin(math.pi * t)), abs(c - math.cos(math.pi * t)))
    # absolute: math.sin(pi * t) itself carries the rounding of pi * t (up to ~4e-16 near t = 2)
    assert worst <= 1e-15, worst
    s, c = sincospi_tab(0.5, tabs)
    assert s == 1.0 and abs(c) < 1e-300
