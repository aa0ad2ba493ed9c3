"""The constant tables build.py writes for the kernels, checked against their
definitions by independent means (the math library, exact rational arithmetic,
identities the values must satisfy).  No GPU needed."""
import math
import re
from fractions import Fraction

import numpy as np

from paper_2404_08867_gb300 import build


def _hex_values(src, name):
    body = src.split(name, 1)[1].split("};", 1)[0]
    return [float.fromhex(v) for v in re.findall(r"(-?0x[0-9a-fA-Fp.+-]+),", body)]


def test_cheb_table_matches_its_definition():
    src = build.cheb_table_source()
    xs = _hex_values(src, "kChebXiGen")
    ws = _hex_values(src, "kChebBwGen")
    assert len(xs) == len(ws) == 32 * 33 // 2
    for P in range(1, 33):
        off = P * (P - 1) // 2
        for p in range(P):
            th = math.pi * (2 * p + 1) / (2 * P)
            # within the libm values' own error: theta rounded to double moves cos and
            # sin by up to ulp(pi) = 4.4e-16, and 1 + cos loses up to half an ulp of 1
            assert abs(xs[off + p] - 0.5 * (1.0 + math.cos(th))) <= 6.7e-16
            assert abs(ws[off + p] - (-1) ** p * math.sin(th)) <= 6.7e-16
            # first-kind points lie strictly inside (0, 1), in decreasing order
            assert 0.0 < xs[off + p] < 1.0
            if p:
                assert xs[off + p] < xs[off + p - 1]
        # mirror symmetry xi_{P-1-p} = 1 - xi_p of the exact points, to rounding
        for p in range(P):
            assert abs(xs[off + p] + xs[off + P - 1 - p] - 1.0) <= 2.3e-16


def test_cheb_table_is_correctly_rounded_where_exact():
    # cos(pi/4) = sqrt(2)/2 (P = 2, p = 0): the node (1 + sqrt(2)/2)/2 rounded once;
    # P = 1: xi = 1/2, weight 1; P = 3, p = 1: theta = pi/2, xi = 1/2, weight -1.
    src = build.cheb_table_source()
    xs = _hex_values(src, "kChebXiGen")
    ws = _hex_values(src, "kChebBwGen")
    assert xs[0] == 0.5 and ws[0] == 1.0
    assert xs[3 + 1] == 0.5 and ws[3 + 1] == -1.0
    # sqrt(2)/2 to 40 digits, then (1 + s)/2, rounded to nearest double by Fraction
    s = Fraction(7071067811865475244008443621048490392848, 10 ** 40)
    assert xs[1] == float((1 + s) / 2)
    assert ws[1] == float(s)


def test_cheb_table_interpolates_polynomials():
    # With these points and weights the barycentric formula reproduces a polynomial
    # of degree < P to rounding (the defining property of the weights).
    src = build.cheb_table_source()
    xs = np.array(_hex_values(src, "kChebXiGen"))
    ws = np.array(_hex_values(src, "kChebBwGen"))
    rng = np.random.default_rng(5)
    for P in (2, 8, 16, 32):
        off = P * (P - 1) // 2
        x, w = xs[off:off + P], ws[off:off + P]
        coef = rng.standard_normal(P)
        f = np.polynomial.polynomial.polyval(x, coef)
        for u in rng.random(7):
            r = w / (u - x)
            got = np.dot(r, f) / r.sum()
            want = np.polynomial.polynomial.polyval(u, coef)
            assert abs(got - want) <= 1e-12 * max(1.0, np.abs(coef).sum())


def test_exp64_constants():
    src = build.exp64_constants_source()
    T = _hex_values(src, "kExp2TableD")
    assert len(T) == 256
    for j in range(256):
        assert abs(T[j] - 2.0 ** (j / 256.0)) <= 2.3e-16 * T[j]
    l1 = float.fromhex(re.search(r"kExp64L1 = (\S+);", src).group(1))
    l2 = float.fromhex(re.search(r"kExp64L2 = (\S+);", src).group(1))
    # L1 has at most 33 significant bits, so n L1 is exact for |n| < 2^20
    m, e = math.frexp(l1)
    assert (Fraction(m) * 2 ** 33).denominator == 1
    assert abs((l1 + l2) - math.log(2) / 256) <= 1e-18
