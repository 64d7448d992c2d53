"""The radial kernel's phase reduction inside the table lookup, in exact
arithmetic.

For a record's phase rate dmh (turns per unit radius, a float) and a node's
float radius rh, the kernel forms m = fl(rh dmh + mt) with one FMA, where
mt = 1.5 * 2^16 - j/128 carries the node's dither of j table steps; the
table index is the low 7 bits of m, nk = mt - m, and the residual is
u = fl(rh dmh + nk) with a second FMA. This replays those steps with exact
rational arithmetic and float32 rounding (round to nearest, ties to even) and
checks what the kernel relies on: nk is -k/128 for an integer k, the index is
k - j mod 128, u is within half a float32 ulp of rh dmh - k/128, |u| <= 1/256
(+ that half ulp), so the pair's phase is (index + j)/128 + u turns up to
2^-33, for every |rh dmh| < 2^13, the range the kernel feeds to the lookup.
"""
from fractions import Fraction

import numpy as np
import pytest

MAGIC_TURNS = Fraction(3 * 2 ** 15)  # 1.5 * 2^16


def round_f32(x):
    """x (a Fraction) rounded to the nearest float32, ties to even."""
    if x == 0:
        return Fraction(0)
    sign = -1 if x < 0 else 1
    a = abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    ulp = Fraction(2) ** (e - 23)  # 24 significant bits (normal range only)
    return sign * round(a / ulp) * ulp


def f32(x):
    return Fraction(float(np.float32(x)))


@pytest.mark.parametrize("scale", [1e-3, 1.0, 40.0, 8191.0])
def test_lookup_steps_are_exact(scale):
    rng = np.random.default_rng(int(scale * 10) + 3)
    for _ in range(400):
        rh = f32(rng.uniform(0.0, 256.0))
        dmh = f32(rng.uniform(-1.0, 1.0) * scale / 256.0)
        j = int(rng.integers(-64, 64))
        mt = MAGIC_TURNS - Fraction(j, 128)
        assert round_f32(mt) == mt  # exact as a float
        P = rh * dmh  # the exact product inside the FMA
        assert abs(P) < 2 ** 13
        m = round_f32(P + mt)
        assert 2 ** 16 <= m < 2 ** 17  # one exponent: the float grid there is 2^-7
        bits_low = int(m * 128) % 128  # low 7 mantissa bits of m
        nk = mt - m
        assert round_f32(nk) == nk  # the subtraction is exact
        k = -nk * 128
        assert k.denominator == 1  # a whole number of table steps
        assert bits_low == (int(k) - j) % 128  # the index, moved by the dither
        u = round_f32(P + nk)  # second FMA: one rounding
        exact = P - k / 128
        assert abs(exact) <= Fraction(1, 256)
        assert abs(u - exact) <= Fraction(1, 2 ** 33)
        # the phase the table entry and the residual represent, mod 1
        phase = (Fraction(bits_low + j, 128) + u) % 1
        assert abs((phase - P % 1 + Fraction(1, 2)) % 1 - Fraction(1, 2)) <= Fraction(1, 2 ** 33)


def test_the_range_limit_is_real():
    """Past |rh dmh| = 2^15 the sum leaves the exponent where the grid is the
    table step, so the kernel must not feed such phases to the lookup (it
    switches to the reduced form at 2^13)."""
    mt = MAGIC_TURNS
    m = round_f32(Fraction(40000) + Fraction(1, 300) + mt)
    assert m >= 2 ** 17 and (m * 128).denominator == 1 and int(m * 128) % 2 == 0  # grid 2^-6: steps lost


def test_lattice_lookup_steps_are_exact():
    """The lattice kernel's variant: the record holds its phase at i = 0, t0h
    (reduced mod 1, a float), as S0 table steps inside mt0 = 1.5 * 2^16 +
    S0/128 plus t0r = t0h - S0/128; the pair's phase i rh + t0h is then table
    entry K + S0 (the low bits of fl(i rh + mt0)) plus the residual
    fl(i rh - K/128) + t0r, at most two table steps."""
    rng = np.random.default_rng(5)
    for _ in range(2000):
        t0h = f32(rng.uniform(-0.5, 0.5))
        rh = f32(rng.uniform(-1.0, 1.0))
        i = int(rng.integers(-64, 65))
        S0 = round(t0h * 128)  # rintf (ties to even) of an exact product
        mt0 = MAGIC_TURNS + Fraction(S0, 128)
        assert round_f32(mt0) == mt0
        t0r = round_f32(t0h - Fraction(S0, 128))
        assert t0r == t0h - Fraction(S0, 128) and abs(t0r) <= Fraction(1, 256)  # exact
        P = i * rh  # exact inside the FMA
        m = round_f32(P + mt0)
        idx = int(m * 128) % 128
        nk = mt0 - m
        assert round_f32(nk) == nk and (nk * 128).denominator == 1
        u = round_f32(P + nk)
        v = round_f32(u + t0r)
        assert abs(v) <= Fraction(1, 128) + Fraction(1, 2 ** 30)
        phase = (Fraction(idx, 128) + v) % 1
        assert abs((phase - (P + t0h) % 1 + Fraction(1, 2)) % 1 - Fraction(1, 2)) <= Fraction(1, 2 ** 31)
