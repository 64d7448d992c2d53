"""The residual polynomials of the mixed kernels' table exponential.

exp(-2 pi i tau) is a table entry (128 steps per turn) times exp(-2 pi i v)
for a residual v in turns; the kernels evaluate cos(2 pi v) - 1 and
sin(2 pi v) as short polynomials in v whose leading constants are float
pairs (`expm_residual` for |v| <= 1/256 + a few 2^-24, `expm_residual_wide`
for |v| <= 1/128 + a few 2^-24 in the lattice kernel). This reads the
constants from the CUDA header and checks them against the mathematics: the
float pairs add up to (2 pi)^2 / 2 and 2 pi, the other coefficients are the
Taylor coefficients to float precision, the truncation errors stay below the
bounds the header states (7.5e-11 and 1.5e-13), and so does the whole error
with the float coefficients, up to their own rounding. A wrong digit in any
coefficient fails one of these.
"""
import math
import os
import re

import numpy as np
import pytest

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2304_06340_b300", "csrc",
                      "wd_math.cuh")
TWO_PI = 2.0 * math.pi


def function_body(name):
    src = open(HEADER).read()
    i = src.index("void %s(" % name)
    return src[i:src.index("\n}\n", i)]


def float_literals(body, pattern):
    """The float32 values of the `f` literals that pattern captures."""
    m = re.search(pattern, body, re.S)
    assert m, pattern
    return [float(np.float32(float(x.rstrip("f")))) for x in m.groups()]


def constants(name):
    body = function_body(name)
    num = r"(-?[0-9.]+(?:e[-+]?[0-9]+)?f)"
    if name == "expm_residual":
        c2h, c4, c2l = float_literals(body, r"dc = fmaf\(v2, %s, v2 \* fmaf\(v2, %s, %s\)\)" % (num, num, num))
        s1h, s3, s1l = float_literals(body, r"sx = fmaf\(v, %s, v \* fmaf\(v2, %s, %s\)\)" % (num, num, num))
        return {"c2": (c2h, c2l), "c4": c4, "c6": 0.0, "s1": (s1h, s1l), "s3": s3, "s5": 0.0}
    c2h, c6, c4, c2l = float_literals(
        body, r"dc = fmaf\(v2, %s,\s*v2 \* fmaf\(v2, fmaf\(v2, %s, %s\), %s\)\)" % (num, num, num, num))
    s1h, s5, s3, s1l = float_literals(
        body, r"sx = fmaf\(v, %s,\s*v \* fmaf\(v2, fmaf\(v2, %s, %s\), %s\)\)" % (num, num, num, num))
    return {"c2": (c2h, c2l), "c4": c4, "c6": c6, "s1": (s1h, s1l), "s3": s3, "s5": s5}


@pytest.mark.parametrize("name", ["expm_residual", "expm_residual_wide"])
def test_leading_constants_are_exact_float_pairs(name):
    k = constants(name)
    c2h, c2l = k["c2"]
    s1h, s1l = k["s1"]
    # high + low is the constant to about 2^-48 (the low part is itself a float)
    assert abs((c2h + c2l) - (-TWO_PI ** 2 / 2)) < 1e-14 * TWO_PI ** 2
    assert abs((s1h + s1l) - TWO_PI) < 1e-14 * TWO_PI
    # the low parts carry what the float high part misses (2.9e-8 and 2.8e-8 relative)
    assert abs(c2l) > 1e-8 * TWO_PI ** 2 / 2 and abs(s1l) > 1e-8 * TWO_PI


@pytest.mark.parametrize("name", ["expm_residual", "expm_residual_wide"])
def test_higher_coefficients_are_the_taylor_coefficients(name):
    k = constants(name)
    assert abs(k["c4"] - TWO_PI ** 4 / 24) < 1e-7 * TWO_PI ** 4 / 24
    assert abs(k["s3"] - (-TWO_PI ** 3 / 6)) < 1e-7 * TWO_PI ** 3 / 6
    if name == "expm_residual_wide":
        assert abs(k["c6"] - (-TWO_PI ** 6 / 720)) < 1e-7 * TWO_PI ** 6 / 720
        assert abs(k["s5"] - TWO_PI ** 5 / 120) < 1e-7 * TWO_PI ** 5 / 120


@pytest.mark.parametrize("name, vmax, trunc, total", [("expm_residual", 1.0 / 256 + 1e-6, 7.5e-11, 7.6e-11),
                                                      ("expm_residual_wide", 1.0 / 128 + 1e-6, 1.5e-13, 1e-12)])
def test_truncation_below_the_stated_bound(name, vmax, trunc, total):
    k = constants(name)
    wide = name == "expm_residual_wide"
    v = np.linspace(-vmax, vmax, 20001)
    v2 = v * v
    exact_c, exact_s = np.cos(TWO_PI * v) - 1.0, np.sin(TWO_PI * v)
    # truncation alone: the exact Taylor coefficients cut where the kernel cuts
    c4, s3 = TWO_PI ** 4 / 24, -TWO_PI ** 3 / 6
    c6, s5 = (-TWO_PI ** 6 / 720, TWO_PI ** 5 / 120) if wide else (0.0, 0.0)
    err_c = np.abs(v2 * (-TWO_PI ** 2 / 2 + v2 * (c4 + v2 * c6)) - exact_c).max()
    err_s = np.abs(v * (TWO_PI + v2 * (s3 + v2 * s5)) - exact_s).max()
    assert err_c < trunc and err_s < trunc, (err_c, err_s)
    # with the kernel's float coefficients (their rounding adds up to 6e-13 in
    # the wide form, through the cubic term), still far below the 6e-8 rounding
    # of the result
    dc = v2 * (sum(k["c2"]) + v2 * (k["c4"] + v2 * k["c6"]))
    sx = v * (sum(k["s1"]) + v2 * (k["s3"] + v2 * k["s5"]))
    err_c, err_s = np.abs(dc - exact_c).max(), np.abs(sx - exact_s).max()
    assert err_c < total and err_s < total, (err_c, err_s)
    # and the polynomials are not trivially accurate: dropping the last cosine term fails
    last = v2 * v2 * (v2 * k["c6"] if wide else k["c4"])
    assert np.abs(dc - last - exact_c).max() > 10 * trunc
