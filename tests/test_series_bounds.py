"""The truncation bounds that the mixed kernels rely on for the centred Taylor
form of the triangle transform (Eq. simplex32_ft, Sec. 3.1).

For vertex phases t_a, t_b, t_c with centroid t_m and centred phases
y = t - t_m, F_T = gamma exp(-i t_m) Psi(y) with
Psi(y) = sum_n (-i)^n h_n(y) / (n+2)!, h_n the complete homogeneous symmetric
polynomial of degree n. The kernels keep n <= 12 while the largest gap is
below 3, the radial kernel keeps n <= 9 for whole rows whose largest gap is
below 1.5, and the lattice kernel keeps n <= 6 for whole rows whose largest
gap is below 0.6. The exact Psi comes from the oracle's long-double transform
of one triangle whose phases are the x coordinates of its vertices (xi = e_x).
"""
import math

import numpy as np
import pytest

import oracle


def h(n, y):
    a, b, c = y
    return sum(a ** i * b ** j * c ** (n - i - j) for i in range(n + 1) for j in range(n + 1 - i))


def psi_truncated(y, n_max):
    return sum((-1j) ** n * h(n, y) / math.factorial(n + 2) for n in range(n_max + 1))


@pytest.mark.parametrize("gap, n_max, bound", [(0.6, 6, 2.1e-9), (1.5, 9, 1.1e-9), (3.0, 12, 3.2e-9)])
def test_centred_series_remainder_below_the_kernel_bound(gap, n_max, bound):
    rng = np.random.default_rng(7)
    worst = 0.0
    for _ in range(300):
        t = np.sort(rng.uniform(0.0, 1.0, 3))
        t = (t - t[0]) / (t[2] - t[0]) * gap + rng.uniform(-5.0, 5.0)  # largest gap = gap
        rng.shuffle(t)
        v = np.array([[t[0], 0.0, 0.0], [t[1], 1.0, 0.0], [t[2], 0.0, 1.0]])
        tri = np.array([[0, 1, 2]], dtype=np.int32)
        gamma = np.linalg.norm(np.cross(v[1] - v[0], v[2] - v[0]))
        tm = t.mean()
        exact = oracle.mesh_ft(v, tri, np.array([[1.0, 0.0, 0.0]]))[0] * np.exp(1j * tm) / gamma
        worst = max(worst, abs(exact - psi_truncated(t - tm, n_max)))
    assert worst < bound, worst
    # and the bound is not loose by orders of magnitude: the dropped terms matter
    assert worst > bound / 20, worst
