"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

None of these re-types the oracle's own formulas: each compares it with an
independent route (brute-force quadrature in numpy, the paper's explicit
three-term formula in 40-digit mpmath, closed-form integrals, the Bessel form
of the sphere transform, exact symmetries of the rule, finite differences).
"""
import math

import mpmath
import numpy as np
import pytest
import scipy.integrate as si
import scipy.special as sp

import oracle
import synth

RNG = np.random.default_rng(12345)


def _rand_tri(scale=1.0):
    p = RNG.standard_normal((3, 3)) * scale
    return p[0], p[1], p[2]


def _brute_triangle(a, b, c, xi, order=120):
    """Duffy-collapsed tensor Gauss-Legendre quadrature of exp(-i xi.x) over the triangle."""
    g, wg = np.polynomial.legendre.leggauss(order)
    u = 0.5 * (g + 1.0)
    wu = 0.5 * wg
    U, S = np.meshgrid(u, u, indexing="ij")
    W = np.outer(wu, wu) * (1.0 - U)
    V = (1.0 - U) * S
    P = a[None, None, :] + U[..., None] * (b - a) + V[..., None] * (c - a)
    jac = np.linalg.norm(np.cross(b - a, c - a))
    return jac * (W * np.exp(-1j * (P @ xi))).sum()


def _paper_three_term(a, b, c, xi, dps=40):
    """Eq. (simplex32_ft) verbatim in the 2 pi convention at eta = xi / 2 pi."""
    with mpmath.workdps(dps):
        p = [[mpmath.mpf(float(x)) for x in v] for v in (a, b, c)]
        eta = [mpmath.mpf(float(x)) / (2 * mpmath.pi) for x in xi]
        dot = lambda u, v: sum(ui * vi for ui, vi in zip(u, v))
        e1 = [p[1][j] - p[0][j] for j in range(3)]
        e2 = [p[2][j] - p[0][j] for j in range(3)]
        cr = [e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]]
        gamma = mpmath.sqrt(dot(cr, cr))  # area ratio to the standard simplex (area 1/2)
        tot = mpmath.mpc(0)
        for i in range(3):
            den = mpmath.mpf(1)
            for j in range(3):
                if j != i:
                    den *= dot(eta, [p[i][k] - p[j][k] for k in range(3)])
            tot += mpmath.exp(-2j * mpmath.pi * dot(eta, p[i])) / den
        return complex(-gamma / (4 * mpmath.pi ** 2) * tot)


def _unit_interval_ft(k):
    """int_0^1 exp(-i k x) dx = exp(-i k/2) sin(k/2)/(k/2), via numpy's normalised sinc."""
    return np.exp(-0.5j * k) * np.sinc(k / (2 * np.pi))


# ----------------------------------------------------------------- rule
def test_gauss_legendre_matches_numpy_and_is_exact():
    for n in (1, 2, 5, 24, 48, 96, 192, 256):
        x, w = oracle.gauss_legendre(n)
        xn, wn = np.polynomial.legendre.leggauss(n)
        assert np.abs(x - xn).max() < 5e-15
        assert np.abs(w - wn).max() < 1e-13
        # exact for polynomials of degree < 2n
        for k in range(0, min(2 * n, 40), 2):
            assert abs((w * x ** k).sum() - 2.0 / (k + 1)) < 2e-14


@pytest.mark.parametrize("herm", [False, True])
def test_ball_rule_moments_are_exact(herm):
    R = 7.5
    xi, w = oracle.ball_rule(R, 12, 8, 9, herm)
    assert len(xi) == 12 * (4 if herm else 8) * 9
    vol = 4.0 / 3.0 * math.pi * R ** 3
    r2 = (xi ** 2).sum(1)
    assert abs(w.sum() - vol) < 1e-13 * vol
    assert abs((w * r2).sum() - 4 * math.pi * R ** 5 / 5) < 1e-13 * R ** 5 * 4
    for j in range(3):  # isotropy of the second moments (GL in u, trapezoid in phi)
        assert abs((w * xi[:, j] ** 2).sum() - 4 * math.pi * R ** 5 / 15) < 1e-12 * R ** 5
    assert np.abs(np.sqrt(r2)).max() <= R


def test_ball_rule_rejects_bad_descriptors():
    with pytest.raises(ValueError):
        oracle.ball_rule(8.0, 4, 5, 4, True)  # odd polar count with Hermitian halving
    with pytest.raises(ValueError):
        oracle.ball_rule(-1.0, 4, 4, 4, False)


# ----------------------------------------------------------------- triangle FT
def test_triangle_ft_at_zero_is_area():
    for _ in range(20):
        a, b, c = _rand_tri()
        area = 0.5 * np.linalg.norm(np.cross(b - a, c - a))
        f = oracle.triangle_ft(a, b, c, np.zeros(3))
        assert abs(f.real - area) <= 4.5e-16 * area and f.imag == 0.0  # numpy area: 1-2 ulp


def test_triangle_ft_matches_bruteforce_quadrature():
    for _ in range(25):
        a, b, c = _rand_tri(0.5)
        diam = max(np.linalg.norm(a - b), np.linalg.norm(b - c), np.linalg.norm(a - c))
        xi = RNG.standard_normal(3)
        xi *= RNG.uniform(0.0, 40.0) / (np.linalg.norm(xi) * diam)
        area = 0.5 * np.linalg.norm(np.cross(b - a, c - a))
        f = oracle.triangle_ft(a, b, c, xi)
        g = _brute_triangle(a, b, c, xi)
        assert abs(f - g) < 1e-13 * area, (xi, f, g)


def test_triangle_ft_matches_paper_three_term_formula():
    # generic frequencies, all phase gaps well away from zero
    for _ in range(25):
        a, b, c = _rand_tri()
        xi = RNG.standard_normal(3) * RNG.uniform(0.5, 60.0)
        area = 0.5 * np.linalg.norm(np.cross(b - a, c - a))
        f = oracle.triangle_ft(a, b, c, xi)
        g = _paper_three_term(a, b, c, xi)
        assert abs(f - g) < 1e-15 * max(area, 1.0) * 10, (f, g)


def test_square_and_cube_surface_closed_forms():
    """Two triangles tiling the unit square give the product of 1D integrals;
    twelve tiling the unit cube's surface give the sum over its six faces.
    The frequencies include exact phase coincidences (confluent nodes)."""
    o, x, y, xy = (np.array(p, dtype=float) for p in ([0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0]))
    freqs = [np.array(v, dtype=float) for v in
             ([0, 0, 0], [3, 0, 0], [0, -2, 5], [2.5, 2.5, 0], [4, -4, 1], [1e-9, 2e-9, 0],
              [1e-3, -1e-3, 0], [0.004, 0.011, 0], [17.3, -0.2, 3], [30, 30, 30], [5e-3, 5e-3, 7])]
    for xi in freqs:
        f = oracle.triangle_ft(o, x, xy, xi) + oracle.triangle_ft(o, xy, y, xi)
        g = _unit_interval_ft(xi[0]) * _unit_interval_ft(xi[1])
        assert abs(f - g) < 2e-15, (xi, f, g)
    # unit cube [0,1]^3
    verts = np.array([[i, j, k] for i in (0, 1) for j in (0, 1) for k in (0, 1)], dtype=float)
    idx = {tuple(v): n for n, v in enumerate(verts.astype(int))}
    tris = []
    for axis in range(3):
        for side in (0, 1):
            quad = []
            for (u, v) in ((0, 0), (1, 0), (1, 1), (0, 1)):
                p = [0, 0, 0]
                p[axis] = side
                p[(axis + 1) % 3] = u
                p[(axis + 2) % 3] = v
                quad.append(idx[tuple(p)])
            tris += [(quad[0], quad[1], quad[2]), (quad[0], quad[2], quad[3])]
    tris = np.array(tris, dtype=np.int32)
    xis = np.array(freqs[1:] + [np.array([0.7, -2.2, 9.1])])
    got = oracle.mesh_ft(verts, tris, xis, nthreads=1)
    for xi, f in zip(xis, got):
        I = [_unit_interval_ft(k) for k in xi]
        want = 0
        for axis in range(3):
            rest = I[(axis + 1) % 3] * I[(axis + 2) % 3]
            want += rest * (1.0 + np.exp(-1j * xi[axis]))
        assert abs(f - want) < 1e-14, (xi, f, want)


def test_triangle_ft_symmetries():
    for _ in range(10):
        a, b, c = _rand_tri()
        xi = RNG.standard_normal(3) * 8.0
        f = oracle.triangle_ft(a, b, c, xi)
        # real measure: F(-xi) = conj F(xi)
        assert abs(oracle.triangle_ft(a, b, c, -xi) - np.conj(f)) < 1e-15
        # vertex order is irrelevant (remark after the affine-simplex definition)
        for perm in ((b, c, a), (c, a, b), (b, a, c), (a, c, b), (c, b, a)):
            assert abs(oracle.triangle_ft(*perm, xi) - f) < 1e-15
        # translation x -> x + d multiplies by exp(-i xi.d)
        d = RNG.standard_normal(3)
        g = oracle.triangle_ft(a + d, b + d, c + d, xi)
        assert abs(g - np.exp(-1j * xi @ d) * f) < 1e-14
        # Eq. (simplex32_ft_orth): a shift of xi along the normal only changes the phase
        n = np.cross(b - a, c - a)
        n /= np.linalg.norm(n)
        for alpha in (0.3, 5.0, -40.0):
            h = oracle.triangle_ft(a, b, c, xi + alpha * n)
            assert abs(h - np.exp(-1j * alpha * (n @ a)) * f) < 1e-13


def test_triangle_ft_continuous_across_taylor_seam():
    """The oracle switches to the Taylor series below a phase spread of 1e-2;
    both sides of that switch must agree with brute force."""
    a, b, c = np.array([0.0, 0, 0]), np.array([1.0, 0.2, 0]), np.array([0.3, 0.9, 0.1])
    direction = np.array([0.6, -0.3, 0.74])
    # phase spread is linear in |xi|; bracket the threshold from both sides
    t = np.array([a @ direction, b @ direction, c @ direction])
    spread = t.max() - t.min()
    for target in (0.5e-2, 0.999e-2, 1.0e-2, 1.001e-2, 2e-2):
        xi = direction * target / spread
        assert abs(oracle.triangle_ft(a, b, c, xi) - _brute_triangle(a, b, c, xi, 40)) < 1e-15


def test_divided_difference_special_cases():
    G = lambda t: -np.exp(-1j * t)
    for x in (0.0, 0.7, -3.1, 250.3):
        # confluent nodes give derivatives: G[x,x] = G', G[x,x,x] = G''/2, G[x,x,x,x] = G'''/6
        assert abs(oracle.divided_difference([x, x]) - 1j * np.exp(-1j * x)) < 1e-15
        assert abs(oracle.divided_difference([x, x, x]) - np.exp(-1j * x) / 2) < 1e-15
        assert abs(oracle.divided_difference([x, x, x, x]) + 1j * np.exp(-1j * x) / 6) < 1e-15
    for _ in range(20):
        t = RNG.uniform(-20, 20, 4)
        # well-separated nodes: the explicit sums in 40-digit arithmetic
        with mpmath.workdps(40):
            tm = [mpmath.mpf(float(v)) for v in t]
            for k in (1, 2, 3):
                want = mpmath.mpc(0)
                for i in range(k + 1):
                    den = mpmath.mpf(1)
                    for j in range(k + 1):
                        if j != i:
                            den *= tm[i] - tm[j]
                    want += -mpmath.exp(-1j * tm[i]) / den
                got = oracle.divided_difference(t[: k + 1])
                assert abs(got - complex(want)) < 1e-14 * max(1.0, abs(complex(want)))
        # the derivative of G[a,b,c] in a is G[a,a,b,c] (used by the gradient)
        a, b, c = t[:3]
        eps = 1e-5
        fd = (oracle.divided_difference([a + eps, b, c]) - oracle.divided_difference([a - eps, b, c])) / (2 * eps)
        assert abs(fd - oracle.divided_difference([a, a, b, c])) < 1e-9


# ----------------------------------------------------------------- sphere
def test_sphere_ft_matches_bessel_form():
    """Eq. (ft_nsphere): 2 pi |eta|^(-1/2) J_{1/2}(2 pi |eta|) at eta = xi / 2 pi."""
    xis = RNG.standard_normal((30, 3)) * RNG.uniform(0.01, 300.0, (30, 1))
    got = oracle.sphere_ft(xis)
    for xi, f in zip(xis, got):
        eta = mpmath.mpf(float(np.linalg.norm(xi))) / (2 * mpmath.pi)
        want = 2 * mpmath.pi / mpmath.sqrt(eta) * mpmath.besselj(0.5, 2 * mpmath.pi * eta)
        assert abs(f - complex(want)) < 1e-13 and f.imag == 0.0
    assert oracle.sphere_ft(np.zeros((1, 3)))[0] == pytest.approx(4 * math.pi, rel=1e-16)


def test_sphere_ft_radius_and_center_by_surface_quadrature():
    rho, c = 0.7, np.array([0.2, -0.4, 1.1])
    g, wg = np.polynomial.legendre.leggauss(200)
    phi = 2 * np.pi * np.arange(400) / 400
    U, P = np.meshgrid(g, phi, indexing="ij")
    W = np.outer(wg, np.full(400, 2 * np.pi / 400))
    st = np.sqrt(1 - U ** 2)
    pts = c + rho * np.stack([st * np.cos(P), st * np.sin(P), U], -1)
    for xi in (np.array([1.0, 2.0, 3.0]), np.array([-20.0, 5.0, 0.5]), np.zeros(3)):
        want = rho ** 2 * (W * np.exp(-1j * (pts @ xi))).sum()
        got = oracle.sphere_ft(xi[None], rho, c)[0]
        assert abs(got - want) < 1e-12


def test_sphere_norm_one_dimensional_reduction():
    """With mu = 0 the rule sum is 64 pi^3 sum_i w_i sin^2(r_i) (1+r_i^2)^-s
    (polar weights sum to 2, azimuth weights to 2 pi), which converges to the 1D
    integral 64 pi^3 int_0^R sin^2 r (1 + r^2)^-s dr."""
    empty_v, empty_t = np.zeros((0, 3)), np.zeros((0, 3), np.int32)
    for (R, nr, npol, naz, s) in ((32.0, 96, 6, 5, 1.0), (128.0, 192, 8, 4, 2.0), (20.0, 80, 2, 1, 3.0)):
        xi, w = oracle.ball_rule(R, nr, npol, naz, False)
        d = oracle.distance(xi, w, s, empty_v, empty_t)
        q = 64 * math.pi ** 3 * si.quad(lambda r: math.sin(r) ** 2 * (1 + r * r) ** (-s), 0, R,
                                        limit=4000, epsabs=1e-300, epsrel=2e-14)[0]
        assert abs(d - q) < 2e-13 * q, (R, d, q)
        # and numpy's own Gauss-Legendre for the radial sum at the same order
        g, wg = np.polynomial.legendre.leggauss(nr)
        r = 0.5 * R * (g + 1)
        qq = 64 * math.pi ** 3 * (0.5 * R * wg * np.sin(r) ** 2 * (1 + r * r) ** (-s)).sum()
        assert abs(d - qq) < 1e-13 * qq


def test_sphere_norm_closed_form():
    """Angular-convention analogue of Eq. (sphere_sobolev_exact):
    64 pi^3 int_0^inf sin^2 r (1+r^2)^-s dr = 16 pi^(7/2)/Gamma(s) [Gamma(s-1/2) - 2 K_{s-1/2}(2)];
    the paper's own form (2 pi convention, order s_p < -1/2) is checked too."""
    for s in (1.0, 2.0, 3.0, 5.5):
        cf = 16 * math.pi ** 3.5 / sp.gamma(s) * (sp.gamma(s - 0.5) - 2 * sp.kv(s - 0.5, 2.0))
        # sin^2 = (1 - cos 2r)/2: the constant part by quad, the oscillatory part by quadosc
        a = si.quad(lambda r: 0.5 * (1 + r * r) ** (-s), 0, np.inf, epsabs=1e-300, epsrel=1e-13)[0]
        b = float(mpmath.quadosc(lambda r: 0.5 * mpmath.cos(2 * r) * (1 + r * r) ** (-s),
                                 [0, mpmath.inf], omega=2))
        assert abs(64 * math.pi ** 3 * (a - b) - cf) < 1e-11 * cf
    assert 16 * math.pi ** 4 * (1 - math.exp(-2)) == pytest.approx(
        16 * math.pi ** 3.5 * (sp.gamma(0.5) - 2 * sp.kv(0.5, 2.0)), rel=1e-14)
    for s_p in (-1.0, -2.0, -5.0, -10.0):
        cf = 4 * math.pi ** 1.5 / sp.gamma(-s_p) * (
            sp.gamma(-s_p - 0.5) - 2 * (2 * math.pi) ** (-s_p - 0.5) * sp.kv(-s_p - 0.5, 4 * math.pi))
        a = si.quad(lambda e: 8 * math.pi * (1 + e * e) ** s_p, 0, np.inf, epsabs=1e-300, epsrel=1e-13)[0]
        b = float(mpmath.quadosc(lambda e: 8 * mpmath.pi * mpmath.cos(4 * mpmath.pi * e) * (1 + e * e) ** s_p,
                                 [0, mpmath.inf], omega=4 * mpmath.pi))
        assert abs((a - b) - cf) < 1e-11 * cf


# ----------------------------------------------------------------- meshes
@pytest.mark.parametrize("herm", [False, True])
def test_cube_rule_is_the_product_trapezoid(herm):
    # Sec. 3.2, Eqs. (def_trap_grid), (trap_rule_R3): the 3-D trapezoidal rule
    # on [-xmax, xmax]^3 is the product of 1-D trapezoidal rules, so on a
    # separable (even, for the Hermitian half) integrand it equals the product
    # of numpy's 1-D trapezoid sums; nodes are 2 pi times the lattice.
    xmax, M = 1.3, 6
    xi, w = oracle.cube_rule(xmax, M, herm)
    n_full = (M + 1) ** 3
    assert len(xi) == ((n_full + 1) // 2 if herm else n_full)
    eta = xi / (2 * np.pi)
    grid = np.linspace(-xmax, xmax, M + 1)
    assert np.allclose(np.sort(np.unique(np.round(eta[:, 0], 12))), grid, atol=1e-12)
    fa = lambda x: np.cos(1.7 * x) + x ** 2  # noqa: E731
    fb = lambda y: np.exp(-0.6 * y ** 2)  # noqa: E731
    fc = lambda z: np.cosh(0.9 * z)  # noqa: E731
    lhs = np.sum(w * fa(eta[:, 0]) * fb(eta[:, 1]) * fc(eta[:, 2]))
    rhs = np.trapezoid(fa(grid), grid) * np.trapezoid(fb(grid), grid) * np.trapezoid(fc(grid), grid)
    assert lhs == pytest.approx(rhs, rel=1e-14)
    assert np.sum(w) == pytest.approx((2 * xmax) ** 3, rel=1e-14)
    if not herm:  # odd factors integrate to zero on the symmetric lattice
        assert abs(np.sum(w * eta[:, 0] * fb(eta[:, 1]))) < 1e-14


def test_cube_rule_sphere_norm_as_the_paper_reports():
    # Sec. 4.1 (Fig. 1b): with xmax = 5 the cube trapezoidal rule for the
    # unit sphere's H_s norm, against the closed form Eq.
    # (sphere_sobolev_exact), is limited by truncation at about 1e-7 for
    # s = -5, while for s = -10 it keeps converging to round-off; the paper's
    # convention is the weight (1 + |eta|^2)^s at xi = 2 pi eta.
    empty_v, empty_t = np.zeros((0, 3)), np.zeros((0, 3), dtype=np.int32)
    sphere = ("sphere", 1.0, (0.0, 0.0, 0.0))

    def rel_err(M, s_p):
        xi, w = oracle.cube_rule(5.0, M, True)
        cf = 4 * math.pi ** 1.5 / sp.gamma(-s_p) * (
            sp.gamma(-s_p - 0.5) - 2 * (2 * math.pi) ** (-s_p - 0.5) * sp.kv(-s_p - 0.5, 4 * math.pi))
        d = oracle.distance(xi, w, -s_p, empty_v, empty_t, nu=sphere, wscale=oracle.PAPER_WSCALE)
        return abs(d - cf) / cf

    e5_64, e5_128 = rel_err(64, -5.0), rel_err(128, -5.0)
    assert 1e-8 < e5_64 < 1e-7 and 1e-8 < e5_128 < 1e-7          # truncation plateau
    assert abs(e5_128 - e5_64) < 0.05 * e5_64
    assert rel_err(32, -10.0) > 1e-3 and rel_err(64, -10.0) < 1e-6  # fast convergence
    assert rel_err(128, -10.0) < 1e-12
    # the Hermitian half equals the full lattice
    xf, wf = oracle.cube_rule(5.0, 32, False)
    xh, wh = oracle.cube_rule(5.0, 32, True)
    df = oracle.distance(xf, wf, 10.0, empty_v, empty_t, nu=sphere, wscale=oracle.PAPER_WSCALE)
    dh = oracle.distance(xh, wh, 10.0, empty_v, empty_t, nu=sphere, wscale=oracle.PAPER_WSCALE)
    assert dh == pytest.approx(df, rel=1e-14)


def test_simplex_atoms_integrate_monomials_exactly():
    # Sec. 3.1 (Eq. change_variable_approx with the 8-point Gauss-Legendre rule
    # applied twice): exact for u1^a u2^b up to total degree 14, against the
    # simplex moment a! b! / (a + b + 2)!
    u1, u2, q = oracle.simplex_atoms()
    assert np.all(q > 0) and np.all(u1 > 0) and np.all(u2 > 0) and np.all(u1 + u2 < 1)
    for a in range(15):
        for b in range(15 - a):
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            assert np.sum(q * u1 ** a * u2 ** b) == pytest.approx(exact, rel=1e-13), (a, b)
    # total degree 15 is not: the outer integrand u1^a (1 - u1)^(b+1) / (b+1)
    # then has degree 16 > 2 * 8 - 1
    for a, b in ((15, 0), (8, 7), (0, 15)):
        exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
        assert abs(np.sum(q * u1 ** a * u2 ** b) - exact) > 1e-9 * exact, (a, b)


def test_atomic_transform_approaches_the_exact_one():
    # the atoms reproduce the exact triangle transform (Eq. simplex32_ft) with
    # an error falling like (|xi| h)^15: tiny at |xi| h ~ 1, visible at ~10
    v, t = synth.icosphere(2)
    h = synth.mean_edge_length(v, t)
    rng = np.random.default_rng(4)
    dirs = rng.normal(size=(8, 3))
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    errs = []
    for kh in (0.5, 2.0, 8.0, 16.0):
        xi = dirs * (kh / h)
        exact = oracle.mesh_ft(v, t, xi)
        atoms = oracle.mesh_ft_atoms(v, t, xi)
        errs.append(np.abs(atoms - exact).max() / (4 * np.pi))
    assert errs[0] < 1e-15 and errs[1] < 1e-12
    assert errs[2] < errs[3] and errs[3] > 1e-8
    # at xi = 0 the atoms give the area
    z = oracle.mesh_ft_atoms(v, t, np.zeros((1, 3)))
    assert z[0].real == pytest.approx(oracle.mesh_ft(v, t, np.zeros((1, 3)))[0].real, rel=1e-15)


def test_icosahedral_counts_and_total_area():
    for N in range(0, 5):
        v, t = synth.icosphere(2 ** N)
        assert len(v) == 10 * 4 ** N + 2 and len(t) == 20 * 4 ** N  # Sec. 4.2
    v, t = synth.icosphere(1)
    a = 1.0 / math.sin(2 * math.pi / 5)  # edge of the icosahedron inscribed in S^2
    area = 5 * math.sqrt(3) * a * a
    mu0 = oracle.mesh_ft(v, t, np.zeros((1, 3)))[0]
    assert abs(mu0 - area) < 1e-14 * area
    prev = area
    deficit = []
    for n in (2, 4, 8, 16):
        v, t = synth.icosphere(n)
        mu0 = oracle.mesh_ft(v, t, np.zeros((1, 3)))[0].real
        numpy_area = 0.5 * np.linalg.norm(np.cross(v[t[:, 1]] - v[t[:, 0]], v[t[:, 2]] - v[t[:, 0]]), axis=1).sum()
        assert abs(mu0 - numpy_area) < 1e-13 * numpy_area
        assert prev < mu0 < 4 * math.pi
        prev = mu0
        deficit.append(4 * math.pi - mu0)
    # the area deficit of an inscribed polyhedron is O(h^2) = O(n^-2)
    assert 3.5 < deficit[-2] / deficit[-1] < 4.5


def test_distance_zeros_and_rule_symmetries():
    v, t = synth.icosphere(2)
    v = synth.jitter_isotropic(v, 0.02, 3)
    xi, w = oracle.ball_rule(16.0, 16, 8, 12, False)
    assert oracle.distance(xi, w, 1.0, v, t, nu=("mesh", v, t)) == 0.0
    d = oracle.distance(xi, w, 1.0, v, t)
    # rotation by one azimuthal step permutes the nodes
    vr = v @ synth.rotation_z(2 * math.pi / 12).T
    assert abs(oracle.distance(xi, w, 1.0, vr, t) - d) < 1e-13 * d
    # reflection z -> -z maps the polar nodes onto each other
    vm = v * np.array([1.0, 1.0, -1.0])
    assert abs(oracle.distance(xi, w, 1.0, vm, t) - d) < 1e-13 * d
    # Hermitian halving gives the same sum
    xh, wh = oracle.ball_rule(16.0, 16, 8, 12, True)
    assert abs(oracle.distance(xh, wh, 1.0, v, t) - d) < 1e-13 * d
    # a general rotation only changes D by the rule's anisotropy
    vq = v @ synth.haar_rotation(5).T
    assert abs(oracle.distance(xi, w, 1.0, vq, t) - d) < 0.2 * d


def test_distance_converges_quadratically():
    """Sec. 4.2: the icosahedral error in the Sobolev norm is O(4^-N) = O(n^-2),
    so the squared distance D falls like n^-4 until truncation dominates."""
    xi, w = oracle.ball_rule(24.0, 48, 16, 32, True)
    ns = (2, 4, 8)
    ds = [oracle.distance(xi, w, 2.0, *synth.icosphere(n)) for n in ns]
    slope = np.polyfit(np.log(ns), np.log(ds), 1)[0]
    assert -4.5 < slope < -3.5, (ds, slope)


def test_gradient_matches_central_differences():
    v, t = synth.icosphere(2)
    v = synth.jitter_isotropic(v, 0.01, 0)
    xi, w = oracle.ball_rule(8.0, 12, 8, 10, True)
    d, g = oracle.distance_grad(xi, w, 1.0, v, t)
    assert d == pytest.approx(oracle.distance(xi, w, 1.0, v, t), rel=1e-15)
    h = 1e-6
    fd = np.zeros_like(v)
    for i in range(len(v)):
        for j in range(3):
            vp = v.copy()
            vm = v.copy()
            vp[i, j] += h
            vm[i, j] -= h
            fd[i, j] = (oracle.distance(xi, w, 1.0, vp, t) - oracle.distance(xi, w, 1.0, vm, t)) / (2 * h)
    assert np.linalg.norm(fd - g) < 1e-7 * np.linalg.norm(g)
    # identical measures are a minimum of D: zero gradient
    _, g0 = oracle.distance_grad(xi, w, 1.0, v, t, nu=("mesh", v, t))
    assert np.abs(g0).max() == 0.0


def _central_differences(f, v, h=1e-6):
    fd = np.zeros_like(v)
    for i in range(len(v)):
        for j in range(3):
            vp = v.copy()
            vm = v.copy()
            vp[i, j] += h
            vm[i, j] -= h
            fd[i, j] = (f(vp) - f(vm)) / (2 * h)
    return fd


@pytest.mark.parametrize("case", ["other_mesh", "shifted_sphere", "paper_lattice"])
def test_gradient_matches_central_differences_for_other_references(case):
    # The residual is zero when nu is mu itself, so that pin cannot see the
    # reference measure's part of the gradient; here nu differs from mu: a
    # second mesh, a sphere of another radius and centre, and the paper's
    # lattice with its 1/(4 pi^2) weight scale (Eqs. for the cube rule, Sec. 3.2)
    v, t = synth.icosphere(1)
    v = synth.jitter_isotropic(v, 0.02, 11)
    xi, w = oracle.ball_rule(8.0, 10, 6, 8, True)
    s, nu, wscale = 1.0, None, 1.0
    if case == "other_mesh":
        v2, t2 = synth.icosphere(2)
        nu = ("mesh", synth.jitter_isotropic(v2, 0.01, 12), t2)
    elif case == "shifted_sphere":
        nu = ("sphere", 0.9, (0.1, -0.05, 0.02))
    else:
        xi, w = oracle.cube_rule(1.5, 8, True)
        s, wscale = 2.0, oracle.PAPER_WSCALE
    d, g = oracle.distance_grad(xi, w, s, v, t, nu=nu, wscale=wscale)
    assert d == pytest.approx(oracle.distance(xi, w, s, v, t, nu=nu, wscale=wscale), rel=1e-15)
    fd = _central_differences(lambda x: oracle.distance(xi, w, s, x, t, nu=nu, wscale=wscale), v)
    assert np.linalg.norm(fd - g) < 1e-7 * np.linalg.norm(g)


def test_invalid_mesh_is_rejected():
    v, t = synth.icosphere(1)
    bad = t.copy()
    bad[3, 1] = len(v)
    with pytest.raises(ValueError):
        oracle.mesh_ft(v, bad, np.zeros((1, 3)))
