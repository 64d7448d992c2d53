/*
 * wd_oracle.c -- plain, slow CPU oracle for the H^{-s} weak distance between a
 * triangulated surface and a reference measure (Koga, "Computing weak distance
 * between the 2-sphere and its nonsmooth approximations", arXiv 2304.06340).
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark load this file's library. It shares no source, header,
 * table or helper with the CUDA library, and the CUDA library never loads it.
 *
 * Everything is evaluated in x87 long double (64-bit mantissa) and returned
 * rounded to double. Conventions (angular Fourier transform, the paper's Eq.
 * (ft_measure) with xi -> xi / 2pi):
 *
 *   mu^(xi) = int exp(-i xi.x) dmu(x)
 *   D       = sum_k W_k |mu^(xi_k) - nu^(xi_k)|^2,  W_k = w_k (1 + |xi_k|^2)^(-s)
 *
 * which is the ball-truncated quadrature of the Plancherel form of the squared
 * Sobolev norm, Eq. (sobolev_2), with order -s and no (2 pi)^-3 factor.
 *
 * or_cube_rule gives the paper's own lattice rule in its 2 pi convention; the
 * weighted sums take a weight scale for it (see weight_ld).
 *
 * Parity status of every function is stated in its comment; the pins live in
 * tests/test_oracle_pins.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef long double ld;

#define OR_PI 3.141592653589793238462643383279502884L

/* ------------------------------------------------------------------ */
/* Gauss-Legendre rule on [-1, 1] (used for the radial and polar factors of the
 * ball rule, Sec. 3.2 closing remark on ball-centred rules). Newton iteration on
 * P_n evaluated by the three-term recurrence, started from the asymptotic guess
 * cos(pi (i - 1/4) / (n + 1/2)). Nodes ascending.
 * Pinned against numpy.polynomial.legendre.leggauss and polynomial exactness. */
int or_gauss_legendre(int n, double* x_out, double* w_out)
{
    if (n < 1) return -1;
    for (int i = 1; i <= n; ++i) {
        ld x = cosl(OR_PI * ((ld)i - 0.25L) / ((ld)n + 0.5L));
        ld dp = 0.0L;
        for (int it = 0; it < 100; ++it) {
            ld p0 = 1.0L, p1 = x;
            for (int k = 1; k < n; ++k) {
                ld p2 = ((2.0L * k + 1.0L) * x * p1 - (ld)k * p0) / ((ld)k + 1.0L);
                p0 = p1;
                p1 = p2;
            }
            /* p1 = P_n(x), p0 = P_{n-1}(x) */
            dp = (ld)n * (x * p1 - p0) / (x * x - 1.0L);
            ld dx = p1 / dp;
            x -= dx;
            if (fabsl(dx) < 1e-19L) break;
        }
        {   /* derivative at the converged node */
            ld p0 = 1.0L, p1 = x;
            for (int k = 1; k < n; ++k) {
                ld p2 = ((2.0L * k + 1.0L) * x * p1 - (ld)k * p0) / ((ld)k + 1.0L);
                p0 = p1;
                p1 = p2;
            }
            dp = (ld)n * (x * p1 - p0) / (x * x - 1.0L);
        }
        /* i = 1 is the largest node; store ascending */
        x_out[n - i] = (double)x;
        w_out[n - i] = (double)(2.0L / ((1.0L - x * x) * dp * dp));
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Cube trapezoid rule of the paper's experiments (Sec. 3.2, the lattice of
 * Eq. (def_trap_grid) with the three-dimensional trapezoidal rule of Eq.
 * (trap_rule_R3)), in the paper's 2 pi convention: eta_{ijk} = (i, j, k) h,
 * h = 2 xmax / M, i, j, k = -M/2 .. M/2, weight h^3 times 1/2 per coordinate
 * on the boundary (1 inside, 1/2 on faces, 1/4 on edges, 1/8 at corners).
 * The nodes are returned in the angular convention, xi = 2 pi eta, so that
 * mu^(xi) is the paper's transform at eta; the paper's weight
 * (1 + |eta|^2)^(-s) is (1 + wscale |xi|^2)^(-s) with wscale = 1/(4 pi^2).
 * With `hermitian`, the half eta_z > 0, or eta_z = 0 and eta_y > 0, or
 * eta_z = eta_y = 0 and eta_x >= 0 is kept, every node but the origin with
 * doubled weight. Node order: k outermost, then j, then i (fastest).
 * Returns the node count, or -1 on invalid arguments (M even, >= 2). */
int64_t or_cube_rule(double xmax, int M, int hermitian, double* xi, double* w_geom)
{
    if (!(xmax > 0.0) || M < 2 || (M % 2)) return -1;
    const int m = M / 2;
    const ld h = 2.0L * (ld)xmax / (ld)M;
    int64_t cnt = 0;
    for (int k = hermitian ? 0 : -m; k <= m; ++k)
        for (int j = -m; j <= m; ++j)
            for (int i = -m; i <= m; ++i) {
                if (hermitian && (k == 0) && (j < 0 || (j == 0 && i < 0))) continue;
                if (xi) {
                    const ld fi = (i == m || i == -m) ? 0.5L : 1.0L;
                    const ld fj = (j == m || j == -m) ? 0.5L : 1.0L;
                    const ld fk = (k == m || k == -m) ? 0.5L : 1.0L;
                    const int origin = (i == 0 && j == 0 && k == 0);
                    const ld dup = (hermitian && !origin) ? 2.0L : 1.0L;
                    xi[3 * cnt] = (double)(2.0L * OR_PI * h * i);
                    xi[3 * cnt + 1] = (double)(2.0L * OR_PI * h * j);
                    xi[3 * cnt + 2] = (double)(2.0L * OR_PI * h * k);
                    w_geom[cnt] = (double)(h * h * h * fi * fj * fk * dup);
                }
                ++cnt;
            }
    return cnt;
}

/* ------------------------------------------------------------------ */
/* Ball rule |xi| <= R in spherical coordinates:
 *   r   = Gauss-Legendre on [0, R]           (n_r nodes, weight includes r^2)
 *   u   = cos(theta), Gauss-Legendre on [-1,1] (n_polar nodes)
 *   phi = 2 pi k / n_azim, trapezoid         (weight 2 pi / n_azim)
 *   xi  = r (sqrt(1-u^2) cos phi, sqrt(1-u^2) sin phi, u)
 * With `hermitian`, only u > 0 is kept and its weight doubled: the integrand
 * |mu^ - nu^|^2 is even in xi for real measures (mu^(-xi) = conj mu^(xi)).
 * Node order: r outermost, then u ascending, then phi (fastest).
 * Returns the node count, or -1 on invalid arguments. xi is n x 3 (AoS). */
int64_t or_ball_rule(double R, int n_r, int n_polar, int n_azim, int hermitian,
                     double* xi, double* w_geom)
{
    if (!(R > 0.0) || n_r < 1 || n_polar < 1 || n_azim < 1) return -1;
    if (hermitian && (n_polar % 2)) return -1;
    double* xr = malloc(sizeof(double) * n_r);
    double* wr = malloc(sizeof(double) * n_r);
    double* xu = malloc(sizeof(double) * n_polar);
    double* wu = malloc(sizeof(double) * n_polar);
    or_gauss_legendre(n_r, xr, wr);
    or_gauss_legendre(n_polar, xu, wu);
    int64_t k = 0;
    for (int i = 0; i < n_r; ++i) {
        ld r = 0.5L * (ld)R * (1.0L + (ld)xr[i]);
        ld wrr = 0.5L * (ld)R * (ld)wr[i] * r * r;
        for (int j = 0; j < n_polar; ++j) {
            ld u = (ld)xu[j];
            if (hermitian && !(u > 0.0L)) continue;
            ld wuu = (ld)wu[j] * (hermitian ? 2.0L : 1.0L);
            ld st = sqrtl(1.0L - u * u);
            for (int m = 0; m < n_azim; ++m) {
                ld ph = 2.0L * OR_PI * (ld)m / (ld)n_azim;
                if (xi) {
                    xi[3 * k + 0] = (double)(r * st * cosl(ph));
                    xi[3 * k + 1] = (double)(r * st * sinl(ph));
                    xi[3 * k + 2] = (double)(r * u);
                }
                if (w_geom) w_geom[k] = (double)(wrr * wuu * 2.0L * OR_PI / (ld)n_azim);
                ++k;
            }
        }
    }
    free(xr); free(wr); free(xu); free(wu);
    return k;
}

/* ------------------------------------------------------------------ */
/* Divided differences of G(t) = -exp(-i t).
 *
 * The Fourier transform of the surface measure of a triangle with vertices
 * a, b, c (Eq. (simplex32_ft), angular convention) is
 *     F(xi) = gamma * G[t_a, t_b, t_c],   t_v = xi . v,
 *     gamma = |(b - a) x (c - a)| = area ratio to the standard simplex,
 * because by the Hermite-Genocchi formula the second divided difference of G
 * is the integral of G'' = exp(-i t) over the standard simplex, which is the
 * change of variables of Eq. (change_variable). The explicit three-term form
 * of Eq. (simplex32_ft) is the same divided difference written out; here it is
 * evaluated by the divided-difference recurrence, whose first-order step has
 * the exact closed form
 *     G[x, y] = i exp(-i (x + y)/2) sinc((y - x)/2),
 * and, when all nodes are within TAYLOR_GAP, by the Taylor series about their
 * mean c (y_j = x_j - c, h_n the complete homogeneous symmetric polynomial):
 *     G[x_0..x_k] = -(-i)^k exp(-i c) sum_n (-i)^n h_n(y) / (n + k)!
 */
#define TAYLOR_GAP 1e-2L
#define TAYLOR_TERMS 14

static void cmul(ld ar, ld ai, ld br, ld bi, ld* cr, ld* ci)
{
    *cr = ar * br - ai * bi;
    *ci = ar * bi + ai * br;
}

/* complete homogeneous symmetric polynomial of degree n in y[0..m-1] */
static ld hpoly(int n, const ld* y, int m)
{
    if (m == 1) {
        ld p = 1.0L;
        for (int j = 0; j < n; ++j) p *= y[0];
        return p;
    }
    ld s = 0.0L, p = 1.0L;
    for (int j = 0; j <= n; ++j) {
        s += p * hpoly(n - j, y + 1, m - 1);
        p *= y[0];
    }
    return s;
}

static ld factl(int n)
{
    ld f = 1.0L;
    for (int j = 2; j <= n; ++j) f *= (ld)j;
    return f;
}

/* (-i)^p as (re, im) */
static void mipow(int p, ld* re, ld* im)
{
    switch (((p % 4) + 4) % 4) {
    case 0: *re = 1; *im = 0; break;
    case 1: *re = 0; *im = -1; break;
    case 2: *re = -1; *im = 0; break;
    default: *re = 0; *im = 1; break;
    }
}

static void dd_taylor(const ld* x, int k, ld* re, ld* im)
{
    ld c = 0.0L;
    for (int j = 0; j <= k; ++j) c += x[j];
    c /= (ld)(k + 1);
    ld y[8];
    for (int j = 0; j <= k; ++j) y[j] = x[j] - c;
    ld sr = 0.0L, si = 0.0L;
    for (int n = 0; n <= TAYLOR_TERMS; ++n) {
        ld pr, pi;
        mipow(n, &pr, &pi);
        ld t = hpoly(n, y, k + 1) / factl(n + k);
        sr += pr * t;
        si += pi * t;
    }
    /* prefactor -(-i)^k exp(-i c) */
    ld kr, ki, er = cosl(c), ei = -sinl(c), fr, fi;
    mipow(k, &kr, &ki);
    cmul(-kr, -ki, er, ei, &fr, &fi);
    cmul(fr, fi, sr, si, re, im);
}

static void sort_ld(ld* x, int n)
{
    for (int i = 1; i < n; ++i)
        for (int j = i; j > 0 && x[j - 1] > x[j]; --j) {
            ld t = x[j]; x[j] = x[j - 1]; x[j - 1] = t;
        }
}

/* G[x_0..x_k] for k = 1, 2, 3 (order of the nodes is irrelevant) */
static void dd(const ld* xin, int k, ld* re, ld* im)
{
    ld x[8];
    memcpy(x, xin, sizeof(ld) * (k + 1));
    sort_ld(x, k + 1);
    if (k == 1) {
        ld h = 0.5L * (x[1] - x[0]), m = 0.5L * (x[0] + x[1]);
        ld sc = (h == 0.0L) ? 1.0L : sinl(h) / h;
        *re = sinl(m) * sc; /* i (cos m - i sin m) = sin m + i cos m */
        *im = cosl(m) * sc;
        return;
    }
    ld spread = x[k] - x[0];
    if (spread < TAYLOR_GAP) {
        dd_taylor(x, k, re, im);
        return;
    }
    ld ar, ai, br, bi;
    dd(x + 1, k - 1, &ar, &ai); /* G[x_1..x_k] */
    dd(x, k - 1, &br, &bi);     /* G[x_0..x_{k-1}] */
    *re = (ar - br) / spread;
    *im = (ai - bi) / spread;
}

static ld dotl(const double* a, const double* b)
{
    return (ld)a[0] * b[0] + (ld)a[1] * b[1] + (ld)a[2] * b[2];
}

/* gamma = |(b - a) x (c - a)| and the unit normal, in long double */
static ld tri_gamma(const double* a, const double* b, const double* c, ld* nrm)
{
    ld e1[3], e2[3], n[3];
    for (int j = 0; j < 3; ++j) { e1[j] = (ld)b[j] - a[j]; e2[j] = (ld)c[j] - a[j]; }
    n[0] = e1[1] * e2[2] - e1[2] * e2[1];
    n[1] = e1[2] * e2[0] - e1[0] * e2[2];
    n[2] = e1[0] * e2[1] - e1[1] * e2[0];
    ld g = sqrtl(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    if (nrm) for (int j = 0; j < 3; ++j) nrm[j] = g > 0 ? n[j] / g : 0.0L;
    return g;
}

/* Fourier transform of one triangle's surface measure at xi, Eq. (simplex32_ft). */
static void tri_ft_ld(const double* a, const double* b, const double* c, const double* xi,
                      ld* re, ld* im)
{
    ld g = tri_gamma(a, b, c, NULL);
    ld t[3] = {dotl(xi, a), dotl(xi, b), dotl(xi, c)};
    ld gr, gi;
    dd(t, 2, &gr, &gi);
    *re = g * gr;
    *im = g * gi;
}

void or_triangle_ft(const double* a, const double* b, const double* c, const double* xi,
                    double* re, double* im)
{
    ld r, i;
    tri_ft_ld(a, b, c, xi, &r, &i);
    *re = (double)r;
    *im = (double)i;
}

/* G[t_0, .., t_k] for external tests of the divided-difference machinery. */
void or_divided_difference(const double* t, int k, double* re, double* im)
{
    ld x[8], r, i;
    for (int j = 0; j <= k; ++j) x[j] = t[j];
    dd(x, k, &r, &i);
    *re = (double)r;
    *im = (double)i;
}

/* ------------------------------------------------------------------ */
/* Mesh Fourier transform: mu^(xi) = sum_T F_T(xi) (linearity, Sec. 3.1). */
static void mesh_ft_node_ld(const double* verts, const int32_t* tris, int64_t nt,
                            const double* xi, ld* re, ld* im)
{
    ld sr = 0.0L, si = 0.0L;
    for (int64_t t = 0; t < nt; ++t) {
        ld fr, fi;
        tri_ft_ld(verts + 3 * (int64_t)tris[3 * t], verts + 3 * (int64_t)tris[3 * t + 1],
                  verts + 3 * (int64_t)tris[3 * t + 2], xi, &fr, &fi);
        sr += fr;
        si += fi;
    }
    *re = sr;
    *im = si;
}

static int mesh_ok(int64_t nv, const int32_t* tris, int64_t nt)
{
    for (int64_t j = 0; j < 3 * nt; ++j)
        if (tris[j] < 0 || tris[j] >= nv) return 0;
    return 1;
}

int or_mesh_ft(const double* verts, int64_t nv, const int32_t* tris, int64_t nt,
               const double* xi, int64_t n, double* re, double* im, int nthreads)
{
    if (!mesh_ok(nv, tris, nt)) return -1;
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
    for (int64_t k = 0; k < n; ++k) {
        ld r, i;
        mesh_ft_node_ld(verts, tris, nt, xi + 3 * k, &r, &i);
        re[k] = (double)r;
        im[k] = (double)i;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* The paper's atomic approximation of a triangle's surface measure (Sec. 3.1,
 * Eqs. (change_variable), (change_variable_approx)): the 8-point Gauss-Legendre
 * rule applied twice to the standard simplex Q_0 = {u1, u2 >= 0, u1 + u2 <= 1}
 * as the iterated integral of u2 over [0, 1 - u1] inside u1 over [0, 1]:
 * 64 atoms u = (x_i, (1 - x_i) x_j) with weights q = w_i w_j (1 - x_i), where
 * (x, w) is the Gauss-Legendre rule moved to [0, 1]. On a triangle (a, b, c)
 * they sit at a + u1 (b - a) + u2 (c - a) with weights q gamma.
 * Writes the 64 atoms of Q_0 (u1, u2, q); returns 0.
 * Pinned against the exact simplex moments: u1^a u2^b integrates to
 * a! b! / (a + b + 2)!, exactly for a + b <= 14. */
int or_simplex_atoms(double* u1, double* u2, double* q)
{
    double x[8], w[8];
    if (or_gauss_legendre(8, x, w) != 0) return -1;
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) {
            const ld xi = 0.5L * (1.0L + (ld)x[i]), wi = 0.5L * (ld)w[i];
            const ld xj = 0.5L * (1.0L + (ld)x[j]), wj = 0.5L * (ld)w[j];
            u1[8 * i + j] = (double)xi;
            u2[8 * i + j] = (double)((1.0L - xi) * xj);
            q[8 * i + j] = (double)(wi * wj * (1.0L - xi));
        }
    return 0;
}

/* mu^ of the atomic approximation above, sum over triangles and atoms of
 * q gamma exp(-i xi.x), at n nodes (long double sums). */
int or_mesh_ft_atoms(const double* verts, int64_t nv, const int32_t* tris, int64_t nt,
                     const double* xi, int64_t n, double* re, double* im, int nthreads)
{
    if (!mesh_ok(nv, tris, nt)) return -1;
    double u1[64], u2[64], q[64];
    or_simplex_atoms(u1, u2, q);
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
    for (int64_t k = 0; k < n; ++k) {
        const double* x = xi + 3 * k;
        ld sr = 0.0L, si = 0.0L;
        for (int64_t t = 0; t < nt; ++t) {
            const double* a = verts + 3 * (int64_t)tris[3 * t];
            const double* b = verts + 3 * (int64_t)tris[3 * t + 1];
            const double* c = verts + 3 * (int64_t)tris[3 * t + 2];
            const ld g = tri_gamma(a, b, c, NULL);
            const ld ta = dotl(x, a), tb = dotl(x, b), tc = dotl(x, c);
            for (int m = 0; m < 64; ++m) {
                const ld ph = ta + (ld)u1[m] * (tb - ta) + (ld)u2[m] * (tc - ta);
                sr += g * (ld)q[m] * cosl(ph);
                si -= g * (ld)q[m] * sinl(ph);
            }
        }
        re[k] = (double)sr;
        im[k] = (double)si;
    }
    return 0;
}

/* Sphere of radius rho centred at c: nu^(xi) = 4 pi rho sin(rho |xi|)/|xi| exp(-i xi.c),
 * Eq. (ft_nsphere_sinc) in the angular convention, scaled and translated. */
static void sphere_ft_ld(const double* xi, double rho, const double* c, ld* re, ld* im)
{
    ld r = sqrtl(dotl(xi, xi));
    ld a = (r == 0.0L) ? 4.0L * OR_PI * (ld)rho * rho
                       : 4.0L * OR_PI * (ld)rho * sinl((ld)rho * r) / r;
    ld ph = c ? dotl(xi, c) : 0.0L;
    *re = a * cosl(ph);
    *im = -a * sinl(ph);
}

void or_sphere_ft(const double* xi, int64_t n, double rho, const double* c, double* re, double* im)
{
    for (int64_t k = 0; k < n; ++k) {
        ld r, i;
        sphere_ft_ld(xi + 3 * k, rho, c, &r, &i);
        re[k] = (double)r;
        im[k] = (double)i;
    }
}

/* ------------------------------------------------------------------ */
/* Reference measure nu: kind 0 = sphere (radius, center), kind 1 = second mesh. */
typedef struct {
    int kind;
    double radius;
    const double* center;
    const double* verts;
    int64_t nv;
    const int32_t* tris;
    int64_t nt;
} nu_desc;

static void nu_ft_ld(const nu_desc* nu, const double* xi, ld* re, ld* im)
{
    if (nu->kind == 0) sphere_ft_ld(xi, nu->radius, nu->center, re, im);
    else mesh_ft_node_ld(nu->verts, nu->tris, nu->nt, xi, re, im);
}

/* W = w (1 + wscale |xi|^2)^(-s): wscale = 1 in the angular convention, and
 * 1/(4 pi^2) for the paper's (1 + |eta|^2)^(-s) at xi = 2 pi eta. */
static ld weight_ld(const double* xi, double w_geom, double s, double wscale)
{
    return (ld)w_geom * powl(1.0L + (ld)wscale * dotl(xi, xi), -(ld)s);
}

/* D = sum_k W_k |mu^ - nu^|^2 over explicit nodes (Eq. (sobolev_2) as a
 * quadrature sum). Optional per-node outputs of mu^ (may be NULL). */
double or_distance(const double* xi, const double* w_geom, int64_t n, double s, double wscale,
                   const double* verts, int64_t nv, const int32_t* tris, int64_t nt,
                   int nu_kind, double radius, const double* center,
                   const double* verts2, int64_t nv2, const int32_t* tris2, int64_t nt2,
                   double* mu_re, double* mu_im, int nthreads)
{
    if (!mesh_ok(nv, tris, nt)) return NAN;
    if (nu_kind == 1 && !mesh_ok(nv2, tris2, nt2)) return NAN;
    nu_desc nu = {nu_kind, radius, center, verts2, nv2, tris2, nt2};
    ld* term = malloc(sizeof(ld) * (n > 0 ? n : 1));
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
    for (int64_t k = 0; k < n; ++k) {
        ld mr, mi, vr, vi;
        mesh_ft_node_ld(verts, tris, nt, xi + 3 * k, &mr, &mi);
        nu_ft_ld(&nu, xi + 3 * k, &vr, &vi);
        ld dr = mr - vr, di = mi - vi;
        term[k] = weight_ld(xi + 3 * k, w_geom[k], s, wscale) * (dr * dr + di * di);
        if (mu_re) mu_re[k] = (double)mr;
        if (mu_im) mu_im[k] = (double)mi;
    }
    ld d = 0.0L;
    for (int64_t k = 0; k < n; ++k) d += term[k];
    free(term);
    return (double)d;
}

/* ------------------------------------------------------------------ */
/* Gradient of D with respect to the vertices of mu:
 *   dD/dv = sum_k 2 W_k Re( conj(mu^ - nu^)(xi_k) * d mu^(xi_k)/dv ),
 *   dF_T/da = (d gamma/da) G[t_a,t_b,t_c] + gamma G[t_a,t_a,t_b,t_c] xi,
 *   d gamma/da = (b - c) x n,  d gamma/db = (c - a) x n,  d gamma/dc = (a - b) x n,
 * n the unit normal of (b - a) x (c - a); the derivative of a divided
 * difference in one node is the divided difference with that node repeated.
 * A degenerate triangle (gamma = 0) contributes zero. grad is nv x 3. */
double or_distance_grad(const double* xi, const double* w_geom, int64_t n, double s, double wscale,
                        const double* verts, int64_t nv, const int32_t* tris, int64_t nt,
                        int nu_kind, double radius, const double* center,
                        const double* verts2, int64_t nv2, const int32_t* tris2, int64_t nt2,
                        double* grad, int nthreads)
{
    if (!mesh_ok(nv, tris, nt)) return NAN;
    if (nu_kind == 1 && !mesh_ok(nv2, tris2, nt2)) return NAN;
    nu_desc nu = {nu_kind, radius, center, verts2, nv2, tris2, nt2};
    ld* res_r = malloc(sizeof(ld) * (n > 0 ? n : 1)); /* 2 W (mu^ - nu^) */
    ld* res_i = malloc(sizeof(ld) * (n > 0 ? n : 1));
    ld* term = malloc(sizeof(ld) * (n > 0 ? n : 1));
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
    for (int64_t k = 0; k < n; ++k) {
        ld mr, mi, vr, vi;
        mesh_ft_node_ld(verts, tris, nt, xi + 3 * k, &mr, &mi);
        nu_ft_ld(&nu, xi + 3 * k, &vr, &vi);
        ld w = weight_ld(xi + 3 * k, w_geom[k], s, wscale);
        ld dr = mr - vr, di = mi - vi;
        term[k] = w * (dr * dr + di * di);
        res_r[k] = 2.0L * w * dr;
        res_i[k] = 2.0L * w * di;
    }
    ld d = 0.0L;
    for (int64_t k = 0; k < n; ++k) d += term[k];

    ld* gt = calloc((size_t)(nt > 0 ? nt : 1) * 9, sizeof(ld)); /* per triangle, per vertex */
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads)
    for (int64_t t = 0; t < nt; ++t) {
        const double* p[3] = {verts + 3 * (int64_t)tris[3 * t], verts + 3 * (int64_t)tris[3 * t + 1],
                              verts + 3 * (int64_t)tris[3 * t + 2]};
        ld nrm[3];
        ld g = tri_gamma(p[0], p[1], p[2], nrm);
        if (!(g > 0.0L)) continue;
        /* d gamma / d p_j = (p_{j+1} - p_{j+2}) x n */
        ld dg[3][3];
        for (int j = 0; j < 3; ++j) {
            const double* q1 = p[(j + 1) % 3];
            const double* q2 = p[(j + 2) % 3];
            ld e[3] = {(ld)q1[0] - q2[0], (ld)q1[1] - q2[1], (ld)q1[2] - q2[2]};
            dg[j][0] = e[1] * nrm[2] - e[2] * nrm[1];
            dg[j][1] = e[2] * nrm[0] - e[0] * nrm[2];
            dg[j][2] = e[0] * nrm[1] - e[1] * nrm[0];
        }
        ld acc[3][3] = {{0}};
        for (int64_t k = 0; k < n; ++k) {
            const double* x = xi + 3 * k;
            ld tt[3] = {dotl(x, p[0]), dotl(x, p[1]), dotl(x, p[2])};
            ld gr, gi;
            dd(tt, 2, &gr, &gi);
            /* Re(conj(res) * z) = res_r z_r + res_i z_i */
            ld a0 = res_r[k] * gr + res_i[k] * gi;
            for (int j = 0; j < 3; ++j) {
                ld q[4] = {tt[j], tt[0], tt[1], tt[2]};
                ld hr, hi;
                dd(q, 3, &hr, &hi);
                ld a1 = g * (res_r[k] * hr + res_i[k] * hi);
                for (int c = 0; c < 3; ++c) acc[j][c] += a0 * dg[j][c] + a1 * (ld)x[c];
            }
        }
        for (int j = 0; j < 3; ++j)
            for (int c = 0; c < 3; ++c) gt[9 * t + 3 * j + c] = acc[j][c];
    }
    for (int64_t v = 0; v < 3 * nv; ++v) grad[v] = 0.0;
    ld* gv = calloc((size_t)(nv > 0 ? nv : 1) * 3, sizeof(ld));
    for (int64_t t = 0; t < nt; ++t)
        for (int j = 0; j < 3; ++j)
            for (int c = 0; c < 3; ++c) gv[3 * (int64_t)tris[3 * t + j] + c] += gt[9 * t + 3 * j + c];
    for (int64_t v = 0; v < 3 * nv; ++v) grad[v] = (double)gv[v];
    free(gv); free(gt); free(res_r); free(res_i); free(term);
    return (double)d;
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
