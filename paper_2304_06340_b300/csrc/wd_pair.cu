// Mesh staging and the (triangle, frequency-node) pair kernels.
//
// For a triangle T with vertices a, b, c and a node xi, the transform of the
// surface measure (Eq. (simplex32_ft), angular convention) is
//     F_T(xi) = gamma * G[t_a, t_b, t_c],  G(t) = -exp(-i t),  t_v = xi.v,
// the second divided difference of G times gamma = |(b - a) x (c - a)|.
// With the centroid phase t_m = xi.m, the edge gaps g1 = xi.(b - a),
// g2 = xi.(c - a), g3 = g2 - g1 and the centred phases
//     y_a = -(g1 + g2)/3,  y_b = (2 g1 - g2)/3,  y_c = (2 g2 - g1)/3,
// two evaluations are used:
//   * all gaps below DELTA: the Taylor series about t_m,
//       G = exp(-i t_m) sum_n (-i)^n h_n(y_a, y_b, y_c) / (n + 2)!,
//     where, because y_a + y_b + y_c = 0, the complete homogeneous symmetric
//     polynomials satisfy h_n = p h_{n-2} + q h_{n-3} with
//     p = (g1^2 - g1 g2 + g2^2)/3 and q = y_a y_b y_c (h_0 = 1, h_1 = 0);
//   * otherwise the divided-difference recurrence over the pair (x, z) with
//     the largest gap D = t_z - t_x and the middle node w,
//       G = (G[t_w, t_z] - G[t_x, t_w]) / D,
//       G[u, v] = i exp(-i (u + v)/2) sinc((v - u)/2),
//     each first-order term being exact and cancellation-free, so the only
//     cancellation is the final difference, bounded by the machine epsilon
//     over D >= DELTA.
// Per node the transforms are summed over all triangles (linearity,
// Sec. 3.1); the distance epilogue subtracts nu^, weights by
// w_k (1 + c |xi_k|^2)^(-s) (c = 1, or 1/(4 pi^2) for the paper's lattice
// rule) and reduces (the quadrature of Eq. (sobolev_2)).
//
// Kernels: pair_kernel (one node per thread; float64 path, and the mixed path
// for explicit node lists), pair_kernel_precise (the mixed per-node form's
// extended-precision blocks), pair_kernel_lattice (mixed path, the paper's
// lattice rule: per-(line, triangle) records), pair_kernel_radial (mixed path,
// ball rules: per-(direction, triangle) records, radius per thread) and the
// serving loop's batched kernels, which run the same item bodies.
#include <cstdint>
#include <type_traits>

#include "wd_internal.h"
#include "wd_math.cuh"

namespace {

// ------------------------------------------------------------------ staging (a1)
template <bool MIXED>
__global__ void stage_kernel(const double* __restrict__ verts, int64_t nv,
                             const int32_t* __restrict__ tris, int64_t nt, double sign,
                             void* __restrict__ rec_out, int* __restrict__ flags)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nt;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t ia = tris[3 * t], ib = tris[3 * t + 1], ic = tris[3 * t + 2];
        bool ok = ia >= 0 && ia < nv && ib >= 0 && ib < nv && ic >= 0 && ic < nv;
        double a[3] = {0, 0, 0}, b[3] = {0, 0, 0}, c[3] = {0, 0, 0};
        if (ok) {
            for (int j = 0; j < 3; ++j) {
                a[j] = verts[3 * ia + j];
                b[j] = verts[3 * ib + j];
                c[j] = verts[3 * ic + j];
                ok = ok && isfinite(a[j]) && isfinite(b[j]) && isfinite(c[j]);
            }
        }
        if (!ok) {
            atomicOr(&flags[0], 1);
            for (int j = 0; j < 3; ++j) a[j] = b[j] = c[j] = 0.0;
        }
        double m[3], e1[3], e2[3];
        for (int j = 0; j < 3; ++j) {
            m[j] = (a[j] + b[j] + c[j]) * (1.0 / 3.0);
            e1[j] = b[j] - a[j];
            e2[j] = c[j] - a[j];
        }
        const double nx = e1[1] * e2[2] - e1[2] * e2[1];
        const double ny = e1[2] * e2[0] - e1[0] * e2[2];
        const double nz = e1[0] * e2[1] - e1[1] * e2[0];
        const double gam = sign * sqrt(nx * nx + ny * ny + nz * nz);
        if (MIXED) {
            TriRecF r;
            for (int j = 0; j < 3; ++j) {
                r.mh[j] = (float)m[j];
                r.ml[j] = (float)(m[j] - (double)r.mh[j]);
                r.e1[j] = (float)e1[j];
                r.e2[j] = (float)e2[j];
            }
            r.gam = (float)gam;
            r.gam_lo = (float)(gam - (double)r.gam);
            r.pad[0] = r.pad[1] = 0.0f;
            static_cast<TriRecF*>(rec_out)[t] = r;
        } else {
            TriRecD r;
            for (int j = 0; j < 3; ++j) {
                r.m[j] = m[j];
                r.e1[j] = e1[j];
                r.e2[j] = e2[j];
            }
            r.gam = gam;
            static_cast<TriRecD*>(rec_out)[t] = r;
        }
    }
}

// ------------------------------------------------------------------ shared pieces
// Taylor branch bounds: below a largest gap DELTA the centred phases satisfy
// |y| <= 2 DELTA / 3. float64: DELTA = 1, series to n = 18 (remainder < 1e-18);
// mixed: DELTA = 3, series to n = 12 (p <= 3, remainder < 3.2e-9); in the
// radial kernel also DELTA_S = 1.5 with the series to n = 9 (remainder
// < 1.1e-9). Both bounds sum C(j+k, k) p^j |q|^k / (n+2)! over the dropped
// n = 2j + 3k, with p <= DELTA^2 / 3 and |q| <= 2 (p/3)^(3/2).
constexpr double kDelta64 = 1.0;
constexpr int kTerms64 = 18;
constexpr float kDelta32 = 3.0f;
constexpr float kDeltaShort32 = 1.5f;

// 1/(n+2)! for n = 0..22
__device__ constexpr double kInvFact2[23] = {
    1.0 / 2, 1.0 / 6, 1.0 / 24, 1.0 / 120, 1.0 / 720, 1.0 / 5040, 1.0 / 40320, 1.0 / 362880,
    1.0 / 3628800, 1.0 / 39916800, 1.0 / 479001600, 1.0 / 6227020800.0, 1.0 / 87178291200.0,
    1.0 / 1307674368000.0, 1.0 / 20922789888000.0, 1.0 / 355687428096000.0,
    1.0 / 6402373705728000.0, 1.0 / 121645100408832000.0, 1.0 / 2432902008176640000.0,
    1.0 / 51090942171709440000.0, 1.0 / 1124000727777607680000.0,
    1.0 / 25852016738884976640000.0, 1.0 / 620448401733239439360000.0};

// sum_n (-i)^n h_n / (n+2)! with h_n = p h_{n-2} + q h_{n-3}, from n = N0
// (N0 = 0: the full series; N0 = 3: the tail after the 1/2 and -p/24 terms)
template <typename Real, int NT, int N0 = 0>
__device__ __forceinline__ void taylor_sum(Real p, Real q, Real& sr, Real& si)
{
    Real h[NT + 1];
    h[0] = Real(1);
    if (NT >= 1) h[1] = Real(0);
    if (NT >= 2) h[2] = p;
    if (NT >= 3) h[3] = q;
#pragma unroll
    for (int n = 4; n <= NT; ++n) h[n] = p * h[n - 2] + q * h[n - 3];
    sr = Real(0);
    si = Real(0);
#pragma unroll
    for (int n = NT; n >= N0; --n) {
        // (-i)^n: 1, -i, -1, i
        const Real c = Real(kInvFact2[n]);
        switch (n & 3) {
        case 0: sr += c * h[n]; break;
        case 1: si -= c * h[n]; break;
        case 2: sr -= c * h[n]; break;
        default: si += c * h[n]; break;
        }
    }
}

// ------------------------------------------------------------------ float64 pair (a3, a4)
__device__ __forceinline__ double sinc64(double x)
{
    return x == 0.0 ? 1.0 : sin(x) / x;
}

struct NodeD {
    double x, y, z;
};

__device__ __forceinline__ void pair_f64(const NodeD& q, const TriRecD& t, double& fr, double& fi)
{
    const double tm = fma(q.x, t.m[0], fma(q.y, t.m[1], q.z * t.m[2]));
    const double g1 = fma(q.x, t.e1[0], fma(q.y, t.e1[1], q.z * t.e1[2]));
    const double g2 = fma(q.x, t.e2[0], fma(q.y, t.e2[1], q.z * t.e2[2]));
    const double g3 = g2 - g1;
    const double a1 = fabs(g1), a2 = fabs(g2), a3 = fabs(g3);
    const double gmax = fmax(a1, fmax(a2, a3));
    const double ya = -(g1 + g2) * (1.0 / 3.0);
    const double yb = (2.0 * g1 - g2) * (1.0 / 3.0);
    const double yc = (2.0 * g2 - g1) * (1.0 / 3.0);
    double gr, gi;
    if (gmax < kDelta64) {
        const double p = (g1 * g1 - g1 * g2 + g2 * g2) * (1.0 / 3.0);
        const double qq = ya * yb * yc;
        double sr, si;
        taylor_sum<double, kTerms64>(p, qq, sr, si);
        double s, c;
        sincos(tm, &s, &c);
        // exp(-i tm) (sr + i si)
        gr = c * sr + s * si;
        gi = c * si - s * sr;
    } else {
        // largest gap: A = (a, c) with g2, B = (a, b) with g1, C = (b, c) with g3;
        // P is the first-order term on the far side, Q on the near side.
        // Edge midpoints relative to the centroid: (a+b)/2 -> -y_c/2,
        // (b+c)/2 -> -y_a/2, (a+c)/2 -> -y_b/2.
        const bool caseA = (a2 >= a1) && (a2 >= a3);
        const bool caseB = !caseA && (a1 >= a3);
        const bool caseC = !caseA && !caseB;
        const double offP = caseC ? -0.5 * yb : -0.5 * ya;  // C: (a,c) ; A, B: (b,c)
        const double hP = caseC ? 0.5 * g2 : 0.5 * g3;
        const double offQ = caseB ? -0.5 * yb : -0.5 * yc;  // B: (a,c) ; A, C: (a,b)
        const double hQ = caseB ? 0.5 * g2 : 0.5 * g1;
        const double D = caseA ? g2 : (caseB ? g1 : g3);
        double sP, cP, sQ, cQ;
        sincos(tm + offP, &sP, &cP);
        sincos(tm + offQ, &sQ, &cQ);
        const double scP = sinc64(hP), scQ = sinc64(hQ);
        // S_P - S_Q with S = exp(-i theta) sinc(h); G = i (S_P - S_Q) / D
        const double dr = cP * scP - cQ * scQ;
        const double di = sQ * scQ - sP * scP;
        gr = -di / D;
        gi = dr / D;
    }
    fr = t.gam * gr;
    fi = t.gam * gi;
}

// Largest gap >= DELTA (mixed): the divided-difference recurrence over the
// pair with the largest gap, phases in turns about the dithered centroid
// phase (tau, tlo); returns gamma G with gamma = gam + gam_lo.
__device__ __forceinline__ void pair_mixed_divdiff(const TabEntry* __restrict__ tab, float tau, float tlo, float g1,
                                                   float g2, float gam, float gam_lo, float& fr, float& fi,
                                                   float magic)
{
    const float g3 = g2 - g1;
    const float a1 = fabsf(g1), a2 = fabsf(g2), a3 = fabsf(g3);
    const float ya = -(g1 + g2) * (1.0f / 3.0f);
    const float yb = (2.0f * g1 - g2) * (1.0f / 3.0f);
    const float yc = (2.0f * g2 - g1) * (1.0f / 3.0f);
    const bool caseA = (a2 >= a1) && (a2 >= a3);
    const bool caseB = !caseA && (a1 >= a3);
    const bool caseC = !caseA && !caseB;
    const float inv4pi = 0.0795774715459476679f;  // offsets -y/2 in turns: -y/(4 pi)
    const float offP = caseC ? -inv4pi * yb : -inv4pi * ya;
    const float hP = caseC ? 0.5f * g2 : 0.5f * g3;
    const float offQ = caseB ? -inv4pi * yb : -inv4pi * yc;
    const float hQ = caseB ? 0.5f * g2 : 0.5f * g1;
    const float D = caseA ? g2 : (caseB ? g1 : g3);
    float cP, sP, cQ, sQ;  // exp(-i theta) = (c, s)
    expm_turns(tab, tau + offP, tlo, cP, sP, magic);
    expm_turns(tab, tau + offQ, tlo, cQ, sQ, magic);
    const float scP = sinc32(hP), scQ = sinc32(hQ);
    // S_P - S_Q, G = i (S_P - S_Q) / D
    const float dr = cP * scP - cQ * scQ;
    const float di = sP * scP - sQ * scQ;
    const float inv = 1.0f / D;
    const float gr = -di * inv;
    const float gi = dr * inv;
    // gamma carried as a float pair: its rounding is identical for congruent triangles
    fr = fmaf(gam, gr, gam_lo * gr);
    fi = fmaf(gam, gi, gam_lo * gi);
}

// Taylor branch, last step: gamma exp(-i t_m) (1/2 + sr + i si) with the
// dithered phase (tau, tlo). The tail must not be added to the exactly
// representable c/2 on its own: below half an ulp it would be rounded away
// every time, and it has one sign (-p/24), so the loss would be a bias. It is
// added inside the final rounding with gamma, where gamma c/2 is a full-width
// product off the float grid.
// gamma (c + i s)(1/2 + sr + i si) = g2 (c + i s) + (c + i s)(ar + i ai) with
// g2 = gamma/2, ar = gamma sr + gamma_lo/2, ai = gamma si, (c, s) = exp(-i t);
// gamma_lo times the tail (2^-24 of a zero-mean term) is left out
__device__ __forceinline__ void taylor_gamma(float c, float s, float sr, float si, float gam, float gam_lo, float& fr,
                                             float& fi)
{
    const float g2 = 0.5f * gam;  // exact
    const float ar = fmaf(gam, sr, 0.5f * gam_lo);
    const float ai = gam * si;
    fr = fmaf(g2, c, fmaf(c, ar, -s * ai));
    fi = fmaf(g2, s, fmaf(s, ar, c * ai));
}

// FAST: expm_turns_fast
template <bool FAST = false>
__device__ __forceinline__ void taylor_combine(const TabEntry* __restrict__ tab, float tau, float tlo, float sr,
                                               float si, float gam, float gam_lo, float& fr, float& fi, float magic)
{
    float c, s;
    // (c, s) = exp(-i (t_m - 2 pi dith + 2 pi shift))
    if (FAST) expm_turns_fast(tab, tau, tlo, c, s, magic);
    else expm_turns(tab, tau, tlo, c, s, magic);
    taylor_gamma(c, s, sr, si, gam, gam_lo, fr, fi);
}

__device__ __forceinline__ void pair_mixed_gaps(const TabEntry* __restrict__ tab, float tau, float tlo, float g1,
                                                float g2, float gam, float gam_lo, float& fr, float& fi, float magic);

__device__ __forceinline__ void pair_mixed(const TabEntry* __restrict__ tab, const NodeF& q, const TriRecF& t,
                                           float& fr, float& fi, float magic)
{
    // centroid phase in turns: exact high products reduced mod 1, plus the low terms
    const float p0 = q.hx * t.mh[0], p1 = q.hy * t.mh[1], p2 = q.hz * t.mh[2];
    const float r0 = fmaf(q.hx, t.mh[0], -p0);
    const float r1 = fmaf(q.hy, t.mh[1], -p1);
    const float r2 = fmaf(q.hz, t.mh[2], -p2);
    float f = (p0 - rintf(p0)) + (p1 - rintf(p1));
    f -= rintf(f);
    f += p2 - rintf(p2);
    f -= rintf(f);
    float lo = r0 + r1 + r2;
    lo = fmaf(q.hx, t.ml[0], lo);
    lo = fmaf(q.hy, t.ml[1], lo);
    lo = fmaf(q.hz, t.ml[2], lo);
    lo = fmaf(q.lx, t.mh[0], lo);
    lo = fmaf(q.ly, t.mh[1], lo);
    lo = fmaf(q.lz, t.mh[2], lo);
    // phase in turns as the pair (tau, tlo), shifted by the node's dither; the
    // rounding of f - dith (below 2^-25 turns) varies pseudo-randomly with the
    // dithered phase and averages out over the triangles
    const float tau = f - q.dith;
    const float g1 = fmaf(q.x, t.e1[0], fmaf(q.y, t.e1[1], q.z * t.e1[2]));
    const float g2 = fmaf(q.x, t.e2[0], fmaf(q.y, t.e2[1], q.z * t.e2[2]));
    pair_mixed_gaps(tab, tau, lo, g1, g2, t.gam, t.gam_lo, fr, fi, magic);
}

// F_T from the dithered centroid phase (tau, tlo) in turns and the edge gaps
// g1, g2: the centred Taylor series below DELTA, else the largest-gap
// recurrence.
__device__ __forceinline__ void pair_mixed_gaps(const TabEntry* __restrict__ tab, float tau, float tlo, float g1,
                                                float g2, float gam, float gam_lo, float& fr, float& fi, float magic)
{
    const float g3 = g2 - g1;
    const float a1 = fabsf(g1), a2 = fabsf(g2), a3 = fabsf(g3);
    const float gmax = fmaxf(a1, fmaxf(a2, a3));
    const float ya = -(g1 + g2) * (1.0f / 3.0f);
    const float yb = (2.0f * g1 - g2) * (1.0f / 3.0f);
    const float yc = (2.0f * g2 - g1) * (1.0f / 3.0f);
    if (gmax < kDelta32) {
        const float p = (g1 * g1 - g1 * g2 + g2 * g2) * (1.0f / 3.0f);
        const float qq = ya * yb * yc;
        // The series value depends only on the gaps, so its rounding repeats at
        // neighbouring nodes; the exact leading 1/2 is therefore kept out of it
        // and applied with the (dithered) phase factor, and only the small tail
        // sr + i si = Psi - 1/2 = O(p) is rounded independently of the phase.
        // Psi - 1/2 = sum_{n>=2} (-i)^n h_n / (n+2)! in Horner form, with
        // h_n = sum_{2j+3k=n} C(j+k, k) p^j q^k, to n = 12. The -p/24 term is
        // formed as -A/72 with A = g1^2 - g1 g2 + g2^2 and 1/72 as a float
        // pair: a rounded 1/3 or 1/24 would bias it alike for every triangle.
        const float A = fmaf(g1, g1 - g2, g2 * g2);
        const float q2 = qq * qq;
        float re = fmaf(p, 1.0f / 87178291200.0f, -1.0f / 479001600.0f);
        re = fmaf(re, p, 1.0f / 3628800.0f);
        re = fmaf(re, p, -1.0f / 40320.0f);
        re = fmaf(re, p, 1.0f / 720.0f);
        float rq = fmaf(p, 10.0f / 87178291200.0f, -6.0f / 479001600.0f);
        rq = fmaf(rq, p, 3.0f / 3628800.0f);
        rq = fmaf(rq, p, -1.0f / 40320.0f);
        rq = fmaf(q2, 1.0f / 87178291200.0f, rq);
        float sr = fmaf(re, p * p, q2 * rq);
        sr = fmaf(A, -1.388888899e-02f, fmaf(A, 1.034802868e-10f, sr));  // -A (1/72 hi + lo)
        float im = fmaf(p, 5.0f / 6227020800.0f, -4.0f / 39916800.0f);
        im = fmaf(im, p, 3.0f / 362880.0f);
        im = fmaf(im, p, -2.0f / 5040.0f);
        im = fmaf(im, p, 1.0f / 120.0f);
        const float iq = fmaf(p, 4.0f / 6227020800.0f, -1.0f / 39916800.0f);
        const float si = qq * fmaf(q2, iq, im);
        taylor_combine(tab, tau, tlo, sr, si, gam, gam_lo, fr, fi, magic);
        return;
    }
    pair_mixed_divdiff(tab, tau, tlo, g1, g2, gam, gam_lo, fr, fi, magic);
}

// ------------------------------------------------------------------ extended-precision per-node pair
// On lattice rules with a steep weight (the paper's H_{-10}), D is carried by
// a few thousand low-frequency nodes, where mu^ - nu^ is 1e-5 of mu^ and
// every triangle's term has nearly the same phase: the float32 rounding of the
// pairs, though independent across triangles, leaves each node's transform
// about 2e-10 of its size off, which at so few nodes moves D by 1e-6 (Sec. 4.2
// experiment at N = 6, 7). Node blocks that hold such nodes take this variant:
// the centroid phase keeps the rounding errors of its mod-1 sums and of the
// dither (two-sums), exp(-i theta) stays an unevaluated float pair (table
// entry plus correction), gamma/2 times it is formed exactly, and the pairs
// are summed with every rounding error kept. Per pair the relative error falls
// from ~6e-8 to ~1e-9. The Taylor tail, O(p) of the leading 1/2, keeps float32
// arithmetic, and the largest-gap branch (large |xi| h, where mu^ - nu^ is not
// small) is the float32 one.


// float32 sum carried as (s, c) with every addend's rounding error kept in c;
// an addend's low part goes to c directly
struct PairAcc {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float hi, float lo)
    {
        const float t = s + hi;
        c += two_sum_err(s, hi, t) + lo;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// exp(-2 pi i tau) as float pairs: cos = ch + cl, -sin = sh + sl (expm_turns
// without its last rounding: the table entry stays the high part)
__device__ __forceinline__ void expm_turns_pair(const TabEntry* __restrict__ tl, float tau, float tlo, float& ch,
                                                float& cl, float& sh, float& sl, float magic)
{
    const float km = fmaf(tau, (float)kTab, magic);
    const int idx = __float_as_int(km) & (kTab - 1);
    const float k = km - magic;
    const float u = fmaf(-1.0f / kTab, k, tau);
    const float xh = u * 6.28318548202514648f;
    float xl = fmaf(u, 6.28318548202514648f, -xh);
    xl = fmaf(u, -1.74845553e-7f, xl);
    xl = fmaf(tlo, 6.28318548202514648f, xl);
    const float x2 = xh * xh;
    const float dc = fmaf(x2, fmaf(x2, 1.0f / 24.0f, -0.5f), -xh * xl);
    const float ds = fmaf(xh * x2, -1.0f / 6.0f, xl);
    const TabEntry t = tl[idx * kTabRep];
    ch = t.ch;
    cl = fmaf(t.ch, dc, fmaf(-t.sh, xh, fmaf(-t.sh, ds, t.cl)));
    sh = -t.sh;
    sl = -fmaf(t.sh, dc, fmaf(t.ch, xh, fmaf(t.ch, ds, t.sl)));
}

// F_T at node q as float pairs (frh + frl, fih + fil)
__device__ __forceinline__ void pair_mixed_precise(const TabEntry* __restrict__ tab, const NodeF& q, const TriRecF& t,
                                                   float& frh, float& frl, float& fih, float& fil, float magic)
{
    const float p0 = q.hx * t.mh[0], p1 = q.hy * t.mh[1], p2 = q.hz * t.mh[2];
    const float a0 = p0 - rintf(p0), a1 = p1 - rintf(p1), a2 = p2 - rintf(p2);  // exact
    float f = a0 + a1;
    float lo = two_sum_err(a0, a1, f);
    f -= rintf(f);
    const float f2 = f + a2;
    lo += two_sum_err(f, a2, f2);
    f = f2 - rintf(f2);
    const float tau = f - q.dith;
    lo += two_sum_err(f, -q.dith, tau);
    lo += fmaf(q.hx, t.mh[0], -p0) + fmaf(q.hy, t.mh[1], -p1) + fmaf(q.hz, t.mh[2], -p2);
    lo = fmaf(q.hx, t.ml[0], lo);
    lo = fmaf(q.hy, t.ml[1], lo);
    lo = fmaf(q.hz, t.ml[2], lo);
    lo = fmaf(q.lx, t.mh[0], lo);
    lo = fmaf(q.ly, t.mh[1], lo);
    lo = fmaf(q.lz, t.mh[2], lo);
    const float g1 = fmaf(q.x, t.e1[0], fmaf(q.y, t.e1[1], q.z * t.e1[2]));
    const float g2 = fmaf(q.x, t.e2[0], fmaf(q.y, t.e2[1], q.z * t.e2[2]));
    const float g3 = g2 - g1;
    const float gmax = fmaxf(fabsf(g1), fmaxf(fabsf(g2), fabsf(g3)));
    if (gmax < kDelta32) {
        // the tail Psi - 1/2 as in pair_mixed
        const float ya = -(g1 + g2) * (1.0f / 3.0f);
        const float yb = (2.0f * g1 - g2) * (1.0f / 3.0f);
        const float yc = (2.0f * g2 - g1) * (1.0f / 3.0f);
        const float p = (g1 * g1 - g1 * g2 + g2 * g2) * (1.0f / 3.0f);
        const float qq = ya * yb * yc;
        const float A = fmaf(g1, g1 - g2, g2 * g2);
        const float q2 = qq * qq;
        float re = fmaf(p, 1.0f / 87178291200.0f, -1.0f / 479001600.0f);
        re = fmaf(re, p, 1.0f / 3628800.0f);
        re = fmaf(re, p, -1.0f / 40320.0f);
        re = fmaf(re, p, 1.0f / 720.0f);
        float rq = fmaf(p, 10.0f / 87178291200.0f, -6.0f / 479001600.0f);
        rq = fmaf(rq, p, 3.0f / 3628800.0f);
        rq = fmaf(rq, p, -1.0f / 40320.0f);
        rq = fmaf(q2, 1.0f / 87178291200.0f, rq);
        float sr = fmaf(re, p * p, q2 * rq);
        sr = fmaf(A, -1.388888899e-02f, fmaf(A, 1.034802868e-10f, sr));
        float im = fmaf(p, 5.0f / 6227020800.0f, -4.0f / 39916800.0f);
        im = fmaf(im, p, 3.0f / 362880.0f);
        im = fmaf(im, p, -2.0f / 5040.0f);
        im = fmaf(im, p, 1.0f / 120.0f);
        const float iq = fmaf(p, 4.0f / 6227020800.0f, -1.0f / 39916800.0f);
        const float si = qq * fmaf(q2, iq, im);
        float ch, cl, sh, sl;
        expm_turns_pair(tab, tau, lo, ch, cl, sh, sl, magic);
        // gamma (c + i s)(1/2 + sr + i si) with gamma/2 = g (exact) and the
        // gamma-scaled tail ar + i ai (ar carries gamma_lo / 2): the product
        // g ch exactly (high part and its error), g times the low parts, and
        // the tail times the rounded c and s (the tail reaches 1/8 of 1/2 at
        // gaps near DELTA, so it takes the whole of c and s)
        const float g = 0.5f * t.gam;
        const float ar = fmaf(t.gam, sr, 0.5f * t.gam_lo);
        const float ai = t.gam * si;
        const float c = ch + cl, sn = sh + sl;
        frh = g * ch;
        frl = fmaf(g, ch, -frh) + fmaf(g, cl, fmaf(c, ar, -sn * ai));
        fih = g * sh;
        fil = fmaf(g, sh, -fih) + fmaf(g, sl, fmaf(sn, ar, c * ai));
        return;
    }
    float fr, fi;
    pair_mixed_divdiff(tab, tau, lo, g1, g2, t.gam, t.gam_lo, fr, fi, magic);
    frh = fr;
    frl = 0.0f;
    fih = fi;
    fil = 0.0f;
}

// ------------------------------------------------------------------ block reduction
__device__ __forceinline__ double block_sum(double v, double* red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = (l < (int)(blockDim.x >> 5)) ? red[l] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    return s;  // valid in warp 0
}

// mu^(0) = sum_T gamma_T / 2 exactly: the float64 sum, in fixed order, of the
// records' float-pair gamma, returned to every thread of the block. Used for a
// node at the origin in the mixed path: there every pair has the same phase,
// so the float32 roundings of the pairs repeat for congruent triangles and add
// up instead of averaging out, while the origin carries a full weight in
// lattice rules.
__device__ __noinline__ double origin_transform(const TriRecF* __restrict__ rec, int64_t T, double* red)
{
    double v = 0.0;
    for (int64_t j = threadIdx.x; j < T; j += blockDim.x) v += (double)rec[j].gam + (double)rec[j].gam_lo;
    const double s = block_sum(v, red);
    __syncthreads();
    if (threadIdx.x == 0) red[0] = s;
    __syncthreads();
    const double tot = red[0];
    __syncthreads();
    return 0.5 * tot;
}

// Per-node end of one work item, called by every thread of the block with its
// K nodes: combine the triangle chunks of the node block in fixed order (the
// last chunk to finish does it), undo the mixed path's phase dither, then
// write mu^ (FT) or subtract nu^, weight, write the residual (RESID) and reduce
// D in fixed order (the last node block to finish adds the block sums).
// ORIGIN: the node list may contain xi = 0 (not for ball rules: their radii
// are Gauss-Legendre nodes inside (0, R)).
// Chunk partial sums of a node: partial[2 (chunk * stride + slot)] (re, im).
// The plain forms use slot = node and stride = n; the extended-precision
// blocks have their own buffer, indexed by the block's place in their list.
struct PartialSlots {
    double* base;
    int64_t stride;
};

template <bool MIXED, int MODE, int K, bool ORIGIN = true>
__device__ __forceinline__ void node_epilogue(const PairArgs& a, const PairPlan& p, int64_t nb, int chunk,
                                              const int64_t* node, const bool* active, const float* dith,
                                              const double* acc_r, const double* acc_i, double* red, int& s_last,
                                              const PartialSlots& ps, const int64_t* slot)
{
    const int64_t n = a.n;
    double mr[K], mi[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
        mr[q] = acc_r[q];
        mi[q] = acc_i[q];
    }
    // ---- combine triangle chunks of this node block (fixed order)
    if (p.nchunks > 1) {
#pragma unroll
        for (int q = 0; q < K; ++q)
            if (active[q]) {
                ps.base[2 * ((int64_t)chunk * ps.stride + slot[q])] = acc_r[q];
                ps.base[2 * ((int64_t)chunk * ps.stride + slot[q]) + 1] = acc_i[q];
            }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) s_last = (atomicAdd(&a.cnt[nb], 1) == p.nchunks - 1);
        __syncthreads();
        if (!s_last) return;
        __threadfence();
#pragma unroll
        for (int q = 0; q < K; ++q) {
            mr[q] = 0.0;
            mi[q] = 0.0;
            if (active[q])
                for (int c = 0; c < p.nchunks; ++c) {
                    mr[q] += __ldcg(&ps.base[2 * ((int64_t)c * ps.stride + slot[q])]);
                    mi[q] += __ldcg(&ps.base[2 * ((int64_t)c * ps.stride + slot[q]) + 1]);
                }
        }
        if (threadIdx.x == 0) a.cnt[nb] = 0;  // ready for the next launch
    }

    if (MIXED) {
        bool origin[K], any = false;
#pragma unroll
        for (int q = 0; q < K; ++q) {
            // undo the phase dither: mu^ = S exp(-2 pi i dith), in float64
            double sd, cd;
            sincospi(2.0 * (double)dith[q], &sd, &cd);
            const double r_ = mr[q] * cd + mi[q] * sd;
            mi[q] = mi[q] * cd - mr[q] * sd;
            mr[q] = r_;
            origin[q] = ORIGIN && active[q] && a.xi[node[q]] == 0.0 && a.xi[n + node[q]] == 0.0 &&
                        a.xi[2 * n + node[q]] == 0.0;
            any = any || origin[q];
        }
        // a node at the origin takes the exact total (block-uniform branch)
        if (ORIGIN && __syncthreads_or(any)) {
            const double m0 = origin_transform(static_cast<const TriRecF*>(a.tris), a.T, red);
#pragma unroll
            for (int q = 0; q < K; ++q)
                if (origin[q]) {
                    mr[q] = m0;
                    mi[q] = 0.0;
                }
        }
    }

    if (MODE == MODE_FT) {
#pragma unroll
        for (int q = 0; q < K; ++q)
            if (active[q]) {
                a.out[node[q]] = mr[q];
                a.out_im[node[q]] = mi[q];
            }
        return;
    }

    // ---- distance epilogue (a6, a7): subtract nu^, weight, reduce
    double term = 0.0;
#pragma unroll
    for (int q = 0; q < K; ++q)
        if (active[q]) {
            double dr = mr[q], di = mi[q];
            if (a.nu) {
                dr -= a.nu[2 * node[q]];
                di -= a.nu[2 * node[q] + 1];
            }
            term += a.W[node[q]] * (dr * dr + di * di);
            if (MODE == MODE_RESID) {
                a.resid[2 * node[q]] = 2.0 * a.W[node[q]] * dr;
                a.resid[2 * node[q] + 1] = 2.0 * a.W[node[q]] * di;
            }
        }
    const double bsum = block_sum(term, red);
    if (threadIdx.x == 0) {
        a.blockD[nb] = bsum;
        __threadfence();
        s_last = (atomicAdd(a.done, 1) == (int)(p.n_nb - 1));
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        double v = 0.0;
        for (int64_t i = threadIdx.x; i < p.n_nb; i += WD_NPB) v += __ldcg(&a.blockD[i]);
        const double tot = block_sum(v, red);
        if (threadIdx.x == 0) {
            a.out[0] = tot;
            *a.done = 0;
        }
    }
}

// ------------------------------------------------------------------ pair kernel (a3..a7)
// Shared memory of the per-node form: a tile of raw triangle records and the
// exponential table (mixed path).
template <bool MIXED>
struct NodeSmem {
    using Rec = typename std::conditional<MIXED, TriRecF, TriRecD>::type;
    Rec tile[WD_TILE];
    TabEntry etab[MIXED ? kTab * kTabRep : 1];
};

// One work item (node block nb, triangle chunk) of the per-node form: one node
// per thread, tiles of raw records, then the epilogue. Called by every thread
// of the block (barriers inside); etab is filled. PRECISE: the
// extended-precision pairs and sums (mixed only); its chunk partials live in
// their own buffer at slot li * WD_NPB + thread, li the block's list index.
template <bool MIXED, int MODE, bool PRECISE = false>
__device__ __forceinline__ void pair_item(const PairArgs& a, const PairPlan& p, int64_t nb, int chunk, int64_t li,
                                          NodeSmem<MIXED>& sm, double* red, int& s_last)
{
    static_assert(MIXED || !PRECISE, "the extended-precision variant is a mixed-path form");
    using Rec = typename NodeSmem<MIXED>::Rec;
    const int64_t n = a.n;
    const int64_t node = nb * WD_NPB + threadIdx.x;
    const bool active = node < n;
    const double x = active ? a.xi[node] : 0.0;
    const double y = active ? a.xi[n + node] : 0.0;
    const double z = active ? a.xi[2 * n + node] : 0.0;

    double acc_r = 0.0, acc_i = 0.0;
    NodeD qd{x, y, z};
    NodeF qf;
    if (MIXED) {
        const double inv2pi = 0.15915494309189533576888376337251;
        const double X = x * inv2pi, Y = y * inv2pi, Z = z * inv2pi;
        qf.x = (float)x;
        qf.y = (float)y;
        qf.z = (float)z;
        qf.hx = (float)X;
        qf.hy = (float)Y;
        qf.hz = (float)Z;
        qf.lx = (float)(X - (double)qf.hx);
        qf.ly = (float)(Y - (double)qf.hy);
        qf.lz = (float)(Z - (double)qf.hz);
        qf.dith = node_dither(node);
    }
    const int64_t t0 = (int64_t)chunk * p.tiles_per_chunk * WD_TILE;
    int64_t t1 = t0 + (int64_t)p.tiles_per_chunk * WD_TILE;
    if (t1 > a.T) t1 = a.T;
    for (int64_t tb = t0; tb < t1; tb += WD_TILE) {
        const int cnt = (int)((t1 - tb) < WD_TILE ? (t1 - tb) : WD_TILE);
        __syncthreads();
        // the mixed path reads the tile in groups of 4: pad with zero
        // records, which contribute exactly zero (gamma = 0)
        const int cnt4 = MIXED ? ((cnt + 3) & ~3) : cnt;
        {
            const uint4* src = reinterpret_cast<const uint4*>(static_cast<const Rec*>(a.tris) + tb);
            uint4* dst = reinterpret_cast<uint4*>(sm.tile);
            const int nvec = cnt * (int)(sizeof(Rec) / 16);
            const int nvec4 = cnt4 * (int)(sizeof(Rec) / 16);
            for (int i = threadIdx.x; i < nvec4; i += WD_NPB)
                dst[i] = i < nvec ? __ldg(src + i) : make_uint4(0u, 0u, 0u, 0u);
        }
        __syncthreads();
        if (PRECISE) {
            const int shift = tile_shift(node, tb / WD_TILE);
            const float magic = kMagic + (float)shift;
            PairAcc kr, ki;
            for (int j = 0; j < cnt4; j += 4) {
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    float frh, frl, fih, fil;
                    pair_mixed_precise(exp_table_lane(sm.etab), qf, reinterpret_cast<const TriRecF*>(sm.tile)[j + jj],
                                       frh, frl, fih, fil, magic);
                    kr.add(frh, frl);
                    ki.add(fih, fil);
                }
            }
            unshift_add(sm.etab, shift, kr.value(), ki.value(), acc_r, acc_i);
        } else if (MIXED) {
            // plain float32 sums over groups of 4 pairs (their phases are
            // dithered, so the roundings are random), Kahan across groups;
            // each tile with its own phase shift
            const int shift = tile_shift(node, tb / WD_TILE);
            const float magic = kMagic + (float)shift;
            Kahan kr, ki;
            for (int j = 0; j < cnt4; j += 4) {
                float br = 0.0f, bi = 0.0f;
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    float fr, fi;
                    pair_mixed(exp_table_lane(sm.etab), qf, reinterpret_cast<const TriRecF*>(sm.tile)[j + jj], fr,
                               fi, magic);
                    br += fr;
                    bi += fi;
                }
                kr.add(br);
                ki.add(bi);
            }
            unshift_add(sm.etab, shift, kr.value(), ki.value(), acc_r, acc_i);
        } else {
            for (int j = 0; j < cnt; ++j) {
                double fr, fi;
                pair_f64(qd, reinterpret_cast<const TriRecD*>(sm.tile)[j], fr, fi);
                acc_r += fr;
                acc_i += fi;
            }
        }
    }

    const float dith = MIXED ? qf.dith : 0.0f;
    const PartialSlots ps{PRECISE ? a.precise_partial : a.partial, PRECISE ? (int64_t)a.n_precise * WD_NPB : a.n};
    const int64_t slot = PRECISE ? li * WD_NPB + threadIdx.x : node;
    node_epilogue<MIXED, MODE, 1>(a, p, nb, chunk, &node, &active, &dith, &acc_r, &acc_i, red, s_last, ps, &slot);
}

// The per-node form over every node block, skipping the blocks that the
// extended-precision kernel takes (a.precise_flag, mixed path).
template <bool MIXED, int MODE>
__global__ void __launch_bounds__(WD_NPB) pair_kernel(const PairArgs a, const PairPlan p)
{
    __shared__ __align__(16) NodeSmem<MIXED> sm;
    __shared__ double red[WD_NPB / 32];
    __shared__ int s_last;
    if (MIXED) fill_exp_table(sm.etab);  // visible after the first tile barrier
    for (int64_t item = blockIdx.x; item < p.n_items; item += gridDim.x) {
        const int64_t nb = item / p.nchunks;
        if (MIXED && a.precise_flag && a.precise_flag[nb]) continue;  // block-uniform
        pair_item<MIXED, MODE>(a, p, nb, (int)(item - nb * p.nchunks), 0, sm, red, s_last);
    }
}

// The extended-precision blocks a.precise_list[0 .. n_precise), with the
// triangle chunks of their own plan pp (more chunks: few blocks).
template <int MODE>
__global__ void __launch_bounds__(WD_NPB) pair_kernel_precise(const PairArgs a, const PairPlan pp)
{
    __shared__ __align__(16) NodeSmem<true> sm;
    __shared__ double red[WD_NPB / 32];
    __shared__ int s_last;
    fill_exp_table(sm.etab);
    const int64_t n_items = (int64_t)a.n_precise * pp.nchunks;
    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int64_t li = item / pp.nchunks;
        pair_item<true, MODE, true>(a, pp, a.precise_list[li], (int)(item - li * pp.nchunks), li, sm, red, s_last);
    }
}

// ------------------------------------------------------------------ lattice-line kernel (mixed, cube rules)
// The paper's lattice rule (Sec. 3.2, Eq. (def_trap_grid)) puts its nodes on
// lines xi = 2 pi (h i, eta_y, eta_z), i = i0 .. i0 + count - 1, stored
// consecutively. Along a line every per-pair quantity that is linear in xi is
// affine in i: the centroid phase tau(i) = tau0 + i rho (turns), the gaps
// g(i) = G + i d, hence A = g1^2 - g1 g2 + g2^2 (= 3p) is quadratic and
// q = y_a y_b y_c cubic in i. A node block of the per-node plan (256
// consecutive nodes) touches at most three lines; for each tile of triangles
// it builds one record per (line, triangle) with these coefficients, and each
// thread evaluates its pairs from its line's records and its own i.
//
// Dither: node i of line L gets d(i) = d0(L) + i delta(L) (mod 1), both on
// the 2^-20 grid from a hash of L, folded into the record's tau0 and rho, so
// it costs nothing per pair; the epilogue undoes it as for any node. The
// phase is the float pair tau0 + i rho with the exact error of the high
// product kept, as in the radial kernel.
//
// Rows (per warp and tile, as in the radial kernel): where every gap the warp
// meets in the tile is below DELTA_T = 0.6, the centred series to h_6
// (remainder < 2.1e-9); below DELTA = 3 the series to h_12; else the per-pair
// choice between the series and the largest-gap recurrence.
constexpr float kDeltaTiny32 = 0.6f;
constexpr int LAT_TILE = 64;   // triangles per record tile
constexpr int LAT_SLOTS = 3;   // lines a node block can touch (lines hold >= WD_NPB / 2 + 1 nodes)

__device__ __forceinline__ uint32_t mix32(uint32_t h)
{
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

// the line's dither: d(i) = (d0u + i du) 2^-20 - 1/2 (mod 1)
__device__ __forceinline__ void line_dither(int64_t L, uint32_t& d0u, uint32_t& du)
{
    d0u = mix32((uint32_t)L * 0x9E3779B9u + 0x3C6EF372u) & 0xFFFFFu;
    du = mix32((uint32_t)L * 0x7F4A7C15u + 0xA54FF53Au) & 0xFFFFFu;
}

__device__ __forceinline__ float line_node_dither(uint32_t d0u, uint32_t du, int i)
{
    return (float)((d0u + (uint32_t)i * du) & 0xFFFFFu) * 9.5367431640625e-7f - 0.5f;  // exact
}

// Per-(line, triangle) record, grouped by 16 bytes in the order the rows read
// them: the series rows read groups 0-3, the per-pair rows 0, 1 (gamma), 3, 4.
// The dithered phase at i = 0 is the float pair t0h + t0l, t0h reduced mod 1,
// held as t0h = S0 / kTab + t0r (S0 whole table steps, |t0r| <= 1/256): mt0 =
// kMagicTurns + S0 / kTab is the magic constant of the series rows' table
// lookup, which then adds the steps of t0h to those of i rh for free.
struct __align__(16) LatRec {
    float mt0, t0r;        // kMagicTurns + S0 / kTab (exact) and t0h - S0 / kTab
    float rh, rl;          // dithered phase per step of i, float pair
    float A0, A1, A2;      // A(i) = A0 + A1 i + A2 i^2
    float gam;             // twice the area, high part (0 for padding)
    float Q0, Q1, Q2, Q3;  // q(i) = y_a y_b y_c
    float gam_lo;
    float gmax;            // bound of the largest |gap| over the block's nodes on this line
    float t0l;             // low part of the phase at i = 0
    float pad;
    float G1, d1, G2, d2;  // gaps g1 = G1 + i d1, g2 = G2 + i d2 (radians)
};
static_assert(sizeof(LatRec) == 80, "LatRec layout");

__device__ __forceinline__ void make_latrec(const TriRecF& t, const LatLine& ln, int64_t L, float hh, float hl,
                                            int ia, int ib, LatRec& o)
{
    // phase at i = 0 in turns, eta_y m_y + eta_z m_z, in float-pair
    // arithmetic: exact high products reduced mod 1, two-summed, low terms
    const float u1 = ln.yh * t.mh[1], u2 = ln.zh * t.mh[2];
    const float a1 = u1 - rintf(u1), a2 = u2 - rintf(u2);
    float f = a1 + a2;
    float lo = two_sum_err(a1, a2, f);
    lo += fmaf(ln.yh, t.mh[1], -u1) + fmaf(ln.zh, t.mh[2], -u2);
    lo = fmaf(ln.yh, t.ml[1], lo);
    lo = fmaf(ln.yl, t.mh[1], lo);
    lo = fmaf(ln.zh, t.ml[2], lo);
    lo = fmaf(ln.zl, t.mh[2], lo);
    uint32_t d0u, du;
    line_dither(L, d0u, du);
    const float d0 = (float)d0u * 9.5367431640625e-7f - 0.5f;
    const float f2 = f - d0;
    lo += two_sum_err(f, -d0, f2);
    f = f2 - rintf(f2);
    const float t0h = f + lo;
    o.t0l = lo - (t0h - f);
    const float S0 = rintf(t0h * (float)kTab);  // |S0| <= kTab / 2
    o.mt0 = kMagicTurns + S0 * (1.0f / kTab);     // exact
    o.t0r = fmaf(S0, -1.0f / kTab, t0h);          // exact
    // rate per step of i: h m_x - du 2^-20
    const float pr = hh * t.mh[0];
    float rlo = fmaf(hh, t.mh[0], -pr) + fmaf(hh, t.ml[0], hl * t.mh[0]);
    const float dd = (float)du * 9.5367431640625e-7f;
    const float r1 = pr - dd;
    rlo += two_sum_err(pr, -dd, r1);
    o.rh = r1 + rlo;
    o.rl = rlo - (o.rh - r1);
    // gaps (radians): g = 2 pi (h i e_x + eta_y e_y + eta_z e_z)
    const float tpi = 6.28318530717958648f;
    o.G1 = tpi * fmaf(ln.yh, t.e1[1], ln.zh * t.e1[2]);
    o.d1 = tpi * hh * t.e1[0];
    o.G2 = tpi * fmaf(ln.yh, t.e2[1], ln.zh * t.e2[2]);
    o.d2 = tpi * hh * t.e2[0];
    // A = g1^2 - g1 g2 + g2^2 and q = y_a y_b y_c as polynomials in i
    o.A2 = fmaf(o.d1, o.d1 - o.d2, o.d2 * o.d2);
    o.A1 = fmaf(2.0f * o.G1, o.d1, fmaf(2.0f * o.G2, o.d2, -fmaf(o.G1, o.d2, o.G2 * o.d1)));
    o.A0 = fmaf(o.G1, o.G1 - o.G2, o.G2 * o.G2);
    const float ya0 = -(o.G1 + o.G2) * (1.0f / 3.0f), ya1 = -(o.d1 + o.d2) * (1.0f / 3.0f);
    const float yb0 = (2.0f * o.G1 - o.G2) * (1.0f / 3.0f), yb1 = (2.0f * o.d1 - o.d2) * (1.0f / 3.0f);
    const float yc0 = (2.0f * o.G2 - o.G1) * (1.0f / 3.0f), yc1 = (2.0f * o.d2 - o.d1) * (1.0f / 3.0f);
    o.Q3 = ya1 * yb1 * yc1;
    o.Q2 = fmaf(ya0, yb1 * yc1, fmaf(ya1, yb0 * yc1, ya1 * yb1 * yc0));
    o.Q1 = fmaf(ya0, yb0 * yc1, fmaf(ya0, yb1 * yc0, ya1 * yb0 * yc0));
    o.Q0 = ya0 * yb0 * yc0;
    o.gam = t.gam;
    o.gam_lo = t.gam_lo;
    // the largest |gap| over i in [ia, ib] (each gap is affine in i)
    const float fa = (float)ia, fb = (float)ib;
    const float G3 = o.G2 - o.G1, d3 = o.d2 - o.d1;
    float gm = fmaxf(fabsf(fmaf(fa, o.d1, o.G1)), fabsf(fmaf(fb, o.d1, o.G1)));
    gm = fmaxf(gm, fmaxf(fabsf(fmaf(fa, o.d2, o.G2)), fabsf(fmaf(fb, o.d2, o.G2))));
    gm = fmaxf(gm, fmaxf(fabsf(fmaf(fa, d3, G3)), fabsf(fmaf(fb, d3, G3))));
    o.gmax = t.gam != 0.0f ? gm : 0.0f;
    o.pad = 0.0f;
}

struct LatSmem {
    LatRec rec[LAT_SLOTS][LAT_TILE];
    TabEntry etab[kTab * kTabRep];
    unsigned int gmax[LAT_SLOTS * (LAT_TILE / 32)];  // largest gmax of every 32 records, as bits
    int line[LAT_SLOTS], ia[LAT_SLOTS], ib[LAT_SLOTS];
    int n_slots;
};

// Rows: VAR 0 per-pair choice (gaps from G + i d), 1 series to h_12 from
// A(i), q(i), 2 series to h_6 (every gap below DELTA_T).
template <int VAR>
__device__ __forceinline__ void lattice_row(const TabEntry* __restrict__ tl, const LatRec* __restrict__ rec, int cnt4,
                                            float fi, float magic, Kahan& kr, Kahan& ki)
{
    for (int j = 0; j < cnt4; j += 4) {
        float br = 0.0f, bi = 0.0f;
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const LatRec& t = rec[j + jj];
            float fr, fim;
            if (VAR == 0) {
                const float P = fi * t.rh;
                const float lo = fmaf(fi, t.rl, fmaf(fi, t.rh, -P) + t.t0l);
                const float tau = (P - rintf(P)) + ((t.mt0 - kMagicTurns) + t.t0r);  // t0h, exact
                pair_mixed_gaps(tl, tau, lo, fmaf(fi, t.d1, t.G1), fmaf(fi, t.d2, t.G2), t.gam, t.gam_lo, fr, fim,
                                magic);
            } else {
                const float A = fmaf(fmaf(t.A2, fi, t.A1), fi, t.A0);
                const float qq = fmaf(fmaf(fmaf(t.Q3, fi, t.Q2), fi, t.Q1), fi, t.Q0);
                const float p = A * (1.0f / 3.0f);
                float sr, si;
                if (VAR == 2) {
                    // Psi - 1/2 to h_6: -p/24 + p^2/720 - (p^3 + q^2)/8! + i (q/120 - 2 p q/7!)
                    const float t2 = fmaf(p * p, fmaf(p, -1.0f / 40320.0f, 1.0f / 720.0f), qq * qq * (-1.0f / 40320.0f));
                    sr = fmaf(A, -1.388888899e-02f, fmaf(A, 1.034802868e-10f, t2));  // -A (1/72 hi + lo)
                    si = qq * fmaf(p, -2.0f / 5040.0f, 1.0f / 120.0f);
                } else {
                    // to h_12, as in pair_mixed
                    const float q2 = qq * qq;
                    float re = fmaf(p, 1.0f / 87178291200.0f, -1.0f / 479001600.0f);
                    re = fmaf(re, p, 1.0f / 3628800.0f);
                    re = fmaf(re, p, -1.0f / 40320.0f);
                    re = fmaf(re, p, 1.0f / 720.0f);
                    float rq = fmaf(p, 10.0f / 87178291200.0f, -6.0f / 479001600.0f);
                    rq = fmaf(rq, p, 3.0f / 3628800.0f);
                    rq = fmaf(rq, p, -1.0f / 40320.0f);
                    rq = fmaf(q2, 1.0f / 87178291200.0f, rq);
                    sr = fmaf(re, p * p, q2 * rq);
                    sr = fmaf(A, -1.388888899e-02f, fmaf(A, 1.034802868e-10f, sr));
                    float im = fmaf(p, 5.0f / 6227020800.0f, -4.0f / 39916800.0f);
                    im = fmaf(im, p, 3.0f / 362880.0f);
                    im = fmaf(im, p, -2.0f / 5040.0f);
                    im = fmaf(im, p, 1.0f / 120.0f);
                    const float iq = fmaf(p, 4.0f / 6227020800.0f, -1.0f / 39916800.0f);
                    si = qq * fmaf(q2, iq, im);
                }
                // the phase i (rh + rl) + t0h + t0l with its reduction in the
                // table lookup: adding mt0 to the exact product i rh rounds it
                // to K table steps and leaves the index K + S0 in the low bits;
                // mt0 minus that sum is -K / kTab exactly, one more FMA gives
                // the residual i rh - K / kTab with a single rounding, and t0r
                // (at most one more table step) joins it
                const float m = fmaf(fi, t.rh, t.mt0);
                const int idx = __float_as_int(m) & (kTab - 1);
                const float u = fmaf(fi, t.rh, t.mt0 - m);
                const float v = (u + t.t0r) + fmaf(fi, t.rl, t.t0l);
                float c, s;
                expm_residual_wide(tl, idx, v, c, s);
                taylor_gamma(c, s, sr, si, t.gam, t.gam_lo, fr, fim);
            }
            br += fr;
            bi += fim;
        }
        kr.add(br);
        ki.add(bi);
    }
}

// One work item (node block nb, triangle chunk) of the lattice form. Called by
// every thread of the block (barriers inside); etab is filled.
template <int MODE>
__device__ __forceinline__ void lattice_item(const PairArgs& a, const PairPlan& p, int64_t nb, int chunk, LatSmem& sm,
                                             double* red, int& s_last)
{
    const int64_t n = a.n;
    const int64_t node = nb * WD_NPB + threadIdx.x;
    const bool active = node < n;
    // the block's lines: slot s is line lblk.x + s over the block's nodes
    const int2 bd = a.lblk[nb];
    __syncthreads();  // the previous item is done with sm
    if (threadIdx.x == 0) {
        const int64_t last = (n - nb * WD_NPB) < WD_NPB ? n - nb * WD_NPB : WD_NPB;  // nodes in the block
        int64_t L = bd.x, pos = bd.y, left = last;
        int ns = 0;
        while (left > 0 && ns < LAT_SLOTS) {
            const LatLine ln = a.lines[L];
            const int64_t take = (ln.count - pos) < left ? (ln.count - pos) : left;
            sm.line[ns] = (int)L;
            sm.ia[ns] = ln.i0 + (int)pos;
            sm.ib[ns] = ln.i0 + (int)(pos + take - 1);
            ++ns;
            left -= take;
            pos = 0;
            ++L;
        }
        sm.n_slots = ns;
    }
    __syncthreads();
    // this thread's slot and i
    int slot = 0, i = 0;
    {
        int pos = threadIdx.x;
        for (int s = 0; s < sm.n_slots; ++s) {
            const int len = sm.ib[s] - sm.ia[s] + 1;
            if (pos < len || s == sm.n_slots - 1) {
                slot = s;
                i = sm.ia[s] + pos;
                break;
            }
            pos -= len;
        }
    }
    uint32_t d0u = 0, du = 0;
    line_dither(sm.line[slot], d0u, du);
    const float dith = line_node_dither(d0u, du, i);
    const float fi = (float)i;
    const TabEntry* tl = exp_table_lane(sm.etab);
    // slots of the warp's first and last active lane (a warp spans at most two lines)
    const int s_lo = __reduce_min_sync(0xffffffffu, active ? slot : LAT_SLOTS);
    const int s_hi = __reduce_max_sync(0xffffffffu, active ? slot : 0);

    double acc_r = 0.0, acc_i = 0.0;
    const int64_t t0 = (int64_t)chunk * p.tiles_per_chunk * WD_TILE;
    int64_t t1 = t0 + (int64_t)p.tiles_per_chunk * WD_TILE;
    if (t1 > a.T) t1 = a.T;
    const TriRecF* tris = static_cast<const TriRecF*>(a.tris);
    // one compensated float32 sum per node over the item, converted once; the
    // per-node kernel's per-tile phase shift is not needed here: the line
    // dither varies along the line and the nodes that carry D at a steep
    // weight are in the extended-precision blocks (mixed vs float64 within
    // 3e-8 on the paper's ladder either way)
    Kahan kr, ki;
    for (int64_t tb = t0; tb < t1; tb += LAT_TILE) {
        const int cnt = (int)((t1 - tb) < LAT_TILE ? (t1 - tb) : LAT_TILE);
        const int cnt4 = (cnt + 3) & ~3;
        __syncthreads();
        for (int k = threadIdx.x; k < LAT_SLOTS * LAT_TILE; k += WD_NPB) {
            const int sl = k / LAT_TILE, j = k % LAT_TILE;
            float gm = 0.0f;
            if (sl < sm.n_slots && j < cnt4) {
                LatRec o;
                if (j < cnt) {
                    make_latrec(tris[tb + j], a.lines[sm.line[sl]], sm.line[sl], a.lat_hh, a.lat_hl, sm.ia[sl],
                                sm.ib[sl], o);
                } else {
                    o = LatRec{};
                }
                gm = o.gmax;
                sm.rec[sl][j] = o;
            }
            const unsigned int wm = __reduce_max_sync(0xffffffffu, __float_as_uint(gm));
            if ((threadIdx.x & 31) == 0) sm.gmax[k / 32] = wm;
        }
        __syncthreads();
        if (s_lo > s_hi) continue;  // no active lane in this warp (warp-uniform)
        unsigned int gu = 0u;
        for (int s = s_lo; s <= s_hi; ++s)
            for (int part = 0; part < LAT_TILE / 32; ++part) gu = max(gu, sm.gmax[s * (LAT_TILE / 32) + part]);
        const float gap_row = __uint_as_float(gu);
        // the node's per-tile phase shift in whole table steps, undone in float64
        const float magic = kMagic;
        const LatRec* rec = sm.rec[slot];
        if (gap_row < kDeltaTiny32)
            lattice_row<2>(tl, rec, cnt4, fi, magic, kr, ki);
        else if (gap_row < kDelta32)
            lattice_row<1>(tl, rec, cnt4, fi, magic, kr, ki);
        else
            lattice_row<0>(tl, rec, cnt4, fi, magic, kr, ki);
    }
    acc_r = kr.value();
    acc_i = ki.value();
    const PartialSlots ps{a.partial, a.n};
    node_epilogue<true, MODE, 1>(a, p, nb, chunk, &node, &active, &dith, &acc_r, &acc_i, red, s_last, ps, &node);
}

// The lattice form over every node block, skipping the blocks that the
// extended-precision kernel takes.
template <int MODE>
__global__ void __launch_bounds__(WD_NPB) pair_kernel_lattice(const PairArgs a, const PairPlan p)
{
    __shared__ __align__(16) LatSmem sm;
    __shared__ double red[WD_NPB / 32];
    __shared__ int s_last;
    fill_exp_table(sm.etab);  // visible after the first barrier
    for (int64_t item = blockIdx.x; item < p.n_items; item += gridDim.x) {
        const int64_t nb = item / p.nchunks;
        if (a.precise_flag && a.precise_flag[nb]) continue;  // block-uniform
        lattice_item<MODE>(a, p, nb, (int)(item - nb * p.nchunks), sm, red, s_last);
    }
}

// ------------------------------------------------------------------ radial pair kernel (mixed, ball rules)
// Ball-rule nodes factor as xi = r omega (radius r, unit direction omega), so
// every per-pair quantity that is linear in xi is a per-(direction, triangle)
// rate times r: the centroid phase t_m = r (omega.m), the gaps g1 = r (omega.e1),
// g2 = r (omega.e2). In the Taylor branch p = r^2 p0 and q = r^3 q0, so the
// tail Psi - 1/2 = sr + i si is a polynomial in rho = r^2:
//     sr = rho (R1 + rho (R2 + ... + rho R6)),  si = r^3 (I0 + rho (I1 + ... + rho I4)),
// the same terms (h_n to n = 12) as the per-node kernel, regrouped by powers of
// r. A block covers WD_NPB / NR directions x NR radii (RadShape); for each tile of
// triangles it first computes one record of rates and coefficients per
// (direction, triangle), in float32 (float pairs for the phase rate: the
// float64 pipe of this GPU is too narrow for it), then every thread runs
// over the tile with its own radius. A warp holds 32 radii of one direction,
// so the record loads are broadcasts.
// The fields are grouped by 16 bytes in the order the branches read them:
// the short Taylor form reads the first three groups, the full one the first
// four, the divided difference the first and the last three.
struct __align__(16) RadRec {
    float dmh, dml;      // omega.m / 2 pi in turns per unit radius, float pair
    float g2;            // gamma / 2, high part (0 for padding)
    float l2;            // gamma / 2, low part
    float R[4];          // real tail coefficients R1..R4 (h_2..h_8), times gamma
    float I[4];          // imaginary tail coefficients I0..I3 (h_3..h_9), times gamma
    float R5, R6, I4;    // the h_10, h_12 and h_11 terms, times gamma
    float gmax0;         // largest |gap| per unit radius
    // divided-difference branch, per unit radius: phase offsets of the two
    // first differences about the centroid (turns), their half gaps, 2 /
    // (largest gap) and the half gaps' reciprocals (0 for a zero half gap);
    // the case (which vertex pair has the largest gap) does not depend on r
    float oP, oQ, hP, hQ;
    float iD2, ihP, ihQ;
    float pad;
};
static_assert(sizeof(RadRec) == 96, "RadRec layout");

__device__ __forceinline__ void make_radrec(const TriRecF& t, const float* __restrict__ dir, int64_t n_dir,
                                            int64_t d, RadRec& o)
{
    const float fx = dir[d], fy = dir[n_dir + d], fz = dir[2 * n_dir + d];
    const float hx = dir[3 * n_dir + d], hy = dir[4 * n_dir + d], hz = dir[5 * n_dir + d];
    const float lx = dir[6 * n_dir + d], ly = dir[7 * n_dir + d], lz = dir[8 * n_dir + d];
    // omega.m / 2 pi in float-pair arithmetic (relative error ~2^-46): exact
    // high products, their exact two-sums, and the first-order low terms
    const float u0 = hx * t.mh[0], u1 = hy * t.mh[1], u2 = hz * t.mh[2];
    const float v0 = fmaf(hx, t.mh[0], -u0), v1 = fmaf(hy, t.mh[1], -u1), v2 = fmaf(hz, t.mh[2], -u2);
    const float s1 = u0 + u1;
    float bv = s1 - u0;
    float err = (u0 - (s1 - bv)) + (u1 - bv);
    const float s2 = s1 + u2;
    bv = s2 - s1;
    err += (s1 - (s2 - bv)) + (u2 - bv);
    float lo = err + (v0 + v1 + v2);
    lo = fmaf(hx, t.ml[0], lo);
    lo = fmaf(hy, t.ml[1], lo);
    lo = fmaf(hz, t.ml[2], lo);
    lo = fmaf(lx, t.mh[0], lo);
    lo = fmaf(ly, t.mh[1], lo);
    lo = fmaf(lz, t.mh[2], lo);
    o.dmh = s2 + lo;
    o.dml = lo - (o.dmh - s2);
    const float d1 = fmaf(fx, t.e1[0], fmaf(fy, t.e1[1], fz * t.e1[2]));
    const float d2 = fmaf(fx, t.e2[0], fmaf(fy, t.e2[1], fz * t.e2[2]));
    const float d3 = d2 - d1;
    const float a1 = fabsf(d1), a2 = fabsf(d2), a3 = fabsf(d3);
    o.gmax0 = fmaxf(a1, fmaxf(a2, a3));
    o.g2 = 0.5f * t.gam;  // exact
    o.l2 = 0.5f * t.gam_lo;
    const float ya = -(d1 + d2) * (1.0f / 3.0f);
    const float yb = (2.0f * d1 - d2) * (1.0f / 3.0f);
    const float yc = (2.0f * d2 - d1) * (1.0f / 3.0f);
    const float p0 = (d1 * d1 - d1 * d2 + d2 * d2) * (1.0f / 3.0f);
    const float A0 = fmaf(d1, d1 - d2, d2 * d2);  // 3 p0
    const float q0 = ya * yb * yc;
    const float q02 = q0 * q0;
    const float p2 = p0 * p0, p3 = p2 * p0, p4 = p2 * p2;
    // -A0/72 with 1/72 as a float pair (a rounded 1/72 would bias every triangle alike)
    o.R[0] = fmaf(A0, -1.388888899e-02f, A0 * 1.034802868e-10f);
    o.R[1] = p2 * (1.0f / 720.0f);
    o.R[2] = -(p3 + q02) * (1.0f / 40320.0f);
    o.R[3] = fmaf(3.0f * q02, p0, p4) * (1.0f / 3628800.0f);
    o.R5 = -fmaf(6.0f * q02, p2, p4 * p0) * (1.0f / 479001600.0f);
    o.R6 = fmaf(10.0f * q02, p3, fmaf(p3, p3, q02 * q02)) * (1.0f / 87178291200.0f);
    o.I[0] = q0 * (1.0f / 120.0f);
    o.I[1] = -2.0f * q0 * p0 * (1.0f / 5040.0f);
    o.I[2] = 3.0f * q0 * p2 * (1.0f / 362880.0f);
    o.I[3] = -q0 * fmaf(4.0f, p3, q02) * (1.0f / 39916800.0f);
    o.I4 = q0 * fmaf(5.0f, p4, 4.0f * q02 * p0) * (1.0f / 6227020800.0f);
    // scaled by gamma (high part), so that the pair's tail comes out already
    // multiplied by gamma; the smallest scaled coefficients reach the float32
    // subnormal range only where their terms are far below the rounding of F
    for (int k = 0; k < 4; ++k) o.R[k] *= t.gam;
    for (int k = 0; k < 4; ++k) o.I[k] *= t.gam;
    o.R5 *= t.gam;
    o.R6 *= t.gam;
    o.I4 *= t.gam;
    // largest gap: A = (a, c) with d2, B = (a, b) with d1, C = (b, c) with d3,
    // as in pair_mixed_divdiff
    const bool caseA = (a2 >= a1) && (a2 >= a3);
    const bool caseB = !caseA && (a1 >= a3);
    const bool caseC = !caseA && !caseB;
    const float inv4pi = 0.0795774715459476679f;
    o.oP = caseC ? -inv4pi * yb : -inv4pi * ya;
    o.hP = caseC ? 0.5f * d2 : 0.5f * d3;
    o.oQ = caseB ? -inv4pi * yb : -inv4pi * yc;
    o.hQ = caseB ? 0.5f * d2 : 0.5f * d1;
    const float D0 = caseA ? d2 : (caseB ? d1 : d3);
    o.iD2 = D0 != 0.0f ? 2.0f / D0 : 0.0f;  // gmax0 = 0 never takes this branch
    o.ihP = o.hP != 0.0f ? 1.0f / o.hP : 0.0f;
    o.ihQ = o.hQ != 0.0f ? 1.0f / o.hQ : 0.0f;
    o.pad = 0.0f;
}

// Divided-difference branch of the radial kernel: the per-node version
// (pair_mixed_divdiff) with its radius-independent choices taken from the
// record; rinv = 1/r. Returns gamma G.
__device__ __forceinline__ void radial_divdiff(const TabEntry* __restrict__ tl, float tau, float tlo, float r,
                                               float rinv, const RadRec& t, float& fr, float& fi, float magic)
{
    float cP, sP, cQ, sQ;  // exp(-i theta) = (c, s)
    expm_turns_fast(tl, fmaf(r, t.oP, tau), tlo, cP, sP, magic);
    expm_turns_fast(tl, fmaf(r, t.oQ, tau), tlo, cQ, sQ, magic);
    const float scP = sinc32_inv(r * t.hP, rinv * t.ihP), scQ = sinc32_inv(r * t.hQ, rinv * t.ihQ);
    // 2 G = i (S_P - S_Q) (2 / D)
    const float dr = cP * scP - cQ * scQ;
    const float di = sP * scP - sQ * scQ;
    const float inv = t.iD2 * rinv;
    const float gr = -di * inv;
    const float gi = dr * inv;
    fr = fmaf(t.g2, gr, t.l2 * gr);  // (gamma/2)(2 G), gamma as a float pair
    fi = fmaf(t.g2, gi, t.l2 * gi);
}

// Taylor branch end for the radial kernel, (c, s) = exp(-i theta). With
// g2 = gamma/2 and l2 = gamma_lo/2 (both exact), the gamma-scaled tail
// gamma (sr + i si) as (ar - l2) + i ai, i.e. ar = l2 + gamma sr:
//     F = gamma (c + i s)(1/2 + sr + i si)
//       = g2 (c + i s) + (c + i s)(ar + i ai),
// in one final rounding per component as in taylor_combine. The product
// gamma_lo * tail (2^-24 of a zero-mean term already below the float32
// rounding of F) is left out.
__device__ __forceinline__ void taylor_combine_half(float c, float s, float ar, float ai, float g2, float& fr,
                                                    float& fi)
{
    fr = fmaf(g2, c, fmaf(c, ar, -s * ai));
    fi = fmaf(g2, s, fmaf(s, ar, c * ai));
}

// One thread's nodes in a radial node block: with radius group NR, block nb
// covers directions [dg ND, +ND) x radii [rg NR, +NR), ND = WD_NPB / NR;
// thread t takes direction t / TPD (warp-uniform) and the WD_RAD_RPT radii
// t % TPD + q TPD, q < WD_RAD_RPT, of the block's radius group, TPD = NR /
// WD_RAD_RPT. A warp always holds 32 consecutive radii of one direction.
struct RadThread {
    int64_t dg;
    int dl;
    bool dir_ok;
    int64_t node[WD_RAD_RPT];
    bool active[WD_RAD_RPT];
    float rh[WD_RAD_RPT], rlo[WD_RAD_RPT];   // radius as a float pair
    float rho[WD_RAD_RPT], r3[WD_RAD_RPT];   // r^2, r^3
    float thr[WD_RAD_RPT];                   // Taylor branch while gmax0 < thr = DELTA / r
    float rinv[WD_RAD_RPT];                  // 1 / r
    float mt[WD_RAD_RPT];                    // kMagicTurns - j / kTab: the node's dither of j table steps
};

// dith_base: index, in the full rule, of the first node of a radial window
// (the dither is a function of that index, so a window's nodes keep theirs)
template <int NR>
__device__ __forceinline__ RadThread radial_thread(const double* __restrict__ rad, int n_rad, int64_t n_dir,
                                                   int64_t nb, int n_rg, int64_t dith_base)
{
    using S = RadShape<NR>;
    RadThread h;
    h.dl = threadIdx.x / S::TPD;
    const int rl = threadIdx.x % S::TPD;
    h.dg = nb / n_rg;
    const int rg = (int)(nb - h.dg * n_rg);
    const int64_t d = h.dg * S::ND + h.dl;
    h.dir_ok = d < n_dir;
#pragma unroll
    for (int q = 0; q < WD_RAD_RPT; ++q) {
        const int ir = rg * NR + rl + q * S::TPD;
        h.active[q] = h.dir_ok && ir < n_rad;
        h.node[q] = h.active[q] ? (int64_t)ir * n_dir + d : 0;
        const double r = h.active[q] ? rad[ir] : 0.0;
        h.rh[q] = (float)r;
        h.rlo[q] = (float)(r - (double)h.rh[q]);
        h.rho[q] = (float)(r * r);
        h.r3[q] = (float)(r * r * r);
        h.thr[q] = h.active[q] ? (float)((double)kDelta32 / r) : 3.402823466e38f;
        h.rinv[q] = h.active[q] ? (float)(1.0 / r) : 0.0f;
        h.mt[q] = kMagicTurns - (float)node_dither_steps(dith_base + h.node[q]) * (1.0f / kTab);  // exact
        // A warp holds 32 consecutive radii of one direction, and the branch
        // test r gmax0 < DELTA splits it wherever a record's seam falls inside
        // its radius range; the split warp then runs both branches. Where the
        // warp's radii lie within a factor of 2 (every warp but the innermost
        // ones), the whole warp takes the branch of its largest radius
        // instead: Taylor only where every lane's gap is below DELTA (so the
        // remainder bound holds), the divided difference otherwise, which
        // then sees gaps of at least DELTA r_min / r_max > DELTA / 2.
        const unsigned int umax = __reduce_max_sync(0xffffffffu, h.active[q] ? __float_as_uint(h.rh[q]) : 0u);
        const unsigned int umin =
            __reduce_min_sync(0xffffffffu, h.active[q] ? __float_as_uint(h.rh[q]) : 0x7f7fffffu);
        const float rmax = __uint_as_float(umax), rmin = __uint_as_float(umin);
        if (rmax > 0.0f && rmax < 2.0f * rmin) h.thr[q] = (float)((double)kDelta32 / (double)rmax);
    }
    return h;
}

// Centroid phase in turns of record t at the thread's q-th radius,
// (rh + rlo)(dmh + dml) as the pair (P, lo): P the rounded high product, lo
// its exact rounding error plus the low products.
__device__ __forceinline__ void radial_phase(const RadRec& t, const RadThread& h, int q, float& P, float& lo)
{
    P = h.rh[q] * t.dmh;
    const float e = fmaf(h.rh[q], t.dmh, -P);
    lo = fmaf(h.rh[q], t.dml, fmaf(h.rlo[q], t.dmh, e));
}

// exp(-2 pi i (rh + rlo)(dmh + dml)) exp(2 pi i j / kTab) of record t at the
// thread's q-th radius, j the node's dither in table steps, with the phase
// reduction folded into the table lookup: adding mt = kMagicTurns - j / kTab
// to the exact product rh dmh rounds it to k table steps (|rh dmh| < 2^13,
// see radial_sum) and leaves the index k - j in the low bits; mt minus that
// sum is -k / kTab exactly, and one FMA with the exact product again gives
// the residual rh dmh - k / kTab with a single rounding (below 2.5e-10
// turns). The low products are summed apart and added once: added one by
// one to the residual, each would be rounded away wherever it is below half
// the residual's ulp, i.e. the pair would be evaluated at the float radius
// rh and the float rate dmh, a coherent error that moved D on low-frequency
// shells by 8e-8. No rounding of the whole phase enters the pair.
__device__ __forceinline__ void radial_expm(const TabEntry* __restrict__ tl, const RadRec& t, const RadThread& h,
                                            int q, float& er, float& ei)
{
    const float m = fmaf(h.rh[q], t.dmh, h.mt[q]);
    const int idx = __float_as_int(m) & (kTab - 1);
    const float nk = h.mt[q] - m;  // exact
    const float u = fmaf(h.rh[q], t.dmh, nk);
    const float w = fmaf(h.rh[q], t.dml, h.rlo[q] * t.dmh);
    expm_residual(tl, idx, u + w, er, ei);
}

// The gamma-scaled Taylor tail of record t at the thread's q-th radius as a
// polynomial in rho = r^2 (ar including gamma_lo / 2), to h_12 or, when every
// gap is below DELTA_S, to h_9
template <bool SHORT>
__device__ __forceinline__ void radial_tail(const RadRec& t, const RadThread& h, int q, float& ar, float& ai)
{
    const float rho = h.rho[q];
    if (SHORT) {
        ar = fmaf(fmaf(t.R[3], rho, t.R[2]), rho, t.R[1]);
        ai = fmaf(fmaf(t.I[3], rho, t.I[2]), rho, t.I[1]);
    } else {
        ar = fmaf(fmaf(fmaf(fmaf(t.R6, rho, t.R5), rho, t.R[3]), rho, t.R[2]), rho, t.R[1]);
        ai = fmaf(fmaf(fmaf(t.I4, rho, t.I[3]), rho, t.I[2]), rho, t.I[1]);
    }
    ar = fmaf(fmaf(ar, rho, t.R[0]), rho, t.l2);
    ai = fmaf(ai, rho, t.I[0]) * h.r3[q];
}

// Taylor branch of record t at the thread's q-th radius
template <bool SHORT>
__device__ __forceinline__ void radial_taylor(const TabEntry* __restrict__ tl, const RadRec& t, const RadThread& h,
                                              int q, float& fr, float& fi)
{
    float ar, ai, c, s;
    radial_tail<SHORT>(t, h, q, ar, ai);
    radial_expm(tl, t, h, q, c, s);
    taylor_combine_half(c, s, ar, ai, t.g2, fr, fi);
}

// F_T of record t at the thread's q-th radius (dithered phase, Taylor branch
// as a polynomial in r^2 or the largest-gap branch); REDUCE takes the phase
// mod 1 first (exact) in both branches, for rows whose phases reach 2^13
// turns, beyond radial_expm's range
template <bool REDUCE>
__device__ __forceinline__ void radial_pair(const TabEntry* __restrict__ tl, const RadRec& t, const RadThread& h,
                                            int q, float& fr, float& fi)
{
    const float magic = h.mt[q] * (float)kTab;  // kMagic - j, exact
    if (!REDUCE && t.gmax0 < h.thr[q]) {
        radial_taylor<false>(tl, t, h, q, fr, fi);
        return;
    }
    float P, lo;
    radial_phase(t, h, q, P, lo);
    P -= rintf(P);  // exact
    if (REDUCE) {
        // at these phases lo (the high product's rounding error and the low
        // products) can reach table steps: fold it into the reduced phase
        // with its exact rounding error, so that the residual stays small
        const float Pl = P + lo;
        lo = two_sum_err(P, lo, Pl);
        P = Pl;
    }
    if (REDUCE && t.gmax0 < h.thr[q]) {
        float ar, ai, c, s;
        radial_tail<false>(t, h, q, ar, ai);
        expm_turns_fast(tl, P, lo, c, s, magic);
        taylor_combine_half(c, s, ar, ai, t.g2, fr, fi);
    } else {  // the offsets r oP, r oQ are added to the reduced phase
        radial_divdiff(tl, P, lo, h.rh[q], h.rinv[q], t, fr, fi, magic);
    }
}

// One tile row of records at the thread's radii, in groups of 8 pairs
// (float32 sums, dithered phases: random roundings), Kahan across groups.
// VAR 0: per-pair branch choice; 1: every pair in the Taylor branch; 2: every
// pair in the Taylor branch with all gaps below DELTA_S (short series); 3: as
// 0 with the phase reduced mod 1 first (phases of 2^13 turns or more).
template <int VAR>
__device__ __forceinline__ void radial_row(const TabEntry* __restrict__ tl, const RadRec* __restrict__ rec, int cnt8,
                                           const RadThread& h, Kahan* kr, Kahan* ki)
{
    for (int j = 0; j < cnt8; j += 8) {
        float br[WD_RAD_RPT], bi[WD_RAD_RPT];
#pragma unroll
        for (int q = 0; q < WD_RAD_RPT; ++q) br[q] = bi[q] = 0.0f;
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
            const RadRec& t = rec[j + jj];
#pragma unroll
            for (int q = 0; q < WD_RAD_RPT; ++q) {
                float fr, fi;
                if (VAR == 0 || VAR == 3)
                    radial_pair<VAR == 3>(tl, t, h, q, fr, fi);
                else
                    radial_taylor<VAR == 2>(tl, t, h, q, fr, fi);
                br[q] += fr;
                bi[q] += fi;
            }
        }
#pragma unroll
        for (int q = 0; q < WD_RAD_RPT; ++q) {
            kr[q].add(br[q]);
            ki[q].add(bi[q]);
        }
    }
}

// Sums of F_T over the triangle records [t0, t1) at the thread's nodes, in
// tiles of TILE = NR triangles: the block first fills the tile's (direction,
// triangle) records, then every thread runs over its direction's row, in
// segments of 64 records. Called by every thread of the block (barriers
// inside). Every choice that shapes a node's float32 operations (the row form
// per 64 records, the branch threshold per warp of 32 radii, groups of 8
// pairs from t0) is independent of NR, so a node's sum is the same bits for
// every radius group, radial window and serving batch.
template <int NR>
__device__ __forceinline__ void radial_sum(RadRec* tile, const TabEntry* __restrict__ tab,
                                           const TriRecF* __restrict__ tris, int64_t t0, int64_t t1,
                                           const float* __restrict__ dir, int64_t n_dir, const RadThread& h,
                                           double* acc_r, double* acc_i)
{
    using S = RadShape<NR>;
    static_assert(S::TILE % 64 == 0 && WD_NPB % 32 == 0, "a warp builds records of one direction");
    __shared__ unsigned int s_gmax[WD_NPB / 32];  // largest gmax0 per 32 records, as bits
    __shared__ unsigned int s_pmax[WD_NPB / 32];  // largest |dmh| per 32 records, as bits
    __shared__ float s_rmax[WD_NPB / 32];         // largest active radius per warp
    {
        float rm = 0.0f;
#pragma unroll
        for (int q = 0; q < WD_RAD_RPT; ++q) rm = fmaxf(rm, h.active[q] ? h.rh[q] : 0.0f);
        const unsigned int u = __reduce_max_sync(0xffffffffu, __float_as_uint(rm));
        if ((threadIdx.x & 31) == 0) s_rmax[threadIdx.x >> 5] = __uint_as_float(u);  // read after a barrier
    }
    const TabEntry* tl = exp_table_lane(tab);
    // one compensated float32 sum per node over the whole triangle range (the
    // pair (s, c) goes to float64 once, at the end: a float64 conversion per
    // tile kept this GPU's narrow float64 pipe 10 % busy)
    Kahan kr[WD_RAD_RPT], ki[WD_RAD_RPT];
    for (int64_t tb = t0; tb < t1; tb += S::TILE) {
        const int cnt = (int)((t1 - tb) < S::TILE ? (t1 - tb) : S::TILE);
        const int cnt8 = (cnt + 7) & ~7;
        __syncthreads();
        // records for ND directions x cnt8 triangles (zero padding: gamma =
        // 0, gmax0 = 0), one per thread, and the largest gmax0 of every 32
        // of them (gmax0 >= 0, so its bits order like its value)
        {
            const int i = threadIdx.x;
            const int di = i / S::TILE, j = i % S::TILE;
            const int64_t dd = h.dg * S::ND + di;
            float gm = 0.0f, pm = 0.0f;
            if (j < cnt8) {
                RadRec o;
                if (j < cnt && dd < n_dir) {
                    const TriRecF tr = tris[tb + j];
                    make_radrec(tr, dir, n_dir, dd, o);
                } else {
                    o = RadRec{};
                }
                gm = o.gmax0;
                pm = fabsf(o.dmh);
                tile[i] = o;
            }
            const unsigned int wm = __reduce_max_sync(0xffffffffu, __float_as_uint(gm));
            const unsigned int pmx = __reduce_max_sync(0xffffffffu, __float_as_uint(pm));
            if ((threadIdx.x & 31) == 0) {
                s_gmax[i / 32] = wm;
                s_pmax[i / 32] = pmx;
            }
        }
        __syncthreads();
        bool any_node = false;
#pragma unroll
        for (int q = 0; q < WD_RAD_RPT; ++q) any_node = any_node || h.active[q];
        if (!h.dir_ok || !__any_sync(0xffffffffu, any_node)) continue;  // warp-uniform: no node here
        const RadRec* rec = tile + h.dl * S::TILE;
        const float rmax = s_rmax[threadIdx.x >> 5];
        // No per-tile phase shift here: on ball rules the weight spreads over
        // many nodes and the shift's float64 rotation cost 3% of the
        // throughput without a measurable gain in accuracy (see the per-node
        // kernel for the lattice case). Where every record of a 64-record
        // segment keeps every lane of the warp in the Taylor branch, the
        // segment runs without the per-pair branch test, and with the short
        // series where every gap is below DELTA_S; the choice is the same for
        // the whole warp.
        for (int seg = 0; seg < cnt8; seg += 64) {
            const int n8 = cnt8 - seg < 64 ? cnt8 - seg : 64;
            const int k = (h.dl * S::TILE + seg) >> 5;  // the segment's two 32-record maxima
            const float gap = __uint_as_float(max(s_gmax[k], s_gmax[k + 1])) * rmax;  // bounds every lane's gaps
            // radial_expm takes the unreduced phase P while |P| < 2^13 turns,
            // well inside the [-2^15, 2^15) where adding kMagicTurns keeps the
            // sum on the grid of table steps
            if (__uint_as_float(max(s_pmax[k], s_pmax[k + 1])) * rmax >= 8192.0f)
                radial_row<3>(tl, rec + seg, n8, h, kr, ki);
            else if (gap < kDeltaShort32)
                radial_row<2>(tl, rec + seg, n8, h, kr, ki);
            else if (gap < kDelta32)
                radial_row<1>(tl, rec + seg, n8, h, kr, ki);
            else
                radial_row<0>(tl, rec + seg, n8, h, kr, ki);
        }
    }
#pragma unroll
    for (int q = 0; q < WD_RAD_RPT; ++q) {
        acc_r[q] = kr[q].value();
        acc_i[q] = ki[q].value();
    }
}

struct RadSmem {
    RadRec tile[WD_NPB];  // ND directions x TILE triangles, direction-major
    TabEntry etab[kTab * kTabRep];
};

// One work item (radial node block nb, triangle chunk) of the radial form.
// Called by every thread of the block (barriers inside); etab is filled.
template <int MODE, int NR>
__device__ __forceinline__ void radial_item(const PairArgs& a, const PairPlan& p, int64_t item, RadSmem& sm,
                                            double* red, int& s_last)
{
    const int64_t nb = item / p.nchunks;
    const int chunk = (int)(item - nb * p.nchunks);
    const RadThread h = radial_thread<NR>(a.rad, a.n_rad, a.n_dir, nb, p.n_rg, a.dith_base);
    const int64_t t0 = (int64_t)chunk * p.tiles_per_chunk * WD_TILE;
    int64_t t1 = t0 + (int64_t)p.tiles_per_chunk * WD_TILE;
    if (t1 > a.T) t1 = a.T;
    double acc_r[WD_RAD_RPT], acc_i[WD_RAD_RPT];
    radial_sum<NR>(sm.tile, sm.etab, static_cast<const TriRecF*>(a.tris), t0, t1, a.dir, a.n_dir, h, acc_r,
                   acc_i);
    float dith[WD_RAD_RPT];  // j / kTab turns, exact
#pragma unroll
    for (int q = 0; q < WD_RAD_RPT; ++q) dith[q] = kMagicTurns - h.mt[q];
    const PartialSlots ps{a.partial, a.n};
    node_epilogue<true, MODE, WD_RAD_RPT, false>(a, p, nb, chunk, h.node, h.active, dith, acc_r, acc_i, red,
                                                 s_last, ps, h.node);
}

template <int MODE, int NR>
__global__ void __launch_bounds__(WD_NPB, WD_RAD_RPT == 1 ? 4 : 3) pair_kernel_radial(const PairArgs a,
                                                                                      const PairPlan p)
{
    __shared__ __align__(16) RadSmem sm;
    __shared__ double red[WD_NPB / 32];
    __shared__ int s_last;
    fill_exp_table(sm.etab);  // visible after the first tile barrier
    for (int64_t item = blockIdx.x; item < p.n_items; item += gridDim.x)
        radial_item<MODE, NR>(a, p, item, sm, red, s_last);
}

template <bool MIXED, int MODE>
int resident_blocks(wd_ctx* ctx)
{
    return wd_resident(ctx, OCC_PAIR + 3 * (MIXED ? 1 : 0) + MODE, pair_kernel<MIXED, MODE>, WD_NPB);
}

template <int MODE>
int resident_lattice(wd_ctx* ctx)
{
    return wd_resident(ctx, OCC_LATTICE + MODE, pair_kernel_lattice<MODE>, WD_NPB);
}

int resident_lattice_for(wd_ctx* ctx, int mode)
{
    if (mode == MODE_FT) return resident_lattice<MODE_FT>(ctx);
    if (mode == MODE_RESID) return resident_lattice<MODE_RESID>(ctx);
    return resident_lattice<MODE_DIST>(ctx);
}

template <int MODE>
int resident_precise(wd_ctx* ctx)
{
    return wd_resident(ctx, OCC_PRECISE + MODE, pair_kernel_precise<MODE>, WD_NPB);
}

int resident_precise_for(wd_ctx* ctx, int mode)
{
    if (mode == MODE_FT) return resident_precise<MODE_FT>(ctx);
    if (mode == MODE_RESID) return resident_precise<MODE_RESID>(ctx);
    return resident_precise<MODE_DIST>(ctx);
}

template <int MODE, int NR>
int resident_radial(wd_ctx* ctx)
{
    return wd_resident(ctx, OCC_RADIAL + 3 * MODE + RadShape<NR>::IDX, pair_kernel_radial<MODE, NR>, WD_NPB);
}

template <int MODE>
int resident_radial_mode(wd_ctx* ctx, int nr)
{
    if (nr == 256) return resident_radial<MODE, 256>(ctx);
    if (nr == 128) return resident_radial<MODE, 128>(ctx);
    return resident_radial<MODE, 64>(ctx);
}

// The radius group for a ball rule with n_rad radii: the one that leaves the
// fewest idle threads, the larger on a tie.
int radial_group(int n_rad)
{
    int best = 64;
    int64_t best_slots = 0;
    for (int nr : {64, 128, 256}) {
        const int64_t slots = (int64_t)((n_rad + nr - 1) / nr) * nr;  // threads per direction
        if (best_slots == 0 || slots <= best_slots) {
            best = nr;
            best_slots = slots;
        }
    }
    return best;
}

int resident_radial_for(wd_ctx* ctx, int mode, int nr)
{
    if (mode == MODE_FT) return resident_radial_mode<MODE_FT>(ctx, nr);
    if (mode == MODE_RESID) return resident_radial_mode<MODE_RESID>(ctx, nr);
    return resident_radial_mode<MODE_DIST>(ctx, nr);
}

// Split the triangle range into chunks only when the node blocks alone cannot
// fill the GPU (about four waves of resident blocks).
void plan_chunks(PairPlan& p, int64_t resident)
{
    p.n_tiles = (p.n_tris + WD_TILE - 1) / WD_TILE;
    const int64_t target = 4 * resident;
    int64_t nchunks = 1;
    if (p.n_nb > 0 && p.n_nb < target && p.n_tiles > 1) {
        nchunks = (target + p.n_nb - 1) / p.n_nb;
        if (nchunks > p.n_tiles) nchunks = p.n_tiles;
    }
    int64_t tpc = p.n_tiles > 0 ? (p.n_tiles + nchunks - 1) / nchunks : 0;
    if (tpc > 0) nchunks = (p.n_tiles + tpc - 1) / tpc;
    if (nchunks < 1) nchunks = 1;
    p.tiles_per_chunk = (int)tpc;
    p.nchunks = (int)nchunks;
    p.n_items = p.n_nb * p.nchunks;
    p.grid = (int)(p.n_items < resident ? p.n_items : resident);
}

int resident_for(wd_ctx* ctx, int precision, int mode)
{
    if (precision == WD_MIXED) {
        if (mode == MODE_FT) return resident_blocks<true, MODE_FT>(ctx);
        if (mode == MODE_RESID) return resident_blocks<true, MODE_RESID>(ctx);
        return resident_blocks<true, MODE_DIST>(ctx);
    }
    if (mode == MODE_FT) return resident_blocks<false, MODE_FT>(ctx);
    if (mode == MODE_RESID) return resident_blocks<false, MODE_RESID>(ctx);
    return resident_blocks<false, MODE_DIST>(ctx);
}

// ------------------------------------------------------------------ batched serving kernels
// A launch of the serving loop runs work items of many requests. Each request
// brings the arguments and plan of its own wd_distance launch; the table lists
// contiguous ranges of its items (a range per request and launch). Blocks
// take launch-local item indices from a counter, find their range (binary
// search over the prefix sums) and run the same item body as pair_kernel or
// pair_kernel_radial with the request's arguments. A request's node blocks
// combine their triangle chunks and its final sum is formed in the fixed
// order of its plan, by whichever launch finishes its last item, so the
// result does not depend on what else shares the launches.
__device__ __forceinline__ int64_t serve_next_item(int* counter, int* s_item)
{
    if (threadIdx.x == 0) *s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int64_t it = *s_item;
    __syncthreads();  // every thread has read s_item before it is written again
    return it;
}

__device__ __forceinline__ const ServeRange& serve_find_range(const ServeRange* __restrict__ rg, int n, int64_t it)
{
    int lo = 0, hi = n - 1;  // largest r with rg[r].start <= it
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (rg[mid].start <= it) lo = mid;
        else hi = mid - 1;
    }
    return rg[lo];
}

// one radial work item of a served request, compiled on its own (a call per
// item) so that the three radius groups do not share one register allocation
template <int NR>
__device__ __noinline__ void serve_radial_item(const ServeReq& rq, int64_t item, RadSmem& sm, double* red,
                                               int& s_last)
{
    radial_item<MODE_DIST, NR>(rq.a, rq.p, item, sm, red, s_last);
}

__global__ void __launch_bounds__(WD_NPB, WD_RAD_RPT == 1 ? 4 : 3) serve_kernel_radial(
    ServeTable* __restrict__ head, const ServeRange* __restrict__ ranges, const ServeReq* __restrict__ reqs)
{
    __shared__ __align__(16) RadSmem sm;
    __shared__ double red[WD_NPB / 32];
    __shared__ int s_last, s_item;
    const int64_t n_items = head->n_items[SERVE_RADIAL];
    if (n_items == 0) return;
    fill_exp_table(sm.etab);  // visible after the first tile barrier
    const int n_rg = head->n_ranges[SERVE_RADIAL];
    for (;;) {
        const int64_t it = serve_next_item(&head->next[SERVE_RADIAL], &s_item);
        if (it >= n_items) break;
        const ServeRange& r = serve_find_range(ranges, n_rg, it);
        const ServeReq& rq = reqs[r.req];
        const int64_t item = r.first + (it - r.start);
        if (rq.p.rad_nr == 256)  // block-uniform: the request's radius group
            serve_radial_item<256>(rq, item, sm, red, s_last);
        else if (rq.p.rad_nr == 128)
            serve_radial_item<128>(rq, item, sm, red, s_last);
        else
            serve_radial_item<64>(rq, item, sm, red, s_last);
    }
}

template <bool MIXED>
__global__ void __launch_bounds__(WD_NPB) serve_kernel_node(ServeTable* __restrict__ head,
                                                            const ServeRange* __restrict__ ranges,
                                                            const ServeReq* __restrict__ reqs)
{
    __shared__ __align__(16) NodeSmem<MIXED> sm;
    __shared__ double red[WD_NPB / 32];
    __shared__ int s_last, s_item;
    const int64_t n_items = head->n_items[SERVE_NODE];
    if (n_items == 0) return;
    if (MIXED) fill_exp_table(sm.etab);
    const ServeRange* rg = ranges + WD_SERVE_RANGES;
    const int n_rg = head->n_ranges[SERVE_NODE];
    for (;;) {
        const int64_t it = serve_next_item(&head->next[SERVE_NODE], &s_item);
        if (it >= n_items) break;
        const ServeRange& r = serve_find_range(rg, n_rg, it);
        const ServeReq& rq = reqs[r.req];
        const int64_t item = r.first + (it - r.start);
        const int64_t nb = item / rq.p.nchunks;
        if (MIXED && rq.a.precise_flag && rq.a.precise_flag[nb]) continue;  // the precise form's block
        pair_item<MIXED, MODE_DIST>(rq.a, rq.p, nb, (int)(item - nb * rq.p.nchunks), 0, sm, red, s_last);
    }
}

// Requests with a lattice plan (mixed path, cube rules): the lattice form.
__global__ void __launch_bounds__(WD_NPB) serve_kernel_lattice(ServeTable* __restrict__ head,
                                                               const ServeRange* __restrict__ ranges,
                                                               const ServeReq* __restrict__ reqs)
{
    __shared__ __align__(16) LatSmem sm;
    __shared__ double red[WD_NPB / 32];
    __shared__ int s_last, s_item;
    const int64_t n_items = head->n_items[SERVE_LATTICE];
    if (n_items == 0) return;
    fill_exp_table(sm.etab);
    const ServeRange* rg = ranges + 3 * WD_SERVE_RANGES;
    const int n_rg = head->n_ranges[SERVE_LATTICE];
    for (;;) {
        const int64_t it = serve_next_item(&head->next[SERVE_LATTICE], &s_item);
        if (it >= n_items) break;
        const ServeRange& r = serve_find_range(rg, n_rg, it);
        const ServeReq& rq = reqs[r.req];
        const int64_t item = r.first + (it - r.start);
        const int64_t nb = item / rq.p.nchunks;
        if (rq.a.precise_flag && rq.a.precise_flag[nb]) continue;  // the precise form's block
        lattice_item<MODE_DIST>(rq.a, rq.p, nb, (int)(item - nb * rq.p.nchunks), sm, red, s_last);
    }
}

// The extended-precision blocks of requests with a mixed per-node plan: item
// i of a request is chunk i mod pp.nchunks of its listed block i / pp.nchunks.
__global__ void __launch_bounds__(WD_NPB) serve_kernel_precise(ServeTable* __restrict__ head,
                                                               const ServeRange* __restrict__ ranges,
                                                               const ServeReq* __restrict__ reqs)
{
    __shared__ __align__(16) NodeSmem<true> sm;
    __shared__ double red[WD_NPB / 32];
    __shared__ int s_last, s_item;
    const int64_t n_items = head->n_items[SERVE_PRECISE];
    if (n_items == 0) return;
    fill_exp_table(sm.etab);
    const ServeRange* rg = ranges + 2 * WD_SERVE_RANGES;
    const int n_rg = head->n_ranges[SERVE_PRECISE];
    for (;;) {
        const int64_t it = serve_next_item(&head->next[SERVE_PRECISE], &s_item);
        if (it >= n_items) break;
        const ServeRange& r = serve_find_range(rg, n_rg, it);
        const ServeReq& rq = reqs[r.req];
        const int64_t item = r.first + (it - r.start);
        const int64_t li = item / rq.pp.nchunks;
        pair_item<true, MODE_DIST, true>(rq.a, rq.pp, rq.a.precise_list[li], (int)(item - li * rq.pp.nchunks), li,
                                         sm, red, s_last);
    }
}

}  // namespace

size_t wd_tri_record_bytes(int precision)
{
    return precision == WD_MIXED ? sizeof(TriRecF) : sizeof(TriRecD);
}

wd_status wd_launch_stage(wd_ctx* ctx, int precision, const double* d_verts, int64_t nv,
                          const int32_t* d_tris, int64_t nt, double sign, void* d_rec,
                          int64_t rec_offset, cudaStream_t st)
{
    if (nt == 0) return WD_OK;
    int64_t g = (nt + 255) / 256;
    const int64_t cap = (int64_t)ctx->num_sms * 8;
    if (g > cap) g = cap;
    if (precision == WD_MIXED)
        stage_kernel<true><<<(int)g, 256, 0, st>>>(d_verts, nv, d_tris, nt, sign,
                                                     static_cast<TriRecF*>(d_rec) + rec_offset, ctx->d_flags);
    else
        stage_kernel<false><<<(int)g, 256, 0, st>>>(d_verts, nv, d_tris, nt, sign,
                                                      static_cast<TriRecD*>(d_rec) + rec_offset, ctx->d_flags);
    ctx->launches++;
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}

wd_status wd_plan_pair(wd_ctx* ctx, int precision, int mode, int64_t n_nodes, int64_t n_tris,
                       PairPlan* plan)
{
    PairPlan p;
    p.n_nodes = n_nodes;
    p.n_tris = n_tris;
    p.n_nb = (n_nodes + WD_NPB - 1) / WD_NPB;
    plan_chunks(p, resident_for(ctx, precision, mode));
    *plan = p;
    return WD_OK;
}

wd_status wd_plan_pair_rule(wd_ctx* ctx, const wd_rule* rule, int precision, int mode, int64_t n_tris,
                            PairPlan* plan)
{
    if (precision == WD_MIXED && rule->d_lines) {
        // lattice rules: the per-node blocks, evaluated with line records
        PairPlan p;
        p.lattice = true;
        p.n_nodes = rule->n_eval;
        p.n_tris = n_tris;
        p.n_nb = (rule->n_eval + WD_NPB - 1) / WD_NPB;
        plan_chunks(p, resident_lattice_for(ctx, mode));
        *plan = p;
        return WD_OK;
    }
    if (precision != WD_MIXED || !rule->d_rad || rule->n_dir <= 0)
        return wd_plan_pair(ctx, precision, mode, rule->n_eval, n_tris, plan);
    PairPlan p;
    p.radial = true;
    p.rad_nr = radial_group(rule->n_rad);
    const int nd = WD_NPB / p.rad_nr;  // directions per block
    p.n_nodes = rule->n_eval;
    p.n_tris = n_tris;
    p.n_dg = (rule->n_dir + nd - 1) / nd;
    p.n_rg = (rule->n_rad + p.rad_nr - 1) / p.rad_nr;
    p.n_nb = p.n_dg * p.n_rg;
    plan_chunks(p, resident_radial_for(ctx, mode, p.rad_nr));
    *plan = p;
    return WD_OK;
}

PairPlan wd_precise_plan(wd_ctx* ctx, const PairPlan& plan, int n_precise, int mode)
{
    PairPlan q = plan;
    const int64_t resident = resident_precise_for(ctx, mode);
    const int64_t target = 4 * resident;
    int64_t nch = 1;
    if (n_precise > 0 && n_precise < target && q.n_tiles > 1) {
        nch = (target + n_precise - 1) / n_precise;
        if (nch > q.n_tiles) nch = q.n_tiles;
    }
    const int64_t tpc = q.n_tiles > 0 ? (q.n_tiles + nch - 1) / nch : 0;
    if (tpc > 0) nch = (q.n_tiles + tpc - 1) / tpc;
    if (nch < 1) nch = 1;
    q.tiles_per_chunk = (int)tpc;
    q.nchunks = (int)nch;
    q.n_items = (int64_t)n_precise * nch;
    q.grid = (int)(q.n_items < resident ? q.n_items : resident);
    return q;
}

size_t wd_precise_partial_bytes(const PairPlan& pp, int n_precise)
{
    return pp.nchunks > 1 ? sizeof(double) * 2 * (size_t)pp.nchunks * (size_t)n_precise * WD_NPB : 0;
}

void wd_pair_args_rule(const wd_rule* rule, PairArgs& a)
{
    a.xi = rule->d_xi;
    a.n = rule->n_eval;
    a.rad = rule->d_rad;
    a.dir = rule->d_dir;
    a.n_rad = rule->n_rad;
    a.n_dir = rule->n_dir;
    a.dith_base = (int64_t)rule->shell0 * rule->n_dir;
    a.lines = rule->d_lines;
    a.lblk = rule->d_lblk;
    a.lat_hh = rule->lat_hh;
    a.lat_hl = rule->lat_hl;
}

template <int MODE>
void launch_radial_mode(const PairPlan& plan, const PairArgs& args, cudaStream_t st)
{
    if (plan.rad_nr == 256)
        pair_kernel_radial<MODE, 256><<<plan.grid, WD_NPB, 0, st>>>(args, plan);
    else if (plan.rad_nr == 128)
        pair_kernel_radial<MODE, 128><<<plan.grid, WD_NPB, 0, st>>>(args, plan);
    else
        pair_kernel_radial<MODE, 64><<<plan.grid, WD_NPB, 0, st>>>(args, plan);
}

void launch_radial(int mode, const PairPlan& plan, const PairArgs& args, cudaStream_t st)
{
    if (mode == MODE_FT) launch_radial_mode<MODE_FT>(plan, args, st);
    else if (mode == MODE_RESID) launch_radial_mode<MODE_RESID>(plan, args, st);
    else launch_radial_mode<MODE_DIST>(plan, args, st);
}

wd_status wd_launch_pair(wd_ctx* ctx, int precision, int mode, const PairPlan& plan,
                         const PairArgs& args, cudaStream_t st)
{
    if (plan.n_items == 0) return WD_OK;
    if (plan.radial) {
        if (precision != WD_MIXED || !args.rad || !args.dir) {
            wd_set_error("internal: radial plan without a mixed ball rule");
            return WD_EINVAL;
        }
        launch_radial(mode, plan, args, st);
    } else if (precision == WD_MIXED) {
        if (plan.lattice) {
            if (!args.lines || !args.lblk) {
                wd_set_error("internal: lattice plan without the rule's lines");
                return WD_EINVAL;
            }
            if (mode == MODE_FT) pair_kernel_lattice<MODE_FT><<<plan.grid, WD_NPB, 0, st>>>(args, plan);
            else if (mode == MODE_RESID) pair_kernel_lattice<MODE_RESID><<<plan.grid, WD_NPB, 0, st>>>(args, plan);
            else pair_kernel_lattice<MODE_DIST><<<plan.grid, WD_NPB, 0, st>>>(args, plan);
        } else if (mode == MODE_FT) {
            pair_kernel<true, MODE_FT><<<plan.grid, WD_NPB, 0, st>>>(args, plan);
        } else if (mode == MODE_RESID) {
            pair_kernel<true, MODE_RESID><<<plan.grid, WD_NPB, 0, st>>>(args, plan);
        } else {
            pair_kernel<true, MODE_DIST><<<plan.grid, WD_NPB, 0, st>>>(args, plan);
        }
        if (args.n_precise > 0) {
            WD_CUDA(cudaGetLastError());
            ctx->launches++;
            const PairPlan pp = wd_precise_plan(ctx, plan, args.n_precise, mode);
            if (pp.nchunks > 1 && !args.precise_partial) {
                wd_set_error("internal: extended-precision blocks without their partial buffer");
                return WD_EINVAL;
            }
            if (mode == MODE_FT) pair_kernel_precise<MODE_FT><<<pp.grid, WD_NPB, 0, st>>>(args, pp);
            else if (mode == MODE_RESID) pair_kernel_precise<MODE_RESID><<<pp.grid, WD_NPB, 0, st>>>(args, pp);
            else pair_kernel_precise<MODE_DIST><<<pp.grid, WD_NPB, 0, st>>>(args, pp);
        }
    } else {
        if (mode == MODE_FT) pair_kernel<false, MODE_FT><<<plan.grid, WD_NPB, 0, st>>>(args, plan);
        else if (mode == MODE_RESID) pair_kernel<false, MODE_RESID><<<plan.grid, WD_NPB, 0, st>>>(args, plan);
        else pair_kernel<false, MODE_DIST><<<plan.grid, WD_NPB, 0, st>>>(args, plan);
    }
    ctx->launches++;
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}

int wd_serve_resident(wd_ctx* ctx, int precision, int form)
{
    if (form == SERVE_RADIAL) return wd_resident(ctx, OCC_SERVE, serve_kernel_radial, WD_NPB);
    if (form == SERVE_PRECISE) return wd_resident(ctx, OCC_SERVE_PRECISE, serve_kernel_precise, WD_NPB);
    if (form == SERVE_LATTICE) return wd_resident(ctx, OCC_SERVE_LATTICE, serve_kernel_lattice, WD_NPB);
    return precision == WD_MIXED ? wd_resident(ctx, OCC_SERVE + 2, serve_kernel_node<true>, WD_NPB)
                                 : wd_resident(ctx, OCC_SERVE + 1, serve_kernel_node<false>, WD_NPB);
}

wd_status wd_plan_pair_serve(wd_ctx* ctx, const wd_rule* rule, int precision, int64_t n_tris, int max_tiles,
                             PairPlan* plan)
{
    PairPlan p;
    wd_status st = wd_plan_pair_rule(ctx, rule, precision, MODE_DIST, n_tris, &p);
    if (st != WD_OK) return st;
    if (max_tiles >= 1 && p.tiles_per_chunk > max_tiles) {
        p.tiles_per_chunk = max_tiles;
        p.nchunks = (int)((p.n_tiles + max_tiles - 1) / max_tiles);
        p.n_items = p.n_nb * p.nchunks;
    }
    *plan = p;
    return WD_OK;
}

wd_status wd_launch_serve(wd_ctx* ctx, int precision, ServeTable* d_head, const ServeRange* d_ranges,
                          const ServeReq* d_reqs, cudaStream_t st)
{
    if (precision == WD_MIXED) {
        serve_kernel_radial<<<wd_serve_resident(ctx, precision, SERVE_RADIAL), WD_NPB, 0, st>>>(d_head, d_ranges,
                                                                                              d_reqs);
        WD_CUDA(cudaGetLastError());
        serve_kernel_node<true><<<wd_serve_resident(ctx, precision, SERVE_NODE), WD_NPB, 0, st>>>(d_head, d_ranges,
                                                                                                d_reqs);
        WD_CUDA(cudaGetLastError());
        serve_kernel_precise<<<wd_serve_resident(ctx, precision, SERVE_PRECISE), WD_NPB, 0, st>>>(d_head, d_ranges,
                                                                                                d_reqs);
        WD_CUDA(cudaGetLastError());
        serve_kernel_lattice<<<wd_serve_resident(ctx, precision, SERVE_LATTICE), WD_NPB, 0, st>>>(d_head, d_ranges,
                                                                                                d_reqs);
    } else {
        serve_kernel_node<false><<<wd_serve_resident(ctx, precision, SERVE_NODE), WD_NPB, 0, st>>>(d_head, d_ranges,
                                                                                                 d_reqs);
    }
    WD_CUDA(cudaGetLastError());
    ctx->launches += precision == WD_MIXED ? 4 : 1;
    return WD_OK;
}
