// Adjoint of the distance: dD/d(vertices of mu).
//
// D = sum_k W_k |mu^(xi_k) - nu^(xi_k)|^2 and mu^ = sum_T gamma_T G[t_a, t_b, t_c]
// with G(t) = -exp(-i t) and t_v = xi.v (Eq. (simplex32_ft), angular convention),
// so with the residual r_k = 2 W_k (mu^ - nu^)(xi_k) from the forward pass,
//     dD/dp_j = sum_T [ (d gamma_T/dp_j) Re(conj r . G)
//                       + gamma_T sum_k Re(conj r_k . dG/dt_j) xi_k ],
//     d gamma/da = (b - c) x n,  d gamma/db = (c - a) x n,  d gamma/dc = (a - b) x n,
// n the unit normal. Writing G = exp(-i t_m) Psi(g1, g2) with t_m the centroid
// phase, g1 = t_b - t_a, g2 = t_c - t_a, the phase derivatives are
//     dG/dt_b = exp(-i t_m) (-i Psi/3 + Psi_1),  dG/dt_c = exp(-i t_m) (-i Psi/3 + Psi_2),
//     dG/dt_a = exp(-i t_m) (-i Psi/3 - Psi_1 - Psi_2),
// Psi_k = dPsi/dg_k (their sum is -i G: a common shift of all phases only
// changes exp(-i t_m)). Psi and its partials come from the same two branches as
// the forward transform: the centred Taylor series (with the recurrences of
// h_n differentiated in p and q) and the largest-gap divided difference (with
// sinc' = (cos h - sinc h)/h, by its series for small h).
//
// Three kernels produce the ten per-triangle sums sum Re(conj r G),
// sum rho_i xi, sum rho_1 xi, sum rho_2 xi over a chunk of nodes:
//   * adjoint_kernel_f64 (float64) and adjoint_kernel_mixed (mixed, explicit
//     node lists): work items (block of 128 triangles, chunk of nodes), one
//     thread per triangle over node tiles staged in shared memory;
//   * adjoint_kernel_radial (mixed, ball rules): work items (tile of 32
//     triangles, chunk of directions), a warp per (direction, triangle) with
//     its lanes on the radii (see its comment).
// A finalize kernel adds the chunks in fixed order and applies the geometry; a
// scatter kernel adds the corner contributions to the vertices with float64
// atomic adds made exact by rounding to a per-(vertex, component) grid, so the
// gradient has the same bits on every run.
#include <cstdint>

#include "wd_internal.h"
#include "wd_math.cuh"

namespace {

constexpr int ADJ_TPB = 128;  // triangles per block, one per thread
constexpr int ADJ_NPT = 128;  // nodes per shared-memory tile
constexpr double kDeltaA = 1.0;
constexpr int kTermsA = 18;

__device__ constexpr double kInvFactA[23] = {
    1.0 / 2, 1.0 / 6, 1.0 / 24, 1.0 / 120, 1.0 / 720, 1.0 / 5040, 1.0 / 40320, 1.0 / 362880,
    1.0 / 3628800, 1.0 / 39916800, 1.0 / 479001600, 1.0 / 6227020800.0, 1.0 / 87178291200.0,
    1.0 / 1307674368000.0, 1.0 / 20922789888000.0, 1.0 / 355687428096000.0,
    1.0 / 6402373705728000.0, 1.0 / 121645100408832000.0, 1.0 / 2432902008176640000.0,
    1.0 / 51090942171709440000.0, 1.0 / 1124000727777607680000.0,
    1.0 / 25852016738884976640000.0, 1.0 / 620448401733239439360000.0};

struct Cplx {
    double r, i;
};

// accumulate c (-i)^n x into z
__device__ __forceinline__ void add_mi(Cplx& z, int n, double x)
{
    switch (n & 3) {
    case 0: z.r += x; break;
    case 1: z.i -= x; break;
    case 2: z.r -= x; break;
    default: z.i += x; break;
    }
}

// Psi = sum (-i)^n h_n/(n+2)! and its partials in p and q
__device__ __forceinline__ void taylor_psi(double p, double q, Cplx& P, Cplx& Pp, Cplx& Pq)
{
    double h[kTermsA + 1], hp[kTermsA + 1], hq[kTermsA + 1];
    h[0] = 1.0; h[1] = 0.0; h[2] = p; h[3] = q;
    hp[0] = 0.0; hp[1] = 0.0; hp[2] = 1.0; hp[3] = 0.0;
    hq[0] = 0.0; hq[1] = 0.0; hq[2] = 0.0; hq[3] = 1.0;
#pragma unroll
    for (int n = 4; n <= kTermsA; ++n) {
        h[n] = p * h[n - 2] + q * h[n - 3];
        hp[n] = h[n - 2] + p * hp[n - 2] + q * hp[n - 3];
        hq[n] = h[n - 3] + p * hq[n - 2] + q * hq[n - 3];
    }
    P = Cplx{0.0, 0.0};
    Pp = Cplx{0.0, 0.0};
    Pq = Cplx{0.0, 0.0};
#pragma unroll
    for (int n = kTermsA; n >= 0; --n) {
        const double c = kInvFactA[n];
        add_mi(P, n, c * h[n]);
        add_mi(Pp, n, c * hp[n]);
        add_mi(Pq, n, c * hq[n]);
    }
}

// sinc(h) and its derivative (series below |h| = 0.5: remainder < 1e-18)
__device__ __forceinline__ void sinc_d(double h, double& sc, double& dsc, double& s, double& c)
{
    sincos(h, &s, &c);
    if (fabs(h) < 0.5) {
        const double h2 = h * h;
        // sinc = sum (-1)^k h^2k/(2k+1)!, sinc' = sum_{k>=1} (-1)^k 2k h^(2k-1)/(2k+1)!
        double a = 1.0 / 6227020800.0, b = 12.0 / 6227020800.0;  // k = 6 terms
        a = a * h2 - 1.0 / 39916800.0;
        b = b * h2 - 10.0 / 39916800.0;
        a = a * h2 + 1.0 / 362880.0;
        b = b * h2 + 8.0 / 362880.0;
        a = a * h2 - 1.0 / 5040.0;
        b = b * h2 - 6.0 / 5040.0;
        a = a * h2 + 1.0 / 120.0;
        b = b * h2 + 4.0 / 120.0;
        a = a * h2 - 1.0 / 6.0;
        b = b * h2 - 2.0 / 6.0;
        sc = a * h2 + 1.0;
        dsc = b * h;
    } else {
        sc = s / h;
        dsc = (c - sc) / h;
    }
}

// G/E, Psi_1 and Psi_2 (centred, without exp(-i t_m)) for gaps g1, g2
__device__ __forceinline__ void psi_and_partials(double g1, double g2, Cplx& P, Cplx& P1, Cplx& P2)
{
    const double g3 = g2 - g1;
    const double a1 = fabs(g1), a2 = fabs(g2), a3 = fabs(g3);
    const double gmax = fmax(a1, fmax(a2, a3));
    const double ya = -(g1 + g2) * (1.0 / 3.0);
    const double yb = (2.0 * g1 - g2) * (1.0 / 3.0);
    const double yc = (2.0 * g2 - g1) * (1.0 / 3.0);
    if (gmax < kDeltaA) {
        const double p = (g1 * g1 - g1 * g2 + g2 * g2) * (1.0 / 3.0);
        const double q = ya * yb * yc;
        Cplx Pp, Pq;
        taylor_psi(p, q, P, Pp, Pq);
        // dp/dg1 = y_b, dp/dg2 = y_c; dq/dg from y' = (-1/3, 2/3, -1/3) and (-1/3, -1/3, 2/3)
        const double dq1 = (-yb * yc + 2.0 * ya * yc - ya * yb) * (1.0 / 3.0);
        const double dq2 = (-yb * yc - ya * yc + 2.0 * ya * yb) * (1.0 / 3.0);
        P1 = Cplx{Pp.r * yb + Pq.r * dq1, Pp.i * yb + Pq.i * dq1};
        P2 = Cplx{Pp.r * yc + Pq.r * dq2, Pp.i * yc + Pq.i * dq2};
        return;
    }
    // largest gap: A = (a, c) with g2, B = (a, b) with g1, C = (b, c) with g3.
    // S = exp(-i off) sinc(h) for the far (P) and near (Q) first differences,
    // off and h linear in (g1, g2); Psi = i (S_P - S_Q) / D.
    const bool caseA = (a2 >= a1) && (a2 >= a3);
    const bool caseB = !caseA && (a1 >= a3);
    double oP1, oP2, hP1, hP2, oQ1, oQ2, hQ1, hQ2, D, D1, D2;
    if (caseA) {
        oP1 = 1.0 / 6; oP2 = 1.0 / 6; hP1 = -0.5; hP2 = 0.5;
        oQ1 = 1.0 / 6; oQ2 = -1.0 / 3; hQ1 = 0.5; hQ2 = 0.0;
        D = g2; D1 = 0.0; D2 = 1.0;
    } else if (caseB) {
        oP1 = 1.0 / 6; oP2 = 1.0 / 6; hP1 = -0.5; hP2 = 0.5;
        oQ1 = -1.0 / 3; oQ2 = 1.0 / 6; hQ1 = 0.0; hQ2 = 0.5;
        D = g1; D1 = 1.0; D2 = 0.0;
    } else {
        oP1 = -1.0 / 3; oP2 = 1.0 / 6; hP1 = 0.0; hP2 = 0.5;
        oQ1 = 1.0 / 6; oQ2 = -1.0 / 3; hQ1 = 0.5; hQ2 = 0.0;
        D = g3; D1 = -1.0; D2 = 1.0;
    }
    const double offP = oP1 * g1 + oP2 * g2, hP = hP1 * g1 + hP2 * g2;
    const double offQ = oQ1 * g1 + oQ2 * g2, hQ = hQ1 * g1 + hQ2 * g2;
    double so, co, scP, dscP, scQ, dscQ, tmp1, tmp2;
    sinc_d(hP, scP, dscP, tmp1, tmp2);
    sinc_d(hQ, scQ, dscQ, tmp1, tmp2);
    sincos(offP, &so, &co);
    const Cplx eP{co, -so};  // exp(-i offP)
    sincos(offQ, &so, &co);
    const Cplx eQ{co, -so};
    const Cplx SP{eP.r * scP, eP.i * scP}, SQ{eQ.r * scQ, eQ.i * scQ};
    const double inv = 1.0 / D;
    // Psi = i (SP - SQ) / D
    const Cplx dS{SP.r - SQ.r, SP.i - SQ.i};
    P = Cplx{-dS.i * inv, dS.r * inv};
    // dS/dg = S (-i doff) + exp(-i off) sinc'(h) dh
    Cplx dSP1{SP.i * oP1 + eP.r * dscP * hP1, -SP.r * oP1 + eP.i * dscP * hP1};
    Cplx dSP2{SP.i * oP2 + eP.r * dscP * hP2, -SP.r * oP2 + eP.i * dscP * hP2};
    Cplx dSQ1{SQ.i * oQ1 + eQ.r * dscQ * hQ1, -SQ.r * oQ1 + eQ.i * dscQ * hQ1};
    Cplx dSQ2{SQ.i * oQ2 + eQ.r * dscQ * hQ2, -SQ.r * oQ2 + eQ.i * dscQ * hQ2};
    // dPsi/dg = (i (dSP - dSQ) - Psi dD) / D
    const Cplx d1{dSP1.r - dSQ1.r, dSP1.i - dSQ1.i}, d2{dSP2.r - dSQ2.r, dSP2.i - dSQ2.i};
    P1 = Cplx{(-d1.i - P.r * D1) * inv, (d1.r - P.i * D1) * inv};
    P2 = Cplx{(-d2.i - P.r * D2) * inv, (d2.r - P.i * D2) * inv};
}

__global__ void __launch_bounds__(ADJ_TPB) adjoint_kernel_f64(const double* __restrict__ xi, int64_t n,
                                                              const double* __restrict__ resid,
                                                              const TriRecD* __restrict__ rec, int64_t nt,
                                                              const AdjPlan p, double* __restrict__ partial)
{
    __shared__ double sx[ADJ_NPT], sy[ADJ_NPT], sz[ADJ_NPT], srr[ADJ_NPT], sri[ADJ_NPT];
    for (int64_t item = blockIdx.x; item < p.n_items; item += gridDim.x) {
        const int64_t tb = item / p.nchunks;
        const int chunk = (int)(item - tb * p.nchunks);
        const int64_t tri = tb * ADJ_TPB + threadIdx.x;
        const bool active = tri < nt;
        TriRecD t{};
        if (active) t = rec[tri];
        double acc[10];
#pragma unroll
        for (int c = 0; c < 10; ++c) acc[c] = 0.0;
        const int64_t k0 = (int64_t)chunk * p.tiles_per_chunk * ADJ_NPT;
        int64_t k1 = k0 + (int64_t)p.tiles_per_chunk * ADJ_NPT;
        if (k1 > n) k1 = n;
        for (int64_t kb = k0; kb < k1; kb += ADJ_NPT) {
            const int cnt = (int)((k1 - kb) < ADJ_NPT ? (k1 - kb) : ADJ_NPT);
            __syncthreads();
            for (int i = threadIdx.x; i < cnt; i += ADJ_TPB) {
                sx[i] = xi[kb + i];
                sy[i] = xi[n + kb + i];
                sz[i] = xi[2 * n + kb + i];
                srr[i] = resid[2 * (kb + i)];
                sri[i] = resid[2 * (kb + i) + 1];
            }
            __syncthreads();
            if (!active) continue;
            for (int k = 0; k < cnt; ++k) {
                const double x = sx[k], y = sy[k], z = sz[k], rr = srr[k], ri = sri[k];
                const double tm = fma(x, t.m[0], fma(y, t.m[1], z * t.m[2]));
                const double g1 = fma(x, t.e1[0], fma(y, t.e1[1], z * t.e1[2]));
                const double g2 = fma(x, t.e2[0], fma(y, t.e2[1], z * t.e2[2]));
                Cplx P, P1, P2;
                psi_and_partials(g1, g2, P, P1, P2);
                double se, ce;
                sincos(tm, &se, &ce);  // E = exp(-i tm) = (ce, -se)
                const Cplx G{ce * P.r + se * P.i, ce * P.i - se * P.r};
                const Cplx V1{ce * P1.r + se * P1.i, ce * P1.i - se * P1.r};
                const Cplx V2{ce * P2.r + se * P2.i, ce * P2.i - se * P2.r};
                // Re(conj(r) z) = rr zr + ri zi; (-i G)/3 = (G.i, -G.r)/3
                const double rho0 = rr * G.r + ri * G.i;
                const double rhoi = (rr * G.i - ri * G.r) * (1.0 / 3.0);
                const double rho1 = rr * V1.r + ri * V1.i;
                const double rho2 = rr * V2.r + ri * V2.i;
                acc[0] += rho0;
                acc[1] = fma(rhoi, x, acc[1]);
                acc[2] = fma(rhoi, y, acc[2]);
                acc[3] = fma(rhoi, z, acc[3]);
                acc[4] = fma(rho1, x, acc[4]);
                acc[5] = fma(rho1, y, acc[5]);
                acc[6] = fma(rho1, z, acc[6]);
                acc[7] = fma(rho2, x, acc[7]);
                acc[8] = fma(rho2, y, acc[8]);
                acc[9] = fma(rho2, z, acc[9]);
            }
        }
        if (active)
#pragma unroll
            for (int c = 0; c < 10; ++c) partial[((int64_t)chunk * nt + tri) * 10 + c] = acc[c];
    }
}

// ------------------------------------------------------------------ mixed adjoint
// The same quantities in float32 arithmetic with the forward mixed path's
// safeguards: centroid phase in turns from float pairs, a per-node phase
// dither (undone by rotating the node's residual by exp(2 pi i d)), the
// table-driven exp(-i theta), the Taylor series in Horner form together with
// its p and q derivatives, and separate accumulators for the exact 1/2 part of
// Psi, so that the tail is never rounded against it. Per-node-tile sums are
// float32, flushed to float64.
constexpr float kDeltaAM = 3.0f;

struct AdjNodeF {
    NodeF q;
    float rr, ri;  // residual times exp(2 pi i d)
};

// sinc(h) and sinc'(h) in float32: their Taylor series below |h| = 1
// (remainders < 1e-12); otherwise sin r and cos r from Taylor polynomials
// after reducing h by the nearest multiple of pi, r = h - k pi with a
// two-constant split of pi, |r| <= pi/2 (remainders < 1e-9)
__device__ __forceinline__ void sincd32(float h, float& sc, float& dsc)
{
    const float h2 = h * h;
    if (fabsf(h) < 1.0f) {
        float a = fmaf(h2, 1.0f / 6227020800.0f, -1.0f / 39916800.0f);
        a = fmaf(a, h2, 1.0f / 362880.0f);
        a = fmaf(a, h2, -1.0f / 5040.0f);
        a = fmaf(a, h2, 1.0f / 120.0f);
        a = fmaf(a, h2, -1.0f / 6.0f);
        sc = fmaf(a, h2, 1.0f);
        float b = fmaf(h2, 1.0f / 518918400.0f, -1.0f / 3991680.0f);
        b = fmaf(b, h2, 1.0f / 45360.0f);
        b = fmaf(b, h2, -1.0f / 840.0f);
        b = fmaf(b, h2, 1.0f / 30.0f);
        b = fmaf(b, h2, -1.0f / 3.0f);
        dsc = b * h;
        return;
    }
    const float k = rintf(h * 0.318309886183790672f);
    float r = fmaf(-k, 3.14159274101257324f, h);
    r = fmaf(-k, -8.74227766e-8f, r);
    const float r2 = r * r;
    float sp = fmaf(r2, 1.0f / 6227020800.0f, -1.0f / 39916800.0f);
    sp = fmaf(sp, r2, 1.0f / 362880.0f);
    sp = fmaf(sp, r2, -1.0f / 5040.0f);
    sp = fmaf(sp, r2, 1.0f / 120.0f);
    sp = fmaf(sp, r2, -1.0f / 6.0f);
    const float sr = fmaf(r * r2, sp, r);
    float cp = fmaf(r2, -1.0f / 87178291200.0f, 1.0f / 479001600.0f);
    cp = fmaf(cp, r2, -1.0f / 3628800.0f);
    cp = fmaf(cp, r2, 1.0f / 40320.0f);
    cp = fmaf(cp, r2, -1.0f / 720.0f);
    cp = fmaf(cp, r2, 1.0f / 24.0f);
    cp = fmaf(cp, r2, -0.5f);
    const float cr = fmaf(cp, r2, 1.0f);
    const float half = 0.5f * k;
    const float sgn = (half == rintf(half)) ? 1.0f : -1.0f;
    const float inv = 1.0f / h;
    sc = sgn * sr * inv;
    dsc = (sgn * cr - sc) * inv;
}

// sincd32 given invh = 1/h (anything where h = 0): the reduction by the
// nearest multiple of pi with a magic-number add (1.5 * 2^23 is even, so the
// low bit of the sum is the parity of k) and multiplications by invh in place
// of the division
__device__ __forceinline__ void sincd32_inv(float h, float invh, float& sc, float& dsc)
{
    const float h2 = h * h;
    if (fabsf(h) < 1.0f) {
        float a = fmaf(h2, 1.0f / 6227020800.0f, -1.0f / 39916800.0f);
        a = fmaf(a, h2, 1.0f / 362880.0f);
        a = fmaf(a, h2, -1.0f / 5040.0f);
        a = fmaf(a, h2, 1.0f / 120.0f);
        a = fmaf(a, h2, -1.0f / 6.0f);
        sc = fmaf(a, h2, 1.0f);
        float b = fmaf(h2, 1.0f / 518918400.0f, -1.0f / 3991680.0f);
        b = fmaf(b, h2, 1.0f / 45360.0f);
        b = fmaf(b, h2, -1.0f / 840.0f);
        b = fmaf(b, h2, 1.0f / 30.0f);
        b = fmaf(b, h2, -1.0f / 3.0f);
        dsc = b * h;
        return;
    }
    const float km = fmaf(h, 0.318309886183790672f, 12582912.0f);
    const float k = km - 12582912.0f;  // exact
    float r = fmaf(-k, 3.14159274101257324f, h);
    r = fmaf(-k, -8.74227766e-8f, r);
    const float r2 = r * r;
    float sp = fmaf(r2, 1.0f / 6227020800.0f, -1.0f / 39916800.0f);
    sp = fmaf(sp, r2, 1.0f / 362880.0f);
    sp = fmaf(sp, r2, -1.0f / 5040.0f);
    sp = fmaf(sp, r2, 1.0f / 120.0f);
    sp = fmaf(sp, r2, -1.0f / 6.0f);
    const float sr = fmaf(r * r2, sp, r);
    float cp = fmaf(r2, -1.0f / 87178291200.0f, 1.0f / 479001600.0f);
    cp = fmaf(cp, r2, -1.0f / 3628800.0f);
    cp = fmaf(cp, r2, 1.0f / 40320.0f);
    cp = fmaf(cp, r2, -1.0f / 720.0f);
    cp = fmaf(cp, r2, 1.0f / 24.0f);
    cp = fmaf(cp, r2, -0.5f);
    const float cr = fmaf(cp, r2, 1.0f);
    // (-1)^k sin r and (-1)^k cos r: the parity of k in the sign bits
    const int odd = __float_as_int(km) << 31;
    const float ssr = __int_as_float(__float_as_int(sr) ^ odd), scr = __int_as_float(__float_as_int(cr) ^ odd);
    sc = ssr * invh;
    dsc = (scr - sc) * invh;
}

__global__ void __launch_bounds__(ADJ_TPB) adjoint_kernel_mixed(const double* __restrict__ xi, int64_t n,
                                                                const double* __restrict__ resid,
                                                                const TriRecF* __restrict__ rec, int64_t nt,
                                                                const AdjPlan p, double* __restrict__ partial)
{
    __shared__ AdjNodeF sn[ADJ_NPT];
    __shared__ TabEntry etab[kTab * kTabRep];
    fill_exp_table(etab);
    const TabEntry* tl = exp_table_lane(etab);
    for (int64_t item = blockIdx.x; item < p.n_items; item += gridDim.x) {
        const int64_t tb = item / p.nchunks;
        const int chunk = (int)(item - tb * p.nchunks);
        const int64_t tri = tb * ADJ_TPB + threadIdx.x;
        const bool active = tri < nt;
        TriRecF t{};
        if (active) t = rec[tri];
        // float64 totals: 1/2-part and tail of rho_0, of rho_i xi, and rho_1 xi, rho_2 xi
        double A0h = 0.0, A0t = 0.0, Aih[3] = {0, 0, 0}, Ait[3] = {0, 0, 0}, A1[3] = {0, 0, 0}, A2[3] = {0, 0, 0};
        const int64_t k0 = (int64_t)chunk * p.tiles_per_chunk * ADJ_NPT;
        int64_t k1 = k0 + (int64_t)p.tiles_per_chunk * ADJ_NPT;
        if (k1 > n) k1 = n;
        for (int64_t kb = k0; kb < k1; kb += ADJ_NPT) {
            const int cnt = (int)((k1 - kb) < ADJ_NPT ? (k1 - kb) : ADJ_NPT);
            __syncthreads();
            for (int i = threadIdx.x; i < cnt; i += ADJ_TPB) {
                const int64_t k = kb + i;
                const double x = xi[k], y = xi[n + k], z = xi[2 * n + k];
                const double inv2pi = 0.15915494309189533576888376337251;
                const double X = x * inv2pi, Y = y * inv2pi, Z = z * inv2pi;
                AdjNodeF a;
                a.q.x = (float)x;
                a.q.y = (float)y;
                a.q.z = (float)z;
                a.q.hx = (float)X;
                a.q.hy = (float)Y;
                a.q.hz = (float)Z;
                a.q.lx = (float)(X - (double)a.q.hx);
                a.q.ly = (float)(Y - (double)a.q.hy);
                a.q.lz = (float)(Z - (double)a.q.hz);
                a.q.dith = node_dither(k);
                double sd, cd;
                sincospi(2.0 * (double)a.q.dith, &sd, &cd);
                const double r0 = resid[2 * k], r1 = resid[2 * k + 1];
                a.rr = (float)(r0 * cd - r1 * sd);
                a.ri = (float)(r0 * sd + r1 * cd);
                sn[i] = a;
            }
            __syncthreads();
            if (!active) continue;
            float b0h = 0.0f, b0t = 0.0f, bih[3] = {0, 0, 0}, bit[3] = {0, 0, 0}, b1[3] = {0, 0, 0}, b2[3] = {0, 0, 0};
            for (int kk = 0; kk < cnt; ++kk) {
                const AdjNodeF& a = sn[kk];
                const NodeF& q = a.q;
                // centroid phase in turns (as in the forward mixed pair), dithered
                const float p0 = q.hx * t.mh[0], p1 = q.hy * t.mh[1], p2 = q.hz * t.mh[2];
                const float e0 = fmaf(q.hx, t.mh[0], -p0);
                const float e1 = fmaf(q.hy, t.mh[1], -p1);
                const float e2 = fmaf(q.hz, t.mh[2], -p2);
                float f = (p0 - rintf(p0)) + (p1 - rintf(p1));
                f -= rintf(f);
                f += p2 - rintf(p2);
                f -= rintf(f);
                float lo = e0 + e1 + e2;
                lo = fmaf(q.hx, t.ml[0], lo);
                lo = fmaf(q.hy, t.ml[1], lo);
                lo = fmaf(q.hz, t.ml[2], lo);
                lo = fmaf(q.lx, t.mh[0], lo);
                lo = fmaf(q.ly, t.mh[1], lo);
                lo = fmaf(q.lz, t.mh[2], lo);
                const float tau = f - q.dith;
                const float g1 = fmaf(q.x, t.e1[0], fmaf(q.y, t.e1[1], q.z * t.e1[2]));
                const float g2 = fmaf(q.x, t.e2[0], fmaf(q.y, t.e2[1], q.z * t.e2[2]));
                const float g3 = g2 - g1;
                const float a1 = fabsf(g1), a2 = fabsf(g2), a3 = fabsf(g3);
                const float gmax = fmaxf(a1, fmaxf(a2, a3));
                const float ya = -(g1 + g2) * (1.0f / 3.0f);
                const float yb = (2.0f * g1 - g2) * (1.0f / 3.0f);
                const float yc = (2.0f * g2 - g1) * (1.0f / 3.0f);
                const float rr = a.rr, ri = a.ri;
                float rho0h = 0.0f, rho0t, rhoih = 0.0f, rhoit, rho1, rho2;
                if (gmax < kDeltaAM) {
                    const float pp = (g1 * g1 - g1 * g2 + g2 * g2) * (1.0f / 3.0f);
                    const float qq = ya * yb * yc;
                    const float A = fmaf(g1, g1 - g2, g2 * g2);
                    const float q2 = qq * qq;
                    // tail = Psi - 1/2 (as in the forward pass)
                    float re = fmaf(pp, 1.0f / 87178291200.0f, -1.0f / 479001600.0f);
                    re = fmaf(re, pp, 1.0f / 3628800.0f);
                    re = fmaf(re, pp, -1.0f / 40320.0f);
                    re = fmaf(re, pp, 1.0f / 720.0f);
                    float rq = fmaf(pp, 10.0f / 87178291200.0f, -6.0f / 479001600.0f);
                    rq = fmaf(rq, pp, 3.0f / 3628800.0f);
                    rq = fmaf(rq, pp, -1.0f / 40320.0f);
                    const float rq4 = fmaf(q2, 1.0f / 87178291200.0f, rq);
                    float sr = fmaf(re, pp * pp, q2 * rq4);
                    sr = fmaf(A, -1.388888899e-02f, fmaf(A, 1.034802868e-10f, sr));
                    float im = fmaf(pp, 5.0f / 6227020800.0f, -4.0f / 39916800.0f);
                    im = fmaf(im, pp, 3.0f / 362880.0f);
                    im = fmaf(im, pp, -2.0f / 5040.0f);
                    im = fmaf(im, pp, 1.0f / 120.0f);
                    const float iq = fmaf(pp, 4.0f / 6227020800.0f, -1.0f / 39916800.0f);
                    const float si = qq * fmaf(q2, iq, im);
                    // d tail / dp and d tail / dq
                    float dre = fmaf(pp, 6.0f / 87178291200.0f, -5.0f / 479001600.0f);
                    dre = fmaf(dre, pp, 4.0f / 3628800.0f);
                    dre = fmaf(dre, pp, -3.0f / 40320.0f);
                    dre = fmaf(dre, pp, 2.0f / 720.0f);
                    float drq = fmaf(pp, 30.0f / 87178291200.0f, -12.0f / 479001600.0f);
                    drq = fmaf(drq, pp, 3.0f / 3628800.0f);
                    const float Ppr = fmaf(dre, pp, fmaf(q2, drq, -1.0f / 24.0f));
                    const float Pqr = qq * fmaf(2.0f, rq, 4.0f * q2 / 87178291200.0f);
                    float dim = fmaf(pp, 20.0f / 6227020800.0f, -12.0f / 39916800.0f);
                    dim = fmaf(dim, pp, 6.0f / 362880.0f);
                    dim = fmaf(dim, pp, -2.0f / 5040.0f);
                    const float Ppi = qq * fmaf(q2, 4.0f / 6227020800.0f, dim);
                    const float Pqi = fmaf(3.0f * q2, iq, im);
                    // dq/dg1, dq/dg2; dp/dg1 = y_b, dp/dg2 = y_c
                    const float dq1 = (-yb * yc + 2.0f * ya * yc - ya * yb) * (1.0f / 3.0f);
                    const float dq2 = (-yb * yc - ya * yc + 2.0f * ya * yb) * (1.0f / 3.0f);
                    const float P1r = fmaf(Ppr, yb, Pqr * dq1), P1i = fmaf(Ppi, yb, Pqi * dq1);
                    const float P2r = fmaf(Ppr, yc, Pqr * dq2), P2i = fmaf(Ppi, yc, Pqi * dq2);
                    float c, s;
                    expm_turns(tl, tau, lo, c, s);  // exp(-i (t_m - 2 pi d)) = (c, s)
                    // Z = conj(r') E
                    const float Zr = fmaf(rr, c, ri * s), Zi = fmaf(rr, s, -ri * c);
                    rho0h = Zr;
                    rho0t = fmaf(Zr, sr, -Zi * si);
                    rhoih = Zi;
                    rhoit = fmaf(Zr, si, Zi * sr);
                    // Re(Z P1), Re(Z P2)
                    rho1 = fmaf(Zr, P1r, -Zi * P1i);
                    rho2 = fmaf(Zr, P2r, -Zi * P2i);
                } else {
                    const bool caseA = (a2 >= a1) && (a2 >= a3);
                    const bool caseB = !caseA && (a1 >= a3);
                    float oP1, oP2, hP1, hP2, oQ1, oQ2, hQ1, hQ2, D, D1, D2;
                    if (caseA) {
                        oP1 = 1.0f / 6; oP2 = 1.0f / 6; hP1 = -0.5f; hP2 = 0.5f;
                        oQ1 = 1.0f / 6; oQ2 = -1.0f / 3; hQ1 = 0.5f; hQ2 = 0.0f;
                        D = g2; D1 = 0.0f; D2 = 1.0f;
                    } else if (caseB) {
                        oP1 = 1.0f / 6; oP2 = 1.0f / 6; hP1 = -0.5f; hP2 = 0.5f;
                        oQ1 = -1.0f / 3; oQ2 = 1.0f / 6; hQ1 = 0.0f; hQ2 = 0.5f;
                        D = g1; D1 = 1.0f; D2 = 0.0f;
                    } else {
                        oP1 = -1.0f / 3; oP2 = 1.0f / 6; hP1 = 0.0f; hP2 = 0.5f;
                        oQ1 = 1.0f / 6; oQ2 = -1.0f / 3; hQ1 = 0.5f; hQ2 = 0.0f;
                        D = g3; D1 = -1.0f; D2 = 1.0f;
                    }
                    const float offP = oP1 * g1 + oP2 * g2, hP = hP1 * g1 + hP2 * g2;
                    const float offQ = oQ1 * g1 + oQ2 * g2, hQ = hQ1 * g1 + hQ2 * g2;
                    const float inv2pif = 0.159154943091895336f;
                    float cP, sP, cQ, sQ;
                    expm_turns(tl, tau + offP * inv2pif, lo, cP, sP);
                    expm_turns(tl, tau + offQ * inv2pif, lo, cQ, sQ);
                    float scP, dscP, scQ, dscQ;
                    sincd32(hP, scP, dscP);
                    sincd32(hQ, scQ, dscQ);
                    const float SPr = cP * scP, SPi = sP * scP, SQr = cQ * scQ, SQi = sQ * scQ;
                    const float inv = 1.0f / D;
                    const float Gr = -(SPi - SQi) * inv, Gi = (SPr - SQr) * inv;
                    // dS/dg = S (-i doff) + E sinc' dh ; -i o S = o (S.i, -S.r)
                    const float dP1r = fmaf(SPi, oP1, cP * dscP * hP1), dP1i = fmaf(-SPr, oP1, sP * dscP * hP1);
                    const float dP2r = fmaf(SPi, oP2, cP * dscP * hP2), dP2i = fmaf(-SPr, oP2, sP * dscP * hP2);
                    const float dQ1r = fmaf(SQi, oQ1, cQ * dscQ * hQ1), dQ1i = fmaf(-SQr, oQ1, sQ * dscQ * hQ1);
                    const float dQ2r = fmaf(SQi, oQ2, cQ * dscQ * hQ2), dQ2i = fmaf(-SQr, oQ2, sQ * dscQ * hQ2);
                    // V = (i (dS_P - dS_Q) - G dD) / D (already including the phase factor)
                    const float V1r = (-(dP1i - dQ1i) - Gr * D1) * inv, V1i = ((dP1r - dQ1r) - Gi * D1) * inv;
                    const float V2r = (-(dP2i - dQ2i) - Gr * D2) * inv, V2i = ((dP2r - dQ2r) - Gi * D2) * inv;
                    rho0t = fmaf(rr, Gr, ri * Gi);
                    rhoit = fmaf(rr, Gi, -ri * Gr);  // 3 rho_i
                    rho1 = fmaf(rr, V1r, ri * V1i);
                    rho2 = fmaf(rr, V2r, ri * V2i);
                }
                const float xs[3] = {q.x, q.y, q.z};
                b0h += rho0h;
                b0t += rho0t;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    bih[c] = fmaf(rhoih, xs[c], bih[c]);
                    bit[c] = fmaf(rhoit, xs[c], bit[c]);
                    b1[c] = fmaf(rho1, xs[c], b1[c]);
                    b2[c] = fmaf(rho2, xs[c], b2[c]);
                }
            }
            A0h += b0h;
            A0t += b0t;
            for (int c = 0; c < 3; ++c) {
                Aih[c] += bih[c];
                Ait[c] += bit[c];
                A1[c] += b1[c];
                A2[c] += b2[c];
            }
        }
        if (active) {
            double* o = partial + ((int64_t)chunk * nt + tri) * 10;
            o[0] = 0.5 * A0h + A0t;
            for (int c = 0; c < 3; ++c) {
                o[1 + c] = (0.5 * Aih[c] + Ait[c]) * (1.0 / 3.0);
                o[4 + c] = A1[c];
                o[7 + c] = A2[c];
            }
        }
    }
}

// ------------------------------------------------------------------ radial mixed adjoint (ball rules)
// Ball-rule nodes are xi = r omega, so per (direction, triangle) the phase,
// the gaps and the Taylor polynomials are fixed rates and coefficients in r,
// as in the radial pair kernel. For each direction of its chunk a block forms,
// per triangle of its tile, the phase rate omega.m / 2 pi (float pair), the
// tail T = Psi - 1/2 and its partials T_p, T_q as polynomials in rho = r^2:
//     T   = rho (R1 + ... + rho^5 R6) + i r^3 (I0 + ... + rho^4 I4),
//     T_p = (-1/24 + rho a1 + ... + rho^5 a5) + i r^3 (b0 + ... + rho^3 b3),
//     T_q = r^3 (c0 + ... + rho^3 c3) + i (1/120 + rho e1 + ... + rho^4 e4),
// then a warp per triangle runs over the radii (node data staged per
// direction in shared memory).
// With Z = conj(r'_k) exp(-i t_m) and y_b = r yb0, dq/dg1 = r^2 dq1_0 (and
// y_c, dq/dg2 likewise), Psi_1 = T_p y_b + T_q dq/dg1 gives
//     sum_r rho_1 r = yb0 sum_r rho Re(Z T_p) + dq1_0 sum_r r^3 Re(Z T_q),
// so the Taylor branch needs two derivative sums per direction. In the
// largest-gap branch the case constants and D = r D0 factor out of the radius
// sum, leaving five sums. The per-direction results, times omega, go into ten
// float64 per-triangle totals kept in shared memory.
constexpr int ADJ_RMAX = 256;  // radii per direction the radial adjoint stages
constexpr int ADJ_TT = 32;     // triangles per tile of the radial adjoint (one warp of records)

// 48 bytes: a quarter-warp's 128-bit loads of consecutive entries then fall
// in 8 different bank groups (a 32-byte stride would pair them up)
struct __align__(16) AdjRad {
    float rh, rlo;  // radius as a float pair
    float rho, r3;  // r^2, r^3
    float rinv;     // 1 / r
    float thr;      // Taylor branch while gmax0 < thr = DELTA / r
    float pad[6];
};
static_assert(sizeof(AdjRad) == 48, "AdjRad layout");

// Residual rotated by the node's dither, direction-major: nd[d n_rad + ir] =
// (Re, Im of r_k exp(2 pi i d_k), d_k, 0) for node k = ir n_dir + d.
__global__ void adjoint_prep_radial(const double* __restrict__ resid, int n_rad, int64_t n_dir,
                                    int64_t dith_base, float4* __restrict__ nd)
{
    const int64_t n = (int64_t)n_rad * n_dir;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t ir = k / n_dir, d = k - ir * n_dir;
        const float dith = node_dither(dith_base + k);
        double sd, cd;
        sincospi(2.0 * (double)dith, &sd, &cd);
        const double r0 = resid[2 * k], r1 = resid[2 * k + 1];
        nd[d * n_rad + ir] = make_float4((float)(r0 * cd - r1 * sd), (float)(r0 * sd + r1 * cd), dith, 0.0f);
    }
}

// Per-(direction, triangle) quantities of the radial adjoint.
struct AdjDirTri {
    float dmh, dml, gmax0;
    float R[6], I[5];            // T
    float a[5], b[4], c[4], e[4];  // T_p, T_q (constant terms -1/24 and 1/120 implicit)
    float oPt, oQt, hP0, hQ0;    // largest-gap branch: offsets (turns) and half gaps per unit radius
};

__device__ __forceinline__ void adj_dirtri(const TriRecF& t, const float* __restrict__ dir, int64_t n_dir, int64_t d,
                                           AdjDirTri& o, float& d1, float& d2)
{
    const float fx = dir[d], fy = dir[n_dir + d], fz = dir[2 * n_dir + d];
    const float hx = dir[3 * n_dir + d], hy = dir[4 * n_dir + d], hz = dir[5 * n_dir + d];
    const float lx = dir[6 * n_dir + d], ly = dir[7 * n_dir + d], lz = dir[8 * n_dir + d];
    // omega.m / 2 pi as a float pair (as in the radial pair kernel)
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
    d1 = fmaf(fx, t.e1[0], fmaf(fy, t.e1[1], fz * t.e1[2]));
    d2 = fmaf(fx, t.e2[0], fmaf(fy, t.e2[1], fz * t.e2[2]));
    const float d3 = d2 - d1;
    const float a1 = fabsf(d1), a2 = fabsf(d2), a3 = fabsf(d3);
    o.gmax0 = fmaxf(a1, fmaxf(a2, a3));
    const float ya = -(d1 + d2) * (1.0f / 3.0f);
    const float yb = (2.0f * d1 - d2) * (1.0f / 3.0f);
    const float yc = (2.0f * d2 - d1) * (1.0f / 3.0f);
    const float p0 = (d1 * d1 - d1 * d2 + d2 * d2) * (1.0f / 3.0f);
    const float A0 = fmaf(d1, d1 - d2, d2 * d2);
    const float q0 = ya * yb * yc;
    const float q02 = q0 * q0;
    const float p2 = p0 * p0, p3 = p2 * p0, p4 = p2 * p2;
    // T: as in the radial pair kernel (not doubled)
    o.R[0] = fmaf(A0, -1.388888899e-02f, A0 * 1.034802868e-10f);
    o.R[1] = p2 * (1.0f / 720.0f);
    o.R[2] = -(p3 + q02) * (1.0f / 40320.0f);
    o.R[3] = fmaf(3.0f * q02, p0, p4) * (1.0f / 3628800.0f);
    o.R[4] = -fmaf(6.0f * q02, p2, p4 * p0) * (1.0f / 479001600.0f);
    o.R[5] = fmaf(10.0f * q02, p3, fmaf(p3, p3, q02 * q02)) * (1.0f / 87178291200.0f);
    o.I[0] = q0 * (1.0f / 120.0f);
    o.I[1] = -2.0f * q0 * p0 * (1.0f / 5040.0f);
    o.I[2] = 3.0f * q0 * p2 * (1.0f / 362880.0f);
    o.I[3] = -q0 * fmaf(4.0f, p3, q02) * (1.0f / 39916800.0f);
    o.I[4] = q0 * fmaf(5.0f, p4, 4.0f * q02 * p0) * (1.0f / 6227020800.0f);
    // Re T_p = -1/24 + p dre(p) + q^2 drq(p), in rho (a_j multiplies rho^j)
    o.a[0] = 2.0f * p0 * (1.0f / 720.0f);
    o.a[1] = -3.0f * p2 * (1.0f / 40320.0f);
    o.a[2] = fmaf(4.0f, p3, 3.0f * q02) * (1.0f / 3628800.0f);
    o.a[3] = -fmaf(5.0f, p4, 12.0f * q02 * p0) * (1.0f / 479001600.0f);
    o.a[4] = fmaf(6.0f, p4 * p0, 30.0f * q02 * p2) * (1.0f / 87178291200.0f);
    // Im T_p = q (dim(p) + 4 q^2 / 13!) = r^3 (b0 + rho b1 + rho^2 b2 + rho^3 b3)
    o.b[0] = -2.0f * q0 * (1.0f / 5040.0f);
    o.b[1] = 6.0f * q0 * p0 * (1.0f / 362880.0f);
    o.b[2] = -12.0f * q0 * p2 * (1.0f / 39916800.0f);
    o.b[3] = q0 * fmaf(20.0f, p3, 4.0f * q02) * (1.0f / 6227020800.0f);
    // Re T_q = q (2 rq(p) + 4 q^2 / 14!) = r^3 (c0 + ... + rho^3 c3)
    o.c[0] = -2.0f * q0 * (1.0f / 40320.0f);
    o.c[1] = 6.0f * q0 * p0 * (1.0f / 3628800.0f);
    o.c[2] = -12.0f * q0 * p2 * (1.0f / 479001600.0f);
    o.c[3] = q0 * fmaf(20.0f, p3, 4.0f * q02) * (1.0f / 87178291200.0f);
    // Im T_q = im(p) + 3 q^2 iq(p) = 1/120 + rho e1 + ... + rho^4 e4
    o.e[0] = -2.0f * p0 * (1.0f / 5040.0f);
    o.e[1] = 3.0f * p2 * (1.0f / 362880.0f);
    o.e[2] = -fmaf(4.0f, p3, 3.0f * q02) * (1.0f / 39916800.0f);
    o.e[3] = fmaf(5.0f, p4, 12.0f * q02 * p0) * (1.0f / 6227020800.0f);
    // largest-gap branch: A = (a, c) with d2, B = (a, b) with d1, C = (b, c) with d3
    const bool caseA = (a2 >= a1) && (a2 >= a3);
    const bool caseB = !caseA && (a1 >= a3);
    const bool caseC = !caseA && !caseB;
    const float inv4pi = 0.0795774715459476679f;
    o.oPt = caseC ? -inv4pi * yb : -inv4pi * ya;
    o.hP0 = caseC ? 0.5f * d2 : 0.5f * d3;
    o.oQt = caseB ? -inv4pi * yb : -inv4pi * yc;
    o.hQ0 = caseB ? 0.5f * d2 : 0.5f * d1;
}

// Per-(direction, triangle) record of the radial adjoint in shared memory.
struct __align__(16) AdjRec {
    AdjDirTri q;
    float d1, d2;    // omega.e1, omega.e2 (the largest-gap case and the Psi_1/Psi_2 factors)
    float ihP, ihQ;  // 1 / hP0, 1 / hQ0 (0 where the half gap is 0)
    float pad;
};
static_assert(sizeof(AdjRec) % 16 == 0, "AdjRec layout");

// One lane's radii of a (direction, triangle) record in the radial adjoint:
// lane l takes radii l, l + 32, ... and adds into its partial sums. BIG folds
// the phase's rounding error into the reduced phase (phases of 2^13 turns or
// more, where it can reach table steps); the record decides, warp-uniformly.
template <bool BIG>
__device__ __forceinline__ void adj_lane_radii(const AdjRad* __restrict__ rt, const float4* __restrict__ sn,
                                               const AdjRec& rec, const TabEntry* __restrict__ tl, int lane, int n_rad,
                                               float& S0h, float& S0t, float& Sih, float& Sit, float& SA, float& SB,
                                               float& xP, float& yP, float& xQ, float& yQ, float& G0)
{
    const AdjDirTri& q = rec.q;
    for (int ir = lane; ir < n_rad; ir += 32) {
        const AdjRad a = rt[ir];
        const float4 w = sn[ir];
        const float rr = w.x, ri = w.y;
        const float P = a.rh * q.dmh;
        const float e = fmaf(a.rh, q.dmh, -P);
        float lo = fmaf(a.rh, q.dml, fmaf(a.rlo, q.dmh, e));
        float tau = (P - rintf(P)) - w.z;
        if (BIG) {
            const float tl2 = tau + lo;
            lo = two_sum_err(tau, lo, tl2);
            tau = tl2;
        }
        if (q.gmax0 < a.thr) {
            float c, s;
            expm_turns_fast(tl, tau, lo, c, s);
            const float Zr = fmaf(rr, c, ri * s), Zi = fmaf(rr, s, -ri * c);
            const float rho = a.rho, r3 = a.r3;
            float sr = fmaf(fmaf(fmaf(fmaf(q.R[5], rho, q.R[4]), rho, q.R[3]), rho, q.R[2]), rho, q.R[1]);
            sr = fmaf(sr, rho, q.R[0]) * rho;
            float si = fmaf(fmaf(fmaf(q.I[4], rho, q.I[3]), rho, q.I[2]), rho, q.I[1]);
            si = fmaf(si, rho, q.I[0]) * r3;
            S0h += Zr;
            S0t = fmaf(Zr, sr, fmaf(-Zi, si, S0t));
            Sih = fmaf(Zi, a.rh, Sih);
            Sit = fmaf(fmaf(Zr, si, Zi * sr), a.rh, Sit);
            float Ap = fmaf(fmaf(fmaf(fmaf(q.a[4], rho, q.a[3]), rho, q.a[2]), rho, q.a[1]), rho, q.a[0]);
            Ap = fmaf(Ap, rho, -1.0f / 24.0f);
            const float Bp = fmaf(fmaf(fmaf(q.b[3], rho, q.b[2]), rho, q.b[1]), rho, q.b[0]) * r3;
            const float Cq = fmaf(fmaf(fmaf(q.c[3], rho, q.c[2]), rho, q.c[1]), rho, q.c[0]) * r3;
            float Eq = fmaf(fmaf(fmaf(q.e[3], rho, q.e[2]), rho, q.e[1]), rho, q.e[0]);
            Eq = fmaf(Eq, rho, 1.0f / 120.0f);
            SA = fmaf(rho, fmaf(Zr, Ap, -Zi * Bp), SA);
            SB = fmaf(r3, fmaf(Zr, Cq, -Zi * Eq), SB);
        } else {
            float cP, sP, cQ, sQ;
            expm_turns_fast(tl, fmaf(a.rh, q.oPt, tau), lo, cP, sP);
            expm_turns_fast(tl, fmaf(a.rh, q.oQt, tau), lo, cQ, sQ);
            float scP, dscP, scQ, dscQ;
            sincd32_inv(a.rh * q.hP0, a.rinv * rec.ihP, scP, dscP);
            sincd32_inv(a.rh * q.hQ0, a.rinv * rec.ihQ, scQ, dscQ);
            // X = E sinc(h), Y = i E sinc'(h); x = Re(conj r' X), y = Re(conj r' Y)
            const float XPr = cP * scP, XPi = sP * scP, XQr = cQ * scQ, XQi = sQ * scQ;
            xP = fmaf(rr, XPr, fmaf(ri, XPi, xP));
            xQ = fmaf(rr, XQr, fmaf(ri, XQi, xQ));
            yP = fmaf(dscP, fmaf(ri, cP, -rr * sP), yP);
            yQ = fmaf(dscQ, fmaf(ri, cQ, -rr * sQ), yQ);
            // Re(conj r' i (X_P - X_Q)) / r
            G0 = fmaf(fmaf(ri, XPr - XQr, -rr * (XPi - XQi)), a.rinv, G0);
        }
    }
}

// A warp per (direction, triangle), its lanes on the radii: lane l takes radii
// l, l + 32, ... of the direction, so the Taylor / largest-gap choice, which
// moves with r, splits a warp at most once per record. Each lane combines its
// partial sums into the direction's four results with the record's
// warp-uniform constants; a warp reduction gives the direction's results,
// which one thread per triangle adds, times omega, to the triangle's float64
// totals in shared memory after the next barrier.
__global__ void __launch_bounds__(ADJ_TPB) adjoint_kernel_radial(const TriRecF* __restrict__ rec, int64_t nt,
                                                                 const float4* __restrict__ nd,
                                                                 const double* __restrict__ rad, int n_rad,
                                                                 const float* __restrict__ dir, int64_t n_dir,
                                                                 const AdjPlan p, double* __restrict__ partial)
{
    __shared__ AdjRad rt[ADJ_RMAX];
    __shared__ float4 sn[ADJ_RMAX];
    __shared__ AdjRec srec[ADJ_TT];
    __shared__ double acc[10][ADJ_TT];
    __shared__ float4 tres[ADJ_TT];  // a direction's results per triangle: (T0, Ti, T1, T2)
    __shared__ TabEntry etab[kTab * kTabRep];
    __shared__ int s_rbits;  // the largest radius, as bits (radii are positive)
    fill_exp_table(etab);
    const TabEntry* tl = exp_table_lane(etab);
    if (threadIdx.x == 0) s_rbits = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n_rad; i += ADJ_TPB) {
        const double r = rad[i];
        AdjRad a;
        a.rh = (float)r;
        atomicMax(&s_rbits, __float_as_int(a.rh));  // read after the item loop's first barrier
        a.rlo = (float)(r - (double)a.rh);
        a.rho = (float)(r * r);
        a.r3 = (float)(r * r * r);
        a.rinv = (float)(1.0 / r);
        // Lanes take radii i = lane + 32 k, so the radii of one pass of a warp
        // are the group of 32 consecutive ones holding i. Where the group's
        // radii lie within a factor of 2, all of them take the branch of the
        // group's largest radius (as in the radial pair kernel), so that no
        // warp runs both: Taylor only below DELTA, the largest-gap branch
        // from DELTA / 2 up.
        const int g0 = i & ~31, g1 = min(g0 + 32, n_rad);
        double rmin = rad[g0], rmax = rad[g0];
        for (int k = g0 + 1; k < g1; ++k) {
            rmin = fmin(rmin, rad[k]);
            rmax = fmax(rmax, rad[k]);
        }
        a.thr = (float)((double)kDeltaAM / (rmax < 2.0 * rmin ? rmax : r));
        for (int k = 0; k < 6; ++k) a.pad[k] = 0.0f;
        rt[i] = a;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t item = blockIdx.x; item < p.n_items; item += gridDim.x) {
        const int64_t tt = item / p.nchunks;
        const int chunk = (int)(item - tt * p.nchunks);
        const int64_t tri0 = tt * ADJ_TT;
        __syncthreads();  // the previous item's totals have been written out
        for (int i = threadIdx.x; i < 10 * ADJ_TT; i += ADJ_TPB) acc[i / ADJ_TT][i % ADJ_TT] = 0.0;
        const int64_t d0 = (int64_t)chunk * p.dirs_per_chunk;
        int64_t d1e = d0 + p.dirs_per_chunk;
        if (d1e > n_dir) d1e = n_dir;
        for (int64_t d = d0; d <= d1e; ++d) {
            __syncthreads();
            // the previous direction's results, times its omega, into the
            // triangles' float64 totals: one thread per triangle
            if (d > d0 && threadIdx.x < ADJ_TT && tri0 + threadIdx.x < nt) {
                const int64_t dp = d - 1;
                const double ux = dir[dp], uy = dir[n_dir + dp], uz = dir[2 * n_dir + dp];
                const float4 r = tres[threadIdx.x];
                const int j = threadIdx.x;
                acc[0][j] += (double)r.x;
                acc[1][j] += ux * r.y;
                acc[2][j] += uy * r.y;
                acc[3][j] += uz * r.y;
                acc[4][j] += ux * r.z;
                acc[5][j] += uy * r.z;
                acc[6][j] += uz * r.z;
                acc[7][j] += ux * r.w;
                acc[8][j] += uy * r.w;
                acc[9][j] += uz * r.w;
            }
            if (d == d1e) break;
            for (int i = threadIdx.x; i < n_rad; i += ADJ_TPB) sn[i] = nd[d * n_rad + i];
            if (threadIdx.x < ADJ_TT) {
                AdjRec r{};
                const int64_t tri = tri0 + threadIdx.x;
                if (tri < nt) {
                    adj_dirtri(rec[tri], dir, n_dir, d, r.q, r.d1, r.d2);
                    r.ihP = r.q.hP0 != 0.0f ? 1.0f / r.q.hP0 : 0.0f;
                    r.ihQ = r.q.hQ0 != 0.0f ? 1.0f / r.q.hQ0 : 0.0f;
                }
                srec[threadIdx.x] = r;
            }
            __syncthreads();
            for (int j = warp; j < ADJ_TT; j += ADJ_TPB / 32) {
                if (tri0 + j >= nt) break;  // warp-uniform
                const AdjDirTri& q = srec[j].q;
                // phases of 2^13 turns or more (a mesh far from the origin):
                // lo, the high product's rounding error and the low products,
                // can then reach table steps and is folded into tau with its
                // exact rounding error (warp-uniform)
                const bool big = fabsf(q.dmh) * __int_as_float(s_rbits) >= 8192.0f;
                float S0h = 0.0f, S0t = 0.0f, Sih = 0.0f, Sit = 0.0f, SA = 0.0f, SB = 0.0f;
                float xP = 0.0f, yP = 0.0f, xQ = 0.0f, yQ = 0.0f, G0 = 0.0f;
                if (big)
                    adj_lane_radii<true>(rt, sn, srec[j], tl, lane, n_rad, S0h, S0t, Sih, Sit, SA, SB, xP, yP, xQ, yQ,
                                         G0);
                else
                    adj_lane_radii<false>(rt, sn, srec[j], tl, lane, n_rad, S0h, S0t, Sih, Sit, SA, SB, xP, yP, xQ,
                                          yQ, G0);
                // this lane's share of sum_r rho_0, sum_r rho_i r, sum_r rho_1 r, sum_r rho_2 r
                const float g1d = srec[j].d1, g2d = srec[j].d2;
                const float ya = -(g1d + g2d) * (1.0f / 3.0f);
                const float yb = (2.0f * g1d - g2d) * (1.0f / 3.0f);
                const float yc = (2.0f * g2d - g1d) * (1.0f / 3.0f);
                const float dq1 = (-yb * yc + 2.0f * ya * yc - ya * yb) * (1.0f / 3.0f);
                const float dq2 = (-yb * yc - ya * yc + 2.0f * ya * yb) * (1.0f / 3.0f);
                float T0 = fmaf(0.5f, S0h, S0t);
                float Ti = fmaf(0.5f, Sih, Sit) * (1.0f / 3.0f);
                float T1 = fmaf(yb, SA, dq1 * SB);
                float T2 = fmaf(yc, SA, dq2 * SB);
                if (q.gmax0 > 0.0f) {  // warp-uniform; with gmax0 = 0 no radius takes the largest-gap branch
                    const float g3d = g2d - g1d;
                    const float a1 = fabsf(g1d), a2 = fabsf(g2d), a3 = fabsf(g3d);
                    const bool caseA = (a2 >= a1) && (a2 >= a3);
                    const bool caseB = !caseA && (a1 >= a3);
                    float oP1, oP2, hP1, hP2, oQ1, oQ2, hQ1, hQ2, D0, D1, D2;
                    if (caseA) {
                        oP1 = 1.0f / 6; oP2 = 1.0f / 6; hP1 = -0.5f; hP2 = 0.5f;
                        oQ1 = 1.0f / 6; oQ2 = -1.0f / 3; hQ1 = 0.5f; hQ2 = 0.0f;
                        D0 = g2d; D1 = 0.0f; D2 = 1.0f;
                    } else if (caseB) {
                        oP1 = 1.0f / 6; oP2 = 1.0f / 6; hP1 = -0.5f; hP2 = 0.5f;
                        oQ1 = -1.0f / 3; oQ2 = 1.0f / 6; hQ1 = 0.0f; hQ2 = 0.5f;
                        D0 = g1d; D1 = 1.0f; D2 = 0.0f;
                    } else {
                        oP1 = -1.0f / 3; oP2 = 1.0f / 6; hP1 = 0.0f; hP2 = 0.5f;
                        oQ1 = 1.0f / 6; oQ2 = -1.0f / 3; hQ1 = 0.5f; hQ2 = 0.0f;
                        D0 = g3d; D1 = -1.0f; D2 = 1.0f;
                    }
                    const float iD = 1.0f / D0;
                    const float G0D = G0 * iD;
                    T0 += G0D;
                    Ti = fmaf(xP - xQ, iD * (1.0f / 3.0f), Ti);
                    T1 += fmaf(oP1 * xP + hP1 * yP - oQ1 * xQ - hQ1 * yQ, iD, -D1 * G0D * iD);
                    T2 += fmaf(oP2 * xP + hP2 * yP - oQ2 * xQ - hQ2 * yQ, iD, -D2 * G0D * iD);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    T0 += __shfl_xor_sync(0xffffffffu, T0, o);
                    Ti += __shfl_xor_sync(0xffffffffu, Ti, o);
                    T1 += __shfl_xor_sync(0xffffffffu, T1, o);
                    T2 += __shfl_xor_sync(0xffffffffu, T2, o);
                }
                if (lane == 0) tres[j] = make_float4(T0, Ti, T1, T2);
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < 10 * ADJ_TT; i += ADJ_TPB) {
            const int j = i / 10, c = i % 10;
            const int64_t tri = tri0 + j;
            if (tri < nt) partial[((int64_t)chunk * nt + tri) * 10 + c] = acc[c][j];
        }
    }
}

// Sum the node chunks per triangle (fixed order), apply d gamma/dp_j and gamma,
// and store the three corner contributions. Each (vertex, component) records
// the largest binary exponent among its contributions, and each vertex its
// number of incident corners, for the order-independent scatter below.
__global__ void adjoint_finalize(const double* __restrict__ partial, int nchunks, const TriRecD* __restrict__ rec,
                                 int64_t nt, const int32_t* __restrict__ tris, int64_t nv,
                                 double* __restrict__ corner, int* __restrict__ expo, int* __restrict__ deg)
{
    for (int64_t tri = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; tri < nt;
         tri += (int64_t)gridDim.x * blockDim.x) {
        double S[10];
#pragma unroll
        for (int c = 0; c < 10; ++c) S[c] = 0.0;
        for (int ch = 0; ch < nchunks; ++ch)
#pragma unroll
            for (int c = 0; c < 10; ++c) S[c] += partial[((int64_t)ch * nt + tri) * 10 + c];
        const TriRecD t = rec[tri];
        const double gam = t.gam;
        double* out = corner + 9 * tri;
        if (!(gam > 0.0)) {  // degenerate triangles contribute nothing
#pragma unroll
            for (int c = 0; c < 9; ++c) out[c] = 0.0;
            continue;
        }
        const double* e1 = t.e1;
        const double* e2 = t.e2;
        double nrm[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        for (int c = 0; c < 3; ++c) nrm[c] /= gam;
        // p_b - p_c = e1 - e2, p_c - p_a = e2, p_a - p_b = -e1
        const double ea[3] = {e1[0] - e2[0], e1[1] - e2[1], e1[2] - e2[2]};
        const double eb[3] = {e2[0], e2[1], e2[2]};
        const double ec[3] = {-e1[0], -e1[1], -e1[2]};
        const double* ev[3] = {ea, eb, ec};
        for (int j = 0; j < 3; ++j) {
            const int64_t v = tris[3 * tri + j];
            const bool ok = v >= 0 && v < nv;
            if (ok) atomicAdd(&deg[v], 1);
            const double* e = ev[j];
            const double dg[3] = {e[1] * nrm[2] - e[2] * nrm[1], e[2] * nrm[0] - e[0] * nrm[2],
                                  e[0] * nrm[1] - e[1] * nrm[0]};
            for (int c = 0; c < 3; ++c) {
                // sum_k Re(conj r dG/dt_j) xi_c: a -> rho_i - rho_1 - rho_2, b -> rho_i + rho_1, c -> rho_i + rho_2
                const double si = S[1 + c], s1 = S[4 + c], s2 = S[7 + c];
                const double sj = (j == 0) ? si - s1 - s2 : (j == 1 ? si + s1 : si + s2);
                const double val = S[0] * dg[c] + gam * sj;
                out[3 * j + c] = val;
                // |val| < 2^E with E = (biased exponent field) - 1022, also for
                // subnormals; stored as E + 2048 > 0, so 0 means "all zero"
                const int biased = (int)((__double_as_longlong(val) >> 52) & 0x7ff);
                if (ok && val != 0.0) atomicMax(&expo[3 * v + c], biased - 1022 + 2048);
            }
        }
    }
}

// Add the corner contributions into grad in an order-independent way: each
// contribution to (vertex v, component c) is rounded to a multiple of 2^g,
// g = E + L - 53, where every contribution there is below 2^E in magnitude and
// L = ceil(log2(number of corners at v)). Every partial sum is then an integer
// times 2^g of magnitude at most 2^53 * 2^g, exact in float64, so the float64
// atomic adds give the same bits in any order. The rounding error per
// contribution is at most 2^(E + L - 54), the size of one float64 rounding of
// the sum itself.
__global__ void adjoint_scatter(const double* __restrict__ corner, const int32_t* __restrict__ tris, int64_t nt,
                                int64_t nv, const int* __restrict__ expo, const int* __restrict__ deg,
                                double* __restrict__ grad)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < 3 * nt;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = tris[k];
        if (v < 0 || v >= nv) continue;
        const int d = deg[v];
        const int L = 32 - __clz(d - 1);
        for (int c = 0; c < 3; ++c) {
            const int es = expo[3 * v + c];
            const double val = corner[3 * k + c];
            if (es == 0 || val == 0.0) continue;
            const int g = es - 2048 + L - 53;
            const double r = ldexp(rint(ldexp(val, -g)), g);
            if (r != 0.0) atomicAdd(&grad[3 * v + c], r);
        }
    }
}

int resident_adjoint(wd_ctx* ctx, int precision, bool radial = false)
{
    if (radial) return wd_resident(ctx, OCC_ADJOINT + 2, adjoint_kernel_radial, ADJ_TPB);
    if (precision == WD_MIXED) return wd_resident(ctx, OCC_ADJOINT + 1, adjoint_kernel_mixed, ADJ_TPB);
    return wd_resident(ctx, OCC_ADJOINT, adjoint_kernel_f64, ADJ_TPB);
}

}  // namespace

wd_status wd_plan_adjoint(wd_ctx* ctx, int precision, int64_t n_nodes, int64_t n_tris, AdjPlan* plan)
{
    AdjPlan p;
    p.n_tb = (n_tris + ADJ_TPB - 1) / ADJ_TPB;
    p.n_node_tiles = (n_nodes + ADJ_NPT - 1) / ADJ_NPT;
    const int64_t resident = resident_adjoint(ctx, precision);
    const int64_t target = 4 * resident;
    int64_t nchunks = 1;
    if (p.n_tb > 0 && p.n_tb < target && p.n_node_tiles > 1) {
        nchunks = (target + p.n_tb - 1) / p.n_tb;
        if (nchunks > p.n_node_tiles) nchunks = p.n_node_tiles;
    }
    int64_t tpc = p.n_node_tiles > 0 ? (p.n_node_tiles + nchunks - 1) / nchunks : 0;
    if (tpc > 0) nchunks = (p.n_node_tiles + tpc - 1) / tpc;
    if (nchunks < 1) nchunks = 1;
    p.tiles_per_chunk = (int)tpc;
    p.nchunks = (int)nchunks;
    p.n_items = p.n_tb * p.nchunks;
    p.grid = (int)(p.n_items < resident ? p.n_items : resident);
    *plan = p;
    return WD_OK;
}

wd_status wd_plan_adjoint_rule(wd_ctx* ctx, const wd_rule* rule, int precision, int64_t n_tris, AdjPlan* plan)
{
    if (precision != WD_MIXED || !rule->d_rad || rule->n_rad > ADJ_RMAX || rule->n_dir <= 0)
        return wd_plan_adjoint(ctx, precision, rule->n_eval, n_tris, plan);
    AdjPlan p;
    p.radial = true;
    p.n_tb = (n_tris + ADJ_TT - 1) / ADJ_TT;  // tiles of ADJ_TT triangles
    const int64_t resident = resident_adjoint(ctx, precision, true);
    const int64_t target = 4 * resident;
    int64_t nchunks = 1;
    if (p.n_tb > 0 && p.n_tb < target) nchunks = (target + p.n_tb - 1) / p.n_tb;
    if (nchunks > rule->n_dir) nchunks = rule->n_dir;
    p.dirs_per_chunk = (rule->n_dir + nchunks - 1) / nchunks;
    p.nchunks = (int)((rule->n_dir + p.dirs_per_chunk - 1) / p.dirs_per_chunk);
    p.n_items = p.n_tb * p.nchunks;
    p.grid = (int)(p.n_items < resident ? p.n_items : resident);
    *plan = p;
    return WD_OK;
}

size_t wd_adjoint_radial_bytes(const wd_rule* rule)
{
    return sizeof(float4) * (size_t)(rule->n_eval > 0 ? rule->n_eval : 1);
}

size_t wd_adjoint_scatter_bytes(int64_t nt, int64_t nv)
{
    const size_t corner = ((sizeof(double) * 9 * (size_t)(nt > 0 ? nt : 1)) + 255) & ~size_t(255);
    return corner + sizeof(int) * 4 * (size_t)(nv > 0 ? nv : 1);
}

wd_status wd_launch_adjoint(wd_ctx* ctx, int precision, const AdjPlan& plan, const wd_rule* rule,
                            const double* d_resid, const void* d_rec, const void* d_rec_mixed, int64_t nt,
                            void* d_radial, double* d_partial, void* d_scatter, const int32_t* d_tris, int64_t nv,
                            double* d_grad, cudaStream_t st)
{
    if (nt == 0) return WD_OK;
    const double* d_xi = rule->d_xi;
    const int64_t n = rule->n_eval;
    if (plan.radial && plan.n_items > 0) {
        if (precision != WD_MIXED || !rule->d_rad || !d_radial) {
            wd_set_error("internal: radial adjoint plan without a mixed ball rule");
            return WD_EINVAL;
        }
        float4* nd = static_cast<float4*>(d_radial);
        int64_t g = (n + 255) / 256;
        const int64_t cap = (int64_t)ctx->num_sms * 8;
        if (g > cap) g = cap;
        adjoint_prep_radial<<<(int)g, 256, 0, st>>>(d_resid, rule->n_rad, rule->n_dir,
                                                    (int64_t)rule->shell0 * rule->n_dir, nd);
        ctx->launches++;
        WD_CUDA(cudaGetLastError());
        adjoint_kernel_radial<<<plan.grid, ADJ_TPB, 0, st>>>(static_cast<const TriRecF*>(d_rec_mixed), nt, nd,
                                                            rule->d_rad, rule->n_rad, rule->d_dir, rule->n_dir,
                                                            plan, d_partial);
        ctx->launches++;
        WD_CUDA(cudaGetLastError());
    } else if (plan.n_items > 0) {
        if (precision == WD_MIXED)
            adjoint_kernel_mixed<<<plan.grid, ADJ_TPB, 0, st>>>(d_xi, n, d_resid,
                                                               static_cast<const TriRecF*>(d_rec_mixed), nt, plan,
                                                               d_partial);
        else
            adjoint_kernel_f64<<<plan.grid, ADJ_TPB, 0, st>>>(d_xi, n, d_resid, static_cast<const TriRecD*>(d_rec),
                                                             nt, plan, d_partial);
        ctx->launches++;
        WD_CUDA(cudaGetLastError());
    }
    const size_t corner_bytes = ((sizeof(double) * 9 * (size_t)nt) + 255) & ~size_t(255);
    double* corner = static_cast<double*>(d_scatter);
    int* expo = reinterpret_cast<int*>(static_cast<unsigned char*>(d_scatter) + corner_bytes);
    int* deg = expo + 3 * (nv > 0 ? nv : 1);
    WD_CUDA(cudaMemsetAsync(expo, 0, sizeof(int) * 4 * (size_t)(nv > 0 ? nv : 1), st));
    const int64_t cap = (int64_t)ctx->num_sms * 8;
    int64_t g = (nt + 255) / 256;
    if (g > cap) g = cap;
    adjoint_finalize<<<(int)g, 256, 0, st>>>(d_partial, plan.n_items > 0 ? plan.nchunks : 0,
                                             static_cast<const TriRecD*>(d_rec), nt, d_tris, nv, corner, expo, deg);
    ctx->launches++;
    WD_CUDA(cudaGetLastError());
    g = (3 * nt + 255) / 256;
    if (g > cap) g = cap;
    adjoint_scatter<<<(int)g, 256, 0, st>>>(corner, d_tris, nt, nv, expo, deg, d_grad);
    ctx->launches++;
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}
