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
// Work items are (block of 128 triangles, chunk of frequency nodes); nodes are
// staged in shared-memory tiles; each thread keeps the ten per-triangle sums
// sum Re(conj r G), sum rho_i xi, sum rho_1 xi, sum rho_2 xi in float64. A
// second kernel adds the chunks in fixed order, applies the geometry and
// scatters to the vertices with float64 atomic adds.
#include <cstdint>

#include "wd_internal.h"

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

// Sum the node chunks per triangle (fixed order), apply d gamma/dp_j and gamma,
// and add the three vertex contributions to grad (float64 atomics).
__global__ void adjoint_finalize(const double* __restrict__ partial, int nchunks, const TriRecD* __restrict__ rec,
                                 int64_t nt, const int32_t* __restrict__ tris, int64_t nv, double* __restrict__ grad)
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
        if (!(gam > 0.0)) continue;  // degenerate triangles contribute nothing
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
            if (v < 0 || v >= nv) continue;
            const double* e = ev[j];
            const double dg[3] = {e[1] * nrm[2] - e[2] * nrm[1], e[2] * nrm[0] - e[0] * nrm[2],
                                  e[0] * nrm[1] - e[1] * nrm[0]};
            for (int c = 0; c < 3; ++c) {
                // sum_k Re(conj r dG/dt_j) xi_c: a -> rho_i - rho_1 - rho_2, b -> rho_i + rho_1, c -> rho_i + rho_2
                const double si = S[1 + c], s1 = S[4 + c], s2 = S[7 + c];
                const double sj = (j == 0) ? si - s1 - s2 : (j == 1 ? si + s1 : si + s2);
                atomicAdd(&grad[3 * v + c], S[0] * dg[c] + gam * sj);
            }
        }
    }
}

int resident_adjoint(wd_ctx* ctx)
{
    static int cached[64] = {0};
    int& c = cached[ctx->device & 63];
    if (c == 0) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, adjoint_kernel_f64, ADJ_TPB, 0) != cudaSuccess ||
            per_sm < 1) {
            cudaGetLastError();
            per_sm = 1;
        }
        c = per_sm * ctx->num_sms;
    }
    return c;
}

}  // namespace

wd_status wd_plan_adjoint(wd_ctx* ctx, int, int64_t n_nodes, int64_t n_tris, AdjPlan* plan)
{
    AdjPlan p;
    p.n_tb = (n_tris + ADJ_TPB - 1) / ADJ_TPB;
    p.n_node_tiles = (n_nodes + ADJ_NPT - 1) / ADJ_NPT;
    const int64_t resident = resident_adjoint(ctx);
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

wd_status wd_launch_adjoint(wd_ctx* ctx, int, const AdjPlan& plan, const double* d_xi, int64_t n,
                            const double* d_resid, const void* d_rec, int64_t nt, double* d_partial,
                            const int32_t* d_tris, int64_t nv, double* d_grad, cudaStream_t st)
{
    if (nt == 0) return WD_OK;
    if (plan.n_items > 0) {
        adjoint_kernel_f64<<<plan.grid, ADJ_TPB, 0, st>>>(d_xi, n, d_resid, static_cast<const TriRecD*>(d_rec), nt,
                                                         plan, d_partial);
        ctx->launches++;
        WD_CUDA(cudaGetLastError());
    }
    int64_t g = (nt + 255) / 256;
    const int64_t cap = (int64_t)ctx->num_sms * 8;
    if (g > cap) g = cap;
    adjoint_finalize<<<(int)g, 256, 0, st>>>(d_partial, plan.n_items > 0 ? plan.nchunks : 0,
                                             static_cast<const TriRecD*>(d_rec), nt, d_tris, nv, d_grad);
    ctx->launches++;
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}
