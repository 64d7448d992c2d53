// Device building blocks of the mixed-precision path, shared by the pair
// kernels (wd_pair.cu) and the adjoint (wd_adjoint.cu).
#pragma once

#include <cstdint>

struct NodeF {
    float x, y, z;     // xi (radians), float32
    float hx, hy, hz;  // xi / 2 pi, high float32 part
    float lx, ly, lz;  // xi / 2 pi - high part
    float dith;        // per-node phase origin shift in turns, [-1/2, 1/2)
};

// Per-node phase dither. The float32 rounding of each pair's terms is a
// deterministic function of its phases; at low frequency neighbouring nodes
// see nearly equal phases, round alike, and the per-node errors add up
// coherently in the weighted sum against mu^ - nu^, which is small there.
// Shifting every phase of node k by a pseudo-random turn offset d_k and
// rotating the node's sum back by exp(-2 pi i d_k) in float64 leaves the
// result unchanged (translation theorem) while making the rounding errors of
// different nodes independent, so they average out in the quadrature sum.
// The shift lies in [-1/2, 1/2) on a 2^-20 grid: the reduced phase f is in
// [-1/2, 1/2], so f - d stays below 1 in magnitude, and when f itself lies on
// a coarse grid (large high products, e.g. a frequency component exactly 0)
// f - d is exact. A shift in [0, 1) would push half the phases past 1, where
// rounding to the 2^-23 grid depends on d's last bit alone, the same for every
// triangle of the node: a coherent phase error.
__device__ __forceinline__ float node_dither(int64_t node)
{
    uint32_t h = (uint32_t)node * 0x9E3779B9u + 0x7F4A7C15u;
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return (float)(h >> 12) * 9.5367431640625e-7f - 0.5f;  // 20 bits, exact in float32
}

// The same hash as a whole number of exp-table steps, j in [-kTab/2, kTab/2)
// (kTab = 128 steps per turn), for a kernel that feeds its unreduced phase
// tau straight to the table exponential with the magic constant kMagic - j:
// the table index moves by -j while the residual u stays exact, so every pair
// of the node comes out multiplied by exp(2 pi i j / kTab), undone in float64
// as the dither d = j / kTab. No rounding enters the phase itself.
__device__ __forceinline__ int node_dither_steps(int64_t node)
{
    uint32_t h = (uint32_t)node * 0x9E3779B9u + 0x7F4A7C15u;
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return (int)(h >> 25) - 64;
}

// sin(x)/x: reduction by the nearest multiple of pi (two-constant split) and
// the Taylor polynomial of sin(r)/r on |r| <= pi/2 (remainder < 5e-10).
__device__ __forceinline__ float sinc32(float x)
{
    const float k = rintf(x * 0.318309886183790672f);
    float r = fmaf(-k, 3.14159274101257324f, x);
    r = fmaf(-k, -8.74227766e-8f, r);
    const float r2 = r * r;
    float P = -1.0f / 1307674368000.0f;
    P = fmaf(P, r2, 1.0f / 6227020800.0f);
    P = fmaf(P, r2, -1.0f / 39916800.0f);
    P = fmaf(P, r2, 1.0f / 362880.0f);
    P = fmaf(P, r2, -1.0f / 5040.0f);
    P = fmaf(P, r2, 1.0f / 120.0f);
    P = fmaf(P, r2, -1.0f / 6.0f);
    P = fmaf(P, r2, 1.0f);
    // sin(x) = (-1)^k r P; for k = 0, r == x exactly
    const float half = 0.5f * k;
    const float sgn = (half == rintf(half)) ? 1.0f : -1.0f;
    const float qf = (k == 0.0f) ? 1.0f : __fdividef(sgn * r, x);
    return P * qf;
}

// sin(x)/x given invx = 1/x (anything where x = 0): sinc32 with the multiple
// k of pi found by a magic-number add (1.5 * 2^23 is even, so the low bit of
// the sum is the parity of k, which sets the sign of sin(x) = (-1)^k sin(r))
// and a multiplication by invx in place of the division.
__device__ __forceinline__ float sinc32_inv(float x, float invx)
{
    const float km = fmaf(x, 0.318309886183790672f, 12582912.0f);
    const float k = km - 12582912.0f;  // exact
    float r = fmaf(-k, 3.14159274101257324f, x);
    r = fmaf(-k, -8.74227766e-8f, r);
    const float r2 = r * r;
    float P = -1.0f / 1307674368000.0f;
    P = fmaf(P, r2, 1.0f / 6227020800.0f);
    P = fmaf(P, r2, -1.0f / 39916800.0f);
    P = fmaf(P, r2, 1.0f / 362880.0f);
    P = fmaf(P, r2, -1.0f / 5040.0f);
    P = fmaf(P, r2, 1.0f / 120.0f);
    P = fmaf(P, r2, -1.0f / 6.0f);
    P = fmaf(P, r2, 1.0f);
    // for k = 0, r == x exactly and sinc = P
    const float rs = __int_as_float(__float_as_int(r) ^ (__float_as_int(km) << 31));
    const float qf = (k == 0.0f) ? 1.0f : rs * invx;
    return P * qf;
}

// exp(-i 2 pi tau) for a phase in turns given as the unevaluated float pair
// tau + tlo, without rounding 2 pi into the argument. tau = j/128 + u with j
// the nearest multiple (found with a magic-number add, so no float-to-int
// conversion) and |u| <= 1/256 exactly; exp(-2 pi i j/128) comes from a table
// of float pairs (hi + lo, from float64 sincospi), exp(-i x), x = 2 pi u, from
// short Taylor polynomials (|x| <= pi/128: cos remainder 3e-13; the sin
// remainder, 7e-11, is odd in x and moves the mean amplitude by 5e-13), and
// the two are combined in pair arithmetic. Unlike a float32 polynomial on a
// quarter turn, whose rounded coefficients bias its mean amplitude by about
// 1e-9, this has a mean relative bias near 1e-11, which matters because the
// phases of a node's triangles are uniformly spread and any mean bias scales
// mu^.
//
// The table lives in shared memory as kTabRep interleaved replicas (entry j
// of replica c at j * kTabRep + c) and lane l reads replica l mod kTabRep: the
// eight lanes served together by a 128-bit shared load then always fall in
// different bank groups, whatever their (data-dependent) entries.
constexpr int kTab = 128;
constexpr int kTabRep = 8;
struct __align__(16) TabEntry {
    float ch, cl, sh, sl;  // cos and sin of 2 pi j / 128 as float pairs
};

// fills kTab * kTabRep entries; visible after the caller's next barrier
__device__ __forceinline__ void fill_exp_table(TabEntry* tab)
{
    for (int j = threadIdx.x; j < kTab; j += blockDim.x) {
        double sd, cd;
        sincospi(2.0 * j / kTab, &sd, &cd);
        TabEntry e;
        e.ch = (float)cd;
        e.cl = (float)(cd - (double)e.ch);
        e.sh = (float)sd;
        e.sl = (float)(sd - (double)e.sh);
#pragma unroll
        for (int c = 0; c < kTabRep; ++c) tab[j * kTabRep + c] = e;
    }
}

// this thread's replica of the table
__device__ __forceinline__ const TabEntry* exp_table_lane(const TabEntry* tab)
{
    return tab + (threadIdx.x & (kTabRep - 1));
}

// kMagic = 1.5 * 2^23: tau * kTab + kMagic rounds to an integer in the low
// bits. A caller may pass kMagic + s (s an integer, 0 <= s < kTab) instead:
// the table index then moves by s while u stays the same, i.e. the result is
// exp(-2 pi i (tau + s / kTab)) exactly (a phase shift by whole table steps).
constexpr float kMagic = 12582912.0f;

__device__ __forceinline__ void expm_turns(const TabEntry* __restrict__ tl, float tau, float tlo,
                                           float& er, float& ei, float magic = kMagic)
{
    const float km = fmaf(tau, (float)kTab, magic);
    const int idx = __float_as_int(km) & (kTab - 1);
    const float k = km - magic;                   // exact
    const float u = fmaf(-1.0f / kTab, k, tau);   // exact, |u| <= 1/256
    const float xh = u * 6.28318548202514648f;
    float xl = fmaf(u, 6.28318548202514648f, -xh);
    xl = fmaf(u, -1.74845553e-7f, xl);            // 2 pi - float(2 pi)
    xl = fmaf(tlo, 6.28318548202514648f, xl);
    const float x2 = xh * xh;
    // cos x - 1 and sin x - xh
    const float dc = fmaf(x2, fmaf(x2, 1.0f / 24.0f, -0.5f), -xh * xl);
    const float ds = fmaf(xh * x2, -1.0f / 6.0f, xl);
    const TabEntry t = tl[idx * kTabRep];
    // cos(theta) = Tc (1 + dc) - Ts sin x, sin(theta) = Ts (1 + dc) + Tc sin x,
    // with the table's low parts applied to the leading 1 only: their products
    // with x (below 1e-9, zero mean over the phases) are left out
    const float c = t.ch + fmaf(t.ch, dc, fmaf(-t.sh, xh, fmaf(-t.sh, ds, t.cl)));
    const float s = t.sh + fmaf(t.sh, dc, fmaf(t.ch, xh, fmaf(t.ch, ds, t.sl)));
    er = c;   // exp(-i theta) = cos theta - i sin theta
    ei = -s;
}

// The residual part of the fast table exponential: table entry idx (of the
// lane's replica) times exp(-2 pi i v), as (er, ei), for a residual v in turns,
// |v| <= 1/256 + a few 2^-24. cos(2 pi v) - 1 and sin(2 pi v) are polynomials
// in v with the powers of 2 pi folded into their coefficients, sin(2 pi v) as
// one float instead of a float pair: one instruction fewer than a residual in
// radians. The leading coefficients (2 pi)^2 / 2 and 2 pi are float pairs whose high
// products enter each final FMA exactly. Rounded alone they would scale
// every residual sine by 1 + 2.8e-8 and every cos - 1 by 1 - 2.9e-8; a kernel
// whose residual v is not dithered (see node_dither_steps) sees those as a
// coherent frequency-scale error and a coherent real scale error of ~3e-12 at
// low frequency, which move D against mu^ - nu^ there (measured: twice the
// random spread of D on a low-frequency shell window for the cosine alone).
// |v| <= 1/256 + |tlo|: the rounding of v is below 2.5e-10 turns, that of
// sin(2 pi v) below 1.5e-9, and the dropped v^5 (sine) and v^6 (cosine)
// terms below 7.5e-11, all far below the 6e-8 rounding of the result.
__device__ __forceinline__ void expm_residual(const TabEntry* __restrict__ tl, int idx, float v, float& er,
                                              float& ei)
{
    const float v2 = v * v;
    // cos 2 pi v - 1 = -(2 pi)^2 v^2 / 2 + (2 pi)^4 v^4 / 24 and
    // sin 2 pi v = 2 pi v - (2 pi)^3 v^3 / 6, the leading constants split
    const float dc = fmaf(v2, -19.7392082214355469f, v2 * fmaf(v2, 64.9393940226682914f, -5.80743176215037e-07f));
    const float sx = fmaf(v, 6.28318548202514648f, v * fmaf(v2, -41.3417022403997534f, -1.74845553146951715e-07f));
    const TabEntry t = tl[idx * kTabRep];
    const float c = t.ch + fmaf(t.ch, dc, fmaf(-t.sh, sx, t.cl));
    const float s = t.sh + fmaf(t.sh, dc, fmaf(t.ch, sx, t.sl));
    er = c;
    ei = -s;
}

// expm_residual for |v| <= 1/128 + a few 2^-24 (two table steps): the sine to
// v^5 and the cosine to v^6 (the first dropped terms below 1.5e-13; the float
// cubic coefficient adds up to 6e-13), for a kernel whose residual is the sum
// of two table-step residuals.
__device__ __forceinline__ void expm_residual_wide(const TabEntry* __restrict__ tl, int idx, float v, float& er,
                                                   float& ei)
{
    const float v2 = v * v;
    // cos 2 pi v - 1 = -(2 pi)^2 v^2 / 2 + (2 pi)^4 v^4 / 24 - (2 pi)^6 v^6 / 720 and
    // sin 2 pi v = 2 pi v - (2 pi)^3 v^3 / 6 + (2 pi)^5 v^5 / 120, the leading constants split
    const float dc = fmaf(v2, -19.7392082214355469f,
                          v2 * fmaf(v2, fmaf(v2, -85.4568172066937f, 64.9393940226682914f), -5.80743176215037e-07f));
    const float sx = fmaf(v, 6.28318548202514648f,
                          v * fmaf(v2, fmaf(v2, 81.6052492760750f, -41.3417022403997534f), -1.74845553146951715e-07f));
    const TabEntry t = tl[idx * kTabRep];
    const float c = t.ch + fmaf(t.ch, dc, fmaf(-t.sh, sx, t.cl));
    const float s = t.sh + fmaf(t.sh, dc, fmaf(t.ch, sx, t.sl));
    er = c;
    ei = -s;
}

// expm_turns with the residual u + tlo in turns (expm_residual)
__device__ __forceinline__ void expm_turns_fast(const TabEntry* __restrict__ tl, float tau, float tlo, float& er,
                                                float& ei, float magic = kMagic)
{
    const float km = fmaf(tau, (float)kTab, magic);
    const int idx = __float_as_int(km) & (kTab - 1);
    const float k = km - magic;                   // exact
    const float u = fmaf(-1.0f / kTab, k, tau);   // exact, |u| <= 1/256
    expm_residual(tl, idx, u + tlo, er, ei);
}

// kMagic in turns, 1.5 * 2^16: adding it to a phase in turns (|phase| < 2^15)
// rounds the phase to whole table steps, 2^-7 turns, whose count mod kTab is
// then the low 7 bits of the sum. kMagicTurns - j / kTab (j an integer,
// |j| <= kTab / 2) is exact and moves the index by -j the same way.
constexpr float kMagicTurns = kMagic / kTab;

// Per-(node, triangle tile) phase shift in whole table steps, s in [0, kTab):
// a second dither that varies across the tiles of one node. At low frequency
// the phases of all triangles of a node are close, so with the node's dither
// alone their float32 roundings stay correlated; shifting each tile by its own
// s (undone on the tile's sum in float64) makes the tiles' roundings
// independent.
__device__ __forceinline__ int tile_shift(int64_t node, int64_t tile)
{
    uint32_t h = (uint32_t)node * 0x9E3779B9u ^ ((uint32_t)tile * 0x85EBCA6Bu + 0x165667B1u);
    h ^= h >> 15;
    h *= 0x2C1B3C6Du;
    h ^= h >> 12;
    h *= 0x297A2D39u;
    h ^= h >> 15;
    return (int)(h & (kTab - 1));
}

// Rotate a tile's float32 sum (sr, si), evaluated with tile shift s, back by
// exp(+2 pi i s / kTab) in float64 (table entry s, replica 0, as a float pair)
// and add it to (ar, ai).
__device__ __forceinline__ void unshift_add(const TabEntry* __restrict__ tab, int s, double sr, double si,
                                            double& ar, double& ai)
{
    const TabEntry e = tab[s * kTabRep];
    const double c = (double)e.ch + (double)e.cl, sn = (double)e.sh + (double)e.sl;
    ar += sr * c - si * sn;
    ai += sr * sn + si * c;
}

// rounding error of s = fl(a + b): a + b = s + err exactly (Knuth's two-sum)
__device__ __forceinline__ float two_sum_err(float a, float b, float s)
{
    const float bb = s - a;
    return (a - (s - bb)) + (b - bb);
}

// Kahan-compensated float32 accumulation: the per-tile sum of nearly equal
// terms at low frequency would otherwise round the same way at neighbouring
// nodes, a coherent error that the mesh-minus-sphere difference magnifies.
struct Kahan {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x)
    {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

