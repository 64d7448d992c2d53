// The paper's atomic approximation of a mesh's surface measure (Sec. 3.1,
// Eqs. (change_variable) and (change_variable_approx)): every triangle
// (a, b, c) is replaced by 64 atoms a + u1 (b - a) + u2 (c - a) with weights
// q gamma, from the 8-point Gauss-Legendre rule applied twice to the standard
// simplex as the iterated integral of u2 over [0, 1 - u1] inside u1 over
// [0, 1]: u = (x_i, (1 - x_i) x_j), q = w_i w_j (1 - x_i), (x, w) the rule on
// [0, 1]. The transform is the atoms' plane-wave sum, in float64. It
// approximates the exact transform of wd_pair.cu with an error that falls like
// (|xi| h)^15 on triangles of size h, at 64 exponentials per (triangle, node)
// pair where the exact formula needs one or two.
#include <cmath>
#include <mutex>
#include <set>
#include <vector>

#include "wd_internal.h"

namespace {

constexpr int kAtoms = 64;
constexpr int ATOM_TPB = 256;
constexpr int ATOM_TILE = 128;

__constant__ double c_u1[kAtoms], c_u2[kAtoms], c_q[kAtoms];

std::mutex g_atoms_mu;
std::set<int> g_atoms_ready;  // devices whose constant memory holds the atoms

// One node per thread; triangle records (float64 staging) in shared-memory
// tiles; per (node, triangle) the vertex phase t_a = xi.a and the two edge
// phases, then the 64 atoms.
__global__ void __launch_bounds__(ATOM_TPB) atoms_kernel(const double* __restrict__ xi, int64_t n,
                                                         const TriRecD* __restrict__ rec, int64_t T,
                                                         double* __restrict__ out_re, double* __restrict__ out_im)
{
    __shared__ TriRecD tile[ATOM_TILE];
    const int64_t n_nb = (n + ATOM_TPB - 1) / ATOM_TPB;
    for (int64_t nb = blockIdx.x; nb < n_nb; nb += gridDim.x) {
        const int64_t node = nb * ATOM_TPB + threadIdx.x;
        const bool active = node < n;
        const double x = active ? xi[node] : 0.0;
        const double y = active ? xi[n + node] : 0.0;
        const double z = active ? xi[2 * n + node] : 0.0;
        double ar = 0.0, ai = 0.0;
        for (int64_t tb = 0; tb < T; tb += ATOM_TILE) {
            const int cnt = (int)((T - tb) < ATOM_TILE ? (T - tb) : ATOM_TILE);
            __syncthreads();
            for (int i = threadIdx.x; i < cnt; i += ATOM_TPB) tile[i] = rec[tb + i];
            __syncthreads();
            if (!active) continue;
            for (int j = 0; j < cnt; ++j) {
                const TriRecD& t = tile[j];
                // vertex a from the record: a = m - (e1 + e2) / 3
                const double ax = t.m[0] - (t.e1[0] + t.e2[0]) * (1.0 / 3.0);
                const double ay = t.m[1] - (t.e1[1] + t.e2[1]) * (1.0 / 3.0);
                const double az = t.m[2] - (t.e1[2] + t.e2[2]) * (1.0 / 3.0);
                const double ta = fma(x, ax, fma(y, ay, z * az));
                const double g1 = fma(x, t.e1[0], fma(y, t.e1[1], z * t.e1[2]));
                const double g2 = fma(x, t.e2[0], fma(y, t.e2[1], z * t.e2[2]));
                double sr = 0.0, si = 0.0;
#pragma unroll 4
                for (int m = 0; m < kAtoms; ++m) {
                    double s, c;
                    sincos(fma(c_u1[m], g1, fma(c_u2[m], g2, ta)), &s, &c);
                    sr = fma(c_q[m], c, sr);
                    si = fma(-c_q[m], s, si);
                }
                ar = fma(t.gam, sr, ar);
                ai = fma(t.gam, si, ai);
            }
        }
        if (active) {
            out_re[node] = ar;
            out_im[node] = ai;
        }
    }
}

// The 64 atoms of the standard simplex, built once per device in long double.
wd_status atoms_setup(wd_ctx* ctx)
{
    std::lock_guard<std::mutex> lk(g_atoms_mu);
    if (g_atoms_ready.count(ctx->device)) return WD_OK;
    std::vector<double> x, w;
    wd_legendre_rule(8, x, w);
    double u1[kAtoms], u2[kAtoms], q[kAtoms];
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) {
            const long double xi = 0.5L * (1.0L + (long double)x[i]), wi = 0.5L * (long double)w[i];
            const long double xj = 0.5L * (1.0L + (long double)x[j]), wj = 0.5L * (long double)w[j];
            u1[8 * i + j] = (double)xi;
            u2[8 * i + j] = (double)((1.0L - xi) * xj);
            q[8 * i + j] = (double)(wi * wj * (1.0L - xi));
        }
    WD_CUDA(cudaMemcpyToSymbol(c_u1, u1, sizeof(u1)));
    WD_CUDA(cudaMemcpyToSymbol(c_u2, u2, sizeof(u2)));
    WD_CUDA(cudaMemcpyToSymbol(c_q, q, sizeof(q)));
    g_atoms_ready.insert(ctx->device);
    return WD_OK;
}

}  // namespace

wd_status wd_launch_atoms(wd_ctx* ctx, const double* d_xi, int64_t n, const void* d_rec, int64_t T, double* d_re,
                          double* d_im, cudaStream_t st)
{
    if (n == 0) return WD_OK;
    wd_status s = atoms_setup(ctx);
    if (s != WD_OK) return s;
    int64_t g = (n + ATOM_TPB - 1) / ATOM_TPB;
    const int64_t cap = (int64_t)ctx->num_sms * 8;
    if (g > cap) g = cap;
    atoms_kernel<<<(int)g, ATOM_TPB, 0, st>>>(d_xi, n, static_cast<const TriRecD*>(d_rec), T, d_re, d_im);
    ctx->launches++;
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}
