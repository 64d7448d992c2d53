// Frequency rules (Sec. 3.2) and the per-rule device caches: the s-dependent
// weights and the reference sphere's transform (Eq. (ft_nsphere_sinc)).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "wd_internal.h"

namespace {

constexpr long double kPi = 3.141592653589793238462643383279502884L;

// Gauss-Legendre nodes and weights on [-1, 1], ascending. Newton's method on
// P_n with P_n and P_n' from the joint three-term recurrences
//   (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1},   P'_{k+1} = P'_{k-1} + (2k+1) P_k,
// started from Tricomi's asymptotic node estimate. Host long double.
void legendre_rule(int n, std::vector<double>& x, std::vector<double>& w)
{
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < (n + 1) / 2; ++i) {
        // i-th largest root
        long double th = kPi * (4.0L * (i + 1) - 1.0L) / (4.0L * n + 2.0L);
        long double z = (1.0L - (n - 1.0L) / (8.0L * n * n * n)) * cosl(th);
        long double dp = 1.0L;
        for (int it = 0; it < 60; ++it) {
            long double pm1 = 1.0L, p = z, dpm1 = 0.0L;
            dp = 1.0L;
            for (int k = 1; k < n; ++k) {
                long double pn = ((2.0L * k + 1.0L) * z * p - k * pm1) / (k + 1.0L);
                long double dpn = dpm1 + (2.0L * k + 1.0L) * p;
                pm1 = p;
                p = pn;
                dpm1 = dp;
                dp = dpn;
            }
            long double step = p / dp;
            z -= step;
            if (fabsl(step) <= 1e-19L * (1.0L + fabsl(z))) {
                // one more derivative evaluation at the final z
                long double qm1 = 1.0L, q = z, dqm1 = 0.0L, dq = 1.0L;
                for (int k = 1; k < n; ++k) {
                    long double qn = ((2.0L * k + 1.0L) * z * q - k * qm1) / (k + 1.0L);
                    long double dqn = dqm1 + (2.0L * k + 1.0L) * q;
                    qm1 = q;
                    q = qn;
                    dqm1 = dq;
                    dq = dqn;
                }
                dp = dq;
                break;
            }
        }
        long double wt = 2.0L / ((1.0L - z * z) * dp * dp);
        // symmetric pair (the middle node of odd n is 0)
        int hi = n - 1 - i, lo = i;
        x[hi] = (double)z;
        x[lo] = (double)(-z);
        w[hi] = w[lo] = (double)wt;
        if (hi == lo) x[hi] = 0.0;
    }
}

__global__ void weights_kernel(const double* __restrict__ xi, const double* __restrict__ wg,
                               int64_t n, double s, double wscale, double* __restrict__ w)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        double x = xi[k], y = xi[n + k], z = xi[2 * n + k];
        double r2 = fma(x, x, fma(y, y, z * z));
        w[k] = wg[k] * exp(-s * log1p(wscale * r2));
    }
}

// nu^(xi) = 4 pi rho sin(rho r)/r exp(-i xi.c), r = |xi|; 4 pi rho^2 at r = 0.
__global__ void sphere_kernel(const double* __restrict__ xi, int64_t n, double rho, double cx,
                              double cy, double cz, double* __restrict__ re, double* __restrict__ im,
                              double* __restrict__ inter)
{
    const double four_pi = 12.566370614359172953850573533118;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        double x = xi[k], y = xi[n + k], z = xi[2 * n + k];
        double r = sqrt(fma(x, x, fma(y, y, z * z)));
        double a = (r == 0.0) ? four_pi * rho * rho : four_pi * rho * sin(rho * r) / r;
        double ph = fma(x, cx, fma(y, cy, z * cz));
        double sp, cp;
        sincos(ph, &sp, &cp);
        double vr = a * cp, vi = -a * sp;
        if (re) re[k] = vr;
        if (im) im[k] = vi;
        if (inter) { inter[2 * k] = vr; inter[2 * k + 1] = vi; }
    }
}

int grid_for(wd_ctx* ctx, int64_t n)
{
    int64_t g = (n + 255) / 256;
    int64_t cap = (int64_t)ctx->num_sms * 8;
    return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

wd_status upload_rule(wd_ctx* ctx, wd_rule* r)
{
    const int64_t n = r->n_eval;
    if (n > 0) {
        WD_CUDA(wd_dev_alloc(&r->d_xi, sizeof(double) * 3 * n, "rule nodes"));
        WD_CUDA(wd_dev_alloc(&r->d_wg, sizeof(double) * n, "rule weights"));
        WD_CUDA(cudaMemcpy(r->d_xi, r->h_xi.data(), sizeof(double) * 3 * n, cudaMemcpyHostToDevice));
        WD_CUDA(cudaMemcpy(r->d_wg, r->h_wg.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
    }
    if (!r->h_rad.empty()) {
        WD_CUDA(wd_dev_alloc(&r->d_rad, sizeof(double) * r->h_rad.size(), "rule radii"));
        WD_CUDA(wd_dev_alloc(&r->d_dir, sizeof(float) * r->h_dir.size(), "rule directions"));
        WD_CUDA(cudaMemcpy(r->d_rad, r->h_rad.data(), sizeof(double) * r->h_rad.size(), cudaMemcpyHostToDevice));
        WD_CUDA(cudaMemcpy(r->d_dir, r->h_dir.data(), sizeof(float) * r->h_dir.size(), cudaMemcpyHostToDevice));
    }
    r->ctx = ctx;
    return WD_OK;
}

void release_rule(wd_rule* r)
{
    if (!r) return;
    cudaFree(r->d_xi);
    cudaFree(r->d_wg);
    cudaFree(r->d_rad);
    cudaFree(r->d_dir);
    cudaFree(r->d_lines);
    cudaFree(r->d_lblk);
    for (auto& kv : r->w_cache) cudaFree(kv.second);
    for (auto& kv : r->precise_cache) {
        cudaFree(kv.second.d_list);
        cudaFree(kv.second.d_flag);
    }
    for (auto& kv : r->nu_cache) cudaFree(kv.second);
    delete r;
}

// A cache entry is filled on the stream of the call that first needs it. Wait
// for it there (unless the stream is being captured into a graph) so that later
// calls on other streams see a complete array.
wd_status settle_cache_fill(cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    WD_CUDA(cudaStreamIsCapturing(st, &cs));
    if (cs == cudaStreamCaptureStatusNone) WD_CUDA(cudaStreamSynchronize(st));
    return WD_OK;
}

bool same_desc(const wd_rule_desc& a, const wd_rule_desc& b)
{
    return a.kind == b.kind && a.R == b.R && a.n_r == b.n_r && a.n_polar == b.n_polar &&
           a.n_azim == b.n_azim && (a.hermitian != 0) == (b.hermitian != 0);
}

}  // namespace

wd_status wd_launch_weights(wd_ctx* ctx, const double* d_xi, const double* d_wg, int64_t n,
                            double s, double wscale, double* d_w, cudaStream_t st)
{
    if (n == 0) return WD_OK;
    weights_kernel<<<grid_for(ctx, n), 256, 0, st>>>(d_xi, d_wg, n, s, wscale, d_w);
    ctx->launches++;
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}

wd_status wd_launch_sphere(wd_ctx* ctx, const double* d_xi, int64_t n, double radius,
                           const double* center, double* d_re, double* d_im, double* d_inter,
                           cudaStream_t st)
{
    if (n == 0) return WD_OK;
    sphere_kernel<<<grid_for(ctx, n), 256, 0, st>>>(d_xi, n, radius, center[0], center[1],
                                                     center[2], d_re, d_im, d_inter);
    ctx->launches++;
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}

wd_status wd_rule_weights(wd_ctx* ctx, wd_rule* rule, double s, const double** d_w, cudaStream_t st)
{
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    auto it = rule->w_cache.find(s);
    if (it != rule->w_cache.end()) {
        *d_w = it->second;
        return WD_OK;
    }
    double* w = nullptr;
    cudaError_t e = wd_dev_alloc(&w, sizeof(double) * (rule->n_eval > 0 ? rule->n_eval : 1), "weights cache");
    if (e != cudaSuccess) {
        cudaGetLastError();
        wd_set_error("out of device memory for rule weights");
        return WD_ENOMEM;
    }
    wd_status stt = wd_launch_weights(ctx, rule->d_xi, rule->d_wg, rule->n_eval, s, rule->wscale, w, st);
    if (stt != WD_OK) {
        cudaFree(w);
        return stt;
    }
    rule->w_cache[s] = w;
    *d_w = w;
    return settle_cache_fill(st);
}

wd_status wd_rule_sphere(wd_ctx* ctx, wd_rule* rule, double radius, const double* center,
                         const double** d_nu, cudaStream_t st)
{
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    std::array<double, 4> key{radius, center[0], center[1], center[2]};
    auto it = rule->nu_cache.find(key);
    if (it != rule->nu_cache.end()) {
        *d_nu = it->second;
        return WD_OK;
    }
    double* nu = nullptr;
    cudaError_t e = wd_dev_alloc(&nu, sizeof(double) * 2 * (rule->n_eval > 0 ? rule->n_eval : 1), "sphere cache");
    if (e != cudaSuccess) {
        cudaGetLastError();
        wd_set_error("out of device memory for the cached sphere transform");
        return WD_ENOMEM;
    }
    wd_status stt = wd_launch_sphere(ctx, rule->d_xi, rule->n_eval, radius, center, nullptr,
                                     nullptr, nu, st);
    if (stt != WD_OK) {
        cudaFree(nu);
        return stt;
    }
    rule->nu_cache[key] = nu;
    *d_nu = nu;
    return settle_cache_fill(st);
}

wd_status wd_rule_precise(wd_ctx* ctx, wd_rule* rule, double s, const PreciseSet** out)
{
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    auto it = rule->precise_cache.find(s);
    if (it != rule->precise_cache.end()) {
        *out = &it->second;
        return WD_OK;
    }
    // the weights in float64 on the host, from the rule's host copy; the
    // choice only has to be deterministic, not bitwise the device's weights
    const int64_t n = rule->n_eval;
    const int64_t n_nb = (n + WD_NPB - 1) / WD_NPB;
    std::vector<double> W(n);
    double wmax = 0.0;
    for (int64_t k = 0; k < n; ++k) {
        const double x = rule->h_xi[k], y = rule->h_xi[n + k], z = rule->h_xi[2 * n + k];
        W[k] = std::fabs(rule->h_wg[k]) * std::exp(-s * std::log1p(rule->wscale * (x * x + y * y + z * z)));
        wmax = std::max(wmax, W[k]);
    }
    std::vector<unsigned char> flag(n_nb > 0 ? n_nb : 1, 0);
    std::vector<int> list;
    for (int64_t b = 0; b < n_nb; ++b) {
        bool hit = false;
        for (int64_t k = b * WD_NPB; k < std::min(n, (b + 1) * WD_NPB) && !hit; ++k)
            hit = W[k] >= kPreciseWeightFrac * wmax;
        if (hit) {
            flag[b] = 1;
            list.push_back((int)b);
        }
    }
    PreciseSet ps;
    ps.n = (int)list.size();
    if (ps.n > 0) {
        if (wd_dev_alloc(&ps.d_flag, flag.size(), "precise-block flags") != cudaSuccess ||
            wd_dev_alloc(&ps.d_list, sizeof(int) * list.size(), "precise-block list") != cudaSuccess) {
            cudaGetLastError();
            cudaFree(ps.d_flag);
            cudaFree(ps.d_list);
            wd_set_error("out of device memory for the extended-precision block list");
            return WD_ENOMEM;
        }
        WD_CUDA(cudaMemcpy(ps.d_flag, flag.data(), flag.size(), cudaMemcpyHostToDevice));
        WD_CUDA(cudaMemcpy(ps.d_list, list.data(), sizeof(int) * list.size(), cudaMemcpyHostToDevice));
    }
    wd_log(4, "rule %p, s=%g: %d of %lld node blocks in extended precision", (void*)rule, s, ps.n, (long long)n_nb);
    auto ins = rule->precise_cache.emplace(s, ps).first;
    *out = &ins->second;
    return WD_OK;
}

// ------------------------------------------------------------------ C ABI
// The paper's cube trapezoid rule (Sec. 3.2), nodes at xi = 2 pi eta: see
// WD_RULE_CUBE_TRAP in wd.h. Built in long double like the ball rule.
static wd_status build_cube_rule(wd_ctx* ctx, const wd_rule_desc* d, wd_rule** out)
{
    WD_CHECK(std::isfinite(d->R) && d->R > 0.0, WD_EINVAL, "xi_max must be finite and > 0");
    WD_CHECK(d->n_r >= 2 && d->n_r % 2 == 0, WD_EINVAL, "cube rule: M (n_r) must be even and >= 2");
    const int64_t side = (int64_t)d->n_r + 1;
    const int64_t n_total = side * side * side;
    WD_CHECK(n_total <= (int64_t)1 << 31, WD_EINVAL, "rule too large (more than 2^31 nodes)");
    wd_rule_desc key = *d;
    key.n_polar = key.n_azim = 0;
    key.hermitian = d->hermitian ? 1 : 0;
    wd_status st = wd_activate(ctx);
    if (st != WD_OK) return st;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    for (wd_rule* r : ctx->rules)
        if (same_desc(r->desc, key)) {
            *out = r;
            return WD_OK;
        }
    const int m = d->n_r / 2;
    const bool herm = key.hermitian != 0;
    wd_rule* r = new wd_rule();
    r->desc = key;
    r->cached = true;
    r->n_total = n_total;
    r->n_eval = herm ? (n_total + 1) / 2 : n_total;
    r->wscale = 1.0 / (4.0 * (double)(kPi * kPi));
    const int64_t n = r->n_eval;
    r->h_xi.resize(3 * n);
    r->h_wg.resize(n);
    const long double h = 2.0L * (long double)d->R / (long double)d->n_r;
    const long double tpih = 2.0L * kPi * h;
    int64_t k = 0;
    for (int iz = herm ? 0 : -m; iz <= m; ++iz)
        for (int iy = -m; iy <= m; ++iy)
            for (int ix = -m; ix <= m; ++ix) {
                if (herm && iz == 0 && (iy < 0 || (iy == 0 && ix < 0))) continue;
                const long double fx = (ix == m || ix == -m) ? 0.5L : 1.0L;
                const long double fy = (iy == m || iy == -m) ? 0.5L : 1.0L;
                const long double fz = (iz == m || iz == -m) ? 0.5L : 1.0L;
                const bool origin = ix == 0 && iy == 0 && iz == 0;
                r->h_xi[k] = (double)(tpih * ix);
                r->h_xi[n + k] = (double)(tpih * iy);
                r->h_xi[2 * n + k] = (double)(tpih * iz);
                r->h_wg[k] = (double)(h * h * h * fx * fy * fz * ((herm && !origin) ? 2.0L : 1.0L));
                ++k;
            }
    // the lattice lines (fixed j, k) in node order, and each node block's first
    // line; with full lines of 2m + 1 >= WD_NPB / 2 + 1 nodes a block of WD_NPB
    // consecutive nodes touches at most three lines (the one half line of a
    // Hermitian rule comes first), which the lattice kernel relies on; for
    // smaller M the per-node kernel serves the rule
    const bool lattice = 2 * m + 1 >= WD_NPB / 2 + 1;
    std::vector<LatLine> lines;
    for (int iz = herm ? 0 : -m; iz <= m && lattice; ++iz)
        for (int iy = -m; iy <= m; ++iy) {
            if (herm && iz == 0 && iy < 0) continue;
            LatLine ln;
            const long double ey = h * iy, ez = h * iz;
            ln.yh = (float)ey;
            ln.yl = (float)(ey - (long double)ln.yh);
            ln.zh = (float)ez;
            ln.zl = (float)(ez - (long double)ln.zh);
            ln.i0 = (herm && iz == 0 && iy == 0) ? 0 : -m;
            ln.count = m - ln.i0 + 1;
            ln.node0 = lines.empty() ? 0 : lines.back().node0 + lines.back().count;
            lines.push_back(ln);
        }
    const int64_t n_nb = lattice ? (n + WD_NPB - 1) / WD_NPB : 0;
    std::vector<int2> lblk(n_nb > 0 ? n_nb : 1);
    for (int64_t b = 0, L = 0; b < n_nb; ++b) {
        const int64_t node = b * WD_NPB;
        while (node >= lines[L].node0 + lines[L].count) ++L;
        lblk[b] = make_int2((int)L, (int)(node - lines[L].node0));
    }
    r->n_lines = (int64_t)lines.size();
    r->lat_hh = (float)h;
    r->lat_hl = (float)(h - (long double)r->lat_hh);
    st = upload_rule(ctx, r);
    if (st == WD_OK && lattice) {
        if (wd_dev_alloc(&r->d_lines, sizeof(LatLine) * lines.size(), "lattice lines") != cudaSuccess ||
            wd_dev_alloc(&r->d_lblk, sizeof(int2) * lblk.size(), "lattice block lines") != cudaSuccess) {
            cudaGetLastError();
            wd_set_error("out of device memory for the lattice lines");
            st = WD_ENOMEM;
        } else if (cudaMemcpy(r->d_lines, lines.data(), sizeof(LatLine) * lines.size(), cudaMemcpyHostToDevice) !=
                       cudaSuccess ||
                   cudaMemcpy(r->d_lblk, lblk.data(), sizeof(int2) * lblk.size(), cudaMemcpyHostToDevice) !=
                       cudaSuccess) {
            st = wd_cuda_status(cudaGetLastError(), "lattice line upload");
        }
    }
    if (st != WD_OK) {
        release_rule(r);
        return st;
    }
    ctx->rules.push_back(r);
    wd_log(3, "cube rule xi_max=%g M=%d hermitian=%d: %lld nodes on %lld lines", d->R, d->n_r, key.hermitian,
           (long long)n, (long long)r->n_lines);
    *out = r;
    return WD_OK;
}

// The ball rule (Sec. 3.2, rules over balls centred at the origin) on its
// radial shells [s0, s1): Gauss-Legendre radii on [0, R] with the r^2
// Jacobian, Gauss-Legendre u = cos(theta), trapezoid phi. [0, n_r) is the
// full rule.
static wd_status build_ball_rule(wd_ctx* ctx, const wd_rule_desc* d, int s0, int s1, wd_rule** out)
{
    WD_CHECK(d->kind == WD_RULE_BALL, WD_EINVAL, "rule kind must be WD_RULE_BALL or WD_RULE_CUBE_TRAP");
    WD_CHECK(std::isfinite(d->R) && d->R > 0.0, WD_EINVAL, "R must be finite and > 0");
    WD_CHECK(d->n_r >= 1 && d->n_polar >= 1 && d->n_azim >= 1, WD_EINVAL, "node counts must be >= 1");
    WD_CHECK(!d->hermitian || d->n_polar % 2 == 0, WD_EINVAL,
             "hermitian halving needs an even polar node count");
    WD_CHECK(s0 >= 0 && s0 < s1 && s1 <= d->n_r, WD_EINVAL,
             "radial shell window must satisfy 0 <= shell_begin < shell_end <= n_r");
    int64_t n_total = (int64_t)(s1 - s0) * d->n_polar * d->n_azim;
    WD_CHECK((int64_t)d->n_r * d->n_polar * d->n_azim <= (int64_t)1 << 31, WD_EINVAL,
             "rule too large (more than 2^31 nodes)");
    wd_status st = wd_activate(ctx);
    if (st != WD_OK) return st;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    for (wd_rule* r : ctx->rules)
        if (same_desc(r->desc, *d) && r->shell0 == s0 && r->shell1 == s1) {
            *out = r;
            return WD_OK;
        }
    std::vector<double> xr, wr, xu, wu;
    legendre_rule(d->n_r, xr, wr);
    legendre_rule(d->n_polar, xu, wu);
    const int n_u = d->hermitian ? d->n_polar / 2 : d->n_polar;
    const int u0 = d->hermitian ? d->n_polar / 2 : 0;  // ascending: upper half starts here
    wd_rule* r = new wd_rule();
    r->desc = *d;
    r->desc.hermitian = d->hermitian ? 1 : 0;
    r->cached = true;
    r->n_total = n_total;
    r->n_eval = (int64_t)(s1 - s0) * n_u * d->n_azim;
    r->shell0 = s0;
    r->shell1 = s1;
    const int64_t n = r->n_eval;
    r->h_xi.resize(3 * n);
    r->h_wg.resize(n);
    std::vector<long double> cph(d->n_azim), sph(d->n_azim);
    for (int m = 0; m < d->n_azim; ++m) {
        long double ph = 2.0L * kPi * m / d->n_azim;
        cph[m] = cosl(ph);
        sph[m] = sinl(ph);
    }
    const long double w_phi = 2.0L * kPi / d->n_azim;
    const long double half_R = 0.5L * (long double)d->R;
    // the same nodes factored as radius x unit direction, for the radial kernel
    r->n_rad = s1 - s0;
    r->n_dir = (int64_t)n_u * d->n_azim;
    r->h_rad.resize(r->n_rad);
    r->h_dir.resize(9 * r->n_dir);
    for (int i = s0; i < s1; ++i) r->h_rad[i - s0] = (double)(half_R * (1.0L + xr[i]));
    for (int j = 0, kd = 0; j < n_u; ++j) {
        const long double u = xu[u0 + j], sn = sqrtl(1.0L - u * u);
        for (int m = 0; m < d->n_azim; ++m, ++kd) {
            const long double w[3] = {sn * cph[m], sn * sph[m], u};
            for (int c = 0; c < 3; ++c) {
                const long double t = w[c] / (2.0L * kPi);
                const float hi = (float)t;
                r->h_dir[c * r->n_dir + kd] = (float)w[c];
                r->h_dir[(3 + c) * r->n_dir + kd] = hi;
                r->h_dir[(6 + c) * r->n_dir + kd] = (float)(t - (long double)hi);
            }
        }
    }
    int64_t k = 0;
    for (int i = s0; i < s1; ++i) {
        long double rr = half_R * (1.0L + xr[i]);
        long double w_r = half_R * wr[i] * rr * rr;  // Jacobian r^2 of spherical coordinates
        for (int j = 0; j < n_u; ++j) {
            long double u = xu[u0 + j];
            long double w_u = wu[u0 + j] * (d->hermitian ? 2.0L : 1.0L);
            long double sn = sqrtl(1.0L - u * u);
            for (int m = 0; m < d->n_azim; ++m, ++k) {
                r->h_xi[k] = (double)(rr * sn * cph[m]);
                r->h_xi[n + k] = (double)(rr * sn * sph[m]);
                r->h_xi[2 * n + k] = (double)(rr * u);
                r->h_wg[k] = (double)(w_r * w_u * w_phi);
            }
        }
    }
    st = upload_rule(ctx, r);
    if (st != WD_OK) {
        release_rule(r);
        return st;
    }
    ctx->rules.push_back(r);
    *out = r;
    return WD_OK;
}

extern "C" wd_status wd_build_freq_rule(wd_ctx* ctx, const wd_rule_desc* d, wd_rule** out)
{
    WdRange nvtx_range("wd_build_freq_rule");
    WD_CHECK(ctx && d && out, WD_EINVAL, "null argument");
    if (d->kind == WD_RULE_CUBE_TRAP) return build_cube_rule(ctx, d, out);
    return build_ball_rule(ctx, d, 0, d->n_r, out);
}

extern "C" wd_status wd_build_freq_rule_shells(wd_ctx* ctx, const wd_rule_desc* d, int shell_begin, int shell_end,
                                               wd_rule** out)
{
    WdRange nvtx_range("wd_build_freq_rule_shells");
    WD_CHECK(ctx && d && out, WD_EINVAL, "null argument");
    WD_CHECK(d->kind == WD_RULE_BALL, WD_EINVAL, "radial shell windows exist for ball rules only");
    return build_ball_rule(ctx, d, shell_begin, shell_end, out);
}

extern "C" wd_status wd_rule_from_nodes(wd_ctx* ctx, const double* xi, const double* w_geom,
                                        int64_t n, wd_rule** out)
{
    WD_CHECK(ctx && out && (n == 0 || (xi && w_geom)), WD_EINVAL, "null argument");
    WD_CHECK(n >= 0 && n <= ((int64_t)1 << 31), WD_EINVAL, "node count out of range");
    for (int64_t k = 0; k < 3 * n; ++k)
        WD_CHECK(std::isfinite(xi[k]), WD_EINVAL, "non-finite frequency node");
    for (int64_t k = 0; k < n; ++k)
        WD_CHECK(std::isfinite(w_geom[k]), WD_EINVAL, "non-finite node weight");
    wd_status st = wd_activate(ctx);
    if (st != WD_OK) return st;
    wd_rule* r = new wd_rule();
    r->desc.kind = WD_RULE_EXPLICIT;
    r->n_eval = r->n_total = n;
    r->h_xi.assign(xi, xi + 3 * n);
    r->h_wg.assign(w_geom, w_geom + n);
    st = upload_rule(ctx, r);
    if (st != WD_OK) {
        release_rule(r);
        return st;
    }
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    ctx->explicit_rules.push_back(r);
    *out = r;
    return WD_OK;
}

extern "C" wd_status wd_rule_info(const wd_rule* r, int64_t* n_eval, int64_t* n_total)
{
    WD_CHECK(r, WD_EINVAL, "null rule");
    if (n_eval) *n_eval = r->n_eval;
    if (n_total) *n_total = r->n_total;
    return WD_OK;
}

extern "C" wd_status wd_rule_copy_nodes(const wd_rule* r, double* xi, double* w_geom)
{
    WD_CHECK(r, WD_EINVAL, "null rule");
    if (xi && !r->h_xi.empty()) std::memcpy(xi, r->h_xi.data(), sizeof(double) * r->h_xi.size());
    if (w_geom && !r->h_wg.empty()) std::memcpy(w_geom, r->h_wg.data(), sizeof(double) * r->h_wg.size());
    return WD_OK;
}

extern "C" void wd_rule_free(wd_rule* r)
{
    if (!r || !r->ctx) return;
    wd_ctx* ctx = r->ctx;
    if (wd_activate(ctx) != WD_OK) return;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    cudaDeviceSynchronize();  // the rule's arrays may be in use by queued work
    for (auto* lst : {&ctx->rules, &ctx->explicit_rules})
        for (size_t i = 0; i < lst->size(); ++i)
            if ((*lst)[i] == r) {
                lst->erase(lst->begin() + i);
                release_rule(r);
                return;
            }
}

void wd_release_all_rules(wd_ctx* ctx)
{
    for (wd_rule* r : ctx->rules) release_rule(r);
    for (wd_rule* r : ctx->explicit_rules) release_rule(r);
    ctx->rules.clear();
    ctx->explicit_rules.clear();
}

void wd_legendre_rule(int n, std::vector<double>& x, std::vector<double>& w) { legendre_rule(n, x, w); }
