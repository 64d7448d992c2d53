// C ABI entry points: context, scratch, transforms and the distance.
#include <cmath>
#include <cstring>
#include <string>

#include "wd_internal.h"

void wd_release_all_rules(wd_ctx* ctx);

namespace {

thread_local std::string g_last_error;

constexpr size_t align_up(size_t v) { return (v + 255) & ~size_t(255); }

bool host_mesh_ok(const wd_mesh* m, std::string* why)
{
    if (!m) { *why = "null mesh"; return false; }
    if (m->n_verts < 0 || m->n_tris < 0) { *why = "negative mesh size"; return false; }
    if ((m->n_verts > 0 && !m->verts) || (m->n_tris > 0 && !m->tris)) { *why = "null mesh array"; return false; }
    if (m->n_tris > ((int64_t)1 << 31)) { *why = "too many triangles"; return false; }
    for (int64_t i = 0; i < 3 * m->n_verts; ++i)
        if (!std::isfinite(m->verts[i])) { *why = "non-finite vertex coordinate"; return false; }
    for (int64_t i = 0; i < 3 * m->n_tris; ++i)
        if (m->tris[i] < 0 || m->tris[i] >= m->n_verts) { *why = "triangle index out of range"; return false; }
    return true;
}

wd_status check_common(wd_ctx* ctx, const wd_rule* rule, int precision)
{
    WD_CHECK(ctx && rule, WD_EINVAL, "null context or rule");
    WD_CHECK(rule->ctx == ctx, WD_EINVAL, "rule belongs to another context");
    WD_CHECK(precision == WD_FP64 || precision == WD_MIXED, WD_EINVAL, "precision must be WD_FP64 or WD_MIXED");
    return WD_OK;
}

wd_status check_nu(const wd_measure* nu)
{
    WD_CHECK(nu, WD_EINVAL, "null reference measure");
    if (nu->kind == WD_NU_SPHERE) {
        WD_CHECK(std::isfinite(nu->radius) && nu->radius > 0.0, WD_EINVAL, "sphere radius must be finite and > 0");
        for (int j = 0; j < 3; ++j)
            WD_CHECK(std::isfinite(nu->center[j]), WD_EINVAL, "non-finite sphere center");
        return WD_OK;
    }
    WD_CHECK(nu->kind == WD_NU_MESH, WD_EINVAL, "unknown reference-measure kind");
    WD_CHECK(nu->mesh, WD_EINVAL, "WD_NU_MESH needs a mesh");
    WD_CHECK(nu->mesh->n_verts >= 0 && nu->mesh->n_tris >= 0, WD_EINVAL, "negative mesh size");
    WD_CHECK(nu->mesh->n_tris == 0 || (nu->mesh->verts && nu->mesh->tris), WD_EINVAL,
             "reference mesh: null mesh array");
    return WD_OK;
}

// Layout of one pair evaluation inside the context scratch, from offset `base`.
// With a weight (s > 0) a mixed per-node plan also gets the rule's
// extended-precision node blocks for s and room for their chunk partials.
struct CoreLayout {
    PairPlan plan;
    const PreciseSet* precise = nullptr;
    size_t rec = 0, partial = 0, ppartial = 0, blockD = 0, end = 0;
};

wd_status core_layout(wd_ctx* ctx, wd_rule* rule, int precision, int mode, int64_t n_rec, size_t base, double s,
                      CoreLayout* out)
{
    CoreLayout L;
    const int64_t n_nodes = rule->n_eval;
    wd_plan_pair_rule(ctx, rule, precision, mode, n_rec, &L.plan);
    if (precision == WD_MIXED && !L.plan.radial && mode != MODE_FT && s > 0.0 && L.plan.n_items > 0) {
        wd_status st = wd_rule_precise(ctx, rule, s, &L.precise);
        if (st != WD_OK) return st;
        if (L.precise->n == 0) L.precise = nullptr;
    }
    size_t off = align_up(base);
    L.rec = off;
    off += align_up((size_t)n_rec * wd_tri_record_bytes(precision));
    L.partial = off;
    if (L.plan.nchunks > 1) off += align_up((size_t)L.plan.nchunks * n_nodes * 2 * sizeof(double));
    L.ppartial = off;
    if (L.precise)
        off += align_up(wd_precise_partial_bytes(wd_precise_plan(ctx, L.plan, L.precise->n, mode), L.precise->n));
    L.blockD = off;
    off += align_up((size_t)(L.plan.n_nb > 0 ? L.plan.n_nb : 1) * sizeof(double));
    L.end = off;
    *out = L;
    return WD_OK;
}

// the extended-precision blocks of a layout into the pair arguments
void set_precise_args(wd_ctx* ctx, const CoreLayout& L, PairArgs& a)
{
    if (!L.precise) return;
    a.precise_flag = L.precise->d_flag;
    a.precise_list = L.precise->d_list;
    a.n_precise = L.precise->n;
    a.precise_partial = reinterpret_cast<double*>(ctx->ws + L.ppartial);
}

// Stage mu (and a mesh nu, negated) and run the pair kernel in `mode`.
// Device pointers only; scratch must already hold `L.end` bytes.
wd_status run_core(wd_ctx* ctx, wd_rule* rule, const CoreLayout& L, int precision, int mode,
                   const double* d_verts, int64_t nv, const int32_t* d_tris, int64_t nt,
                   const wd_measure* nu, double s, double* d_out, double* d_out_im, cudaStream_t st)
{
    void* rec = ctx->ws + L.rec;
    wd_status r = wd_launch_stage(ctx, precision, d_verts, nv, d_tris, nt, 1.0, rec, 0, st);
    if (r != WD_OK) return r;
    PairArgs a;
    wd_pair_args_rule(rule, a);
    a.tris = rec;
    a.T = L.plan.n_tris;
    if (mode == MODE_DIST) {
        if (nu->kind == WD_NU_MESH) {
            r = wd_launch_stage(ctx, precision, nu->mesh->verts, nu->mesh->n_verts, nu->mesh->tris,
                                nu->mesh->n_tris, -1.0, rec, nt, st);
            if (r != WD_OK) return r;
        } else {
            r = wd_rule_sphere(ctx, rule, nu->radius, nu->center, &a.nu, st);
            if (r != WD_OK) return r;
        }
        r = wd_rule_weights(ctx, rule, s, &a.W, st);
        if (r != WD_OK) return r;
    }
    a.partial = reinterpret_cast<double*>(ctx->ws + L.partial);
    set_precise_args(ctx, L, a);
    a.cnt = ctx->d_counters;
    a.blockD = reinterpret_cast<double*>(ctx->ws + L.blockD);
    a.done = ctx->d_flags + 1;
    a.out = d_out;
    a.out_im = d_out_im;
    if (L.plan.n_items == 0) {
        // no nodes: D = 0, nothing to transform
        if (mode == MODE_DIST) WD_CUDA(cudaMemsetAsync(d_out, 0, sizeof(double), st));
        return WD_OK;
    }
    return wd_launch_pair(ctx, precision, mode, L.plan, a, st);
}

wd_status finish_host(wd_ctx* ctx, cudaStream_t st)
{
    WD_CUDA(cudaStreamSynchronize(st));
    int flag = 0;
    WD_CUDA(cudaMemcpy(&flag, ctx->d_flags, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        WD_CUDA(cudaMemset(ctx->d_flags, 0, sizeof(int)));
        wd_set_error("invalid mesh input (index out of range or non-finite vertex)");
        return WD_EINVAL;
    }
    return WD_OK;
}

wd_status upload_mesh(wd_ctx* ctx, const wd_mesh* m, size_t ov, size_t ot, cudaStream_t st)
{
    if (m->n_verts > 0)
        WD_CUDA(cudaMemcpyAsync(ctx->ws + ov, m->verts, sizeof(double) * 3 * m->n_verts,
                                cudaMemcpyHostToDevice, st));
    if (m->n_tris > 0)
        WD_CUDA(cudaMemcpyAsync(ctx->ws + ot, m->tris, sizeof(int32_t) * 3 * m->n_tris,
                                cudaMemcpyHostToDevice, st));
    return WD_OK;
}

}  // namespace

// ------------------------------------------------------------------ internals
void wd_set_error(const std::string& msg)
{
    g_last_error = msg;
    wd_log(1, "%s", msg.c_str());
}

wd_status wd_cuda_status(cudaError_t e, const char* what)
{
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    wd_log(1, "%s", g_last_error.c_str());
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return WD_ENOMEM;
    }
    return WD_ECUDA;
}

wd_status wd_activate(wd_ctx* ctx)
{
    WD_CUDA(cudaSetDevice(ctx->device));
    return WD_OK;
}

wd_status wd_ws_reserve(wd_ctx* ctx, size_t bytes)
{
    if (bytes <= ctx->ws_bytes) return WD_OK;
    size_t want = bytes + bytes / 4;
    WD_CUDA(cudaDeviceSynchronize());
    cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
    if (wd_dev_alloc(&ctx->ws, want, "context scratch") != cudaSuccess) {
        cudaGetLastError();
        ctx->ws = nullptr;
        wd_set_error("out of device memory for scratch (" + std::to_string(want) + " bytes)");
        return WD_ENOMEM;
    }
    ctx->ws_bytes = want;
    return WD_OK;
}

wd_status wd_counters_reserve(wd_ctx* ctx, int64_t n)
{
    if (n <= ctx->n_counters) return WD_OK;
    int64_t want = n + n / 4 + 64;
    WD_CUDA(cudaDeviceSynchronize());
    cudaFree(ctx->d_counters);
    ctx->d_counters = nullptr;
    ctx->n_counters = 0;
    if (wd_dev_alloc(&ctx->d_counters, sizeof(int) * want, "completion counters") != cudaSuccess) {
        cudaGetLastError();
        wd_set_error("out of device memory for completion counters");
        return WD_ENOMEM;
    }
    WD_CUDA(cudaMemset(ctx->d_counters, 0, sizeof(int) * want));
    ctx->n_counters = want;
    return WD_OK;
}

// ------------------------------------------------------------------ C ABI
extern "C" const char* wd_last_error(const wd_ctx*) { return g_last_error.c_str(); }

extern "C" wd_status wd_create(int device, wd_ctx** out)
{
    WD_CHECK(out, WD_EINVAL, "null output pointer");
    *out = nullptr;
    int count = 0;
    WD_CUDA(cudaGetDeviceCount(&count));
    WD_CHECK(device >= 0 && device < count, WD_EINVAL, "no such CUDA device");
    WD_CUDA(cudaSetDevice(device));
    wd_ctx* c = new wd_ctx();
    c->device = device;
    cudaError_t e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = wd_dev_alloc(&c->d_flags, 4 * sizeof(int), "context flags");
    if (e == cudaSuccess) e = cudaMemset(c->d_flags, 0, 4 * sizeof(int));
    if (e == cudaSuccess) e = wd_dev_alloc(&c->d_scalar, 4 * sizeof(double), "context scalars");
    if (e != cudaSuccess) {
        wd_status st = wd_cuda_status(e, "wd_create");
        cudaFree(c->d_flags);
        cudaFree(c->d_scalar);
        delete c;
        return st;
    }
    wd_log(3, "context created on device %d (%d SMs)", device, c->num_sms);
    *out = c;
    return WD_OK;
}

extern "C" void wd_destroy(wd_ctx* ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    wd_release_all_rules(ctx);
    cudaFree(ctx->ws);
    cudaFree(ctx->d_counters);
    cudaFree(ctx->d_flags);
    cudaFree(ctx->d_scalar);
    delete ctx;
}

extern "C" int64_t wd_launch_count(const wd_ctx* ctx) { return ctx ? ctx->launches.load() : 0; }

extern "C" wd_status wd_sync(wd_ctx* ctx, void* stream)
{
    WD_CHECK(ctx, WD_EINVAL, "null context");
    wd_status st = wd_activate(ctx);
    if (st != WD_OK) return st;
    return finish_host(ctx, (cudaStream_t)stream);
}

// ---- transforms
extern "C" wd_status wd_mesh_ft_dev(wd_ctx* ctx, const wd_rule* rule_c, const double* d_verts,
                                    int64_t nv, const int32_t* d_tris, int64_t nt, int precision,
                                    double* d_re, double* d_im, void* stream)
{
    WdRange nvtx_range("wd_mesh_ft_dev");
    wd_status st = check_common(ctx, rule_c, precision);
    if (st != WD_OK) return st;
    WD_CHECK(nv >= 0 && nt >= 0 && nt <= ((int64_t)1 << 31), WD_EINVAL, "mesh size out of range");
    WD_CHECK((nt == 0 || (d_verts && d_tris)) && (rule_c->n_eval == 0 || (d_re && d_im)),
             WD_EINVAL, "null device pointer");
    if ((st = wd_activate(ctx)) != WD_OK) return st;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    wd_rule* rule = const_cast<wd_rule*>(rule_c);
    cudaStream_t s = (cudaStream_t)stream;
    CoreLayout L;
    if ((st = core_layout(ctx, rule, precision, MODE_FT, nt, 0, 0.0, &L)) != WD_OK) return st;
    if ((st = wd_ws_reserve(ctx, L.end)) != WD_OK) return st;
    if ((st = wd_counters_reserve(ctx, L.plan.n_nb)) != WD_OK) return st;
    return run_core(ctx, rule, L, precision, MODE_FT, d_verts, nv, d_tris, nt, nullptr, 0.0, d_re, d_im, s);
}

extern "C" wd_status wd_mesh_ft_atoms(wd_ctx* ctx, const wd_rule* rule_c, const wd_mesh* mesh, double* out_re,
                                      double* out_im)
{
    WdRange nvtx_range("wd_mesh_ft_atoms");
    wd_status st = check_common(ctx, rule_c, WD_FP64);
    if (st != WD_OK) return st;
    std::string why;
    WD_CHECK(host_mesh_ok(mesh, &why), WD_EINVAL, why);
    const int64_t n = rule_c->n_eval;
    WD_CHECK(n == 0 || (out_re && out_im), WD_EINVAL, "null output array");
    if ((st = wd_activate(ctx)) != WD_OK) return st;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    const int64_t nt = mesh->n_tris;
    size_t ov = 0, ot = align_up(sizeof(double) * 3 * mesh->n_verts);
    size_t orc = ot + align_up(sizeof(int32_t) * 3 * nt);
    size_t oo = orc + align_up(sizeof(TriRecD) * (size_t)(nt > 0 ? nt : 1));
    size_t end = oo + 2 * align_up(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if ((st = wd_ws_reserve(ctx, end)) != WD_OK) return st;
    cudaStream_t s = 0;
    if ((st = upload_mesh(ctx, mesh, ov, ot, s)) != WD_OK) return st;
    void* rec = ctx->ws + orc;
    if ((st = wd_launch_stage(ctx, WD_FP64, reinterpret_cast<const double*>(ctx->ws + ov), mesh->n_verts,
                              reinterpret_cast<const int32_t*>(ctx->ws + ot), nt, 1.0, rec, 0, s)) != WD_OK)
        return st;
    double* d_re = reinterpret_cast<double*>(ctx->ws + oo);
    double* d_im = reinterpret_cast<double*>(ctx->ws + oo + align_up(sizeof(double) * (size_t)(n > 0 ? n : 1)));
    if ((st = wd_launch_atoms(ctx, rule_c->d_xi, n, rec, nt, d_re, d_im, s)) != WD_OK) return st;
    if (n > 0) {
        WD_CUDA(cudaMemcpyAsync(out_re, d_re, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
        WD_CUDA(cudaMemcpyAsync(out_im, d_im, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    }
    return finish_host(ctx, s);
}

extern "C" wd_status wd_mesh_ft(wd_ctx* ctx, const wd_rule* rule_c, const wd_mesh* mesh, int precision,
                                double* out_re, double* out_im)
{
    WdRange nvtx_range("wd_mesh_ft");
    wd_status st = check_common(ctx, rule_c, precision);
    if (st != WD_OK) return st;
    std::string why;
    WD_CHECK(host_mesh_ok(mesh, &why), WD_EINVAL, why);
    const int64_t n = rule_c->n_eval;
    WD_CHECK(n == 0 || (out_re && out_im), WD_EINVAL, "null output array");
    if ((st = wd_activate(ctx)) != WD_OK) return st;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    wd_rule* rule = const_cast<wd_rule*>(rule_c);
    size_t ov = 0, ot = align_up(sizeof(double) * 3 * mesh->n_verts);
    size_t oo = ot + align_up(sizeof(int32_t) * 3 * mesh->n_tris);
    size_t base = oo + 2 * align_up(sizeof(double) * n);
    CoreLayout L;
    if ((st = core_layout(ctx, rule, precision, MODE_FT, mesh->n_tris, base, 0.0, &L)) != WD_OK) return st;
    if ((st = wd_ws_reserve(ctx, L.end)) != WD_OK) return st;
    if ((st = wd_counters_reserve(ctx, L.plan.n_nb)) != WD_OK) return st;
    cudaStream_t s = 0;
    if ((st = upload_mesh(ctx, mesh, ov, ot, s)) != WD_OK) return st;
    double* d_re = reinterpret_cast<double*>(ctx->ws + oo);
    double* d_im = reinterpret_cast<double*>(ctx->ws + oo + align_up(sizeof(double) * n));
    st = run_core(ctx, rule, L, precision, MODE_FT, reinterpret_cast<const double*>(ctx->ws + ov),
                  mesh->n_verts, reinterpret_cast<const int32_t*>(ctx->ws + ot), mesh->n_tris, nullptr,
                  0.0, d_re, d_im, s);
    if (st != WD_OK) return st;
    if (n > 0) {
        WD_CUDA(cudaMemcpyAsync(out_re, d_re, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
        WD_CUDA(cudaMemcpyAsync(out_im, d_im, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    }
    return finish_host(ctx, s);
}

extern "C" wd_status wd_sphere_ft_dev(wd_ctx* ctx, const wd_rule* rule, double radius, const double center[3],
                                      double* d_re, double* d_im, void* stream)
{
    WdRange nvtx_range("wd_sphere_ft_dev");
    wd_status st = check_common(ctx, rule, WD_FP64);
    if (st != WD_OK) return st;
    WD_CHECK(center, WD_EINVAL, "null center");
    WD_CHECK(std::isfinite(radius) && radius > 0.0, WD_EINVAL, "radius must be finite and > 0");
    for (int j = 0; j < 3; ++j) WD_CHECK(std::isfinite(center[j]), WD_EINVAL, "non-finite center");
    WD_CHECK(rule->n_eval == 0 || (d_re && d_im), WD_EINVAL, "null device pointer");
    if ((st = wd_activate(ctx)) != WD_OK) return st;
    return wd_launch_sphere(ctx, rule->d_xi, rule->n_eval, radius, center, d_re, d_im, nullptr,
                            (cudaStream_t)stream);
}

extern "C" wd_status wd_sphere_ft(wd_ctx* ctx, const wd_rule* rule, double radius, const double center[3],
                                  double* out_re, double* out_im)
{
    WdRange nvtx_range("wd_sphere_ft");
    wd_status st = check_common(ctx, rule, WD_FP64);
    if (st != WD_OK) return st;
    const int64_t n = rule->n_eval;
    WD_CHECK(n == 0 || (out_re && out_im), WD_EINVAL, "null output array");
    if ((st = wd_activate(ctx)) != WD_OK) return st;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    if ((st = wd_ws_reserve(ctx, 2 * align_up(sizeof(double) * (n > 0 ? n : 1)))) != WD_OK) return st;
    double* d_re = reinterpret_cast<double*>(ctx->ws);
    double* d_im = reinterpret_cast<double*>(ctx->ws + align_up(sizeof(double) * (n > 0 ? n : 1)));
    st = wd_sphere_ft_dev(ctx, rule, radius, center, d_re, d_im, nullptr);
    if (st != WD_OK) return st;
    if (n > 0) {
        WD_CUDA(cudaMemcpy(out_re, d_re, sizeof(double) * n, cudaMemcpyDeviceToHost));
        WD_CUDA(cudaMemcpy(out_im, d_im, sizeof(double) * n, cudaMemcpyDeviceToHost));
    }
    return finish_host(ctx, 0);
}

// ---- distance
extern "C" wd_status wd_distance_dev(wd_ctx* ctx, const wd_rule* rule_c, const double* d_verts,
                                     int64_t nv, const int32_t* d_tris, int64_t nt, const wd_measure* nu,
                                     double s, int precision, double* d_dist2, void* stream)
{
    WdRange nvtx_range("wd_distance_dev");
    wd_status st = check_common(ctx, rule_c, precision);
    if (st != WD_OK) return st;
    if ((st = check_nu(nu)) != WD_OK) return st;
    WD_CHECK(std::isfinite(s) && s > 0.0, WD_EINVAL, "s must be finite and > 0");
    WD_CHECK(nv >= 0 && nt >= 0, WD_EINVAL, "negative mesh size");
    WD_CHECK((nt == 0 || (d_verts && d_tris)) && d_dist2, WD_EINVAL, "null device pointer");
    const int64_t nt2 = nu->kind == WD_NU_MESH ? nu->mesh->n_tris : 0;
    WD_CHECK(nt + nt2 <= ((int64_t)1 << 31), WD_EINVAL, "too many triangles");
    if ((st = wd_activate(ctx)) != WD_OK) return st;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    wd_rule* rule = const_cast<wd_rule*>(rule_c);
    CoreLayout L;
    if ((st = core_layout(ctx, rule, precision, MODE_DIST, nt + nt2, 0, s, &L)) != WD_OK) return st;
    if ((st = wd_ws_reserve(ctx, L.end)) != WD_OK) return st;
    if ((st = wd_counters_reserve(ctx, L.plan.n_nb)) != WD_OK) return st;
    return run_core(ctx, rule, L, precision, MODE_DIST, d_verts, nv, d_tris, nt, nu, s, d_dist2, nullptr,
                    (cudaStream_t)stream);
}

extern "C" wd_status wd_distance(wd_ctx* ctx, const wd_rule* rule_c, const wd_mesh* mu, const wd_measure* nu,
                                 double s, int precision, double* dist2)
{
    WdRange nvtx_range("wd_distance");
    wd_status st = check_common(ctx, rule_c, precision);
    if (st != WD_OK) return st;
    if ((st = check_nu(nu)) != WD_OK) return st;
    WD_CHECK(std::isfinite(s) && s > 0.0, WD_EINVAL, "s must be finite and > 0");
    WD_CHECK(dist2, WD_EINVAL, "null output");
    std::string why;
    WD_CHECK(host_mesh_ok(mu, &why), WD_EINVAL, why);
    if (nu->kind == WD_NU_MESH) WD_CHECK(host_mesh_ok(nu->mesh, &why), WD_EINVAL, "reference mesh: " + why);
    if ((st = wd_activate(ctx)) != WD_OK) return st;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    wd_rule* rule = const_cast<wd_rule*>(rule_c);
    const wd_mesh* m2 = nu->kind == WD_NU_MESH ? nu->mesh : nullptr;
    const int64_t nt2 = m2 ? m2->n_tris : 0;
    size_t ov = 0, ot = align_up(sizeof(double) * 3 * mu->n_verts);
    size_t ov2 = ot + align_up(sizeof(int32_t) * 3 * mu->n_tris);
    size_t ot2 = ov2 + (m2 ? align_up(sizeof(double) * 3 * m2->n_verts) : 0);
    size_t base = ot2 + (m2 ? align_up(sizeof(int32_t) * 3 * m2->n_tris) : 0);
    CoreLayout L;
    if ((st = core_layout(ctx, rule, precision, MODE_DIST, mu->n_tris + nt2, base, s, &L)) != WD_OK) return st;
    if ((st = wd_ws_reserve(ctx, L.end)) != WD_OK) return st;
    if ((st = wd_counters_reserve(ctx, L.plan.n_nb)) != WD_OK) return st;
    cudaStream_t strm = 0;
    if ((st = upload_mesh(ctx, mu, ov, ot, strm)) != WD_OK) return st;
    wd_mesh dm2{};
    wd_measure dnu = *nu;
    if (m2) {
        if ((st = upload_mesh(ctx, m2, ov2, ot2, strm)) != WD_OK) return st;
        dm2.verts = reinterpret_cast<const double*>(ctx->ws + ov2);
        dm2.n_verts = m2->n_verts;
        dm2.tris = reinterpret_cast<const int32_t*>(ctx->ws + ot2);
        dm2.n_tris = m2->n_tris;
        dnu.mesh = &dm2;
    }
    st = run_core(ctx, rule, L, precision, MODE_DIST, reinterpret_cast<const double*>(ctx->ws + ov),
                  mu->n_verts, reinterpret_cast<const int32_t*>(ctx->ws + ot), mu->n_tris, &dnu, s,
                  ctx->d_scalar, nullptr, strm);
    if (st != WD_OK) return st;
    WD_CUDA(cudaMemcpyAsync(dist2, ctx->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, strm));
    return finish_host(ctx, strm);
}

// Scratch layout of the gradient from offset `base`: the forward pass's
// records, chunk partials and block sums, then the residual, the float64
// records of the adjoint, its per-(chunk, triangle) sums, the scatter scratch
// and the radial adjoint's tables.
struct GradLayout {
    CoreLayout core;
    AdjPlan ap;
    size_t res = 0, rec64 = 0, adj = 0, sc = 0, rad = 0, end = 0;
};

static wd_status grad_layout(wd_ctx* ctx, wd_rule* rule, int precision, int64_t nt, int64_t nt2, int64_t nv,
                             size_t base, double s, GradLayout* out)
{
    GradLayout G;
    const int64_t n = rule->n_eval;
    wd_status st = core_layout(ctx, rule, precision, MODE_RESID, nt + nt2, base, s, &G.core);
    if (st != WD_OK) return st;
    wd_plan_adjoint_rule(ctx, rule, precision, nt, &G.ap);
    size_t off = G.core.end;
    G.res = off;
    off += align_up(sizeof(double) * 2 * (size_t)(n > 0 ? n : 1));
    G.rec64 = off;
    off += align_up(sizeof(TriRecD) * (size_t)(nt > 0 ? nt : 1));
    G.adj = off;
    off += align_up(sizeof(double) * 10 * (size_t)(G.ap.nchunks > 0 ? G.ap.nchunks : 1) * (size_t)(nt > 0 ? nt : 1));
    G.sc = off;
    off += align_up(wd_adjoint_scatter_bytes(nt, nv));
    G.rad = off;
    if (G.ap.radial) off += align_up(wd_adjoint_radial_bytes(rule));
    G.end = off;
    *out = G;
    return WD_OK;
}

// Gradient core on device pointers: forward pass in `precision` writing D and
// the residual 2 W (mu^ - nu^), then the adjoint in the same precision over
// mu's triangles.
static wd_status grad_core(wd_ctx* ctx, wd_rule* rule, int precision, const double* d_verts, int64_t nv,
                           const int32_t* d_tris, int64_t nt, const wd_measure* nu, double s, double* d_dist2,
                           double* d_grad, size_t base, cudaStream_t st)
{
    const int64_t nt2 = nu->kind == WD_NU_MESH ? nu->mesh->n_tris : 0;
    const int64_t n = rule->n_eval;
    GradLayout G;
    wd_status st_ = grad_layout(ctx, rule, precision, nt, nt2, nv, base, s, &G);
    if (st_ != WD_OK) return st_;
    const CoreLayout& L = G.core;
    const AdjPlan& ap = G.ap;
    st_ = wd_ws_reserve(ctx, G.end);
    if (st_ != WD_OK) return st_;
    if ((st_ = wd_counters_reserve(ctx, L.plan.n_nb)) != WD_OK) return st_;
    double* resid = reinterpret_cast<double*>(ctx->ws + G.res);
    if (n > 0) WD_CUDA(cudaMemsetAsync(resid, 0, sizeof(double) * 2 * n, st));
    if (nv > 0) WD_CUDA(cudaMemsetAsync(d_grad, 0, sizeof(double) * 3 * nv, st));
    // forward (same staging as the distance), with the residual written per node
    void* rec = ctx->ws + L.rec;
    if ((st_ = wd_launch_stage(ctx, precision, d_verts, nv, d_tris, nt, 1.0, rec, 0, st)) != WD_OK) return st_;
    PairArgs a;
    wd_pair_args_rule(rule, a);
    a.tris = rec;
    a.T = L.plan.n_tris;
    if (nu->kind == WD_NU_MESH) {
        if ((st_ = wd_launch_stage(ctx, precision, nu->mesh->verts, nu->mesh->n_verts, nu->mesh->tris,
                                   nu->mesh->n_tris, -1.0, rec, nt, st)) != WD_OK)
            return st_;
    } else if ((st_ = wd_rule_sphere(ctx, rule, nu->radius, nu->center, &a.nu, st)) != WD_OK) {
        return st_;
    }
    if ((st_ = wd_rule_weights(ctx, rule, s, &a.W, st)) != WD_OK) return st_;
    a.partial = reinterpret_cast<double*>(ctx->ws + L.partial);
    set_precise_args(ctx, L, a);
    a.cnt = ctx->d_counters;
    a.blockD = reinterpret_cast<double*>(ctx->ws + L.blockD);
    a.done = ctx->d_flags + 1;
    a.out = d_dist2;
    a.resid = resid;
    if (L.plan.n_items == 0) {
        WD_CUDA(cudaMemsetAsync(d_dist2, 0, sizeof(double), st));
        return WD_OK;
    }
    if ((st_ = wd_launch_pair(ctx, precision, MODE_RESID, L.plan, a, st)) != WD_OK) return st_;
    // adjoint over mu's triangles, staged in float64
    void* rec64 = ctx->ws + G.rec64;
    if ((st_ = wd_launch_stage(ctx, WD_FP64, d_verts, nv, d_tris, nt, 1.0, rec64, 0, st)) != WD_OK) return st_;
    return wd_launch_adjoint(ctx, precision, ap, rule, resid, rec64, precision == WD_MIXED ? rec : nullptr, nt,
                             ap.radial ? ctx->ws + G.rad : nullptr, reinterpret_cast<double*>(ctx->ws + G.adj),
                             ctx->ws + G.sc, d_tris, nv, d_grad, st);
}

extern "C" wd_status wd_distance_grad_dev(wd_ctx* ctx, const wd_rule* rule_c, const double* d_verts,
                                          int64_t nv, const int32_t* d_tris, int64_t nt, const wd_measure* nu,
                                          double s, int precision, double* d_dist2, double* d_grad, void* stream)
{
    WdRange nvtx_range("wd_distance_grad_dev");
    wd_status st = check_common(ctx, rule_c, precision);
    if (st != WD_OK) return st;
    if ((st = check_nu(nu)) != WD_OK) return st;
    WD_CHECK(std::isfinite(s) && s > 0.0, WD_EINVAL, "s must be finite and > 0");
    WD_CHECK(nv >= 0 && nt >= 0, WD_EINVAL, "negative mesh size");
    WD_CHECK((nt == 0 || (d_verts && d_tris)) && d_dist2 && (nv == 0 || d_grad), WD_EINVAL,
             "null device pointer");
    const int64_t nt2 = nu->kind == WD_NU_MESH ? nu->mesh->n_tris : 0;
    WD_CHECK(nt + nt2 <= ((int64_t)1 << 31), WD_EINVAL, "too many triangles");
    if ((st = wd_activate(ctx)) != WD_OK) return st;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    return grad_core(ctx, const_cast<wd_rule*>(rule_c), precision, d_verts, nv, d_tris, nt, nu, s, d_dist2, d_grad,
                     0, (cudaStream_t)stream);
}

extern "C" wd_status wd_distance_grad(wd_ctx* ctx, const wd_rule* rule_c, const wd_mesh* mu, const wd_measure* nu,
                                      double s, int precision, double* dist2, double* grad_verts)
{
    WdRange nvtx_range("wd_distance_grad");
    wd_status st = check_common(ctx, rule_c, precision);
    if (st != WD_OK) return st;
    if ((st = check_nu(nu)) != WD_OK) return st;
    WD_CHECK(std::isfinite(s) && s > 0.0, WD_EINVAL, "s must be finite and > 0");
    WD_CHECK(dist2 && (mu == nullptr || mu->n_verts == 0 || grad_verts), WD_EINVAL, "null output");
    std::string why;
    WD_CHECK(host_mesh_ok(mu, &why), WD_EINVAL, why);
    if (nu->kind == WD_NU_MESH) WD_CHECK(host_mesh_ok(nu->mesh, &why), WD_EINVAL, "reference mesh: " + why);
    if ((st = wd_activate(ctx)) != WD_OK) return st;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    wd_rule* rule = const_cast<wd_rule*>(rule_c);
    const wd_mesh* m2 = nu->kind == WD_NU_MESH ? nu->mesh : nullptr;
    // upload area: mu, nu mesh, gradient; the core's scratch follows
    size_t ov = 0, ot = align_up(sizeof(double) * 3 * mu->n_verts);
    size_t ov2 = ot + align_up(sizeof(int32_t) * 3 * mu->n_tris);
    size_t ot2 = ov2 + (m2 ? align_up(sizeof(double) * 3 * m2->n_verts) : 0);
    size_t og = ot2 + (m2 ? align_up(sizeof(int32_t) * 3 * m2->n_tris) : 0);
    size_t base = og + align_up(sizeof(double) * 3 * (size_t)(mu->n_verts > 0 ? mu->n_verts : 1));
    // reserve the upload area first; grad_core grows the scratch beyond `base`
    // before it touches any of it, and the uploads are issued after that
    if ((st = wd_ws_reserve(ctx, base)) != WD_OK) return st;
    cudaStream_t strm = 0;
    // grad_core reserves the scratch for its own layout, and a reallocation
    // there would lose the uploads; reserve that same layout before uploading
    GradLayout G;
    if ((st = grad_layout(ctx, rule, precision, mu->n_tris, m2 ? m2->n_tris : 0, mu->n_verts, base, s, &G)) != WD_OK)
        return st;
    if ((st = wd_ws_reserve(ctx, G.end)) != WD_OK) return st;
    if ((st = upload_mesh(ctx, mu, ov, ot, strm)) != WD_OK) return st;
    wd_mesh dm2{};
    wd_measure dnu = *nu;
    if (m2) {
        if ((st = upload_mesh(ctx, m2, ov2, ot2, strm)) != WD_OK) return st;
        dm2.verts = reinterpret_cast<const double*>(ctx->ws + ov2);
        dm2.n_verts = m2->n_verts;
        dm2.tris = reinterpret_cast<const int32_t*>(ctx->ws + ot2);
        dm2.n_tris = m2->n_tris;
        dnu.mesh = &dm2;
    }
    double* d_grad = reinterpret_cast<double*>(ctx->ws + og);
    st = grad_core(ctx, rule, precision, reinterpret_cast<const double*>(ctx->ws + ov), mu->n_verts,
                   reinterpret_cast<const int32_t*>(ctx->ws + ot), mu->n_tris, &dnu, s, ctx->d_scalar, d_grad, base,
                   strm);
    if (st != WD_OK) return st;
    WD_CUDA(cudaMemcpyAsync(dist2, ctx->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, strm));
    if (mu->n_verts > 0)
        WD_CUDA(cudaMemcpyAsync(grad_verts, d_grad, sizeof(double) * 3 * mu->n_verts, cudaMemcpyDeviceToHost, strm));
    return finish_host(ctx, strm);
}
