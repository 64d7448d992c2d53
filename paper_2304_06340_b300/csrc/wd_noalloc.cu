// Distance entry point that performs no device allocation.
//
// Some callers cannot allocate device memory at the moment they need a
// distance: an application whose memory manager owns the whole device and
// forbids stray cudaMalloc calls, a latency-critical loop that must never hit
// the allocator (cudaMalloc and cudaFree can synchronise the device), or a
// plugin that only receives buffers from its host. wd_distance_dev_noalloc
// serves them: the caller passes every input and the output as device arrays,
// and all intermediate storage (staged triangles, weights, the sphere's
// transform, per-block partial sums and completion counters) lives in one
// fixed-size array in the library's static device memory. Every device that
// loads the library reserves that array until the process exits.
#include <cmath>
#include <mutex>

#include "wd_internal.h"

namespace {

constexpr size_t kScratchBytes = WD_NOALLOC_SCRATCH_BYTES;

// The shared scratch. In host code this name is only a stand-in for the
// device symbol; kernels receive its device address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr size_t align_up(size_t v) { return (v + 255) & ~size_t(255); }

struct DeviceSetup {
    bool ready = false;
    unsigned char* scratch = nullptr;  // device address of g_noalloc_scratch
    wd_ctx ctx;                        // launch bookkeeping only: no workspace is ever attached
};

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
DeviceSetup g_setup[kMaxDevices];

// One-time set-up per device, with that device current: resolve the device
// address of the scratch array and record the SM count used by the planner.
wd_status setup_device(int dev, DeviceSetup** out)
{
    WD_CHECK(dev >= 0 && dev < kMaxDevices, WD_EINVAL, "device ordinal out of range");
    DeviceSetup& s = g_setup[dev];
    if (!s.ready) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return wd_cuda_status(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        int sms = 0;
        WD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        s.ctx.device = dev;
        s.ctx.num_sms = sms;
        s.scratch = static_cast<unsigned char*>(p);
        s.ready = true;
    }
    *out = &s;
    return WD_OK;
}

}  // namespace

extern "C" wd_status wd_distance_dev_noalloc(const double* d_xi, const double* d_w_geom, int64_t n_nodes,
                                             const double* d_verts, int64_t n_verts, const int32_t* d_tris,
                                             int64_t n_tris, double s, double radius, const double center[3],
                                             int precision, double* d_dist2, void* stream)
{
    WdRange nvtx_range("wd_distance_dev_noalloc");
    WD_CHECK(precision == WD_FP64 || precision == WD_MIXED, WD_EINVAL, "precision must be WD_FP64 or WD_MIXED");
    WD_CHECK(std::isfinite(s) && s > 0.0, WD_EINVAL, "s must be finite and > 0");
    WD_CHECK(std::isfinite(radius) && radius > 0.0, WD_EINVAL, "sphere radius must be finite and > 0");
    WD_CHECK(center, WD_EINVAL, "null sphere center");
    for (int j = 0; j < 3; ++j) WD_CHECK(std::isfinite(center[j]), WD_EINVAL, "non-finite sphere center");
    WD_CHECK(n_nodes >= 0 && n_verts >= 0 && n_tris >= 0, WD_EINVAL, "negative size");
    WD_CHECK(n_nodes <= ((int64_t)1 << 31) && n_tris <= ((int64_t)1 << 31), WD_EINVAL, "size out of range");
    WD_CHECK(d_dist2 && (n_nodes == 0 || (d_xi && d_w_geom)) && (n_tris == 0 || (d_verts && d_tris)),
             WD_EINVAL, "null device pointer");

    int dev = 0;
    WD_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_setup_mu);
    DeviceSetup* S = nullptr;
    wd_status st = setup_device(dev, &S);
    if (st != WD_OK) return st;
    wd_ctx* ctx = &S->ctx;

    // scratch layout: weights, sphere transform, triangle records, chunk
    // partials, block sums, then the counters and flags that must start at zero
    PairPlan plan;
    wd_plan_pair(ctx, precision, MODE_DIST, n_nodes, n_tris, &plan);
    size_t off = 0;
    const size_t o_w = off;
    off += align_up(sizeof(double) * (size_t)n_nodes);
    const size_t o_nu = off;
    off += align_up(2 * sizeof(double) * (size_t)n_nodes);
    const size_t o_rec = off;
    off += align_up(wd_tri_record_bytes(precision) * (size_t)n_tris);
    const size_t o_part = off;
    if (plan.nchunks > 1) off += align_up((size_t)plan.nchunks * (size_t)n_nodes * 2 * sizeof(double));
    const size_t o_blk = off;
    off += align_up(sizeof(double) * (size_t)(plan.n_nb > 0 ? plan.n_nb : 1));
    const size_t o_zero = off;
    const size_t o_cnt = off;
    off += align_up(sizeof(int) * (size_t)(plan.n_nb > 0 ? plan.n_nb : 1));
    const size_t o_flags = off;
    off += align_up(4 * sizeof(int));
    if (off > kScratchBytes) {
        wd_set_error("wd_distance_dev_noalloc: problem needs " + std::to_string(off) +
                     " bytes of scratch, more than the fixed " + std::to_string(kScratchBytes) +
                     " (use wd_distance_dev for larger problems)");
        return WD_EINVAL;
    }

    unsigned char* base = S->scratch;
    cudaStream_t strm = (cudaStream_t)stream;
    // the array keeps the previous call's contents: clear counters and flags
    WD_CUDA(cudaMemsetAsync(base + o_zero, 0, off - o_zero, strm));
    ctx->d_flags = reinterpret_cast<int*>(base + o_flags);

    double* W = reinterpret_cast<double*>(base + o_w);
    double* nu = reinterpret_cast<double*>(base + o_nu);
    if ((st = wd_launch_weights(ctx, d_xi, d_w_geom, n_nodes, s, 1.0, W, strm)) != WD_OK) return st;
    if ((st = wd_launch_sphere(ctx, d_xi, n_nodes, radius, center, nullptr, nullptr, nu, strm)) != WD_OK)
        return st;
    void* rec = base + o_rec;
    if ((st = wd_launch_stage(ctx, precision, d_verts, n_verts, d_tris, n_tris, 1.0, rec, 0, strm)) != WD_OK)
        return st;
    if (plan.n_items == 0) {
        WD_CUDA(cudaMemsetAsync(d_dist2, 0, sizeof(double), strm));
        return WD_OK;
    }
    PairArgs a;
    a.xi = d_xi;
    a.n = n_nodes;
    a.tris = rec;
    a.T = n_tris;
    a.W = W;
    a.nu = nu;
    a.partial = reinterpret_cast<double*>(base + o_part);
    a.cnt = reinterpret_cast<int*>(base + o_cnt);
    a.blockD = reinterpret_cast<double*>(base + o_blk);
    a.done = ctx->d_flags + 1;
    a.out = d_dist2;
    return wd_launch_pair(ctx, precision, MODE_DIST, plan, a, strm);
}
