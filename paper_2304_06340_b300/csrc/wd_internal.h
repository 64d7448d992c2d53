// Internal declarations shared by the libwd translation units.
#pragma once

#include <cuda_runtime.h>

#include <array>
#include <atomic>
#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "wd.h"

// ------------------------------------------------------------------ runtime support (wd_runtime.cu)
int wd_log_level();
void wd_log(int level, const char* fmt, ...);  // 1 error, 2 warn, 3 info, 4 debug (stderr, WD_LOG)
// device allocation: honours WD_FAULT_ALLOC and WD_POISON_SCRATCH
cudaError_t wd_dev_alloc(void** p, size_t bytes, const char* what);
template <typename T>
cudaError_t wd_dev_alloc(T** p, size_t bytes, const char* what)
{
    void* q = nullptr;
    cudaError_t e = wd_dev_alloc(&q, bytes, what);
    *p = static_cast<T*>(q);
    return e;
}
int wd_fault_drop_completion();  // WD_FAULT_DROP_COMPLETION (0: off)

// NVTX range for the duration of a scope (shows in Nsight timelines)
struct WdRange {
    explicit WdRange(const char* name);
    ~WdRange();
};

// ------------------------------------------------------------------ errors
void wd_set_error(const std::string& msg);
wd_status wd_cuda_status(cudaError_t e, const char* what);

#define WD_CUDA(call)                                              \
    do {                                                           \
        cudaError_t e__ = (call);                                  \
        if (e__ != cudaSuccess) return wd_cuda_status(e__, #call); \
    } while (0)

#define WD_CHECK(cond, code, msg)       \
    do {                                \
        if (!(cond)) {                  \
            wd_set_error(msg);          \
            return (code);              \
        }                               \
    } while (0)

// ------------------------------------------------------------------ records
// One triangle as the float64 pair kernel reads it (80 bytes).
struct __align__(16) TriRecD {
    double m[3];   // centroid
    double e1[3];  // b - a
    double e2[3];  // c - a
    double gam;    // |(b - a) x (c - a)| = twice the area (negative for a subtracted mesh)
};

// One triangle as the mixed pair kernel reads it (64 bytes).
struct __align__(16) TriRecF {
    float mh[3];   // centroid, high float32 part
    float ml[3];   // centroid - high part, as float32
    float e1[3];
    float e2[3];
    float gam;     // twice the area, high float32 part (negative for a subtracted mesh)
    float gam_lo;  // remainder of gam
    float pad[2];
};

// ------------------------------------------------------------------ rule
// Node blocks (WD_NPB consecutive nodes) of a rule that the mixed per-node
// kernel evaluates in extended precision for one s: those holding a node whose
// weight W_k = w_k (1 + c |xi_k|^2)^(-s) is at least kPreciseWeightFrac of the
// largest. Where the weight is that concentrated, D rests on few nodes and
// their float32 rounding does not average out.
constexpr double kPreciseWeightFrac = 1e-3;
struct PreciseSet {
    int n = 0;                          // listed blocks
    int* d_list = nullptr;              // their indices, ascending
    unsigned char* d_flag = nullptr;    // per node block: 1 if listed
};

// Lattice (cube) rules: nodes on lines of fixed (eta_y, eta_z) = h (j, k),
// eta_x = h i for i = i0 .. i0 + count - 1, stored consecutively.
struct LatLine {
    float yh, yl, zh, zl;  // eta_y, eta_z (turns per unit length) as float pairs
    int i0, count;
    int64_t node0;         // index of the line's first node
};

struct wd_rule {
    wd_ctx* ctx = nullptr;
    wd_rule_desc desc{};
    bool cached = false;              // owned by the context's descriptor cache
    int64_t n_eval = 0, n_total = 0;
    std::vector<double> h_xi;         // SoA, 3 * n_eval
    std::vector<double> h_wg;         // s-free weights
    std::vector<double> h_rad;        // ball rules: radii
    std::vector<float> h_dir;         // ball rules: directions, layout of d_dir
    double* d_xi = nullptr;           // SoA on the device
    double* d_wg = nullptr;
    double wscale = 1.0;              // W = w (1 + wscale |xi|^2)^(-s); 1/(4 pi^2) for cube rules
    // ball rules only: node k = rad[k / n_dir] * omega[k % n_dir] (radius outer)
    int shell0 = 0, shell1 = 0;       // radial window [shell0, shell1) of the desc's n_r radii
    int n_rad = 0;
    int64_t n_dir = 0;
    double* d_rad = nullptr;          // radial nodes, n_rad
    float* d_dir = nullptr;           // per direction, SoA 9 * n_dir: omega (x, y, z) in float32,
                                      // then omega / 2 pi as float pairs: high (x, y, z), low (x, y, z)
    // cube rules: the lattice lines and, per node block of WD_NPB nodes, the
    // first line it touches and the block's first node's place in that line
    int64_t n_lines = 0;
    LatLine* d_lines = nullptr;
    int2* d_lblk = nullptr;
    float lat_hh = 0.0f, lat_hl = 0.0f;   // lattice step h as a float pair
    std::map<double, double*> w_cache;                  // s -> W_k
    std::map<double, PreciseSet> precise_cache;         // s -> extended-precision node blocks
    std::map<std::array<double, 4>, double*> nu_cache;  // (radius, center) -> nu^ (re, im interleaved)
};

// ------------------------------------------------------------------ context
struct wd_ctx {
    int device = 0;
    int num_sms = 0;
    std::recursive_mutex mu;
    std::vector<wd_rule*> rules;      // descriptor cache
    std::vector<wd_rule*> explicit_rules;
    // growable scratch
    char* ws = nullptr;
    size_t ws_bytes = 0;
    // per-node-block completion counters (self-resetting) and the flags word
    int* d_counters = nullptr;
    int64_t n_counters = 0;
    int* d_flags = nullptr;           // [0]: invalid-input flag, [1]: final-block counter
    double* d_scalar = nullptr;       // staging for host-variant scalar results
    std::atomic<int64_t> launches{0};
    // resident blocks of each kernel on this context's device (0: not yet
    // queried); written once per slot, any thread may fill a slot
    std::atomic<int> occupancy[32] = {};  // OccSlot
};

// resident-block slots of wd_ctx::occupancy
enum OccSlot {
    OCC_PAIR = 0,          // + 3 * mixed + mode (6 slots)
    OCC_RADIAL = 6,        // + 3 * mode + radius group index (9 slots)
    OCC_SERVE = 15,        // + form, mixed per-node form at + 2 (3 slots)
    OCC_ADJOINT = 18,      // + 0 float64, 1 mixed, 2 radial (3 slots)
    OCC_PRECISE = 21,      // + mode (3 slots)
    OCC_SERVE_PRECISE = 24,
    OCC_LATTICE = 25,      // + mode (3 slots)
    OCC_SERVE_LATTICE = 28,
};
// the cached count of slot `slot`, or query(kernel) * SMs stored there
template <typename K>
int wd_resident(wd_ctx* ctx, int slot, K kernel, int threads)
{
    int c = ctx->occupancy[slot].load(std::memory_order_relaxed);
    if (c == 0) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess ||
            per_sm < 1) {
            cudaGetLastError();
            per_sm = 1;
        }
        c = per_sm * ctx->num_sms;
        ctx->occupancy[slot].store(c, std::memory_order_relaxed);
    }
    return c;
}

// make ctx's device current
wd_status wd_activate(wd_ctx* ctx);
// grow the scratch area to at least `bytes`
wd_status wd_ws_reserve(wd_ctx* ctx, size_t bytes);
wd_status wd_counters_reserve(wd_ctx* ctx, int64_t n);

// cached per-rule device arrays
wd_status wd_rule_weights(wd_ctx* ctx, wd_rule* rule, double s, const double** d_w, cudaStream_t st);
wd_status wd_rule_sphere(wd_ctx* ctx, wd_rule* rule, double radius, const double* center,
                         const double** d_nu, cudaStream_t st);
// the extended-precision node blocks of the mixed per-node plan for s (built
// on the host and uploaded synchronously on first use, then cached)
wd_status wd_rule_precise(wd_ctx* ctx, wd_rule* rule, double s, const PreciseSet** out);

// ------------------------------------------------------------------ kernels
enum PairMode { MODE_DIST = 0, MODE_FT = 1, MODE_RESID = 2 };

struct PairPlan {
    bool radial = false;      // radius x direction node blocks (ball rules, mixed path)
    int rad_nr = 0;           // radial plan: radii per block (radius group)
    bool lattice = false;     // per-node blocks with lattice-line records (cube rules, mixed path)
    int64_t n_dg = 0;         // radial plan: direction groups
    int n_rg = 0;             // radial plan: radius groups
    int64_t n_nodes = 0;
    int64_t n_tris = 0;       // records (mu and, for a mesh nu, its negated triangles)
    int64_t n_nb = 0;         // node blocks
    int64_t n_tiles = 0;
    int tiles_per_chunk = 0;
    int nchunks = 0;
    int64_t n_items = 0;
    int grid = 0;
};

struct PairArgs {
    const double* xi = nullptr;   // SoA nodes
    int64_t n = 0;
    const void* tris = nullptr;   // TriRecD or TriRecF
    int64_t T = 0;
    const double* W = nullptr;    // MODE_DIST: weights
    const double* nu = nullptr;   // MODE_DIST: sphere nu^ (re, im) or null
    double* partial = nullptr;    // nchunks * n * 2 when nchunks > 1
    int* cnt = nullptr;           // n_nb counters
    double* blockD = nullptr;     // n_nb partial sums
    int* done = nullptr;          // final-block counter
    double* out = nullptr;        // MODE_DIST: D; MODE_FT: re[n]
    double* out_im = nullptr;     // MODE_FT: im[n]
    double* resid = nullptr;      // MODE_RESID: 2 W_k (mu^ - nu^)(xi_k), (re, im) interleaved
    const double* rad = nullptr;  // radial plan: radii (n_rad) and directions (wd_rule::d_dir layout)
    const float* dir = nullptr;
    int n_rad = 0;
    int64_t n_dir = 0;
    int64_t dith_base = 0;        // radial plan: node index of the window's first node in the full rule
    const LatLine* lines = nullptr;  // lattice plan: lines, per-block (first line, offset), h
    const int2* lblk = nullptr;
    float lat_hh = 0.0f, lat_hl = 0.0f;
    // mixed per-node plan: node blocks evaluated in extended precision (see
    // wd_rule_precise), their chunk partials (wd_precise_partial_bytes)
    const unsigned char* precise_flag = nullptr;  // per node block
    const int* precise_list = nullptr;
    int n_precise = 0;
    double* precise_partial = nullptr;
};

constexpr int WD_NPB = 256;   // nodes per block: one node per thread
constexpr int WD_TILE = 128;  // triangles per shared-memory tile
// radial plan (ball rules, mixed path): a block of WD_NPB threads covers
// WD_NPB / NR directions x NR radii (a radius group), one radius per thread;
// NR in {64, 128, 256} is chosen per rule (radial_group). Per tile of NR
// triangles the block builds one record per (direction, triangle), so a
// larger group spreads each record and each tile barrier over more pairs.
constexpr int WD_RAD_RPT = 1;  // radii per thread; 2 (3 blocks per SM) ran 7 % faster on all-Taylor rows but 25 % slower where rows mix branches
template <int NR>
struct RadShape {
    static_assert(NR == 64 || NR == 128 || NR == 256, "radius group of 64, 128 or 256");
    static constexpr int TPD = NR / WD_RAD_RPT;  // threads per direction
    static constexpr int ND = WD_NPB / TPD;      // directions per block
    static constexpr int TILE = WD_NPB / ND;     // triangles per record tile (one record per thread)
    static constexpr int IDX = NR == 64 ? 0 : (NR == 128 ? 1 : 2);
};

size_t wd_tri_record_bytes(int precision);
// stage triangles (a1): records for mu (sign +1) at offset 0 and optionally a
// second mesh (sign -1) after them
wd_status wd_launch_stage(wd_ctx* ctx, int precision, const double* d_verts, int64_t nv,
                          const int32_t* d_tris, int64_t nt, double sign, void* d_rec,
                          int64_t rec_offset, cudaStream_t st);
wd_status wd_plan_pair(wd_ctx* ctx, int precision, int mode, int64_t n_nodes, int64_t n_tris,
                       PairPlan* plan);
// plan for a rule: the radial kernel for ball rules in the mixed path, else as above
wd_status wd_plan_pair_rule(wd_ctx* ctx, const wd_rule* rule, int precision, int mode, int64_t n_tris,
                            PairPlan* plan);
// node arrays of a rule into the pair arguments (xi, n and, for ball rules, rad/dir)
void wd_pair_args_rule(const wd_rule* rule, PairArgs& a);
// the plan of the extended-precision kernel for n_precise listed blocks
// (the plan's node blocks, triangle chunks of their own) and the bytes of its
// chunk partials
PairPlan wd_precise_plan(wd_ctx* ctx, const PairPlan& plan, int n_precise, int mode);
size_t wd_precise_partial_bytes(const PairPlan& precise_plan, int n_precise);
// launches the plan's kernel, then, for a mixed per-node plan with
// args.n_precise > 0, the extended-precision kernel over the listed blocks
wd_status wd_launch_pair(wd_ctx* ctx, int precision, int mode, const PairPlan& plan,
                         const PairArgs& args, cudaStream_t st);
wd_status wd_launch_sphere(wd_ctx* ctx, const double* d_xi, int64_t n, double radius,
                           const double* center, double* d_re, double* d_im, double* d_inter,
                           cudaStream_t st);
// adjoint (wd_adjoint.cu): gradient of D with respect to the vertices of mu
struct AdjPlan {
    bool radial = false;     // radial mixed adjoint: chunks are ranges of directions
    int64_t dirs_per_chunk = 0;
    int64_t n_tb = 0;        // triangle blocks
    int64_t n_node_tiles = 0;
    int tiles_per_chunk = 0;
    int nchunks = 0;
    int64_t n_items = 0;
    int grid = 0;
};
wd_status wd_plan_adjoint(wd_ctx* ctx, int precision, int64_t n_nodes, int64_t n_tris, AdjPlan* plan);
// plan for a rule: the radial adjoint for ball rules in the mixed path, else as above
wd_status wd_plan_adjoint_rule(wd_ctx* ctx, const wd_rule* rule, int precision, int64_t n_tris, AdjPlan* plan);
// scratch of the radial adjoint (the rotated residual, direction-major)
size_t wd_adjoint_radial_bytes(const wd_rule* rule);
// d_rec: float64 records of mu (geometry for the final scatter, and the
// float64 adjoint); d_rec_mixed: mixed records of mu (mixed adjoint);
// d_scatter: wd_adjoint_scatter_bytes(nt, nv) bytes of scratch. d_grad must
// be zeroed by the caller; the result is bitwise independent of launch order.
size_t wd_adjoint_scatter_bytes(int64_t nt, int64_t nv);
// d_radial: wd_adjoint_radial_bytes(rule) bytes when plan.radial, else unused
wd_status wd_launch_adjoint(wd_ctx* ctx, int precision, const AdjPlan& plan, const wd_rule* rule,
                            const double* d_resid, const void* d_rec, const void* d_rec_mixed, int64_t nt,
                            void* d_radial, double* d_partial, void* d_scatter, const int32_t* d_tris, int64_t nv,
                            double* d_grad, cudaStream_t st);

// batched serving kernels (wd_pair.cu), driven by a device descriptor table.
// Every admitted request carries the arguments and the plan of its own
// wd_distance launch (radial or per-node form); a launch runs contiguous
// ranges of each request's work items, so a request's items may spread over
// several launches and still sum in the order of its plan.
struct ServeReq {
    PairArgs a;             // out -> the request's result slot
    PairPlan p;
    PairPlan pp;            // mixed per-node plan: its extended-precision blocks (items after p's)
};
struct ServeRange {         // items [first, first + count) of request `req`
    int req;
    int count;
    int64_t first;
    int64_t start;          // launch-local index of the range's first item (prefix sum)
};
enum { SERVE_RADIAL = 0, SERVE_NODE = 1, SERVE_PRECISE = 2, SERVE_LATTICE = 3, SERVE_FORMS = 4 };
struct ServeTable {         // laid out in pinned host memory and copied whole per launch
    int n_ranges[SERVE_FORMS];  // per kernel form
    int64_t n_items[SERVE_FORMS];
    int next[SERVE_FORMS];  // dynamic item counters (zero in the host copy)
};
constexpr int WD_SERVE_RANGES = 512;  // ranges per form and launch
// table layout: ServeTable, then WD_SERVE_RANGES ranges per form, then the requests
wd_status wd_launch_serve(wd_ctx* ctx, int precision, ServeTable* d_head, const ServeRange* d_ranges,
                          const ServeReq* d_reqs, cudaStream_t st);
int wd_serve_resident(wd_ctx* ctx, int precision, int form);
// the plan of a request: wd_plan_pair_rule's, with at most max_tiles tiles per item
wd_status wd_plan_pair_serve(wd_ctx* ctx, const wd_rule* rule, int precision, int64_t n_tris, int max_tiles,
                             PairPlan* plan);

// Gauss-Legendre nodes and weights on [-1, 1], ascending (host, long double)
void wd_legendre_rule(int n, std::vector<double>& x, std::vector<double>& w);
// the paper's atomic transform (wd_atoms.cu): d_rec holds float64 records
wd_status wd_launch_atoms(wd_ctx* ctx, const double* d_xi, int64_t n, const void* d_rec, int64_t T, double* d_re,
                          double* d_im, cudaStream_t st);

wd_status wd_launch_weights(wd_ctx* ctx, const double* d_xi, const double* d_wg, int64_t n,
                            double s, double wscale, double* d_w, cudaStream_t st);
