/*
 * wd.h -- C ABI of libwd: the H^{-s} weak distance between a triangulated
 * surface and a reference measure, evaluated on one NVIDIA B300 (sm_103a).
 *
 * Method (Koga, arXiv 2304.06340): identify a surface with its surface
 * measure mu, take the Fourier transform of the measure on R^3 (Sec. 2.1,
 * Eq. (ft_measure)), and compare two measures in the inhomogeneous Sobolev
 * norm of negative order through the Plancherel form (Eq. (sobolev_2)).
 * This library uses the angular convention
 *
 *     mu^(xi) = int_{R^3} exp(-i xi.x) dmu(x)
 *     D       = ||mu - nu||^2 = int (1 + |xi|^2)^(-s) |mu^(xi) - nu^(xi)|^2 dxi
 *
 * (the paper's 2 pi convention maps by xi = 2 pi eta; its order s_p < 0 is -s
 * here), truncated to the ball |xi| <= R and discretised by a quadrature rule
 * {xi_k, w_k}: D = sum_k w_k (1 + |xi_k|^2)^(-s) |mu^(xi_k) - nu^(xi_k)|^2.
 * No (2 pi)^-3 factor is applied. For a mesh, mu^ is the sum over triangles
 * (linearity, Sec. 3.1) of the exact transform of each flat triangle
 * (Eq. (simplex32_ft)); the unit sphere's transform is 4 pi sin|xi|/|xi|
 * (Eq. (ft_nsphere_sinc)).
 *
 * Conventions of every call:
 *   - The return value is a wd_status; calls never abort or exit.
 *   - wd_last_error() returns a message for the last failing call of the
 *     calling thread. The string is owned by the library.
 *   - The caller owns every input and output array. Host inputs are copied
 *     as needed before the call returns; nothing keeps a caller pointer.
 *   - Host-pointer variants are synchronous. `_dev` variants take device
 *     pointers and a CUDA stream (passed as void*, a cudaStream_t; NULL is the
 *     legacy default stream); they are asynchronous on that stream.
 *   - Meshes: vertices are float64, n_verts x 3 (x, y, z interleaved);
 *     triangles are int32, n_tris x 3 vertex indices. Vertex order inside a
 *     triangle is irrelevant (Sec. 2.2). A degenerate triangle (zero area)
 *     contributes zero.
 *   - Frequency rule nodes are stored structure-of-arrays (x[n], y[n], z[n]).
 *   - A wd_ctx owns a device workspace; calls on one context must not overlap
 *     in time (serialise them on one stream or use one context per stream).
 *     The first call at a new problem size may grow that workspace, which
 *     synchronises the device; make such a call before capturing a graph.
 */
#ifndef WD_H
#define WD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    WD_OK = 0,
    WD_EINVAL = 1,     /* invalid argument: bad index, non-finite input, s <= 0, R <= 0, ... */
    WD_ENOMEM = 2,     /* device allocation failed or a memory cap was exceeded */
    WD_ECUDA = 3,      /* a CUDA runtime error; its text is in wd_last_error() */
    WD_EBUSY = 4,      /* no free slot (serving) */
    WD_ETIMEOUT = 5,   /* a bounded wait ran out */
    WD_ENOTFOUND = 6,  /* unknown ticket or handle */
    WD_ECANCELLED = 7  /* the request was cancelled */
} wd_status;

enum { WD_FP64 = 0, WD_MIXED = 1 };               /* arithmetic of the pair kernel */
enum { WD_RULE_BALL = 0, WD_RULE_CUBE_TRAP = 1, WD_RULE_EXPLICIT = 2 };  /* frequency-rule kinds */
enum { WD_NU_SPHERE = 0, WD_NU_MESH = 1 };        /* reference-measure kinds */

typedef struct wd_ctx wd_ctx;
typedef struct wd_rule wd_rule;

/* ----------------------------------------------------------------- context */

/* Create a context on CUDA device `device`. The library makes that device
 * current on the calling thread at every call that takes the context. */
wd_status wd_create(int device, wd_ctx** out);
void wd_destroy(wd_ctx* ctx);

/* Message of the calling thread's last failure ("" if none). ctx may be NULL. */
const char* wd_last_error(const wd_ctx* ctx);

/* Wait for all work of `stream` and report deferred errors of earlier `_dev`
 * calls on this context: WD_EINVAL if a staged mesh had a triangle index
 * outside [0, n_verts) or a non-finite vertex (that triangle was treated as
 * degenerate), WD_ECUDA on a CUDA error. Clears the deferred flag. */
wd_status wd_sync(wd_ctx* ctx, void* stream);

/* ------------------------------------------------------------ frequency rule */

/* Ball-centred rule for |xi| <= R (Sec. 3.2, closing remark on rules over balls
 * centred at the origin, justified by the radial symmetry of the weight):
 *   r   : Gauss-Legendre on [0, R], n_r nodes (the weight carries r^2)
 *   u   : cos(theta), Gauss-Legendre on [-1, 1], n_polar nodes
 *   phi : 2 pi k / n_azim, trapezoid
 *   xi  = r (sqrt(1 - u^2) cos phi, sqrt(1 - u^2) sin phi, u)
 * hermitian != 0 keeps only u > 0 and doubles its weight, which is exact for
 * real measures because |mu^ - nu^|^2 is even in xi (n_polar must be even).
 * Node order: r outermost, then u ascending, then phi fastest. */
/* WD_RULE_CUBE_TRAP is the rule of the paper's own experiments (Sec. 3.2:
 * the lattice of Eq. (def_trap_grid) with the trapezoidal rule of Eq.
 * (trap_rule_R3)), in the paper's 2 pi convention (Eq. (ft_measure)):
 *   eta_{ijk} = (i, j, k) h,  h = 2 R / n_r,  i, j, k = -n_r/2 .. n_r/2,
 *   weight h^3 x (1/2 per coordinate on the boundary of [-R, R]^3),
 * with R = xi_max in the paper's frequency units and n_r = M (even, >= 2);
 * n_polar and n_azim are ignored. The rule's nodes are stored in this
 * library's angular convention, xi = 2 pi eta, so mu^(xi) is the paper's
 * transform at eta, and its per-call weight is the paper's
 * (1 + |eta|^2)^(-s) = (1 + |xi|^2 / (4 pi^2))^(-s): with this kind, D is the
 * paper's squared H_{-s} norm of mu - nu, Eq. (sobolev_2), quadrature of
 * Eq. (trap_rule_R3). hermitian != 0 keeps the half eta_z > 0, or eta_z = 0
 * and eta_y > 0, or eta_z = eta_y = 0 and eta_x >= 0, doubling every weight
 * but the origin's. Node order: eta_z outermost, then eta_y, eta_x fastest. */
typedef struct {
    int kind;      /* WD_RULE_BALL or WD_RULE_CUBE_TRAP */
    double R;      /* ball: truncation radius; cube: xi_max (paper units); > 0 */
    int n_r;       /* ball: radial nodes, >= 1; cube: M, even, >= 2 */
    int n_polar;   /* ball: polar nodes, >= 1 (even when hermitian) */
    int n_azim;    /* ball: azimuthal nodes, >= 1 */
    int hermitian; /* 0 or 1 */
} wd_rule_desc;

/* Build (or fetch from the context's cache: an equal descriptor returns the
 * same handle) a rule and upload it to the device. The handle belongs to the
 * context; wd_rule_free is optional and only drops it from the cache. */
wd_status wd_build_freq_rule(wd_ctx* ctx, const wd_rule_desc* desc, wd_rule** out);

/* The ball rule of `desc` restricted to its radial shells [shell_begin,
 * shell_end) of the n_r Gauss-Legendre radii (0 <= shell_begin < shell_end <=
 * n_r): the same nodes and weights as the full rule's nodes with those radial
 * indices, in the same order. The quadrature is a sum over nodes, so D over
 * windows that partition [0, n_r) adds up to D over the full rule; a window is
 * the unit in which radial shells are split between calls, streams or GPUs
 * (Sec. 3.2, rules over balls centred at the origin). The mixed path assigns
 * every node the same phase dither as in the full rule, so for windows whose
 * bounds are multiples of 32 each node's transform is evaluated with the same
 * float32 operations as in the full rule. desc->kind must be WD_RULE_BALL.
 * Cached like wd_build_freq_rule (by descriptor and window). */
wd_status wd_build_freq_rule_shells(wd_ctx* ctx, const wd_rule_desc* desc, int shell_begin, int shell_end,
                                    wd_rule** out);

/* A rule from explicit host nodes: xi is SoA (x[n], y[n], z[n]), w_geom[n] the
 * s-free weights (the factor (1 + |xi|^2)^(-s) is applied per call). Used for
 * sub-rules and user rules. Not cached by descriptor; free with wd_rule_free. */
wd_status wd_rule_from_nodes(wd_ctx* ctx, const double* xi, const double* w_geom, int64_t n,
                             wd_rule** out);

/* Number of nodes the kernels evaluate, and the size of the full rule before
 * Hermitian halving (equal when hermitian == 0). */
wd_status wd_rule_info(const wd_rule* rule, int64_t* n_nodes_evaluated, int64_t* n_nodes_total);

/* Copy the evaluated nodes (SoA, 3 * n doubles) and s-free weights (n) to host
 * arrays; either pointer may be NULL. */
wd_status wd_rule_copy_nodes(const wd_rule* rule, double* xi, double* w_geom);
void wd_rule_free(wd_rule* rule);

/* ------------------------------------------------------------ transforms */

typedef struct {
    const double* verts;  /* n_verts x 3 */
    int64_t n_verts;
    const int32_t* tris;  /* n_tris x 3 */
    int64_t n_tris;
} wd_mesh;

/* mu^(xi_k) of the mesh's surface measure at every evaluated node: the sum over
 * triangles of gamma_T * G[xi.a, xi.b, xi.c], the second divided difference of
 * G(t) = -exp(-i t) with gamma_T twice the area (Eq. (simplex32_ft) in the
 * angular convention; Sec. 3.1 for the sum). precision is WD_FP64 (every step
 * in float64) or WD_MIXED (float64 staging and per-node accumulation, phase
 * reduction in extended float32 pairs, float32 transcendental and
 * divided-difference arithmetic). out_re/out_im: n_nodes_evaluated doubles. */
wd_status wd_mesh_ft(wd_ctx* ctx, const wd_rule* rule, const wd_mesh* mesh, int precision,
                     double* out_re, double* out_im);
wd_status wd_mesh_ft_dev(wd_ctx* ctx, const wd_rule* rule, const double* d_verts, int64_t n_verts,
                         const int32_t* d_tris, int64_t n_tris, int precision,
                         double* d_out_re, double* d_out_im, void* stream);

/* The paper's atomic approximation of the same transform (Sec. 3.1, Eqs.
 * (change_variable) and (change_variable_approx)). Each triangle is replaced by
 * 64 weighted atoms from the 8-point Gauss-Legendre rule applied twice to the
 * standard simplex as an iterated integral, and mu^ is their plane-wave sum,
 * in float64. It approximates wd_mesh_ft with an error falling like
 * (|xi| h)^15 for triangles of size h. It costs 64 exponentials per
 * (triangle, node) pair where the exact formula needs one or two. Arguments,
 * errors and outputs as for wd_mesh_ft. */
wd_status wd_mesh_ft_atoms(wd_ctx* ctx, const wd_rule* rule, const wd_mesh* mesh, double* out_re, double* out_im);

/* Transform of the surface measure of the sphere |x - center| = radius:
 * 4 pi radius sin(radius |xi|)/|xi| exp(-i xi.center) (Eq. (ft_nsphere_sinc),
 * angular convention, scaled and translated), in float64. */
wd_status wd_sphere_ft(wd_ctx* ctx, const wd_rule* rule, double radius, const double center[3],
                       double* out_re, double* out_im);
wd_status wd_sphere_ft_dev(wd_ctx* ctx, const wd_rule* rule, double radius, const double center[3],
                           double* d_out_re, double* d_out_im, void* stream);

/* ------------------------------------------------------------ distance */

/* Reference measure nu: a sphere (radius > 0, center) or a second mesh. */
typedef struct {
    int kind;              /* WD_NU_SPHERE or WD_NU_MESH */
    double radius;
    double center[3];
    const wd_mesh* mesh;   /* WD_NU_MESH: host mesh for wd_distance; for the _dev
                              variants its verts/tris are device pointers */
} wd_measure;

/* D = sum_k w_k (1 + |xi_k|^2)^(-s) |mu^(xi_k) - nu^(xi_k)|^2 (the rule's
 * quadrature of Eq. (sobolev_2) with order -s, no (2 pi)^-3), mu the mesh.
 * s > 0 (finite for every truncated rule; the untruncated norm of a surface
 * measure needs s > 1/2, Sec. 2.2). One fused kernel evaluates every
 * (triangle, node) pair, sums per node, subtracts nu^, weights and reduces;
 * the final sum has a fixed order, so results are reproducible run to run. */
wd_status wd_distance(wd_ctx* ctx, const wd_rule* rule, const wd_mesh* mu, const wd_measure* nu,
                      double s, int precision, double* dist2);
/* d_dist2: one device double, written when the stream reaches the call. */
wd_status wd_distance_dev(wd_ctx* ctx, const wd_rule* rule, const double* d_verts, int64_t n_verts,
                          const int32_t* d_tris, int64_t n_tris, const wd_measure* nu, double s,
                          int precision, double* d_dist2, void* stream);

/* D and its gradient with respect to the vertices of mu (n_verts x 3):
 *   dD/dv = sum_k 2 W_k Re(conj(mu^ - nu^)(xi_k) d mu^(xi_k)/dv),
 *   dF_T/da = (d gamma/da) G[t_a,t_b,t_c] + gamma G[t_a,t_a,t_b,t_c] xi.
 * Precision as for wd_distance. */
wd_status wd_distance_grad(wd_ctx* ctx, const wd_rule* rule, const wd_mesh* mu, const wd_measure* nu,
                           double s, int precision, double* dist2, double* grad_verts);
wd_status wd_distance_grad_dev(wd_ctx* ctx, const wd_rule* rule, const double* d_verts,
                               int64_t n_verts, const int32_t* d_tris, int64_t n_tris,
                               const wd_measure* nu, double s, int precision, double* d_dist2,
                               double* d_grad_verts, void* stream);

/* Number of kernel launches issued by this context since creation (all entry
 * points). Used to report launch counts. */
int64_t wd_launch_count(const wd_ctx* ctx);

/* ------------------------------------------------------------ serving */

/* Continuous batching of distance queries (mesh vs the unit sphere) on one GPU.
 * Not in the paper, which times single evaluations (Sec. 4.3); this serves many
 * queries of uneven size at once. A worker thread admits queued queries while
 * request slots and a fixed device memory arena allow. Each admitted query gets
 * the work plan of its own wd_distance_dev launch (node blocks x triangle
 * chunks; chunks are capped at 8192 triangles so that a work item stays short).
 * Every batched launch replays a captured CUDA graph over a budget of work
 * items drawn round-robin from all admitted queries; a query's items may span
 * launches, and its chunks, node blocks and final sum combine in its plan's
 * fixed order. Queries that arrive while others run join the next launch, and
 * the worker prepares launch k + 1 while launch k runs. Results are the same
 * bits alone and in any mix, and equal those of wd_distance_dev with the same
 * rule and precision whenever the chunk cap leaves the plan unchanged (within
 * rounding of the chunk sums otherwise). */
#define WD_SERVE_MAX_SLOTS 256

typedef struct wd_server wd_server;

typedef struct {
    int64_t mem_cap_bytes;     /* device arena for admitted queries (meshes, records, partials) */
    int max_slots;             /* queries admitted at once, 1..WD_SERVE_MAX_SLOTS */
    int max_pending;           /* queue length at which submit returns WD_EBUSY */
    int timeout_ms;            /* a query still queued after this long ends with WD_ETIMEOUT (0: never) */
    int precision;             /* WD_FP64 or WD_MIXED */
    int64_t pairs_per_launch;  /* (triangle, node) pairs per batched launch */
    int n_rules;               /* 1..4 frequency rules, selected per query by R */
    wd_rule_desc rules[4];
} wd_serve_config;

typedef struct {
    int64_t submitted, admitted, completed, rejected, timeouts, cancelled, failed, launches;
    int64_t pending, active, arena_used_bytes;
    double pairs;              /* (triangle, node) pairs of the queries completed */
    double p50_us, p99_us, max_us, mean_us;  /* submit-to-result latency of completed queries */
    double qps;                /* completed queries per second, first submit to last result */
    double gpu_busy;           /* device time of the batched launches (events) over that span */
} wd_serve_stats_t;

/* Start the worker; builds the rules and captures the graph. */
wd_status wd_serve_start(wd_ctx* ctx, const wd_serve_config* cfg, wd_server** out);
/* Queue a query (the mesh is copied). WD_EBUSY: queue full; WD_ENOMEM: larger
 * than the arena; WD_EINVAL: bad mesh, s <= 0 or no rule for R. */
wd_status wd_serve_submit(wd_server* sv, const wd_mesh* mesh, double s, double R, uint64_t* ticket);
/* Non-blocking: done = 1 once the query finished (req_status tells how). */
wd_status wd_serve_poll(wd_server* sv, uint64_t ticket, int* done, double* dist2, wd_status* req_status);
/* Blocks for at most timeout_ms; WD_ETIMEOUT if the query is not finished by then. */
wd_status wd_serve_wait(wd_server* sv, uint64_t ticket, int timeout_ms, double* dist2);
/* Cancel a queued or running query; it finishes with WD_ECANCELLED. */
wd_status wd_serve_cancel(wd_server* sv, uint64_t ticket);
wd_status wd_serve_stats(wd_server* sv, wd_serve_stats_t* out);
/* Cancel queued queries, let admitted ones finish, free everything. */
wd_status wd_serve_stop(wd_server* sv);

/* ------------------------------------------------------------ allocation-free variant */

/* Fixed size of the library's static device scratch used below (64 MiB). */
#define WD_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)

/* The paper has no counterpart to this entry point; it exists for callers that
 * must not allocate device memory while they run: applications whose own
 * memory manager owns the device, latency-critical loops that may not touch
 * cudaMalloc/cudaFree (which can synchronise the device), and plugins that
 * only get buffers from their host. It computes the same D as wd_distance_dev
 * with a sphere as reference, using the same kernels, but takes every input
 * as a caller-owned device array and needs no context and no rule handle:
 *   d_xi      frequency nodes, SoA (x[n], y[n], z[n]) float64
 *   d_w_geom  s-free node weights, n float64 (as from wd_rule_copy_nodes)
 *   d_verts, d_tris  the mesh, as for wd_distance_dev
 *   radius, center   the reference sphere
 *   d_dist2   one float64 output, written when the stream reaches the call
 * It runs on the calling thread's current device. All intermediate storage
 * lives in one static array of WD_NOALLOC_SCRATCH_BYTES that every device
 * loading the library reserves until the process exits; a problem needing
 * more is rejected with WD_EINVAL and a message giving the size. The call
 * makes no device allocation. Its first call on a device resolves the array's
 * device address (cudaGetSymbolAddress); make that first call before any
 * stream capture. All calls share the one array, and counters in it are
 * cleared at each call: calls whose work overlaps on the GPU (different
 * streams, or other host threads) race and must be serialised by the caller.
 * Triangle indices are not validated on the host: an out-of-range index or a
 * non-finite vertex makes that triangle contribute zero. */
wd_status wd_distance_dev_noalloc(const double* d_xi, const double* d_w_geom, int64_t n_nodes,
                                  const double* d_verts, int64_t n_verts, const int32_t* d_tris,
                                  int64_t n_tris, double s, double radius, const double center[3],
                                  int precision, double* d_dist2, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* WD_H */
