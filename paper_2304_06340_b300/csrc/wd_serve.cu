// Serving loop: continuous batching of distance queries on one GPU.
//
// submit() copies a query (mesh, s, R) into host memory and queues it. A worker
// thread admits queued queries while request slots and device memory (a fixed
// arena, first-fit) are free, stages their meshes, and gives each the plan of
// its own wd_distance launch: node blocks x triangle chunks, chunks capped so
// that one work item stays short. Each batched launch replays a captured CUDA
// graph that copies a descriptor table from pinned memory, runs the batched
// pair kernels over contiguous ranges of the admitted queries' work items
// (a share of a pair budget per query, round-robin, largest items first) and
// copies the result slots back. Blocks take items from a counter. A query's
// chunks, node blocks and final sum combine in the fixed order of its plan in
// whichever launch runs its last item, so results do not depend on the mix.
// Two tables alternate: the worker builds and enqueues launch k + 1 while
// launch k runs, then retires the queries that launch k finished. Queries that
// arrive meanwhile join the next launch; the frequency rules, their weights
// and the sphere's transform stay resident on the device.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "wd_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

constexpr int kMaxSlots = WD_SERVE_MAX_SLOTS;
constexpr int kRoundItems = 8;    // work items taken per query per round-robin round
constexpr int kMaxItemTiles = 64; // triangle tiles per work item (2^21 pairs of a 256-node block)
constexpr int kBuffers = 2;       // launch tables in flight

size_t align_up(size_t v) { return (v + 255) & ~size_t(255); }

// LOST: finished, but its completion dropped by WD_FAULT_DROP_COMPLETION, so
// the client never sees it done (its waits run out)
enum ReqState { PENDING = 0, ADMITTED = 1, DONE = 2, FAILED = 3, LOST = 4 };

struct Request {
    uint64_t ticket = 0;
    std::vector<double> verts;
    std::vector<int32_t> tris;
    double s = 1.0;
    int rule = 0;
    Clock::time_point t_submit, t_done;
    ReqState state = PENDING;
    wd_status status = WD_OK;
    double result = 0.0;
    bool cancel = false;
    std::string why;            // failure reason, for wd_last_error of the waiting client
    // device side
    size_t off = 0, bytes = 0;
    int slot = -1;
    PairPlan plan;
    const PreciseSet* precise = nullptr;  // mixed per-node plan: extended-precision blocks for s
    PairPlan pplan;             // their plan; their items follow plan's
    int64_t n_items = 0;        // plan.n_items (+ pplan.n_items)
    int64_t next_item = 0;      // first item not yet given to a launch
    int64_t last_seq = -1;      // last launch that runs items of this query
    int64_t finish_seq = -1;    // the launch that runs its last item (result valid once it completes)
};

// Arena layout of one request: records, chunk partials, block sums, counters
// (node blocks, then the final-block counter), vertices, triangles.
struct ReqLayout {
    size_t rec = 0, partial = 0, ppartial = 0, blockD = 0, cnt = 0, done = 0, verts = 0, tris = 0, end = 0;
};

// First-fit allocator over one device arena.
struct Arena {
    char* base = nullptr;
    size_t cap = 0;
    std::map<size_t, size_t> free_;  // offset -> size
    size_t used = 0;
    void init(char* b, size_t c)
    {
        base = b;
        cap = c;
        free_.clear();
        free_[0] = c;
        used = 0;
    }
    bool alloc(size_t bytes, size_t* off)
    {
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t o = it->first;
                free_.erase(it);
                if (rest) free_[o + bytes] = rest;
                used += bytes;
                return true;
            }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        used -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct RuleEntry {
    wd_rule* rule = nullptr;
    const double* nu = nullptr;
    std::map<double, const double*> W;
};

}  // namespace

struct wd_server {
    wd_ctx* ctx = nullptr;
    wd_serve_config cfg{};
    cudaStream_t stream = nullptr;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stopping = false;
    uint64_t next_ticket = 1;
    std::deque<Request*> pending;
    std::vector<Request*> slots;  // admitted requests by slot
    std::unordered_map<uint64_t, Request*> all;
    Arena arena;
    char* d_arena = nullptr;
    std::vector<RuleEntry> rules;
    // descriptor tables: per buffer a pinned host copy and a device copy with
    // the same layout (ServeTable, ranges of both forms, request descriptors)
    size_t table_bytes = 0, off_ranges = 0, off_reqs = 0;
    char* h_table[kBuffers] = {nullptr, nullptr};
    char* d_table[kBuffers] = {nullptr, nullptr};
    double* h_results[kBuffers] = {nullptr, nullptr};
    double* d_results = nullptr;
    cudaGraphExec_t graph[kBuffers] = {nullptr, nullptr};
    cudaEvent_t ev_start[kBuffers] = {nullptr, nullptr}, ev_end[kBuffers] = {nullptr, nullptr};
    int kernels_per_launch = 0;
    // statistics
    wd_serve_stats_t st{};
    std::vector<double> lat_us;
    Clock::time_point t_first_submit{}, t_last_done{};
    bool any_submit = false;
    double busy_s = 0.0;          // device time of completed launches (events)
    wd_status fatal = WD_OK;
    std::string fatal_msg;
    int drop_nth = 0;        // WD_FAULT_DROP_COMPLETION at start (0: off)
    int64_t n_ok_seen = 0;   // successful completions so far
};

namespace {

ReqLayout request_layout(const wd_server* sv, const Request* r)
{
    const int64_t T = (int64_t)r->tris.size() / 3;
    const int64_t V = (int64_t)r->verts.size() / 3;
    const PairPlan& p = r->plan;
    ReqLayout L;
    size_t o = 0;
    L.rec = o;
    o += align_up(wd_tri_record_bytes(sv->cfg.precision) * (size_t)(T > 0 ? T : 1));
    L.partial = o;
    if (p.nchunks > 1) o += align_up(sizeof(double) * 2 * (size_t)p.nchunks * (size_t)p.n_nodes);
    L.ppartial = o;
    if (r->precise) o += align_up(wd_precise_partial_bytes(r->pplan, r->precise->n));
    L.blockD = o;
    o += align_up(sizeof(double) * (size_t)(p.n_nb > 0 ? p.n_nb : 1));
    L.cnt = o;
    L.done = L.cnt + sizeof(int) * (size_t)(p.n_nb > 0 ? p.n_nb : 1);
    o += align_up(L.done + sizeof(int) - L.cnt);
    L.verts = o;
    o += align_up(sizeof(double) * 3 * (size_t)(V > 0 ? V : 1));
    L.tris = o;
    o += align_up(sizeof(int32_t) * 3 * (size_t)(T > 0 ? T : 1));
    L.end = o;
    return L;
}

void finish(wd_server* sv, Request* r, wd_status status, double result)
{
    if (status == WD_OK && sv->drop_nth > 0 && ++sv->n_ok_seen == sv->drop_nth) {
        // injected fault: the work is done but the completion never reaches the client
        wd_log(2, "injected fault: completion of ticket %llu dropped", (unsigned long long)r->ticket);
        r->state = LOST;
        r->verts.clear();
        r->tris.clear();
        sv->st.completed++;
        return;
    }
    r->state = status == WD_OK ? DONE : FAILED;
    r->status = status;
    r->result = result;
    r->t_done = Clock::now();
    r->verts.clear();
    r->verts.shrink_to_fit();
    r->tris.clear();
    r->tris.shrink_to_fit();
    if (status == WD_OK) {
        sv->st.completed++;
        sv->lat_us.push_back(std::chrono::duration<double, std::micro>(r->t_done - r->t_submit).count());
        sv->t_last_done = r->t_done;
    } else if (status == WD_ETIMEOUT) {
        sv->st.timeouts++;
    } else if (status == WD_ECANCELLED) {
        sv->st.cancelled++;
    } else {
        sv->st.failed++;
    }
}

void release_slot(wd_server* sv, Request* r)
{
    if (r->slot >= 0) {
        sv->slots[r->slot] = nullptr;
        r->slot = -1;
    }
    if (r->bytes) {
        sv->arena.release(r->off, r->bytes);
        r->bytes = 0;
    }
}

ServeTable* table_head(wd_server* sv, int b) { return reinterpret_cast<ServeTable*>(sv->h_table[b]); }
ServeRange* table_ranges(wd_server* sv, int b) { return reinterpret_cast<ServeRange*>(sv->h_table[b] + sv->off_ranges); }
ServeReq* table_reqs(wd_server* sv, int b) { return reinterpret_cast<ServeReq*>(sv->h_table[b] + sv->off_reqs); }

// One graph per table buffer: table in, batched kernels, result slots out.
// (The worker brackets each replay with events recorded on the stream.)
wd_status capture_graph(wd_server* sv, int b)
{
    cudaStream_t s = sv->stream;
    ServeTable* d_head = reinterpret_cast<ServeTable*>(sv->d_table[b]);
    const ServeRange* d_ranges = reinterpret_cast<const ServeRange*>(sv->d_table[b] + sv->off_ranges);
    const ServeReq* d_reqs = reinterpret_cast<const ServeReq*>(sv->d_table[b] + sv->off_reqs);
    WD_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaMemcpyAsync(sv->d_table[b], sv->h_table[b], sv->table_bytes, cudaMemcpyHostToDevice, s);
    const int64_t before = sv->ctx->launches;
    wd_status st = WD_OK;
    if (e == cudaSuccess) st = wd_launch_serve(sv->ctx, sv->cfg.precision, d_head, d_ranges, d_reqs, s);
    sv->kernels_per_launch = (int)(sv->ctx->launches - before);
    sv->ctx->launches = before;  // counted per replay instead
    if (e == cudaSuccess && st == WD_OK)
        e = cudaMemcpyAsync(sv->h_results[b], sv->d_results, sizeof(double) * kMaxSlots, cudaMemcpyDeviceToHost, s);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(s, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return wd_cuda_status(e, "serve graph capture");
    }
    if (st != WD_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e2 != cudaSuccess) return wd_cuda_status(e2, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&sv->graph[b], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return wd_cuda_status(e, "cudaGraphInstantiate");
    return WD_OK;
}

// Stage one admitted request: copy its mesh, build its triangle records, clear
// its completion counters and make sure the weights for its s exist.
wd_status stage_request(wd_server* sv, Request* r)
{
    const int64_t T = (int64_t)r->tris.size() / 3;
    const int64_t V = (int64_t)r->verts.size() / 3;
    const ReqLayout L = request_layout(sv, r);
    char* base = sv->d_arena + r->off;
    if (V > 0)
        WD_CUDA(cudaMemcpyAsync(base + L.verts, r->verts.data(), sizeof(double) * 3 * V, cudaMemcpyHostToDevice,
                                sv->stream));
    if (T > 0)
        WD_CUDA(cudaMemcpyAsync(base + L.tris, r->tris.data(), sizeof(int32_t) * 3 * T, cudaMemcpyHostToDevice,
                                sv->stream));
    WD_CUDA(cudaMemsetAsync(base + L.cnt, 0, L.done + sizeof(int) - L.cnt, sv->stream));
    wd_status st = wd_launch_stage(sv->ctx, sv->cfg.precision, reinterpret_cast<const double*>(base + L.verts), V,
                                   reinterpret_cast<const int32_t*>(base + L.tris), T, 1.0, base + L.rec, 0,
                                   sv->stream);
    if (st != WD_OK) return st;
    RuleEntry& re = sv->rules[r->rule];
    if (!re.W.count(r->s)) {
        const double* w = nullptr;
        if ((st = wd_rule_weights(sv->ctx, re.rule, r->s, &w, sv->stream)) != WD_OK) return st;
        re.W[r->s] = w;
    }
    // the request's descriptor, the same in both tables
    ServeReq q;
    wd_pair_args_rule(re.rule, q.a);
    q.a.tris = base + L.rec;
    q.a.T = T;
    q.a.W = re.W[r->s];
    q.a.nu = re.nu;
    q.a.partial = reinterpret_cast<double*>(base + L.partial);
    q.a.blockD = reinterpret_cast<double*>(base + L.blockD);
    q.a.cnt = reinterpret_cast<int*>(base + L.cnt);
    q.a.done = reinterpret_cast<int*>(base + L.done);
    q.a.out = sv->d_results + r->slot;
    if (r->precise) {
        q.a.precise_flag = r->precise->d_flag;
        q.a.precise_list = r->precise->d_list;
        q.a.n_precise = r->precise->n;
        q.a.precise_partial = reinterpret_cast<double*>(base + L.ppartial);
    }
    q.p = r->plan;
    q.pp = r->pplan;
    for (int b = 0; b < kBuffers; ++b) table_reqs(sv, b)[r->slot] = q;
    return WD_OK;
}

int64_t item_pairs(const Request* r) { return (int64_t)r->plan.tiles_per_chunk * WD_TILE * WD_NPB; }

// Fill table b for launch `seq`: round-robin shares of the pair budget over
// the admitted queries, queries with the largest items first; one contiguous
// range per query and kernel form (a per-node query's run of items may cross
// from its plain items into its extended-precision ones). Lock held.
int64_t build_launch(wd_server* sv, int b, int64_t seq, double* pairs_out)
{
    ServeTable* head = table_head(sv, b);
    ServeRange* ranges = table_ranges(sv, b);
    std::vector<Request*> act;
    for (Request* r : sv->slots)
        if (r && !r->cancel && r->next_item < r->n_items) act.push_back(r);
    std::stable_sort(act.begin(), act.end(), [](const Request* x, const Request* y) {
        return item_pairs(x) > item_pairs(y);
    });
    std::vector<int64_t> take(act.size(), 0);
    double pairs = 0.0;
    bool progress = true;
    while (progress && pairs < (double)sv->cfg.pairs_per_launch) {
        progress = false;
        for (size_t i = 0; i < act.size() && pairs < (double)sv->cfg.pairs_per_launch; ++i) {
            const int64_t left = act[i]->n_items - act[i]->next_item - take[i];
            if (left <= 0) continue;
            const int64_t k = left < kRoundItems ? left : kRoundItems;
            take[i] += k;
            pairs += (double)k * (double)item_pairs(act[i]);
            progress = true;
        }
    }
    int n_rg[SERVE_FORMS] = {0, 0, 0, 0};
    int64_t n_it[SERVE_FORMS] = {0, 0, 0, 0};
    auto add_range = [&](int f, int slot, int64_t first, int64_t count) {
        ServeRange& g = ranges[f * WD_SERVE_RANGES + n_rg[f]++];
        g.req = slot;
        g.count = (int)count;
        g.first = first;
        g.start = n_it[f];
        n_it[f] += count;
    };
    for (size_t i = 0; i < act.size(); ++i) {
        if (take[i] == 0) continue;
        Request* r = act[i];
        const int64_t a = r->next_item, e = r->next_item + take[i];
        if (r->plan.radial) {
            add_range(SERVE_RADIAL, r->slot, a, e - a);
        } else {
            const int64_t m = r->plan.n_items;  // plain items [0, m), then the precise ones
            if (a < m) add_range(r->plan.lattice ? SERVE_LATTICE : SERVE_NODE, r->slot, a, std::min(e, m) - a);
            if (e > m) add_range(SERVE_PRECISE, r->slot, std::max(a, m) - m, e - std::max(a, m));
        }
        r->next_item = e;
        r->last_seq = seq;
        if (r->next_item == r->n_items) r->finish_seq = seq;
    }
    for (int f = 0; f < SERVE_FORMS; ++f) {
        head->n_ranges[f] = n_rg[f];
        head->n_items[f] = n_it[f];
        head->next[f] = 0;
    }
    *pairs_out = pairs;
    return n_it[0] + n_it[1] + n_it[2] + n_it[3];
}

// Retire launch `seq` (complete on the device): deliver the queries it
// finished and free cancelled queries with no work left in flight. Lock held.
void retire_launch(wd_server* sv, int64_t seq)
{
    const int b = (int)(seq % kBuffers);
    bool any = false;
    for (Request* r : sv->slots) {
        if (!r) continue;
        if (r->finish_seq == seq) {
            const double d = sv->h_results[b][r->slot];
            sv->st.pairs += (double)r->plan.n_tris * (double)r->plan.n_nodes;
            release_slot(sv, r);
            finish(sv, r, r->cancel ? WD_ECANCELLED : WD_OK, d);
            any = true;
        } else if (r->cancel && r->last_seq <= seq) {
            release_slot(sv, r);
            finish(sv, r, WD_ECANCELLED, 0.0);
            any = true;
        }
    }
    if (any) sv->cv_done.notify_all();
}

// after a CUDA error of the worker (its text is this thread's last error)
void fail_all(wd_server* sv, wd_status status)
{
    sv->fatal = status;
    sv->fatal_msg = wd_last_error(nullptr);
    for (Request*& r : sv->slots)
        if (r) {
            Request* q = r;
            q->why = sv->fatal_msg;
            release_slot(sv, q);
            finish(sv, q, status, 0.0);
        }
    sv->cv_done.notify_all();
}

void worker_main(wd_server* sv)
{
    cudaSetDevice(sv->ctx->device);
    std::vector<Request*> to_stage;
    int64_t seq = 0;        // launches issued
    int64_t retired = 0;    // launches retired (all below are complete)
    for (;;) {
        to_stage.clear();
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            for (;;) {
                const auto now = Clock::now();
                // expire queued requests past their admission deadline
                if (sv->cfg.timeout_ms > 0)
                    for (auto it = sv->pending.begin(); it != sv->pending.end();) {
                        if (now - (*it)->t_submit > std::chrono::milliseconds(sv->cfg.timeout_ms)) {
                            finish(sv, *it, WD_ETIMEOUT, 0.0);
                            it = sv->pending.erase(it);
                        } else {
                            ++it;
                        }
                    }
                // drop cancelled requests that are queued
                for (auto it = sv->pending.begin(); it != sv->pending.end();) {
                    if ((*it)->cancel) {
                        finish(sv, *it, WD_ECANCELLED, 0.0);
                        it = sv->pending.erase(it);
                    } else {
                        ++it;
                    }
                }
                // cancelled admitted requests with nothing in flight
                for (Request* r : sv->slots)
                    if (r && r->cancel && r->last_seq < retired) {
                        release_slot(sv, r);
                        finish(sv, r, WD_ECANCELLED, 0.0);
                        sv->cv_done.notify_all();
                    }
                // admit in arrival order while a slot and arena space are free
                while (!sv->pending.empty()) {
                    Request* r = sv->pending.front();
                    int slot = -1;
                    for (int i = 0; i < sv->cfg.max_slots; ++i)
                        if (!sv->slots[i]) {
                            slot = i;
                            break;
                        }
                    if (slot < 0) break;
                    const size_t need = request_layout(sv, r).end;
                    size_t off = 0;
                    if (!sv->arena.alloc(need, &off)) break;
                    r->off = off;
                    r->bytes = need;
                    r->slot = slot;
                    r->state = ADMITTED;
                    sv->slots[slot] = r;
                    sv->pending.pop_front();
                    sv->st.admitted++;
                    to_stage.push_back(r);
                }
                bool work = !to_stage.empty() || seq > retired;
                for (Request* r : sv->slots) work = work || r != nullptr;
                if (work) break;
                if (sv->stopping) return;
                sv->cv_work.wait_for(lk, std::chrono::milliseconds(sv->cfg.timeout_ms > 0 ? 1 : 20));
            }
        }
        // stage newly admitted requests (outside the lock; stream-ordered
        // before the next launch)
        for (Request* r : to_stage) {
            wd_status st = stage_request(sv, r);
            if (st != WD_OK) {
                std::lock_guard<std::mutex> lk(sv->mu);
                r->why = wd_last_error(nullptr);
                release_slot(sv, r);
                finish(sv, r, st, 0.0);
                sv->cv_done.notify_all();
            }
        }
        // build and enqueue launch `seq` into the buffer of launch seq - 2,
        // which is retired (at most kBuffers launches are in flight)
        int64_t n_items = 0;
        double pairs = 0.0;
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            if (seq - retired < kBuffers) n_items = build_launch(sv, (int)(seq % kBuffers), seq, &pairs);
        }
        if (n_items > 0) {
            WdRange nvtx_range("wd_serve launch");
            const int b = (int)(seq % kBuffers);
            cudaError_t e = cudaEventRecord(sv->ev_start[b], sv->stream);
            if (e == cudaSuccess) e = cudaGraphLaunch(sv->graph[b], sv->stream);
            if (e == cudaSuccess) e = cudaEventRecord(sv->ev_end[b], sv->stream);
            std::lock_guard<std::mutex> lk(sv->mu);
            if (e != cudaSuccess) {
                fail_all(sv, wd_cuda_status(e, "serve launch"));
                return;
            }
            sv->ctx->launches += sv->kernels_per_launch;
            sv->st.launches++;
            ++seq;
        }
        // retire the oldest launch once the next one is queued behind it (or
        // when nothing else can be queued)
        if (seq > retired && (seq - retired >= kBuffers || n_items == 0)) {
            const int b = (int)(retired % kBuffers);
            const cudaError_t e = cudaEventSynchronize(sv->ev_end[b]);
            float ms = 0.0f;
            if (e == cudaSuccess && cudaEventElapsedTime(&ms, sv->ev_start[b], sv->ev_end[b]) != cudaSuccess) {
                cudaGetLastError();  // no timing for this launch; the work itself completed
                ms = 0.0f;
            }
            std::lock_guard<std::mutex> lk(sv->mu);
            if (e != cudaSuccess) {
                fail_all(sv, wd_cuda_status(e, "serve launch"));
                return;
            }
            sv->busy_s += 1e-3 * ms;
            retire_launch(sv, retired);
            ++retired;
        }
    }
}

}  // namespace

// ------------------------------------------------------------------ C ABI
extern "C" wd_status wd_serve_start(wd_ctx* ctx, const wd_serve_config* cfg, wd_server** out)
{
    WD_CHECK(ctx && cfg && out, WD_EINVAL, "null argument");
    WD_CHECK(cfg->precision == WD_FP64 || cfg->precision == WD_MIXED, WD_EINVAL, "bad precision");
    WD_CHECK(cfg->max_slots >= 1 && cfg->max_slots <= kMaxSlots, WD_EINVAL, "max_slots out of range");
    WD_CHECK(cfg->mem_cap_bytes > 0 && cfg->pairs_per_launch > 0 && cfg->max_pending >= 1, WD_EINVAL,
             "memory cap, pending limit and launch budget must be > 0");
    WD_CHECK(cfg->n_rules >= 1 && cfg->n_rules <= 4, WD_EINVAL, "n_rules must be 1..4");
    wd_status st = wd_activate(ctx);
    if (st != WD_OK) return st;
    wd_server* sv = new wd_server();
    sv->ctx = ctx;
    sv->cfg = *cfg;
    sv->slots.assign(cfg->max_slots, nullptr);
    auto release_all = [](wd_server* v) {
        for (int b = 0; b < kBuffers; ++b) {
            if (v->graph[b]) cudaGraphExecDestroy(v->graph[b]);
            if (v->ev_start[b]) cudaEventDestroy(v->ev_start[b]);
            if (v->ev_end[b]) cudaEventDestroy(v->ev_end[b]);
            cudaFree(v->d_table[b]);
            cudaFreeHost(v->h_table[b]);
            cudaFreeHost(v->h_results[b]);
        }
        if (v->stream) cudaStreamDestroy(v->stream);
        cudaFree(v->d_arena);
        cudaFree(v->d_results);
    };
    auto fail = [&](wd_status s) {
        release_all(sv);
        delete sv;
        return s;
    };
    for (int i = 0; i < cfg->n_rules; ++i) {
        RuleEntry re;
        st = wd_build_freq_rule(ctx, &cfg->rules[i], &re.rule);
        if (st != WD_OK) return fail(st);
        const double c0[3] = {0.0, 0.0, 0.0};
        st = wd_rule_sphere(ctx, re.rule, 1.0, c0, &re.nu, nullptr);
        if (st != WD_OK) return fail(st);
        sv->rules.push_back(re);
    }
    if (cudaStreamCreateWithFlags(&sv->stream, cudaStreamNonBlocking) != cudaSuccess)
        return fail(wd_cuda_status(cudaGetLastError(), "cudaStreamCreate"));
    if (wd_dev_alloc(&sv->d_arena, (size_t)cfg->mem_cap_bytes, "serving arena") != cudaSuccess) {
        cudaGetLastError();
        wd_set_error("cannot allocate the serving arena");
        return fail(WD_ENOMEM);
    }
    sv->arena.init(sv->d_arena, (size_t)cfg->mem_cap_bytes);
    sv->off_ranges = align_up(sizeof(ServeTable));
    sv->off_reqs = sv->off_ranges + align_up(sizeof(ServeRange) * SERVE_FORMS * WD_SERVE_RANGES);
    sv->table_bytes = sv->off_reqs + align_up(sizeof(ServeReq) * kMaxSlots);
    bool ok = wd_dev_alloc(&sv->d_results, sizeof(double) * kMaxSlots, "serving results") == cudaSuccess;
    for (int b = 0; ok && b < kBuffers; ++b)
        ok = cudaHostAlloc(&sv->h_table[b], sv->table_bytes, cudaHostAllocDefault) == cudaSuccess &&
             cudaHostAlloc(&sv->h_results[b], sizeof(double) * kMaxSlots, cudaHostAllocDefault) == cudaSuccess &&
             wd_dev_alloc(&sv->d_table[b], sv->table_bytes, "serving table") == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        wd_set_error("cannot allocate the serving tables");
        return fail(WD_ENOMEM);
    }
    for (int b = 0; b < kBuffers; ++b) {
        std::memset(sv->h_table[b], 0, sv->table_bytes);
        if (cudaEventCreate(&sv->ev_start[b]) != cudaSuccess || cudaEventCreate(&sv->ev_end[b]) != cudaSuccess)
            return fail(wd_cuda_status(cudaGetLastError(), "cudaEventCreate"));
    }
    // occupancy queries before the capture (they are cached per context)
    for (int f = 0; f < SERVE_FORMS; ++f) wd_serve_resident(ctx, cfg->precision, f);
    for (int b = 0; b < kBuffers; ++b)
        if ((st = capture_graph(sv, b)) != WD_OK) return fail(st);
    sv->drop_nth = wd_fault_drop_completion();
    wd_log(3, "server started: %d slots, arena %lld bytes, %d rules, %d kernels per launch", cfg->max_slots,
           (long long)cfg->mem_cap_bytes, cfg->n_rules, sv->kernels_per_launch);
    sv->worker = std::thread(worker_main, sv);
    *out = sv;
    return WD_OK;
}

extern "C" wd_status wd_serve_submit(wd_server* sv, const wd_mesh* m, double s, double R, uint64_t* ticket)
{
    WD_CHECK(sv && m && ticket, WD_EINVAL, "null argument");
    WD_CHECK(std::isfinite(s) && s > 0.0, WD_EINVAL, "s must be finite and > 0");
    WD_CHECK(m->n_verts >= 0 && m->n_tris >= 0 && (m->n_verts == 0 || m->verts) && (m->n_tris == 0 || m->tris),
             WD_EINVAL, "bad mesh");
    int rule = -1;
    for (int i = 0; i < sv->cfg.n_rules; ++i)
        if (sv->cfg.rules[i].R == R) rule = i;
    WD_CHECK(rule >= 0, WD_EINVAL, "no serving rule with this truncation radius R");
    for (int64_t i = 0; i < 3 * m->n_tris; ++i)
        WD_CHECK(m->tris[i] >= 0 && m->tris[i] < m->n_verts, WD_EINVAL, "triangle index out of range");
    for (int64_t i = 0; i < 3 * m->n_verts; ++i)
        WD_CHECK(std::isfinite(m->verts[i]), WD_EINVAL, "non-finite vertex coordinate");
    Request* r = new Request();
    r->verts.assign(m->verts, m->verts + 3 * m->n_verts);
    r->tris.assign(m->tris, m->tris + 3 * m->n_tris);
    r->s = s;
    r->rule = rule;
    {
        // the plan of this query's own wd_distance launch, items capped in size
        wd_rule* ru = sv->rules[rule].rule;
        wd_status pst = wd_plan_pair_serve(sv->ctx, ru, sv->cfg.precision, m->n_tris, kMaxItemTiles, &r->plan);
        if (pst == WD_OK && sv->cfg.precision == WD_MIXED && !r->plan.radial) {
            // the extended-precision blocks of wd_distance's per-node plan
            pst = wd_rule_precise(sv->ctx, ru, s, &r->precise);
            if (pst == WD_OK && r->precise->n == 0) r->precise = nullptr;
            if (pst == WD_OK && r->precise) r->pplan = wd_precise_plan(sv->ctx, r->plan, r->precise->n, MODE_DIST);
        }
        if (pst != WD_OK) {
            delete r;
            return pst;
        }
        r->n_items = r->plan.n_items + (r->precise ? r->pplan.n_items : 0);
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->fatal != WD_OK) {
        delete r;
        wd_set_error("the serving loop stopped after a CUDA error: " + sv->fatal_msg);
        return sv->fatal;
    }
    if ((int)sv->pending.size() >= sv->cfg.max_pending) {
        sv->st.rejected++;
        delete r;
        wd_set_error("serving queue full");
        return WD_EBUSY;
    }
    if (request_layout(sv, r).end > (size_t)sv->cfg.mem_cap_bytes) {
        sv->st.rejected++;
        delete r;
        wd_set_error("query larger than the serving memory cap");
        return WD_ENOMEM;
    }
    r->ticket = sv->next_ticket++;
    r->t_submit = Clock::now();
    if (!sv->any_submit) {
        sv->any_submit = true;
        sv->t_first_submit = r->t_submit;
    }
    sv->st.submitted++;
    sv->all[r->ticket] = r;
    sv->pending.push_back(r);
    *ticket = r->ticket;
    sv->cv_work.notify_one();
    return WD_OK;
}

extern "C" wd_status wd_serve_poll(wd_server* sv, uint64_t ticket, int* done, double* dist2, wd_status* req_status)
{
    WD_CHECK(sv && done, WD_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    WD_CHECK(it != sv->all.end(), WD_ENOTFOUND, "unknown ticket");
    Request* r = it->second;
    *done = (r->state == DONE || r->state == FAILED) ? 1 : 0;
    if (*done && dist2) *dist2 = r->result;
    if (req_status) *req_status = *done ? r->status : WD_OK;
    return WD_OK;
}

extern "C" wd_status wd_serve_wait(wd_server* sv, uint64_t ticket, int timeout_ms, double* dist2)
{
    WD_CHECK(sv, WD_EINVAL, "null server");
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    WD_CHECK(it != sv->all.end(), WD_ENOTFOUND, "unknown ticket");
    Request* r = it->second;
    const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms > 0 ? timeout_ms : 0);
    while (r->state != DONE && r->state != FAILED) {
        if (sv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && r->state != DONE &&
            r->state != FAILED) {
            wd_set_error("timed out waiting for the query");
            return WD_ETIMEOUT;
        }
    }
    if (r->state == FAILED) {
        wd_set_error("query failed: " + r->why);
        return r->status;
    }
    if (dist2) *dist2 = r->result;
    return WD_OK;
}

extern "C" wd_status wd_serve_cancel(wd_server* sv, uint64_t ticket)
{
    WD_CHECK(sv, WD_EINVAL, "null server");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    WD_CHECK(it != sv->all.end(), WD_ENOTFOUND, "unknown ticket");
    it->second->cancel = true;
    sv->cv_work.notify_one();
    return WD_OK;
}

extern "C" wd_status wd_serve_stats(wd_server* sv, wd_serve_stats_t* out)
{
    WD_CHECK(sv && out, WD_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    *out = sv->st;
    std::vector<double> l = sv->lat_us;
    std::sort(l.begin(), l.end());
    if (!l.empty()) {
        out->p50_us = l[l.size() / 2];
        out->p99_us = l[std::min(l.size() - 1, (size_t)(0.99 * l.size()))];
        out->max_us = l.back();
        double sum = 0.0;
        for (double x : l) sum += x;
        out->mean_us = sum / l.size();
    }
    const double span = std::chrono::duration<double>(sv->t_last_done - sv->t_first_submit).count();
    out->qps = (span > 0.0) ? sv->st.completed / span : 0.0;
    out->gpu_busy = (span > 0.0) ? std::min(1.0, sv->busy_s / span) : 0.0;
    out->pending = (int64_t)sv->pending.size();
    int act = 0;
    for (Request* r : sv->slots) act += r != nullptr;
    out->active = act;
    out->arena_used_bytes = (int64_t)sv->arena.used;
    return WD_OK;
}

extern "C" wd_status wd_serve_stop(wd_server* sv)
{
    if (!sv) return WD_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stopping = true;
        // queued requests are cancelled; admitted ones drain
        for (Request* r : sv->pending) finish(sv, r, WD_ECANCELLED, 0.0);
        sv->pending.clear();
        sv->cv_work.notify_all();
        sv->cv_done.notify_all();
    }
    if (sv->worker.joinable()) sv->worker.join();
    cudaSetDevice(sv->ctx->device);
    cudaStreamSynchronize(sv->stream);
    for (int b = 0; b < kBuffers; ++b) {
        if (sv->graph[b]) cudaGraphExecDestroy(sv->graph[b]);
        if (sv->ev_start[b]) cudaEventDestroy(sv->ev_start[b]);
        if (sv->ev_end[b]) cudaEventDestroy(sv->ev_end[b]);
        cudaFree(sv->d_table[b]);
        cudaFreeHost(sv->h_table[b]);
        cudaFreeHost(sv->h_results[b]);
    }
    cudaStreamDestroy(sv->stream);
    cudaFree(sv->d_arena);
    cudaFree(sv->d_results);
    for (auto& kv : sv->all) delete kv.second;
    const wd_status fatal = sv->fatal;
    if (fatal != WD_OK) wd_set_error("the serving loop had stopped after a CUDA error: " + sv->fatal_msg);
    delete sv;
    return fatal;
}
