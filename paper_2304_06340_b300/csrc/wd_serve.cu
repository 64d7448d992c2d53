// Serving loop: continuous batching of distance queries on one GPU.
//
// submit() copies a query (mesh, s, R) into host memory and queues it. A worker
// thread admits queued queries while request slots and device memory (a fixed
// arena, first-fit) are free, stages their meshes, and then repeatedly replays
// one captured CUDA graph: copy the descriptor table from pinned memory, run
// the batched pair kernel over a budget of (request, node block) items drawn
// round-robin from every admitted query, sum the blocks of the queries that
// finished, and copy their results back. Queries that arrive while a launch is
// running join the next one, so short and long queries share the device and a
// long query never holds back the short ones. The frequency rules, their
// weights and the sphere's transform stay resident on the device.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "wd_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

constexpr int kMaxSlots = WD_SERVE_MAX_SLOTS;
constexpr int kMaxItems = 1 << 17;
constexpr int kRoundRobinBlocks = 8;  // node blocks taken per request per round

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
    // device side
    size_t off = 0, bytes = 0;
    int slot = -1;
    int n_nb = 0, next_nb = 0;
    bool staged = false;
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
    // descriptor table: pinned host copy and device copy with the same layout
    size_t table_bytes = 0, off_reqs = 0, off_items = 0, off_fin = 0;
    char* h_table = nullptr;
    char* d_table = nullptr;
    double* h_results = nullptr;
    double* d_results = nullptr;
    cudaGraphExec_t graph = nullptr;
    int grid = 0;
    // statistics
    wd_serve_stats_t st{};
    std::vector<double> lat_us;
    Clock::time_point t_first_submit{}, t_last_done{};
    bool any_submit = false;
    double busy_s = 0.0;
    wd_status fatal = WD_OK;
    int drop_nth = 0;        // WD_FAULT_DROP_COMPLETION at start (0: off)
    int64_t n_ok_seen = 0;   // successful completions so far
};

namespace {

size_t request_bytes(const wd_server* sv, const Request* r)
{
    const int64_t T = (int64_t)r->tris.size() / 3;
    const int64_t V = (int64_t)r->verts.size() / 3;
    return align_up(wd_tri_record_bytes(sv->cfg.precision) * (size_t)(T > 0 ? T : 1)) +
           align_up(sizeof(double) * (size_t)(r->n_nb > 0 ? r->n_nb : 1)) +
           align_up(sizeof(double) * 3 * (size_t)(V > 0 ? V : 1)) + align_up(sizeof(int32_t) * 3 * (size_t)(T > 0 ? T : 1));
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

wd_status capture_graph(wd_server* sv)
{
    cudaStream_t s = sv->stream;
    const ServeTable* d_head = reinterpret_cast<const ServeTable*>(sv->d_table);
    const ServeReq* d_reqs = reinterpret_cast<const ServeReq*>(sv->d_table + sv->off_reqs);
    const ServeItem* d_items = reinterpret_cast<const ServeItem*>(sv->d_table + sv->off_items);
    const ServeFin* d_fin = reinterpret_cast<const ServeFin*>(sv->d_table + sv->off_fin);
    WD_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaMemcpyAsync(sv->d_table, sv->h_table, sv->table_bytes, cudaMemcpyHostToDevice, s);
    wd_status st = WD_OK;
    if (e == cudaSuccess)
        st = wd_launch_serve(sv->ctx, sv->cfg.precision, sv->grid, d_head, d_reqs, d_items, d_fin, sv->d_results, s);
    if (e == cudaSuccess && st == WD_OK)
        e = cudaMemcpyAsync(sv->h_results, sv->d_results, sizeof(double) * kMaxSlots, cudaMemcpyDeviceToHost, s);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(s, &g);
    if (e != cudaSuccess) return wd_cuda_status(e, "serve graph capture");
    if (st != WD_OK) return st;
    if (e2 != cudaSuccess) return wd_cuda_status(e2, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&sv->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return wd_cuda_status(e, "cudaGraphInstantiate");
    return WD_OK;
}

// Stage one admitted request: copy its mesh and build its triangle records.
wd_status stage_request(wd_server* sv, Request* r)
{
    const int64_t T = (int64_t)r->tris.size() / 3;
    const int64_t V = (int64_t)r->verts.size() / 3;
    char* base = sv->d_arena + r->off;
    const size_t o_rec = 0;
    const size_t o_bd = o_rec + align_up(wd_tri_record_bytes(sv->cfg.precision) * (size_t)(T > 0 ? T : 1));
    const size_t o_v = o_bd + align_up(sizeof(double) * (size_t)(r->n_nb > 0 ? r->n_nb : 1));
    const size_t o_t = o_v + align_up(sizeof(double) * 3 * (size_t)(V > 0 ? V : 1));
    if (V > 0)
        WD_CUDA(cudaMemcpyAsync(base + o_v, r->verts.data(), sizeof(double) * 3 * V, cudaMemcpyHostToDevice,
                                sv->stream));
    if (T > 0)
        WD_CUDA(cudaMemcpyAsync(base + o_t, r->tris.data(), sizeof(int32_t) * 3 * T, cudaMemcpyHostToDevice,
                                sv->stream));
    wd_status st = wd_launch_stage(sv->ctx, sv->cfg.precision, reinterpret_cast<const double*>(base + o_v), V,
                                   reinterpret_cast<const int32_t*>(base + o_t), T, 1.0, base + o_rec, 0, sv->stream);
    if (st != WD_OK) return st;
    RuleEntry& re = sv->rules[r->rule];
    if (!re.W.count(r->s)) {
        const double* w = nullptr;
        if ((st = wd_rule_weights(sv->ctx, re.rule, r->s, &w, sv->stream)) != WD_OK) return st;
        re.W[r->s] = w;
    }
    r->staged = true;
    return WD_OK;
}

void worker_main(wd_server* sv)
{
    cudaSetDevice(sv->ctx->device);
    ServeTable* head = reinterpret_cast<ServeTable*>(sv->h_table);
    ServeReq* reqs = reinterpret_cast<ServeReq*>(sv->h_table + sv->off_reqs);
    ServeItem* items = reinterpret_cast<ServeItem*>(sv->h_table + sv->off_items);
    ServeFin* fin = reinterpret_cast<ServeFin*>(sv->h_table + sv->off_fin);
    std::vector<Request*> to_stage;
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
                    const size_t need = request_bytes(sv, r);
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
                bool active = false;
                for (Request* r : sv->slots) active = active || r != nullptr;
                if (active || !to_stage.empty()) break;
                if (sv->stopping) return;
                sv->cv_work.wait_for(lk, std::chrono::milliseconds(sv->cfg.timeout_ms > 0 ? 1 : 20));
            }
        }
        // stage newly admitted requests (outside the lock)
        for (Request* r : to_stage) {
            wd_status st = stage_request(sv, r);
            if (st != WD_OK) {
                std::lock_guard<std::mutex> lk(sv->mu);
                release_slot(sv, r);
                finish(sv, r, st, 0.0);
                sv->cv_done.notify_all();
            }
        }
        // build the launch: round-robin node blocks of every admitted request
        std::vector<Request*> finishing;
        int n_items = 0;
        double pairs = 0.0;
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            for (int i = 0; i < sv->cfg.max_slots; ++i) {
                Request* r = sv->slots[i];
                if (r && r->cancel) {
                    release_slot(sv, r);
                    finish(sv, r, WD_ECANCELLED, 0.0);
                    sv->cv_done.notify_all();
                    r = nullptr;
                }
                if (!r) continue;
                RuleEntry& re = sv->rules[r->rule];
                char* base = sv->d_arena + r->off;
                const int64_t T = (int64_t)r->tris.size() / 3;
                ServeReq q;
                q.rec = base;
                q.T = T;
                q.xi = re.rule->d_xi;
                q.n = re.rule->n_eval;
                const bool radial = sv->cfg.precision == WD_MIXED && re.rule->d_rad;
                q.rad = radial ? re.rule->d_rad : nullptr;
                q.dir = radial ? re.rule->d_dir : nullptr;
                q.n_rad = re.rule->n_rad;
                q.n_rg = (re.rule->n_rad + WD_RAD_NR - 1) / WD_RAD_NR;
                q.n_dir = re.rule->n_dir;
                q.W = re.W[r->s];
                q.nu = re.nu;
                q.blockD = reinterpret_cast<double*>(
                    base + align_up(wd_tri_record_bytes(sv->cfg.precision) * (size_t)(T > 0 ? T : 1)));
                reqs[i] = q;
            }
            bool progress = true;
            while (progress && n_items < kMaxItems && pairs < (double)sv->cfg.pairs_per_launch) {
                progress = false;
                for (int i = 0; i < sv->cfg.max_slots && n_items < kMaxItems; ++i) {
                    Request* r = sv->slots[i];
                    if (!r || r->next_nb >= r->n_nb) continue;
                    const int64_t T = reqs[i].T;
                    for (int b = 0; b < kRoundRobinBlocks && r->next_nb < r->n_nb && n_items < kMaxItems; ++b) {
                        items[n_items].req = i;
                        items[n_items].nb = r->next_nb++;
                        n_items++;
                        pairs += (double)T * WD_NPB;
                    }
                    if (r->next_nb >= r->n_nb) finishing.push_back(r);
                    progress = true;
                }
            }
            head->n_items = n_items;
            head->n_fin = (int)finishing.size();
            for (size_t f = 0; f < finishing.size(); ++f) {
                fin[f].req = finishing[f]->slot;
                fin[f].n_nb = finishing[f]->n_nb;
                fin[f].out = finishing[f]->slot;
            }
        }
        if (n_items == 0 && finishing.empty()) continue;
        const auto t0 = Clock::now();
        WdRange nvtx_range("wd_serve launch");
        cudaError_t e = cudaGraphLaunch(sv->graph, sv->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(sv->stream);
        const auto t1 = Clock::now();
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->busy_s += std::chrono::duration<double>(t1 - t0).count();
        sv->st.launches++;
        sv->st.pairs += pairs;
        if (e != cudaSuccess) {
            wd_cuda_status(e, "serve launch");
            sv->fatal = WD_ECUDA;
            for (Request*& r : sv->slots)
                if (r) {
                    Request* q = r;
                    release_slot(sv, q);
                    finish(sv, q, WD_ECUDA, 0.0);
                }
            sv->cv_done.notify_all();
            return;
        }
        for (Request* r : finishing) {
            const double d = sv->h_results[r->slot];
            release_slot(sv, r);
            finish(sv, r, r->cancel ? WD_ECANCELLED : WD_OK, d);
        }
        if (!finishing.empty()) sv->cv_done.notify_all();
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
    auto fail = [&](wd_status s) {
        if (sv->graph) cudaGraphExecDestroy(sv->graph);
        if (sv->stream) cudaStreamDestroy(sv->stream);
        cudaFree(sv->d_arena);
        cudaFree(sv->d_table);
        cudaFree(sv->d_results);
        cudaFreeHost(sv->h_table);
        cudaFreeHost(sv->h_results);
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
    sv->off_reqs = align_up(sizeof(ServeTable));
    sv->off_items = sv->off_reqs + align_up(sizeof(ServeReq) * kMaxSlots);
    sv->off_fin = sv->off_items + align_up(sizeof(ServeItem) * kMaxItems);
    sv->table_bytes = sv->off_fin + align_up(sizeof(ServeFin) * kMaxSlots);
    if (cudaHostAlloc(&sv->h_table, sv->table_bytes, cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc(&sv->h_results, sizeof(double) * kMaxSlots, cudaHostAllocDefault) != cudaSuccess ||
        wd_dev_alloc(&sv->d_table, sv->table_bytes, "serving table") != cudaSuccess ||
        wd_dev_alloc(&sv->d_results, sizeof(double) * kMaxSlots, "serving results") != cudaSuccess) {
        cudaGetLastError();
        wd_set_error("cannot allocate the serving tables");
        return fail(WD_ENOMEM);
    }
    std::memset(sv->h_table, 0, sv->table_bytes);
    sv->grid = wd_serve_resident(ctx, cfg->precision);
    if ((st = capture_graph(sv)) != WD_OK) return fail(st);
    sv->drop_nth = wd_fault_drop_completion();
    wd_log(3, "server started: %d slots, arena %lld bytes, %d rules, grid %d", cfg->max_slots,
           (long long)cfg->mem_cap_bytes, cfg->n_rules, sv->grid);
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
        // node blocks: radius x direction blocks for ball rules in the mixed path
        const wd_rule* ru = sv->rules[rule].rule;
        if (sv->cfg.precision == WD_MIXED && ru->d_rad)
            r->n_nb = (int)(((ru->n_dir + WD_RAD_ND - 1) / WD_RAD_ND) * ((ru->n_rad + WD_RAD_NR - 1) / WD_RAD_NR));
        else
            r->n_nb = (int)((ru->n_eval + WD_NPB - 1) / WD_NPB);
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->fatal != WD_OK) {
        delete r;
        wd_set_error("the serving loop stopped after a CUDA error");
        return sv->fatal;
    }
    if ((int)sv->pending.size() >= sv->cfg.max_pending) {
        sv->st.rejected++;
        delete r;
        wd_set_error("serving queue full");
        return WD_EBUSY;
    }
    if (request_bytes(sv, r) > (size_t)sv->cfg.mem_cap_bytes) {
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
        wd_set_error("query failed");
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
    if (sv->graph) cudaGraphExecDestroy(sv->graph);
    cudaStreamDestroy(sv->stream);
    cudaFree(sv->d_arena);
    cudaFree(sv->d_table);
    cudaFree(sv->d_results);
    cudaFreeHost(sv->h_table);
    cudaFreeHost(sv->h_results);
    for (auto& kv : sv->all) delete kv.second;
    const wd_status fatal = sv->fatal;
    delete sv;
    return fatal;
}
