// Continuous-batching server for streams of WCSP / DCOP instances.
//
// Planning: srv_submit copies the problem and queues it; a pool of planner
// threads computes each plan (ordering, buckets, work decomposition; no GPU
// work), so the caller's thread is not held by host planning and plans of
// many requests are computed in parallel.  A plan's device need (its arena
// size, from the separator sizes, i.e. the induced width) is known before
// anything is allocated; a request that can never fit the budget fails with
// GPUBE_ENOMEM (srv_result).
//
// Admission: planned requests are admitted in submission order while a slot
// is free and a first-fit allocator finds room for them in the server's
// memory budget; their tables stay resident until they finish.  While no
// request waits for memory, a planner thread that finds room for its request
// also binds it (descriptors, uploads on the thread's own stream), so the
// serving thread only merges launches and retires results.
//
// Batching: each server step merges, for every admitted request, the tasks
// of its next elimination-tree level into ONE persistent UTIL launch (the
// same kernel and device work queue as a single instance's batched level).
// A request admitted while others are running joins the next launch, so the
// work of requests of different sizes overlaps on the device.  A request
// whose last level has run gets its VALUE kernel and an asynchronous copy of
// its result; it is retired (memory returned) once that copy has landed.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "gpube_internal.h"

using namespace gpube;

namespace {

#define SRV_TRY(call)                                           \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_error(e_, #call);    \
    } while (0)

size_t al(size_t x, size_t a) { return (x + a - 1) / a * a; }

// First-fit allocator over [0, size) with coalescing on free.
struct FirstFit {
    std::map<size_t, size_t> free_blocks;  // offset -> bytes
    size_t used = 0, peak = 0;
    void init(size_t size)
    {
        free_blocks.clear();
        if (size) free_blocks[0] = size;
        used = peak = 0;
    }
    bool alloc(size_t bytes, size_t *off)
    {
        bytes = al(bytes, 256);
        for (auto it = free_blocks.begin(); it != free_blocks.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, at = it->first + bytes;
                free_blocks.erase(it);
                if (rest) free_blocks[at] = rest;
                used += bytes;
                peak = std::max(peak, used);
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = al(bytes, 256);
        used -= bytes;
        auto it = free_blocks.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_blocks.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_blocks.erase(nx);
        }
        if (it != free_blocks.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_blocks.erase(it);
            }
        }
    }
};

enum { kQueued = 0, kActive = 1, kValue = 2, kDone = 3, kFailed = 4, kPlanning = 5 };

struct Request {
    int64_t id = 0;
    // the submission: a reference to the problem, copies of the arrays (the
    // caller may free its own right after submit)
    wcsp *prob = nullptr;
    int32_t kind = 0, i_bound = 0;
    solve_opts opts{};
    std::vector<int32_t> parent, order, opt_parent, ev_vars;
    std::string err;  // planning failure message
    util_state *st = nullptr;
    size_t off = 0, bytes = 0;
    int slot = -1, next_level = 0, state = kQueued, rc = 0;
    bool bound = false;  // admitted and bound by a planner thread
    double t_submit = 0, t_admit = 0, t_done = 0;
    cudaEvent_t up_ev = nullptr, done_ev = nullptr;
    bool up_waited = false;
    std::vector<int32_t> sigma;
    solve_result res{};
};

}  // namespace

struct gpube_server {
    size_t budget = 0;
    int max_slots = 1;
    unsigned char *base = nullptr;
    bool owns = false;
    cudaStream_t stream = nullptr, up_stream = nullptr;
    FirstFit alloc;
    std::deque<Request *> queue;
    std::map<int64_t, Request *> reqs;
    std::vector<Request *> active;
    std::vector<int> free_slots;
    std::vector<unsigned char *> pinned;   // per slot: status, result, assignment
    std::vector<cudaEvent_t> slot_up, slot_done;  // per slot: upload done, result copied
    std::vector<size_t> pinned_cap;
    int64_t next_id = 0;
    // merged launch descriptors (double buffered)
    unsigned char *dbuf[2] = {nullptr, nullptr};
    unsigned char *hbuf[2] = {nullptr, nullptr};  // pinned host staging of dbuf
    size_t dcap[2] = {0, 0};
    cudaEvent_t dev_ev[2] = {nullptr, nullptr};
    bool dev_used[2] = {false, false};
    int flip = 0;
    int64_t key_turn = 0;  // which group of compatible requests launches next
    // planner pool: submitted requests wait in to_plan; finished plans (or
    // failures) wait in planned until srv_step takes them
    std::vector<std::thread> planners;
    std::mutex pmu;
    std::condition_variable pcv;
    std::deque<Request *> to_plan;
    std::vector<Request *> planned;
    std::vector<std::pair<util_state *, wcsp *>> to_free;  // finished requests' plans and problems
    std::deque<Request *> to_bind;         // admitted (memory and slot reserved), to be bound
    std::vector<cudaStream_t> planner_up;  // per planner thread: its upload stream
    std::mutex amu;                        // guards alloc and free_slots
    std::atomic<int64_t> waiting{0};       // requests queued for memory (planners then leave admission alone)
    int dev = 0;
    bool stopping = false;
    int64_t planning = 0;  // requests submitted and not yet taken by srv_step (guarded by pmu)
    int32_t *work = nullptr;  // [0..1] counters, [2] status
    int num_sms = 0, threads = 256;
    int64_t launches = 0, max_inflight = 0;
    double t0 = 0;
};

// Bind an admitted request (memory offset and slot assigned): its result
// buffer, descriptors and uploads (on stream up), the slot's events.
static int bind_request(gpube_server *s, Request *r, cudaStream_t up)
{
    const size_t need = 24 + 4 * static_cast<size_t>(std::max(r->st->w->n, 1));
    if (s->pinned_cap[r->slot] < need) {  // grown geometrically: rare
        const size_t cap = std::max(need, 2 * s->pinned_cap[r->slot]);
        if (s->pinned[r->slot]) cudaFreeHost(s->pinned[r->slot]);
        s->pinned[r->slot] = nullptr;
        s->pinned_cap[r->slot] = 0;
        SRV_TRY(cudaMallocHost(reinterpret_cast<void **>(&s->pinned[r->slot]), cap));
        s->pinned_cap[r->slot] = cap;
    }
    // uploads go to a side stream so that admission does not wait for the
    // launches in flight; the compute stream waits on them by event
    int rc = util_bind(r->st, s->base + r->off, r->bytes, up);
    if (rc) return rc;
    // the slot's events (created on the slot's first use, reused after)
    if (!s->slot_up[r->slot]) SRV_TRY(cudaEventCreateWithFlags(&s->slot_up[r->slot], cudaEventDisableTiming));
    if (!s->slot_done[r->slot]) SRV_TRY(cudaEventCreateWithFlags(&s->slot_done[r->slot], cudaEventDisableTiming));
    r->up_ev = s->slot_up[r->slot];
    r->done_ev = s->slot_done[r->slot];
    SRV_TRY(cudaEventRecord(r->up_ev, up));
    r->st->stream = s->stream;  // everything after the upload runs on the compute stream
    r->next_level = 0;
    r->t_admit = now_ms() - s->t0;
    return GPUBE_OK;
}

// Memory and a slot for a request, if both are free now.
static bool reserve(gpube_server *s, Request *r)
{
    std::lock_guard<std::mutex> g(s->amu);
    if (s->free_slots.empty()) return false;
    size_t off;
    if (!s->alloc.alloc(r->bytes, &off)) return false;
    r->off = off;
    r->slot = s->free_slots.back();
    s->free_slots.pop_back();
    return true;
}

static void unreserve(gpube_server *s, Request *r)
{
    std::lock_guard<std::mutex> g(s->amu);
    s->alloc.release(r->off, r->bytes);
    s->free_slots.push_back(r->slot);
    r->slot = -1;
}

// Planner thread: plan queued requests until the server stops; bind them
// too when nothing waits for memory and they fit now.
static void planner_loop(gpube_server *s, int idx)
{
    cudaSetDevice(s->dev);
    const cudaStream_t up = s->planner_up[idx];
    for (;;) {
        Request *r = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->pmu);
            s->pcv.wait(lk, [&] {
                return s->stopping || !s->to_plan.empty() || !s->to_free.empty() || !s->to_bind.empty();
            });
            if (!s->to_bind.empty()) {  // admitted by the serving thread: bind it here
                Request *b = s->to_bind.front();
                s->to_bind.pop_front();
                lk.unlock();
                int brc = bind_request(s, b, up);
                if (brc) {
                    cudaStreamSynchronize(up);  // no copy may still land in the released memory
                    unreserve(s, b);
                }
                std::lock_guard<std::mutex> lk2(s->pmu);
                b->rc = brc;
                b->bound = brc == 0;
                if (brc) b->err = last_error();
                s->planned.push_back(b);
                continue;
            }
            if (!s->to_free.empty()) {
                auto f = s->to_free.back();
                s->to_free.pop_back();
                lk.unlock();
                util_state_free(f.first);
                wcsp_unref(f.second);
                continue;
            }
            if (s->to_plan.empty()) return;  // stopping
            r = s->to_plan.front();
            s->to_plan.pop_front();
        }
        util_state *st = nullptr;
        int rc = util_plan(r->prob, r->kind, r->i_bound, r->parent.empty() ? nullptr : r->parent.data(),
                           &r->opts, &st);
        if (!rc && al(st->arena_bytes, 256) > s->budget) {
            rc = set_error(GPUBE_ENOMEM, "request needs %zu bytes, the budget is %zu", st->arena_bytes, s->budget);
            util_state_free(st);
            st = nullptr;
        }
        if (!rc) gpube_prepack(st);  // the tables' device layout, ready for the upload at admission
        r->st = st;
        bool bound = false;
        if (!rc && s->waiting.load() == 0) {
            r->bytes = st->arena_bytes;
            if (reserve(s, r)) {
                rc = bind_request(s, r, up);
                if (rc) {
                    cudaStreamSynchronize(up);  // no copy may still land in the released memory
                    unreserve(s, r);
                } else {
                    bound = true;
                }
            }
        }
        std::lock_guard<std::mutex> lk(s->pmu);
        r->rc = rc;
        r->bound = bound;
        if (rc) r->err = last_error();
        s->planned.push_back(r);
    }
}

extern "C" int srv_create(size_t budget_bytes, int32_t max_slots, void *arena, size_t arena_bytes, void *stream,
                          gpube_server **out)
{
    if (!out || budget_bytes == 0 || max_slots < 1) return set_error(GPUBE_EINVAL, "bad server arguments");
    *out = nullptr;
    int dev = 0;
    SRV_TRY(cudaGetDevice(&dev));
    gpube_server *s = new gpube_server();
    s->budget = budget_bytes;
    s->max_slots = max_slots;
    s->stream = static_cast<cudaStream_t>(stream);
    cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaError_t e0 = kernels_init_device(); e0 != cudaSuccess) {
        delete s;
        return cuda_error(e0, "kernel attributes");
    }
    if (arena) {
        if (arena_bytes < budget_bytes || reinterpret_cast<uintptr_t>(arena) % 256) {
            delete s;
            return set_error(GPUBE_EINVAL, "arena smaller than the budget or not 256-byte aligned");
        }
        s->base = static_cast<unsigned char *>(arena);
    } else {
        void *p = nullptr;
        if (cudaMalloc(&p, budget_bytes) != cudaSuccess) {
            cudaGetLastError();
            delete s;
            return set_error(GPUBE_ENOMEM, "cudaMalloc of the %zu-byte budget failed", budget_bytes);
        }
        s->base = static_cast<unsigned char *>(p);
        s->owns = true;
    }
    s->alloc.init(budget_bytes);
    for (int i = max_slots - 1; i >= 0; --i) s->free_slots.push_back(i);
    s->pinned.assign(max_slots, nullptr);
    s->slot_up.assign(max_slots, nullptr);
    s->slot_done.assign(max_slots, nullptr);
    s->pinned_cap.assign(max_slots, 0);
    cudaError_t e = cudaStreamCreateWithFlags(&s->up_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&s->work), 64);
    // result buffers: 16 KB per slot up front (problems of up to ~4,000 variables)
    for (int i = 0; i < max_slots && e == cudaSuccess; ++i) {
        e = cudaMallocHost(reinterpret_cast<void **>(&s->pinned[i]), 16384);
        if (e == cudaSuccess) s->pinned_cap[i] = 16384;
    }
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = cudaEventCreateWithFlags(&s->dev_ev[b], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->work, 0, 64, s->stream);
    if (e != cudaSuccess) {
        int rc = cuda_error(e, "srv_create");
        srv_free(s);
        return rc;
    }
    s->t0 = now_ms();
    const unsigned hw = std::thread::hardware_concurrency();
    const int n_planners = static_cast<int>(std::max(1u, std::min(8u, hw > 1 ? hw - 1 : 1u)));
    s->dev = dev;
    s->planner_up.assign(n_planners, nullptr);
    for (int i = 0; i < n_planners; ++i) {
        if (cudaError_t e2 = cudaStreamCreateWithFlags(&s->planner_up[i], cudaStreamNonBlocking); e2 != cudaSuccess) {
            int rc = cuda_error(e2, "planner stream");
            srv_free(s);
            return rc;
        }
    }
    for (int i = 0; i < n_planners; ++i) s->planners.emplace_back(planner_loop, s, i);
    *out = s;
    return GPUBE_OK;
}

extern "C" int64_t srv_submit(gpube_server *s, wcsp *w, int32_t kind, int32_t i_bound, const int32_t *parent,
                              const solve_opts *opts)
{
    if (!s || !w) return set_error(GPUBE_EINVAL, "null argument");
    if (kind < GPUBE_KIND_BE || kind > GPUBE_KIND_SUM_MBE) return set_error(GPUBE_EINVAL, "unknown kind %d", kind);
    Request *r = new Request();
    solve_opts &o = r->opts;
    if (opts) o = *opts;
    else solve_opts_init(&o);
    o.block_threads = s->threads;  // one CTA size for every merged launch
    o.batched = 1;
    o.use_graph = 0;
    o.autotune_cache = nullptr;
    o.device = s->dev;
    // small requests: inner row blocks of two CTAs' width keep the per-task
    // offset tables (one row per inner row) small
    if (o.lo_target <= 0) o.lo_target = 2 * s->threads;
    // merged launches take the largest shared-memory need of their tasks:
    // keep staged tables at the default limit
    if (o.stage_max_entries == 0 || o.stage_max_entries > 4096) o.stage_max_entries = 4096;
    // copies of everything the plan reads, owned by the request
    const int n = w->n;
    wcsp_ref(w);
    r->prob = w;
    if (parent) r->parent.assign(parent, parent + n);
    if (o.order) {
        r->order.assign(o.order, o.order + n);
        o.order = r->order.data();
    }
    if (o.parent) {
        r->opt_parent.assign(o.parent, o.parent + n);
        o.parent = r->opt_parent.data();
    }
    if (o.n_evidence_vars > 0 && o.evidence_vars) {
        r->ev_vars.assign(o.evidence_vars, o.evidence_vars + o.n_evidence_vars);
        o.evidence_vars = r->ev_vars.data();
    }
    r->kind = kind;
    r->i_bound = i_bound;
    r->state = kPlanning;
    r->id = s->next_id++;
    r->t_submit = now_ms() - s->t0;
    s->reqs[r->id] = r;
    {
        std::lock_guard<std::mutex> lk(s->pmu);
        s->to_plan.push_back(r);
        s->planning++;
    }
    s->pcv.notify_one();
    return r->id;
}

static int admit(gpube_server *s)
{
    // in order: reserve memory and a slot, then hand the binding (descriptors,
    // uploads) to the planner threads; bound requests come back through
    // take_planned
    int handed = 0;
    while (!s->queue.empty()) {
        Request *r = s->queue.front();
        if (!reserve(s, r)) break;  // wait until memory and a slot free up
        s->queue.pop_front();
        std::lock_guard<std::mutex> lk(s->pmu);
        s->to_bind.push_back(r);
        s->planning++;
        ++handed;
    }
    if (handed) s->pcv.notify_all();
    s->waiting.store(static_cast<int64_t>(s->queue.size()));
    s->max_inflight = std::max<int64_t>(s->max_inflight, static_cast<int64_t>(s->active.size()));
    return GPUBE_OK;
}

static int retire(gpube_server *s)
{
    for (size_t i = 0; i < s->active.size();) {
        Request *r = s->active[i];
        if (r->state == kValue && cudaEventQuery(r->done_ev) == cudaSuccess) {
            const unsigned char *pb = s->pinned[r->slot];
            int32_t status;
            memcpy(&status, pb, 4);
            double rr[2];
            memcpy(rr, pb + 8, 16);
            const int n = r->st->w->n;
            const bool sum = kind_sum(r->st->plan.kind);  // no assignment, no Eq. 1 cost
            if (!sum)
                r->sigma.assign(reinterpret_cast<const int32_t *>(pb + 24),
                                reinterpret_cast<const int32_t *>(pb + 24) + n);
            r->res.bound = rr[0];
            r->res.cost = sum ? NAN : rr[1];
            const Plan &P = r->st->plan;
            r->res.induced_width = P.width;
            r->res.n_tasks = static_cast<int32_t>(P.tasks.size());
            r->res.n_levels = P.n_levels;
            r->res.util_entries = P.util_entries;
            r->res.alg_bytes = alg_bytes_of(P);
            r->res.plan_ms = r->st->plan_ms;
            r->rc = status ? GPUBE_ETIMEDOUT : GPUBE_OK;
            r->state = status ? kFailed : kDone;
            r->t_done = now_ms() - s->t0;
            {
                std::lock_guard<std::mutex> g(s->amu);
                s->alloc.release(r->off, r->bytes);
                s->free_slots.push_back(r->slot);
            }
            r->up_ev = r->done_ev = nullptr;  // the slot's events, reused
            r->st->sync_on_free = false;  // its work is complete (done_ev)
            {
                // freeing a plan's host structures is left to the planner threads
                std::lock_guard<std::mutex> lk(s->pmu);
                s->to_free.push_back({r->st, r->prob});
            }
            s->pcv.notify_one();
            r->st = nullptr;
            r->prob = nullptr;
            s->active.erase(s->active.begin() + i);
        } else {
            ++i;
        }
    }
    return GPUBE_OK;
}

// Take the finished plans: failures end their request, the others join the
// admission queue in submission order.
static void take_planned(gpube_server *s)
{
    std::vector<Request *> got;
    {
        std::lock_guard<std::mutex> lk(s->pmu);
        got.swap(s->planned);
        s->planning -= static_cast<int64_t>(got.size());
    }
    for (Request *r : got) {
        if (r->rc) {  // planning or binding failed
            r->state = kFailed;
            r->t_done = now_ms() - s->t0;
            if (r->st) {
                r->st->sync_on_free = false;
                util_state_free(r->st);
                r->st = nullptr;
            }
            wcsp_unref(r->prob);
            r->prob = nullptr;
            continue;
        }
        r->bytes = r->st->arena_bytes;
        if (r->bound) {  // admitted and bound by its planner thread
            r->state = kActive;
            s->active.push_back(r);
            continue;
        }
        r->state = kQueued;
        auto it = std::upper_bound(s->queue.begin(), s->queue.end(), r,
                                   [](const Request *a, const Request *b) { return a->id < b->id; });
        s->queue.insert(it, r);
    }
    s->waiting.store(static_cast<int64_t>(s->queue.size()));
    s->max_inflight = std::max<int64_t>(s->max_inflight, static_cast<int64_t>(s->active.size()));
}

extern "C" int srv_step(gpube_server *s)
{
    if (!s) return set_error(GPUBE_EINVAL, "null server");
    take_planned(s);
    int rc = retire(s);
    if (!rc) rc = admit(s);
    if (rc) return rc;
    // merge the next level of every running request into one launch.  One
    // launch runs one kernel instantiation with one top cost, so only the
    // requests that share them are merged; when the running requests differ
    // (integer / fp32 costs, sum-product, another top cost) the groups take
    // turns, one per step.
    std::vector<std::pair<int, uint32_t>> keys;
    for (Request *r : s->active)
        if (r->state == kActive && r->next_level < r->st->plan.n_levels) {
            const std::pair<int, uint32_t> k(r->st->ktype, r->st->w->top_k);
            if (std::find(keys.begin(), keys.end(), k) == keys.end()) keys.push_back(k);
        }
    std::pair<int, uint32_t> key(kKTypeInt, 0u);
    if (!keys.empty()) key = keys[static_cast<size_t>(s->key_turn++) % keys.size()];
    std::vector<TaskDev> tds;
    std::vector<Request *> finishing;
    int smem = 0, pipe_b = 0;
    for (Request *r : s->active) {
        if (r->state != kActive) continue;
        if (!r->up_waited) {
            SRV_TRY(cudaStreamWaitEvent(s->stream, r->up_ev, 0));
            r->up_waited = true;
        }
        const Plan &P = r->st->plan;
        if (r->next_level < P.n_levels && r->st->ktype == key.first && r->st->w->top_k == key.second) {
            const TaskDev *td = reinterpret_cast<const TaskDev *>(
                r->st->host_blob.data() + (r->st->dl.taskdev - r->st->desc_off));
            for (int i = P.level_off[r->next_level]; i < P.level_off[r->next_level + 1]; ++i) {
                tds.push_back(td[i]);
                smem = std::max(smem, td[i].stage_bytes);
                if (td[i].pipe) pipe_b = std::max(pipe_b, pipe_bytes_per_thread(td[i].d));
            }
            r->next_level++;
        }
        if (r->next_level >= P.n_levels) finishing.push_back(r);
    }
    if (!tds.empty()) {
        const int b = s->flip;
        s->flip ^= 1;
        if (s->dev_used[b]) SRV_TRY(cudaEventSynchronize(s->dev_ev[b]));
        const size_t nt = tds.size();
        const size_t bytes = al(sizeof(TaskDev) * nt, 16) + 4 * (nt + 1);
        if (s->dcap[b] < bytes) {
            if (s->dbuf[b]) cudaFree(s->dbuf[b]);
            if (s->hbuf[b]) cudaFreeHost(s->hbuf[b]);
            s->dbuf[b] = s->hbuf[b] = nullptr;
            s->dcap[b] = 0;
            const size_t cap = std::max<size_t>(bytes * 2, 1 << 16);
            SRV_TRY(cudaMalloc(reinterpret_cast<void **>(&s->dbuf[b]), cap));
            SRV_TRY(cudaMallocHost(reinterpret_cast<void **>(&s->hbuf[b]), cap));
            s->dcap[b] = cap;
        }
        // pinned staging: the copy is queued without waiting for the stream
        // (the buffer's previous launch has completed, dev_ev[b] above)
        unsigned char *host = s->hbuf[b];
        memcpy(host, tds.data(), sizeof(TaskDev) * nt);
        int32_t *pre = reinterpret_cast<int32_t *>(host + al(sizeof(TaskDev) * nt, 16));
        int64_t tot = 0;
        for (size_t i = 0; i < nt; ++i) {
            pre[i] = static_cast<int32_t>(tot);
            tot += tds[i].n_items;
        }
        pre[nt] = static_cast<int32_t>(tot);
        if (tot > INT32_MAX / 2) return set_error(GPUBE_ENOMEM, "merged launch has too many work items");
        SRV_TRY(cudaMemcpyAsync(s->dbuf[b], host, bytes, cudaMemcpyHostToDevice, s->stream));
        LaunchDev L{};
        L.tasks = reinterpret_cast<const TaskDev *>(s->dbuf[b]);
        L.prefix = reinterpret_cast<const int32_t *>(s->dbuf[b] + al(sizeof(TaskDev) * nt, 16));
        L.n_tasks = static_cast<int32_t>(nt);
        L.total_items = static_cast<int32_t>(tot);
        L.counter = s->work + b;
        L.status = s->work + 2;
        L.top_k = key.second;
        L.arows_off = static_cast<int32_t>(al(smem, 16));
        L.pipe_off = L.arows_off + (pipe_b ? kMaxPipeRows * 16 : 0);
        if (pipe_b) smem = L.pipe_off + s->threads * pipe_b;
        smem = place_prefix_smem(L, smem);
        SRV_TRY(cudaMemsetAsync(L.counter, 0, 4, s->stream));
        const int64_t cap = static_cast<int64_t>(util_max_blocks_per_sm(key.first, s->threads, smem)) * s->num_sms;
        const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(tot, cap)));
        SRV_TRY(launch_util(L, key.first, grid, s->threads, smem, s->stream));
        SRV_TRY(cudaEventRecord(s->dev_ev[b], s->stream));
        s->dev_used[b] = true;
        s->launches++;
    }
    // the VALUE phases of the requests whose last level ran: one launch per
    // value-kernel instantiation (integer / fp32 costs), one CTA per request,
    // then each request's result copy and completion event
    for (int vk = 0; vk < 2; ++vk) {
        const bool want_int = vk == 0;
        std::vector<Request *> grp;
        for (Request *r : finishing)
            if ((r->st->ktype == kKTypeInt) == want_int) grp.push_back(r);
        for (size_t a = 0; a < grp.size(); a += kMaxValueBatch) {
            const size_t b = std::min(grp.size(), a + kMaxValueBatch);
            ValueBatch vb{};
            int smem = 0;
            for (size_t i = a; i < b; ++i) {
                vb.v[vb.n++] = grp[i]->st->vdev;
                smem = std::max(smem, grp[i]->st->value_smem);
                grp[i]->st->ran = true;
            }
            SRV_TRY(launch_value_batch(vb, want_int ? kKTypeInt : kKTypeFloat, smem, s->stream));
            for (size_t i = a; i < b; ++i) {
                Request *r = grp[i];
                util_state *st = r->st;
                const size_t need = 24 + 4 * static_cast<size_t>(std::max(st->w->n, 1));
                SRV_TRY(cudaMemcpyAsync(s->pinned[r->slot], st->base + st->status_off, need,
                                        cudaMemcpyDeviceToHost, s->stream));
                SRV_TRY(cudaEventRecord(r->done_ev, s->stream));
                r->state = kValue;
            }
        }
    }
    int64_t planning;
    {
        std::lock_guard<std::mutex> lk(s->pmu);
        planning = s->planning;
    }
    return static_cast<int>(planning + static_cast<int64_t>(s->queue.size() + s->active.size()));
}

extern "C" int srv_result(gpube_server *s, int64_t id, int32_t *assignment, solve_result *res)
{
    if (!s) return set_error(GPUBE_EINVAL, "null server");
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return set_error(GPUBE_EINVAL, "unknown request %lld", static_cast<long long>(id));
    Request *r = it->second;
    if (r->state == kFailed)
        return set_error(r->rc, "request %lld failed%s%s", static_cast<long long>(id), r->err.empty() ? "" : ": ",
                         r->err.c_str());
    if (r->state != kDone) return GPUBE_EAGAIN;
    if (assignment) std::copy(r->sigma.begin(), r->sigma.end(), assignment);
    if (res) {
        int32_t *keep = res->assignment;
        *res = r->res;
        res->assignment = keep;
        if (keep && keep != assignment) std::copy(r->sigma.begin(), r->sigma.end(), keep);
    }
    return GPUBE_OK;
}

extern "C" int srv_times(gpube_server *s, int64_t id, double *t_submit, double *t_admit, double *t_done)
{
    if (!s) return set_error(GPUBE_EINVAL, "null server");
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return set_error(GPUBE_EINVAL, "unknown request");
    Request *r = it->second;
    if (t_submit) *t_submit = r->t_submit * 1e-3;
    if (t_admit) *t_admit = r->t_admit * 1e-3;
    if (t_done) *t_done = r->t_done * 1e-3;
    return r->state == kDone ? GPUBE_OK : GPUBE_EAGAIN;
}

extern "C" int srv_stats(gpube_server *s, int64_t *launches, int64_t *peak_bytes, int64_t *max_inflight)
{
    if (!s) return set_error(GPUBE_EINVAL, "null server");
    if (launches) *launches = s->launches;
    if (peak_bytes) {
        std::lock_guard<std::mutex> g(s->amu);
        *peak_bytes = static_cast<int64_t>(s->alloc.peak);
    }
    if (max_inflight) *max_inflight = s->max_inflight;
    return GPUBE_OK;
}

extern "C" void srv_free(gpube_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->pmu);
        s->stopping = true;
        s->to_plan.clear();  // requests not planned yet are never planned
    }
    s->pcv.notify_all();
    for (auto &t : s->planners) t.join();
    for (auto st_ : s->planner_up)
        if (st_) {
            cudaStreamSynchronize(st_);
            cudaStreamDestroy(st_);
        }
    for (auto &f : s->to_free) {
        util_state_free(f.first);
        wcsp_unref(f.second);
    }
    cudaStreamSynchronize(s->stream);
    if (s->up_stream) {
        cudaStreamSynchronize(s->up_stream);
        cudaStreamDestroy(s->up_stream);
    }
    for (auto &kv : s->reqs) {
        Request *r = kv.second;
        if (r->st) util_state_free(r->st);
        wcsp_unref(r->prob);
        delete r;
    }
    for (auto e : s->slot_up)
        if (e) cudaEventDestroy(e);
    for (auto e : s->slot_done)
        if (e) cudaEventDestroy(e);
    for (int b = 0; b < 2; ++b) {
        if (s->dbuf[b]) cudaFree(s->dbuf[b]);
        if (s->hbuf[b]) cudaFreeHost(s->hbuf[b]);
        if (s->dev_ev[b]) cudaEventDestroy(s->dev_ev[b]);
    }
    for (auto p : s->pinned)
        if (p) cudaFreeHost(p);
    if (s->work) cudaFree(s->work);
    if (s->owns && s->base) cudaFree(s->base);
    delete s;
}
