// serve.cu -- continuous batching of scenario requests (mhc_submit / mhc_poll / mhc_release).
//
// Each lane (small and large requests) has a scheduler thread that owns its admission: while a stream slot
// of the lane is idle and the lane's queue is not empty it takes requests from the queue head as long as
// the batch limits hold and the largest free pool block could hold them, lays them out as one batch
// without the lock (a batch of one request reuses the layout built at submission), allocates its blocks
// first fit (putting the requests back if the pool has no room), and enqueues on the slot's stream:
// descriptor upload, the fused batch kernels, the copy of the batch's risk outputs to the slot's pinned
// buffer and a host callback.  The callback (a CUDA driver thread; no CUDA calls) copies the outputs into
// the batch's host memory, frees the batch's scratch block and wakes pollers and the schedulers.  Poses,
// table and device risk outputs stay resident in the batch's block until every request of the batch is
// released.  Small requests run on high-priority streams of their own, so the thread-block scheduler starts
// their CTAs ahead of those of a large batch in flight, and the host work of a large batch does not hold
// up the small lane.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "runtime.h"

using namespace mhc;
using namespace mhc::host;

namespace {

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

constexpr size_t kSlotPinned = 4u << 20;   // initial mapped pinned staging per slot and direction

struct Server;
struct Batch;

struct Request {
    uint64_t ticket = 0;
    std::vector<mhc_object> objs;                 // the copied scenario
    std::vector<std::vector<float>> arrays;       // its grids and parameters
    std::vector<std::vector<float>> weights;      // per object (empty: uniform)
    bool has_w = false;
    mhc_scenario sc{};
    long long tests = 0;
    size_t bytes = 0;                             // device bytes alone (resident + scratch)
    bool small = true;
    Layout L;                                     // the request's own layout (built at submission), reused by a
    bool has_layout = false;                      // batch of this request alone
    enum State { kQueued, kTaken, kRunning, kDone, kFailed } state = kQueued;   // kTaken: being laid out
    Batch *batch = nullptr;
    int index = 0;
    int64_t t_submit = 0, t_launch = 0, t_done = 0;
    bool released = false;
};

struct Batch {
    Server *srv = nullptr;
    std::vector<Request *> reqs;
    Layout L;
    std::vector<float> w;
    size_t res_off = 0, res_bytes = 0;            // poses, table, risk outputs (resident)
    size_t scr_off = 0, scr_bytes = 0;            // descriptors, weights, bounds, risk scratch
    bool scr_held = false;
    mhc_poses poses{};
    int16_t *table = nullptr;
    mhc_risk dev{};
    size_t out_bytes = 0;
    std::vector<char> host;                       // the risk outputs, copied at completion
    int slot = -1;
    int live = 0;                                 // requests not yet released
    bool complete = false, failed = false;
};

struct Slot {
    cudaStream_t st = nullptr;
    bool small = true;
    Batch *busy = nullptr;
    char *stage = nullptr;   size_t stage_cap = 0;     // mapped pinned: descriptors of the batch
    char *pinned = nullptr;  size_t pinned_cap = 0;    // mapped pinned: risk outputs of the batch
    char *stage_dev = nullptr, *pinned_dev = nullptr;  // their device addresses
    std::vector<char *> retired;                        // outgrown pinned buffers (freed at stop)
};

struct Server {
    mhc_ctx *ctx = nullptr;
    mhc_ctx shadow;                               // collision configuration for the loop's launches
    mhc_ctx shadow_large;                         // the same with the large lane's CTA cap
    char *base = nullptr;
    mhc_pool *pool = nullptr;
    size_t pool_bytes = 0;
    mhc_serve_config cfg{};
    std::mutex mu;
    std::condition_variable cv, cv_done;
    std::deque<Request *> q_small, q_large;
    std::unordered_map<uint64_t, Request *> reqs;
    std::vector<Slot> slots;
    std::thread th_small, th_large;               // one scheduler per lane
    bool stopping = false, paused = false;
    uint64_t next_ticket = 1;
    long long n_submitted = 0, n_completed = 0, n_batches = 0;
};

void delete_batch(Server *S, Batch *b) {
    for (Request *r : b->reqs) delete r;
    if (b->res_bytes) pool_free(S->pool, b->res_off);
    if (b->scr_held) pool_free(S->pool, b->scr_off);
    delete b;
}

// Frees a batch once it is complete and every request of it is released (caller holds mu).
void maybe_retire(Server *S, Batch *b) {
    if (b->complete && b->live == 0) delete_batch(S, b);
}

void CUDART_CB on_batch_done(void *arg) {
    Batch *b = static_cast<Batch *>(arg);
    Server *S = b->srv;
    std::lock_guard<std::mutex> lk(S->mu);
    Slot &sl = S->slots[b->slot];
    b->host.assign(sl.pinned, sl.pinned + b->out_bytes);
    const int64_t t = now_ns();
    for (Request *r : b->reqs) {
        r->state = Request::kDone;
        r->t_done = t;
    }
    S->n_completed += (long long)b->reqs.size();
    pool_free(S->pool, b->scr_off);
    b->scr_held = false;
    b->complete = true;
    sl.busy = nullptr;
    S->cv_done.notify_all();
    S->cv.notify_all();
    maybe_retire(S, b);
}

// Marks a batch failed (its work is no longer in flight: caller synchronised the stream or nothing was
// enqueued).  Caller holds mu.
void fail_batch(Server *S, Batch *b) {
    for (Request *r : b->reqs) {
        r->state = Request::kFailed;
        r->t_done = now_ns();
    }
    b->failed = true;
    b->complete = true;
    if (b->scr_held) { pool_free(S->pool, b->scr_off); b->scr_held = false; }
    if (b->slot >= 0) S->slots[b->slot].busy = nullptr;
    S->cv_done.notify_all();
    maybe_retire(S, b);
}

size_t resident_bytes(const Layout &L) {
    return 4 * align_up(sizeof(float) * (size_t)L.n_pose) + align_up(sizeof(int16_t) * (size_t)L.n_entries) +
           risk_output_bytes(L) + kAlign;
}

// Takes requests for an idle slot from the head of its lane's queue (holds mu): as many as the batch limits
// allow and the largest free pool block could hold.  They are marked taken, so a release meanwhile only
// flags them.
std::vector<Request *> take_requests(Server *S, const Slot &sl) {
    std::deque<Request *> &q = sl.small ? S->q_small : S->q_large;
    std::vector<Request *> take;
    size_t need = 0;
    long long tests = 0;
    const size_t largest = pool_largest(S->pool);
    while (!q.empty() && (int)take.size() < S->cfg.max_batch) {
        Request *r = q.front();
        if (!take.empty() && sl.small && tests + r->tests > S->cfg.max_batch_tests) break;
        if (need + r->bytes > largest) break;
        take.push_back(r);
        q.pop_front();
        r->state = Request::kTaken;
        need += r->bytes;
        tests += r->tests;
    }
    return take;
}

// Puts taken requests back at the head of their queue, in order (holds mu); those released meanwhile go.
void untake(Server *S, std::vector<Request *> &take, bool small) {
    std::deque<Request *> &q = small ? S->q_small : S->q_large;
    for (auto it = take.rbegin(); it != take.rend(); ++it) {
        Request *r = *it;
        if (r->released) { delete r; continue; }
        r->state = Request::kQueued;
        q.push_front(r);
    }
    take.clear();
}

// The batch of taken requests laid out (without mu: the host work of a large scenario does not hold up
// the other lane, submissions or polls).  A batch of one request reuses the layout built at submission.
Batch *build_batch(Server *S, std::vector<Request *> &take) {
    Batch *b = new Batch();
    b->srv = S;
    std::vector<const float *> wp;
    bool any_w = false;
    for (Request *r : take)
        for (size_t o = 0; o < r->objs.size(); ++o) {
            wp.push_back(r->has_w && !r->weights[o].empty() ? r->weights[o].data() : nullptr);
            any_w |= wp.back() != nullptr;
        }
    bool ok;
    if (take.size() == 1 && take[0]->has_layout) {
        b->L = take[0]->L;
        ok = true;
    } else {
        std::vector<mhc_scenario> scs;
        for (Request *r : take) scs.push_back(r->sc);
        ok = build_layout(scs.data(), (int)scs.size(), b->L) == MHC_OK;
        if (ok) plan_generation(b->L, S->shadow.n_sm, S->shadow.gen_scan);
    }
    if (ok) ok = gather_weights(b->L, any_w ? wp.data() : nullptr, b->w) == MHC_OK;
    if (ok) {
        b->res_bytes = resident_bytes(b->L);
        b->scr_bytes = scratch_of(b->L, !b->w.empty()).total + kAlign;
    }
    if (!ok) { delete b; return nullptr; }
    return b;
}

// The batch's pool blocks and its requests' states (holds mu).  False: the pool has no room (the caller
// puts the requests back).
bool admit_batch(Server *S, Batch *b, std::vector<Request *> &take) {
    if (!pool_alloc(S->pool, b->res_bytes, &b->res_off)) { b->res_bytes = 0; return false; }
    if (!(b->scr_held = pool_alloc(S->pool, b->scr_bytes, &b->scr_off))) {
        pool_free(S->pool, b->res_off);
        b->res_bytes = 0;
        return false;
    }
    b->reqs = take;
    b->live = (int)take.size();
    const int64_t t = now_ns();
    for (size_t q2 = 0; q2 < take.size(); ++q2) {
        take[q2]->state = Request::kRunning;
        take[q2]->batch = b;
        take[q2]->index = (int)q2;
        take[q2]->t_launch = t;
        if (take[q2]->released) --b->live;
    }
    return true;
}

// Host work and enqueue of one batch on its slot (without mu).  Returns false if the callback was not
// enqueued; the stream has then been synchronised.
bool launch_batch(Server *S, Batch *b, Slot &sl) {
    cudaError_t e = cudaSuccess;
    int rc = MHC_OK;
    char *res = S->base + b->res_off, *scr = S->base + b->scr_off;
    Bump rb{res, b->res_bytes, 0};
    const size_t plane = sizeof(float) * (size_t)b->L.n_pose;
    b->poses.x = static_cast<float *>(rb.take(plane));
    b->poses.y = static_cast<float *>(rb.take(plane));
    b->poses.c = static_cast<float *>(rb.take(plane));
    b->poses.s = static_cast<float *>(rb.take(plane));
    b->table = static_cast<int16_t *>(rb.take(sizeof(int16_t) * (size_t)b->L.n_entries));
    if (!take_risk_outputs(rb, b->L, b->dev)) return false;
    b->out_bytes = risk_output_bytes(b->L);
    DevDesc D;
    const std::vector<float> *w = b->w.empty() ? nullptr : &b->w;
    const size_t desc = pack_descriptors(b->L, w, nullptr, scr, D);
    // pinned buffers only grow, and a replaced one is freed at mhc_serve_stop: cudaFreeHost waits for the
    // device, which would hold this thread (and every admission) behind the batches in flight
    if (sl.stage_cap < desc) {
        char *nb = nullptr, *nd = nullptr;
        if (alloc_mapped(desc * 2, &nb, &nd) != cudaSuccess) return false;
        if (sl.stage) sl.retired.push_back(sl.stage);
        sl.stage = nb;
        sl.stage_dev = nd;
        sl.stage_cap = desc * 2;
    }
    if (sl.pinned_cap < b->out_bytes) {
        char *nb = nullptr, *nd = nullptr;
        if (alloc_mapped(b->out_bytes * 2, &nb, &nd) != cudaSuccess) return false;
        if (sl.pinned) sl.retired.push_back(sl.pinned);
        sl.pinned = nb;
        sl.pinned_dev = nd;
        sl.pinned_cap = b->out_bytes * 2;
    }
    pack_descriptors(b->L, w, sl.stage, scr, D);
    e = launch_copy(scr, sl.stage_dev, desc, sl.st);
    if (e == cudaSuccess) {
        Bump sb{scr, b->scr_bytes, align_up(desc)};
        rc = launch_all(sl.small ? &S->shadow : &S->shadow_large, b->L, D, sb, &b->poses, &b->poses, b->table, true,
                        &b->dev, sl.st, true, true);
    }
    if (e == cudaSuccess && rc == MHC_OK)
        e = launch_copy(sl.pinned_dev, b->dev.count, b->out_bytes, sl.st, !(sl.small ? S->shadow : S->shadow_large).profile);
    if (e == cudaSuccess && rc == MHC_OK) e = cudaLaunchHostFunc(sl.st, on_batch_done, b);
    if (e == cudaSuccess && rc == MHC_OK) return true;
    cudaStreamSynchronize(sl.st);
    return false;
}

// One scheduler thread per lane: while a slot of its lane is idle and the lane's queue is not empty it
// takes requests, lays them out, admits them into the pool and enqueues the batch.
void scheduler(Server *S, bool small_lane) {
    cudaSetDevice(S->ctx->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->stopping) {
        // a batch whose stream reports an error never gets its callback: fail it here
        for (Slot &sl : S->slots) {
            if (sl.small != small_lane || !sl.busy) continue;
            const cudaError_t q = cudaStreamQuery(sl.st);
            if (q != cudaSuccess && q != cudaErrorNotReady) fail_batch(S, sl.busy);
        }
        bool launched = false;
        if (!S->paused) {
            for (size_t s = 0; s < S->slots.size(); ++s) {
                Slot &sl = S->slots[s];
                if (sl.small != small_lane || sl.busy) continue;
                std::vector<Request *> take = take_requests(S, sl);
                if (take.empty()) continue;
                lk.unlock();
                Batch *b = build_batch(S, take);
                lk.lock();
                if (S->stopping || !b || !admit_batch(S, b, take)) {   // no room (or stopping): back to the queue
                    delete b;
                    untake(S, take, small_lane);
                    break;
                }
                b->slot = (int)s;
                sl.busy = b;
                ++S->n_batches;
                lk.unlock();
                const bool ok = launch_batch(S, b, sl);
                lk.lock();
                if (!ok) fail_batch(S, b);
                launched = true;
            }
        }
        if (!launched) S->cv.wait_for(lk, std::chrono::microseconds(500));
    }
}

Server *server_of(mhc_ctx *ctx) { return ctx ? static_cast<Server *>(ctx->server) : nullptr; }

int copy_outputs(const Batch *b, int s, const mhc_risk *out) {
    const Layout &L = b->L;
    const ScenDesc &S = L.scens[s];
    const int p0 = L.pair0[s], np = L.pair0[s + 1] - L.pair0[s];
    const long long k0 = np ? L.pairs[p0].kofs : 0, N = S.n_steps, e0 = S.e_base, he = S.h_e;
    const char *hb = b->host.data();
    auto src = [&](const void *dev_field) { return hb + (static_cast<const char *>(dev_field) -
                                                          reinterpret_cast<const char *>(b->dev.count)); };
    struct Cp { void *dst; const char *from; size_t n; } cps[] = {
        {out->count, src(b->dev.count) + 8 * p0, 8 * (size_t)np},
        {out->count_k, src(b->dev.count_k) + 8 * k0, 8 * (size_t)(np * N)},
        {out->P, src(b->dev.P) + 8 * p0, 8 * (size_t)np},
        {out->H, src(b->dev.H) + 8 * k0, 8 * (size_t)(np * N)},
        {out->naive, src(b->dev.naive) + 8 * e0, 8 * (size_t)he},
        {out->cond, src(b->dev.cond) + 8 * e0, 8 * (size_t)he},
        {out->indep, src(b->dev.indep) + 8 * e0, 8 * (size_t)he},
        {out->hits, src(b->dev.hits) + 4 * e0, 4 * (size_t)he},
        {out->attr_obj, src(b->dev.attr_obj) + 8 * (size_t)S.obj0, 8 * (size_t)S.n_obj},
        {out->attr_step, src(b->dev.attr_step) + 8 * S.step_base, 8 * (size_t)N},
        {out->scalars, src(b->dev.scalars) + 32 * (size_t)s, 32},
        {out->escape, src(b->dev.escape) + 4 * e0, 4 * (size_t)he},
        {out->n_escape, src(b->dev.n_escape) + 4 * (size_t)s, 4},
    };
    for (const Cp &c : cps)
        if (c.dst && c.n) std::memcpy(c.dst, c.from, c.n);
    return MHC_OK;
}

}  // namespace

namespace mhc {
namespace host {
void serve_shutdown(mhc_ctx *ctx) { mhc_serve_stop(ctx); }
}  // namespace host
}  // namespace mhc

extern "C" {

int mhc_serve_start(mhc_ctx *ctx, void *pool, size_t pool_bytes, const mhc_serve_config *cfg) {
    if (int r = check_ctx(ctx)) return r;
    if (ctx->server) return fail(MHC_E_INVALID, "a serving loop already runs on this context");
    if (!pool || pool_bytes < (1u << 20)) return fail(MHC_E_INVALID, "the pool must be non-NULL and at least 1 MiB");
    if (reinterpret_cast<uintptr_t>(pool) % kAlign) return fail(MHC_E_INVALID, "the pool must be 256-byte aligned");
    mhc_serve_config c{3, 1, 64, 4096, 1LL << 31, 1LL << 34};
    if (cfg) c = *cfg;
    if (c.small_slots < 1 || c.small_slots > 8 || c.large_slots < 1 || c.large_slots > 8 || c.max_batch < 1 ||
        c.max_batch > 4096 || c.max_queue < 1 || c.small_tests < 0 || c.max_batch_tests < 1)
        return fail(MHC_E_INVALID, "serve config out of range");
    MHC_CUDA(cudaSetDevice(ctx->device));
    int least = 0, greatest = 0;
    MHC_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    Server *S = new Server();
    S->ctx = ctx;
    S->base = static_cast<char *>(pool);
    S->pool = pool_new(pool_bytes);
    S->pool_bytes = pool_bytes & ~(kAlign - 1);
    S->cfg = c;
    S->shadow.device = ctx->device;
    S->shadow.n_sm = ctx->n_sm;
    S->shadow.cull = ctx->cull;
    S->shadow.variant = ctx->variant;
    S->shadow.gen_scan = ctx->gen_scan;
    // the large lane may cap its collision kernels' CTAs (collide_max_ctas) to leave SM room to the small
    // lane; measured at 2000 requests/s, a cap of 3 CTAs per SM slowed the large requests past their
    // arrival rate, so it is off
    S->shadow_large = S->shadow;
    S->shadow.tuned = ctx->tuned;
    S->slots.resize(c.small_slots + c.large_slots);
    for (size_t s = 0; s < S->slots.size(); ++s) {
        Slot &sl = S->slots[s];
        sl.small = (int)s < c.small_slots;
        cudaError_t e = cudaStreamCreateWithPriority(&sl.st, cudaStreamNonBlocking, sl.small ? greatest : least);
        // pinned staging sized for typical batches up front (growth allocates, see launch_batch)
        if (e == cudaSuccess && (e = alloc_mapped(kSlotPinned, &sl.stage, &sl.stage_dev)) == cudaSuccess)
            sl.stage_cap = kSlotPinned;
        if (e == cudaSuccess && (e = alloc_mapped(kSlotPinned, &sl.pinned, &sl.pinned_dev)) == cudaSuccess)
            sl.pinned_cap = kSlotPinned;
        if (e != cudaSuccess) {
            for (Slot &x : S->slots) {
                if (x.stage) cudaFreeHost(x.stage);
                if (x.pinned) cudaFreeHost(x.pinned);
            }
            for (Slot &x : S->slots) if (x.st) cudaStreamDestroy(x.st);
            pool_delete(S->pool);
            delete S;
            return cuda_fail(e, "serving streams and pinned staging");
        }
    }
    ctx->server = S;
    S->th_small = std::thread(scheduler, S, true);
    S->th_large = std::thread(scheduler, S, false);
    return MHC_OK;
}

int mhc_serve_stop(mhc_ctx *ctx) {
    Server *S = server_of(ctx);
    if (!S) return fail(MHC_E_NOTFOUND, "no serving loop on this context");
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
    }
    S->cv.notify_all();
    S->th_small.join();
    S->th_large.join();
    for (Slot &sl : S->slots) cudaStreamSynchronize(sl.st);   // callbacks of the batches in flight run
    std::lock_guard<std::mutex> lk(S->mu);
    std::vector<Batch *> batches;
    for (auto &kv : S->reqs) {
        Request *r = kv.second;
        if (r->batch) {
            bool seen = false;
            for (Batch *b : batches) seen |= b == r->batch;
            if (!seen) batches.push_back(r->batch);
        }
    }
    for (Request *r : S->q_small) delete r;
    for (Request *r : S->q_large) delete r;
    for (Batch *b : batches) delete_batch(S, b);   // deletes its requests
    for (Slot &sl : S->slots) {
        if (sl.st) cudaStreamDestroy(sl.st);
        if (sl.stage) cudaFreeHost(sl.stage);
        if (sl.pinned) cudaFreeHost(sl.pinned);
        for (char *p : sl.retired) cudaFreeHost(p);
    }
    pool_delete(S->pool);
    ctx->server = nullptr;
    S->reqs.clear();
    S->q_small.clear();
    S->q_large.clear();
    delete S;
    return MHC_OK;
}

int mhc_submit(mhc_ctx *ctx, const mhc_scenario *scen, const float *const *traj_weights, uint64_t *ticket) {
    Server *S = server_of(ctx);
    if (!S) return fail(MHC_E_NOTFOUND, "no serving loop on this context");
    if (!ticket) return fail(MHC_E_INVALID, "ticket is NULL");
    Layout L;
    if (int r = build_layout(scen, L)) return r;
    std::vector<float> wcheck;
    if (int r = gather_weights(L, traj_weights, wcheck)) return r;
    Request *r = new Request();
    r->objs.assign(scen->objects, scen->objects + scen->n_objects);
    r->arrays.reserve(3 * scen->n_objects);
    r->weights.resize(scen->n_objects);
    for (int o = 0; o < scen->n_objects; ++o) {
        mhc_object &d = r->objs[o];
        const mhc_object &s = scen->objects[o];
        r->arrays.emplace_back(s.grid_a, s.grid_a + s.n_a);
        d.grid_a = r->arrays.back().data();
        r->arrays.emplace_back(s.grid_b, s.grid_b + s.n_b);
        d.grid_b = r->arrays.back().data();
        if (s.veh_params) {
            r->arrays.emplace_back(s.veh_params, s.veh_params + 6);
            d.veh_params = r->arrays.back().data();
        }
        if (traj_weights && traj_weights[o]) {
            r->weights[o].assign(traj_weights[o], traj_weights[o] + (size_t)s.n_a * s.n_b);
            r->has_w = true;
        }
    }
    r->sc = *scen;
    r->sc.objects = r->objs.data();
    for (const PairDesc &p : L.pairs) r->tests += (long long)L.objs[p.a].h * L.objs[p.b].h * p.n_steps;
    r->bytes = resident_bytes(L) + scratch_of(L, r->has_w).total + 2 * kAlign;
    r->small = r->tests <= S->cfg.small_tests;
    plan_generation(L, S->shadow.n_sm, S->shadow.gen_scan);
    r->L = std::move(L);
    r->has_layout = true;
    std::lock_guard<std::mutex> lk(S->mu);
    if (r->bytes > S->pool_bytes) {
        delete r;
        return fail(MHC_E_NOMEM, "the request alone needs more device memory than the pool holds");
    }
    if ((long long)(S->q_small.size() + S->q_large.size()) >= S->cfg.max_queue) {
        delete r;
        return fail(MHC_E_BUSY, "request queue full");
    }
    r->ticket = S->next_ticket++;
    r->t_submit = now_ns();
    S->reqs.emplace(r->ticket, r);
    (r->small ? S->q_small : S->q_large).push_back(r);
    ++S->n_submitted;
    *ticket = r->ticket;
    S->cv.notify_all();
    return MHC_OK;
}

int mhc_poll(mhc_ctx *ctx, uint64_t ticket, const mhc_risk *out, int32_t timeout_us) {
    Server *S = server_of(ctx);
    if (!S) return fail(MHC_E_NOTFOUND, "no serving loop on this context");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(MHC_E_NOTFOUND, "unknown or released ticket");
    Request *r = it->second;
    auto finished = [&] { return r->state == Request::kDone || r->state == Request::kFailed; };
    if (!finished() && timeout_us != 0) {
        if (timeout_us < 0) S->cv_done.wait(lk, finished);
        else S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), finished);
    }
    if (r->state == Request::kFailed) return fail(MHC_E_CUDA, "the request's batch failed on the device");
    if (r->state != Request::kDone) return MHC_PENDING;
    if (out) copy_outputs(r->batch, r->index, out);
    return MHC_OK;
}

int mhc_release(mhc_ctx *ctx, uint64_t ticket) {
    Server *S = server_of(ctx);
    if (!S) return fail(MHC_E_NOTFOUND, "no serving loop on this context");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(MHC_E_NOTFOUND, "unknown or released ticket");
    Request *r = it->second;
    S->reqs.erase(it);
    r->released = true;
    if (r->state == Request::kQueued) {
        std::deque<Request *> &q = r->small ? S->q_small : S->q_large;
        for (auto qi = q.begin(); qi != q.end(); ++qi)
            if (*qi == r) { q.erase(qi); break; }
        delete r;
        return MHC_OK;
    }
    if (r->state == Request::kTaken) return MHC_OK;   // its scheduler admits it (or puts it back) and counts the flag
    Batch *b = r->batch;
    --b->live;
    maybe_retire(S, b);
    S->cv.notify_all();
    return MHC_OK;
}

int mhc_request_buffers(mhc_ctx *ctx, uint64_t ticket, mhc_poses *poses, int16_t **table, mhc_risk *dev_out) {
    Server *S = server_of(ctx);
    if (!S) return fail(MHC_E_NOTFOUND, "no serving loop on this context");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(MHC_E_NOTFOUND, "unknown or released ticket");
    Request *r = it->second;
    if (r->state != Request::kDone) return r->state == Request::kFailed ? fail(MHC_E_CUDA, "the batch failed") : MHC_PENDING;
    const Batch *b = r->batch;
    const Layout &L = b->L;
    const int s = r->index;
    const ScenDesc &SD = L.scens[s];
    const long long pose0 = L.objs[SD.obj0].pose_base;
    if (poses) {
        poses->x = b->poses.x + pose0;
        poses->y = b->poses.y + pose0;
        poses->c = b->poses.c + pose0;
        poses->s = b->poses.s + pose0;
    }
    if (table) *table = b->table + L.entry0[s];
    if (dev_out) {
        const int p0 = L.pair0[s], np = L.pair0[s + 1] - L.pair0[s];
        const long long k0 = np ? L.pairs[p0].kofs : 0, e0 = SD.e_base;
        dev_out->count = b->dev.count + p0;
        dev_out->count_k = b->dev.count_k + k0;
        dev_out->P = b->dev.P + p0;
        dev_out->H = b->dev.H + k0;
        dev_out->naive = b->dev.naive + e0;
        dev_out->cond = b->dev.cond + e0;
        dev_out->indep = b->dev.indep + e0;
        dev_out->hits = b->dev.hits + e0;
        dev_out->attr_obj = b->dev.attr_obj + SD.obj0;
        dev_out->attr_step = b->dev.attr_step + SD.step_base;
        dev_out->scalars = b->dev.scalars + 4 * s;
        dev_out->escape = b->dev.escape + e0;
        dev_out->n_escape = b->dev.n_escape + s;
    }
    return MHC_OK;
}

int mhc_request_times(mhc_ctx *ctx, uint64_t ticket, int64_t ns[3], int32_t *batch_size) {
    Server *S = server_of(ctx);
    if (!S) return fail(MHC_E_NOTFOUND, "no serving loop on this context");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(MHC_E_NOTFOUND, "unknown or released ticket");
    const Request *r = it->second;
    if (ns) { ns[0] = r->t_submit; ns[1] = r->t_launch; ns[2] = r->t_done; }
    if (batch_size) *batch_size = r->batch ? (int32_t)r->batch->reqs.size() : 0;
    return MHC_OK;
}

int mhc_serve_stats_read(mhc_ctx *ctx, mhc_serve_stats *st) {
    Server *S = server_of(ctx);
    if (!S) return fail(MHC_E_NOTFOUND, "no serving loop on this context");
    if (!st) return fail(MHC_E_INVALID, "stats is NULL");
    std::lock_guard<std::mutex> lk(S->mu);
    st->submitted = S->n_submitted;
    st->completed = S->n_completed;
    st->batches = S->n_batches;
    st->queued = (int64_t)(S->q_small.size() + S->q_large.size());
    long long running = 0;
    for (const Slot &sl : S->slots) running += sl.busy ? (long long)sl.busy->reqs.size() : 0;
    st->running = running;
    st->pool_free = pool_free_bytes(S->pool);
    st->pool_largest = pool_largest(S->pool);
    return MHC_OK;
}

int mhc_serve_pause(mhc_ctx *ctx, int32_t paused) {
    Server *S = server_of(ctx);
    if (!S) return fail(MHC_E_NOTFOUND, "no serving loop on this context");
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->paused = paused != 0;
    }
    S->cv.notify_all();
    return MHC_OK;
}

}  // extern "C"
