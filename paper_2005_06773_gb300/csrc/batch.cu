// batch.cu -- batches of uneven scenarios in one launch sequence, and plans: a batch whose descriptors
// live in caller-owned device scratch and whose launch sequence is captured once as a CUDA graph and
// replayed (new initial states are written into the plan's pinned copy of the descriptors between
// replays).  The kernels are those of the single-scenario path; every descriptor carries its scenario's
// horizon and accumulator bases, so a batch is one generation launch over all hypotheses, one collision
// launch over all tiles of all pairs and one risk walk over all EGO hypotheses.
#include <algorithm>
#include <cstring>

#include "runtime.h"

using namespace mhc;
using namespace mhc::host;

// One group of a pipelined plan: a run of consecutive scenarios with its own layout, descriptors (at
// desc_off in the plan's scratch and in its pinned copy) and work scratch, writing into its slices of the
// batch's poses, table and risk outputs.
struct PlanGroup {
    int s0 = 0, n = 0;                 // scenarios [s0, s0 + n)
    Layout L;
    std::vector<float> w;
    size_t desc_off = 0, desc_bytes = 0;
    char *work = nullptr;              // its scratch past the descriptors
    size_t work_bytes = 0;
    DevDesc D{};
    mhc_poses poses{};
    int16_t *table = nullptr;
    mhc_risk out{};
};

struct mhc_plan {
    mhc_ctx *ctx = nullptr;
    Layout L;
    std::vector<float> w;
    bool has_w = false;
    char *dev = nullptr;               // caller's device scratch
    size_t dev_bytes = 0;
    char *host = nullptr;              // mapped pinned copy of the descriptors (source of each launch's upload)
    char *host_dev = nullptr;          // its device address
    size_t desc_bytes = 0;
    DevDesc D{};
    mhc_poses poses{};
    int16_t *table = nullptr;
    mhc_risk out{};
    std::vector<PlanGroup> groups;     // more than one: the pipelined launch sequence (see plan_enqueue)
    cudaStream_t cap = nullptr;        // capture stream
    cudaStream_t side = nullptr;       // the pipeline's second stream
    std::vector<cudaEvent_t> ev;       // fork, join, and one per group's generation
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;        // recorded after each launch
    bool launched = false;
};

namespace {

// Structural fields of two layouts agree (same objects, grids sizes, steps, pairs): only states may differ.
bool same_structure(const Layout &a, const Layout &b) {
    if (a.n_obj != b.n_obj || a.n_scen != b.n_scen || a.pairs.size() != b.pairs.size() ||
        a.grids.size() != b.grids.size() || a.n_traj != b.n_traj || a.n_entries != b.n_entries)
        return false;
    for (int o = 0; o < a.n_obj; ++o) {
        const ObjDesc &x = a.objs[o], &y = b.objs[o];
        if (x.kind != y.kind || x.n_a != y.n_a || x.n_b != y.n_b || x.n_steps != y.n_steps) return false;
    }
    for (size_t p = 0; p < a.pairs.size(); ++p)
        if (a.pairs[p].a != b.pairs[p].a || a.pairs[p].b != b.pairs[p].b) return false;
    return true;
}

// Pipeline groups: runs of consecutive scenarios with about equal collision tiles (kPlanGroups of them from
// kPlanGroupMin scenarios on, else one).
constexpr int kPlanGroups = 4;
constexpr int kPlanGroupMin = 8;

std::vector<std::pair<int, int>> plan_group_ranges(const Layout &L) {
    std::vector<std::pair<int, int>> out;
    const int G = L.n_scen >= kPlanGroupMin ? kPlanGroups : 1;
    std::vector<long long> tiles(L.n_scen, 0);
    long long total = 0;
    for (int q = 0; q < L.n_scen; ++q) {
        for (int p = L.pair0[q]; p < L.pair0[q + 1]; ++p) tiles[q] += (long long)L.pairs[p].tiles_a * L.pairs[p].tiles_b;
        total += tiles[q];
    }
    int s0 = 0;
    long long acc = 0;
    for (int q = 0; q < L.n_scen; ++q) {
        acc += tiles[q];
        const int g = (int)out.size();
        const bool last_group = g == G - 1;
        if (!last_group && (acc * G >= total * (g + 1)) && L.n_scen - (q + 1) >= G - 1 - g) {
            out.push_back({s0, q + 1 - s0});
            s0 = q + 1;
        }
    }
    if (s0 < L.n_scen) out.push_back({s0, L.n_scen - s0});
    return out;
}

// Device scratch of a plan: the batch as one launch sequence, or the pipeline's groups (their
// descriptors first, then each group's work scratch), whichever is larger.
size_t plan_scratch_bytes(const mhc_scenario *scens, const Layout &L, bool with_w) {
    const size_t single = scratch_of(L, with_w).total;
    const auto ranges = plan_group_ranges(L);
    if (ranges.size() <= 1) return single;
    size_t sum = 0;
    for (const auto &r : ranges) {
        Layout G;
        if (build_layout(scens + r.first, r.second, G) != MHC_OK) return single;
        sum += scratch_of(G, with_w).total + 2 * kAlign;
    }
    return std::max(single, sum);
}

// The plan's launch sequence on `st`: descriptor upload from the pinned copy, then the fused path.  A
// pipelined plan uploads every group's descriptors at once, then runs the groups alternately on `st` and
// the plan's second stream: group g's generation waits for group g - 1's generation only, and the rest of
// its sequence (risk preparation, bounds and the table's -1s, collision, risk walk) follows its own
// generation on its stream, so that one group's generation and table fill may run beside another group's
// collision kernel.  The end joins both streams on `st`.  Measured on the 256-scenario batch it is not
// faster (15.26 ms against 14.87 ms as graphs): the large-scene collision kernel holds every SM's
// register file, so the generation CTAs wait for its CTAs to retire; it stays an option (MHC_PLAN_PIPELINE).
int plan_enqueue(mhc_plan *p, cudaStream_t st) {
    MHC_CUDA(launch_copy(p->dev, p->host_dev, p->desc_bytes, st));
    if (p->groups.size() <= 1) {
        Bump bump{p->dev, p->dev_bytes, align_up(p->desc_bytes)};
        return launch_all(p->ctx, p->L, p->D, bump, &p->poses, &p->poses, p->table, true, &p->out, st, true, true);
    }
    cudaEvent_t fork = p->ev[0], join = p->ev[1];
    MHC_CUDA(cudaEventRecord(fork, st));
    MHC_CUDA(cudaStreamWaitEvent(p->side, fork, 0));
    for (size_t g = 0; g < p->groups.size(); ++g) {
        PlanGroup &G = p->groups[g];
        cudaStream_t sg = g % 2 == 0 ? st : p->side;
        if (g > 0) MHC_CUDA(cudaStreamWaitEvent(sg, p->ev[2 + g - 1], 0));
        Bump bump{G.work, G.work_bytes, 0};
        if (int r = launch_all(p->ctx, G.L, G.D, bump, &G.poses, nullptr, G.table, false, nullptr, sg, false)) return r;
        MHC_CUDA(cudaEventRecord(p->ev[2 + g], sg));
        if (int r = launch_all(p->ctx, G.L, G.D, bump, nullptr, &G.poses, G.table, true, &G.out, sg, true)) return r;
    }
    MHC_CUDA(cudaEventRecord(join, p->side));
    MHC_CUDA(cudaStreamWaitEvent(st, join, 0));
    return MHC_OK;
}

// The group's slices of the batch's buffers (scenario s0's offsets in the whole layout).
void group_slices(const mhc_plan *p, PlanGroup &G) {
    const Layout &L = p->L;
    const ScenDesc &S = L.scens[G.s0];
    const long long pose0 = L.objs[S.obj0].pose_base, entry0 = L.entry0[G.s0];
    const int pair0 = L.pair0[G.s0];
    const long long kofs0 = L.pair0[G.s0] < (int)L.pairs.size() ? L.pairs[pair0].kofs : L.n_kofs;
    const long long e0 = S.e_base, step0 = S.step_base, obj0 = S.obj0;
    G.poses.x = p->poses.x + pose0; G.poses.y = p->poses.y + pose0;
    G.poses.c = p->poses.c + pose0; G.poses.s = p->poses.s + pose0;
    G.table = p->table + entry0;
    const mhc_risk &o = p->out;
    mhc_risk &r = G.out;
    r = o;
    r.count = o.count + pair0; r.P = o.P + pair0;
    r.count_k = o.count_k + kofs0; r.H = o.H + kofs0;
    r.naive = o.naive + e0; r.cond = o.cond + e0; r.indep = o.indep + e0; r.hits = o.hits + e0;
    r.escape = o.escape + e0;
    r.attr_obj = o.attr_obj + obj0; r.attr_step = o.attr_step + step0;
    r.scalars = o.scalars + 4LL * G.s0; r.n_escape = o.n_escape + G.s0;
}

// Lays the plan's groups out (their layouts from `scens`) and packs their descriptors into `host` (the
// pinned copy, or null to size them).  Returns the descriptors' total bytes, or 0 on a layout error.
size_t plan_groups_pack(mhc_plan *p, const mhc_scenario *scens, const float *const *traj_weights, char *host,
                        bool keep_weights = false) {
    size_t off = 0;
    for (PlanGroup &G : p->groups) {
        if (build_layout(scens + G.s0, G.n, G.L) != MHC_OK) return 0;
        plan_generation(G.L, p->ctx->n_sm, p->ctx->gen_scan);
        const float *const *wg = traj_weights ? traj_weights + p->L.scens[G.s0].obj0 : nullptr;
        if (!keep_weights && gather_weights(G.L, wg, G.w) != MHC_OK) return 0;
        G.desc_off = off;
        G.desc_bytes = pack_descriptors(G.L, G.w.empty() ? nullptr : &G.w, host ? host + off : nullptr,
                                        p->dev + off, G.D);
        off = align_up(off + G.desc_bytes);
    }
    return off;
}

}  // namespace

extern "C" {

int mhc_batch_layout(const mhc_scenario *scens, int32_t n_scen, mhc_batch_info *info, mhc_batch_slice *slices) {
    Layout L;
    if (int r = build_layout(scens, n_scen, L)) return r;
    if (info) {
        std::memset(info, 0, sizeof *info);
        info->n_traj = L.n_traj;
        info->n_poses = L.n_pose;
        info->n_entries = L.n_entries;
        info->n_step_entries = L.n_kofs;
        info->n_scen_steps = L.n_steps_total;
        info->h_ego = L.h_e;
        info->n_pairs = (int32_t)L.pairs.size();
        info->n_objects = L.n_obj;
        info->n_scenarios = L.n_scen;
        info->max_steps = L.max_steps;
        info->scratch = kReserved + scratch_of(L, true).total;
        info->plan_bytes = plan_scratch_bytes(scens, L, true);
    }
    if (slices) {
        for (int s = 0; s < L.n_scen; ++s) {
            const ScenDesc &S = L.scens[s];
            mhc_batch_slice &q = slices[s];
            q.obj0 = S.obj0;
            q.n_objects = S.n_obj;
            q.pair0 = L.pair0[s];
            q.n_pairs = L.pair0[s + 1] - L.pair0[s];
            q.n_steps = S.n_steps;
            q.ego = S.ego - S.obj0;
            q.traj0 = L.objs[S.obj0].traj_off;
            q.pose0 = L.objs[S.obj0].pose_base;
            q.entry0 = L.entry0[s];
            q.step_entry0 = q.n_pairs ? L.pairs[q.pair0].kofs : 0;
            q.ego0 = S.e_base;
            q.step0 = S.step_base;
        }
    }
    return MHC_OK;
}

int mhc_batch_pair_table(const mhc_scenario *scens, int32_t n_scen, int32_t *pair_a, int32_t *pair_b,
                         int64_t *pair_off) {
    Layout L;
    if (int r = build_layout(scens, n_scen, L)) return r;
    for (size_t p = 0; p < L.pairs.size(); ++p) {
        if (pair_a) pair_a[p] = L.pairs[p].a;
        if (pair_b) pair_b[p] = L.pairs[p].b;
        if (pair_off) pair_off[p] = L.pairs[p].off;
    }
    if (pair_off) pair_off[L.pairs.size()] = L.n_entries;
    return MHC_OK;
}

int mhc_evaluate_batch(mhc_ctx *ctx, const mhc_scenario *scens, int32_t n_scen, const float *const *traj_weights,
                       const mhc_poses *poses, int16_t *table, const mhc_risk *out, void *stream) {
    return evaluate_impl(ctx, scens, n_scen, traj_weights, poses, table, out, stream);
}

int mhc_autotune_batch(mhc_ctx *ctx, const mhc_scenario *scens, int32_t n_scen, const mhc_poses *poses,
                       int16_t *table, int fused, int32_t *best_variant, int32_t *best_cull, void *stream) {
    return autotune_impl(ctx, scens, n_scen, poses, table, fused, best_variant, best_cull, stream);
}

void mhc_plan_destroy(mhc_plan *p) {
    if (!p) return;
    if (p->ctx) cudaSetDevice(p->ctx->device);
    if (p->done) { cudaEventSynchronize(p->done); cudaEventDestroy(p->done); }
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    for (cudaEvent_t e : p->ev) if (e) cudaEventDestroy(e);
    if (p->side) cudaStreamDestroy(p->side);
    if (p->cap) cudaStreamDestroy(p->cap);
    if (p->host) cudaFreeHost(p->host);
    delete p;
}

int mhc_plan_create(mhc_ctx *ctx, const mhc_scenario *scens, int32_t n_scen, const float *const *traj_weights,
                    const mhc_poses *poses, int16_t *table, const mhc_risk *out, void *scratch,
                    size_t scratch_bytes, int32_t flags, mhc_plan **plan) {
    if (!plan) return fail(MHC_E_INVALID, "plan is NULL");
    *plan = nullptr;
    if (int r = check_ctx(ctx)) return r;
    if (!poses || !poses->x || !poses->y || !poses->c || !poses->s || !table || !out || !scratch)
        return fail(MHC_E_INVALID, "poses, table, out and scratch must be non-NULL");
    if (reinterpret_cast<uintptr_t>(scratch) % kAlign) return fail(MHC_E_INVALID, "scratch must be 256-byte aligned");
    if (int r = check_device_arrays(poses, table, out)) return r;
    if (flags & ~(MHC_PLAN_GRAPH | MHC_PLAN_PIPELINE)) return fail(MHC_E_INVALID, "unknown plan flags");
    mhc_plan *p = new mhc_plan();
    p->ctx = ctx;
    int rc = build_layout(scens, n_scen, p->L);
    if (rc == MHC_OK) rc = gather_weights(p->L, traj_weights, p->w);
    if (rc != MHC_OK) { delete p; return rc; }
    plan_generation(p->L, ctx->n_sm, ctx->gen_scan);
    p->has_w = !p->w.empty();
    p->dev = static_cast<char *>(scratch);
    p->dev_bytes = scratch_bytes;
    p->poses = *poses;
    p->table = table;
    p->out = *out;
    if (flags & MHC_PLAN_PIPELINE) {
        const auto ranges = plan_group_ranges(p->L);
        if (ranges.size() > 1)
            for (const auto &r : ranges) {
                PlanGroup G;
                G.s0 = r.first;
                G.n = r.second;
                p->groups.push_back(std::move(G));
            }
    }
    if (p->groups.size() > 1) {   // the pipeline: descriptors of every group first, then each group's work scratch
        const size_t desc = plan_groups_pack(p, scens, traj_weights, nullptr);
        if (!desc) { delete p; return fail(MHC_E_INVALID, "plan group layout failed"); }
        size_t off = desc;
        for (PlanGroup &G : p->groups) {
            const Scratch SG = scratch_of(G.L, !G.w.empty());
            G.work = p->dev + off;
            G.work_bytes = SG.total - SG.desc - SG.weights + 2 * kAlign;
            off = align_up(off + G.work_bytes);
            group_slices(p, G);
        }
        if (scratch_bytes < off) {
            delete p;
            return fail(MHC_E_NOMEM, "plan scratch smaller than mhc_batch_info.plan_bytes");
        }
        p->desc_bytes = desc;
    } else {
        p->groups.clear();
        const Scratch S = scratch_of(p->L, p->has_w);
        if (scratch_bytes < S.total) {
            delete p;
            return fail(MHC_E_NOMEM, "plan scratch smaller than mhc_batch_info.plan_bytes");
        }
        p->desc_bytes = pack_descriptors(p->L, p->has_w ? &p->w : nullptr, nullptr, p->dev, p->D);
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e == cudaSuccess) e = alloc_mapped(p->desc_bytes, &p->host, &p->host_dev);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess && p->groups.size() > 1) {
        e = cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking);
        p->ev.assign(2 + p->groups.size(), nullptr);
        for (size_t q = 0; q < p->ev.size() && e == cudaSuccess; ++q)
            e = cudaEventCreateWithFlags(&p->ev[q], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) { mhc_plan_destroy(p); return cuda_fail(e, "plan set-up"); }
    if (p->groups.size() > 1) plan_groups_pack(p, scens, traj_weights, p->host);
    else pack_descriptors(p->L, p->has_w ? &p->w : nullptr, p->host, p->dev, p->D);
    if (flags & MHC_PLAN_GRAPH) {
        // one un-captured pass first (kernel attributes are set outside the capture), then the capture;
        // the context's profiling events stay out of the graph
        const bool prof = ctx->profile;
        ctx->profile = false;
        rc = plan_enqueue(p, p->cap);
        if (rc == MHC_OK) {
            e = cudaStreamSynchronize(p->cap);
            if (e != cudaSuccess) rc = cuda_fail(e, "plan warm-up");
        }
        if (rc == MHC_OK) {
            e = cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) rc = cuda_fail(e, "cudaStreamBeginCapture");
        }
        if (rc == MHC_OK) {
            const int rq = plan_enqueue(p, p->cap);
            cudaGraph_t g = nullptr;
            e = cudaStreamEndCapture(p->cap, &g);
            p->graph = g;
            if (rq != MHC_OK) rc = rq;
            else if (e != cudaSuccess) rc = cuda_fail(e, "cudaStreamEndCapture");
        }
        if (rc == MHC_OK) {
            e = cudaGraphInstantiate(&p->exec, p->graph, 0);
            if (e != cudaSuccess) rc = cuda_fail(e, "cudaGraphInstantiate");
        }
        ctx->profile = prof;
        if (rc != MHC_OK) { mhc_plan_destroy(p); return rc; }
    }
    *plan = p;
    return MHC_OK;
}

int mhc_plan_update(mhc_plan *p, const mhc_scenario *scens, int32_t n_scen) {
    if (!p) return fail(MHC_E_INVALID, "plan is NULL");
    Layout L;
    if (int r = build_layout(scens, n_scen, L)) return r;
    if (!same_structure(L, p->L)) return fail(MHC_E_INVALID, "scenarios differ from the plan's in structure");
    plan_generation(L, p->ctx->n_sm, p->ctx->gen_scan);
    MHC_CUDA(cudaSetDevice(p->ctx->device));
    if (p->launched) MHC_CUDA(cudaEventSynchronize(p->done));   // the previous launch has read the copy
    p->L = std::move(L);
    if (p->groups.size() > 1) {   // the groups keep their structure with the batch's; only their contents change
        if (!plan_groups_pack(p, scens, nullptr, p->host, true)) return fail(MHC_E_INVALID, "plan group layout failed");
        return MHC_OK;
    }
    DevDesc D;
    pack_descriptors(p->L, p->has_w ? &p->w : nullptr, p->host, p->dev, D);
    return MHC_OK;
}

int mhc_plan_launch(mhc_plan *p, void *stream) {
    if (!p) return fail(MHC_E_INVALID, "plan is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    MHC_CUDA(cudaSetDevice(p->ctx->device));
    if (p->launched) MHC_CUDA(cudaStreamWaitEvent(st, p->done, 0));   // launches of a plan never overlap
    if (p->exec) {
        MHC_CUDA(cudaGraphLaunch(p->exec, st));
    } else {
        if (int r = plan_enqueue(p, st)) return r;
    }
    MHC_CUDA(cudaEventRecord(p->done, st));
    p->launched = true;
    p->ctx->h2d = (long long)p->desc_bytes;
    p->ctx->d2h = 0;
    return MHC_OK;
}

}  // extern "C"
