// batch.cu -- batches of uneven scenarios in one launch sequence, and plans: a batch whose descriptors
// live in caller-owned device scratch and whose launch sequence is captured once as a CUDA graph and
// replayed (new initial states are written into the plan's pinned copy of the descriptors between
// replays).  The kernels are those of the single-scenario path; every descriptor carries its scenario's
// horizon and accumulator bases, so a batch is one generation launch over all hypotheses, one collision
// launch over all tiles of all pairs and one risk walk over all EGO hypotheses.
#include <cstring>

#include "runtime.h"

using namespace mhc;
using namespace mhc::host;

struct mhc_plan {
    mhc_ctx *ctx = nullptr;
    Layout L;
    std::vector<float> w;
    bool has_w = false;
    char *dev = nullptr;               // caller's device scratch
    size_t dev_bytes = 0;
    char *host = nullptr;              // pinned copy of the descriptors (source of each launch's upload)
    size_t desc_bytes = 0;
    DevDesc D{};
    mhc_poses poses{};
    int16_t *table = nullptr;
    mhc_risk out{};
    cudaStream_t cap = nullptr;        // capture stream
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

// The plan's launch sequence on `st`: descriptor upload from the pinned copy, then the fused path.
int plan_enqueue(mhc_plan *p, cudaStream_t st) {
    MHC_CUDA(cudaMemcpyAsync(p->dev, p->host, p->desc_bytes, cudaMemcpyHostToDevice, st));
    Bump bump{p->dev, p->dev_bytes, align_up(p->desc_bytes)};
    return launch_all(p->ctx, p->L, p->D, bump, &p->poses, &p->poses, p->table, true, &p->out, st, true);
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
        info->plan_bytes = scratch_of(L, true).total;
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
    if (flags & ~MHC_PLAN_GRAPH) return fail(MHC_E_INVALID, "unknown plan flags");
    mhc_plan *p = new mhc_plan();
    p->ctx = ctx;
    int rc = build_layout(scens, n_scen, p->L);
    if (rc == MHC_OK) rc = gather_weights(p->L, traj_weights, p->w);
    if (rc != MHC_OK) { delete p; return rc; }
    plan_generation(p->L, ctx->n_sm, ctx->gen_scan);
    p->has_w = !p->w.empty();
    const Scratch S = scratch_of(p->L, p->has_w);
    if (scratch_bytes < S.total) {
        delete p;
        return fail(MHC_E_NOMEM, "plan scratch smaller than mhc_batch_info.plan_bytes");
    }
    p->dev = static_cast<char *>(scratch);
    p->dev_bytes = scratch_bytes;
    p->desc_bytes = pack_descriptors(p->L, p->has_w ? &p->w : nullptr, nullptr, p->dev, p->D);
    p->poses = *poses;
    p->table = table;
    p->out = *out;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void **>(&p->host), p->desc_bytes, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) { mhc_plan_destroy(p); return cuda_fail(e, "plan set-up"); }
    pack_descriptors(p->L, p->has_w ? &p->w : nullptr, p->host, p->dev, p->D);
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
