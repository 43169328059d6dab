// runtime.h -- host runtime shared by the C-ABI entry points (api.cu, plan.cu, serve.cu): the batch
// layout of scenarios, the context, the arena bump allocator, descriptor upload and the launch sequence.
#pragma once
#include <cmath>
#include <string>
#include <vector>

#include "../../include/mhc.h"
#include "mhc_internal.cuh"

namespace mhc {
namespace host {

int fail(int code, const std::string &why);
int check_device_arrays(const mhc_poses *p, const int16_t *table, const mhc_risk *r);
// Copies `bytes` with a kernel on `st` between addresses the device can use (device memory or the device
// address of mapped pinned host memory), both 16-byte aligned.  pdl: launched as a programmatic dependent
// of the kernel just before it on `st` (the copy waits for that kernel before it reads).
cudaError_t launch_copy(void *dst, const void *src, size_t bytes, cudaStream_t st, bool pdl = false);
// Mapped pinned host memory: its host address and the address kernels use.
cudaError_t alloc_mapped(size_t bytes, char **host, char **dev);
int cuda_fail(cudaError_t e, const char *what);

#define MHC_CUDA(call)                                            \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return ::mhc::host::cuda_fail(e_, #call); \
    } while (0)

constexpr size_t kAlign = 256;
constexpr size_t kReserved = 4096;    // persistent words at the start of the arena (counters)
constexpr int kSlots = 4;
constexpr long long kFillInCollideMax = 1LL << 25;   // table entries up to which the collision kernel fills
constexpr long long kItemsMax = 1LL << 22;             // step items (8 B each) up to which variant 6 applies
constexpr long long kItemsMaxEntries = 1LL << 26;      // and table entries (4 B of first-step scratch each)
constexpr long long kBlockListMax = 1LL << 19;         // 32 x 32 blocks (128 B records) up to which variant 8 applies

// The object fields a pair descriptor carries for the collision kernels.
inline void copy_object_fields(PairDesc &p, const ObjDesc &A, const ObjDesc &B) {
    p.pose_a = A.pose_base; p.pose_b = B.pose_base;
    p.bounds_a = A.bounds_base; p.bounds_b = B.bounds_base;
    p.traj_a = A.traj_off; p.traj_b = B.traj_off;
    p.h_a = A.h; p.h_b = B.h;
    p.hl_a = A.hl; p.hw_a = A.hw; p.rad_a = A.rad;
    p.hl_b = B.hl; p.hw_b = B.hw; p.rad_b = B.rad;
}
constexpr long long kGenScanMaxTraj = 4096;           // a scenario's hypotheses up to which generation is parallel in time

inline size_t align_up(size_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }
inline bool finite(float v) { return std::isfinite(v); }

// Host-side layout of a batch of scenarios (one scenario is a batch of one): every descriptor the
// kernels read.  Objects, pairs, hypotheses, poses, table entries and per-step outputs of the scenarios
// are concatenated in batch order; each descriptor carries its scenario's horizon and accumulator bases.
struct Layout {
    int n_obj = 0, n_scen = 0, max_steps = 0;
    std::vector<ObjDesc> objs;
    std::vector<PairDesc> pairs;
    std::vector<PairDesc> pairs_c;                   // the same in collision-grid order (closest pairs first)
    std::vector<ScenDesc> scens;
    std::vector<float> grids;
    std::vector<Regime> regimes;                     // per vehicle and acceleration value
    std::vector<PolyVertex> polys;                   // vehicles' outlines in scenarios that have convex outlines
    std::vector<float> paths;                        // path sections of the vehicles that follow paths
    std::vector<int> warp_obj, warp_first;          // 32-hypothesis bound tiles
    std::vector<int> gen_obj, gen_first;            // generation tasks: n_gen_scan_objs (object, first warp)
                                                     // ranges of a warp per hypothesis, then (object, first
                                                     // hypothesis) tasks of gen_lanes hypotheses
    std::vector<int> pair0;                         // first pair of each scenario (n_scen + 1 entries)
    std::vector<long long> entry0;                  // first table entry of each scenario
    int gen_lanes = 32;
    int n_gen_scan = 0;                              // the first n_gen_scan generation warps: a warp per hypothesis
    int n_gen_scan_objs = 0;                         // objects those warps cover
    int n_gen_warps = 0;                             // generation warps in all
    long long n_traj = 0, n_pose = 0, n_entries = 0, n_tiles = 0, n_bounds = 0;
    long long h_e = 0, n_kofs = 0, n_steps_total = 0, n_lsum = 0, n_mass = 0;
    int n_tiles32 = 0;
};

int build_layout(const mhc_scenario *sc, int n_scen, Layout &L);
int build_layout(const mhc_scenario *sc, Layout &L);
void plan_generation(Layout &L, int n_sm, int mode);   // mode: MHC_OPT_GEN_SCAN
long long acc_words(const Layout &L);
bool items_eligible(const Layout &L);

// Device scratch each call needs (besides caller buffers).
struct Scratch {
    size_t desc = 0, bounds = 0, prob = 0, acc = 0, weights = 0, items = 0, total = 0;
    long long acc_words = 0;
};

Scratch scratch_of(const Layout &L, bool with_weights);

// Bump allocator over the arena for one call.
struct Bump {
    char *base;
    size_t cap, off;
    void *take(size_t n) {
        n = align_up(n);
        if (off + n > cap) return nullptr;
        void *p = base + off;
        off += n;
        return p;
    }
};

// Pack the descriptors into a mapped pinned staging slot and copy them to `dev` on `st` with the copy kernel.
struct DevDesc {
    ObjDesc *objs;
    PairDesc *pairs;
    PairDesc *pairs_c;
    ScenDesc *scens;
    float *grids;
    int *warp_obj, *warp_first;
    int *gen_obj, *gen_first;
    Regime *regimes;
    PolyVertex *polys;       // null when the batch has no outlines
    float *paths;            // null when no vehicle follows paths
    float *weights;
};


}  // namespace host
}  // namespace mhc

struct mhc_ctx {
    int device = 0;
    char *arena = nullptr;
    size_t arena_bytes = 0;
    bool owns = false;
    char *stage[mhc::host::kSlots] = {};
    char *stage_dev[mhc::host::kSlots] = {};     // the same buffers as kernels address them (mapped)
    size_t stage_cap[mhc::host::kSlots] = {};
    cudaEvent_t stage_ev[mhc::host::kSlots] = {};
    int slot = 0;
    cudaEvent_t done_ev = nullptr;
    cudaStream_t last_stream = nullptr;
    bool has_last = false;
    int cull = 1;
    int variant = 0;
    int collide_max_ctas = 0;        // > 0: CTA cap of the warp-per-block collision layouts (serving's large lane)
    int gen_scan = 2;
    bool score = false;                            // MHC_OPT_SCORE                // generation: 1 a warp per hypothesis (parallel in time), 0 a thread each, 2 auto
    int n_sm = 152;
    // autotuned collision configuration per size class (log2 of the tile count, log2 of the steps)
    struct Tuned { int tiles_log2, steps_log2, fused, variant, cull; };
    std::vector<Tuned> tuned;
    unsigned long long *counters = nullptr;
    // kernel timing
    bool profile = false;
    struct Timed { cudaEvent_t a, b; int kind; int launches; };
    std::vector<Timed> timed;
    std::vector<cudaEvent_t> ev_pool;
    double prof_ms[MHC_K_COUNT] = {};
    long long prof_n[MHC_K_COUNT] = {};
    long long h2d = 0, d2h = 0;
    void *server = nullptr;          // the serving loop (serve.cu), if started
    char *out_stage = nullptr;       // mapped pinned staging of mhc_run's outputs
    char *out_stage_dev = nullptr;   // its device address
    size_t out_stage_cap = 0;
};

namespace mhc {
namespace host {

cudaEvent_t pooled_event(mhc_ctx *ctx);

// Records an event pair around the launches made in its scope when profiling is on.
struct TimedScope {
    mhc_ctx *ctx;
    cudaStream_t st;
    int kind, launches;
    cudaEvent_t a = nullptr;
    TimedScope(mhc_ctx *c, cudaStream_t s, int k, int n) : ctx(c), st(s), kind(k), launches(n) {
        if (ctx->profile && (a = pooled_event(ctx))) cudaEventRecord(a, st);
    }
    ~TimedScope() {
        if (!a) return;
        cudaEvent_t b = pooled_event(ctx);
        if (!b) { ctx->ev_pool.push_back(a); return; }
        cudaEventRecord(b, st);
        ctx->timed.push_back({a, b, kind, launches});
    }
};

int begin_call(mhc_ctx *ctx, cudaStream_t st);
int end_call(mhc_ctx *ctx, cudaStream_t st);
int check_ctx(mhc_ctx *ctx);
// Packs every descriptor (and the weights) into `host` (if non-null) laid out as at `dev`; fills `out` with
// the device addresses and returns the bytes.
size_t pack_descriptors(const Layout &L, const std::vector<float> *weights, char *host, char *dev, DevDesc &out);
int upload(mhc_ctx *ctx, const Layout &L, const std::vector<float> *weights, char *dev, cudaStream_t st,
           DevDesc &out);
int gather_weights(const Layout &L, const float *const *w, std::vector<float> &out);
int make_risk_args(const Layout &L, const DevDesc &D, Bump &bump, const int16_t *table, const mhc_risk *rout,
                   RiskArgs &r);
int log2_floor(long long v);
void pick_collide_config(const mhc_ctx *ctx, const Layout &L, bool fused, int &variant, int &cull);
bool take_risk_outputs(Bump &bump, const Layout &L, mhc_risk &R);
size_t risk_output_bytes(const Layout &L);
int launch_all(mhc_ctx *ctx, const Layout &L, const DevDesc &D, Bump &bump, const mhc_poses *gen_out,
               const mhc_poses *coll_in, int16_t *table, bool risk, const mhc_risk *rout, cudaStream_t st,
               bool fused = false, bool after_upload = false);
// after_upload: the last operation on `st` is the descriptor copy kernel (launch_copy), so the generation
// kernel may be a programmatic dependent launch of it
int evaluate_impl(mhc_ctx *ctx, const mhc_scenario *scen, int n_scen, const float *const *traj_weights,
                  const mhc_poses *poses, int16_t *table, const mhc_risk *out, void *stream);
int autotune_impl(mhc_ctx *ctx, const mhc_scenario *scen, int n_scen, const mhc_poses *poses, int16_t *table,
                  int fused, int32_t *best_variant, int32_t *best_cull, void *stream);

// first-fit allocator of pool.cu
bool pool_alloc(mhc_pool *p, size_t bytes, size_t *offset);
bool pool_free(mhc_pool *p, size_t offset);
size_t pool_largest(const mhc_pool *p);
size_t pool_free_bytes(const mhc_pool *p);
mhc_pool *pool_new(size_t bytes);
void pool_delete(mhc_pool *p);
void serve_shutdown(mhc_ctx *ctx);   // stops the serving loop of ctx (serve.cu)

}  // namespace host
}  // namespace mhc
