// mhc_internal.cuh -- device descriptors and launch interfaces shared by the library's translation units.
//
// Layouts (all in the context arena unless the caller passes buffers):
//   poses   SoA planes x, y, c, s; pose (object a, step k, hypothesis i) at N * traj_off[a] + k * h_a + i.
//   table   int16, pair p block of h_a x h_b at pair_off[p], row-major (row = hypothesis of a).
//   bounds  per 32-hypothesis tile of an object and per step: float4 {xmin, ymin, xmax, ymax} of the
//           tile's pose centres, at (tile_base[a] + tile) * N + k.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mhc {

constexpr int kVehicle = 0;
constexpr int kPedestrian = 1;
constexpr int kModelOT = 0;
constexpr int kModelKin = 1;
constexpr int kPedAccelGrid = 1;
constexpr float kVMin = 2.0f;      // below this speed the one-track model gives way to its kinematic limit
constexpr double kVMinD = 2.0;

constexpr int kTile = 64;           // collision tile edge (hypotheses per side)
constexpr int kCollideVariants = 8; // thread layouts of the collision kernel (MHC_OPT_COLLIDE_VARIANT 1..8)
constexpr int kBoundTile = 32;     // hypotheses per bounding-box tile (one warp)
constexpr int16_t kNoHit = 0x7fff; // in-kernel sentinel, stored as -1

// Per-object descriptor (device).  Objects of every scenario of a batch are listed one after another.
struct ObjDesc {
    int kind, flags, n_a, n_b;
    int h;              // hypotheses n_a * n_b
    int grid_off;       // grid_a at grids[grid_off], grid_b right after
    int tile_base;      // first 32-wide bound tile of this object
    int n_tiles32;
    long long traj_off; // global index of hypothesis 0
    long long pose_base;// first pose: poses of the object are [step][hypothesis] from here
    long long bounds_base;  // first bound box: [tile][step] from here
    float hl, hw, rad;  // half length, half width, disc radius
    float circ;         // circumradius about the pose point
    float x0, y0, psi0, v0, v_max;
    float m, Iz, lf, lr, caf, car;
    // the object's scenario
    int scen;           // scenario index in the batch
    int n_steps, substeps, model;
    float tau;
    int regime_off;     // vehicles: the speed regimes of grid_a[0..n_a) at regimes[regime_off ..]
    double tau_i_d;     // (double)tau / substeps, the sub-step of the speed recurrence
    int poly_off;       // vehicles of scenarios with convex outlines: the outline's vertices at
    int n_poly;         // polys[poly_off .. + n_poly) (a rectangle as its 4 corners); n_poly = 0 otherwise
    int path_off;       // vehicles with paths: path i_b's three sections (x, y, psi) at paths[9 (path_off +
                        // i_b) ..]; -1 for constant steering angles
    int path_n1, path_n2;   // the first sub-steps of the second and third sections (t >= 1.0 s, t >= 1.5 s)
};

// One vertex of a convex outline in the body frame with the outward unit normal of the edge to the next
// vertex (counter-clockwise order): {x, y, n_x, n_y}.
using PolyVertex = float4;

// Per-object-pair descriptor (device).
struct PairDesc {
    int a, b;                 // global object indices
    int tiles_a, tiles_b;     // 64-wide tiles along each side
    long long off;            // table offset of the pair's block
    long long tile_start;     // first global collision tile of this pair
    float rc2;                // (R_a + R_b)^2, R = circumradius about the pose point
    float r_cull;             // R_a + R_b plus a margin, for bounding-box culling
    int combo;                // 0 rect-rect, 1 rect(a)-disc(b), 2 disc(a)-rect(b), 3 disc-disc,
                              // 4 outline-outline, 5 outline(a)-disc(b), 6 disc(a)-outline(b)
    int ego_side;             // 0: a is its scenario's EGO object, 1: b is, -1: neither
    int n_steps;              // steps of the pair's scenario
    int scen;
    long long kofs;           // first of the pair's n_steps entries in the per-step outputs (count_k, H)
    // accumulators of the scenario's EGO hypotheses (used when ego_side >= 0)
    long long lsum_base;      // cells [EGO hypothesis][step][CO object of the scenario]
    long long mass_base;      // [EGO hypothesis][CO object of the scenario]
    long long hits_base;      // [EGO hypothesis]
    int n_obj_s;              // objects in the scenario
    int co_local;             // the CO object's index in its scenario
    int index;                // the pair's position in table order (per-pair outputs count, P)
    int poly_a, nv_a;         // combos 4..6: the outlines' vertices (ObjDesc::poly_off, n_poly)
    int poly_b, nv_b;
    int pad_;
    // copies of the two objects' fields the collision kernels read (one load less on their chain)
    long long pose_a, pose_b;     // ObjDesc::pose_base
    long long bounds_a, bounds_b; // ObjDesc::bounds_base
    long long traj_a, traj_b;     // ObjDesc::traj_off
    int h_a, h_b;                 // hypotheses
    float hl_a, hw_a, rad_a, hl_b, hw_b, rad_b;   // half extents, disc radii
};

// Per-scenario descriptor of a batch (device; risk stage).
struct ScenDesc {
    int ego;                  // global object index of the EGO object
    int n_obj, n_steps, h_e;
    int obj0;                 // global index of the scenario's first object
    int pad_;
    long long e_base;         // first global EGO hypothesis (per-EGO-hypothesis outputs, hits)
    long long lsum_base, mass_base;
    long long step_base;      // the scenario's n_steps entries of attr_step
    long long e_traj;         // global index of the EGO object's hypothesis 0 (its probabilities)
};

// Sub-steps of a vehicle hypothesis's low-speed regime [low_lo, low_hi) and its stop sub-step (n_stop = N K
// if it never stops), decided on the FP64 speed v_0 + n vdot tau_i; one entry per acceleration value.
struct Regime {
    int low_lo, low_hi, n_stop, pad_;
};

// The risk preparation (prepare.cuh): accumulators to zero, escape lists to fill, weights to normalise.
struct PrepArgs {
    unsigned long long *base;      // accumulator words to zero
    long long n_words;
    int *escape;                   // [h_e] escape lists (may be null)
    long long h_e;
    const ObjDesc *objs;
    int n_obj;
    const float *weights;          // [n_traj] raw weights, or null for uniform (or scored)
    double *prob;                  // [n_traj] normalised probabilities
    float *probf;                  // [n_traj] the same rounded to FP32
    unsigned long long *pfix;      // [n_traj] or null: to_fixed(probf, kFixProb)
    unsigned long long *lfix;      // [n_traj] or null: to_fixed(neg_log_survival(probf), kFixLog)
    int score;                     // no weights: 1 scores every hypothesis by Eq. normTraj, 0 uniform
    const float *grids;            // the hypothesis grids and paths the scores read
    const float *paths;
};

struct GenArgs {
    const ObjDesc *objs;
    const Regime *regimes;
    const float *grids;
    const int *warp_obj;      // object of each warp task
    const int *warp_first;    // first hypothesis of each warp task
    int n_warps;
    int lanes;                // hypotheses per warp task (1..32): fewer than 32 spreads small workloads
                              // over more warp schedulers, since each hypothesis is a sequential chain
    int gen_blocks;           // set by launch_generate: CTAs of the generation tasks
    int prep_blocks;          // > 0: that many further CTAs run the risk preparation `prep` (fused path)
    PrepArgs prep;
    int n_scan;               // warps [0, n_scan): one hypothesis each, parallel in time: warp w belongs to
                              // the last entry k < n_scan_objs with warp_first[k] <= w (object warp_obj[k],
                              // hypothesis w - warp_first[k]); warp w >= n_scan: entry n_scan_objs + w -
                              // n_scan, `lanes` hypotheses from warp_first of object warp_obj, a thread each
    int n_scan_objs;
    const float *paths;       // path sections of the vehicles that follow paths (ObjDesc::path_off)
    float *x, *y, *c, *s;
    int16_t *fill;            // if set: the launch's first fill_blocks CTAs write table[0, n_fill) = -1
    long long n_fill;
    int fill_blocks;          // set by launch_generate
};

struct BoundsArgs {
    const ObjDesc *objs;
    const int *warp_obj, *warp_first;
    int n_warps, max_steps;   // grid covers n_warps x max_steps; steps beyond an object's own are skipped
    const float *x, *y;
    float4 *bounds;
    unsigned long long *zero_counts;   // if set: two words zeroed after the wait (the step-item counters)
    int16_t *fill;            // if set: further CTAs of the launch write table[0, n_fill) = -1 (no collision)
    long long n_fill;
};

// Risk accumulators: one contiguous block of 64-bit words, zeroed before every assessment.  Masses and
// log-survival sums are unsigned fixed point (kFixProb / kFixLog fractional bits): every term is an FP32
// value converted exactly, and integer atomics add them exactly and in any order.
// Programmatic dependent launch.  Every kernel of the library starts with pdl_start(): it lets the next
// kernel of the stream be scheduled as soon as every block of this one is running, then waits until the
// previous kernel of the stream has completed and its writes are visible (a no-op for a kernel launched
// without the attribute).  A dependent's blocks thus sit resident, waiting, while its predecessor's tail
// runs, instead of being launched after it ends.  Because every block waits first, a kernel completes only
// after its predecessor did, so the ordering stays transitive along the chain.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_start() {
    pdl_trigger();
    pdl_wait();
}
// Between pdl_trigger() and pdl_wait() a kernel may read only what was in memory before the first kernel
// of its chain began (the uploaded descriptors): the first kernel after a copy is launched in plain stream
// order, so every later kernel starts after that copy completed.

// kernel<<<grid, block, smem, st>>>(args...), with programmatic stream serialization when pdl is set.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_kernel(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                 bool pdl, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

constexpr int kFixProb = 62;   // probability masses: every accumulated sum is at most 1
constexpr int kFixLog = 40;    // sums of -log(1 - p): each term capped at 2^22

struct RiskScratch {
    unsigned long long *count;     // [n_pairs]
    unsigned long long *count_k;   // [sum over pairs of N]           (per pair at PairDesc::kofs)
    unsigned long long *P, *H;     // [n_pairs], [sum over pairs of N] sum p_a[i] p_b[j]
    unsigned long long *hits;      // [sum h_e]                        colliding (b, j) per EGO hypothesis
    unsigned long long *lsum;      // [sum h_e N n_obj]                sum -log(1 - p_b[j]) per (i, k, b) cell
    unsigned long long *mass;      // [sum h_e n_obj]                  sum p_b[j] per (i, b)
    unsigned long long *attr_obj;  // [total objects]
    unsigned long long *attr_step; // [sum over scenarios of N]
    double *scalars;               // [4 per scenario]
    unsigned long long *n_escape;  // [per scenario] collision-free EGO hypotheses
    unsigned long long *done;      // [1] EGO-walk CTAs finished (the last one converts the totals)
    unsigned long long *base;      // first word of the block
    long long n_words;             // words to zero
};

// A 32 x 32 block of the step-item layout (variant 6) with active steps, recorded by the listing kernel so
// that an item (and the table kernel) needs no descriptor search: table entry (i, j) of the block at
// entry0 + i h_b + j, the pair's squared circumradius sum, the two shapes' half extents and radii, and the
// block's origin in its pair.
struct __align__(16) ItemBlock {
    long long entry0;
    int h_b, pair, rows, cols;
    float rc2, la, wa, ra, lb, wb, rb;
    int i0, j0;               // the block's first row and column within its pair
};

// A 32 x 32 block with at least one active step, recorded by the listing kernel of the block-list layout
// (variant 8) with everything its block kernel needs but the pair's risk fields: table entry (i, j) of the
// block at entry0 + i h_b + j, pose (k, i) of its row object at pose_a + k h_a + i (columns alike), its two
// bound tiles' boxes of step k at bounds_a + k and bounds_b + k, the shapes, and the first 32-step chunk
// with an active step (steps k0 .. k0 + 31, active ones in `mask`).
struct __align__(16) ActiveBlock {
    long long entry0, pose_a, pose_b, bounds_a, bounds_b, traj_a, traj_b;
    int h_a, h_b, n_steps, pair, rows, cols, i0, j0;
    float rcull, rc2, la, wa, ra, lb, wb, rb;
    int k0;
    unsigned mask;
};

// One item of the step-item layout: an active step k of block gw, with the pose indices of the step's first
// row of A and first column of B (pa = pose_a + k h_a, pb = pose_b + k h_b), so that its poses are one
// load away from the item.
struct StepItem {
    long long pa, pb;
    int gw, k;
};

struct CollideArgs {
    const ObjDesc *objs;
    const PairDesc *pairs;    // in collision-grid order (tile_start over that order; index = table order)
    int n_pairs;
    int n_obj;                // objects (the descriptors at objs)
    long long n_tiles;        // total collision tiles over all pairs
    int max_steps;            // the longest horizon of the batch (sizes the per-CTA accumulators)
    int cull;                 // 1: skip steps whose tile bounding boxes cannot meet
    int fill_blocks;          // 1: each warp writes -1 to its own block first (variant 5; no fill launch)
    int max_ctas;             // > 0: at most this many CTAs for variants 4, 5 (the warps loop over the blocks)
    // variant 6: the item list (active (block, step) pairs) and its length, zeroed by the caller
    StepItem *items;
    unsigned long long *item_count;
    int *first32;             // [n_entries] first overlapping step per table entry (INT_MAX: none)
    int *active;              // [4 n_tiles] blocks with at least one active step, and their number (zeroed)
    ItemBlock *blocks;        // [4 n_tiles] the records of the active blocks (indexed by block)
    unsigned long long *active_count;
    ActiveBlock *recs;        // variant 8: [4 n_tiles] the records of the active blocks ([*active_count] valid)
    long long max_items;      // capacity: 4 n_tiles x max_steps
    int variant;              // 1: 256 threads x 4 x 4, 2: 64 threads x 8 x 8, 3: warp per step, 4: warp per tile,
                              // 5: warp per quarter tile, 6: step items, 7: CTA per quarter tile,
                              // 8: CTA per listed active quarter tile
    const float *x, *y, *c, *s;
    const float4 *bounds;
    const PolyVertex *polys;       // convex outlines (pairs of combo 4..6), or null when there are none
    int16_t *table;
    unsigned long long *counters;  // optional: [0] broad-phase tests executed, [1] narrow-phase tests,
                                   // [2 .. 6] narrow-phase tests by shape class (collide.cu narrow_class)
    // fused risk accumulation at first-hit time (probf null: table only)
    const float *probf;            // [n_traj] FP32 probabilities
    const unsigned long long *pfix, *lfix;   // [n_traj] the same and -log(1 - p) in fixed point
    RiskScratch acc;               // accumulators, zeroed beforehand
};

struct RiskArgs {
    const ObjDesc *objs;
    const PairDesc *pairs;
    const ScenDesc *scens;
    int n_pairs, n_obj, n_scen;
    long long h_e;                 // EGO hypotheses over all scenarios
    long long n_kofs, n_steps_total;   // per-pair step entries, per-scenario step entries
    int max_steps;                 // the longest horizon of the batch
    int convert_in_walk;           // set by launch_risk_tail: the EGO walk's last CTA converts the totals
    long long n_tiles;
    const int16_t *table;
    const float *weights;          // [n_traj] raw non-negative weights, or null for uniform (or scored)
    int score;                     // no weights: score the hypotheses by Eq. normTraj (prepare.cuh)
    const float *grids, *paths;
    double *prob;                  // [n_traj] normalised probabilities (scratch)
    float *probf;                  // [n_traj] the same rounded to FP32 (the per-hit arithmetic)
    unsigned long long *pfix;      // [n_traj] each probability in fixed point (kFixProb)
    unsigned long long *lfix;      // [n_traj] each -log(1 - p) in fixed point (kFixLog)
    RiskScratch acc;
    // outputs (device); any may be null
    long long *count, *count_k;
    double *P, *H;
    double *naive, *cond, *indep;
    int *hits;
    double *attr_obj, *attr_step, *scalars;
    int *escape, *n_escape;
};

// ---- per-hit risk accumulation helpers (shared by the risk scan and the fused collision kernel) ----
constexpr float kMaxLogTerm = 4194304.0f;    // 2^22: -log(1 - p) for p = 1 (a certain trajectory)

// Exact unsigned fixed point of a finite w >= 0 with `frac` fractional bits (round to nearest).
__device__ __forceinline__ unsigned long long to_fixed(float w, int frac) {
    const unsigned b = __float_as_uint(w);
    const int e = (int)(b >> 23);
    if (e == 0) return 0ull;                 // zero (and denormals, below 2^-126)
    const unsigned long long m = (b & 0x7fffffu) | 0x800000u;
    const int sh = e - 150 + frac;           // w = m 2^(e - 150)
    if (sh >= 0) return m << sh;
    if (sh <= -25) return 0ull;
    return (m + (1ull << (-sh - 1))) >> -sh;
}

// -log(1 - p) in FP32, capped for p -> 1
__device__ __forceinline__ float neg_log_survival(float p) {
    return p >= 1.0f ? kMaxLogTerm : fminf(-log1pf(-p), kMaxLogTerm);
}

// pdl: the launch follows another kernel of the library on the same stream with nothing in between, so
// it may use programmatic dependent launch (see launch_kernel).
cudaError_t launch_generate(const GenArgs &a, cudaStream_t st, bool pdl = false);
cudaError_t launch_bounds(const BoundsArgs &a, cudaStream_t st, bool pdl = false);
cudaError_t launch_fill_table(int16_t *table, long long n, cudaStream_t st, bool pdl = false);   // table[0, n) = -1
cudaError_t launch_collide(const CollideArgs &a, cudaStream_t st, bool pdl = false);  // stores first hits only
cudaError_t launch_risk_prepare(const RiskArgs &a, cudaStream_t st);             // zero + normalise
int risk_tail_launches(const RiskArgs &a);   // kernels launch_risk_tail launches
cudaError_t launch_risk_tail(const RiskArgs &a, cudaStream_t st, bool pdl = false);   // ego walk + finish
cudaError_t launch_risk(const RiskArgs &a, cudaStream_t st, bool with_prepare = true, bool pdl = false);

}  // namespace mhc
