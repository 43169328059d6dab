/*
 * mhc.h -- C ABI of the GB300 (sm_103a) multi-hypothesis collision-criticality library.
 *
 * The library implements the data-parallel hot path of "Parallel Multi-Hypothesis Algorithm for
 * Criticality Estimation in Traffic and Collision Avoidance" (arXiv 2005.06773):
 *   trajectory generation (Section IV-B)  ->  collision recognition (Section IV-C)  ->  risk (Section IV-D).
 *
 * Conventions shared by every entry point
 *   - Every function returns an mhc_status (0 = MHC_OK, negative = error); nothing crosses the ABI as an
 *     exception.  mhc_status_string() names a code; mhc_last_error() gives a one-line reason for the
 *     most recent failure on the calling thread.
 *   - "host" pointers are read during the call only; the library copies what it needs.  "device"
 *     pointers are global-memory pointers of the context's device; they are owned by the caller, must
 *     stay valid until the work enqueued on `stream` has completed, and must not overlap each other.
 *     Device arrays are aligned to their element size (4 bytes for the FP32 pose planes and int32 outputs,
 *     8 bytes for int64 and double outputs, 2 bytes for the int16 table); a misaligned one is an
 *     MHC_E_INVALID.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  Work is enqueued
 *     asynchronously; the caller synchronises.  Calls on one context may use different streams: the
 *     library orders its internal scratch memory between them on the device.
 *   - One host thread at a time may call into a given context (except mhc_poll, see below).
 *   - Invalid arguments return MHC_E_INVALID before any work is enqueued; CUDA failures return MHC_E_CUDA.
 */
#ifndef MHC_H
#define MHC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MHC_OK = 0,
    MHC_PENDING = 1,        /* mhc_poll: the request has not finished yet */
    MHC_E_INVALID = -1,     /* malformed scenario, sizes out of range, bad weights */
    MHC_E_NOMEM = -2,       /* the context's arena or a host allocation is too small */
    MHC_E_CUDA = -3,        /* a CUDA runtime call or kernel launch failed */
    MHC_E_TIMEOUT = -4,     /* a bounded device-side wait gave up / a request missed its deadline */
    MHC_E_BUSY = -5,        /* mhc_submit: queue full */
    MHC_E_NOTFOUND = -6     /* unknown ticket */
} mhc_status;

enum { MHC_VEHICLE = 0, MHC_PEDESTRIAN = 1 };     /* object kinds: rectangle / disc */
enum { MHC_ALL_PAIRS = 0, MHC_EGO_ONLY = 1 };     /* which object pairs are tested */
enum { MHC_MODEL_OT = 0, MHC_MODEL_KIN = 1 };     /* vehicle motion model */
#define MHC_PED_ACCEL_GRID 1                       /* object flag: pedestrian grid_a holds accelerations */
#define MHC_MAX_STEPS 32767                        /* first-collision steps are stored as int16 */
#define MHC_MAX_OBJECTS 4096                       /* per scenario */
#define MHC_MAX_SCENARIOS 65536                    /* per batch */
#define MHC_MAX_VERTICES 16                        /* vertices of a vehicle's convex outline */

/*
 * One traffic object and the control grid of its hypotheses (Section IV-B; a hypothesis is one
 * acceleration profile combined with one path, Section III).
 *   kind MHC_VEHICLE: rectangle length x width centred on the pose point, body axis along psi.
 *       Hypothesis h = i_a * n_b + i_b drives with constant acceleration grid_a[i_a] (m/s^2) and constant
 *       front steering angle grid_b[i_b] (rad) through the one-track model (Eq. onetrack) integrated
 *       by Eq. (EulerVelocity); model MHC_MODEL_KIN uses the kinematic bicycle instead.
 *   kind MHC_PEDESTRIAN: disc of `radius` moving by Eq. (pedestrianmotion) with constant heading
 *       psi0 + grid_b[i_b]; grid_a holds initial speeds (m/s) or, with flag MHC_PED_ACCEL_GRID,
 *       accelerations from initial speed v0, the speed then limited to [0, v_max] (v_max <= 0: no cap).
 *   veh_params: host pointer to {m, I_z, l_f, l_r, c_af, c_ar} (kg, kg m^2, m, m, N/rad, N/rad), or NULL
 *       for {1500, 2500, 1.2, 1.5, 80000, 80000}.  grid_a / grid_b are host pointers.
 *   n_vertices / vertices (vehicles only; Section IV-C.1 lets an outline be as detailed as needed):
 *       0 draws the vehicle as its length x width rectangle.  3..MHC_MAX_VERTICES draws it as the convex
 *       polygon vertices[2 q], vertices[2 q + 1] (host, metres, body frame: x along the body axis, y to
 *       the left, origin at the pose point), listed in either orientation; length and width stay
 *       required but are not used for collisions.  The polygon must be strictly convex and simple (every
 *       turn in the same direction, one turn in total): anything else, repeated vertices, non-finite
 *       coordinates or an outline on a pedestrian returns MHC_E_INVALID.  The static entry point
 *       (mhc_detect_collisions_static) takes rectangles only.
 *   paths (vehicles; Section IV-B.2b): NULL drives hypothesis (i_a, i_b) with the constant steering angle
 *       grid_b[i_b].  Otherwise hypothesis (i_a, i_b) follows path i_b, and grid_b's values are unused:
 *       paths[9 i_b + 3 s + {0, 1, 2}] = (x, y, psi) of a point on section s and its direction (host,
 *       metres and rad); section 0 is followed for t < 1.0 s, section 1 for t < 1.5 s, section 2 after.
 *       Before every sub-step the lateral controller (Eq. controller) sets the front steering angle, in
 *       degrees, from the speed, the signed distance d_path from the centre of gravity predicted 0.5 s
 *       ahead along the course to the section's line (positive when the line lies to the vehicle's left)
 *       and the yaw error e_psi = psi_section - psi (wrapped to [-pi, pi]); the angle is then held within
 *       0.5 rad and within 0.5 rad/s of the previous sub-step's (0 before the first).  Non-finite values
 *       or paths on a pedestrian return MHC_E_INVALID.  Path hypotheses use the thread-per-hypothesis
 *       generation layout.
 */
typedef struct {
    int32_t kind;
    int32_t flags;
    float length, width, radius;
    float x0, y0, psi0, v0;
    float v_max;
    int32_t n_a, n_b;
    const float *grid_a;
    const float *grid_b;
    const float *veh_params;
    int32_t n_vertices;
    const float *vertices;
    const float *paths;
} mhc_object;

/*
 * A scenario: objects, horizon and pairing.  tau is the output time step (s); each step is integrated
 * in `substeps` equal sub-steps; output step k (0 <= k < n_steps) is the pose at time (k + 1) tau.
 * pair_mode MHC_ALL_PAIRS tests every object pair (a, b), a < b; MHC_EGO_ONLY tests (ego, b) for every
 * b != ego (the paper's choice, Section IV-C.1).  `ego` is the EGO object for the risk measures.
 */
typedef struct {
    int32_t n_objects;
    const mhc_object *objects;    /* host */
    float tau;
    int32_t n_steps;
    int32_t substeps;
    int32_t pair_mode;
    int32_t ego;
    int32_t model;
} mhc_scenario;

/*
 * Device pose planes (FP32): x, y (m) and c = cos(psi), s = sin(psi) of the body axis.  Each plane holds
 * n_steps * n_traj values laid out [object][step][hypothesis]: the pose of hypothesis i of object a at
 * step k is at index n_steps * traj_off[a] + k * h_a + i, where traj_off is the prefix sum of the
 * objects' hypothesis counts h_a = n_a * n_b (Eq. threads:traj counts them).
 */
typedef struct {
    float *x, *y, *c, *s;
} mhc_poses;

/*
 * Risk outputs (Section IV-D).  For mhc_assess_risk they are device pointers, for mhc_run host pointers.
 * Any pointer may be NULL to skip that output.  n_pairs / h_e / N / n_objects as in mhc_layout.
 *   per object pair p (table order):
 *     count[p]   int64  number of colliding trajectory combinations
 *     count_k    int64  [n_pairs][N] of them first colliding at step k
 *     P[p]       double sum over colliding combinations of p_a[i] p_b[j]  (Eq. totalCrashProb per pair)
 *     H          double [n_pairs][N] the same split by first-collision step
 *   per EGO hypothesis i (h_e of them):
 *     naive[i]   double sum over colliding (CO b, j) of p_b[j]
 *     cond[i]    double chronologically scaled collision probability (Eq. p21): the colliding entries
 *                (b, j, k) in ascending (k, b, j) order each contribute S p_b[j] with S the product of
 *                (1 - p) over the earlier ones
 *     indep[i]   double 1 - prod_b (1 - sum_j [collide] p_b[j])  (COs independent)
 *     hits[i]    int32  number of colliding (b, j)
 *   attr_obj     double [n_objects] sum_i p_e[i] * (share of cond[i] due to object b)
 *   attr_step    double [N] the same per step
 *   scalars      double [4]: p_cra (Eq. totalCrashProb), p_cra_cond = sum_i p_e[i] cond[i],
 *                            p_cra_indep = sum_i p_e[i] indep[i], 0
 *   escape       int32 [h_e] collision-free EGO hypotheses, most probable first, ties by index (Section VI-A);
 *                the entries after the n_escape routes are -1
 *   n_escape     int32 [1] their number
 */
typedef struct {
    int64_t *count;
    int64_t *count_k;
    double *P;
    double *H;
    double *naive;
    double *cond;
    double *indep;
    int32_t *hits;
    double *attr_obj;
    double *attr_step;
    double *scalars;
    int32_t *escape;
    int32_t *n_escape;
} mhc_risk;

typedef struct mhc_ctx mhc_ctx;

/* Human-readable name of a status code (static string). */
const char *mhc_status_string(int status);
/* One-line reason for the last error returned on the calling thread ("" if none). */
const char *mhc_last_error(void);
/* Library version string. */
const char *mhc_version(void);

/*
 * Create a context on CUDA device `device`.  `arena` is a device buffer of `arena_bytes` bytes owned by the
 * caller (e.g. a framework allocation; 256-byte aligned) that the library sub-allocates scratch from; with
 * arena == NULL the library allocates `arena_bytes` itself with cudaMalloc and frees it in mhc_destroy.
 * Errors: MHC_E_INVALID (bad device, arena_bytes < 1 MiB, arena not 256-byte aligned), MHC_E_CUDA,
 * MHC_E_NOMEM.
 */
int mhc_create(mhc_ctx **out, int device, void *arena, size_t arena_bytes);
/* Wait for the context's outstanding work and release it (and the arena if the library allocated it). */
void mhc_destroy(mhc_ctx *ctx);

/* Context options (mhc_set_option).
 *   MHC_OPT_CULL  1 (default): the collision kernel skips whole steps of a 64 x 64 hypothesis tile when the
 *                 bounding boxes of the two tiles' pose centres, grown by both circumradii, do not meet.
 *                 The table is identical either way; 0 tests every step (used to check that). */
#define MHC_OPT_CULL 1
/*   MHC_OPT_COLLIDE_VARIANT  thread layout of the collision kernel (same table in every case):
 *                 1: 256 threads per 64 x 64 tile, 4 x 4 micro-tiles, all warps on one step at a time;
 *                 2: 64 threads per tile, 8 x 8 micro-tiles;
 *                 3: 4 warps per tile, each warp testing whole steps (8 x 16 micro-tiles per lane);
 *                 4: one warp per tile walking its steps in order (8 x 16 micro-tiles per lane, pairs that
 *                    already hit dropped from later steps, first hits stored at once);
 *                 5: as 4 with one warp per 32 x 32 quarter tile (4 x 8 micro-tiles, culling per quarter);
 *                 6: every active (quarter tile, step) an item, all tested in parallel by persistent warps (a
 *                    pair's first step by atomicMin in scratch, the table and the risk terms written after);
 *                    for small scenes (at most 2^22 items and 2^26 table entries; larger ones use 5);
 *                 7: one 128-thread CTA per 32 x 32 quarter tile, its active steps spread over the four
 *                    warps (each in ascending order), first hits kept in shared memory and a candidate of a
 *                    pair that already hit at an earlier step dropped before its exact test; the CTA stores
 *                    the first hits and their risk terms (the table's -1s are written beforehand);
 *                 8: as 7 for the quarter tiles with an active step only, listed first by one warp per
 *                    quarter tile (records in scratch; up to 2^19 quarter tiles, larger scenarios use 7);
 *                 0 (default): the one mhc_autotune chose for the scenario's size class, else 4 for at
 *                 least 32 tiles per SM, and 7 below that. */
#define MHC_OPT_COLLIDE_VARIANT 3
/*   MHC_OPT_GEN_SCAN  trajectory generation: 1 one warp per hypothesis, its sub-steps in parallel (warp
 *                 scans of the state maps and of the heading / position increments); 0 one thread per
 *                 hypothesis, sub-steps in order; 2 (default) the first for the objects of scenarios with
 *                 up to 4096 hypotheses, the second for larger scenarios (chosen per scenario, so that a
 *                 scenario gets the same poses alone and in any batch).  Both follow Eqs. onetrack,
 *                 EulerVelocity and pedestrianmotion; they differ in FP32 rounding only. */
#define MHC_OPT_GEN_SCAN 4
/*   MHC_OPT_SCORE  occurrence probabilities when a call passes no weights: 0 (default) uniform per object;
 *                 1 each hypothesis scored by Eq. (normTraj), n_h = (w_acc n_acc + w_str d_str) /
 *                 (c_com c_cou), then L1-normalised per object (Section IV-D.1).  The paper fixes neither
 *                 weights nor factors; the library's defaults: w_acc = w_str = 1/2; vehicles n_acc =
 *                 1 / (1 + |vdot| / 2 m/s^2); constant steering d_str = 1 / (1 + |delta| / 0.05 rad);
 *                 paths, from the lateral offsets o_s of their section points from the vehicle's initial
 *                 line (positive to the left): d_str = 1 / (1 + max |o_s| / 1.75 m), c_com = 1 + (|o_1 -
 *                 o_0| + |o_2 - o_1|) / 3.5 m, c_cou = 2 when max o_s > 1.75 m (the lane to the left
 *                 carries counter traffic), else 1; pedestrians n_acc = 1 / (1 + |v - v0| / 1 m/s) for
 *                 speed grids or 1 / (1 + |vdot| / 2 m/s^2) for acceleration grids, d_str = 1 / (1 +
 *                 |heading offset| / 0.5 rad), c_com = c_cou = 1. */
#define MHC_OPT_SCORE 5
int mhc_set_option(mhc_ctx *ctx, int option, long long value);

/* Work counters of the collision kernel since the last reset, summed over calls on this context (host
   array out, n_out <= MHC_COUNTER_WORDS words written): out[0] = pose-pair broad-phase tests executed
   (after culling, a whole block of hypothesis pairs per active step), out[1] = exact narrow-phase tests,
   out[2 .. 6] = those narrow-phase tests by shape class: rectangle-rectangle, rectangle-disc, disc-disc,
   outline-outline, outline-disc (a rectangle in a pair with an outline counts as an outline).  Synchronises `stream`; reset != 0 zeroes them all afterwards.
   MHC_E_INVALID: out NULL or n_out outside 1..MHC_COUNTER_WORDS. */
#define MHC_COUNTER_WORDS 7
int mhc_collision_counters(mhc_ctx *ctx, uint64_t *out, int32_t n_out, int reset, void *stream);

/* Kernel timing (mhc_set_option(ctx, MHC_OPT_PROFILE, 1)): the library records a CUDA event pair on the
   launching stream around every kernel it launches.  mhc_profile_read synchronises those events and
   returns, per kernel class (MHC_K_GENERATE = the descriptor upload (a copy kernel reading mapped pinned
   host memory) and generation, which on the fused mhc_evaluate / mhc_run path also runs the risk
   preparation in extra CTAs; MHC_K_BOUNDS = the table fill (unless the collision kernel fills) and the
   tile-bounds kernel; MHC_K_COLLIDE; MHC_K_RISK = the risk kernels: prepare (unfused path), table scan
   (unfused path), the EGO walk and, for large batches, the totals conversion, and mhc_run's copy of its
   outputs into mapped pinned host memory), the summed milliseconds and
   the launch counts since the last reset; reset != 0 clears them.  Disabled by default (no events
   recorded); the events add GPU time, so time steps with it off. */
#define MHC_OPT_PROFILE 2
enum { MHC_K_GENERATE = 0, MHC_K_BOUNDS = 1, MHC_K_COLLIDE = 2, MHC_K_RISK = 3, MHC_K_COUNT = 4 };
int mhc_profile_read(mhc_ctx *ctx, double ms[4], int64_t launches[4], int reset);

/* Bytes the most recent call on this context copied host->device (descriptors, weights) and
   device->host (mhc_run: its whole output block, one copy). */
int mhc_transfer_bytes(mhc_ctx *ctx, int64_t *h2d, int64_t *d2h);

/*
 * Sizes of a scenario's buffers (host only, no GPU work).  Any output pointer may be NULL.
 *   n_traj     total hypotheses sum_a h_a (Eq. threads:traj); each pose plane holds n_steps * n_traj floats
 *   n_pairs    object pairs tested
 *   n_entries  trajectory combinations sum_p h_a h_b (Eq. threads:coll); the table holds that many int16
 *   h_ego      hypotheses of the EGO object
 *   scratch    arena bytes a call on this scenario needs (mhc_run needs poses + table on top, reported
 *              by mhc_run_bytes)
 * Errors: MHC_E_INVALID with the reason in mhc_last_error().
 */
int mhc_layout(const mhc_scenario *scen, int64_t *n_traj, int32_t *n_pairs, int64_t *n_entries,
               int32_t *h_ego, size_t *scratch);

/* Pair list in table order: pair_a[n_pairs], pair_b[n_pairs] object indices and pair_off[n_pairs + 1]
   int64 offsets of each pair's h_a x h_b block (row i = hypothesis of a, column j = hypothesis of b). */
int mhc_pair_table(const mhc_scenario *scen, int32_t *pair_a, int32_t *pair_b, int64_t *pair_off);

/*
 * Trajectory generation (Section IV-B, Eqs. onetrack, EulerVelocity, pedestrianmotion): one thread per
 * hypothesis integrates its n_steps * substeps sub-steps in order and writes the FP32 pose planes `out`
 * (device, layout above).  Errors: MHC_E_INVALID, MHC_E_NOMEM (arena), MHC_E_CUDA.
 */
int mhc_generate_trajectories(mhc_ctx *ctx, const mhc_scenario *scen, const mhc_poses *out, void *stream);

/*
 * Collision recognition (Section IV-C): for every listed object pair (a, b) and every hypothesis pair
 * (i, j) writes table[pair_off[p] + i * h_b + j] = the first step k at which the closed shapes of a and b
 * overlap (touching counts), or -1 if they never do within the horizon.  `poses` is the device output of
 * mhc_generate_trajectories (or any poses in that layout); `table` is a device int16 buffer of n_entries.
 * Errors: MHC_E_INVALID, MHC_E_NOMEM (arena), MHC_E_CUDA.
 */
int mhc_detect_collisions(mhc_ctx *ctx, const mhc_scenario *scen, const mhc_poses *poses, int16_t *table,
                          void *stream);

/*
 * Risk assessment (Section IV-D) from a device first-collision table.  traj_weights: host array of
 * n_objects host pointers to each object's h_a non-negative FP32 weights, L1-normalised per object into
 * occurrence probabilities (Section IV-D.1); traj_weights == NULL or a NULL entry means uniform.
 * Outputs (mhc_risk) are device pointers.  Errors: MHC_E_INVALID (negative weights or a zero sum),
 * MHC_E_NOMEM (arena), MHC_E_CUDA.
 */
int mhc_assess_risk(mhc_ctx *ctx, const mhc_scenario *scen, const int16_t *table,
                    const float *const *traj_weights, const mhc_risk *out, void *stream);

/*
 * The whole method on device buffers in one call: generation (Section IV-B) into `poses`, collision
 * recognition (Section IV-C) into `table`, risk (Section IV-D) into the device outputs `out` -- the same
 * results as the three calls above.  The collision kernel accumulates the risk terms at each first hit,
 * so the table is not read a second time.  Asynchronous on `stream`.  Errors as above.
 */
int mhc_evaluate(mhc_ctx *ctx, const mhc_scenario *scen, const float *const *traj_weights, const mhc_poses *poses,
                 int16_t *table, const mhc_risk *out, void *stream);

/*
 * Autotuner of the collision stage: times the collision kernel (its own CUDA events) with every thread
 * layout and with culling on and off, on `poses` / `table` (device buffers as for mhc_detect_collisions),
 * either as mhc_detect_collisions runs it (fused = 0) or as mhc_evaluate / mhc_run run it with the risk
 * terms accumulated inside (fused = 1; outputs go to the arena).  The fastest is kept for scenarios of
 * this size class (floor(log2(tiles)), floor(log2(n_steps))) and that path, and reported; later calls
 * with MHC_OPT_COLLIDE_VARIANT 0 use it.  Synchronises `stream`.
 */
int mhc_autotune(mhc_ctx *ctx, const mhc_scenario *scen, const mhc_poses *poses, int16_t *table, int fused,
                 int32_t *best_variant, int32_t *best_cull, void *stream);

/* Arena bytes mhc_run needs for this scenario (poses + table + scratch). */
int mhc_run_bytes(const mhc_scenario *scen, size_t *bytes);

/*
 * The whole method for one scenario from host inputs to host outputs: uploads the scenario, runs
 * generation, collision recognition and risk in the context's arena, copies the risk outputs (host
 * pointers in `out`) back and synchronises `stream`.  Poses and table live in the arena and are
 * overwritten by the next call.  Errors as above.
 */
int mhc_run(mhc_ctx *ctx, const mhc_scenario *scen, const float *const *traj_weights, const mhc_risk *out,
            void *stream);

/*
 * Batches: many scenarios of different sizes in one launch sequence (one generation launch over every
 * hypothesis, one collision launch over every tile of every object pair, one risk walk over every EGO
 * hypothesis).  The scenarios of a batch are concatenated in batch order: objects, hypotheses (weights),
 * pose-plane elements, object pairs, table entries, per-pair step entries (count_k, H), EGO hypotheses
 * (naive, cond, indep, hits, escape) and per-scenario steps (attr_step) of scenario s follow those of
 * scenario s - 1, each scenario laid out exactly as it is alone; scalars hold 4 doubles and n_escape one
 * int32 per scenario, and escape lists each scenario's routes from its ego0.  A single scenario is the
 * batch of one (its sizes are those of mhc_layout).  Pair lists hold batch-wide object indices.
 */
typedef struct {
    int64_t n_traj;          /* hypotheses of all objects (weights, probabilities) */
    int64_t n_poses;         /* elements of each pose plane: sum over objects of h_a x its scenario's n_steps */
    int64_t n_entries;       /* first-collision table entries */
    int64_t n_step_entries;  /* per-pair step entries: length of count_k and H */
    int64_t n_scen_steps;    /* sum of the scenarios' n_steps: length of attr_step */
    int64_t h_ego;           /* EGO hypotheses of all scenarios */
    int32_t n_pairs, n_objects, n_scenarios, max_steps;
    size_t scratch;          /* arena bytes mhc_evaluate_batch needs */
    size_t plan_bytes;       /* device scratch bytes mhc_plan_create needs */
} mhc_batch_info;

typedef struct {             /* where scenario s sits in the concatenated arrays */
    int32_t obj0, n_objects, pair0, n_pairs, n_steps, ego;   /* ego: index within the scenario */
    int64_t traj0, pose0, entry0, step_entry0, ego0, step0;
} mhc_batch_slice;

/* Sizes of a batch (host only, no GPU work); `slices` (n_scen entries) may be NULL.  Errors: MHC_E_INVALID
   (reason names the scenario), also for n_scen outside [1, MHC_MAX_SCENARIOS]. */
int mhc_batch_layout(const mhc_scenario *scens, int32_t n_scen, mhc_batch_info *info, mhc_batch_slice *slices);

/* Pair list of a batch in table order (as mhc_pair_table, object indices batch-wide). */
int mhc_batch_pair_table(const mhc_scenario *scens, int32_t n_scen, int32_t *pair_a, int32_t *pair_b,
                         int64_t *pair_off);

/* mhc_evaluate over a batch: traj_weights holds n_objects (batch-wide) host pointers or is NULL; poses,
   table and out are device buffers of the batch sizes.  Results per scenario equal those of mhc_evaluate
   on that scenario alone (integers and fixed-point sums exactly; the scalars to rounding of the order of
   their double additions). */
int mhc_evaluate_batch(mhc_ctx *ctx, const mhc_scenario *scens, int32_t n_scen, const float *const *traj_weights,
                       const mhc_poses *poses, int16_t *table, const mhc_risk *out, void *stream);

/* mhc_autotune over a batch (size class of the whole batch: its tiles and max_steps). */
int mhc_autotune_batch(mhc_ctx *ctx, const mhc_scenario *scens, int32_t n_scen, const mhc_poses *poses,
                       int16_t *table, int fused, int32_t *best_variant, int32_t *best_cull, void *stream);

/*
 * Plans: a batch evaluated repeatedly.  mhc_plan_create lays the batch out once into `scratch` (device,
 * caller-owned, at least mhc_batch_info.plan_bytes, 256-byte aligned; used by the plan only) and keeps a
 * pinned host copy of the descriptors.  With flags MHC_PLAN_GRAPH it runs the launch sequence once and
 * captures it (descriptor upload from the pinned copy + the mhc_evaluate_batch kernels) as a CUDA graph;
 * each mhc_plan_launch is then one cudaGraphLaunch on `stream`.  With MHC_PLAN_PIPELINE a plan of at
 * least 8 scenarios is pipelined: its scenarios form 4 runs of about equal collision work, each laid out on
 * its own, and the runs alternate between `stream` and a second stream of the plan, run g's generation
 * waiting for run g - 1's generation only, so that generations and table fills may run beside the
 * collision kernels of earlier runs (the launch ends with both streams joined on `stream`).  The results
 * are those of the batch: integer outputs bit for bit, FP64 scalar totals to rounding.  The collision configuration (autotuned
 * or forced) is the one in force at creation.  mhc_plan_update replaces the scenarios by ones of the same
 * structure (objects, grid sizes, steps, pairs; initial states, grid values and shapes may change): it
 * waits for the plan's previous launch to finish, then rewrites the pinned copy, which the next launch
 * uploads.  Launches of one plan are ordered after each other on the device.  poses / table / out stay
 * the caller's and are rewritten by every launch.  The plan uses ctx (destroy it first) but not the
 * context's arena.  Errors: MHC_E_INVALID, MHC_E_NOMEM (scratch too small), MHC_E_CUDA.
 */
typedef struct mhc_plan mhc_plan;
#define MHC_PLAN_GRAPH 1
#define MHC_PLAN_PIPELINE 2
int mhc_plan_create(mhc_ctx *ctx, const mhc_scenario *scens, int32_t n_scen, const float *const *traj_weights,
                    const mhc_poses *poses, int16_t *table, const mhc_risk *out, void *scratch,
                    size_t scratch_bytes, int32_t flags, mhc_plan **plan);
int mhc_plan_update(mhc_plan *plan, const mhc_scenario *scens, int32_t n_scen);
int mhc_plan_launch(mhc_plan *plan, void *stream);
void mhc_plan_destroy(mhc_plan *plan);

/*
 * Serving (no counterpart in the paper beyond its real-time setting, Section I: a criticality answer per
 * sensor frame).  Continuous batching of scenario requests on one context: mhc_submit copies a scenario
 * and queues it; a scheduler thread of the library admits queued requests into batches while stream slots
 * and pool memory are free, launches each batch (the mhc_evaluate_batch kernels) on its slot's stream and
 * copies the batch's risk outputs to pinned host memory; requests that arrive while other batches run are
 * admitted into the next batch on another slot, so their work overlaps on the device.  Requests up to
 * `small_tests` nominal pose tests go to the small lane (high-priority streams), larger ones to the large
 * lane, so small requests never wait behind a large batch.  A request's poses, table and risk outputs
 * stay resident in the pool until mhc_release.
 *
 * The pool is a device buffer the caller owns (e.g. a torch tensor), at least 1 MiB; admission is by its
 * free bytes (first fit).  One serving loop per context; while it runs, use the context for nothing else
 * but the calls below and mhc_set_option / mhc_autotune before mhc_serve_start (the loop keeps a copy of
 * the collision configuration).  mhc_submit / mhc_poll / mhc_release / mhc_request_* / mhc_serve_stats_read
 * are thread-safe.
 */
typedef struct {
    int32_t small_slots;         /* streams of the small lane, 1..8 (default 3) */
    int32_t large_slots;         /* streams of the large lane, 1..8 (default 1) */
    int32_t max_batch;           /* scenarios per batch, 1..4096 (default 64) */
    int32_t max_queue;           /* queued requests beyond which mhc_submit returns MHC_E_BUSY (default 4096) */
    int64_t small_tests;         /* nominal pose tests up to which a request is small (default 2^31) */
    int64_t max_batch_tests;     /* nominal pose tests per batch of the small lane (default 2^34) */
} mhc_serve_config;

int mhc_serve_start(mhc_ctx *ctx, void *pool, size_t pool_bytes, const mhc_serve_config *cfg /* NULL: defaults */);

/* Stops the scheduler after the batches in flight; queued requests are dropped (their tickets become
   unknown).  Called by mhc_destroy if still running. */
int mhc_serve_stop(mhc_ctx *ctx);

/* Queues a scenario (host inputs copied; weights as for mhc_evaluate).  *ticket identifies the request.
   Errors: MHC_E_INVALID (scenario / weights), MHC_E_NOMEM (the request alone is larger than the pool),
   MHC_E_BUSY (max_queue requests waiting), MHC_E_NOTFOUND (no serving loop). */
int mhc_submit(mhc_ctx *ctx, const mhc_scenario *scen, const float *const *traj_weights, uint64_t *ticket);

/* Waits up to timeout_us (0: no wait, < 0: forever) for the request.  MHC_OK: done, and the host pointers
   of `out` (may be NULL; the single-scenario sizes of mhc_layout, each pointer may be NULL) receive its
   risk outputs; MHC_PENDING: not finished yet; MHC_E_NOTFOUND: unknown or released ticket; MHC_E_CUDA:
   its batch failed. */
int mhc_poll(mhc_ctx *ctx, uint64_t ticket, const mhc_risk *out, int32_t timeout_us);

/* Frees the request's resident device memory (its batch's block once every request of it is released).
   A request still queued is withdrawn; one in flight is released when its batch completes. */
int mhc_release(mhc_ctx *ctx, uint64_t ticket);

/* Device views of a finished request, valid until mhc_release: pose planes and first-collision table in
   the single-scenario layout, and the device risk outputs (NULL arguments skipped). */
int mhc_request_buffers(mhc_ctx *ctx, uint64_t ticket, mhc_poses *poses, int16_t **table, mhc_risk *dev_out);

/* Host steady-clock times (ns) of a request: ns[0] submitted, ns[1] launched in a batch, ns[2] outputs on
   the host (0 where not reached); *batch_size = scenarios in its batch. */
int mhc_request_times(mhc_ctx *ctx, uint64_t ticket, int64_t ns[3], int32_t *batch_size);

typedef struct {
    int64_t submitted, completed, batches, queued, running;
    size_t pool_free, pool_largest;
} mhc_serve_stats;
int mhc_serve_stats_read(mhc_ctx *ctx, mhc_serve_stats *stats);

/* While paused (paused != 0) the scheduler admits nothing; batches in flight complete. */
int mhc_serve_pause(mhc_ctx *ctx, int32_t paused);

/* The pool's first-fit allocator on its own (host only, offsets into a buffer of `bytes`; 256-byte
   blocks).  Errors: MHC_E_NOMEM (no free block fits), MHC_E_NOTFOUND (no block at that offset). */
typedef struct mhc_pool mhc_pool;
int mhc_pool_create(size_t bytes, mhc_pool **out);
int mhc_pool_alloc(mhc_pool *pool, size_t bytes, size_t *offset);
int mhc_pool_free(mhc_pool *pool, size_t offset);
int mhc_pool_info(mhc_pool *pool, size_t *free_bytes, size_t *largest_free, int32_t *n_free_blocks);
void mhc_pool_destroy(mhc_pool *pool);

/*
 * Collision recognition without any allocation (no counterpart in the paper: it serves deployment).
 * Same result as mhc_detect_collisions (same kernels, culling on) for callers that may not allocate memory
 * while running -- real-time or safety controllers with a memory plan fixed at start-up, where an
 * allocation can block, synchronise the device or fail at a deadline, and plugins whose host framework
 * owns all device memory.  It takes no context and calls no cudaMalloc, cudaFree, cudaHostAlloc or host
 * heap allocation.  Its scratch (scenario descriptors and per-tile bounding boxes) is one static device
 * array of 8 MiB that every GPU which loads the library holds until the process exits.  With CUDA's lazy
 * module loading the array (and the kernels) are loaded into a device's context on first use, so the first
 * call on each device is a warm-up that reserves those 8 MiB: make it at start-up; later calls allocate
 * nothing.  Limits: at most 64 objects and 524,288 hypotheses, and descriptors + n_steps x
 * ceil(h_a / 32) summed over objects x 16 bytes must fit in the 8 MiB; larger scenarios return
 * MHC_E_INVALID with the needed size in mhc_last_error().  The device is the calling thread's current one;
 * every call looks up the array's device address there (cudaGetSymbolAddress, a host query).  A stream
 * in capture is refused with MHC_E_INVALID (the descriptors are staged in a static host array that later
 * calls rewrite).  Every call shares the one array (nothing in it needs to start at zero; each call
 * rewrites what it reads): calls whose work overlaps on the GPU -- different streams without ordering, or
 * several host threads -- race, and one host thread at a time may call it.
 * poses / table / stream as for mhc_detect_collisions.
 */
int mhc_detect_collisions_static(const mhc_scenario *scen, const mhc_poses *poses, int16_t *table, void *stream);

/*
 * Street data processing (Section IV-A) and the controller's paths (Section IV-B.2b), on the calling host
 * thread (a few dividers: no device work).  dividers: host, n_dividers (2..4) lane dividers x 3 points
 * (x, y) in the vehicle's frame at t = 0 (x ahead, y to the left), ordered from right to left; each
 * divider is the curve y = a x^2 + b x + c through its points (Gauss-Jordan).  The vehicle's lane is the
 * pair of adjacent dividers enclosing its position (the origin).  At 1.0, 1.5 and 2.0 s the reference
 * position is x = v0 t; the own lane is sampled at 1/4, 1/2 and 3/4 of its width there and each
 * neighbouring lane present at 1/3 and 2/3, right to left (m = 3, 5 or 7 samples per instant); a section
 * passes through a sample along the lane's centre-line direction.  ego = 0: m paths (sample q at every
 * instant); ego != 0: m^3 paths, path (q0 m + q1) m + q2 taking sample q_k at instant k.  paths: host,
 * n_paths x 3 sections x (x, y, psi) in the scenario frame (the vehicle at x0, y0 heading psi0), ready
 * for mhc_object.paths; NULL returns the count only (*n_paths).  MHC_E_INVALID: non-finite input,
 * v0 < 0, repeated abscissae in a divider, or no lane enclosing the vehicle.
 */
int mhc_lane_paths(const float *dividers, int32_t n_dividers, float x0, float y0, float psi0, float v0,
                   int32_t ego, float *paths, int32_t *n_paths);

#ifdef __cplusplus
}
#endif

#endif /* MHC_H */
