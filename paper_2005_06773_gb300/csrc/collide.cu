// collide.cu -- collision recognition (Section IV-C): first overlapping step of every hypothesis pair.
//
// Work decomposition: the hypothesis pairs of each object pair form 64 x 64 tiles, listed pair after pair
// in collision-grid order (closest pairs first).  Eight thread layouts share one result:
//   1, 2  one CTA per tile (256 threads with 4 x 4 register micro-tiles, or 64 threads with 8 x 8); the
//         tile's active steps are staged into shared memory a chunk at a time and tested in any order, the
//         earliest hit kept with a shared atomicMin;
//   3     a CTA of 4 warps per tile, each warp testing whole steps;
//   4, 5  one warp per 64 x 64 tile (4 warps per CTA) or per 32 x 32 quarter (1-warp CTAs) walking the
//         active steps in ascending order: a register mask remembers the pairs that already hit, so only
//         first hits are stored and later candidates of those pairs cost nothing; the warp stages its own
//         poses with the next step's loads in flight, and loops over blocks when the grid is capped;
//   6     step items: (32 x 32 block, active step) pairs listed by one kernel and taken in any order by a
//         persistent kernel that keeps each pair's earliest step with a global atomicMin; a third kernel
//         writes the int16 table (and the fused risk terms) for the blocks with active steps;
//   7     one 128-thread CTA per 32 x 32 block, the block's active steps spread over its four warps, first
//         hits kept in shared memory (the small-scene default);
//   8     as 7 for the blocks with an active step only, listed first by one warp per block.
// The table is -1 outside first hits: a fill kernel (or fill CTAs of the generation or bounds launch) writes
// it first, or variant 5 writes its own blocks (small tables) and variant 6 its active blocks.
//
// Broad phase (per test, 3 FP32 instructions): with h_a = (1 - eps)|p_a|^2 / 2 and
// h_b = ((1 - eps)|p_b|^2 - R^2 - eps0) / 2 precomputed at staging, the pair is a candidate iff
//     x_a x_b + y_a y_b - h_b >= h_a   <=>   |p_a - p_b|^2 <= R^2 + eps0 + eps (|p_a|^2 + |p_b|^2),
// R = sum of circumradii.  eps = 1e-5 exceeds the FP32 rounding error of the expanded form (< 7 * 2^-24
// relative to |p|^2) by more than 10x, so no true candidate is ever rejected; the narrow phase then
// decides exactly on direct coordinate differences.
// Narrow phase: separating-axis test on the four edge normals (rectangle-rectangle), clamped distance in
// the rectangle frame (rectangle-disc), centre distance (disc-disc), separating edges of convex outlines
// (outline kernels only).  Closed sets: touching overlaps.
// Culling: steps at which two blocks' pose-centre bounding boxes, inflated by R, do not meet are skipped
// whole (result-preserving).
#include <algorithm>
#include <cstdint>

#include "mhc_internal.cuh"

namespace mhc {
namespace {

constexpr float kEps = 1e-5f;
constexpr float kEps0 = 1e-4f;
constexpr float kFar = 1.0e6f;   // padding poses far outside any scene

__device__ __forceinline__ bool rect_rect(float dx, float dy, float ca, float sa, float la, float wa,
                                          float cb, float sb, float lb, float wb) {
    const float c = fabsf(fmaf(ca, cb, sa * sb));
    const float s = fabsf(fmaf(sa, cb, -ca * sb));
    const float pau = fabsf(fmaf(dx, ca, dy * sa));
    const float pav = fabsf(fmaf(dy, ca, -dx * sa));
    const float pbu = fabsf(fmaf(dx, cb, dy * sb));
    const float pbv = fabsf(fmaf(dy, cb, -dx * sb));
    return pau <= la + fmaf(lb, c, wb * s) && pav <= wa + fmaf(lb, s, wb * c) &&
           pbu <= lb + fmaf(la, c, wa * s) && pbv <= wb + fmaf(la, s, wa * c);
}

// rectangle at the origin of d (axis (c, s), half extents l, w) against a disc of radius r at offset d
__device__ __forceinline__ bool rect_disc(float dx, float dy, float c, float s, float l, float w, float r) {
    const float ex = fmaxf(fabsf(fmaf(dx, c, dy * s)) - l, 0.0f);
    const float ey = fmaxf(fabsf(fmaf(dy, c, -dx * s)) - w, 0.0f);
    return fmaf(ex, ex, ey * ey) <= r * r;
}

// Convex outlines (Section IV-C.1 lets an outline be as detailed as needed); in a pair with an outline a
// plain rectangle comes as a 4-gon.  Two convex polygons are disjoint iff the supporting line of some edge
// of one has the whole other polygon strictly on its outer side (the edges of their Minkowski difference
// are the edges of the two), so each edge is one test: edge e of A (body-frame vertex v_e, outward unit
// normal n_e, support h_e = n_e . v_e) separates iff min over B's vertices w of
// (R_a n_e) . (d + R_b w) > h_e, d = p_b - p_a.  The normal is turned into B's frame once per edge and B's
// vertices are read as stored.  Only the kernels instantiated for batches with outlines contain it.
__device__ __forceinline__ bool outline_outline(float dx, float dy, float ca, float sa, float cb, float sb,
                                               const PolyVertex *A, int na, const PolyVertex *B, int nb) {
    const float cr = fmaf(ca, cb, sa * sb), sr = fmaf(sa, cb, -ca * sb);   // R_b^T R_a = R(psi_a - psi_b)
    for (int e = 0; e < na; ++e) {
        const float4 v = A[e];
        const float h = fmaf(v.z, v.x, v.w * v.y);
        const float nwx = fmaf(ca, v.z, -sa * v.w), nwy = fmaf(sa, v.z, ca * v.w);
        const float o = fmaf(nwx, dx, nwy * dy);
        const float mx = fmaf(cr, v.z, -sr * v.w), my = fmaf(sr, v.z, cr * v.w);
        float lo = INFINITY;
        for (int q = 0; q < nb; ++q) {
            const float4 w = B[q];
            lo = fminf(lo, fmaf(mx, w.x, my * w.y));
        }
        if (o + lo > h) return false;
    }
    for (int e = 0; e < nb; ++e) {   // B's edges: A's vertices relative to p_b are -d + R_a w
        const float4 v = B[e];
        const float h = fmaf(v.z, v.x, v.w * v.y);
        const float nwx = fmaf(cb, v.z, -sb * v.w), nwy = fmaf(sb, v.z, cb * v.w);
        const float o = -fmaf(nwx, dx, nwy * dy);
        const float mx = fmaf(cr, v.z, sr * v.w), my = fmaf(-sr, v.z, cr * v.w);   // R_a^T R_b = R(psi_b - psi_a)
        float lo = INFINITY;
        for (int q = 0; q < na; ++q) {
            const float4 w = A[q];
            lo = fminf(lo, fmaf(mx, w.x, my * w.y));
        }
        if (o + lo > h) return false;
    }
    return true;
}

// Outline A at the origin of d (axis (c, s)) against a disc of radius r at offset d: the disc's centre in
// A's frame lies inside A, or within r of one of its edges (segment distance).
__device__ __forceinline__ bool outline_disc(float dx, float dy, float c, float s, const PolyVertex *A, int n,
                                            float r) {
    const float qx = fmaf(dx, c, dy * s), qy = fmaf(dy, c, -dx * s);
    float smax = -INFINITY;
    for (int e = 0; e < n; ++e) {
        const float4 v = A[e];
        smax = fmaxf(smax, fmaf(v.z, qx - v.x, v.w * (qy - v.y)));
    }
    if (smax > r) return false;   // beyond some edge's line by more than r
    if (smax <= 0.0f) return true; // centre inside
    float d2 = INFINITY;
    for (int e = 0; e < n; ++e) {
        const float4 v = A[e], w = A[e + 1 == n ? 0 : e + 1];
        const float ex = w.x - v.x, ey = w.y - v.y, px = qx - v.x, py = qy - v.y;
        const float t = fminf(fmaxf(fmaf(px, ex, py * ey) / fmaf(ex, ex, ey * ey), 0.0f), 1.0f);
        const float rx = fmaf(-t, ex, px), ry = fmaf(-t, ey, py);
        d2 = fminf(d2, fmaf(rx, rx, ry * ry));
    }
    return d2 <= r * r;
}

// The exact test of one broad-phase candidate: d = p_b - p_a, (ca, sa) / (cb, sb) the body axes, la / wa
// and lb / wb the half extents of rectangles, ra / rb the radii of discs.  OUTL: the batch has outlines
// (combos 4..6); the kernels without them keep the short rectangle and disc tests alone.
// The shape combination of a pair and its outlines, copied out of the descriptor once per block: a field read
// through the descriptor in a loop with atomics would be read again after every atomic.
struct PairShape {
    int combo, poly_a, nv_a, poly_b, nv_b;
};

__device__ __forceinline__ PairShape shape_of(const PairDesc &P) { return {P.combo, P.poly_a, P.nv_a, P.poly_b, P.nv_b}; }

template <bool OUTL>
__device__ __forceinline__ bool narrow_hit(const PairShape P, const PolyVertex *polys, float dx, float dy,
                                           float2 qa, float2 qb, float la, float wa, float lb, float wb,
                                           float ra, float rb) {
    if (!OUTL) {
        switch (P.combo) {
            case 0: return rect_rect(dx, dy, qa.x, qa.y, la, wa, qb.x, qb.y, lb, wb);
            case 1: return rect_disc(dx, dy, qa.x, qa.y, la, wa, rb);
            case 2: return rect_disc(-dx, -dy, qb.x, qb.y, lb, wb, ra);
            default: return fmaf(dx, dx, dy * dy) <= (ra + rb) * (ra + rb);
        }
    }
    switch (P.combo) {
        case 0: return rect_rect(dx, dy, qa.x, qa.y, la, wa, qb.x, qb.y, lb, wb);
        case 1: return rect_disc(dx, dy, qa.x, qa.y, la, wa, rb);
        case 2: return rect_disc(-dx, -dy, qb.x, qb.y, lb, wb, ra);
        case 3: return fmaf(dx, dx, dy * dy) <= (ra + rb) * (ra + rb);
        case 4: return outline_outline(dx, dy, qa.x, qa.y, qb.x, qb.y, polys + P.poly_a, P.nv_a, polys + P.poly_b, P.nv_b);
        case 5: return outline_disc(dx, dy, qa.x, qa.y, polys + P.poly_a, P.nv_a, rb);
        default: return outline_disc(-dx, -dy, qb.x, qb.y, polys + P.poly_b, P.nv_b, ra);
    }
}

// Narrow-phase work counters by shape class (CollideArgs::counters [2 + class]): 0 rectangle-rectangle,
// 1 rectangle-disc, 2 disc-disc, 3 outline-outline, 4 outline-disc (the PairDesc combos 0, 1|2, 3, 4, 5|6).
__device__ __forceinline__ int narrow_class(int combo) {
    return combo == 0 ? 0 : (combo <= 2 ? 1 : (combo <= 4 ? combo - 1 : 4));
}

__device__ __forceinline__ void count_narrow(const CollideArgs &a, int combo, unsigned long long n) {
    atomicAdd(a.counters + 1, n);
    atomicAdd(a.counters + 2 + narrow_class(combo), n);
}

// Queue slots of one compaction round: each lane brings cnt (0..8) candidates; off = the candidates of the
// lanes below it, total = all of them (one ballot per bit of cnt instead of a shuffle scan: four
// independent instructions, not a chain of five).  Returns false when no lane has any (uniform).
__device__ __forceinline__ bool queue_offsets(int cnt, int lane, int &off, int &total) {
    const unsigned b0 = __ballot_sync(0xffffffffu, cnt & 1), b1 = __ballot_sync(0xffffffffu, cnt & 2);
    const unsigned b2 = __ballot_sync(0xffffffffu, cnt & 4), b3 = __ballot_sync(0xffffffffu, cnt & 8);
    if (!(b0 | b1 | b2 | b3)) return false;
    const unsigned lt = (1u << lane) - 1u;
    off = __popc(b0 & lt) + 2 * __popc(b1 & lt) + 4 * __popc(b2 & lt) + 8 * __popc(b3 & lt);
    total = __popc(b0) + 2 * __popc(b1) + 4 * __popc(b2) + 8 * __popc(b3);
    return true;
}

// Position of the r-th set bit (r counted from 0, below popc(m)) of m, by halving popcounts.
__device__ __forceinline__ int nth_set_bit(unsigned m, int r) {
    int pos = 0, c = __popc(m & 0xffffu);
    if (r >= c) { r -= c; m >>= 16; pos += 16; }
    c = __popc(m & 0xffu);
    if (r >= c) { r -= c; m >>= 8; pos += 8; }
    c = __popc(m & 0xfu);
    if (r >= c) { r -= c; m >>= 4; pos += 4; }
    c = __popc(m & 0x3u);
    if (r >= c) { r -= c; m >>= 2; pos += 2; }
    return pos + (r >= (int)(m & 1u) ? 1 : 0);
}

// Candidate selection without a queue: lane L holds a mask `cand` of its candidates; slot s of the warp's
// candidates in (lane, bit) order belongs to the last lane whose exclusive count is <= s (a 5-step
// shuffle search), and is that lane's (s - its count)-th bit.  Every lane takes one slot per round, so the
// exact tests run with all lanes busy.  Calls fn(owner lane, bit) for each slot (warp-uniform call).
template <typename Fn>
__device__ __forceinline__ void for_each_candidate(unsigned cand, int lane, Fn &&fn) {
    const unsigned cnt = __popc(cand);
    unsigned incl = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned v = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += v;
    }
    const unsigned excl = incl - cnt;
    const unsigned total = __shfl_sync(0xffffffffu, incl, 31);
    for (unsigned s0 = 0; s0 < total; s0 += 32) {
        const unsigned s = s0 + lane;
        int owner = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const unsigned e = __shfl_sync(0xffffffffu, excl, owner + step);
            if (e <= s) owner += step;
        }
        const unsigned m = __shfl_sync(0xffffffffu, cand, owner);
        const unsigned e = __shfl_sync(0xffffffffu, excl, owner);
        if (s < total) fn(owner, nth_set_bit(m, (int)(s - e)));
    }
}

// The pair of collision tile g: the last pair (in collision-grid order) whose first tile is <= g.  A 64-way
// search by the whole warp (every lane must call it with the same g): each round the lanes probe 64
// evenly spaced pairs at once (two each) and keep the span between the last probe <= g and the next, so up
// to 64 pairs take one round of loads and 4,096 two (a binary search is a chain of log2 n dependent loads).
__device__ __forceinline__ int pair_of_tile(const CollideArgs &a, long long g) {
    const int lane = threadIdx.x & 31;
    int lo = 0, hi = a.n_pairs - 1;
    while (lo < hi) {   // 64 probes per round (two per lane): a scene of up to 64 pairs in one round of loads
        const long long span = hi - lo + 1;
        const bool le0 = a.pairs[lo + (int)(span * (2 * lane) / 64)].tile_start <= g;
        const bool le1 = a.pairs[lo + (int)(span * (2 * lane + 1) / 64)].tile_start <= g;
        const unsigned long long m = (unsigned long long)__ballot_sync(0xffffffffu, le0) |
                                     (unsigned long long)__ballot_sync(0xffffffffu, le1) << 32;
        // probe q = 2 lane + (0 | 1) sits at bit lane + 32 (q & 1); probe 0 always holds: pairs[lo] <= g
        const unsigned even = (unsigned)m, odd = (unsigned)(m >> 32);
        const int le = 31 - __clz(even), lo2 = odd ? 31 - __clz(odd) : -1;   // last true even / odd probe
        const int L = 2 * lo2 + 1 > 2 * le ? 2 * lo2 + 1 : 2 * le;           // the true probes form a prefix
        const int nlo = lo + (int)(span * L / 64);
        hi = L == 63 ? hi : lo + (int)(span * (L + 1) / 64) - 1;
        lo = nlo;
    }
    return lo;
}

constexpr int kMaxChunks = (32767 + 31) / 32;   // 32-step activity words for the longest horizon
constexpr int kFusedHistSteps = 1024;            // per-CTA step histograms in shared memory up to this N
constexpr int kFusedCellSteps = 160;             // per-CTA EGO survival cells (64 x N x 8 B) up to this N

// Next active step at or after k (-1 if none), from the per-32-step activity words.
__device__ __forceinline__ int next_active(const unsigned *mask, int n_chunks, int k) {
    int w = k >> 5;
    if (w >= n_chunks) return -1;
    unsigned m = mask[w] & (0xffffffffu << (k & 31));
    while (!m) {
        if (++w >= n_chunks) return -1;
        m = mask[w];
    }
    return (w << 5) + __ffs(m) - 1;
}

// THREADS threads per 64 x 64 tile, each testing an MI x MJ micro-tile (rows ti + TI m, columns tj + TJ n).
// The tile's active steps are taken CH at a time: all their poses are staged into shared memory with
// every load in flight at once, then each warp runs through the CH steps without further barriers.
template <int THREADS, int MI, int MJ, int CH, bool FUSED, bool OUTL>
__global__ void __launch_bounds__(THREADS) collide_kernel(const CollideArgs a) {
    pdl_start();
    constexpr int TI = kTile / MI, TJ = kTile / MJ;
    static_assert(TI * TJ == THREADS, "micro-tiles must cover the tile");
    static_assert(MI * MJ <= 64, "first-hit mask is 64 bits");
    // dynamic shared memory: CH staged steps, then (FUSED) the tile's risk accumulators
    extern __shared__ __align__(16) unsigned char s_dyn[];
    float4 *s_pa = reinterpret_cast<float4 *>(s_dyn);               // [CH][64] x, y, h_a
    float4 *s_pb = s_pa + CH * kTile;                                  // [CH][64] x, y, h_b
    float2 *s_ra = reinterpret_cast<float2 *>(s_pb + CH * kTile);     // [CH][64] c, s
    float2 *s_rb = s_ra + CH * kTile;
    unsigned long long *s_acc = reinterpret_cast<unsigned long long *>(s_rb + CH * kTile);
    __shared__ unsigned s_mask[kMaxChunks];
    __shared__ int s_klist[CH];
    __shared__ int s_nk, s_cursor;
    constexpr int WARPS = THREADS / 32;
    __shared__ unsigned long long s_found[THREADS];          // bit MJ m + n: the thread's pair has hit
    __shared__ unsigned short s_queue[WARPS][32 * MI * MJ];  // per-warp candidates: owner lane << 6 | bit

    const long long g = blockIdx.x;
    if (g >= a.n_tiles) return;
    const int lo = pair_of_tile(a, g);
    const PairDesc P = a.pairs[lo];
    const PairShape shape = shape_of(P);
    const ObjDesc &A = a.objs[P.a];
    const ObjDesc &B = a.objs[P.b];
    const int t = (int)(g - P.tile_start);          // < tiles_a x tiles_b <= n_tiles < 2^31
    const int ta = t / P.tiles_b, tb = t - ta * P.tiles_b;
    const int i0 = ta * kTile, j0 = tb * kTile;
    const int rows = min(kTile, A.h - i0), cols = min(kTile, B.h - j0);
    const int tid = threadIdx.x, ti = tid / TJ, tj = tid % TJ;
    const int N = P.n_steps;
    const int n_chunks = (N + 31) >> 5;

    // activity of every step: the two tiles' centre boxes, grown by both circumradii, must meet
    const int na = (rows + kBoundTile - 1) / kBoundTile, nb = (cols + kBoundTile - 1) / kBoundTile;
    const float4 *bA0 = a.bounds + A.bounds_base + (long long)(ta * 2) * N;
    const float4 *bB0 = a.bounds + B.bounds_base + (long long)(tb * 2) * N;
    for (int w = tid >> 5; w < n_chunks; w += THREADS / 32) {
        const int k = (w << 5) + (tid & 31);
        bool act = k < N;
        if (act && a.cull) {
            float4 ba = bA0[k];
            if (na > 1) {
                const float4 q = bA0[N + k];
                ba = make_float4(fminf(ba.x, q.x), fminf(ba.y, q.y), fmaxf(ba.z, q.z), fmaxf(ba.w, q.w));
            }
            float4 bb = bB0[k];
            if (nb > 1) {
                const float4 q = bB0[N + k];
                bb = make_float4(fminf(bb.x, q.x), fminf(bb.y, q.y), fmaxf(bb.z, q.z), fmaxf(bb.w, q.w));
            }
            const float r = P.r_cull;
            act = (ba.x - r <= bb.z) && (bb.x - r <= ba.z) && (ba.y - r <= bb.w) && (bb.y - r <= ba.w);
        }
        const unsigned m = __ballot_sync(0xffffffffu, act);
        if ((tid & 31) == 0) s_mask[w] = m;
    }
    if (tid == 0) s_cursor = 0;
    __syncthreads();
    if (next_active(s_mask, n_chunks, 0) < 0) return;   // the tiles never come close: nothing to test

    // fused risk accumulation: [N] u64 masses | [N] u32 counts | [64][N] u64 log-survival cells of the
    // tile's EGO hypotheses (when N <= kFusedCellSteps)
    __shared__ float s_prob[2][kTile];
    __shared__ unsigned long long s_emass[kTile];
    __shared__ unsigned s_ehits[kTile];
    unsigned long long *s_H = s_acc;
    unsigned *s_cnt = reinterpret_cast<unsigned *>(s_acc + N);
    unsigned long long *s_L = s_acc + N + (N + 1) / 2;
    const bool smem_hist = FUSED && a.max_steps <= kFusedHistSteps;
    const bool smem_cells = smem_hist && a.max_steps <= kFusedCellSteps && P.ego_side >= 0;
    if (FUSED) {
        if (smem_hist)
            for (int q = tid; q < N; q += THREADS) { s_H[q] = 0ull; s_cnt[q] = 0u; }
        if (smem_cells)
            for (int q = tid; q < kTile * N; q += THREADS) s_L[q] = 0ull;
        for (int q = tid; q < 2 * kTile; q += THREADS) {
            const int r = q & (kTile - 1);
            if (q < kTile) {
                s_prob[0][r] = r < rows ? a.probf[A.traj_off + i0 + r] : 0.0f;
                s_emass[r] = 0ull;
                s_ehits[r] = 0u;
            } else {
                s_prob[1][r] = r < cols ? a.probf[B.traj_off + j0 + r] : 0.0f;
            }
        }
    }
    unsigned long long hit_cnt = 0, hit_mass = 0;

    const float la = A.hl, wa = A.hw, ra = A.rad, lb = B.hl, wb = B.hw, rb = B.rad;
    const float rc2 = P.rc2 + kEps0;     // (R_a + R_b)^2 plus the absolute slack
    const float ka = 0.5f * (1.0f - kEps);
    s_found[tid] = 0ull;                 // bit MJ m + n: pair (ti + TI m, tj + TJ n) has had its first hit
    unsigned long long narrow = 0;
    const int lane = tid & 31, warp = tid >> 5;
    unsigned short *queue = s_queue[warp];
    int active_steps = 0;
    for (;;) {
        if (tid == 0) {   // the next CH active steps
            int c = 0, k = next_active(s_mask, n_chunks, s_cursor);
            while (c < CH && k >= 0) {
                s_klist[c++] = k;
                k = next_active(s_mask, n_chunks, k + 1);
            }
            s_nk = c;
            s_cursor = k < 0 ? N : k;
        }
        __syncthreads();
        const int nk = s_nk;
        if (nk == 0) break;
        // stage: every pose of the chunk's steps, all loads issued before any is needed
#pragma unroll 4
        for (int e = tid; e < nk * 2 * kTile; e += THREADS) {
            const int c = e >> 7, q = e & (2 * kTile - 1);
            const int k = s_klist[c];
            if (q < kTile) {
                float x = kFar, y = 0.0f, cc = 1.0f, ss = 0.0f;
                if (q < rows) {
                    const long long idx = A.pose_base + (long long)k * A.h + i0 + q;
                    x = __ldg(a.x + idx); y = __ldg(a.y + idx); cc = __ldg(a.c + idx); ss = __ldg(a.s + idx);
                }
                s_pa[c * kTile + q] = make_float4(x, y, ka * fmaf(x, x, y * y), 0.0f);
                s_ra[c * kTile + q] = make_float2(cc, ss);
            } else {
                const int r = q - kTile;
                float x = -kFar, y = 0.0f, cc = 1.0f, ss = 0.0f;
                if (r < cols) {
                    const long long idx = B.pose_base + (long long)k * B.h + j0 + r;
                    x = __ldg(a.x + idx); y = __ldg(a.y + idx); cc = __ldg(a.c + idx); ss = __ldg(a.s + idx);
                }
                s_pb[c * kTile + r] = make_float4(x, y, 0.5f * fmaf(1.0f - kEps, fmaf(x, x, y * y), -rc2), 0.0f);
                s_rb[c * kTile + r] = make_float2(cc, ss);
            }
        }
        __syncthreads();
        active_steps += nk;
        for (int c = 0; c < nk; ++c) {
            const int k = s_klist[c];
            const float4 *pa_s = s_pa + c * kTile, *pb_s = s_pb + c * kTile;
            float4 pa[MI], pb[MJ];
#pragma unroll
            for (int m = 0; m < MI; ++m) pa[m] = pa_s[ti + TI * m];
#pragma unroll
            for (int n = 0; n < MJ; ++n) pb[n] = pb_s[tj + TJ * n];
            unsigned rowhit = 0;             // bit m: row m of the micro-tile has a broad-phase candidate
#pragma unroll
            for (int m = 0; m < MI; ++m) {
                bool any = false;
#pragma unroll
                for (int n = 0; n < MJ; ++n)
                    any |= fmaf(pa[m].x, pb[n].x, fmaf(pa[m].y, pb[n].y, -pb[n].z)) >= pa[m].z;
                rowhit |= any ? (1u << m) : 0u;
            }
            // candidates of this thread not yet decided: re-derived from shared memory for flagged rows
            unsigned long long cand = 0ull;
            if (rowhit) {
                const unsigned long long found = s_found[tid];
                while (rowhit) {
                    const int m = __ffs(rowhit) - 1;
                    rowhit &= rowhit - 1;
                    const float4 qa4 = pa_s[ti + TI * m];
#pragma unroll
                    for (int n = 0; n < MJ; ++n) {
                        const float4 qb4 = pb_s[tj + TJ * n];
                        if (fmaf(qa4.x, qb4.x, fmaf(qa4.y, qb4.y, -qb4.z)) >= qa4.z) cand |= 1ull << (MJ * m + n);
                    }
                }
                cand &= ~found;
            }
            // compact the warp's candidates and test them one per lane (the exact test is long: dense lanes)
            const int cnt = __popcll(cand);
            if (!__ballot_sync(0xffffffffu, cnt != 0)) continue;
            int off = cnt;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, off, d);
                if (lane >= d) off += u;
            }
            const int total = __shfl_sync(0xffffffffu, off, 31);
            off -= cnt;
            while (cand) {
                const int bit = __ffsll((long long)cand) - 1;
                cand &= cand - 1;
                queue[off++] = (unsigned short)((lane << 6) | bit);
            }
            __syncwarp();
            narrow += total;   // counted once per warp below (lane 0)
            for (int e = lane; e < total; e += 32) {
                const int ent = queue[e];
                const int owner = (warp << 5) | (ent >> 6), bit = ent & 63;
                const int m = bit / MJ, n = bit - m * MJ;
                const int i = owner / TJ + TI * m, j = owner % TJ + TJ * n;
                const float4 qa4 = pa_s[i], qb4 = pb_s[j];
                const float dx = qb4.x - qa4.x, dy = qb4.y - qa4.y;
                const float2 qa = s_ra[c * kTile + i], qb = s_rb[c * kTile + j];
                const bool hit = narrow_hit<OUTL>(shape, a.polys, dx, dy, qa, qb, la, wa, lb, wb, ra, rb);
                if (!hit) continue;
                atomicOr(s_found + owner, 1ull << bit);
                a.table[P.off + (long long)(i0 + i) * B.h + j0 + j] = (int16_t)k;
                if (FUSED) {   // the risk terms of this first hit (FP32 terms, exact fixed-point sums)
                    const float pa_ = s_prob[0][i], pb_ = s_prob[1][j];
                    const unsigned long long w = to_fixed(pa_ * pb_, kFixProb);
                    ++hit_cnt;
                    hit_mass += w;
                    if (smem_hist) {
                        atomicAdd(s_cnt + k, 1u);
                        atomicAdd(s_H + k, w);
                    } else {
                        atomicAdd(a.acc.count_k + P.kofs + k, 1ull);
                        atomicAdd(a.acc.H + P.kofs + k, w);
                    }
                    if (P.ego_side >= 0) {
                        const int eg = P.ego_side == 0 ? i : j;             // the EGO hypothesis
                        const float pco = P.ego_side == 0 ? pb_ : pa_;      // the CO hypothesis
                        atomicAdd(s_emass + eg, to_fixed(pco, kFixProb));
                        atomicAdd(s_ehits + eg, 1u);
                        const unsigned long long lq = to_fixed(neg_log_survival(pco), kFixLog);
                        if (smem_cells) {
                            atomicAdd(s_L + eg * N + k, lq);
                        } else {
                            const int e0 = P.ego_side == 0 ? i0 : j0;
                            atomicAdd(a.acc.lsum + P.lsum_base + ((long long)(e0 + eg) * N + k) * P.n_obj_s + P.co_local, lq);
                        }
                    }
                }
            }
            __syncwarp();
        }
        __syncthreads();   // the chunk's staged poses are no longer read
    }
    if (a.counters) {   // every lane of a warp counted the warp's exact tests: lane 0 reports them
        if ((tid & 31) == 0 && narrow) count_narrow(a, P.combo, narrow);
        if (tid == 0 && active_steps) atomicAdd(a.counters, (unsigned long long)active_steps * kTile * kTile);
    }
    if (FUSED) {   // merge the tile's risk accumulators into the global ones
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            hit_cnt += __shfl_xor_sync(0xffffffffu, hit_cnt, d);
            hit_mass += __shfl_xor_sync(0xffffffffu, hit_mass, d);
        }
        if ((tid & 31) == 0 && hit_cnt) {
            atomicAdd(a.acc.count + P.index, hit_cnt);
            atomicAdd(a.acc.P + P.index, hit_mass);
        }
        if (smem_hist) {
            for (int q = tid; q < N; q += THREADS) {
                if (s_cnt[q]) {
                    atomicAdd(a.acc.count_k + P.kofs + q, (unsigned long long)s_cnt[q]);
                    atomicAdd(a.acc.H + P.kofs + q, s_H[q]);
                }
            }
        }
        if (P.ego_side >= 0) {
            const int e0 = P.ego_side == 0 ? i0 : j0;
            for (int q = tid; q < kTile; q += THREADS) {
                if (s_ehits[q]) {
                    atomicAdd(a.acc.mass + P.mass_base + (long long)(e0 + q) * P.n_obj_s + P.co_local, s_emass[q]);
                    atomicAdd(a.acc.hits + P.hits_base + e0 + q, (unsigned long long)s_ehits[q]);
                }
            }
            if (smem_cells) {
                for (int q = tid; q < kTile * N; q += THREADS) {
                    const unsigned long long v = s_L[q];
                    if (v) {
                        const int e = q / N, kk = q - e * N;
                        atomicAdd(a.acc.lsum + P.lsum_base + ((long long)(e0 + e) * N + kk) * P.n_obj_s + P.co_local, v);
                    }
                }
            }
        }
    }
}

// Fused risk terms of one first hit (i, j) at step k of pair `pair` (FP32 terms, exact fixed-point sums)
// into the CTA's shared accumulators (or the global ones when they do not fit).
struct TileRisk {
    unsigned long long *s_H;
    unsigned *s_cnt;
    unsigned long long *s_L;
    float *pa, *pb;                     // [64] probabilities of the tile's rows / columns
    unsigned long long *emass;          // [64] per EGO hypothesis of the tile
    unsigned *ehits;
    bool hist, cells;
};

__device__ __forceinline__ void add_hit(const CollideArgs &a, const PairDesc &P, int pair, int N, const TileRisk &R,
                                        int i0, int j0, int i, int j, int k, unsigned long long &cnt,
                                        unsigned long long &mass) {
    const float pa_ = R.pa[i], pb_ = R.pb[j];
    const unsigned long long w = to_fixed(pa_ * pb_, kFixProb);
    ++cnt;
    mass += w;
    if (R.hist) {
        atomicAdd(R.s_cnt + k, 1u);
        atomicAdd(R.s_H + k, w);
    } else {
        atomicAdd(a.acc.count_k + P.kofs + k, 1ull);
        atomicAdd(a.acc.H + P.kofs + k, w);
    }
    if (P.ego_side >= 0) {
        const int e = P.ego_side == 0 ? i : j;                // the EGO hypothesis
        const float pco = P.ego_side == 0 ? pb_ : pa_;        // the CO hypothesis
        atomicAdd(R.emass + e, to_fixed(pco, kFixProb));
        atomicAdd(R.ehits + e, 1u);
        const unsigned long long lq = to_fixed(neg_log_survival(pco), kFixLog);
        if (R.cells) {
            atomicAdd(R.s_L + e * N + k, lq);
        } else {
            const int e0 = P.ego_side == 0 ? i0 : j0;
            atomicAdd(a.acc.lsum + P.lsum_base + ((long long)(e0 + e) * N + k) * P.n_obj_s + P.co_local, lq);
        }
    }
}

// Warp-per-step layout: a CTA of WARPS warps takes a 64 x 64 tile; its active steps are staged CH at a
// time, and warp w tests steps w, w + WARPS, ... of the chunk on its own (no barrier between steps).  A
// lane holds an 8 x 16 micro-tile (rows lr + 8 m, columns lc + 4 n with lr = lane / 4, lc = lane % 4), so
// a warp covers the 4096 pairs of a step and the per-step overhead (candidate compaction) is paid once
// per 4096 tests.  Candidates are tested one per lane; the earliest overlapping step of each pair is
// kept with a shared-memory atomicMin, and the first hits are stored (and their risk terms added) once,
// when the tile is done.
template <int WARPS, int CH, bool FUSED, bool OUTL>
__global__ void __launch_bounds__(WARPS * 32) collide_warp_kernel(const CollideArgs a) {
    pdl_start();
    constexpr int THREADS = WARPS * 32;
    constexpr int QCAP = 256;            // candidates compacted per warp per round
    extern __shared__ __align__(16) unsigned char s_dyn[];
    float4 *s_pa = reinterpret_cast<float4 *>(s_dyn);               // [CH][64] x, y, h_a
    float4 *s_pb = s_pa + CH * kTile;                                  // [CH][64] x, y, h_b
    float2 *s_ra = reinterpret_cast<float2 *>(s_pb + CH * kTile);     // [CH][64] c, s
    float2 *s_rb = s_ra + CH * kTile;
    int *s_first = reinterpret_cast<int *>(s_rb + CH * kTile);        // [64 * 64] earliest hit step
    unsigned long long *s_acc = reinterpret_cast<unsigned long long *>(s_first + kTile * kTile);
    __shared__ unsigned s_mask[kMaxChunks];
    __shared__ int s_klist[CH];
    __shared__ int s_nk, s_cursor;
    __shared__ unsigned short s_queue[WARPS][QCAP];

    const long long g = blockIdx.x;
    if (g >= a.n_tiles) return;
    const int lo = pair_of_tile(a, g);
    const PairDesc P = a.pairs[lo];
    const PairShape shape = shape_of(P);
    const ObjDesc &A = a.objs[P.a];
    const ObjDesc &B = a.objs[P.b];
    const int t = (int)(g - P.tile_start);          // < tiles_a x tiles_b <= n_tiles < 2^31
    const int ta = t / P.tiles_b, tb = t - ta * P.tiles_b;
    const int i0 = ta * kTile, j0 = tb * kTile;
    const int rows = min(kTile, A.h - i0), cols = min(kTile, B.h - j0);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int lr = lane >> 2, lc = lane & 3;
    const int N = P.n_steps;
    const int n_chunks = (N + 31) >> 5;

    const int na = (rows + kBoundTile - 1) / kBoundTile, nb = (cols + kBoundTile - 1) / kBoundTile;
    const float4 *bA0 = a.bounds + A.bounds_base + (long long)(ta * 2) * N;
    const float4 *bB0 = a.bounds + B.bounds_base + (long long)(tb * 2) * N;
    for (int w = warp; w < n_chunks; w += WARPS) {
        const int k = (w << 5) + lane;
        bool act = k < N;
        if (act && a.cull) {
            float4 ba = bA0[k];
            if (na > 1) {
                const float4 q = bA0[N + k];
                ba = make_float4(fminf(ba.x, q.x), fminf(ba.y, q.y), fmaxf(ba.z, q.z), fmaxf(ba.w, q.w));
            }
            float4 bb = bB0[k];
            if (nb > 1) {
                const float4 q = bB0[N + k];
                bb = make_float4(fminf(bb.x, q.x), fminf(bb.y, q.y), fmaxf(bb.z, q.z), fmaxf(bb.w, q.w));
            }
            const float r = P.r_cull;
            act = (ba.x - r <= bb.z) && (bb.x - r <= ba.z) && (ba.y - r <= bb.w) && (bb.y - r <= ba.w);
        }
        const unsigned m = __ballot_sync(0xffffffffu, act);
        if (lane == 0) s_mask[w] = m;
    }
    if (tid == 0) s_cursor = 0;
    __syncthreads();
    if (next_active(s_mask, n_chunks, 0) < 0) return;   // the tiles never come close: nothing to test
    for (int q = tid; q < kTile * kTile; q += THREADS) s_first[q] = kNoHit;

    const float la = A.hl, wa = A.hw, ra = A.rad, lb = B.hl, wb = B.hw, rb = B.rad;
    const float rc2 = P.rc2 + kEps0;
    const float ka = 0.5f * (1.0f - kEps);
    unsigned long long narrow = 0;
    int active_steps = 0;
    unsigned short *queue = s_queue[warp];
    for (;;) {
        if (tid == 0) {   // the next CH active steps
            int c = 0, k = next_active(s_mask, n_chunks, s_cursor);
            while (c < CH && k >= 0) {
                s_klist[c++] = k;
                k = next_active(s_mask, n_chunks, k + 1);
            }
            s_nk = c;
            s_cursor = k < 0 ? N : k;
        }
        __syncthreads();
        const int nk = s_nk;
        if (nk == 0) break;
#pragma unroll 4
        for (int e = tid; e < nk * 2 * kTile; e += THREADS) {
            const int c = e >> 7, q = e & (2 * kTile - 1);
            const int k = s_klist[c];
            if (q < kTile) {
                float x = kFar, y = 0.0f, cc = 1.0f, ss = 0.0f;
                if (q < rows) {
                    const long long idx = A.pose_base + (long long)k * A.h + i0 + q;
                    x = __ldg(a.x + idx); y = __ldg(a.y + idx); cc = __ldg(a.c + idx); ss = __ldg(a.s + idx);
                }
                s_pa[c * kTile + q] = make_float4(x, y, ka * fmaf(x, x, y * y), 0.0f);
                s_ra[c * kTile + q] = make_float2(cc, ss);
            } else {
                const int r = q - kTile;
                float x = -kFar, y = 0.0f, cc = 1.0f, ss = 0.0f;
                if (r < cols) {
                    const long long idx = B.pose_base + (long long)k * B.h + j0 + r;
                    x = __ldg(a.x + idx); y = __ldg(a.y + idx); cc = __ldg(a.c + idx); ss = __ldg(a.s + idx);
                }
                s_pb[c * kTile + r] = make_float4(x, y, 0.5f * fmaf(1.0f - kEps, fmaf(x, x, y * y), -rc2), 0.0f);
                s_rb[c * kTile + r] = make_float2(cc, ss);
            }
        }
        __syncthreads();
        active_steps += nk;
        for (int c = warp; c < nk; c += WARPS) {
            const int k = s_klist[c];
            const float4 *pa_s = s_pa + c * kTile, *pb_s = s_pb + c * kTile;
            float4 pa[8], pb[16];
#pragma unroll
            for (int m = 0; m < 8; ++m) pa[m] = pa_s[lr + 8 * m];
#pragma unroll
            for (int n = 0; n < 16; ++n) pb[n] = pb_s[lc + 4 * n];
            unsigned rowhit = 0;
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                bool any = false;
#pragma unroll
                for (int n = 0; n < 16; ++n)
                    any |= fmaf(pa[m].x, pb[n].x, fmaf(pa[m].y, pb[n].y, -pb[n].z)) >= pa[m].z;
                rowhit |= any ? (1u << m) : 0u;
            }
            if (!__ballot_sync(0xffffffffu, rowhit != 0)) continue;
            // this lane's candidates, 16 bits per flagged row (bit 16 m + n)
            unsigned long long cand_lo = 0ull, cand_hi = 0ull;
            while (rowhit) {
                const int m = __ffs(rowhit) - 1;
                rowhit &= rowhit - 1;
                const float4 qa4 = pa_s[lr + 8 * m];
                unsigned bits = 0;
#pragma unroll
                for (int n = 0; n < 16; ++n) {
                    const float4 qb4 = pb_s[lc + 4 * n];
                    bits |= (fmaf(qa4.x, qb4.x, fmaf(qa4.y, qb4.y, -qb4.z)) >= qa4.z) ? (1u << n) : 0u;
                }
                if (m < 4) cand_lo |= (unsigned long long)bits << (16 * m);
                else cand_hi |= (unsigned long long)bits << (16 * (m - 4));
            }
            // compact and test one candidate per lane, in rounds of at most QCAP
            for (;;) {
                int cnt = 0;
                unsigned short mine[8];
                while (cnt < 8 && (cand_lo | cand_hi)) {
                    int bit;
                    if (cand_lo) { bit = __ffsll((long long)cand_lo) - 1; cand_lo &= cand_lo - 1; }
                    else { bit = 64 + __ffsll((long long)cand_hi) - 1; cand_hi &= cand_hi - 1; }
                    mine[cnt++] = (unsigned short)((lane << 7) | bit);
                }
                if (!__ballot_sync(0xffffffffu, cnt != 0)) break;
                int off = cnt;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const int u = __shfl_up_sync(0xffffffffu, off, d);
                    if (lane >= d) off += u;
                }
                const int total = __shfl_sync(0xffffffffu, off, 31);
                off -= cnt;
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (q < cnt) queue[off + q] = mine[q];
                __syncwarp();
                narrow += total;
                for (int e = lane; e < total; e += 32) {
                    const int ent = queue[e];
                    const int owner = ent >> 7, bit = ent & 127;
                    const int m = bit >> 4, n = bit & 15;
                    const int i = (owner >> 2) + 8 * m, j = (owner & 3) + 4 * n;
                    if (s_first[i * kTile + j] <= k) continue;    // an earlier step already overlaps
                    const float4 qa4 = pa_s[i], qb4 = pb_s[j];
                    const float dx = qb4.x - qa4.x, dy = qb4.y - qa4.y;
                    const float2 qa = s_ra[c * kTile + i], qb = s_rb[c * kTile + j];
                    const bool hit = narrow_hit<OUTL>(shape, a.polys, dx, dy, qa, qb, la, wa, lb, wb, ra, rb);
                    if (hit) atomicMin(s_first + i * kTile + j, k);
                }
                __syncwarp();
            }
        }
        __syncthreads();   // the chunk's staged poses are no longer read
    }
    if (a.counters) {   // every lane counted its warp's exact tests: lane 0 reports them
        if (lane == 0 && narrow) count_narrow(a, P.combo, narrow);
        if (tid == 0 && active_steps) atomicAdd(a.counters, (unsigned long long)active_steps * kTile * kTile);
    }
    // first hits: store them (and add their risk terms)
    __shared__ float s_prob[2][kTile];
    __shared__ unsigned long long s_emass[kTile];
    __shared__ unsigned s_ehits[kTile];
    TileRisk R;
    R.s_H = s_acc;
    R.s_cnt = reinterpret_cast<unsigned *>(s_acc + N);
    R.s_L = s_acc + N + (N + 1) / 2;
    R.pa = s_prob[0];
    R.pb = s_prob[1];
    R.emass = s_emass;
    R.ehits = s_ehits;
    R.hist = FUSED && a.max_steps <= kFusedHistSteps;
    R.cells = R.hist && a.max_steps <= kFusedCellSteps && P.ego_side >= 0;
    if (FUSED) {
        if (R.hist)
            for (int q = tid; q < N; q += THREADS) { R.s_H[q] = 0ull; R.s_cnt[q] = 0u; }
        if (R.cells)
            for (int q = tid; q < kTile * N; q += THREADS) R.s_L[q] = 0ull;
        for (int q = tid; q < 2 * kTile; q += THREADS) {
            const int r = q & (kTile - 1);
            if (q < kTile) {
                s_prob[0][r] = r < rows ? a.probf[A.traj_off + i0 + r] : 0.0f;
                s_emass[r] = 0ull;
                s_ehits[r] = 0u;
            } else {
                s_prob[1][r] = r < cols ? a.probf[B.traj_off + j0 + r] : 0.0f;
            }
        }
        __syncthreads();
    }
    unsigned long long hit_cnt = 0, hit_mass = 0;
    for (int q = tid; q < kTile * kTile; q += THREADS) {
        const int k = s_first[q];
        if (k == kNoHit) continue;
        const int i = q >> 6, j = q & (kTile - 1);
        a.table[P.off + (long long)(i0 + i) * B.h + j0 + j] = (int16_t)k;
        if (FUSED) add_hit(a, P, lo, N, R, i0, j0, i, j, k, hit_cnt, hit_mass);
    }
    if (FUSED) {
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            hit_cnt += __shfl_xor_sync(0xffffffffu, hit_cnt, d);
            hit_mass += __shfl_xor_sync(0xffffffffu, hit_mass, d);
        }
        if (lane == 0 && hit_cnt) {
            atomicAdd(a.acc.count + P.index, hit_cnt);
            atomicAdd(a.acc.P + P.index, hit_mass);
        }
        __syncthreads();
        if (R.hist) {
            for (int q = tid; q < N; q += THREADS) {
                if (R.s_cnt[q]) {
                    atomicAdd(a.acc.count_k + P.kofs + q, (unsigned long long)R.s_cnt[q]);
                    atomicAdd(a.acc.H + P.kofs + q, R.s_H[q]);
                }
            }
        }
        if (P.ego_side >= 0) {
            const int e0 = P.ego_side == 0 ? i0 : j0;
            for (int q = tid; q < kTile; q += THREADS) {
                if (s_ehits[q]) {
                    atomicAdd(a.acc.mass + P.mass_base + (long long)(e0 + q) * P.n_obj_s + P.co_local, s_emass[q]);
                    atomicAdd(a.acc.hits + P.hits_base + e0 + q, (unsigned long long)s_ehits[q]);
                }
            }
            if (R.cells) {
                for (int q = tid; q < kTile * N; q += THREADS) {
                    const unsigned long long v = R.s_L[q];
                    if (v) {
                        const int e = q / N, kk = q - e * N;
                        atomicAdd(a.acc.lsum + P.lsum_base + ((long long)(e0 + e) * N + kk) * P.n_obj_s + P.co_local, v);
                    }
                }
            }
        }
    }
}

// Warp-per-tile layouts: each warp owns one TE x TE block of hypothesis pairs (a whole 64 x 64 tile, or
// one 32 x 32 quarter of it) and walks its active steps in ascending order on its own (no CTA barrier
// anywhere).  A lane holds an MI x MJ micro-block (rows lr + 8 m, columns lc + 4 n, lr = lane / 4,
// lc = lane % 4; 8 x 16 for TE = 64, 4 x 8 for TE = 32) and a register mask of its pairs that have
// already hit: because the steps come in order, the first narrow-phase hit of a pair is its first
// collision step, it is stored at once, and later candidates of that pair are dropped before any further
// work.  The warp stages each step's poses in its own shared-memory slot; the next active step's poses
// are loaded into registers while the current step is tested.  Activity (culling against the blocks'
// bounding boxes) is decided 32 steps at a time with one ballot.  Fused risk terms are added per hit with
// global atomics; the per-step histogram terms of one step's hits are summed over the warp first.
// One TE x TE block (warp task gw) walked by the calling warp; pa_s .. s_new are the warp's own slots.
template <int TE, bool FUSED, bool OUTL>
__device__ __forceinline__ void tile_block(const CollideArgs &a, long long gw, int lane, float4 *pa_s, float4 *pb_s,
                                           float2 *ra_s, float2 *rb_s, float *prob_s) {
    static_assert(TE == 64 || TE == 32, "block edge");
    constexpr int MI = TE / 8, MJ = TE / 4;       // micro-block of a lane
    constexpr int SUB = kTile / TE;               // blocks per tile edge
    const long long g = gw / (SUB * SUB);                 // the 64 x 64 tile
    if (g >= a.n_tiles) return;
    const int quarter = (int)(gw - g * (SUB * SUB));
    const int lo = pair_of_tile(a, g);
    const PairDesc &P = a.pairs[lo];   // fields read where used (fewer live registers)
    const PairShape shape = shape_of(P);
    const ObjDesc &A = a.objs[P.a];
    const ObjDesc &B = a.objs[P.b];
    const int t = (int)(g - P.tile_start);          // < tiles_a x tiles_b <= n_tiles < 2^31
    const int ta = t / P.tiles_b, tb = t - ta * P.tiles_b;
    const int ba_idx = ta * SUB + quarter / SUB, bb_idx = tb * SUB + quarter % SUB;   // blocks along a, b
    const int i0 = ba_idx * TE, j0 = bb_idx * TE;
    const int rows = min(TE, A.h - i0), cols = min(TE, B.h - j0);
    if (rows <= 0 || cols <= 0) return;                    // a quarter past a ragged edge
    const int lr = lane >> 2, lc = lane & 3;
    const int N = P.n_steps;
    const int na = (rows + kBoundTile - 1) / kBoundTile, nb = (cols + kBoundTile - 1) / kBoundTile;
    const float4 *bA0 = a.bounds + A.bounds_base + (long long)(i0 / kBoundTile) * N;
    const float4 *bB0 = a.bounds + B.bounds_base + (long long)(j0 / kBoundTile) * N;
    const float la = A.hl, wa = A.hw, ra = A.rad, lb = B.hl, wb = B.hw, rb = B.rad;
    const float rc2 = P.rc2 + kEps0;
    const float ka = 0.5f * (1.0f - kEps);
    const float r_cull = P.r_cull;
    if (TE == 32 && a.fill_blocks) {   // this block's table entries start as -1 (coalesced 64-byte row stores)
        int16_t *row = a.table + P.off + (long long)i0 * B.h + j0;
        for (int r = 0; r < rows; ++r, row += B.h)
            for (int c = lane; c < cols; c += 32) row[c] = (int16_t)-1;
        __syncwarp();      // the fill is ordered before this warp's first-hit stores
    }
    if (FUSED) {   // the block's probabilities, read at every first hit (kept off the hit path's latency)
#pragma unroll
        for (int u = 0; u < TE / 32; ++u) {
            const int r = lane + 32 * u;
            prob_s[r] = r < rows ? a.probf[A.traj_off + i0 + r] : 0.0f;
            prob_s[TE + r] = r < cols ? a.probf[B.traj_off + j0 + r] : 0.0f;
        }
    }

    // activity of the 32 steps from k0 (one ballot)
    auto chunk_mask = [&](int k0) -> unsigned {
        const int k = k0 + lane;
        bool act = k < N;
        if (act && a.cull) {
            float4 ba = bA0[k];
            if (na > 1) {
                const float4 q = bA0[N + k];
                ba = make_float4(fminf(ba.x, q.x), fminf(ba.y, q.y), fmaxf(ba.z, q.z), fmaxf(ba.w, q.w));
            }
            float4 bb = bB0[k];
            if (nb > 1) {
                const float4 q = bB0[N + k];
                bb = make_float4(fminf(bb.x, q.x), fminf(bb.y, q.y), fmaxf(bb.z, q.z), fmaxf(bb.w, q.w));
            }
            act = (ba.x - r_cull <= bb.z) && (bb.x - r_cull <= ba.z) && (ba.y - r_cull <= bb.w) &&
                  (bb.y - r_cull <= ba.w);
        }
        return __ballot_sync(0xffffffffu, act);
    };
    int k0 = 0;
    unsigned mask = chunk_mask(0);
    // next active step after k (-1: none); advances k0 / mask (warp-uniform)
    auto next_step = [&](int k) -> int {
        unsigned m = k < k0 ? mask : mask & ~((2u << (k - k0)) - 1u);
        while (!m) {
            k0 += 32;
            if (k0 >= N) return -1;
            mask = chunk_mask(k0);
            m = mask;
        }
        return k0 + __ffs(m) - 1;
    };
    // this lane's share of a step's poses: rows lane (+ 32) of A, then columns lane (+ 32) of B
    constexpr int NU = 2 * (TE / 32);
    float px[NU], py[NU], pc[NU], ps[NU];
    auto load_step = [&](int k) {
#pragma unroll
        for (int u = 0; u < NU; ++u) {
            const bool isA = u < NU / 2;
            const int r = lane + 32 * (isA ? u : u - NU / 2);
            const bool ok = isA ? r < rows : r < cols;
            const long long idx = isA ? A.pose_base + (long long)k * A.h + i0 + r
                                      : B.pose_base + (long long)k * B.h + j0 + r;
            px[u] = ok ? __ldg(a.x + idx) : (isA ? kFar : -kFar);
            py[u] = ok ? __ldg(a.y + idx) : 0.0f;
            pc[u] = ok ? __ldg(a.c + idx) : 1.0f;
            ps[u] = ok ? __ldg(a.s + idx) : 0.0f;
        }
    };

    unsigned long long found_lo = 0ull, found_hi = 0ull;   // bit MJ m + n of the lane's pairs
    unsigned long long narrow = 0, hit_cnt = 0, hit_mass = 0;
    int active_steps = 0;
    int k = next_step(-1);
    if (k >= 0) load_step(k);
    while (k >= 0) {
        __syncwarp();                       // the previous step's slot is no longer read
#pragma unroll
        for (int u = 0; u < NU; ++u) {
            const bool isA = u < NU / 2;
            const int r = lane + 32 * (isA ? u : u - NU / 2);
            const float q2 = fmaf(px[u], px[u], py[u] * py[u]);
            if (isA) {
                pa_s[r] = make_float4(px[u], py[u], ka * q2, 0.0f);
                ra_s[r] = make_float2(pc[u], ps[u]);
            } else {
                pb_s[r] = make_float4(px[u], py[u], 0.5f * fmaf(1.0f - kEps, q2, -rc2), 0.0f);
                rb_s[r] = make_float2(pc[u], ps[u]);
            }
        }
        __syncwarp();
        const int kn = next_step(k);
        if (kn >= 0) load_step(kn);         // in flight while this step is tested
        ++active_steps;
        // broad phase: candidate bit MJ m + n (bits 0-63 in c_lo, 64-127 in c_hi)
        float ax[MI], ay[MI], ah[MI];
#pragma unroll
        for (int m = 0; m < MI; ++m) {
            const float4 q = pa_s[lr + 8 * m];
            ax[m] = q.x; ay[m] = q.y; ah[m] = q.z;
        }
        unsigned long long c_lo = 0ull, c_hi = 0ull;
#pragma unroll
        for (int n = 0; n < MJ; ++n) {
            const float4 qb = pb_s[lc + 4 * n];
#pragma unroll
            for (int m = 0; m < MI; ++m) {
                if (fmaf(ax[m], qb.x, fmaf(ay[m], qb.y, -qb.z)) >= ah[m]) {
                    const int bit = MJ * m + n;
                    if (bit < 64) c_lo |= 1ull << bit;
                    else c_hi |= 1ull << (bit - 64);
                }
            }
        }
        c_lo &= ~found_lo;
        c_hi &= ~found_hi;
        if (__ballot_sync(0xffffffffu, (c_lo | c_hi) != 0ull)) {
            bool any_hit = false;
            unsigned long long step_cnt = 0, step_mass = 0;
            // each lane tests the candidates of its own micro-block (a loop as long as the lane with the most;
            // measured faster than compacting them into a warp queue first), so a hit sets its own mask bit
            for (int h = 0; h < 2; ++h) {
                unsigned long long cm = h ? c_hi : c_lo;
                while (cm) {
                    const int bit = 64 * h + __ffsll((long long)cm) - 1;
                    cm &= cm - 1ull;
                    ++narrow;
                    const int m = bit / MJ, n = bit % MJ;
                    const int i = lr + 8 * m, j = lc + 4 * n;
                    const float4 qa4 = pa_s[i], qb4 = pb_s[j];
                    const float dx = qb4.x - qa4.x, dy = qb4.y - qa4.y;
                    const float2 qa = ra_s[i], qb = rb_s[j];
                    if (!narrow_hit<OUTL>(shape, a.polys, dx, dy, qa, qb, la, wa, lb, wb, ra, rb)) continue;
                    any_hit = true;
                    if (h) found_hi |= 1ull << (bit - 64); else found_lo |= 1ull << bit;
                    a.table[P.off + (long long)(i0 + i) * B.h + j0 + j] = (int16_t)k;
                    if (FUSED) {
                        const float pa_ = prob_s[i], pb_ = prob_s[TE + j];
                        const unsigned long long w = to_fixed(pa_ * pb_, kFixProb);
                        ++step_cnt;
                        step_mass += w;
                        if (P.ego_side >= 0) {
                            const int e = P.ego_side == 0 ? i0 + i : j0 + j;     // the EGO hypothesis
                            const float pco = P.ego_side == 0 ? pb_ : pa_;       // the CO hypothesis
                            atomicAdd(a.acc.mass + P.mass_base + (long long)e * P.n_obj_s + P.co_local,
                                      to_fixed(pco, kFixProb));
                            atomicAdd(a.acc.hits + P.hits_base + e, 1ull);
                            atomicAdd(a.acc.lsum + P.lsum_base + ((long long)e * N + k) * P.n_obj_s + P.co_local,
                                      to_fixed(neg_log_survival(pco), kFixLog));
                        }
                    }
                }
            }
            if (__any_sync(0xffffffffu, any_hit)) {
                if (FUSED) {
#pragma unroll
                    for (int d = 16; d > 0; d >>= 1) {
                        step_cnt += __shfl_xor_sync(0xffffffffu, step_cnt, d);
                        step_mass += __shfl_xor_sync(0xffffffffu, step_mass, d);
                    }
                    if (lane == 0) {
                        atomicAdd(a.acc.count_k + P.kofs + k, step_cnt);
                        atomicAdd(a.acc.H + P.kofs + k, step_mass);
                    }
                    hit_cnt += step_cnt;
                    hit_mass += step_mass;
                }
            }
        }
        k = kn;
    }
    if (a.counters) {
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) narrow += __shfl_xor_sync(0xffffffffu, narrow, d);
    }
    if (a.counters && lane == 0) {
        if (narrow) count_narrow(a, P.combo, narrow);
        if (active_steps) atomicAdd(a.counters, (unsigned long long)active_steps * TE * TE);
    }
    if (FUSED && lane == 0 && hit_cnt) {
        atomicAdd(a.acc.count + P.index, hit_cnt);
        atomicAdd(a.acc.P + P.index, hit_mass);
    }
}

// The warp-per-block layouts: each warp takes blocks gw = blockIdx.x * WARPS + warp, then every
// gridDim.x * WARPS further (a grid smaller than the work, max_ctas, leaves SM room to other streams).
template <int WARPS, int TE, bool FUSED, bool OUTL>
__global__ void __launch_bounds__(WARPS * 32, (TE == 64 ? 16 : 24) / WARPS) collide_tile_kernel(const CollideArgs a) {
    pdl_start();
    constexpr int SUB = kTile / TE;
    __shared__ float4 s_pa[WARPS][TE];            // x, y, h_a
    __shared__ float4 s_pb[WARPS][TE];            // x, y, h_b
    __shared__ float2 s_ra[WARPS][TE];            // c, s
    __shared__ float2 s_rb[WARPS][TE];
    __shared__ float s_prob[WARPS][FUSED ? 2 * TE : 1];    // fused: the block's row and column probabilities
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long total = a.n_tiles * (SUB * SUB);
    for (long long gw = (long long)blockIdx.x * WARPS + warp; gw < total; gw += (long long)gridDim.x * WARPS)
        tile_block<TE, FUSED, OUTL>(a, gw, lane, s_pa[warp], s_pb[warp], s_ra[warp], s_rb[warp], s_prob[warp]);
}

// ---- step-item layout (variant 6): the active (block, step) pairs of a small scene in parallel ----------
//
// The warp-per-block layouts walk a block's steps in order, so a block whose objects stay close for many
// steps is one long chain, and on small scenes the launch waits for it.  Here a first kernel lists every
// active step of every 32 x 32 block as an item; then persistent warps test one item each, all steps at
// once, keeping a pair's earliest overlapping step in a 32-bit scratch array with a fire-and-forget
// atomicMin (INT_MAX: none); a third kernel writes the int16 table from it and adds the risk terms of the
// first hits.  Pairs that already hit are retested at later steps (there is no in-order mask).

// the pair of global 32 x 32 block gw (4 per 64 x 64 tile) and the block's origin and extent
struct BlockAt {
    int pair, i0, j0, rows, cols;
};

__device__ __forceinline__ BlockAt block_at(const CollideArgs &a, long long gw) {
    const long long g = gw >> 2;
    const int quarter = (int)(gw & 3);
    const int lo = pair_of_tile(a, g);
    const PairDesc &P = a.pairs[lo];
    const int t = (int)(g - P.tile_start);          // < tiles_a x tiles_b <= n_tiles < 2^31
    const int ta = t / P.tiles_b, tb = t - ta * P.tiles_b;
    BlockAt r;
    r.pair = lo;
    r.i0 = (ta * 2 + (quarter >> 1)) * 32;
    r.j0 = (tb * 2 + (quarter & 1)) * 32;
    r.rows = min(32, a.objs[P.a].h - r.i0);
    r.cols = min(32, a.objs[P.b].h - r.j0);
    return r;
}

// What the listing needs of one block, from the descriptors alone (no output of an earlier kernel).
struct ListBlock {
    BlockAt blk;
    int n, ha, hb;
    float rc;
    long long bounds_a, bounds_b, pose_a, pose_b, entry0;
};

__device__ __forceinline__ ListBlock list_block(const CollideArgs &a, long long gw) {
    ListBlock L;
    L.blk = block_at(a, gw);
    const PairDesc &P = a.pairs[L.blk.pair];
    const ObjDesc &A = a.objs[P.a];
    const ObjDesc &B = a.objs[P.b];
    L.n = P.n_steps;
    L.ha = A.h;
    L.hb = B.h;
    L.rc = P.r_cull;
    L.bounds_a = A.bounds_base + (long long)(L.blk.i0 / kBoundTile) * L.n;
    L.bounds_b = B.bounds_base + (long long)(L.blk.j0 / kBoundTile) * L.n;
    L.pose_a = A.pose_base + L.blk.i0;
    L.pose_b = B.pose_base + L.blk.j0;
    L.entry0 = P.off + (long long)L.blk.i0 * B.h + L.blk.j0;
    return L;
}

// One warp per block (grid-stride): its active steps appended to the item list (one ballot per 32 steps,
// one atomic per ballot); then a block without any writes its table entries (-1) at once, and an active
// block sets its first-step entries to INT_MAX and joins the list of active blocks.  The first block's
// descriptors are read before the wait for the bounds kernel, so their chain of dependent loads (pair
// search, pair, objects) overlaps the bounds kernel's tail.  Bounded to 48 registers (ten CTAs per SM), so
// that one CTA per tile, up to 1520 tiles, is resident at once.
__global__ void __launch_bounds__(128, 10) items_list_kernel(const CollideArgs a) {
    pdl_trigger();
    const int lane = threadIdx.x & 31;
    const long long total = a.n_tiles * 4, stride = (long long)gridDim.x * 4;
    long long gw = (long long)blockIdx.x * 4 + (threadIdx.x >> 5);
    ListBlock L{};
    if (gw < total) L = list_block(a, gw);
    pdl_wait();
    for (bool first = true; gw < total; gw += stride, first = false) {
        if (!first) L = list_block(a, gw);
        const BlockAt &blk = L.blk;
        if (blk.rows <= 0 || blk.cols <= 0) continue;            // a quarter past a ragged edge
        const int N = L.n;
        int n_active = 0;
        const float4 *bA0 = a.bounds + L.bounds_a;
        const float4 *bB0 = a.bounds + L.bounds_b;
        const float rc = L.rc;
        for (int k0 = 0; k0 < N; k0 += 32) {
            const int k = k0 + lane;
            bool act = k < N;
            if (act && a.cull) {
                const float4 ba = bA0[k], bb = bB0[k];
                act = (ba.x - rc <= bb.z) && (bb.x - rc <= ba.z) && (ba.y - rc <= bb.w) && (bb.y - rc <= ba.w);
            }
            const unsigned m = __ballot_sync(0xffffffffu, act);
            if (!m) continue;
            n_active += __popc(m);
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(a.item_count, (unsigned long long)__popc(m));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (act) {
                const unsigned long long at = base + __popc(m & ((1u << lane) - 1u));
                if (at < (unsigned long long)a.max_items) {
                    StepItem itm;
                    itm.pa = L.pose_a + (long long)k * L.ha;
                    itm.pb = L.pose_b + (long long)k * L.hb;
                    itm.gw = (int)gw;
                    itm.k = k;
                    a.items[at] = itm;
                }
            }
        }
        const long long base = L.entry0 + lane;
        if (n_active == 0) {                    // never close: the table entries are final now
            if (lane < blk.cols)
                for (int r = 0; r < blk.rows; ++r) a.table[base + (long long)r * L.hb] = (int16_t)-1;
            continue;
        }
        if (lane < blk.cols)
            for (int r = 0; r < blk.rows; ++r) a.first32[base + (long long)r * L.hb] = 0x7fffffff;
        if (lane == 0) {
            const PairDesc &P = a.pairs[blk.pair];
            const ObjDesc &A = a.objs[P.a];
            const ObjDesc &B = a.objs[P.b];
            const unsigned long long at = atomicAdd(a.active_count, 1ull);
            if (at < (unsigned long long)(a.n_tiles * 4)) a.active[at] = (int)gw;
            ItemBlock rec;
            rec.entry0 = L.entry0;
            rec.h_b = L.hb; rec.pair = blk.pair; rec.rows = blk.rows; rec.cols = blk.cols;
            rec.rc2 = P.rc2; rec.la = A.hl; rec.wa = A.hw; rec.ra = A.rad; rec.lb = B.hl; rec.wb = B.hw; rec.rb = B.rad;
            rec.i0 = blk.i0; rec.j0 = blk.j0;
            a.blocks[gw] = rec;
        }
    }
}

// Persistent warps (kItemWarps independent warps per CTA, 32 per SM) take items it = warp, + warps, ...:
// stage the block's 32 + 32 poses of the item's step, broad phase on a 4 x 8 micro-block per lane,
// candidates compacted and tested one per lane, hits kept with atomicMin on the first-step array (no
// return value: nothing waits on it).  One warp per CTA: on the 11-object scene 1, 2 and 4 warps per CTA
// ran alike, and with octagon outlines one was 12 % faster than two or four.
constexpr int kItemWarps = 1;

template <bool OUTL>
__global__ void __launch_bounds__(32 * kItemWarps, 32 / kItemWarps) items_kernel(const CollideArgs a) {
    pdl_start();
    constexpr int MI = 4, MJ = 8;
    __shared__ float4 pa_w[kItemWarps][32], pb_w[kItemWarps][32];   // x, y, h
    __shared__ float2 ra_w[kItemWarps][32], rb_w[kItemWarps][32];   // c, s
    __shared__ unsigned short queue_w[kItemWarps][256];
    __shared__ unsigned long long ncls_w[kItemWarps][5];             // narrow tests by shape class
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, lr = lane >> 2, lc = lane & 3;
    if (lane < 5) ncls_w[w][lane] = 0ull;
    float4 *pa_s = pa_w[w], *pb_s = pb_w[w];
    float2 *ra_s = ra_w[w], *rb_s = rb_w[w];
    unsigned short *queue = queue_w[w];
    const float ka = 0.5f * (1.0f - kEps);
    const unsigned long long listed = *a.item_count;
    const long long count = listed < (unsigned long long)a.max_items ? (long long)listed : a.max_items;
    const long long first = (long long)blockIdx.x * kItemWarps + w, stride = (long long)gridDim.x * kItemWarps;
    unsigned long long narrow = 0, executed = 0;
    StepItem next;                                                   // one item ahead
    if (first < count) next = a.items[first];
    for (long long it = first; it < count; it += stride) {
        const StepItem item = next;
        if (it + stride < count) next = a.items[it + stride];
        const int k = item.k;
        const ItemBlock bk = a.blocks[item.gw];                      // loaded beside the poses
        const float rc2 = bk.rc2 + kEps0;
        const bool oka = lane < bk.rows, okb = lane < bk.cols;
        const long long ia = item.pa + lane;
        const long long ib = item.pb + lane;
        const float xa = oka ? __ldg(a.x + ia) : kFar, ya = oka ? __ldg(a.y + ia) : 0.0f;
        const float ca = oka ? __ldg(a.c + ia) : 1.0f, sa = oka ? __ldg(a.s + ia) : 0.0f;
        const float xb = okb ? __ldg(a.x + ib) : -kFar, yb = okb ? __ldg(a.y + ib) : 0.0f;
        const float cb = okb ? __ldg(a.c + ib) : 1.0f, sb = okb ? __ldg(a.s + ib) : 0.0f;
        __syncwarp();                           // the previous item's slot is no longer read
        pa_s[lane] = make_float4(xa, ya, ka * fmaf(xa, xa, ya * ya), 0.0f);
        ra_s[lane] = make_float2(ca, sa);
        pb_s[lane] = make_float4(xb, yb, 0.5f * fmaf(1.0f - kEps, fmaf(xb, xb, yb * yb), -rc2), 0.0f);
        rb_s[lane] = make_float2(cb, sb);
        __syncwarp();
        executed += 32 * 32;
        float ax[MI], ay[MI], ah[MI];
#pragma unroll
        for (int m = 0; m < MI; ++m) {
            const float4 q = pa_s[lr + 8 * m];
            ax[m] = q.x; ay[m] = q.y; ah[m] = q.z;
        }
        unsigned cand = 0u;                     // bit MJ m + n
#pragma unroll
        for (int n = 0; n < MJ; ++n) {
            const float4 qb = pb_s[lc + 4 * n];
#pragma unroll
            for (int m = 0; m < MI; ++m)
                if (fmaf(ax[m], qb.x, fmaf(ay[m], qb.y, -qb.z)) >= ah[m]) cand |= 1u << (MJ * m + n);
        }
        if (!__ballot_sync(0xffffffffu, cand != 0u)) continue;
        const PairDesc &P = a.pairs[bk.pair];
        const PairShape shape = shape_of(P);
        const float la = bk.la, wa = bk.wa, ra = bk.ra, lb = bk.lb, wb = bk.wb, rb = bk.rb;
        for (;;) {                              // rounds of at most 8 candidates per lane
            const int cnt = min(__popc(cand), 8);
            int off, total;
            if (!queue_offsets(cnt, lane, off, total)) break;
            for (int q = 0; q < cnt; ++q) {
                const int bit = __ffs(cand) - 1;
                cand &= cand - 1u;
                queue[off + q] = (unsigned short)((lane << 7) | bit);
            }
            __syncwarp();
            narrow += total;
            if (lane == 0) ncls_w[w][narrow_class(P.combo)] += total;
            for (int e = lane; e < total; e += 32) {
                const int ent = queue[e];
                const int owner = ent >> 7, bit = ent & 127;
                const int i = (owner >> 2) + 8 * (bit / MJ), j = (owner & 3) + 4 * (bit % MJ);
                const float4 qa4 = pa_s[i], qb4 = pb_s[j];
                const float dx = qb4.x - qa4.x, dy = qb4.y - qa4.y;
                const float2 qa = ra_s[i], qb = rb_s[j];
                const bool hit = narrow_hit<OUTL>(shape, a.polys, dx, dy, qa, qb, la, wa, lb, wb, ra, rb);
                if (hit) atomicMin(a.first32 + bk.entry0 + (long long)i * bk.h_b + j, k);
            }
            __syncwarp();
        }
    }
    if (a.counters && lane == 0) {
        if (narrow) atomicAdd(a.counters + 1, narrow);
        for (int q = 0; q < 5; ++q)
            if (ncls_w[w][q]) atomicAdd(a.counters + 2 + q, ncls_w[w][q]);
        if (executed) atomicAdd(a.counters, executed);
    }
}

// The table of the step-item layout from the first-step array, and (probf set) the risk terms of its first
// hits: one CTA per active block (grid-stride), lane = column, warp w takes rows 8w .. 8w + 7 (its 8 loads
// in flight together), writes the int16 entries and adds each first hit's terms with the fixed-point
// atomics of the fused layouts (the same sums, in any order).  Four short chains per block instead of one
// warp walking 32 rows: the launch is latency-bound.
constexpr int kTableCtasPerSm = 18;

__global__ void __launch_bounds__(128) items_table_kernel(const CollideArgs a) {
    pdl_start();
    __shared__ float s_pa[32];                       // the block's row probabilities
    __shared__ unsigned long long s_sub[8][16];      // EGO rows: sums of the CO masses of any subset of
                                                     // columns 4q .. 4q + 3 (bit b of m: column 4q + b)
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const bool risk = a.probf != nullptr;
    const unsigned long long listed = *a.active_count;
    const long long total = listed < (unsigned long long)(a.n_tiles * 4) ? (long long)listed : a.n_tiles * 4;
    for (long long q = blockIdx.x; q < total; q += gridDim.x) {
        // the block's record (written by the listing kernel): its first-step rows are one load away, and this
        // warp's 8 rows are loaded before the shared set-up below
        const ItemBlock bk = a.blocks[a.active[q]];
        const int r0 = 8 * w;
        const long long hb = bk.h_b, base = bk.entry0 + lane;
        const bool col_ok = lane < bk.cols;
        int v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
            v[u] = col_ok && r0 + u < bk.rows ? a.first32[base + (long long)(r0 + u) * hb] : 0x7fffffff;
        const PairDesc &P = a.pairs[bk.pair];
        const int N = P.n_steps, ego_side = P.ego_side, n_obj_s = P.n_obj_s, co_local = P.co_local;
        const long long kofs = P.kofs, lsum_base = P.lsum_base;
        const float pb = risk && col_ok ? a.probf[a.objs[P.b].traj_off + bk.j0 + lane] : 0.0f;
        __syncthreads();                             // the previous block's slots are no longer read
        if (w == 0) s_pa[lane] = risk && lane < bk.rows ? a.probf[a.objs[P.a].traj_off + bk.i0 + lane] : 0.0f;
        if (risk && ego_side == 0) {                 // a row's CO mass = the sum over its colliding columns
            const unsigned long long c = to_fixed(pb, kFixProb);   // zero past the block's columns
            const int g = threadIdx.x >> 4, m = threadIdx.x & 15;  // one subset sum per thread
            unsigned long long sum = 0;
#pragma unroll
            for (int bt = 0; bt < 4; ++bt) {
                const unsigned long long cb = __shfl_sync(0xffffffffu, c, 4 * g + bt);   // column 4g + bt (every warp holds them)
                if (m >> bt & 1) sum += cb;
            }
            s_sub[g][m] = sum;
        }
        __syncthreads();
        if (r0 >= bk.rows) continue;                 // a ragged block's missing rows (uniform per warp)
        bool any = false;
#pragma unroll
        for (int u = 0; u < 8; ++u) any |= v[u] != 0x7fffffff;
        if (!__ballot_sync(0xffffffffu, any)) {      // no hit in these 8 rows
            if (col_ok)
                for (int u = 0; u < 8 && r0 + u < bk.rows; ++u) a.table[base + (long long)(r0 + u) * hb] = -1;
            continue;
        }
        // each lane adds its own first hits' terms; an EGO row's totals come from one ballot
        unsigned long long cnt = 0, mass = 0, col_mass = 0;
        unsigned col_hits = 0;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int r = r0 + u;
            if (r >= bk.rows) break;                 // uniform over the warp
            const int k = v[u] == 0x7fffffff ? -1 : v[u];
            if (col_ok) a.table[base + (long long)r * hb] = (int16_t)k;
            if (!risk) continue;
            if (k >= 0) {
                const float pa = s_pa[r];
                const unsigned long long wt = to_fixed(pa * pb, kFixProb);
                ++cnt;
                mass += wt;
                atomicAdd(a.acc.count_k + kofs + k, 1ull);
                atomicAdd(a.acc.H + kofs + k, wt);
                if (ego_side >= 0) {
                    const long long e = ego_side == 0 ? bk.i0 + r : bk.j0 + lane;   // the EGO hypothesis
                    const float pco = ego_side == 0 ? pb : pa;                        // the CO hypothesis
                    atomicAdd(a.acc.lsum + lsum_base + (e * N + k) * n_obj_s + co_local,
                              to_fixed(neg_log_survival(pco), kFixLog));
                    if (ego_side == 1) {
                        col_mass += to_fixed(pco, kFixProb);
                        ++col_hits;
                    }
                }
            }
            if (ego_side == 0) {                     // the row's EGO hypothesis: CO mass and hits
                const unsigned hm = __ballot_sync(0xffffffffu, k >= 0);
                if (hm && lane == 0) {
                    unsigned long long rm = 0;
#pragma unroll
                    for (int g = 0; g < 8; ++g) rm += s_sub[g][(hm >> (4 * g)) & 15];
                    const long long e = bk.i0 + r;
                    atomicAdd(a.acc.mass + P.mass_base + e * n_obj_s + co_local, rm);
                    atomicAdd(a.acc.hits + P.hits_base + e, (unsigned long long)__popc(hm));
                }
            }
        }
        if (!risk) continue;
        if (ego_side == 1 && col_hits) {             // the warp's share of the block's EGO columns
            const long long e = bk.j0 + lane;
            atomicAdd(a.acc.mass + P.mass_base + e * n_obj_s + co_local, col_mass);
            atomicAdd(a.acc.hits + P.hits_base + e, (unsigned long long)col_hits);
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            cnt += __shfl_xor_sync(0xffffffffu, cnt, d);
            mass += __shfl_xor_sync(0xffffffffu, mass, d);
        }
        if (lane == 0 && cnt) {
            atomicAdd(a.acc.count + P.index, cnt);
            atomicAdd(a.acc.P + P.index, mass);
        }
    }
}

// ---- block layout (variant 7): one CTA per 32 x 32 block, its active steps spread over the CTA's warps --
//
// Each CTA owns one 32 x 32 block of hypothesis pairs.  Every warp reads the block's descriptors (before
// the wait for the previous kernel: they are uploaded data) and decides the block's active steps itself
// (one ballot per 32 steps over the tile bounds: the same loads and the same result in every warp, so no
// barrier is needed for it).  Warp w then takes the active steps of rank w, w + W, w + 2W, ... in
// ascending order: the step's 32 + 32 poses staged in its own shared slot (its next step's poses in flight
// meanwhile), the broad phase on a 4 x 8 micro-block per lane, then each lane tests its own candidates (a
// loop as long as the lane with the most: 34.8 us against 37.0 us for a warp-wide selection that hands
// them out one per lane).  The block's first hits live in shared memory (atomicMin per hit); a candidate
// whose pair already holds a step <= k there -- an earlier hit of this warp, or of another warp that got there first -- is
// dropped before its narrow test.  After one barrier the CTA writes the block's int16 table rows and,
// fused, adds the risk terms of its first hits, again one hit per lane (the per-hypothesis fixed-point
// terms come precomputed by the risk preparation).  One launch does what the step-item layout does in three,
// with neither an item list nor a first-step array in global memory, and a block that never comes close
// writes its -1 rows and ends.  A CTA per 32 x 32 block keeps the work fine-grained: a CTA per 64 x 64
// tile (four blocks) was measured at 74.8 us against 43.5 us on the 11-object scene, its heaviest tiles
// holding the launch's tail.
#ifndef MHC_BLOCK_WARPS
#define MHC_BLOCK_WARPS 4
#endif
#ifndef MHC_BLOCK_MIN_CTAS
#define MHC_BLOCK_MIN_CTAS 6
#endif
// Four warps per block and a register bound of six CTAs per SM (80 registers): on the 11-object scene the
// collision stage took 37.8 us so, 39.0 us at eight CTAs per SM (64 registers, small spills), 52-58 us
// with two or eight warps per block.
constexpr int kBlockWarps = MHC_BLOCK_WARPS;
constexpr int kBlockMinCtas = MHC_BLOCK_MIN_CTAS;

// What the block layouts need of one 32 x 32 block: the pair, the table origin (entry (i, j) at
// entry0 + i hb + j), the first pose of its row / column object's block (pose (k, i) at pose_a + k ha + i),
// the bound boxes of step k at bA0[k] / bB0[k], the extent and the shapes.
struct BlockJob {
    const PairDesc *P;
    long long entry0, pose_a, pose_b, traj_a, traj_b;
    const float4 *bA0, *bB0;
    int ha, hb, N, rows, cols, i0, j0;
    float rcull, rc2, la, wa, ra, lb, wb, rb;
};

// Asynchronous 4- and 8-byte copies global -> shared (both addresses aligned to the size); cp_async_wait()
// returns once the calling thread's copies have landed (a barrier then shows them to the CTA).
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Active steps k0 .. k0 + 31 of a block (one ballot over the two bound tiles' boxes; every lane calls it).
__device__ __forceinline__ unsigned block_chunk_mask(const CollideArgs &a, const BlockJob &J, int k0) {
    const int k = k0 + (threadIdx.x & 31);
    bool act = k < J.N;
    if (act && a.cull) {
        const float4 ba = J.bA0[k], bb = J.bB0[k];
        const float rc = J.rcull;
        act = (ba.x - rc <= bb.z) && (bb.x - rc <= ba.z) && (ba.y - rc <= bb.w) && (bb.y - rc <= ba.w);
    }
    return __ballot_sync(0xffffffffu, act);
}

// The work of one block with an active step, by the whole CTA (k0 / mask: the first chunk of 32 steps with
// an active step and its active steps).  The table's -1s are written beforehand; this stores first hits.
template <int W, bool FUSED, bool OUTL>
__device__ __forceinline__ void block_work(const CollideArgs &a, const BlockJob &J, int k0, unsigned mask,
                                           float4 (*s_pa)[32], float4 (*s_pb)[32], float2 (*s_ra)[32],
                                           float2 (*s_rb)[32], int *s_first, float *s_prow, float *s_pcol,
                                           unsigned long long *s_lfix, unsigned long long *s_pfix) {
    constexpr int MI = 4, MJ = 8, ROWS = 32 / W;
    constexpr int kNone = 0x7fffffff;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, lr = lane >> 2, lc = lane & 3;
    const PairDesc &P = *J.P;
    const PairShape shape = shape_of(P);
    const int N = J.N, rows = J.rows, cols = J.cols;
    const bool col_ok = lane < cols;
    for (int q = threadIdx.x; q < 32 * 32; q += W * 32) s_first[q] = kNone;
    // the epilogue's per-hypothesis inputs, copied asynchronously (their latency hides under the step loop):
    // the row and column probabilities and, for an EGO pair, the CO side's fixed-point terms
    if (FUSED && w == 0) {
        if (lane < rows) cp_async4(s_prow + lane, a.probf + J.traj_a + lane); else s_prow[lane] = 0.0f;
        if (col_ok) cp_async4(s_pcol + lane, a.probf + J.traj_b + lane); else s_pcol[lane] = 0.0f;
    }
    if (FUSED && w == (W > 1 ? 1 : 0) && P.ego_side >= 0) {
        const bool co_ok = P.ego_side == 0 ? col_ok : lane < rows;
        const long long co = (P.ego_side == 0 ? J.traj_b : J.traj_a) + lane;
        if (co_ok) {
            cp_async8(s_lfix + lane, a.lfix + co);
            cp_async8(s_pfix + lane, a.pfix + co);
        }
    }

    // ---- the warp's active steps: ranks w, w + W, ... in ascending step order ----
    int rank0 = 0;                                  // active steps before the chunk k0 .. k0 + 31
    auto my_bits = [&](unsigned m) -> unsigned {    // this warp's steps of a chunk (lane b: step k0 + b)
        const bool own = ((m >> lane) & 1u) && (((rank0 + __popc(m & ((1u << lane) - 1u))) & (W - 1)) == w);
        return __ballot_sync(0xffffffffu, own);
    };
    unsigned mine = my_bits(mask);
    auto next_mine = [&]() -> int {                 // warp-uniform; -1 when none is left
        for (;;) {
            if (mine) {
                const int b = __ffs(mine) - 1;
                mine &= mine - 1u;
                return k0 + b;
            }
            rank0 += __popc(mask);
            k0 += 32;
            if (k0 >= N) return -1;
            mask = block_chunk_mask(a, J, k0);
            mine = my_bits(mask);
        }
    };
    const bool oka = lane < rows, okb = col_ok;
    const long long pose_a = J.pose_a + lane, pose_b = J.pose_b + lane;
    const long long ha = J.ha, hb = J.hb;
    float xa = kFar, ya = 0.0f, ca = 1.0f, sa = 0.0f, xb = -kFar, yb = 0.0f, cb = 1.0f, sb = 0.0f;
    auto load = [&](int k) {                        // lane: row `lane` of A and column `lane` of B
        const long long ia = pose_a + (long long)k * ha, ib = pose_b + (long long)k * hb;
        if (oka) { xa = __ldg(a.x + ia); ya = __ldg(a.y + ia); ca = __ldg(a.c + ia); sa = __ldg(a.s + ia); }
        if (okb) { xb = __ldg(a.x + ib); yb = __ldg(a.y + ib); cb = __ldg(a.c + ib); sb = __ldg(a.s + ib); }
    };
    float4 *pa_s = s_pa[w], *pb_s = s_pb[w];
    float2 *ra_s = s_ra[w], *rb_s = s_rb[w];
    const float ka = 0.5f * (1.0f - kEps);
    const float rc2 = J.rc2 + kEps0;
    unsigned narrow = 0;                            // this lane's narrow tests
    int steps = 0;
    int k = next_mine();
    if (k >= 0) load(k);                            // in flight across the barrier
    __syncthreads();                                // s_first initialised
    while (k >= 0) {
        __syncwarp();                               // the previous step's slot is no longer read
        pa_s[lane] = make_float4(xa, ya, ka * fmaf(xa, xa, ya * ya), 0.0f);
        ra_s[lane] = make_float2(ca, sa);
        pb_s[lane] = make_float4(xb, yb, 0.5f * fmaf(1.0f - kEps, fmaf(xb, xb, yb * yb), -rc2), 0.0f);
        rb_s[lane] = make_float2(cb, sb);
        __syncwarp();
        const int kn = next_mine();
        if (kn >= 0) load(kn);                      // in flight while this step is tested
        ++steps;
        float ax[MI], ay[MI], ah[MI];
#pragma unroll
        for (int m = 0; m < MI; ++m) {
            const float4 q = pa_s[lr + 8 * m];
            ax[m] = q.x; ay[m] = q.y; ah[m] = q.z;
        }
        unsigned cand = 0u;                         // bit MJ m + n: pair (lr + 8 m, lc + 4 n)
#pragma unroll
        for (int n = 0; n < MJ; ++n) {
            const float4 qb = pb_s[lc + 4 * n];
#pragma unroll
            for (int m = 0; m < MI; ++m)
                if (fmaf(ax[m], qb.x, fmaf(ay[m], qb.y, -qb.z)) >= ah[m]) cand |= 1u << (MJ * m + n);
        }
        if (__ballot_sync(0xffffffffu, cand != 0u)) {
            while (cand) {                          // each lane its own candidates, in bit order
                const int bit = __ffs(cand) - 1;
                cand &= cand - 1u;
                const int i = lr + 8 * (bit / MJ), j = lc + 4 * (bit % MJ);
                int *first = s_first + 32 * i + j;
                if (*first <= k) continue;          // the pair already hit at this step or earlier
                ++narrow;
                const float4 qa4 = pa_s[i], qb4 = pb_s[j];
                const float dx = qb4.x - qa4.x, dy = qb4.y - qa4.y;
                if (narrow_hit<OUTL>(shape, a.polys, dx, dy, ra_s[i], rb_s[j], J.la, J.wa, J.lb, J.wb, J.ra, J.rb))
                    atomicMin(first, k);
            }
            __syncwarp();
        }
        k = kn;
    }
    if (a.counters) {
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) narrow += __shfl_xor_sync(0xffffffffu, narrow, d);
        if (lane == 0) {
            if (narrow) count_narrow(a, P.combo, narrow);
            if (steps) atomicAdd(a.counters, (unsigned long long)steps * 32 * 32);
        }
    }
    if (FUSED) cp_async_wait();
    __syncthreads();                                // every first hit of the block is in s_first (and the copies)

    // ---- the first hits of this warp's rows, one hit per lane: the table entry and (fused) the risk terms ----
    const int r0 = w * ROWS;
    if (r0 >= rows) return;
    unsigned hits = 0u;                             // bit u: row r0 + u of this lane's column hit
#pragma unroll
    for (int u = 0; u < ROWS; ++u)
        if (r0 + u < rows && col_ok && s_first[32 * (r0 + u) + lane] != kNone) hits |= 1u << u;
    if (!__ballot_sync(0xffffffffu, hits != 0u)) return;
    // the pair's risk fields in registers (read through the descriptor they would be read again after
    // every atomic)
    const int ego_side = P.ego_side, n_obj_s = P.n_obj_s, co_local = P.co_local, pidx = P.index;
    const long long kofs = P.kofs, lsum_base = P.lsum_base, mass_base = P.mass_base, hits_base = P.hits_base;
    unsigned long long cnt = 0, mass = 0;
    int16_t *tab = a.table + J.entry0 + (long long)r0 * hb;
    for_each_candidate(hits, lane, [&](int col, int u) {
        const int r = r0 + u;
        const int kk = s_first[32 * r + col];
        tab[u * hb + col] = (int16_t)kk;
        if (!FUSED) return;
        const unsigned long long wt = to_fixed(s_prow[r] * s_pcol[col], kFixProb);
        ++cnt;
        mass += wt;
        atomicAdd(a.acc.count_k + kofs + kk, 1ull);
        atomicAdd(a.acc.H + kofs + kk, wt);
        if (ego_side >= 0) {
            const long long e = ego_side == 0 ? J.i0 + r : J.j0 + col;                // EGO hypothesis
            const int co = ego_side == 0 ? col : r;                                  // CO hypothesis (block-local)
            atomicAdd(a.acc.lsum + lsum_base + (e * N + kk) * n_obj_s + co_local, s_lfix[co]);
            atomicAdd(a.acc.mass + mass_base + e * n_obj_s + co_local, s_pfix[co]);
            atomicAdd(a.acc.hits + hits_base + e, 1ull);
        }
    });
    if constexpr (FUSED) {
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            cnt += __shfl_xor_sync(0xffffffffu, cnt, d);
            mass += __shfl_xor_sync(0xffffffffu, mass, d);
        }
        if (lane == 0 && cnt) {
            atomicAdd(a.acc.count + pidx, cnt);
            atomicAdd(a.acc.P + pidx, mass);
        }
    }
}

// The block of 32 x 32 block index gw from the descriptors (uploaded data only).
__device__ __forceinline__ BlockJob block_job(const CollideArgs &a, long long gw) {
    const long long g = gw >> 2;
    const int quarter = (int)(gw & 3);
    const int pidx = pair_of_tile(a, g);
    const PairDesc &P = a.pairs[pidx];              // carries the objects' fields: no further load
    const int t = (int)(g - P.tile_start);          // < tiles_a x tiles_b <= n_tiles < 2^31
    const int ta = t / P.tiles_b, tb = t - ta * P.tiles_b;
    BlockJob J;
    J.P = &P;
    J.i0 = (ta * 2 + (quarter >> 1)) * 32;
    J.j0 = (tb * 2 + (quarter & 1)) * 32;
    J.ha = P.h_a;
    J.hb = P.h_b;
    J.rows = min(32, J.ha - J.i0);
    J.cols = min(32, J.hb - J.j0);
    J.N = P.n_steps;
    J.entry0 = P.off + (long long)J.i0 * J.hb + J.j0;
    J.pose_a = P.pose_a + J.i0;
    J.pose_b = P.pose_b + J.j0;
    J.traj_a = P.traj_a + J.i0;
    J.traj_b = P.traj_b + J.j0;
    J.bA0 = a.bounds + P.bounds_a + (long long)(J.i0 / kBoundTile) * J.N;
    J.bB0 = a.bounds + P.bounds_b + (long long)(J.j0 / kBoundTile) * J.N;
    J.rcull = P.r_cull;
    J.rc2 = P.rc2;
    J.la = P.hl_a; J.wa = P.hw_a; J.ra = P.rad_a; J.lb = P.hl_b; J.wb = P.hw_b; J.rb = P.rad_b;
    return J;
}

// Variant 7: one CTA per 32 x 32 block (the hardware hands out blocks as CTAs finish, which balances the
// uneven blocks; persistent CTAs walking a fixed share of the blocks, with the scene's descriptors cached in
// shared memory, were measured at 57 us against 39 us on the 11-object scene).  Every warp reads the block's
// descriptors before the wait for the previous kernel (uploaded data) and decides the activity itself.
template <int W, bool FUSED, bool OUTL>
__global__ void __launch_bounds__(W * 32, kBlockMinCtas) block_kernel(const CollideArgs a) {
    static_assert(W == 1 || W == 2 || W == 4 || W == 8, "warps per block");
    pdl_trigger();
    __shared__ float4 s_pa[W][32], s_pb[W][32];     // x, y, h
    __shared__ float2 s_ra[W][32], s_rb[W][32];     // c, s
    __shared__ int s_first[32 * 32];                // first overlapping step of pair (i, j) at 32 i + j
    __shared__ float s_prow[32], s_pcol[32];        // fused: the block's row and column probabilities
    __shared__ unsigned long long s_lfix[32], s_pfix[32];   // fused EGO pair: the CO side's fixed-point terms
    const BlockJob J = block_job(a, (long long)blockIdx.x);
    pdl_wait();
    if (J.rows <= 0 || J.cols <= 0) return;         // a quarter past a ragged edge (whole CTA)
    int k0 = 0;
    unsigned mask = block_chunk_mask(a, J, 0);
    while (!mask && k0 + 32 < J.N) {
        k0 += 32;
        mask = block_chunk_mask(a, J, k0);
    }
    if (!mask) return;                              // the block never comes close: its entries keep the -1
    block_work<W, FUSED, OUTL>(a, J, k0, mask, s_pa, s_pb, s_ra, s_rb, s_first, s_prow, s_pcol, s_lfix, s_pfix);
}

// ---- block-list layout (variant 8): active blocks listed first, then a CTA per listed block ----
//
// On small scenes most blocks never come close (3,170 of the 11-object scene's 5,780), yet in variant 7 each
// costs a CTA its chain of dependent descriptor and bound loads.  Here one warp per block (4 per CTA, all of
// a small scene's warps resident at once) decides the activity and appends a self-contained record of each
// active block; the block kernel then reads one record per CTA (a single load) and does the work of
// variant 7.  Both CTAs past the list's end and the listing's empty blocks end at once; the table's -1s are
// written beforehand.
__global__ void __launch_bounds__(128, 10) block_list_kernel(const CollideArgs a) {
    pdl_trigger();
    const int lane = threadIdx.x & 31;
    const long long total = a.n_tiles * 4, stride = (long long)gridDim.x * 4;
    long long gw = (long long)blockIdx.x * 4 + (threadIdx.x >> 5);
    BlockJob J{};
    if (gw < total) J = block_job(a, gw);          // uploaded descriptors: before the wait
    pdl_wait();
    for (bool first = true; gw < total; gw += stride, first = false) {
        if (!first) J = block_job(a, gw);
        if (J.rows <= 0 || J.cols <= 0) continue;   // a quarter past a ragged edge
        int k0 = 0;
        unsigned mask = block_chunk_mask(a, J, 0);
        while (!mask && k0 + 32 < J.N) {
            k0 += 32;
            mask = block_chunk_mask(a, J, k0);
        }
        if (!mask) continue;
        if (lane == 0) {
            const unsigned long long at = atomicAdd(a.active_count, 1ull);
            if (at < (unsigned long long)total) {
                ActiveBlock r;
                r.entry0 = J.entry0; r.pose_a = J.pose_a; r.pose_b = J.pose_b;
                r.bounds_a = J.bA0 - a.bounds; r.bounds_b = J.bB0 - a.bounds;
                r.traj_a = J.traj_a; r.traj_b = J.traj_b;
                r.h_a = J.ha; r.h_b = J.hb; r.n_steps = J.N; r.pair = (int)(J.P - a.pairs);
                r.rows = J.rows; r.cols = J.cols; r.i0 = J.i0; r.j0 = J.j0;
                r.rcull = J.rcull; r.rc2 = J.rc2; r.la = J.la; r.wa = J.wa; r.ra = J.ra;
                r.lb = J.lb; r.wb = J.wb; r.rb = J.rb;
                r.k0 = k0;
                r.mask = mask;
                a.recs[at] = r;
            }
        }
    }
}

template <int W, bool FUSED, bool OUTL>
__global__ void __launch_bounds__(W * 32, kBlockMinCtas) block_rec_kernel(const CollideArgs a) {
    pdl_start();                                    // the records are the listing kernel's output
    __shared__ float4 s_pa[W][32], s_pb[W][32];
    __shared__ float2 s_ra[W][32], s_rb[W][32];
    __shared__ int s_first[32 * 32];
    __shared__ float s_prow[32], s_pcol[32];
    __shared__ unsigned long long s_lfix[32], s_pfix[32];
    const unsigned long long listed = *a.active_count;
    const ActiveBlock r = a.recs[blockIdx.x];       // within the array even past the list's end
    if ((unsigned long long)blockIdx.x >= listed) return;
    BlockJob J;
    J.P = a.pairs + r.pair;
    J.entry0 = r.entry0; J.pose_a = r.pose_a; J.pose_b = r.pose_b; J.traj_a = r.traj_a; J.traj_b = r.traj_b;
    J.bA0 = a.bounds + r.bounds_a; J.bB0 = a.bounds + r.bounds_b;
    J.ha = r.h_a; J.hb = r.h_b; J.N = r.n_steps; J.rows = r.rows; J.cols = r.cols; J.i0 = r.i0; J.j0 = r.j0;
    J.rcull = r.rcull; J.rc2 = r.rc2; J.la = r.la; J.wa = r.wa; J.ra = r.ra; J.lb = r.lb; J.wb = r.wb; J.rb = r.rb;
    block_work<W, FUSED, OUTL>(a, J, r.k0, r.mask, s_pa, s_pb, s_ra, s_rb, s_first, s_prow, s_pcol, s_lfix, s_pfix);
}

// table[0, n) = -1 (no collision), 16-byte stores on the aligned body
__global__ void __launch_bounds__(256) fill_kernel(int16_t *table, long long n) {
    pdl_start();
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long head = min(n, (long long)((16 - ((uintptr_t)table & 15)) & 15) / 2);
    if (tid < head) table[tid] = (int16_t)-1;
    const long long body = (n - head) / 8;
    int4 *v = reinterpret_cast<int4 *>(table + head);
    const int4 ones = make_int4(-1, -1, -1, -1);
    for (long long q = tid; q < body; q += stride) v[q] = ones;
    for (long long q = head + body * 8 + tid; q < n; q += stride) table[q] = (int16_t)-1;
}

}  // namespace

cudaError_t launch_fill_table(int16_t *table, long long n, cudaStream_t st, bool pdl) {
    if (n <= 0) return cudaSuccess;
    long long blocks = (n / 8 + 255) / 256 + 1;
    if (blocks > 152 * 16) blocks = 152 * 16;
    return launch_kernel(fill_kernel, dim3((unsigned)blocks), dim3(256), 0, st, pdl, table, n);
}

template <int THREADS, int MI, int MJ, int CH, bool FUSED, bool OUTL>
cudaError_t launch_variant(const CollideArgs &a, cudaStream_t st, bool pdl) {
    size_t smem = (size_t)CH * kTile * (2 * sizeof(float4) + 2 * sizeof(float2));
    if (FUSED) {
        if (a.max_steps <= kFusedHistSteps) smem += 8 * ((size_t)a.max_steps + (a.max_steps + 1) / 2);
        if (a.max_steps <= kFusedCellSteps) smem += 8 * (size_t)kTile * a.max_steps;
    }
    if (smem > 32 * 1024) {   // dynamic + static (about 5 KiB) above the default 48 KiB needs the opt-in
        cudaError_t e = cudaFuncSetAttribute(collide_kernel<THREADS, MI, MJ, CH, FUSED, OUTL>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    return launch_kernel(collide_kernel<THREADS, MI, MJ, CH, FUSED, OUTL>, dim3((unsigned)a.n_tiles), dim3(THREADS),
                         smem, st, pdl, a);
}

template <int WARPS, int CH, bool FUSED, bool OUTL>
cudaError_t launch_warp_variant(const CollideArgs &a, cudaStream_t st, bool pdl) {
    size_t smem = (size_t)CH * kTile * (2 * sizeof(float4) + 2 * sizeof(float2)) + sizeof(int) * kTile * kTile;
    if (FUSED) {
        if (a.max_steps <= kFusedHistSteps) smem += 8 * ((size_t)a.max_steps + (a.max_steps + 1) / 2);
        if (a.max_steps <= kFusedCellSteps) smem += 8 * (size_t)kTile * a.max_steps;
    }
    if (smem > 32 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(collide_warp_kernel<WARPS, CH, FUSED, OUTL>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    return launch_kernel(collide_warp_kernel<WARPS, CH, FUSED, OUTL>, dim3((unsigned)a.n_tiles), dim3(WARPS * 32),
                         smem, st, pdl, a);
}

template <int WARPS, int TE, bool FUSED, bool OUTL>
cudaError_t launch_tile_variant(const CollideArgs &a, cudaStream_t st, bool pdl) {
    constexpr int SUB = kTile / TE;
    const long long warps = a.n_tiles * SUB * SUB;
    long long blocks = (warps + WARPS - 1) / WARPS;
    if (a.max_ctas > 0 && blocks > a.max_ctas) blocks = a.max_ctas;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    return launch_kernel(collide_tile_kernel<WARPS, TE, FUSED, OUTL>, dim3((unsigned)blocks), dim3(WARPS * 32), 0,
                         st, pdl, a);
}

template <bool OUTL>
cudaError_t launch_collide_t(const CollideArgs &a, cudaStream_t st, bool pdl) {
    if (a.n_tiles <= 0) return cudaSuccess;
    if (a.n_tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    if (a.variant == 6) {   // the caller zeroed *item_count and sized items and first32
        if (!a.items || !a.item_count || !a.first32 || !a.active || !a.active_count || !a.blocks ||
            a.n_tiles * 4 > 0x7fffffffLL)
            return cudaErrorInvalidValue;
        long long blocks = (a.n_tiles * 4 + 3) / 4;
        if (blocks > 152 * 16) blocks = 152 * 16;
        cudaError_t e = launch_kernel(items_list_kernel, dim3((unsigned)blocks), dim3(128), 0, st, pdl, a);
        if (e != cudaSuccess) return e;
        int n_sm = 152, dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        e = launch_kernel(items_kernel<OUTL>, dim3((unsigned)(32 / kItemWarps * n_sm)), dim3(32 * kItemWarps), 0, st,
                          true, a);
        if (e != cudaSuccess) return e;
        // one CTA per active block, at most kTableCtasPerSm per SM (the rest grid-stride)
        const long long tblocks = std::min(a.n_tiles * 4, (long long)kTableCtasPerSm * n_sm);
        return launch_kernel(items_table_kernel, dim3((unsigned)tblocks), dim3(128), 0, st, true, a);
    }
    if (a.variant == 8) {   // listing, then one CTA per listed block; the table's -1s and the list's count are
                            // written beforehand
        if (!a.recs || !a.active_count || a.n_tiles * 4 > 0x7fffffffLL) return cudaErrorInvalidValue;
        long long blocks = (a.n_tiles * 4 + 3) / 4;
        if (blocks > 152 * 16) blocks = 152 * 16;
        cudaError_t e = launch_kernel(block_list_kernel, dim3((unsigned)blocks), dim3(128), 0, st, pdl, a);
        if (e != cudaSuccess) return e;
        const dim3 grid((unsigned)(a.n_tiles * 4)), block(32 * kBlockWarps);
        return a.probf ? launch_kernel(block_rec_kernel<kBlockWarps, true, OUTL>, grid, block, 0, st, true, a)
                       : launch_kernel(block_rec_kernel<kBlockWarps, false, OUTL>, grid, block, 0, st, true, a);
    }
    if (a.variant == 7) {   // one CTA per 32 x 32 block; the table's -1s are written beforehand
        if (a.n_tiles * 4 > 0x7fffffffLL) return cudaErrorInvalidValue;
        const dim3 grid((unsigned)(a.n_tiles * 4)), block(32 * kBlockWarps);
        return a.probf ? launch_kernel(block_kernel<kBlockWarps, true, OUTL>, grid, block, 0, st, pdl, a)
                       : launch_kernel(block_kernel<kBlockWarps, false, OUTL>, grid, block, 0, st, pdl, a);
    }
    if (a.variant == 4)
        return a.probf ? launch_tile_variant<4, 64, true, OUTL>(a, st, pdl) : launch_tile_variant<4, 64, false, OUTL>(a, st, pdl);
    if (a.variant == 5)   // one warp per CTA: a finished warp frees its slot at once (small, uneven grids)
        return a.probf ? launch_tile_variant<1, 32, true, OUTL>(a, st, pdl) : launch_tile_variant<1, 32, false, OUTL>(a, st, pdl);
    // variant 1: 4 x 4 micro-tiles with 256 threads (8 warps share each tile's tests); variant 2: 8 x 8 with
    // 64 threads; variant 3: one warp per step (8 x 16 lanes).  The caller picks one (autotuned per size).
    const bool many = a.variant == 2;
    if (a.variant == 3)
        return a.probf ? launch_warp_variant<4, 8, true, OUTL>(a, st, pdl) : launch_warp_variant<4, 8, false, OUTL>(a, st, pdl);
    if (a.probf)
        return many ? launch_variant<64, 8, 8, 8, true, OUTL>(a, st, pdl)
                    : launch_variant<256, 4, 4, 16, true, OUTL>(a, st, pdl);
    return many ? launch_variant<64, 8, 8, 8, false, OUTL>(a, st, pdl)
                : launch_variant<256, 4, 4, 16, false, OUTL>(a, st, pdl);
}

cudaError_t launch_collide(const CollideArgs &a, cudaStream_t st, bool pdl) {
    return a.polys ? launch_collide_t<true>(a, st, pdl) : launch_collide_t<false>(a, st, pdl);
}

}  // namespace mhc
