// collide.cu -- collision recognition (Section IV-C): first overlapping step of every hypothesis pair.
//
// Work decomposition: the table is first filled with -1 (HBM-bound); then one CTA per 64 x 64 tile of
// hypothesis pairs of one object pair walks the active steps in order: per step it stages the 64 + 64
// poses of its tile in shared memory (double buffered, one barrier per step, the next step's poses
// already loading) and every thread tests a register micro-tile (8 x 8 with 64 threads when the launch
// has many tiles, 4 x 4 with 256 threads when it has few and the slowest tile sets the time).  A 64-bit
// register mask remembers which of the thread's pairs have had their first hit; only first hits are
// stored.
//
// Broad phase (per test, 3 FP32 instructions): with h_a = (1 - eps)|p_a|^2 / 2 and
// h_b = ((1 - eps)|p_b|^2 - R^2 - eps0) / 2 precomputed at staging, the pair is a candidate iff
//     x_a x_b + y_a y_b - h_b >= h_a   <=>   |p_a - p_b|^2 <= R^2 + eps0 + eps (|p_a|^2 + |p_b|^2),
// R = sum of circumradii.  eps = 1e-5 exceeds the FP32 rounding error of the expanded form (< 7 * 2^-24
// relative to |p|^2) by more than 10x, so no true candidate is ever rejected; the narrow phase then
// decides exactly on direct coordinate differences.
// Narrow phase: separating-axis test on the four edge normals (rectangle-rectangle), clamped distance in
// the rectangle frame (rectangle-disc), centre distance (disc-disc).  Closed sets: touching overlaps.
// Culling: steps at which the two tiles' bounding boxes, inflated by R, do not meet are skipped whole
// (result-preserving).  The first hit of a pair is kept (steps are visited in ascending order).
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

constexpr int kMaxChunks = (32767 + 31) / 32;   // 32-step activity words for the longest horizon

// One staged pose per (thread, slot): slot q < 64 is hypothesis i0 + q of object a, q >= 64 is
// hypothesis j0 + q - 64 of object b; padding rows and columns sit far away.
__device__ __forceinline__ float4 load_pose(const CollideArgs &a, const ObjDesc &A, const ObjDesc &B, int k, int i0,
                                            int j0, int rows, int cols, int q) {
    if (q < kTile) {
        if (q < rows) {
            const long long idx = A.pose_base + (long long)k * A.h + i0 + q;
            return make_float4(__ldg(a.x + idx), __ldg(a.y + idx), __ldg(a.c + idx), __ldg(a.s + idx));
        }
        return make_float4(kFar, 0.0f, 1.0f, 0.0f);
    }
    q -= kTile;
    if (q < cols) {
        const long long idx = B.pose_base + (long long)k * B.h + j0 + q;
        return make_float4(__ldg(a.x + idx), __ldg(a.y + idx), __ldg(a.c + idx), __ldg(a.s + idx));
    }
    return make_float4(-kFar, 0.0f, 1.0f, 0.0f);
}

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

// THREADS threads per 64 x 64 tile, each testing an MI x MJ micro-tile: rows ti + TI m, columns tj + TJ n.
template <int THREADS, int MI, int MJ>
__global__ void __launch_bounds__(THREADS) collide_kernel(const CollideArgs a) {
    constexpr int TI = kTile / MI, TJ = kTile / MJ;
    static_assert(TI * TJ == THREADS, "micro-tiles must cover the tile");
    static_assert(MI * MJ <= 64, "first-hit mask is 64 bits");
    constexpr int SLOTS = (2 * kTile + THREADS - 1) / THREADS;   // staged poses per thread
    __shared__ float4 s_pa[2][kTile];    // x, y, h_a
    __shared__ float4 s_pb[2][kTile];    // x, y, h_b
    __shared__ float2 s_ra[2][kTile];    // c, s
    __shared__ float2 s_rb[2][kTile];
    __shared__ unsigned s_mask[kMaxChunks];

    const long long g = blockIdx.x;
    if (g >= a.n_tiles) return;
    int lo = 0, hi = a.n_pairs - 1;      // last pair whose first tile is <= g
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (a.pairs[mid].tile_start <= g) lo = mid; else hi = mid - 1;
    }
    const PairDesc P = a.pairs[lo];
    const ObjDesc &A = a.objs[P.a];
    const ObjDesc &B = a.objs[P.b];
    const long long t = g - P.tile_start;
    const int ta = (int)(t / P.tiles_b), tb = (int)(t - (long long)ta * P.tiles_b);
    const int i0 = ta * kTile, j0 = tb * kTile;
    const int rows = min(kTile, A.h - i0), cols = min(kTile, B.h - j0);
    const int tid = threadIdx.x, ti = tid / TJ, tj = tid % TJ;
    const int N = a.n_steps;
    const int n_chunks = (N + 31) >> 5;

    // activity of every step: the two tiles' centre boxes, grown by both circumradii, must meet
    const int na = (rows + kBoundTile - 1) / kBoundTile, nb = (cols + kBoundTile - 1) / kBoundTile;
    const float4 *bA0 = a.bounds + (long long)(A.tile_base + ta * 2) * N;
    const float4 *bB0 = a.bounds + (long long)(B.tile_base + tb * 2) * N;
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
    __syncthreads();

    const float la = A.hl, wa = A.hw, ra = A.rad, lb = B.hl, wb = B.hw, rb = B.rad;
    const float rc2 = P.rc2 + kEps0;     // (R_a + R_b)^2 plus the absolute slack
    const float ka = 0.5f * (1.0f - kEps);
    unsigned long long found = 0ull;     // bit MJ m + n: pair (ti + TI m, tj + TJ n) has had its first hit
    unsigned long long narrow = 0;
    int buf = 0, active_steps = 0;
    int k = next_active(s_mask, n_chunks, 0);
    float4 nxt[SLOTS];
    if (k >= 0) {
#pragma unroll
        for (int q = 0; q < SLOTS; ++q)
            if (tid + q * THREADS < 2 * kTile) nxt[q] = load_pose(a, A, B, k, i0, j0, rows, cols, tid + q * THREADS);
    }
    while (k >= 0) {
#pragma unroll
        for (int q = 0; q < SLOTS; ++q) {
            const int slot = tid + q * THREADS;
            if (slot < kTile) {
                s_pa[buf][slot] = make_float4(nxt[q].x, nxt[q].y, ka * fmaf(nxt[q].x, nxt[q].x, nxt[q].y * nxt[q].y), 0.0f);
                s_ra[buf][slot] = make_float2(nxt[q].z, nxt[q].w);
            } else if (slot < 2 * kTile) {
                const float hb = 0.5f * fmaf(1.0f - kEps, fmaf(nxt[q].x, nxt[q].x, nxt[q].y * nxt[q].y), -rc2);
                s_pb[buf][slot - kTile] = make_float4(nxt[q].x, nxt[q].y, hb, 0.0f);
                s_rb[buf][slot - kTile] = make_float2(nxt[q].z, nxt[q].w);
            }
        }
        const int k_next = next_active(s_mask, n_chunks, k + 1);
        if (k_next >= 0) {   // the next step's poses load while this step is tested
#pragma unroll
            for (int q = 0; q < SLOTS; ++q)
                if (tid + q * THREADS < 2 * kTile)
                    nxt[q] = load_pose(a, A, B, k_next, i0, j0, rows, cols, tid + q * THREADS);
        }
        __syncthreads();
        ++active_steps;
        float4 pa[MI], pb[MJ];
#pragma unroll
        for (int m = 0; m < MI; ++m) pa[m] = s_pa[buf][ti + TI * m];
#pragma unroll
        for (int n = 0; n < MJ; ++n) pb[n] = s_pb[buf][tj + TJ * n];
        unsigned rowhit = 0;                 // bit m: row m of the micro-tile has a broad-phase candidate
#pragma unroll
        for (int m = 0; m < MI; ++m) {
            bool any = false;
#pragma unroll
            for (int n = 0; n < MJ; ++n)
                any |= fmaf(pa[m].x, pb[n].x, fmaf(pa[m].y, pb[n].y, -pb[n].z)) >= pa[m].z;
            rowhit |= any ? (1u << m) : 0u;
        }
        while (rowhit) {   // rare: only the flagged rows are re-derived (from shared memory)
            const int m = __ffs(rowhit) - 1;
            rowhit &= rowhit - 1;
            const int i = ti + TI * m;
            const float4 qa4 = s_pa[buf][i];
#pragma unroll 1
            for (int n = 0; n < MJ; ++n) {
                const unsigned long long bit = 1ull << (MJ * m + n);
                if (found & bit) continue;
                const float4 qb4 = s_pb[buf][tj + TJ * n];
                if (!(fmaf(qa4.x, qb4.x, fmaf(qa4.y, qb4.y, -qb4.z)) >= qa4.z)) continue;
                const int j = tj + TJ * n;
                ++narrow;
                const float dx = qb4.x - qa4.x, dy = qb4.y - qa4.y;
                const float2 qa = s_ra[buf][i], qb = s_rb[buf][j];
                bool hit;
                switch (P.combo) {
                    case 0: hit = rect_rect(dx, dy, qa.x, qa.y, la, wa, qb.x, qb.y, lb, wb); break;
                    case 1: hit = rect_disc(dx, dy, qa.x, qa.y, la, wa, rb); break;
                    case 2: hit = rect_disc(-dx, -dy, qb.x, qb.y, lb, wb, ra); break;
                    default: hit = fmaf(dx, dx, dy * dy) <= (ra + rb) * (ra + rb); break;
                }
                if (hit) {
                    found |= bit;
                    a.table[P.off + (long long)(i0 + i) * B.h + j0 + j] = (int16_t)k;
                }
            }
        }
        buf ^= 1;
        k = k_next;
    }
    if (a.counters) {
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) narrow += __shfl_xor_sync(0xffffffffu, narrow, d);
        if ((tid & 31) == 0 && narrow) atomicAdd(a.counters + 1, narrow);
        if (tid == 0 && active_steps) atomicAdd(a.counters, (unsigned long long)active_steps * kTile * kTile);
    }
}

// table[0, n) = -1 (no collision), 16-byte stores on the aligned body
__global__ void __launch_bounds__(256) fill_kernel(int16_t *table, long long n) {
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

cudaError_t launch_fill_table(int16_t *table, long long n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    long long blocks = (n / 8 + 255) / 256 + 1;
    if (blocks > 152 * 16) blocks = 152 * 16;
    fill_kernel<<<(unsigned)blocks, 256, 0, st>>>(table, n);
    return cudaGetLastError();
}

cudaError_t launch_collide(const CollideArgs &a, cudaStream_t st) {
    if (a.n_tiles <= 0) return cudaSuccess;
    if (a.n_tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    int n_sm = 152, dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (a.n_tiles >= 32LL * n_sm)   // many tiles: throughput, fewest loads per test
        collide_kernel<64, 8, 8><<<(unsigned)a.n_tiles, 64, 0, st>>>(a);
    else                            // few tiles: latency, 8 warps share each tile's tests
        collide_kernel<256, 4, 4><<<(unsigned)a.n_tiles, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace mhc
