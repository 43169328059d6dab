// collide.cu -- collision recognition (Section IV-C): first overlapping step of every hypothesis pair.
//
// Work decomposition: one 64-thread CTA per 64 x 64 tile of hypothesis pairs of one object pair.  The CTA
// walks the steps in order; per step it stages the 64 + 64 poses of its tile in shared memory (double
// buffered, one barrier per step) and every thread tests an 8 x 8 register micro-tile.
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

__global__ void __launch_bounds__(64) collide_kernel(const CollideArgs a) {
    __shared__ float4 s_pa[2][kTile];    // x, y, h_a
    __shared__ float4 s_pb[2][kTile];    // x, y, h_b
    __shared__ float2 s_ra[2][kTile];    // c, s
    __shared__ float2 s_rb[2][kTile];
    __shared__ int16_t s_res[kTile][kTile];
    __shared__ unsigned s_mask[2];

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
    const int tid = threadIdx.x, ti = tid >> 3, tj = tid & 7;
    const int N = a.n_steps;

    for (int e = tid; e < kTile * kTile; e += 64) (&s_res[0][0])[e] = kNoHit;

    const float la = A.hl, wa = A.hw, ra = A.rad, lb = B.hl, wb = B.hw, rb = B.rad;
    const float rc2 = P.rc2 + kEps0;     // (R_a + R_b)^2 plus the absolute slack
    unsigned long long narrow = 0;
    int it = 0, active_steps = 0;

    for (int k0 = 0; k0 < N; k0 += 32) {
        if (tid < 32) {
            const int k = k0 + tid;
            bool act = k < N;
            if (act && a.cull) {
                const int na = (rows + kBoundTile - 1) / kBoundTile, nb = (cols + kBoundTile - 1) / kBoundTile;
                float4 ba = a.bounds[(long long)(A.tile_base + ta * 2) * N + k];
                if (na > 1) {
                    const float4 q = a.bounds[(long long)(A.tile_base + ta * 2 + 1) * N + k];
                    ba = make_float4(fminf(ba.x, q.x), fminf(ba.y, q.y), fmaxf(ba.z, q.z), fmaxf(ba.w, q.w));
                }
                float4 bb = a.bounds[(long long)(B.tile_base + tb * 2) * N + k];
                if (nb > 1) {
                    const float4 q = a.bounds[(long long)(B.tile_base + tb * 2 + 1) * N + k];
                    bb = make_float4(fminf(bb.x, q.x), fminf(bb.y, q.y), fmaxf(bb.z, q.z), fmaxf(bb.w, q.w));
                }
                const float r = P.r_cull;
                act = (ba.x - r <= bb.z) && (bb.x - r <= ba.z) && (ba.y - r <= bb.w) && (bb.y - r <= ba.w);
            }
            const unsigned m = __ballot_sync(0xffffffffu, act);
            if (tid == 0) s_mask[(k0 >> 5) & 1] = m;
        }
        __syncthreads();
        unsigned mask = s_mask[(k0 >> 5) & 1];
        while (mask) {
            const int k = k0 + __ffs(mask) - 1;
            mask &= mask - 1;
            const int buf = it & 1;
            ++it;
            ++active_steps;
            {   // stage step k
                float x, y, c, s;
                if (tid < rows) {
                    const long long idx = A.pose_base + (long long)k * A.h + i0 + tid;
                    x = __ldg(a.x + idx); y = __ldg(a.y + idx); c = __ldg(a.c + idx); s = __ldg(a.s + idx);
                } else {
                    x = kFar; y = 0.0f; c = 1.0f; s = 0.0f;
                }
                s_pa[buf][tid] = make_float4(x, y, 0.5f * (1.0f - kEps) * fmaf(x, x, y * y), 0.0f);
                s_ra[buf][tid] = make_float2(c, s);
                if (tid < cols) {
                    const long long idx = B.pose_base + (long long)k * B.h + j0 + tid;
                    x = __ldg(a.x + idx); y = __ldg(a.y + idx); c = __ldg(a.c + idx); s = __ldg(a.s + idx);
                } else {
                    x = -kFar; y = 0.0f; c = 1.0f; s = 0.0f;
                }
                s_pb[buf][tid] = make_float4(x, y, 0.5f * fmaf(1.0f - kEps, fmaf(x, x, y * y), -rc2), 0.0f);
                s_rb[buf][tid] = make_float2(c, s);
            }
            __syncthreads();
            float4 pa[8], pb[8];
#pragma unroll
            for (int m = 0; m < 8; ++m) pa[m] = s_pa[buf][ti + 8 * m];
#pragma unroll
            for (int n = 0; n < 8; ++n) pb[n] = s_pb[buf][tj + 8 * n];
            bool any = false;
#pragma unroll
            for (int m = 0; m < 8; ++m)
#pragma unroll
                for (int n = 0; n < 8; ++n)
                    any |= fmaf(pa[m].x, pb[n].x, fmaf(pa[m].y, pb[n].y, -pb[n].z)) >= pa[m].z;
            if (any) {   // rare: re-derive the candidates from shared memory (no dynamic register indexing)
#pragma unroll 1
                for (int m = 0; m < 8; ++m) {
                    const float4 qa4 = s_pa[buf][ti + 8 * m];
#pragma unroll 1
                    for (int n = 0; n < 8; ++n) {
                        const float4 qb4 = s_pb[buf][tj + 8 * n];
                        if (!(fmaf(qa4.x, qb4.x, fmaf(qa4.y, qb4.y, -qb4.z)) >= qa4.z)) continue;
                        const int i = ti + 8 * m, j = tj + 8 * n;
                        if (s_res[i][j] != kNoHit) continue;
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
                        if (hit) s_res[i][j] = (int16_t)k;
                    }
                }
            }
        }
    }
    __syncthreads();
    for (int e = tid; e < kTile * kTile; e += 64) {
        const int i = e >> 6, j = e & (kTile - 1);
        if (i < rows && j < cols) {
            const int16_t v = s_res[i][j];
            a.table[P.off + (long long)(i0 + i) * B.h + j0 + j] = v == kNoHit ? (int16_t)-1 : v;
        }
    }
    if (a.counters) {
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) narrow += __shfl_xor_sync(0xffffffffu, narrow, d);
        if ((tid & 31) == 0 && narrow) atomicAdd(a.counters + 1, narrow);
        if (tid == 0 && active_steps) atomicAdd(a.counters, (unsigned long long)active_steps * kTile * kTile);
    }
}

}  // namespace

cudaError_t launch_collide(const CollideArgs &a, cudaStream_t st) {
    if (a.n_tiles <= 0) return cudaSuccess;
    if (a.n_tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    collide_kernel<<<(unsigned)a.n_tiles, 64, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace mhc
