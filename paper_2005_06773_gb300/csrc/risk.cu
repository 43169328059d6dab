// risk.cu -- risk assessment (Section IV-D) from the first-collision table.
//
//   prepare  zero the accumulators; L1-normalise each object's weights into probabilities (Section IV-D.1)
//   scan     one CTA per 64 x 64 table tile (the collision tiling): counts, first-step histograms and
//            probability masses per object pair (Eq. totalCrashProb per pair); for pairs containing the
//            EGO object also per-EGO-hypothesis hit counts, per-(hypothesis, CO object) masses and, per
//            (hypothesis, step, CO object) cell, the sum of -log(1 - p) over the cell's entries
//   ego      one warp per EGO hypothesis walks the cells in ascending (step, object) order: a cell with
//            survival factor 1 - q = exp(-sum) contributes S q and leaves S (1 - q), S being the survival
//            product of the earlier cells -- exactly the entry-by-entry scaling of Eq. p21 summed over
//            the cell (telescoping); plus the per-object independence measure and the scalar totals
//            and the escape-route ranks (Section VI-A); its last CTA converts the totals
//
// Collisions are rare and scattered inside a warp, so the per-hit work uses only FP32 and integer
// instructions: each term (p_a p_b, p, -log(1 - p)) is formed in FP32 and added exactly as unsigned
// 64-bit fixed point by integer atomics (exact, order-independent, bitwise reproducible).  FP64 -- a
// narrow pipe on this GPU -- runs only in dense per-warp steps.
#include "mhc_internal.cuh"
#include "prepare.cuh"

namespace mhc {
namespace {

constexpr int kMaxSmemSteps = 1024;
constexpr int kMaxSmemCells = 256;           // 64 x 256 cells x 8 B = 128 KiB of dynamic shared memory
// value of a fixed-point sum with `frac` fractional bits (the scale is an exact power of two)
__device__ __forceinline__ double from_fixed(unsigned long long v, int frac) {
    return __ull2double_rn(v) * (1.0 / (double)(1ull << frac));
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    return v;
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    return v;
}

// blocks [0, n_obj) normalise one object each; every block zeroes a slice of the accumulators
__global__ void __launch_bounds__(256) prepare_kernel(const PrepArgs a) {
    pdl_start();
    prepare_block(a, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(64) scan_kernel(const RiskArgs a) {
    pdl_start();
    // dynamic: [N] u64 masses | [N] u32 counts | [64][N] u64 log-survival cells of the tile's EGO hypotheses
    extern __shared__ unsigned long long s_dyn64[];
    __shared__ unsigned long long s_row_mass[kTile];
    __shared__ unsigned s_row_hits[kTile];
    const long long g = blockIdx.x;
    if (g >= a.n_tiles) return;
    int lo = 0, hi = a.n_pairs - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (a.pairs[mid].tile_start <= g) lo = mid; else hi = mid - 1;
    }
    const int p = lo;
    const PairDesc P = a.pairs[p];
    const ObjDesc &A = a.objs[P.a];
    const ObjDesc &B = a.objs[P.b];
    const long long t = g - P.tile_start;
    const int ta = (int)(t / P.tiles_b), tb = (int)(t - (long long)ta * P.tiles_b);
    const int i0 = ta * kTile, j0 = tb * kTile;
    const int rows = min(kTile, A.h - i0), cols = min(kTile, B.h - j0);
    const int tid = threadIdx.x;
    const int N = P.n_steps;
    const bool smem_hist = a.max_steps <= kMaxSmemSteps;
    unsigned long long *s_H = s_dyn64;
    unsigned *s_cnt = reinterpret_cast<unsigned *>(s_dyn64 + N);
    unsigned long long *s_L = s_dyn64 + N + (N + 1) / 2;
    const bool smem_cells = smem_hist && a.max_steps <= kMaxSmemCells && P.ego_side >= 0;
    if (smem_hist)
        for (int k = tid; k < N; k += 64) { s_cnt[k] = 0u; s_H[k] = 0ull; }
    if (smem_cells)
        for (int q = tid; q < kTile * N; q += 64) s_L[q] = 0ull;
    s_row_mass[tid] = 0ull;
    s_row_hits[tid] = 0u;
    __syncthreads();

    const int j = tid;
    const bool col_ok = j < cols;
    const float pb = col_ok ? a.probf[B.traj_off + j0 + j] : 0.0f;
    unsigned long long cnt = 0, pm = 0, col_mass = 0;
    unsigned col_hits = 0;
    if (col_ok) {
        const int16_t *row = a.table + P.off + (long long)i0 * B.h + j0 + j;
        const unsigned long long pb_fix = to_fixed(pb, kFixProb);
        for (int ib = 0; ib < rows; ib += 16) {
            int16_t v[16];   // 16 independent loads in flight, then the (rare) hits
#pragma unroll
            for (int q = 0; q < 16; ++q) v[q] = ib + q < rows ? __ldg(row + (long long)(ib + q) * B.h) : (int16_t)-1;
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int T = v[q];
                if (T < 0 || T >= N) continue;   // -1: no collision; >= N cannot come from the collision kernel
                const int i = ib + q;
                const float pa = a.probf[A.traj_off + i0 + i];
                const unsigned long long w = to_fixed(pa * pb, kFixProb);
                ++cnt;
                pm += w;
                if (smem_hist) {
                    atomicAdd(s_cnt + T, 1u);
                    atomicAdd(s_H + T, w);
                } else {
                    atomicAdd(a.acc.count_k + P.kofs + T, 1ull);
                    atomicAdd(a.acc.H + P.kofs + T, w);
                }
                if (P.ego_side == 0) {          // row hypothesis belongs to the EGO object, CO = b
                    atomicAdd(s_row_mass + i, pb_fix);
                    atomicAdd(s_row_hits + i, 1u);
                    const unsigned long long lq = to_fixed(neg_log_survival(pb), kFixLog);
                    if (smem_cells) atomicAdd(s_L + i * N + T, lq);
                    else atomicAdd(a.acc.lsum + P.lsum_base + ((long long)(i0 + i) * N + T) * P.n_obj_s + P.co_local, lq);
                } else if (P.ego_side == 1) {   // column hypothesis belongs to the EGO object, CO = a
                    col_mass += to_fixed(pa, kFixProb);
                    ++col_hits;
                    const unsigned long long lq = to_fixed(neg_log_survival(pa), kFixLog);
                    if (smem_cells) s_L[j * N + T] += lq;   // only this thread owns column j's cells
                    else atomicAdd(a.acc.lsum + P.lsum_base + ((long long)(j0 + j) * N + T) * P.n_obj_s + P.co_local, lq);
                }
            }
        }
    }
    if (P.ego_side == 1 && col_hits) {
        atomicAdd(a.acc.mass + P.mass_base + (long long)(j0 + j) * P.n_obj_s + P.co_local, col_mass);
        atomicAdd(a.acc.hits + P.hits_base + j0 + j, (unsigned long long)col_hits);
    }
    cnt = warp_sum(cnt);
    pm = warp_sum(pm);
    if ((tid & 31) == 0 && cnt) {
        atomicAdd(a.acc.count + p, cnt);
        atomicAdd(a.acc.P + p, pm);
    }
    __syncthreads();
    if (smem_hist) {
        for (int k = tid; k < N; k += 64) {
            if (s_cnt[k]) {
                atomicAdd(a.acc.count_k + P.kofs + k, (unsigned long long)s_cnt[k]);
                atomicAdd(a.acc.H + P.kofs + k, s_H[k]);
            }
        }
    }
    if (smem_cells) {
        const int e0 = P.ego_side == 0 ? i0 : j0;
        for (int q = tid; q < kTile * N; q += 64) {
            const unsigned long long v = s_L[q];
            if (v) {
                const int e = q / N, k = q - e * N;
                atomicAdd(a.acc.lsum + P.lsum_base + ((long long)(e0 + e) * N + k) * P.n_obj_s + P.co_local, v);
            }
        }
    }
    if (P.ego_side == 0 && tid < rows && s_row_hits[tid]) {
        atomicAdd(a.acc.mass + P.mass_base + (long long)(i0 + tid) * P.n_obj_s + P.co_local, s_row_mass[tid]);
        atomicAdd(a.acc.hits + P.hits_base + i0 + tid, (unsigned long long)s_row_hits[tid]);
    }
}

// The caller's outputs from the accumulators (fixed point -> double), in two parts: the pair totals
// (count, P, count_k, H), final once the collision / scan launch has finished, and the totals the EGO walk
// itself accumulates (attr_obj, attr_step, scalars, n_escape).  Threads t of nt; each pass loads four
// elements before storing any, so the loads overlap.
__device__ void convert_pair_totals(const RiskArgs &a, long long t, long long nt) {
    const long long n = a.n_kofs + a.n_pairs;
    for (long long q0 = t; q0 < n; q0 += 4 * nt) {
        unsigned long long c[4], h[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const long long q = q0 + u * nt;
            c[u] = h[u] = 0ull;
            if (q < a.n_kofs) { c[u] = a.acc.count_k[q]; h[u] = a.acc.H[q]; }
            else if (q < n) { c[u] = a.acc.count[q - a.n_kofs]; h[u] = a.acc.P[q - a.n_kofs]; }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const long long q = q0 + u * nt;
            if (q < a.n_kofs) {
                if (a.count_k) a.count_k[q] = (long long)c[u];
                if (a.H) a.H[q] = from_fixed(h[u], kFixProb);
            } else if (q < n) {
                if (a.count) a.count[q - a.n_kofs] = (long long)c[u];
                if (a.P) a.P[q - a.n_kofs] = from_fixed(h[u], kFixProb);
            }
        }
    }
}

__device__ void convert_walk_totals(const RiskArgs &a, long long t, long long nt) {
    for (long long q = t; q < a.n_obj; q += nt)
        if (a.attr_obj) a.attr_obj[q] = from_fixed(a.acc.attr_obj[q], kFixProb);
    for (long long q = t; q < a.n_steps_total; q += nt)
        if (a.attr_step) a.attr_step[q] = from_fixed(a.acc.attr_step[q], kFixProb);
    for (long long q = t; q < 4LL * a.n_scen; q += nt)
        if (a.scalars) a.scalars[q] = (q & 3) < 3 ? a.acc.scalars[q] : 0.0;
    for (long long q = t; q < a.n_scen; q += nt)
        if (a.n_escape) a.n_escape[q] = (int)a.acc.n_escape[q];
}

// One warp per EGO hypothesis of the batch (its scenario found by binary search).
//  * collision-free hypothesis: its escape-route rank (Section VI-A) = the number of collision-free
//    hypotheses of its scenario more probable than it, ties by index, counted 32 at a time with ballots on
//    integer keys (probabilities are non-negative, so their bit patterns order like the values);
//  * otherwise the chronological walk: the (step, object) cells are read in ascending order 32 at a time,
//    384 per group with the twelve loads in flight together; a warp prefix sum of the cells' fixed-point
//    log-survival sums L (exact 64-bit integers) gives each cell the survival S = exp(-sum of the earlier
//    cells' L), and the cell contributes S q with q = 1 - exp(-L) (Eq. p21 over the cell's collisions:
//    the product of their survival factors is exp(-L)).  Every term is formed in FP32 (relative error
//    below 5e-7) and the terms are summed in FP64.
// Every CTA first converts a slice of the pair totals; the last CTA to finish converts the walk's own
// totals (or a separate grid-wide kernel does, for large batches).
constexpr float kLogScale = 1.0f / 1099511627776.0f;   // 2^-40: the fixed point of the log-survival sums

// exp(-x 2^-40) for a fixed-point log-survival sum x: x = hi + lo with hi the nearest FP32 value (exact
// as an integer) and lo the small remainder, so the FP32 rounding of x does not reach the exponent.
__device__ __forceinline__ float survival(unsigned long long x) {
    const float hi = __ull2float_rn(x);
    const long long lo = (long long)(x - __float2ull_rz(hi));
    return expf(-hi * kLogScale) * (1.0f - (float)lo * kLogScale);
}

constexpr int kEscapeBatch = 8;    // escape ranking: 256 EGO hypotheses' keys in flight per round
constexpr int kWalkBatch = 12;     // chronological walk: 384 cells in flight per round

__global__ void __launch_bounds__(64) ego_kernel(const RiskArgs a) {
    pdl_trigger();
    __shared__ bool s_last;
    const int lane = threadIdx.x & 31;
    const long long g = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    // the scenario of EGO hypothesis g and its descriptor: uploaded data, read before the wait
    int lo = 0;
    ScenDesc sd{};
    if (g < a.h_e) {
        int hi = a.n_scen - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.scens[mid].e_base <= g) lo = mid; else hi = mid - 1;
        }
        sd = a.scens[lo];
    }
    pdl_wait();
    convert_pair_totals(a, (long long)blockIdx.x * blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x);
    if (g < a.h_e) {
        const int N = sd.n_steps, n_obj = sd.n_obj;
        const long long i = g - sd.e_base;
        const double pe = a.prob[sd.e_traj + i];
        const float pef = a.probf[sd.e_traj + i];
        const unsigned long long hits = a.acc.hits[g];
        double naive = 0.0, cond = 0.0, indep = 0.0;
        if (!hits) {
            if (a.escape) {
                const long long key = __double_as_longlong(pe);
                int rank = 0;
                for (int q0 = 0; q0 < sd.h_e; q0 += 32 * kEscapeBatch) {   // every load of a batch issued first
                    unsigned long long hq[kEscapeBatch];
                    long long kq[kEscapeBatch];
#pragma unroll
                    for (int u = 0; u < kEscapeBatch; ++u) {
                        const int q = q0 + 32 * u + lane;
                        hq[u] = q < sd.h_e ? a.acc.hits[sd.e_base + q] : 1ull;
                        kq[u] = q < sd.h_e ? __double_as_longlong(a.prob[sd.e_traj + q]) : 0ll;
                    }
#pragma unroll
                    for (int u = 0; u < kEscapeBatch; ++u) {
                        const int q = q0 + 32 * u + lane;
                        const bool above = hq[u] == 0ull && (kq[u] > key || (kq[u] == key && q < i));
                        rank += __popc(__ballot_sync(0xffffffffu, above));
                    }
                }
                if (lane == 0) a.escape[sd.e_base + rank] = (int)i;
            }
            if (lane == 0) atomicAdd(a.acc.n_escape + lo, 1ull);
        } else {
            // per-object masses: naive sum and independence product
            double surv = 1.0, mass_sum = 0.0;
            const unsigned long long *ms = a.acc.mass + sd.mass_base + i * n_obj;
            for (int b = lane; b < n_obj; b += 32) {
                const double m = from_fixed(ms[b], kFixProb);
                mass_sum += m;
                surv *= 1.0 - m;
            }
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) surv *= __shfl_xor_sync(0xffffffffu, surv, d);
            naive = warp_sum(mass_sum);
            indep = 1.0 - surv;
            // chronological walk over the cells, kWalkBatch chunks of 32 loaded at once.  A cell holds
            // L = sum of -log(1 - p) of its collisions in fixed point, so the survival of every earlier cell
            // is exp(-(exact integer prefix sum of L)) and the cell's own collision probability is
            // 1 - exp(-L): the chunks' scans are 64-bit integer additions, independent of each other but
            // for the carried total
            const unsigned long long *lc = a.acc.lsum + sd.lsum_base + i * N * n_obj;
            const long long cells = (long long)N * n_obj;
            unsigned long long carry = 0;     // L summed over every cell before the chunk
            double part = 0.0;
            for (long long g0 = 0; g0 < cells; g0 += 32 * kWalkBatch) {
                unsigned long long lv[kWalkBatch];
#pragma unroll
                for (int u = 0; u < kWalkBatch; ++u) {
                    const long long c = g0 + 32 * u + lane;
                    lv[u] = c < cells ? lc[c] : 0ull;
                }
#pragma unroll
                for (int u = 0; u < kWalkBatch; ++u) {
                    const unsigned long long lf = lv[u];
                    unsigned long long incl = lf;
#pragma unroll
                    for (int d = 1; d < 32; d <<= 1) {
                        const unsigned long long v = __shfl_up_sync(0xffffffffu, incl, d);
                        if (lane >= d) incl += v;
                    }
                    const unsigned long long before = carry + (incl - lf);
                    carry += __shfl_sync(0xffffffffu, incl, 31);
                    if (!lf) continue;                                    // an empty cell adds nothing
                    const long long c = g0 + 32 * u + lane;
                    const float eff = survival(before) * -expm1f(-(float)lf * kLogScale);
                    part += (double)eff;
                    const int k = (int)(c / n_obj), b = (int)(c - (long long)k * n_obj);
                    const unsigned long long w = to_fixed(pef * eff, kFixProb);
                    atomicAdd(a.acc.attr_obj + sd.obj0 + b, w);
                    atomicAdd(a.acc.attr_step + sd.step_base + k, w);
                }
            }
            cond = warp_sum(part);
        }
        if (lane == 0) {
            if (a.naive) a.naive[g] = naive;
            if (a.cond) a.cond[g] = cond;
            if (a.indep) a.indep[g] = indep;
            if (a.hits) a.hits[g] = (int)hits;
            if (naive != 0.0) atomicAdd(a.acc.scalars + 4 * lo + 0, pe * naive);
            if (cond != 0.0) atomicAdd(a.acc.scalars + 4 * lo + 1, pe * cond);
            if (indep != 0.0) atomicAdd(a.acc.scalars + 4 * lo + 2, pe * indep);
        }
    }
    if (!a.convert_in_walk) return;
    // the last CTA converts the totals once every CTA's atomics are visible
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(a.acc.done, 1ull) == (unsigned long long)gridDim.x - 1;
    __syncthreads();
    if (s_last) {
        __threadfence();
        convert_walk_totals(a, threadIdx.x, blockDim.x);
    }
}

// The walk's totals of a large batch, grid-wide after the walk (and the pair totals too when there is no
// EGO hypothesis to walk, which a valid scenario never has).
__global__ void __launch_bounds__(256) totals_kernel(const RiskArgs a) {
    pdl_start();
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x, nt = (long long)gridDim.x * blockDim.x;
    if (a.h_e == 0) convert_pair_totals(a, t, nt);
    convert_walk_totals(a, t, nt);
}

// Up to this many walk totals the walk's last CTA (64 threads) converts them, saving a launch; beyond it a
// grid-wide kernel does.
constexpr long long kConvertInWalk = 512;

long long convert_elements(const RiskArgs &a) {
    return a.n_obj + a.n_steps_total + 5LL * a.n_scen + (a.h_e == 0 ? 2 * (a.n_kofs + a.n_pairs) : 0);
}

}  // namespace

cudaError_t launch_risk_prepare(const RiskArgs &a, cudaStream_t st) {
    const int prep_blocks = a.n_obj > 304 ? a.n_obj : 304;
    prepare_kernel<<<prep_blocks, 256, 0, st>>>(prep_of(a));
    return cudaGetLastError();
}

int risk_tail_launches(const RiskArgs &a) {
    return (a.h_e > 0 ? 1 : 0) + (a.h_e > 0 && convert_elements(a) <= kConvertInWalk ? 0 : 1);
}

cudaError_t launch_risk_tail(const RiskArgs &args, cudaStream_t st, bool pdl) {
    RiskArgs a = args;
    const long long conv = convert_elements(a);
    a.convert_in_walk = a.h_e > 0 && conv <= kConvertInWalk;
    if (a.h_e > 0) {
        cudaError_t e = launch_kernel(ego_kernel, dim3((unsigned)((a.h_e + 1) / 2)), dim3(64), 0, st, pdl, a);
        if (e != cudaSuccess) return e;
        pdl = true;
    }
    if (!a.convert_in_walk) {
        long long blocks = (conv + 255) / 256;
        if (blocks > 152 * 8) blocks = 152 * 8;
        return launch_kernel(totals_kernel, dim3((unsigned)blocks), dim3(256), 0, st, pdl, a);
    }
    return cudaSuccess;
}

cudaError_t launch_risk(const RiskArgs &a, cudaStream_t st, bool with_prepare, bool pdl) {
    cudaError_t e = with_prepare ? launch_risk_prepare(a, st) : cudaSuccess;
    if (e != cudaSuccess) return e;
    pdl = pdl || with_prepare;
    if (a.n_tiles > 0) {
        if (a.n_tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
        size_t smem = 0;
        if (a.max_steps <= kMaxSmemSteps) smem = 8 * ((size_t)a.max_steps + (a.max_steps + 1) / 2);
        if (a.max_steps <= kMaxSmemCells) smem += 8 * (size_t)kTile * a.max_steps;
        if (smem > 48 * 1024) {
            e = cudaFuncSetAttribute(scan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        e = launch_kernel(scan_kernel, dim3((unsigned)a.n_tiles), dim3(64), smem, st, pdl, a);
        if (e != cudaSuccess) return e;
        pdl = true;
    }
    return launch_risk_tail(a, st, pdl);
}

}  // namespace mhc
