// risk.cu -- risk assessment (Section IV-D) from the first-collision table.
//
//   prepare  zero the accumulators; L1-normalise each object's weights into probabilities (Section IV-D.1)
//   scan     one CTA per 64 x 64 table tile (the collision tiling): counts, first-step histograms and
//            probability masses per object pair (Eq. totalCrashProb per pair); for pairs containing the
//            EGO object also per-EGO-hypothesis naive mass, hit counts and, per (step, CO object), the sum
//            of log(1 - p) that the chronological scaling needs
//   ego      one thread per EGO hypothesis walks (step, object) cells in ascending order: a cell whose
//            entries have survival product Q = exp(sum log(1 - p)) contributes S (1 - Q) and leaves
//            S Q, which is exactly the entry-by-entry scaling of Eq. p21 summed over the cell
//            (telescoping); plus the per-object independence measure and the scalar totals
//   finish   escape routes ranked by probability (Section VI-A) and the copy of totals to the outputs
// Probabilities and masses accumulate in FP64 (only colliding entries touch them).
#include "mhc_internal.cuh"

namespace mhc {
namespace {

constexpr int kMaxSmemSteps = 1024;

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
__global__ void __launch_bounds__(256) prepare_kernel(const RiskArgs a) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < a.acc.n_words; w += stride)
        a.acc.base[w] = 0ull;
    if (blockIdx.x >= a.n_obj) return;
    const ObjDesc &o = a.objs[blockIdx.x];
    __shared__ double s_part[8];
    double sum = 0.0;
    if (a.weights) {
        for (int i = threadIdx.x; i < o.h; i += blockDim.x) sum += (double)a.weights[o.traj_off + i];
        sum = warp_sum(sum);
        if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = sum;
        __syncthreads();
        sum = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) sum += s_part[q];
    } else {
        sum = (double)o.h;
    }
    for (int i = threadIdx.x; i < o.h; i += blockDim.x)
        a.prob[o.traj_off + i] = (a.weights ? (double)a.weights[o.traj_off + i] : 1.0) / sum;
}

__global__ void __launch_bounds__(64) scan_kernel(const RiskArgs a) {
    extern __shared__ unsigned char s_dyn[];
    __shared__ double s_row_mass[kTile];
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
    const int N = a.n_steps;
    const bool smem_hist = N <= kMaxSmemSteps;
    unsigned *s_cnt = reinterpret_cast<unsigned *>(s_dyn);
    double *s_H = reinterpret_cast<double *>(s_dyn + sizeof(unsigned) * ((N + 1) & ~1));
    if (smem_hist)
        for (int k = tid; k < N; k += 64) { s_cnt[k] = 0u; s_H[k] = 0.0; }
    s_row_mass[tid] = 0.0;
    s_row_hits[tid] = 0u;
    __syncthreads();

    const int j = tid;
    const bool col_ok = j < cols;
    const double pb = col_ok ? a.prob[B.traj_off + j0 + j] : 0.0;
    const double lq_b = col_ok ? log1p(-pb) : 0.0;
    unsigned long long cnt = 0;
    double pm = 0.0, col_mass = 0.0;
    unsigned col_hits = 0;
    if (col_ok) {
        const int16_t *row = a.table + P.off + (long long)i0 * B.h + j0 + j;
        for (int i = 0; i < rows; ++i) {
            const int T = row[(long long)i * B.h];
            if (T < 0 || T >= N) continue;   // -1: no collision; values >= N cannot come from the collision kernel
            const double pa = a.prob[A.traj_off + i0 + i];
            const double w = pa * pb;
            ++cnt;
            pm += w;
            if (smem_hist) {
                atomicAdd(s_cnt + T, 1u);
                atomicAdd(s_H + T, w);
            } else {
                atomicAdd(a.acc.count_k + (long long)p * N + T, 1ull);
                atomicAdd(a.acc.H + (long long)p * N + T, w);
            }
            if (P.ego_side == 0) {          // row hypothesis belongs to the EGO object, CO = b
                atomicAdd(s_row_mass + i, pb);
                atomicAdd(s_row_hits + i, 1u);
                atomicAdd(a.acc.logq + ((long long)(i0 + i) * N + T) * a.n_obj + P.b, lq_b);
            } else if (P.ego_side == 1) {   // column hypothesis belongs to the EGO object, CO = a
                col_mass += pa;
                ++col_hits;
                atomicAdd(a.acc.logq + ((long long)(j0 + j) * N + T) * a.n_obj + P.a, log1p(-pa));
            }
        }
    }
    if (P.ego_side == 1 && col_hits) {
        atomicAdd(a.acc.naive + j0 + j, col_mass);
        atomicAdd(a.acc.mass + (long long)(j0 + j) * a.n_obj + P.a, col_mass);
        atomicAdd(a.acc.hits + j0 + j, (unsigned long long)col_hits);
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
                atomicAdd(a.acc.count_k + (long long)p * N + k, (unsigned long long)s_cnt[k]);
                atomicAdd(a.acc.H + (long long)p * N + k, s_H[k]);
            }
        }
    }
    if (P.ego_side == 0 && tid < rows && s_row_hits[tid]) {
        atomicAdd(a.acc.naive + i0 + tid, s_row_mass[tid]);
        atomicAdd(a.acc.mass + (long long)(i0 + tid) * a.n_obj + P.b, s_row_mass[tid]);
        atomicAdd(a.acc.hits + i0 + tid, (unsigned long long)s_row_hits[tid]);
    }
}

__global__ void __launch_bounds__(256) ego_kernel(const RiskArgs a) {
    extern __shared__ double s_attr[];   // [n_obj] then [N]
    __shared__ double s_tot[3][8];
    const int N = a.n_steps, n_obj = a.n_obj;
    const bool smem = (n_obj + N) <= 4096;
    if (smem) {
        for (int q = threadIdx.x; q < n_obj + N; q += blockDim.x) s_attr[q] = 0.0;
        __syncthreads();
    }
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double naive = 0.0, cond = 0.0, indep = 0.0, pe = 0.0;
    if (i < a.h_e) {
        const ObjDesc &E = a.objs[a.ego];
        pe = a.prob[E.traj_off + i];
        naive = a.acc.naive[i];
        const double *lq = a.acc.logq + (long long)i * N * n_obj;
        double ls = 0.0;     // log of the survival product of all earlier cells
        for (int k = 0; k < N; ++k) {
            for (int b = 0; b < n_obj; ++b) {
                const double L = lq[(long long)k * n_obj + b];
                if (L == 0.0) continue;
                const double eff = exp(ls) * -expm1(L);
                cond += eff;
                ls += L;
                if (smem) {
                    atomicAdd(s_attr + b, pe * eff);
                    atomicAdd(s_attr + n_obj + k, pe * eff);
                } else {
                    atomicAdd(a.acc.attr_obj + b, pe * eff);
                    atomicAdd(a.acc.attr_step + k, pe * eff);
                }
            }
        }
        double surv = 1.0;
        const double *ms = a.acc.mass + (long long)i * n_obj;
        for (int b = 0; b < n_obj; ++b) surv *= 1.0 - ms[b];
        indep = 1.0 - surv;
        if (a.naive) a.naive[i] = naive;
        if (a.cond) a.cond[i] = cond;
        if (a.indep) a.indep[i] = indep;
        if (a.hits) a.hits[i] = (int)a.acc.hits[i];
    }
    double v0 = warp_sum(pe * naive), v1 = warp_sum(pe * cond), v2 = warp_sum(pe * indep);
    if ((threadIdx.x & 31) == 0) {
        s_tot[0][threadIdx.x >> 5] = v0; s_tot[1][threadIdx.x >> 5] = v1; s_tot[2][threadIdx.x >> 5] = v2;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double s = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += s_tot[threadIdx.x][q];
        atomicAdd(a.acc.scalars + threadIdx.x, s);
    }
    if (smem) {
        for (int q = threadIdx.x; q < n_obj + N; q += blockDim.x) {
            const double v = s_attr[q];
            if (v != 0.0) atomicAdd(q < n_obj ? a.acc.attr_obj + q : a.acc.attr_step + (q - n_obj), v);
        }
    }
}

// single CTA: escape-route ranking and the copy of the totals to the caller's outputs
__global__ void __launch_bounds__(1024) finish_kernel(const RiskArgs a) {
    const int he = a.h_e;
    const ObjDesc &E = a.objs[a.ego];
    const double *pe = a.prob + E.traj_off;
    __shared__ int s_n;
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < he; i += blockDim.x) {
        if (a.acc.hits[i] != 0ull) continue;
        atomicAdd(&s_n, 1);
        if (!a.escape) continue;
        const double p = pe[i];
        int rank = 0;
        for (int q = 0; q < he; ++q)
            if (a.acc.hits[q] == 0ull && (pe[q] > p || (pe[q] == p && q < i))) ++rank;
        a.escape[rank] = i;
    }
    __syncthreads();
    if (threadIdx.x == 0 && a.n_escape) *a.n_escape = s_n;
    const long long npn = (long long)a.n_pairs * a.n_steps;
    for (long long q = threadIdx.x; q < npn; q += blockDim.x) {
        if (a.count_k) a.count_k[q] = (long long)a.acc.count_k[q];
        if (a.H) a.H[q] = a.acc.H[q];
    }
    for (int q = threadIdx.x; q < a.n_pairs; q += blockDim.x) {
        if (a.count) a.count[q] = (long long)a.acc.count[q];
        if (a.P) a.P[q] = a.acc.P[q];
    }
    for (int q = threadIdx.x; q < a.n_obj; q += blockDim.x)
        if (a.attr_obj) a.attr_obj[q] = a.acc.attr_obj[q];
    for (int q = threadIdx.x; q < a.n_steps; q += blockDim.x)
        if (a.attr_step) a.attr_step[q] = a.acc.attr_step[q];
    if (threadIdx.x < 4 && a.scalars) a.scalars[threadIdx.x] = threadIdx.x < 3 ? a.acc.scalars[threadIdx.x] : 0.0;
}

}  // namespace

cudaError_t launch_risk(const RiskArgs &a, cudaStream_t st) {
    const int prep_blocks = a.n_obj > 304 ? a.n_obj : 304;
    prepare_kernel<<<prep_blocks, 256, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (a.n_tiles > 0) {
        if (a.n_tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
        const size_t smem = a.n_steps <= kMaxSmemSteps
                                ? sizeof(unsigned) * ((a.n_steps + 1) & ~1) + sizeof(double) * a.n_steps : 0;
        scan_kernel<<<(unsigned)a.n_tiles, 64, smem, st>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (a.h_e > 0) {
        const size_t smem = (a.n_obj + a.n_steps) <= 4096 ? sizeof(double) * (a.n_obj + a.n_steps) : 0;
        ego_kernel<<<(a.h_e + 255) / 256, 256, smem, st>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    finish_kernel<<<1, 1024, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace mhc
