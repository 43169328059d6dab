// prepare.cuh -- the first step of a risk assessment (Section IV-D.1): zero the accumulators, fill the
// escape lists with -1 and L1-normalise each object's weights into probabilities.  risk.cu launches it on
// its own; on the fused path (generation, then collisions with the risk terms added at each first hit) it
// runs as extra CTAs of the generation launch, since the two are independent.
#pragma once
#include "mhc_internal.cuh"

namespace mhc {

inline PrepArgs prep_of(const RiskArgs &r) {
    PrepArgs p;
    p.base = r.acc.base;
    p.n_words = r.acc.n_words;
    p.escape = r.escape;
    p.h_e = r.h_e;
    p.objs = r.objs;
    p.n_obj = r.n_obj;
    p.weights = r.weights;
    p.prob = r.prob;
    p.probf = r.probf;
    return p;
}

// Block b of nb blocks (blockDim.x a multiple of 32, at most 1024; every thread of the block calls it):
// all blocks zero a slice of the accumulators; blocks [0, n_obj) normalise one object each.
__device__ __forceinline__ void prepare_block(const PrepArgs &a, int b, int nb) {
    __shared__ double s_part[32];
    const long long stride = (long long)nb * blockDim.x;
    for (long long w = (long long)b * blockDim.x + threadIdx.x; w < a.n_words; w += stride) a.base[w] = 0ull;
    if (a.escape)   // entries past each scenario's escape routes read -1
        for (long long w = (long long)b * blockDim.x + threadIdx.x; w < a.h_e; w += stride) a.escape[w] = -1;
    if (b >= a.n_obj) return;                      // the whole block leaves together
    const ObjDesc &o = a.objs[b];
    double sum = 0.0;
    if (a.weights) {
        for (int i = threadIdx.x; i < o.h; i += blockDim.x) sum += (double)a.weights[o.traj_off + i];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, d);
        if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = sum;
        __syncthreads();
        sum = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) sum += s_part[q];
    } else {
        sum = (double)o.h;
    }
    for (int i = threadIdx.x; i < o.h; i += blockDim.x) {
        const double p = (a.weights ? (double)a.weights[o.traj_off + i] : 1.0) / sum;
        a.prob[o.traj_off + i] = p;
        a.probf[o.traj_off + i] = (float)p;
    }
}

}  // namespace mhc
