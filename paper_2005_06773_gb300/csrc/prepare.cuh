// prepare.cuh -- the first step of a risk assessment (Section IV-D.1): zero the accumulators, fill the
// escape lists with -1, L1-normalise each object's weights into probabilities and convert each hypothesis's
// probability p and -log(1 - p) to the fixed point of the risk sums once.  risk.cu launches it on
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
    p.pfix = r.pfix;
    p.lfix = r.lfix;
    p.score = r.score;
    p.grids = r.grids;
    p.paths = r.paths;
    return p;
}

// Eq. (normTraj), n_h = (w_acc n_acc + w_str d_str) / (c_com c_cou), for hypothesis i of object o, with the
// library's default factors (the paper fixes neither): w_acc = w_str = 1/2; vehicles n_acc = 1 / (1 +
// |vdot| / 2 m/s^2); constant steering d_str = 1 / (1 + |delta| / 0.05 rad); paths, from the lateral
// offsets o_s of their section points from the vehicle's initial line: d_str = 1 / (1 + max |o_s| /
// 1.75 m), c_com = 1 + (|o_1 - o_0| + |o_2 - o_1|) / 3.5 m, c_cou = 2 when a section lies more than
// 1.75 m to the left (the counter-traffic lane); pedestrians n_acc = 1 / (1 + |v - v0| / 1 m/s) (speed
// grids) or 1 / (1 + |vdot| / 2 m/s^2) (acceleration grids), d_str = 1 / (1 + |heading offset| / 0.5 rad).
static __device__ __noinline__ double hypothesis_score(const PrepArgs &a, const ObjDesc &o, int i) {
    const int ia = i / o.n_b, ib = i - ia * o.n_b;
    const double ga = a.grids[o.grid_off + ia], gb = a.grids[o.grid_off + o.n_a + ib];
    double n_acc, d_str, c_com = 1.0, c_cou = 1.0;
    if (o.kind == kVehicle) {
        n_acc = 1.0 / (1.0 + fabs(ga) / 2.0);
        if (o.path_off < 0) {
            d_str = 1.0 / (1.0 + fabs(gb) / 0.05);
        } else {
            const float *pth = a.paths + 9LL * (o.path_off + ib);
            const double nx = -sin((double)o.psi0), ny = cos((double)o.psi0);
            double off[3], o_abs = 0.0, o_max = -1e300;
            for (int k = 0; k < 3; ++k) {
                off[k] = ((double)pth[3 * k] - o.x0) * nx + ((double)pth[3 * k + 1] - o.y0) * ny;
                o_abs = fmax(o_abs, fabs(off[k]));
                o_max = fmax(o_max, off[k]);
            }
            d_str = 1.0 / (1.0 + o_abs / 1.75);
            c_com = 1.0 + (fabs(off[1] - off[0]) + fabs(off[2] - off[1])) / 3.5;
            c_cou = o_max > 1.75 ? 2.0 : 1.0;
        }
    } else {
        n_acc = (o.flags & kPedAccelGrid) ? 1.0 / (1.0 + fabs(ga) / 2.0) : 1.0 / (1.0 + fabs(ga - o.v0) / 1.0);
        d_str = 1.0 / (1.0 + fabs(gb) / 0.5);
    }
    return (0.5 * n_acc + 0.5 * d_str) / (c_com * c_cou);
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
    if (a.weights || a.score) {   // raw weights (or scores, kept in prob until normalised) and their sum
        for (int i = threadIdx.x; i < o.h; i += blockDim.x) {
            const double wv = a.weights ? (double)a.weights[o.traj_off + i] : hypothesis_score(a, o, i);
            if (!a.weights) a.prob[o.traj_off + i] = wv;
            sum += wv;
        }
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
        const double p = (a.weights ? (double)a.weights[o.traj_off + i] : (a.score ? a.prob[o.traj_off + i] : 1.0)) / sum;
        a.prob[o.traj_off + i] = p;
        a.probf[o.traj_off + i] = (float)p;
        if (a.pfix) {   // the per-hypothesis terms of every first hit, converted once
            a.pfix[o.traj_off + i] = to_fixed((float)p, kFixProb);
            a.lfix[o.traj_off + i] = to_fixed(neg_log_survival((float)p), kFixLog);
        }
    }
}

}  // namespace mhc
