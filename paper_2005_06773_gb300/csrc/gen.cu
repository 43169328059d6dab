// gen.cu -- trajectory generation (Section IV-B): one thread per hypothesis, sub-steps in order.
//
// Vehicles: one-track model (Eq. onetrack) with constant steering and acceleration, integrated by
// Eq. (EulerVelocity) with sub-step tau / K; the low-speed kinematic limit and the stop rule are applied
// on the sub-steps where the FP64 speed v_0 + n vdot tau_i crosses 2 m/s / zero (the same FP64 decision
// the method's reference arithmetic takes).  Arithmetic is FP32; x, y and psi are carried as
// compensated (hi, lo) sums so that 250+ sub-steps add no more than ~1e-6 m of rounding.
// Pedestrians: Eq. (pedestrianmotion) with a constant acceleration integrates exactly, so every output
// pose is evaluated in closed form (speed saturating at 0 or at the cap).
#include "mhc_internal.cuh"

namespace mhc {
namespace {

// Error-free sum (Knuth's two-sum): s + e == a + b exactly.
__device__ __forceinline__ float two_sum(float a, float b, float &e) {
    const float s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
    return s;
}

// (hi, lo) += d, renormalised so that |lo| <= ulp(hi) / 2; hi + lo carries the running sum.
__device__ __forceinline__ void acc2(float &hi, float &lo, float d) {
    float e;
    const float s = two_sum(hi, d, e);
    const float t = __fadd_rn(lo, e);
    hi = __fadd_rn(s, t);
    lo = __fsub_rn(t, __fsub_rn(hi, s));
}

// sin / cos of the angle (a_hi + a_lo) to first order in the small part a_lo.
__device__ __forceinline__ void sincos2(float a_hi, float a_lo, float &sn, float &cs) {
    float s0, c0;
    sincosf(a_hi, &s0, &c0);
    cs = fmaf(-s0, a_lo, c0);
    sn = fmaf(c0, a_lo, s0);
}

__device__ __forceinline__ double speed_at(double v0, double dv, long long n) {
    return __dadd_rn(v0, __dmul_rn((double)n, dv));
}

// Smallest n in [lo, hi] for which pred(n) holds, pred monotone false..true; hi if none below it.
template <class P>
__device__ long long first_true(long long lo, long long hi, P pred) {
    while (lo < hi) {
        long long mid = lo + ((hi - lo) >> 1);
        if (pred(mid)) hi = mid; else lo = mid + 1;
    }
    return lo;
}

__device__ void vehicle(const ObjDesc &o, float acc, float delta, int model, int N, int K, float tau,
                        double tau_d, long long base, int h, int i, float *X, float *Y, float *C, float *S) {
    const double tau_i_d = __ddiv_rn(tau_d, (double)K);
    const double dv_d = __dmul_rn((double)acc, tau_i_d);
    const double v0_d = (double)o.v0;
    const long long NK = (long long)N * K;
    // low-speed regime: sub-steps with v_n < kVMin (prefix if accelerating, suffix if braking)
    long long low_lo = 0, low_hi = 0;   // low regime on [low_lo, low_hi)
    if (model == kModelKin) {
        low_lo = 0; low_hi = NK;
    } else if (acc > 0.0f) {
        low_hi = first_true(0, NK, [&](long long n) { return speed_at(v0_d, dv_d, n) >= kVMinD; });
    } else if (acc < 0.0f) {
        low_lo = first_true(0, NK, [&](long long n) { return speed_at(v0_d, dv_d, n) < kVMinD; });
        low_hi = NK;
    } else if (v0_d < kVMinD) {
        low_hi = NK;
    }
    long long n_stop = NK;   // sub-step at which v_{n+1} < 0 first holds
    if (acc < 0.0f) n_stop = first_true(0, NK, [&](long long n) { return speed_at(v0_d, dv_d, n + 1) < 0.0; });

    const float ti = (float)tau_i_d;
    const float hti2 = 0.5f * ti * ti;
    const float dv = acc * ti;
    const float L = o.lf + o.lr;
    const float inv_m = 1.0f / o.m, inv_iz = 1.0f / o.Iz;
    const float k11 = -(o.caf + o.car) * inv_m;                 // a11 * v
    const float k12 = (o.car * o.lr - o.caf * o.lf) * inv_m;    // (a12 + 1) * v^2
    const float k21 = (o.car * o.lr - o.caf * o.lf) * inv_iz;   // a21
    const float k22 = -(o.caf * o.lf * o.lf + o.car * o.lr * o.lr) * inv_iz;  // a22 * v
    const float kb1 = o.caf * inv_m;                            // b1 * v
    const float kb2 = o.caf * o.lf * inv_iz;                    // b2
    const float tdel = tanf(delta);
    const float beta_kin = atanf(o.lr * tdel / L);
    const float kappa = cosf(beta_kin) * tdel / L;              // r = v * kappa in the kinematic limit

    float xh = o.x0, xl = 0.0f, yh = o.y0, yl = 0.0f, ph = o.psi0, pl = 0.0f;
    float beta = 0.0f, r = 0.0f, ax = acc, ay = 0.0f;
    bool stopped = false;
    long long n = 0;
    for (int k = 0; k < N; ++k) {
        for (int q = 0; q < K; ++q, ++n) {
            if (stopped) continue;
            const float v = fmaf((float)n, dv, o.v0);
            float bd, rd;
            if (n >= low_lo && n < low_hi) {
                beta = beta_kin;
                r = v * kappa;
                bd = 0.0f;
                rd = 0.0f;
            } else {
                const float iv = 1.0f / v;
                bd = k11 * iv * beta + (k12 * iv * iv - 1.0f) * r + kb1 * iv * delta;
                rd = k21 * beta + k22 * iv * r + kb2 * delta;
            }
            float spb, cpb, e_pb;
            const float pb = two_sum(ph, beta, e_pb);             // course angle psi + beta, split exactly
            sincos2(pb, __fadd_rn(e_pb, pl), spb, cpb);
            if (n == n_stop) {
                const float d = v * v / (2.0f * fabsf(acc));
                acc2(xh, xl, cpb * d);
                acc2(yh, yl, spb * d);
                stopped = true;
                continue;
            }
            float spc, cpc;
            sincos2(ph, pl, spc, cpc);
            const float dx = cpb * v * ti + (cpc * ax - spc * ay) * hti2;
            const float dy = spb * v * ti + (spc * ax + cpc * ay) * hti2;
            float sb, cb;
            sincosf(beta, &sb, &cb);
            const float w = v * (bd + r);
            const float ax_n = cb * acc - sb * w;
            const float ay_n = sb * acc + cb * w;
            const float dpsi = r * ti + rd * hti2;
            beta = fmaf(bd, ti, beta);
            r = fmaf(rd, ti, r);
            ax = ax_n;
            ay = ay_n;
            acc2(xh, xl, dx);
            acc2(yh, yl, dy);
            acc2(ph, pl, dpsi);
        }
        float sp, cp;
        sincos2(ph, pl, sp, cp);
        const long long idx = base + (long long)k * h + i;
        X[idx] = xh + xl;
        Y[idx] = yh + yl;
        C[idx] = cp;
        S[idx] = sp;
    }
}

__device__ void pedestrian(const ObjDesc &o, float ga, float gb, int N, float tau, long long base, int h, int i,
                           float *X, float *Y, float *C, float *S) {
    const bool accel = (o.flags & kPedAccelGrid) != 0;
    const float v0 = accel ? o.v0 : ga;
    const float a = accel ? ga : 0.0f;
    const float th = o.psi0 + gb;
    float st, ct;
    sincosf(th, &st, &ct);
    // saturation time of the speed (cap when accelerating, zero when braking)
    float ts = INFINITY, s_sat = 0.0f, v_sat = v0;
    if (a > 0.0f && o.v_max > 0.0f) {
        if (v0 >= o.v_max) { ts = 0.0f; s_sat = 0.0f; v_sat = v0; }
        else { ts = (o.v_max - v0) / a; s_sat = v0 * ts + 0.5f * a * ts * ts; v_sat = o.v_max; }
    } else if (a < 0.0f) {
        ts = v0 / -a; s_sat = v0 * v0 / (-2.0f * a); v_sat = 0.0f;
    }
    for (int k = 0; k < N; ++k) {
        const float t = (float)(k + 1) * tau;
        const float s = t < ts ? fmaf(0.5f * a * t, t, v0 * t) : fmaf(v_sat, t - ts, s_sat);
        const long long idx = base + (long long)k * h + i;
        X[idx] = fmaf(ct, s, o.x0);
        Y[idx] = fmaf(st, s, o.y0);
        C[idx] = ct;
        S[idx] = st;
    }
}

__global__ void __launch_bounds__(128) gen_kernel(const GenArgs a) {
    const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w >= a.n_warps) return;
    const ObjDesc &o = a.objs[a.warp_obj[w]];
    const int i = a.warp_first[w] + (threadIdx.x & 31);
    if (i >= o.h) return;
    const int ia = i / o.n_b, ib = i - ia * o.n_b;
    const float ga = a.grids[o.grid_off + ia];
    const float gb = a.grids[o.grid_off + o.n_a + ib];
    if (o.kind == kVehicle)
        vehicle(o, ga, gb, a.model, a.n_steps, a.substeps, a.tau, a.tau_d, o.pose_base, o.h, i, a.x, a.y, a.c, a.s);
    else
        pedestrian(o, ga, gb, a.n_steps, a.tau, o.pose_base, o.h, i, a.x, a.y, a.c, a.s);
}

// Bounding box of the 32 pose centres of each bound tile at each step (warp min/max reduction).
__global__ void __launch_bounds__(256) bounds_kernel(const BoundsArgs a) {
    const long long g = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const long long total = (long long)a.n_warps * a.n_steps;
    if (g >= total) return;
    const int w = (int)(g / a.n_steps), k = (int)(g - (long long)w * a.n_steps);
    const ObjDesc &o = a.objs[a.warp_obj[w]];
    const int lane = threadIdx.x & 31;
    const int i = a.warp_first[w] + lane;
    float x0 = INFINITY, y0 = INFINITY, x1 = -INFINITY, y1 = -INFINITY;
    if (i < o.h) {
        const long long idx = o.pose_base + (long long)k * o.h + i;
        x0 = x1 = a.x[idx];
        y0 = y1 = a.y[idx];
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        x0 = fminf(x0, __shfl_xor_sync(0xffffffffu, x0, d));
        y0 = fminf(y0, __shfl_xor_sync(0xffffffffu, y0, d));
        x1 = fmaxf(x1, __shfl_xor_sync(0xffffffffu, x1, d));
        y1 = fmaxf(y1, __shfl_xor_sync(0xffffffffu, y1, d));
    }
    if (lane == 0) a.bounds[(long long)(o.tile_base + a.warp_first[w] / kBoundTile) * a.n_steps + k] =
        make_float4(x0, y0, x1, y1);
}

}  // namespace

cudaError_t launch_generate(const GenArgs &a, cudaStream_t st) {
    if (a.n_warps <= 0) return cudaSuccess;
    // few hypotheses: one warp per block so that the latency-bound integration spreads over all SMs
    const int warps_per_block = a.n_warps < 4 * 152 ? 1 : 4;
    const int blocks = (a.n_warps + warps_per_block - 1) / warps_per_block;
    gen_kernel<<<blocks, 32 * warps_per_block, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_bounds(const BoundsArgs &a, cudaStream_t st) {
    const long long total = (long long)a.n_warps * a.n_steps;
    if (total <= 0) return cudaSuccess;
    const long long blocks = (total + 7) / 8;
    bounds_kernel<<<(unsigned)blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace mhc
