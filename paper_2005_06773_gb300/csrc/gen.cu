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

// Kahan summation: (hi, c) carries the running sum hi - c; c is the compensation of the lost low part.
__device__ __forceinline__ void kahan_add(float &hi, float &c, float d) {
    const float y = __fsub_rn(d, c);
    const float t = __fadd_rn(hi, y);
    c = __fsub_rn(__fsub_rn(t, hi), y);
    hi = t;
}

// sin / cos of the angle (a_hi + a_lo) to first order in the small part a_lo.
__device__ __forceinline__ void sincos2(float a_hi, float a_lo, float &sn, float &cs) {
    float s0, c0;
    sincosf(a_hi, &s0, &c0);
    cs = fmaf(-s0, a_lo, c0);
    sn = fmaf(c0, a_lo, s0);
}

// sin / cos by the Taylor series to x^9 / x^10 (|x| <= 0.5: error < 2e-11), sincosf beyond.
__device__ __forceinline__ void sincos_half(float x, float &sn, float &cs) {
    if (fabsf(x) > 0.5f) {
        sincosf(x, &sn, &cs);
        return;
    }
    const float x2 = x * x;
    float ps = fmaf(x2, 1.0f / 362880.0f, -1.0f / 5040.0f);
    ps = fmaf(x2, ps, 1.0f / 120.0f);
    ps = fmaf(x2, ps, -1.0f / 6.0f);
    sn = fmaf(x * x2, ps, x);
    float pc = fmaf(x2, -1.0f / 3628800.0f, 1.0f / 40320.0f);
    pc = fmaf(x2, pc, -1.0f / 720.0f);
    pc = fmaf(x2, pc, 1.0f / 24.0f);
    pc = fmaf(x2, pc, -0.5f);
    cs = fmaf(x2, pc, 1.0f);
}

// sin / cos by the Taylor series to x^5 / x^6 (|x| <= 0.1: error < 3e-11), sincosf beyond.
__device__ __forceinline__ void sincos_tenth(float x, float &sn, float &cs) {
    if (fabsf(x) > 0.1f) {
        sincosf(x, &sn, &cs);
        return;
    }
    const float x2 = x * x;
    sn = fmaf(x * x2, fmaf(x2, 1.0f / 120.0f, -1.0f / 6.0f), x);
    cs = fmaf(x2, fmaf(x2, fmaf(x2, -1.0f / 720.0f, 1.0f / 24.0f), -0.5f), 1.0f);
}

__device__ __forceinline__ double speed_at(double v0, double dv, int n) {
    return __dadd_rn(v0, __dmul_rn((double)n, dv));
}

// Smallest n in [0, NK] with pred(n) (pred monotone false..true; NK if it never holds before NK), found
// from an FP32 estimate and settled by evaluating the FP64 predicate next to it.
template <class P>
__device__ int first_true(int NK, float estimate, P pred) {
    int n = estimate <= 0.0f ? 0 : (estimate >= (float)NK ? NK : (int)ceilf(estimate));
    while (n > 0 && pred(n - 1)) --n;
    while (n < NK && !pred(n)) ++n;
    return n;
}

__device__ void vehicle(const ObjDesc &o, float acc, float delta, int model, int N, int K, double tau_i_d,
                        long long base, int h, int i, float *X, float *Y, float *C, float *S) {
    const double dv_d = __dmul_rn((double)acc, tau_i_d);
    const double v0_d = (double)o.v0;
    const int NK = N * K;
    const float dvf = (float)dv_d;
    // low-speed regime: sub-steps with v_n < kVMin (a prefix when accelerating, a suffix when braking)
    int low_lo = 0, low_hi = 0;   // low regime on [low_lo, low_hi)
    if (model == kModelKin) {
        low_hi = NK;
    } else if (acc > 0.0f) {
        low_hi = first_true(NK, (kVMin - o.v0) / dvf, [&](int n) { return speed_at(v0_d, dv_d, n) >= kVMinD; });
    } else if (acc < 0.0f) {
        low_lo = first_true(NK, (kVMin - o.v0) / dvf, [&](int n) { return speed_at(v0_d, dv_d, n) < kVMinD; });
        low_hi = NK;
    } else if (v0_d < kVMinD) {
        low_hi = NK;
    }
    int n_stop = NK;   // sub-step at which v_{n+1} < 0 first holds
    if (acc < 0.0f)
        n_stop = first_true(NK, -o.v0 / dvf - 1.0f, [&](int n) { return speed_at(v0_d, dv_d, n + 1) < 0.0; });

    const float ti = (float)tau_i_d;
    const float hti2 = 0.5f * ti * ti;
    const float dv = dvf;
    const float L = o.lf + o.lr;
    const float inv_m = 1.0f / o.m, inv_iz = 1.0f / o.Iz;
    const float k11 = -(o.caf + o.car) * inv_m;                 // a11 * v
    const float k12 = (o.car * o.lr - o.caf * o.lf) * inv_m;    // (a12 + 1) * v^2
    const float k21 = (o.car * o.lr - o.caf * o.lf) * inv_iz;   // a21
    const float k22 = -(o.caf * o.lf * o.lf + o.car * o.lr * o.lr) * inv_iz;  // a22 * v
    const float kb1 = o.caf * inv_m * delta;                    // b1 * v * delta
    const float kb2 = o.caf * o.lf * inv_iz * delta;            // b2 * delta
    const float tdel = tanf(delta);
    const float beta_kin = atanf(o.lr * tdel / L);
    const float kappa = cosf(beta_kin) * tdel / L;              // r = v * kappa in the kinematic limit
    const float stop_den = 0.5f / fabsf(acc == 0.0f ? 1.0f : acc);

    float xh = o.x0, xc = 0.0f, yh = o.y0, yc = 0.0f, ph = o.psi0, pc = 0.0f;   // Kahan sums
    float cps, sps;                      // cos / sin of the heading, carried between output steps
    sincos2(ph, -pc, sps, cps);
    float beta = 0.0f, r = 0.0f, ax = acc, ay = 0.0f;
    bool stopped = false;
    int n = 0;
    for (int k = 0; k < N; ++k) {
        for (int q = 0; q < K; ++q, ++n) {
            // every lane runs the same straight-line sub-step; regime and stop act through selects
            const bool low = n >= low_lo && n < low_hi;
            const bool stop_now = n == n_stop;
            const float v = fmaf((float)n, dv, o.v0);
            const float iv = __fdividef(1.0f, fmaxf(v, 1e-3f));
            const float bd_ot = fmaf(k11 * iv, beta, fmaf(fmaf(k12 * iv, iv, -1.0f), r, kb1 * iv));
            const float rd_ot = fmaf(k21, beta, fmaf(k22 * iv, r, kb2));
            const float b_use = low ? beta_kin : beta;
            const float r_use = low ? v * kappa : r;
            const float bd = low ? 0.0f : bd_ot;
            const float rd = low ? 0.0f : rd_ot;
            float sb, cb;
            sincos_half(b_use, sb, cb);
            const float cpb = fmaf(cps, cb, -sps * sb);          // course angle psi + beta
            const float spb = fmaf(sps, cb, cps * sb);
            const float d_stop = v * v * stop_den;
            const float dx = stop_now ? cpb * d_stop : fmaf(cpb * v, ti, fmaf(cps, ax, -sps * ay) * hti2);
            const float dy = stop_now ? spb * d_stop : fmaf(spb * v, ti, fmaf(sps, ax, cps * ay) * hti2);
            const float w = v * (bd + r_use);
            const float ax_n = fmaf(cb, acc, -sb * w);
            const float ay_n = fmaf(sb, acc, cb * w);
            const float dpsi = fmaf(r_use, ti, rd * hti2);
            const bool move = !stopped && !stop_now;             // a state update beyond the position
            kahan_add(xh, xc, stopped ? 0.0f : dx);
            kahan_add(yh, yc, stopped ? 0.0f : dy);
            kahan_add(ph, pc, move ? dpsi : 0.0f);
            if (move) {
                beta = fmaf(bd, ti, b_use);
                r = fmaf(rd, ti, r_use);
                ax = ax_n;
                ay = ay_n;
                float sd, cd;                                   // rotate (cos, sin) of the heading by dpsi
                sincos_tenth(dpsi, sd, cd);
                const float c2 = fmaf(cps, cd, -sps * sd);
                sps = fmaf(sps, cd, cps * sd);
                cps = c2;
            }
            stopped = stopped || stop_now;
        }
        sincos2(ph, -pc, sps, cps);                              // re-anchor on the exact heading
        const long long idx = base + (long long)k * h + i;
        X[idx] = xh - xc;
        Y[idx] = yh - yc;
        C[idx] = cps;
        S[idx] = sps;
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
    if (w >= a.n_warps || (threadIdx.x & 31) >= a.lanes) return;
    const ObjDesc &o = a.objs[a.warp_obj[w]];
    const int i = a.warp_first[w] + (threadIdx.x & 31);
    if (i >= o.h) return;
    const int ia = i / o.n_b, ib = i - ia * o.n_b;
    const float ga = a.grids[o.grid_off + ia];
    const float gb = a.grids[o.grid_off + o.n_a + ib];
    if (o.kind == kVehicle)
        vehicle(o, ga, gb, o.model, o.n_steps, o.substeps, o.tau_i_d, o.pose_base, o.h, i, a.x, a.y, a.c, a.s);
    else
        pedestrian(o, ga, gb, o.n_steps, o.tau, o.pose_base, o.h, i, a.x, a.y, a.c, a.s);
}

// Bounding box of the 32 pose centres of each bound tile at each step (warp min/max reduction).
__global__ void __launch_bounds__(256) bounds_kernel(const BoundsArgs a) {
    const long long g = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const long long total = (long long)a.n_warps * a.max_steps;
    if (g >= total) return;
    const int w = (int)(g / a.max_steps), k = (int)(g - (long long)w * a.max_steps);
    const ObjDesc &o = a.objs[a.warp_obj[w]];
    if (k >= o.n_steps) return;
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
    if (lane == 0) a.bounds[o.bounds_base + (long long)(a.warp_first[w] / kBoundTile) * o.n_steps + k] =
        make_float4(x0, y0, x1, y1);
}

}  // namespace

cudaError_t launch_generate(const GenArgs &a, cudaStream_t st) {
    if (a.n_warps <= 0) return cudaSuccess;
    // few warps: one warp per block so that the latency-bound integration spreads over all SMs
    const int warps_per_block = a.n_warps < 4 * 152 ? 1 : 4;
    const int blocks = (a.n_warps + warps_per_block - 1) / warps_per_block;
    gen_kernel<<<blocks, 32 * warps_per_block, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_bounds(const BoundsArgs &a, cudaStream_t st) {
    const long long total = (long long)a.n_warps * a.max_steps;
    if (total <= 0) return cudaSuccess;
    const long long blocks = (total + 7) / 8;
    bounds_kernel<<<(unsigned)blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace mhc
