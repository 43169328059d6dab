// gen.cu -- trajectory generation (Section IV-B): a warp per hypothesis with its sub-steps in parallel
// (scenarios with few hypotheses), or a thread per hypothesis with its sub-steps in order.
//
// Vehicles: one-track model (Eq. onetrack) with constant steering and acceleration, integrated by
// Eq. (EulerVelocity) with sub-step tau / K; the low-speed kinematic limit and the stop rule are applied
// on the sub-steps where the FP64 speed v_0 + n vdot tau_i crosses 2 m/s / zero (decided on the host in
// FP64, per object and acceleration value, and read from a table: no FP64 arithmetic runs here).  Arithmetic is FP32; x, y and psi are carried as
// compensated (hi, lo) sums so that 250+ sub-steps add no more than ~1e-6 m of rounding.
// Pedestrians: Eq. (pedestrianmotion) with a constant acceleration integrates exactly, so every output
// pose is evaluated in closed form (speed saturating at 0 or at the cap).
#include <algorithm>

#include "mhc_internal.cuh"
#include "prepare.cuh"

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

__device__ void vehicle(const ObjDesc &o, float acc, float delta, const Regime &g, int N, int K, double tau_i_d,
                        long long base, int h, int i, float *X, float *Y, float *C, float *S) {
    const float dvf = (float)__dmul_rn((double)acc, tau_i_d);
    const int low_lo = g.low_lo, low_hi = g.low_hi, n_stop = g.n_stop;   // low regime on [low_lo, low_hi)

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

// Path hypotheses (Section IV-B.2b): before every sub-step the lateral controller of Eq. (controller) sets
// the front steering angle, in degrees, from the speed, the signed distance d_path from the centre of
// gravity predicted kCtrlTp ahead along the course to the active section's line (positive when the line
// lies to the left) and the yaw error e_psi = psi_section - psi; the angle is held within kDeltaMax and
// within kDeltaRate x tau_i of the previous sub-step's (0 before the first).  The one-track step is then
// the constant-steering one of `vehicle` with that angle.
constexpr float kCtrlTp = 0.5f;       // s: prediction time of the centre of gravity
constexpr float kDeltaMax = 0.5f;     // rad
constexpr float kDeltaRate = 0.5f;    // rad/s
constexpr float kPi = 3.14159265358979f;

__device__ void vehicle_path(const ObjDesc &o, float acc, const float *path, const Regime &g, int N, int K,
                             double tau_i_d, long long base, int h, int i, float *X, float *Y, float *C, float *S) {
    const float dv = (float)__dmul_rn((double)acc, tau_i_d);
    const int low_lo = g.low_lo, low_hi = g.low_hi, n_stop = g.n_stop;
    const float ti = (float)tau_i_d;
    const float hti2 = 0.5f * ti * ti;
    const float L = o.lf + o.lr;
    const float inv_m = 1.0f / o.m, inv_iz = 1.0f / o.Iz;
    const float k11 = -(o.caf + o.car) * inv_m;
    const float k12 = (o.car * o.lr - o.caf * o.lf) * inv_m;
    const float k21 = (o.car * o.lr - o.caf * o.lf) * inv_iz;
    const float k22 = -(o.caf * o.lf * o.lf + o.car * o.lr * o.lr) * inv_iz;
    const float kb1u = o.caf * inv_m;                           // b1 * v per rad of steering
    const float kb2u = o.caf * o.lf * inv_iz;                   // b2 per rad of steering
    const float stop_den = 0.5f / fabsf(acc == 0.0f ? 1.0f : acc);
    const float step_max = kDeltaRate * ti;
    float sec_x[3], sec_y[3], sec_psi[3], sec_nx[3], sec_ny[3];  // sections: point, direction, left normal
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        sec_x[q] = path[3 * q];
        sec_y[q] = path[3 * q + 1];
        sec_psi[q] = path[3 * q + 2];
        float sn, cs;
        sincosf(sec_psi[q], &sn, &cs);
        sec_nx[q] = -sn;
        sec_ny[q] = cs;
    }

    float xh = o.x0, xc = 0.0f, yh = o.y0, yc = 0.0f, ph = o.psi0, pc = 0.0f;   // Kahan sums
    float cps, sps;
    sincos2(ph, -pc, sps, cps);
    float beta = 0.0f, r = 0.0f, ax = acc, ay = 0.0f, delta = 0.0f;
    bool stopped = false;
    int n = 0;
    for (int k = 0; k < N; ++k) {
        for (int q = 0; q < K; ++q, ++n) {
            const bool low = n >= low_lo && n < low_hi;
            const bool stop_now = n == n_stop;
            const float v = fmaf((float)n, dv, o.v0);
            float sb0, cb0;                                      // the course of the state before the step
            sincos_half(beta, sb0, cb0);
            if (!stopped) {   // the controller, on the state before this sub-step
                const int sec = n < o.path_n1 ? 0 : (n < o.path_n2 ? 1 : 2);
                const float px = (xh - xc) + kCtrlTp * v * fmaf(cps, cb0, -sps * sb0);
                const float py = (yh - yc) + kCtrlTp * v * fmaf(sps, cb0, cps * sb0);
                const float d_path = fmaf(sec_x[sec] - px, sec_nx[sec], (sec_y[sec] - py) * sec_ny[sec]);
                float e_psi = sec_psi[sec] - (ph - pc);
                e_psi -= 2.0f * kPi * floorf((e_psi + kPi) * (0.5f / kPi));
                const float gd = fabsf(fmaf(-0.018f, v, 1.5f) * d_path);
                const float cmd = ((gd + 0.5f) * d_path + (9.5f - gd) * (3.8197f * e_psi)) * (kPi / 180.0f);
                delta = fminf(fmaxf(delta + fminf(fmaxf(cmd - delta, -step_max), step_max), -kDeltaMax), kDeltaMax);
            }
            const float kb1 = kb1u * delta, kb2 = kb2u * delta;
            float beta_kin = 0.0f, kappa = 0.0f;
            float sb = sb0, cb = cb0;                            // the one-track step keeps the course
            if (low) {                                           // the kinematic limit at the new angle
                const float tdel = tanf(delta);
                beta_kin = atanf(o.lr * tdel / L);
                kappa = cosf(beta_kin) * tdel / L;
                sincos_half(beta_kin, sb, cb);
            }
            const float iv = __fdividef(1.0f, fmaxf(v, 1e-3f));
            const float bd_ot = fmaf(k11 * iv, beta, fmaf(fmaf(k12 * iv, iv, -1.0f), r, kb1 * iv));
            const float rd_ot = fmaf(k21, beta, fmaf(k22 * iv, r, kb2));
            const float b_use = low ? beta_kin : beta;
            const float r_use = low ? v * kappa : r;
            const float bd = low ? 0.0f : bd_ot;
            const float rd = low ? 0.0f : rd_ot;
            const float cpb = fmaf(cps, cb, -sps * sb);
            const float spb = fmaf(sps, cb, cps * sb);
            const float d_stop = v * v * stop_den;
            const float dx = stop_now ? cpb * d_stop : fmaf(cpb * v, ti, fmaf(cps, ax, -sps * ay) * hti2);
            const float dy = stop_now ? spb * d_stop : fmaf(spb * v, ti, fmaf(sps, ax, cps * ay) * hti2);
            const float w = v * (bd + r_use);
            const float ax_n = fmaf(cb, acc, -sb * w);
            const float ay_n = fmaf(sb, acc, cb * w);
            const float dpsi = fmaf(r_use, ti, rd * hti2);
            const bool move = !stopped && !stop_now;
            kahan_add(xh, xc, stopped ? 0.0f : dx);
            kahan_add(yh, yc, stopped ? 0.0f : dy);
            kahan_add(ph, pc, move ? dpsi : 0.0f);
            if (move) {
                beta = fmaf(bd, ti, b_use);
                r = fmaf(rd, ti, r_use);
                ax = ax_n;
                ay = ay_n;
                float sd, cd;
                sincos_tenth(dpsi, sd, cd);
                const float c2 = fmaf(cps, cd, -sps * sd);
                sps = fmaf(sps, cd, cps * sd);
                cps = c2;
            }
            stopped = stopped || stop_now;
        }
        sincos2(ph, -pc, sps, cps);
        const long long idx = base + (long long)k * h + i;
        X[idx] = xh - xc;
        Y[idx] = yh - yc;
        C[idx] = cps;
        S[idx] = sps;
    }
}

// output steps k0, k0 + dk, ... of one pedestrian hypothesis (closed form)
__device__ void pedestrian(const ObjDesc &o, float ga, float gb, int N, float tau, long long base, int h, int i,
                           float *X, float *Y, float *C, float *S, int k0 = 0, int dk = 1) {
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
    for (int k = k0; k < N; k += dk) {
        const float t = (float)(k + 1) * tau;
        const float s = t < ts ? fmaf(0.5f * a * t, t, v0 * t) : fmaf(v_sat, t - ts, s_sat);
        const long long idx = base + (long long)k * h + i;
        X[idx] = fmaf(ct, s, o.x0);
        Y[idx] = fmaf(st, s, o.y0);
        C[idx] = ct;
        S[idx] = st;
    }
}

// ---- parallel-in-time generation: one warp per hypothesis ----------------------------------------------
//
// Every sub-step maps the lateral state s = (beta, r) affinely: s' = M_n s + c_n, with M_n, c_n functions of
// the speed v_n alone (one-track model: M = I + tau_i A(v_n), c = tau_i b(v_n); kinematic limit: M = 0,
// c = (beta_kin, v_n kappa); stopped: M = I, c = 0).  The warp's lanes take 8 consecutive sub-steps each,
// compose their maps, and one warp scan of the compositions gives every lane its start state; each lane
// then runs its sub-steps in order.  Heading and position are sums of per-sub-step increments, so they
// are prefix sums (double-float: an FP32 (hi, lo) pair per value, exact two-sum additions) over the lanes.

// (hi, lo) + (bh, bl), renormalised
__device__ __forceinline__ void df_add(float &hi, float &lo, float bh, float bl) {
    const float s = __fadd_rn(hi, bh);
    const float bb = __fsub_rn(s, hi);
    float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(bh, bb));
    e = __fadd_rn(e, __fadd_rn(lo, bl));
    hi = __fadd_rn(s, e);
    lo = __fsub_rn(e, __fsub_rn(hi, s));
}

// inclusive warp scan of double-float values (lane order = time order)
__device__ __forceinline__ void df_scan(float &hi, float &lo, int lane) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const float h2 = __shfl_up_sync(0xffffffffu, hi, d), l2 = __shfl_up_sync(0xffffffffu, lo, d);
        if (lane >= d) {
            float th = h2, tl = l2;
            df_add(th, tl, hi, lo);
            hi = th;
            lo = tl;
        }
    }
}

// Affine map of the lateral state: s' = [m00 m01; m10 m11] s + (c0, c1).
struct Aff {
    float m00, m01, m10, m11, c0, c1;
};

// second after first: the map that applies `first`, then `second`
__device__ __forceinline__ Aff aff_then(const Aff &first, const Aff &second) {
    Aff r;
    r.m00 = fmaf(second.m00, first.m00, second.m01 * first.m10);
    r.m01 = fmaf(second.m00, first.m01, second.m01 * first.m11);
    r.m10 = fmaf(second.m10, first.m00, second.m11 * first.m10);
    r.m11 = fmaf(second.m10, first.m01, second.m11 * first.m11);
    r.c0 = fmaf(second.m00, first.c0, fmaf(second.m01, first.c1, second.c0));
    r.c1 = fmaf(second.m10, first.c0, fmaf(second.m11, first.c1, second.c1));
    return r;
}

// One vehicle hypothesis by the whole warp (every lane calls it).  Rounds of 32 x 5 sub-steps; lane L
// takes sub-steps L*5 .. L*5+4 of the round (five per lane keeps the unrolled loops short and out of
// local memory; a 150-sub-step horizon still takes one round).  Per round: compose and scan the lanes'
// state maps, run the lanes' sub-steps from their start states (the same per-sub-step arithmetic as the
// sequential integration), scan the heading increments, form the position increments (heading trig
// exact at the lane's first sub-step, then rotated by each increment as the sequential integration
// rotates it), scan them, and store the poses of the output steps that end in each lane's sub-steps
// (exact heading trig).
__device__ void vehicle_scan(const ObjDesc &o, float acc, float delta, const Regime &g, int N, int K, int lane,
                             long long base, int h, int i, float *X, float *Y, float *C, float *S) {
    constexpr int CS = 5;
    const int NK = N * K;
    const float ti = (float)o.tau_i_d;
    const float hti2 = 0.5f * ti * ti;
    const float dv = (float)__dmul_rn((double)acc, o.tau_i_d);
    const float L = o.lf + o.lr;
    const float inv_m = 1.0f / o.m, inv_iz = 1.0f / o.Iz;
    const float k11 = -(o.caf + o.car) * inv_m;
    const float k12 = (o.car * o.lr - o.caf * o.lf) * inv_m;
    const float k21 = (o.car * o.lr - o.caf * o.lf) * inv_iz;
    const float k22 = -(o.caf * o.lf * o.lf + o.car * o.lr * o.lr) * inv_iz;
    const float kb1 = o.caf * inv_m * delta;
    const float kb2 = o.caf * o.lf * inv_iz * delta;
    const float tdel = tanf(delta);
    const float beta_kin = atanf(o.lr * tdel / L);
    const float kappa = cosf(beta_kin) * tdel / L;
    const float stop_den = 0.5f / fabsf(acc == 0.0f ? 1.0f : acc);

    float beta = 0.0f, r = 0.0f;                      // lateral state at the round's first sub-step
    float ax = acc, ay = 0.0f;                        // acceleration used by the round's first sub-step
    float ph = o.psi0, pl = 0.0f, xh = o.x0, xl = 0.0f, yh = o.y0, yl = 0.0f;
    for (int nr = 0; nr < NK; nr += 32 * CS) {
        // sub-steps per lane this round: CS for full rounds, fewer for the last (100 sub-steps: 4 per lane)
        const int csa = min(CS, (min(NK - nr, 32 * CS) + 31) / 32);
        const int n0 = nr + lane * csa;
        // 1. the lane's state map, composed over its sub-steps, and the warp scan of the maps
        Aff F{1.0f, 0.0f, 0.0f, 1.0f, 0.0f, 0.0f};
#pragma unroll
        for (int c = 0; c < CS; ++c) {
            const int n = n0 + c;
            if (c >= csa || n >= NK || n >= g.n_stop) continue;   // outside the lane / frozen state: identity
            const float v = fmaf((float)n, dv, o.v0);
            Aff m;
            if (n >= g.low_lo && n < g.low_hi) {
                m = Aff{0.0f, 0.0f, 0.0f, 0.0f, beta_kin, v * kappa};
            } else {
                const float iv = __fdividef(1.0f, fmaxf(v, 1e-3f));
                m = Aff{fmaf(ti, k11 * iv, 1.0f), ti * fmaf(k12 * iv, iv, -1.0f), ti * k21, fmaf(ti, k22 * iv, 1.0f),
                        ti * (kb1 * iv), ti * kb2};
            }
            F = aff_then(F, m);
        }
        Aff P = F;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            Aff q;
            q.m00 = __shfl_up_sync(0xffffffffu, P.m00, d); q.m01 = __shfl_up_sync(0xffffffffu, P.m01, d);
            q.m10 = __shfl_up_sync(0xffffffffu, P.m10, d); q.m11 = __shfl_up_sync(0xffffffffu, P.m11, d);
            q.c0 = __shfl_up_sync(0xffffffffu, P.c0, d);   q.c1 = __shfl_up_sync(0xffffffffu, P.c1, d);
            if (lane >= d) P = aff_then(q, P);
        }
        Aff E;   // the maps of the earlier lanes (identity for lane 0)
        E.m00 = __shfl_up_sync(0xffffffffu, P.m00, 1); E.m01 = __shfl_up_sync(0xffffffffu, P.m01, 1);
        E.m10 = __shfl_up_sync(0xffffffffu, P.m10, 1); E.m11 = __shfl_up_sync(0xffffffffu, P.m11, 1);
        E.c0 = __shfl_up_sync(0xffffffffu, P.c0, 1);   E.c1 = __shfl_up_sync(0xffffffffu, P.c1, 1);
        if (lane == 0) E = Aff{1.0f, 0.0f, 0.0f, 1.0f, 0.0f, 0.0f};
        float bs = fmaf(E.m00, beta, fmaf(E.m01, r, E.c0));
        float rs = fmaf(E.m10, beta, fmaf(E.m11, r, E.c1));

        // 2. the lane's sub-steps in order: slip trig, heading increments, next accelerations
        float sbv[CS], cbv[CS], dps[CS], axn[CS], ayn[CS];
        float ax_last = 0.0f, ay_last = 0.0f;             // the acceleration after the lane's last sub-step
#pragma unroll
        for (int c = 0; c < CS; ++c) {
            sbv[c] = 0.0f; cbv[c] = 1.0f; dps[c] = 0.0f; axn[c] = 0.0f; ayn[c] = 0.0f;
            if (c >= csa) continue;
            const int n = n0 + c;
            const bool move = n < NK && n < g.n_stop;
            const bool low = n >= g.low_lo && n < g.low_hi;
            const float v = fmaf((float)n, dv, o.v0);
            const float iv = __fdividef(1.0f, fmaxf(v, 1e-3f));
            const float bd_ot = fmaf(k11 * iv, bs, fmaf(fmaf(k12 * iv, iv, -1.0f), rs, kb1 * iv));
            const float rd_ot = fmaf(k21, bs, fmaf(k22 * iv, rs, kb2));
            const float b_use = low ? beta_kin : bs;
            const float r_use = low ? v * kappa : rs;
            const float bd = low ? 0.0f : bd_ot;
            const float rd = low ? 0.0f : rd_ot;
            float sb, cb;
            sincos_half(b_use, sb, cb);
            sbv[c] = sb;
            cbv[c] = cb;
            const float w = v * (bd + r_use);
            axn[c] = fmaf(cb, acc, -sb * w);
            ayn[c] = fmaf(sb, acc, cb * w);
            dps[c] = move ? fmaf(r_use, ti, rd * hti2) : 0.0f;
            if (move) {
                bs = fmaf(bd, ti, b_use);
                rs = fmaf(rd, ti, r_use);
            }
            ax_last = axn[c];
            ay_last = ayn[c];
        }
        // the next round starts from the state after every lane's maps
        {
            const float m00 = __shfl_sync(0xffffffffu, P.m00, 31), m01 = __shfl_sync(0xffffffffu, P.m01, 31);
            const float m10 = __shfl_sync(0xffffffffu, P.m10, 31), m11 = __shfl_sync(0xffffffffu, P.m11, 31);
            const float c0 = __shfl_sync(0xffffffffu, P.c0, 31), c1 = __shfl_sync(0xffffffffu, P.c1, 31);
            const float b2 = fmaf(m00, beta, fmaf(m01, r, c0));
            r = fmaf(m10, beta, fmaf(m11, r, c1));
            beta = b2;
        }

        // 3. heading at every sub-step start: lane sums, scanned
        float dh = 0.0f, dl = 0.0f;
#pragma unroll
        for (int c = 0; c < CS; ++c) df_add(dh, dl, dps[c], 0.0f);
        float ih = dh, il = dl;
        df_scan(ih, il, lane);
        float hh = ph, hl = pl;                                       // heading at the lane's first sub-step
        {
            const float eh = __shfl_up_sync(0xffffffffu, ih, 1), el = __shfl_up_sync(0xffffffffu, il, 1);
            if (lane > 0) df_add(hh, hl, eh, el);
        }
        const float th = __shfl_sync(0xffffffffu, ih, 31), tl = __shfl_sync(0xffffffffu, il, 31);
        const float h_start = hh, l_start = hl;

        // 4. position increments
        float ax_in = __shfl_up_sync(0xffffffffu, ax_last, 1), ay_in = __shfl_up_sync(0xffffffffu, ay_last, 1);
        if (lane == 0) { ax_in = ax; ay_in = ay; }
        float dxv[CS], dyv[CS];
        float sxh = 0.0f, sxl = 0.0f, syh = 0.0f, syl = 0.0f;
        float sp, cp;                                  // heading trig: exact at the lane start, then rotated
        sincos2(hh, hl, sp, cp);
#pragma unroll
        for (int c = 0; c < CS; ++c) {
            dxv[c] = dyv[c] = 0.0f;
            if (c >= csa) continue;
            const int n = n0 + c;
            const float cpb = fmaf(cp, cbv[c], -sp * sbv[c]);
            const float spb = fmaf(sp, cbv[c], cp * sbv[c]);
            const float axu = c ? axn[c - 1] : ax_in, ayu = c ? ayn[c - 1] : ay_in;
            const float v = fmaf((float)n, dv, o.v0);
            const bool stop_now = n == g.n_stop;
            const float d_stop = v * v * stop_den;
            float dx = stop_now ? cpb * d_stop : fmaf(cpb * v, ti, fmaf(cp, axu, -sp * ayu) * hti2);
            float dy = stop_now ? spb * d_stop : fmaf(spb * v, ti, fmaf(sp, axu, cp * ayu) * hti2);
            if (n >= NK || n > g.n_stop) dx = dy = 0.0f;
            dxv[c] = dx;
            dyv[c] = dy;
            df_add(sxh, sxl, dx, 0.0f);
            df_add(syh, syl, dy, 0.0f);
            if (dps[c] != 0.0f) {                      // rotate (cos, sin) of the heading by the increment
                float sd, cd;
                sincos_tenth(dps[c], sd, cd);
                const float c2 = fmaf(cp, cd, -sp * sd);
                sp = fmaf(sp, cd, cp * sd);
                cp = c2;
            }
        }
        float ixh = sxh, ixl = sxl, iyh = syh, iyl = syl;
        df_scan(ixh, ixl, lane);
        df_scan(iyh, iyl, lane);

        // 5. poses of the output steps ending in this lane's sub-steps
        float px = xh, pxl = xl, py = yh, pyl = yl;
        {
            const float eh = __shfl_up_sync(0xffffffffu, ixh, 1), el = __shfl_up_sync(0xffffffffu, ixl, 1);
            const float fh = __shfl_up_sync(0xffffffffu, iyh, 1), fl = __shfl_up_sync(0xffffffffu, iyl, 1);
            if (lane > 0) {
                df_add(px, pxl, eh, el);
                df_add(py, pyl, fh, fl);
            }
        }
        hh = h_start;
        hl = l_start;
#pragma unroll
        for (int c = 0; c < CS; ++c) {
            if (c >= csa) continue;
            const int n = n0 + c;
            df_add(px, pxl, dxv[c], 0.0f);
            df_add(py, pyl, dyv[c], 0.0f);
            df_add(hh, hl, dps[c], 0.0f);
            if (n < NK && (n + 1) % K == 0) {                // the pose stores the exact heading trig
                const int k = (n + 1) / K - 1;
                float sp, cp;
                sincos2(hh, hl, sp, cp);
                const long long idx = base + (long long)k * h + i;
                X[idx] = __fadd_rn(px, pxl);
                Y[idx] = __fadd_rn(py, pyl);
                C[idx] = cp;
                S[idx] = sp;
            }
        }

        // 6. carried into the next round
        df_add(ph, pl, th, tl);
        df_add(xh, xl, __shfl_sync(0xffffffffu, ixh, 31), __shfl_sync(0xffffffffu, ixl, 31));
        df_add(yh, yl, __shfl_sync(0xffffffffu, iyh, 31), __shfl_sync(0xffffffffu, iyl, 31));
        ax = __shfl_sync(0xffffffffu, ax_last, 31);       // used only after a full round (csa = 8)
        ay = __shfl_sync(0xffffffffu, ay_last, 31);
    }
}

// LAYOUTS: 1 every task is a warp per hypothesis, 2 every task is a thread per hypothesis, 3 both (a kernel
// holding one layout only has a smaller instruction footprint: the integration is latency-bound and
// instruction fetch was its largest stall).  Bounded to 80 registers (six CTAs per SM), where the
// integration has no spills: faster than 64 (eight per SM, all of the 11-object scene's CTAs resident)
// on the 11-object and 32-vehicle scenes.
// table[0, n) = -1 by CTA b of nb (16-byte stores on the aligned body).
__device__ __forceinline__ void fill_part(int16_t *table, long long n, long long b, long long nb) {
    const long long tid = b * blockDim.x + threadIdx.x, stride = nb * blockDim.x;
    const long long head = min(n, (long long)((16 - ((uintptr_t)table & 15)) & 15) / 2);
    if (tid < head) table[tid] = (int16_t)-1;
    const long long body = (n - head) / 8;
    int4 *v = reinterpret_cast<int4 *>(table + head);
    const int4 ones = make_int4(-1, -1, -1, -1);
    for (long long q = tid; q < body; q += stride) v[q] = ones;
    for (long long q = head + body * 8 + tid; q < n; q += stride) table[q] = (int16_t)-1;
}

// CTAs [0, fill_blocks) write the table's -1s (HBM-bound, beside the latency-bound integration: the table is
// read by nothing before the collision kernel), then come the generation CTAs, then the risk preparation.
// The last k in [0, n) with v[k] <= x (v ascending, v[0] <= x), by the whole warp: each round the lanes
// probe 64 evenly spaced entries (two each) and keep the span between the last probe <= x and the next, so
// up to 64 entries take one round of loads.
__device__ __forceinline__ int last_le(const int *v, int n, int x, int lane) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const long long span = hi - lo + 1;
        const bool le0 = v[lo + (int)(span * (2 * lane) / 64)] <= x;
        const bool le1 = v[lo + (int)(span * (2 * lane + 1) / 64)] <= x;
        const unsigned even = __ballot_sync(0xffffffffu, le0), odd = __ballot_sync(0xffffffffu, le1);
        const int le = 31 - __clz(even), lo2 = odd ? 31 - __clz(odd) : -1;   // last true even / odd probe
        const int L = 2 * lo2 + 1 > 2 * le ? 2 * lo2 + 1 : 2 * le;           // the true probes form a prefix
        const int nlo = lo + (int)(span * L / 64);
        hi = L == 63 ? hi : lo + (int)(span * (L + 1) / 64) - 1;
        lo = nlo;
    }
    return lo;
}

template <int LAYOUTS>
__global__ void __launch_bounds__(128, 6) gen_kernel(const GenArgs a) {
    // wait first: launched as a dependent of the descriptor copy kernel, this kernel lets its own dependents
    // (which read descriptors before their wait) start only once the copy is complete
    pdl_wait();
    pdl_trigger();
    if ((int)blockIdx.x < a.fill_blocks) {
        fill_part(a.fill, a.n_fill, blockIdx.x, a.fill_blocks);
        return;
    }
    const int bid = (int)blockIdx.x - a.fill_blocks;
    if (bid >= a.gen_blocks) {                           // the risk preparation, independent of generation
        prepare_block(a.prep, bid - a.gen_blocks, a.prep_blocks);
        return;
    }
    const int w = bid * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w >= a.n_warps) return;                          // whole warps leave
    if ((LAYOUTS & 1) && (LAYOUTS == 1 || w < a.n_scan)) {   // one hypothesis by the whole warp
        const int lane = threadIdx.x & 31;
        const int k = last_le(a.warp_first, a.n_scan_objs, w, lane);
        const ObjDesc &o = a.objs[a.warp_obj[k]];
        const int i = w - a.warp_first[k];
        const int ia = i / o.n_b, ib = i - ia * o.n_b;
        const float ga = a.grids[o.grid_off + ia];
        const float gb = a.grids[o.grid_off + o.n_a + ib];
        if (o.kind == kVehicle)
            vehicle_scan(o, ga, gb, a.regimes[o.regime_off + ia], o.n_steps, o.substeps, lane, o.pose_base, o.h, i,
                         a.x, a.y, a.c, a.s);
        else
            pedestrian(o, ga, gb, o.n_steps, o.tau, o.pose_base, o.h, i, a.x, a.y, a.c, a.s, lane, 32);
        return;
    }
    if (!(LAYOUTS & 2)) return;
    if ((threadIdx.x & 31) >= a.lanes) return;
    const int e = a.n_scan_objs + (w - a.n_scan);
    const ObjDesc &o = a.objs[a.warp_obj[e]];
    const int i = a.warp_first[e] + (threadIdx.x & 31);
    if (i >= o.h) return;
    const int ia = i / o.n_b, ib = i - ia * o.n_b;
    const float ga = a.grids[o.grid_off + ia];
    const float gb = a.grids[o.grid_off + o.n_a + ib];
    if (o.kind == kVehicle && o.path_off >= 0)
        vehicle_path(o, ga, a.paths + 9LL * (o.path_off + ib), a.regimes[o.regime_off + ia], o.n_steps, o.substeps,
                     o.tau_i_d, o.pose_base, o.h, i, a.x, a.y, a.c, a.s);
    else if (o.kind == kVehicle)
        vehicle(o, ga, gb, a.regimes[o.regime_off + ia], o.n_steps, o.substeps, o.tau_i_d, o.pose_base, o.h, i,
                a.x, a.y, a.c, a.s);
    else
        pedestrian(o, ga, gb, o.n_steps, o.tau, o.pose_base, o.h, i, a.x, a.y, a.c, a.s);
}

// Bounding box of the 32 pose centres of each bound tile at each step: one warp per (32-hypothesis group,
// chunk of 8 steps).  Lane i loads hypothesis i's x and y at the chunk's 8 steps (16 loads in flight),
// then a butterfly reduce-scatter over the 32 values (step s, quantity q = x min, y min, x max, y max;
// value 4 s + q) halves the values at each of its five levels, so that lane L ends with the finished value
// L and the 8 boxes go out as one 128-byte store.  The descriptors are read before the wait for the
// generation kernel, the poses after it.  With `fill` set, the CTAs past the bounds write the table's -1s
// (16-byte stores on the aligned body) before the wait: nothing earlier in the launch sequence reads the
// table, so the HBM-rate fill overlaps the generation kernel's tail, and the collision kernel stores first
// hits only.
constexpr int kFillCtas = 152 * 4;
// Fill CTAs of the generation launch (the rest of each SM integrates).  Two per SM spread the fill's stores
// over every SM, which a table much larger than the generation work needs to reach the HBM rate (32-vehicle
// scene: 0.74 ms at two per SM, 0.94 ms at one); when the generation work is comparable, half an SM's worth
// leaves it more room and both finish sooner (256-scenario batch: 1.68 ms against 2.01 ms).
constexpr int kGenFillCtas = 152 * 2;
constexpr int kGenFillCtasShared = 76;
constexpr long long kFillPerHypothesis = 8192;   // table entries per hypothesis above which the fill dominates
constexpr int kBoundSteps = 8;          // steps per warp task

__device__ __forceinline__ float box_op(bool is_max, float u, float v) { return is_max ? fmaxf(u, v) : fminf(u, v); }

__global__ void __launch_bounds__(256) bounds_kernel(const BoundsArgs a) {
    pdl_trigger();
    const int chunks = (a.max_steps + kBoundSteps - 1) / kBoundSteps;
    const long long total = (long long)a.n_warps * chunks;
    const long long bound_ctas = (total + 7) / 8;
    if ((long long)blockIdx.x >= bound_ctas) {   // a fill CTA
        fill_part(a.fill, a.n_fill, (long long)blockIdx.x - bound_ctas, (long long)gridDim.x - bound_ctas);
        pdl_wait();
        return;
    }
    const long long g = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    bool live = g < total;
    int k0 = 0, first = 0, h = 0, n_steps = 0;
    long long pose_base = 0, bounds_base = 0;
    if (live) {
        const int w = (int)(g / chunks);
        k0 = (int)(g - (long long)w * chunks) * kBoundSteps;
        const ObjDesc &o = a.objs[a.warp_obj[w]];
        first = a.warp_first[w];
        h = o.h;
        n_steps = o.n_steps;
        pose_base = o.pose_base;
        bounds_base = o.bounds_base;
    }
    pdl_wait();
    if (a.zero_counts && g == 0 && lane == 0) {
        a.zero_counts[0] = 0ull;
        a.zero_counts[1] = 0ull;
    }
    if (!live || k0 >= n_steps) return;             // uniform over the warp
    const int i = first + lane;
    float v[4 * kBoundSteps];                       // value 4 s + q of step k0 + s
#pragma unroll
    for (int s = 0; s < kBoundSteps; ++s) {
        const bool ok = i < h && k0 + s < n_steps;
        const long long idx = pose_base + (long long)(k0 + s) * h + i;
        const float x = ok ? a.x[idx] : INFINITY, y = ok ? a.y[idx] : INFINITY;
        v[4 * s] = x;
        v[4 * s + 1] = y;
        v[4 * s + 2] = ok ? x : -INFINITY;
        v[4 * s + 3] = ok ? y : -INFINITY;
    }
    // levels 16, 8, 4: the kept values keep their quantity (q = index mod 4)
#pragma unroll
    for (int d = 16, n = 16; d >= 4; d >>= 1, n >>= 1) {
        const bool upper = lane & d;
#pragma unroll
        for (int j = 0; j < n; ++j) {
            const float send = upper ? v[j] : v[j + n], keep = upper ? v[j + n] : v[j];
            v[j] = box_op((j & 3) >= 2, keep, __shfl_xor_sync(0xffffffffu, send, d));
        }
    }
    {   // level 2: values q = 0, 1 (minima) or 2, 3 (maxima) kept
        const bool upper = lane & 2;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const float send = upper ? v[j] : v[j + 2], keep = upper ? v[j + 2] : v[j];
            v[j] = box_op(upper, keep, __shfl_xor_sync(0xffffffffu, send, 2));
        }
    }
    {   // level 1
        const bool upper = lane & 1;
        const float send = upper ? v[0] : v[1], keep = upper ? v[1] : v[0];
        v[0] = box_op(lane & 2, keep, __shfl_xor_sync(0xffffffffu, send, 1));
    }
    const int s = lane >> 2;                        // lane L holds value L: step k0 + L / 4, quantity L % 4
    if (k0 + s < n_steps) {
        float *out = reinterpret_cast<float *>(a.bounds + bounds_base + (long long)(first / kBoundTile) * n_steps + k0);
        out[lane] = v[0];
    }
}

}  // namespace

cudaError_t launch_generate(const GenArgs &args, cudaStream_t st, bool pdl) {
    GenArgs a = args;
    if (a.n_warps <= 0 && a.prep_blocks <= 0) return cudaSuccess;
    // few warps: one warp per block so that the latency-bound integration spreads over all SMs; the
    // preparation CTAs (if any) then have 128 threads as well
    const int warps_per_block = a.n_warps < 4 * 152 ? 1 : 4;
    a.gen_blocks = (a.n_warps + warps_per_block - 1) / warps_per_block;
    const long long hyps = (long long)a.n_scan + (long long)(a.n_warps - a.n_scan) * a.lanes;
    const long long cap = a.n_fill > kFillPerHypothesis * std::max(1LL, hyps) ? kGenFillCtas : kGenFillCtasShared;
    a.fill_blocks = a.fill && a.n_fill > 0 ? (int)std::min(cap, (a.n_fill / 8 + 127) / 128 + 1) : 0;
    const long long blocks = (long long)a.fill_blocks + a.gen_blocks + (a.prep_blocks > 0 ? a.prep_blocks : 0);
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    auto kernel = a.n_scan >= a.n_warps ? gen_kernel<1> : (a.n_scan <= 0 ? gen_kernel<2> : gen_kernel<3>);
    return launch_kernel(kernel, dim3((unsigned)blocks), dim3(32 * warps_per_block), 0, st, pdl, a);
}

cudaError_t launch_bounds(const BoundsArgs &a, cudaStream_t st, bool pdl) {
    const long long total = (long long)a.n_warps * ((a.max_steps + kBoundSteps - 1) / kBoundSteps);
    if (total <= 0) return cudaSuccess;
    long long blocks = (total + 7) / 8;
    if (a.fill && a.n_fill > 0) blocks += std::min((long long)kFillCtas, (a.n_fill / 8 + 255) / 256 + 1);
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    return launch_kernel(bounds_kernel, dim3((unsigned)blocks), dim3(256), 0, st, pdl, a);
}

}  // namespace mhc
