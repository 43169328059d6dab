/*
 * mhc_oracle.c -- plain, slow, FP64 CPU oracle of the multi-hypothesis criticality method.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this file's library.  It shares no code, header, table or constant with the CUDA library:
 * every formula below is written out from the paper (arXiv 2005.06773, "Parallel Multi-Hypothesis
 * Algorithm for Criticality Estimation in Traffic and Collision Avoidance") in its own order and
 * notation, in double precision, without blocking, fusion or reordering.
 *
 * Readings taken where the paper is silent or ambiguous:
 *  R-a  yaw rate update r_{n+1} = r_n + rdot_n tau (omitted in Eq. EulerVelocity).
 *  R-b  a_x,0 = vdot, a_y,0 = 0 (a_{.,n} is used before it is defined); this makes straight-line
 *       constant-acceleration motion exact.
 *  R-c  the state is integrated with sub-step tau_i = tau / K and every K-th state is an output pose;
 *       output step k (k = 0..N-1) is the state at time (k+1) tau; the initial state is not tested.
 *  R-d  speed v_n = v_0 + n vdot tau_i (the Euler recurrence of Eq. EulerVelocity written out);
 *       the low-speed and stop decisions below are taken on this FP64 value.
 *  R-e  below V_MIN = 2 m/s (and always for the kinematic model) the one-track model is replaced by
 *       its kinematic limit: beta = atan(l_r tan(delta) / L), r = v cos(beta) tan(delta) / L,
 *       betadot = rdot = 0.
 *  R-f  no reversing: if v_{n+1} < 0 the vehicle advances by its exact stopping distance
 *       v_n^2 / (2 |vdot|) along the course psi_n + beta_n and stays there.
 *  R-g  pedestrians: constant heading psi_P = psi0 + offset; speed saturates at 0 and, if a cap is
 *       given and the acceleration is positive, at the cap; the saturating sub-step is integrated
 *       exactly piecewise.
 *  R-h  overlap is the intersection of the closed shapes (touching counts); the signed margin is the
 *       Euclidean distance when disjoint and minus the penetration depth when they intersect.
 *  R-i  conditional probability (Eq. p21) is applied per EGO trajectory over its colliding
 *       (CO object, CO trajectory, step) entries in ascending (step, object, trajectory) order.
 *  R-s  path hypotheses (Section IV-B.2b): a vehicle given paths follows path i_b instead of a constant
 *       steering angle; a path is three straight sections (a point and a direction each), the first
 *       followed for t < 1.0 s, the second for t < 1.5 s, the third after (the paper's sampling instants
 *       1.0 / 1.5 / 2.0 s mark the sections' sample points).
 *  R-t  lateral controller, Eq. (controller), evaluated before every sub-step: delta_f in degrees from
 *       v_V = v_n in m/s, d_path in m and e_psi in rad; d_path is the signed distance from the centre of
 *       gravity predicted T_P = 0.5 s ahead along the course (x + T_P v cos(psi + beta), ...) to the
 *       active section's line, positive when the line lies to the vehicle's left; e_psi = psi_section -
 *       psi wrapped to [-pi, pi]; no dynamic weighting (not specified).
 *  R-u  steering limits: |delta_f| <= 0.5 rad and |delta_n - delta_{n-1}| <= 0.5 rad/s x tau_i, with
 *       delta_{-1} = 0 (the current steering angle is not an input).
 *  R-v  lane dividers (Section IV-A) are given in the vehicle's frame at t = 0 (x ahead, y to the left) as
 *       three points each, ordered from right to left; divider j is y = a x^2 + b x + c through its
 *       points (Gauss-Jordan with partial pivoting).  The vehicle's lane is the pair of adjacent dividers
 *       that encloses its position; the lanes beside it (if their dividers are given) are its neighbours.
 *  R-x  trajectory scores (Eq. normTraj; the paper fixes neither its weights nor its factors):
 *       n_h = (w_acc n_acc + w_str d_str) / (c_com c_cou) with w_acc = w_str = 0.5;
 *       vehicles: n_acc = 1 / (1 + |vdot| / 2 m/s^2) (the reference keeps its speed);
 *         constant steering: d_str = 1 / (1 + |delta| / 0.05 rad), c_com = c_cou = 1;
 *         paths: with o_s the lateral offset of section s's point from the vehicle's initial line
 *         (positive to the left), d_str = 1 / (1 + max |o_s| / 1.75 m), c_com = 1 + (|o_1 - o_0| +
 *         |o_2 - o_1|) / 3.5 m, c_cou = 2 if max o_s > 1.75 m (the lane to the left carries counter
 *         traffic), else 1;
 *       pedestrians: n_acc = 1 / (1 + |v - v0| / 1 m/s) for speed grids, 1 / (1 + |vdot| / 2 m/s^2) for
 *         acceleration grids; d_str = 1 / (1 + |heading offset| / 0.5 rad); c_com = c_cou = 1.
 *       orc_scores: parity unpinned beyond this reading's own properties (the paper gives no values).
 *  R-w  path sampling (Section IV-B.2b): at the instants 1.0 / 1.5 / 2.0 s the reference position is
 *       x_t = v0 t ahead; the own lane is sampled at 1/4, 1/2 and 3/4 of its width at x_t, each
 *       neighbouring lane at 1/3 and 2/3 (right to left); a section passes through a sample point with the
 *       direction of the lane's centre line there (atan of its slope).  A CO gets one path per sample
 *       index (the same index at every instant, m paths); the EGO every combination (m^3 paths, index of
 *       the first instant slowest).  Sections are returned in the scenario frame.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_VEHICLE 0
#define ORC_PEDESTRIAN 1
#define ORC_MODEL_OT 0
#define ORC_MODEL_KIN 1
#define ORC_PED_ACCEL_GRID 1
#define ORC_V_MIN 2.0

/* ------------------------------------------------------------------------------------------------
 * Trajectory generation (Section IV-B)
 * ------------------------------------------------------------------------------------------------ */

/* Path following (readings R-s, R-t, R-u). */
#define ORC_PATH_T1 1.0          /* s: end of the first section */
#define ORC_PATH_T2 1.5          /* s: end of the second section */
#define ORC_CTRL_TP 0.5          /* s: prediction time of the centre of gravity */
#define ORC_DELTA_MAX 0.5        /* rad */
#define ORC_DELTA_RATE 0.5       /* rad/s */

static const double ORC_PI = 3.14159265358979323846;

/* Eq. (controller): front steering angle in degrees from the distance and yaw errors. */
static double controller_deg(double v, double d_path, double e_psi) {
    double g = fabs((-0.018 * v + 1.5) * d_path);
    return (g + 0.5) * d_path + (-g + 9.5) * (3.8197 * e_psi);
}

/* Steering angle for sub-step n of a path hypothesis: the controller's command for the active section,
   then the rate and angle limits relative to the previous sub-step's angle. */
static double path_steering(const double *path, long n, double tau_i, double x, double y, double psi,
                            double beta, double v, double delta_prev) {
    double t = (double)n * tau_i;
    int s = t < ORC_PATH_T1 ? 0 : (t < ORC_PATH_T2 ? 1 : 2);
    double sx = path[3 * s], sy = path[3 * s + 1], spsi = path[3 * s + 2];
    double px = x + ORC_CTRL_TP * v * cos(psi + beta);            /* predicted centre of gravity */
    double py = y + ORC_CTRL_TP * v * sin(psi + beta);
    double d_path = (sx - px) * -sin(spsi) + (sy - py) * cos(spsi);   /* line to the left: positive */
    double e_psi = spsi - psi;
    e_psi -= 2.0 * ORC_PI * floor((e_psi + ORC_PI) / (2.0 * ORC_PI));
    double cmd = controller_deg(v, d_path, e_psi) * ORC_PI / 180.0;
    double step = ORC_DELTA_RATE * tau_i;
    double delta = delta_prev + fmin(fmax(cmd - delta_prev, -step), step);
    return fmin(fmax(delta, -ORC_DELTA_MAX), ORC_DELTA_MAX);
}

/* Section IV-A: divider y = a x^2 + b x + c through three points (x_i, y_i), by Gauss-Jordan elimination
   of [x_i^2, x_i, 1 | y_i] with partial pivoting.  Returns 0, or -1 if the points fix no such curve. */
int orc_divider_fit(const double *pts, double *coef) {
    double m[3][4];
    for (int r = 0; r < 3; ++r) {
        double x = pts[2 * r], y = pts[2 * r + 1];
        m[r][0] = x * x; m[r][1] = x; m[r][2] = 1.0; m[r][3] = y;
    }
    for (int col = 0; col < 3; ++col) {
        int piv = col;
        for (int r = col + 1; r < 3; ++r) if (fabs(m[r][col]) > fabs(m[piv][col])) piv = r;
        if (!(fabs(m[piv][col]) > 1e-12)) return -1;
        for (int q = 0; q < 4; ++q) { double t = m[col][q]; m[col][q] = m[piv][q]; m[piv][q] = t; }
        double d = m[col][col];
        for (int q = 0; q < 4; ++q) m[col][q] /= d;
        for (int r = 0; r < 3; ++r) {
            if (r == col) continue;
            double f = m[r][col];
            for (int q = 0; q < 4; ++q) m[r][q] -= f * m[col][q];
        }
    }
    coef[0] = m[0][3]; coef[1] = m[1][3]; coef[2] = m[2][3];
    return 0;
}

/* Paths of one vehicle from its lane dividers (readings R-v, R-w).  div: n_div (2..4) dividers x 3 points
   (x, y) in the vehicle frame, right to left.  Writes up to 343 paths x 3 sections x (x, y, psi) to out and
   returns their number, or -1 if a divider has no fit or no lane encloses the vehicle. */
int orc_lane_paths(const double *div, int n_div, double x0, double y0, double psi0, double v0, int ego,
                   double *out) {
    double cf[4][3];
    if (n_div < 2 || n_div > 4) return -1;
    for (int j = 0; j < n_div; ++j) if (orc_divider_fit(div + 6 * j, cf[j])) return -1;
    int own = -1;                                   /* lane between dividers own and own + 1 */
    for (int j = 0; j + 1 < n_div; ++j)
        if (cf[j][2] <= 0.0 && 0.0 <= cf[j + 1][2]) { own = j; break; }
    if (own < 0) return -1;
    const double times[3] = {1.0, 1.5, 2.0};
    double sy[3][7], spsi[3][7];                    /* per instant: lateral position and direction */
    int m = 0;
    for (int k = 0; k < 3; ++k) {
        double x = v0 * times[k];
        int q = 0;
        for (int lane = own - 1; lane <= own + 1; ++lane) {   /* right neighbour, own, left neighbour */
            if (lane < 0 || lane + 1 >= n_div) continue;
            const double *r = cf[lane], *l = cf[lane + 1];
            double yr = (r[0] * x + r[1]) * x + r[2], yl = (l[0] * x + l[1]) * x + l[2];
            double slope = ((2.0 * r[0] * x + r[1]) + (2.0 * l[0] * x + l[1])) / 2.0;
            int n = lane == own ? 3 : 2;
            for (int u = 1; u <= n; ++u) {
                sy[k][q] = yr + (yl - yr) * u / (n + 1);
                spsi[k][q] = atan(slope);
                ++q;
            }
        }
        m = q;
    }
    const double c = cos(psi0), s = sin(psi0);
    int n_paths = 0;
    for (int i0 = 0; i0 < m; ++i0)
        for (int i1 = 0; i1 < (ego ? m : 1); ++i1)
            for (int i2 = 0; i2 < (ego ? m : 1); ++i2) {
                int idx[3] = {i0, ego ? i1 : i0, ego ? i2 : i0};
                for (int k = 0; k < 3; ++k) {
                    double bx = v0 * times[k], by = sy[k][idx[k]];
                    double *o = out + 9 * n_paths + 3 * k;
                    o[0] = x0 + c * bx - s * by;
                    o[1] = y0 + s * bx + c * by;
                    o[2] = psi0 + spsi[k][idx[k]];
                }
                ++n_paths;
            }
    return n_paths;
}

/* Speed at sub-step n (reading R-d). */
static double speed_at(double v0, double vdot, double tau_i, long n) {
    return v0 + (double)n * (vdot * tau_i);
}

/*
 * One vehicle hypothesis: one-track model (Eq. onetrack) with constant front steering angle delta and
 * constant longitudinal acceleration vdot, pose integration by Eq. (EulerVelocity).
 * params = {m, I_z, l_f, l_r, c_af, c_ar}.  Writes N poses (x, y, psi).
 */
static void vehicle_trajectory(double x0, double y0, double psi0, double v0, double vdot, double delta,
                               const double *path, const double *params, int model, double tau, int n_steps,
                               int substeps, double *ox, double *oy, double *opsi, double *odelta) {
    const double m = params[0], Iz = params[1], lf = params[2], lr = params[3];
    const double caf = params[4], car = params[5];
    const double L = lf + lr;
    const double tau_i = tau / substeps;
    double x = x0, y = y0, psi = psi0;
    double beta = 0.0, r = 0.0;           /* sideslip angle, yaw rate */
    double ax = vdot, ay = 0.0;           /* vehicle-frame accelerations, reading R-b */
    int stopped = 0;
    long n_total = (long)n_steps * substeps;
    if (path) delta = 0.0;                /* reading R-u: delta_{-1} = 0 */
    for (long n = 0; n < n_total; ++n) {
        if (!stopped) {
            double v = speed_at(v0, vdot, tau_i, n);
            double v_next = speed_at(v0, vdot, tau_i, n + 1);
            double betadot, rdot;
            if (path) delta = path_steering(path, n, tau_i, x, y, psi, beta, v, delta);
            if (model == ORC_MODEL_KIN || v < ORC_V_MIN) {
                /* kinematic single-track limit, reading R-e */
                beta = atan(lr * tan(delta) / L);
                r = v * cos(beta) * tan(delta) / L;
                betadot = 0.0;
                rdot = 0.0;
            } else {
                /* Eq. (onetrack): [betadot; psiddot] = A [beta; psidot] + b delta */
                double a11 = -(caf + car) / (m * v);
                double a12 = (car * lr - caf * lf) / (m * v * v) - 1.0;
                double a21 = (car * lr - caf * lf) / Iz;
                double a22 = -(caf * lf * lf + car * lr * lr) / (Iz * v);
                double b1 = caf / (m * v);
                double b2 = caf * lf / Iz;
                betadot = a11 * beta + a12 * r + b1 * delta;
                rdot = a21 * beta + a22 * r + b2 * delta;
            }
            if (v_next < 0.0) {
                /* reading R-f: exact stopping distance along the course */
                double d = v * v / (2.0 * fabs(vdot));
                x += cos(psi + beta) * d;
                y += sin(psi + beta) * d;
                stopped = 1;
            } else {
                /* Eq. (EulerVelocity), position with the accelerations of step n */
                double xn = x + cos(psi + beta) * v * tau_i
                              + cos(psi) * ax * tau_i * tau_i / 2.0
                              - sin(psi) * ay * tau_i * tau_i / 2.0;
                double yn = y + sin(psi + beta) * v * tau_i
                              + sin(psi) * ax * tau_i * tau_i / 2.0
                              + cos(psi) * ay * tau_i * tau_i / 2.0;
                double ax_n = cos(beta) * vdot - sin(beta) * v * (betadot + r);
                double ay_n = sin(beta) * vdot + cos(beta) * v * (betadot + r);
                double psi_n = psi + r * tau_i + rdot * tau_i * tau_i / 2.0;
                double beta_n = beta + betadot * tau_i;
                double r_n = r + rdot * tau_i;          /* reading R-a */
                x = xn; y = yn; psi = psi_n; beta = beta_n; r = r_n; ax = ax_n; ay = ay_n;
            }
        }
        if (odelta) odelta[n] = delta;
        if ((n + 1) % substeps == 0) {
            long k = (n + 1) / substeps - 1;
            ox[k] = x; oy[k] = y; opsi[k] = psi;
        }
    }
}

/*
 * One pedestrian hypothesis, Eq. (pedestrianmotion): x_{n+1} = x_n + (c, s)(psi_P) (v_n tau + vdot tau^2/2),
 * with the speed saturation of reading R-g.
 */
static void pedestrian_trajectory(double x0, double y0, double heading, double v_start, double vdot,
                                  double v_max, double tau, int n_steps, int substeps,
                                  double *ox, double *oy, double *opsi) {
    const double tau_i = tau / substeps;
    double x = x0, y = y0, v = v_start;
    long n_total = (long)n_steps * substeps;
    for (long n = 0; n < n_total; ++n) {
        double s;
        if (vdot > 0.0 && v_max > 0.0 && v >= v_max) {
            s = v * tau_i;                                   /* already at or above the cap */
        } else if (vdot > 0.0 && v_max > 0.0 && v + vdot * tau_i > v_max) {
            double t1 = (v_max - v) / vdot;                  /* reaches the cap inside the sub-step */
            s = v * t1 + vdot * t1 * t1 / 2.0 + v_max * (tau_i - t1);
            v = v_max;
        } else if (vdot < 0.0 && v + vdot * tau_i < 0.0) {
            s = v * v / (2.0 * (-vdot));                     /* comes to rest inside the sub-step */
            v = 0.0;
        } else {
            s = v * tau_i + vdot * tau_i * tau_i / 2.0;
            v = v + vdot * tau_i;
        }
        x += cos(heading) * s;
        y += sin(heading) * s;
        if ((n + 1) % substeps == 0) {
            long k = (n + 1) / substeps - 1;
            ox[k] = x; oy[k] = y; opsi[k] = heading;
        }
    }
}

/* Paths of the objects (set by orc_set_paths; none by default): object o with path_off[o] >= 0 follows
   path i_b at paths[9 (path_off[o] + i_b) ..], three sections of (x, y, psi) each (reading R-s). */
static int g_path_n = 0;
static const long *g_path_off = 0;
static const double *g_path_v = 0;

int orc_set_paths(int n_obj, const long *path_off, const double *paths) {
    g_path_n = n_obj; g_path_off = path_off; g_path_v = paths;
    return 0;
}

static const double *object_path(int o, int ib) {
    if (!g_path_off || o >= g_path_n || g_path_off[o] < 0) return 0;
    return g_path_v + 9 * (g_path_off[o] + ib);
}

/* The steering angle of every sub-step of one path hypothesis (test access to readings R-t, R-u). */
int orc_path_steering(double x0, double y0, double psi0, double v0, double vdot, const double *path,
                      const double *params, int model, double tau, int n_steps, int substeps,
                      double *out_x, double *out_y, double *out_psi, double *out_delta) {
    vehicle_trajectory(x0, y0, psi0, v0, vdot, 0.0, path, params, model, tau, n_steps, substeps,
                       out_x, out_y, out_psi, out_delta);
    return 0;
}

/*
 * Generate every hypothesis of every object.  Inputs are flat per-object arrays; grids are concatenated
 * (grid_a of object o at grid_off[o], then its grid_b).  Hypothesis h of object o uses
 * grid_a[h / n_b] and grid_b[h % n_b].  Output pose of trajectory t (global index traj_off[o] + h) at
 * step k is at index t * n_steps + k.  params: 6 doubles per object (vehicles).  Returns 0.
 */
int orc_generate(int n_obj, const int *kind, const double *x0, const double *y0, const double *psi0,
                 const double *v0, const int *n_a, const int *n_b, const long *grid_off,
                 const double *grids, const double *params, const double *v_max, const int *flags,
                 double tau, int n_steps, int substeps, int model,
                 double *out_x, double *out_y, double *out_psi) {
    long t = 0;
    for (int o = 0; o < n_obj; ++o) {
        const double *ga = grids + grid_off[o];
        const double *gb = ga + n_a[o];
        for (int ia = 0; ia < n_a[o]; ++ia) {
            for (int ib = 0; ib < n_b[o]; ++ib, ++t) {
                double *ox = out_x + t * n_steps, *oy = out_y + t * n_steps, *op = out_psi + t * n_steps;
                if (kind[o] == ORC_VEHICLE) {
                    const double *path = object_path(o, ib);
                    vehicle_trajectory(x0[o], y0[o], psi0[o], v0[o], ga[ia], gb[ib], path, params + 6 * o, model,
                                       tau, n_steps, substeps, ox, oy, op, NULL);
                } else {
                    double heading = psi0[o] + gb[ib];
                    double v_start = (flags[o] & ORC_PED_ACCEL_GRID) ? v0[o] : ga[ia];
                    double vdot = (flags[o] & ORC_PED_ACCEL_GRID) ? ga[ia] : 0.0;
                    pedestrian_trajectory(x0[o], y0[o], heading, v_start, vdot, v_max[o], tau, n_steps,
                                          substeps, ox, oy, op);
                }
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------------------------------
 * Collision recognition (Section IV-C): exact overlap of closed rectangles / discs, reading R-h
 * ------------------------------------------------------------------------------------------------ */

typedef struct {
    int kind;            /* 0 rectangle, 1 disc, 2 convex polygon */
    double hl, hw, rad;  /* half length, half width, radius */
    double x, y, c, s;   /* centre, body axis (c, s) */
    int nv;              /* polygon: vertex count and body-frame vertices (x along the body axis) */
    const double *pv;
} shape;

#define MAX_VERTICES 16

/* World vertices of a rectangle (its four corners) or polygon; returns their number. */
static int world_vertices(const shape *p, double *wx, double *wy);

static double dot2(double ax, double ay, double bx, double by) { return ax * bx + ay * by; }

static void corners(const shape *p, double cx[4], double cy[4]) {
    /* body axis u = (c, s), lateral axis w = (-s, c) */
    double ux = p->c, uy = p->s, wx = -p->s, wy = p->c;
    double sl[4] = {1, 1, -1, -1}, sw[4] = {1, -1, -1, 1};
    for (int q = 0; q < 4; ++q) {
        cx[q] = p->x + sl[q] * p->hl * ux + sw[q] * p->hw * wx;
        cy[q] = p->y + sl[q] * p->hl * uy + sw[q] * p->hw * wy;
    }
}

/* Half extent of rectangle p projected on direction (nx, ny). */
static double support(const shape *p, double nx, double ny) {
    return p->hl * fabs(dot2(p->c, p->s, nx, ny)) + p->hw * fabs(dot2(-p->s, p->c, nx, ny));
}

/* Largest separation gap over the four edge normals (separating-axis theorem for two rectangles).
   <= 0 iff the closed rectangles intersect; then it equals minus the penetration depth. */
static double rect_rect_gap(const shape *a, const shape *b) {
    double axes[4][2] = {{a->c, a->s}, {-a->s, a->c}, {b->c, b->s}, {-b->s, b->c}};
    double dx = b->x - a->x, dy = b->y - a->y;
    double best = -INFINITY;
    for (int q = 0; q < 4; ++q) {
        double nx = axes[q][0], ny = axes[q][1];
        double len = sqrt(nx * nx + ny * ny);
        double gap = (fabs(dot2(dx, dy, nx, ny)) - support(a, nx, ny) - support(b, nx, ny)) / len;
        if (gap > best) best = gap;
    }
    return best;
}

static double point_segment_dist(double px, double py, double ax, double ay, double bx, double by) {
    double ex = bx - ax, ey = by - ay;
    double len2 = ex * ex + ey * ey;
    double t = len2 > 0.0 ? dot2(px - ax, py - ay, ex, ey) / len2 : 0.0;
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    double qx = ax + t * ex - px, qy = ay + t * ey - py;
    return sqrt(qx * qx + qy * qy);
}

/* Euclidean distance between two disjoint convex polygons: smallest vertex-to-edge distance, both ways. */
static double rect_rect_distance(const shape *a, const shape *b) {
    double ax[4], ay[4], bx[4], by[4];
    corners(a, ax, ay);
    corners(b, bx, by);
    double best = INFINITY;
    for (int i = 0; i < 4; ++i) {
        for (int e = 0; e < 4; ++e) {
            int f = (e + 1) % 4;
            double d1 = point_segment_dist(ax[i], ay[i], bx[e], by[e], bx[f], by[f]);
            double d2 = point_segment_dist(bx[i], by[i], ax[e], ay[e], ax[f], ay[f]);
            if (d1 < best) best = d1;
            if (d2 < best) best = d2;
        }
    }
    return best;
}

/* Signed margin of rectangle a and disc b (reading R-h). */
static double rect_disc_margin(const shape *a, const shape *b) {
    double dx = b->x - a->x, dy = b->y - a->y;
    double ulen = sqrt(a->c * a->c + a->s * a->s);
    double qx = dot2(dx, dy, a->c, a->s) / ulen;         /* disc centre in the rectangle's frame */
    double qy = dot2(dx, dy, -a->s, a->c) / ulen;
    double ex = fabs(qx) - a->hl * ulen, ey = fabs(qy) - a->hw * ulen;  /* extents of the drawn rectangle */
    if (ex <= 0.0 && ey <= 0.0) {
        /* centre inside: penetration = radius + distance from the centre to the boundary */
        return (ex > ey ? ex : ey) - b->rad;
    }
    double mx = ex > 0.0 ? ex : 0.0, my = ey > 0.0 ? ey : 0.0;
    return sqrt(mx * mx + my * my) - b->rad;
}

static double disc_disc_margin(const shape *a, const shape *b) {
    double dx = b->x - a->x, dy = b->y - a->y;
    return sqrt(dx * dx + dy * dy) - a->rad - b->rad;
}

static int world_vertices(const shape *p, double *wx, double *wy) {
    if (p->kind == 0) {
        corners(p, wx, wy);
        return 4;
    }
    for (int q = 0; q < p->nv; ++q) {
        double vx = p->pv[2 * q], vy = p->pv[2 * q + 1];
        wx[q] = p->x + p->c * vx - p->s * vy;
        wy[q] = p->y + p->s * vx + p->c * vy;
    }
    return p->nv;
}

/* Separating-axis gap of two convex polygons (or rectangles): the largest separation between their
   projections over all edge normals of both.  <= 0 iff the closed polygons intersect. */
static double poly_poly_gap(const shape *a, const shape *b) {
    double ax[MAX_VERTICES], ay[MAX_VERTICES], bx[MAX_VERTICES], by[MAX_VERTICES];
    int na = world_vertices(a, ax, ay), nb = world_vertices(b, bx, by);
    double best = -INFINITY;
    for (int side = 0; side < 2; ++side) {
        const double *px = side ? bx : ax, *py = side ? by : ay;
        int n = side ? nb : na;
        for (int e = 0; e < n; ++e) {
            int f = (e + 1) % n;
            double nx = -(py[f] - py[e]), ny = px[f] - px[e];
            double len = sqrt(nx * nx + ny * ny);
            nx /= len; ny /= len;
            double amin = INFINITY, amax = -INFINITY, bmin = INFINITY, bmax = -INFINITY;
            for (int q = 0; q < na; ++q) { double t = dot2(ax[q], ay[q], nx, ny); amin = fmin(amin, t); amax = fmax(amax, t); }
            for (int q = 0; q < nb; ++q) { double t = dot2(bx[q], by[q], nx, ny); bmin = fmin(bmin, t); bmax = fmax(bmax, t); }
            double gap = fmax(bmin - amax, amin - bmax);
            if (gap > best) best = gap;
        }
    }
    return best;
}

/* Euclidean distance of two disjoint convex polygons: the smallest vertex-to-edge distance, both ways. */
static double poly_poly_distance(const shape *a, const shape *b) {
    double ax[MAX_VERTICES], ay[MAX_VERTICES], bx[MAX_VERTICES], by[MAX_VERTICES];
    int na = world_vertices(a, ax, ay), nb = world_vertices(b, bx, by);
    double best = INFINITY;
    for (int i = 0; i < na; ++i)
        for (int e = 0; e < nb; ++e) {
            double d = point_segment_dist(ax[i], ay[i], bx[e], by[e], bx[(e + 1) % nb], by[(e + 1) % nb]);
            if (d < best) best = d;
        }
    for (int i = 0; i < nb; ++i)
        for (int e = 0; e < na; ++e) {
            double d = point_segment_dist(bx[i], by[i], ax[e], ay[e], ax[(e + 1) % na], ay[(e + 1) % na]);
            if (d < best) best = d;
        }
    return best;
}

/* Signed margin of convex polygon a and disc b: the centre's distance to the outline minus the radius,
   the distance counted negative when the centre lies inside. */
static double poly_disc_margin(const shape *a, const shape *b) {
    double ax[MAX_VERTICES], ay[MAX_VERTICES];
    int n = world_vertices(a, ax, ay);
    double dmin = INFINITY;
    int pos = 0, neg = 0;
    for (int e = 0; e < n; ++e) {
        int f = (e + 1) % n;
        double cr = (ax[f] - ax[e]) * (b->y - ay[e]) - (ay[f] - ay[e]) * (b->x - ax[e]);
        if (cr > 0.0) ++pos;
        if (cr < 0.0) ++neg;
        double d = point_segment_dist(b->x, b->y, ax[e], ay[e], ax[f], ay[f]);
        if (d < dmin) dmin = d;
    }
    int inside = pos == 0 || neg == 0;      /* on one side of every edge (or on the outline) */
    return (inside ? -dmin : dmin) - b->rad;
}

/* Exact signed separation margin: > 0 disjoint (Euclidean distance), <= 0 overlapping. */
static double shape_margin(const shape *a, const shape *b) {
    if (a->kind == 2 || b->kind == 2) {
        if (a->kind == 1) return poly_disc_margin(b, a);
        if (b->kind == 1) return poly_disc_margin(a, b);
        double g = poly_poly_gap(a, b);
        return g <= 0.0 ? g : poly_poly_distance(a, b);
    }
    if (a->kind == 0 && b->kind == 0) {
        double g = rect_rect_gap(a, b);
        return g <= 0.0 ? g : rect_rect_distance(a, b);
    }
    if (a->kind == 0) return rect_disc_margin(a, b);
    if (b->kind == 0) return rect_disc_margin(b, a);
    return disc_disc_margin(a, b);
}

/* Overlap flag (margin <= 0) without computing the full distance of disjoint rectangles. */
static int shape_overlap(const shape *a, const shape *b) {
    if (a->kind == 0 && b->kind == 0) return rect_rect_gap(a, b) <= 0.0;
    if ((a->kind == 2 && b->kind != 1) || (b->kind == 2 && a->kind != 1)) return poly_poly_gap(a, b) <= 0.0;
    return shape_margin(a, b) <= 0.0;
}

/* The paper's own test (Section IV-C.1): some vertex of one polygon lies in the other, both ways. */
static int point_in_rect(const shape *p, double qx, double qy) {
    double dx = qx - p->x, dy = qy - p->y;
    return fabs(dot2(dx, dy, p->c, p->s)) <= p->hl && fabs(dot2(dx, dy, -p->s, p->c)) <= p->hw;
}

static int rect_rect_pip(const shape *a, const shape *b) {
    double ax[4], ay[4], bx[4], by[4];
    corners(a, ax, ay);
    corners(b, bx, by);
    for (int q = 0; q < 4; ++q)
        if (point_in_rect(b, ax[q], ay[q]) || point_in_rect(a, bx[q], by[q])) return 1;
    return 0;
}

static shape make_shape(int kind, double length, double width, double radius,
                        double x, double y, double c, double s) {
    shape p;
    p.kind = kind; p.hl = length / 2.0; p.hw = width / 2.0; p.rad = radius;
    p.x = x; p.y = y; p.c = c; p.s = s;
    p.nv = 0; p.pv = 0;
    return p;
}

/* Polygon outlines of the objects (set by orc_set_polygons; none by default): object o with nv[o] > 0 has
   the convex outline verts[2 * off[o] ..] (body frame) and shape kind 2. */
static int g_poly_n = 0;
static const int *g_poly_nv = 0;
static const long *g_poly_off = 0;
static const double *g_poly_v = 0;

int orc_set_polygons(int n_obj, const int *nv, const long *off, const double *verts) {
    g_poly_n = n_obj; g_poly_nv = nv; g_poly_off = off; g_poly_v = verts;
    return 0;
}

/* The shape of object o (its polygon outline when one is set). */
static shape object_shape(int o, int kind, double length, double width, double radius,
                          double x, double y, double c, double s) {
    shape p = make_shape(kind, length, width, radius, x, y, c, s);
    if (g_poly_nv && o < g_poly_n && g_poly_nv[o] > 0) {
        p.kind = 2;
        p.nv = g_poly_nv[o];
        p.pv = g_poly_v + 2 * g_poly_off[o];
    }
    return p;
}

double orc_margin(int kind_a, double len_a, double wid_a, double rad_a, double xa, double ya, double ca, double sa,
                  int kind_b, double len_b, double wid_b, double rad_b, double xb, double yb, double cb, double sb) {
    shape a = make_shape(kind_a, len_a, wid_a, rad_a, xa, ya, ca, sa);
    shape b = make_shape(kind_b, len_b, wid_b, rad_b, xb, yb, cb, sb);
    return shape_margin(&a, &b);
}

/* Signed margin (and, *overlap, the closed overlap flag) of two shapes given directly: kind 0 rectangle
   (len, wid), 1 disc (rad), 2 convex polygon (nv body-frame vertices v[2 nv]). */
double orc_margin_shapes(int kind_a, double len_a, double wid_a, double rad_a, int nv_a, const double *va,
                         double xa, double ya, double ca, double sa,
                         int kind_b, double len_b, double wid_b, double rad_b, int nv_b, const double *vb,
                         double xb, double yb, double cb, double sb, int *overlap) {
    shape a = make_shape(kind_a, len_a, wid_a, rad_a, xa, ya, ca, sa);
    shape b = make_shape(kind_b, len_b, wid_b, rad_b, xb, yb, cb, sb);
    a.nv = nv_a; a.pv = va;
    b.nv = nv_b; b.pv = vb;
    if (overlap) *overlap = shape_overlap(&a, &b);
    return shape_margin(&a, &b);
}

int orc_overlap_pip(double len_a, double wid_a, double xa, double ya, double ca, double sa,
                    double len_b, double wid_b, double xb, double yb, double cb, double sb) {
    shape a = make_shape(0, len_a, wid_a, 0.0, xa, ya, ca, sa);
    shape b = make_shape(0, len_b, wid_b, 0.0, xb, yb, cb, sb);
    return rect_rect_pip(&a, &b);
}

/*
 * First-collision table of object pairs (Section IV-C, Eq. threads:coll enumerates the combinations).
 * Poses are given per trajectory t and step k at t * n_steps + k as (x, y, c, s).  For pair p = (a, b):
 * out[pair_off[p] + i * h_b + j] = min{k : overlap at step k} or -1.  Pairs may be listed in either
 * orientation.  Returns 0.
 */
int orc_table(int n_obj, const int *kind, const double *length, const double *width, const double *radius,
              const long *traj_off, int n_steps,
              const double *px, const double *py, const double *pc, const double *ps,
              int n_pairs, const int *pair_a, const int *pair_b, const long *pair_off, int16_t *out) {
    (void)n_obj;
    for (int p = 0; p < n_pairs; ++p) {
        int a = pair_a[p], b = pair_b[p];
        long ha = traj_off[a + 1] - traj_off[a], hb = traj_off[b + 1] - traj_off[b];
        for (long i = 0; i < ha; ++i) {
            for (long j = 0; j < hb; ++j) {
                long ta = traj_off[a] + i, tb = traj_off[b] + j;
                int first = -1;
                for (int k = 0; k < n_steps; ++k) {
                    long ia = ta * n_steps + k, ib = tb * n_steps + k;
                    shape sa = object_shape(a, kind[a], length[a], width[a], radius[a], px[ia], py[ia], pc[ia], ps[ia]);
                    shape sb = object_shape(b, kind[b], length[b], width[b], radius[b], px[ib], py[ib], pc[ib], ps[ib]);
                    if (shape_overlap(&sa, &sb)) { first = k; break; }
                }
                out[pair_off[p] + i * hb + j] = (int16_t)first;
            }
        }
    }
    return 0;
}

/* First-collision step of selected trajectory pairs (same definition as orc_table):
   out[q] for trajectories ta[q] (object oa[q]) and tb[q] (object ob[q]). */
int orc_first(const int *kind, const double *length, const double *width, const double *radius, int n_steps,
              const double *px, const double *py, const double *pc, const double *ps,
              long n_q, const int *oa, const long *ta, const int *ob, const long *tb, int16_t *out) {
    for (long q = 0; q < n_q; ++q) {
        int a = oa[q], b = ob[q], first = -1;
        for (int k = 0; k < n_steps; ++k) {
            long ia = ta[q] * n_steps + k, ib = tb[q] * n_steps + k;
            shape sa = object_shape(a, kind[a], length[a], width[a], radius[a], px[ia], py[ia], pc[ia], ps[ia]);
            shape sb = object_shape(b, kind[b], length[b], width[b], radius[b], px[ib], py[ib], pc[ib], ps[ib]);
            if (shape_overlap(&sa, &sb)) { first = k; break; }
        }
        out[q] = (int16_t)first;
    }
    return 0;
}

/* Per-step signed margins of selected trajectory pairs (for borderline accounting).
   For q < n_q: margins[q * n_steps + k] of trajectories ta[q], tb[q] (objects oa[q], ob[q]). */
int orc_margins(const int *kind, const double *length, const double *width, const double *radius, int n_steps,
                const double *px, const double *py, const double *pc, const double *ps,
                long n_q, const int *oa, const long *ta, const int *ob, const long *tb, double *margins) {
    for (long q = 0; q < n_q; ++q) {
        int a = oa[q], b = ob[q];
        for (int k = 0; k < n_steps; ++k) {
            long ia = ta[q] * n_steps + k, ib = tb[q] * n_steps + k;
            shape sa = object_shape(a, kind[a], length[a], width[a], radius[a], px[ia], py[ia], pc[ia], ps[ia]);
            shape sb = object_shape(b, kind[b], length[b], width[b], radius[b], px[ib], py[ib], pc[ib], ps[ib]);
            margins[q * n_steps + k] = shape_margin(&sa, &sb);
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------------------------------
 * Risk assessment (Section IV-D)
 * ------------------------------------------------------------------------------------------------ */

typedef struct { int k, b; long j; double p; } hit_entry;

static int hit_cmp(const void *x, const void *y) {
    const hit_entry *u = (const hit_entry *)x, *v = (const hit_entry *)y;
    if (u->k != v->k) return u->k < v->k ? -1 : 1;
    if (u->b != v->b) return u->b < v->b ? -1 : 1;
    if (u->j != v->j) return u->j < v->j ? -1 : 1;
    return 0;
}

/*
 * Risk measures from the first-collision tables.
 *  prob: per-trajectory probabilities (already L1-normalised per object, Section IV-D.1), global index.
 *  Per object pair p (Eq. totalCrashProb generalised to every pair):
 *     count[p] = #{T >= 0},  count_k[p*N+k] = #{T = k},
 *     P[p] = sum [T >= 0] p_a[i] p_b[j],  H[p*N+k] = sum [T = k] p_a[i] p_b[j].
 *  EGO object e (pairs that contain e, either orientation):
 *     naive[i] = sum_b sum_j [T >= 0] p_b[j]        (so p_cra = sum_i p_e[i] naive[i], Eq. totalCrashProb)
 *     cond[i]  = sum of eff over colliding entries in chronological order (Eq. p21, reading R-i):
 *                eff = S p_b[j], S <- S (1 - p_b[j]), S starting at 1
 *     indep[i] = 1 - prod_b (1 - sum_j [T >= 0] p_b[j])   (per-object independence)
 *     hits[i]  = number of colliding entries
 *     attr_obj[b] = sum_i p_e[i] sum_{entries of b} eff,  attr_step[k] = same per step
 *  scalars[0] = p_cra, scalars[1] = p_cra_cond = sum_i p_e[i] cond[i], scalars[2] = sum_i p_e[i] indep[i].
 *  escape: EGO trajectories with no colliding entry, by descending p_e, ties by ascending index;
 *  *n_escape receives their number.  Returns 0, or -2 if memory runs out.
 */
int orc_risk(int n_obj, const long *traj_off, int n_steps, int ego,
             int n_pairs, const int *pair_a, const int *pair_b, const long *pair_off, const int16_t *table,
             const double *prob,
             long *count, long *count_k, double *P, double *H,
             double *naive, double *cond, double *indep, int *hits, double *attr_obj, double *attr_step,
             double *scalars, int *escape, int *n_escape) {
    const int N = n_steps;
    for (int p = 0; p < n_pairs; ++p) {
        int a = pair_a[p], b = pair_b[p];
        long ha = traj_off[a + 1] - traj_off[a], hb = traj_off[b + 1] - traj_off[b];
        count[p] = 0; P[p] = 0.0;
        for (int k = 0; k < N; ++k) { count_k[(long)p * N + k] = 0; H[(long)p * N + k] = 0.0; }
        for (long i = 0; i < ha; ++i)
            for (long j = 0; j < hb; ++j) {
                int T = table[pair_off[p] + i * hb + j];
                if (T >= 0) {
                    double w = prob[traj_off[a] + i] * prob[traj_off[b] + j];
                    count[p] += 1;
                    count_k[(long)p * N + T] += 1;
                    P[p] += w;
                    H[(long)p * N + T] += w;
                }
            }
    }
    long he = traj_off[ego + 1] - traj_off[ego];
    for (int b = 0; b < n_obj; ++b) attr_obj[b] = 0.0;
    for (int k = 0; k < N; ++k) attr_step[k] = 0.0;
    double p_cra = 0.0, p_cond = 0.0, p_indep = 0.0;
    long cap = 0;
    for (int p = 0; p < n_pairs; ++p) {
        if (pair_a[p] == ego) cap += traj_off[pair_b[p] + 1] - traj_off[pair_b[p]];
        else if (pair_b[p] == ego) cap += traj_off[pair_a[p] + 1] - traj_off[pair_a[p]];
    }
    hit_entry *list = (hit_entry *)malloc(sizeof(hit_entry) * (size_t)(cap > 0 ? cap : 1));
    double *mass = (double *)malloc(sizeof(double) * (size_t)n_obj);
    if (!list || !mass) { free(list); free(mass); return -2; }
    for (long i = 0; i < he; ++i) {
        long n_hit = 0;
        for (int b = 0; b < n_obj; ++b) mass[b] = 0.0;
        for (int p = 0; p < n_pairs; ++p) {
            int a = pair_a[p], b = pair_b[p];
            if (a != ego && b != ego) continue;
            int co = (a == ego) ? b : a;
            long hco = traj_off[co + 1] - traj_off[co];
            long hb = traj_off[b + 1] - traj_off[b];
            for (long j = 0; j < hco; ++j) {
                /* T(e, i, co, j) read from whichever orientation the pair is stored in (symmetry) */
                long idx = (a == ego) ? pair_off[p] + i * hb + j : pair_off[p] + j * hb + i;
                int T = table[idx];
                if (T >= 0) {
                    hit_entry h;
                    h.k = T; h.b = co; h.j = j; h.p = prob[traj_off[co] + j];
                    list[n_hit++] = h;
                    mass[co] += h.p;
                }
            }
        }
        qsort(list, (size_t)n_hit, sizeof(hit_entry), hit_cmp);
        double S = 1.0, c = 0.0, nv = 0.0;
        double pe = prob[traj_off[ego] + i];
        for (long q = 0; q < n_hit; ++q) {
            double eff = S * list[q].p;
            S = S * (1.0 - list[q].p);
            c += eff;
            nv += list[q].p;
            attr_obj[list[q].b] += pe * eff;
            attr_step[list[q].k] += pe * eff;
        }
        double surv = 1.0;
        for (int b = 0; b < n_obj; ++b) surv *= (1.0 - mass[b]);
        naive[i] = nv;
        cond[i] = c;
        indep[i] = 1.0 - surv;
        hits[i] = (int)n_hit;
        p_cra += pe * nv;
        p_cond += pe * c;
        p_indep += pe * (1.0 - surv);
    }
    scalars[0] = p_cra;
    scalars[1] = p_cond;
    scalars[2] = p_indep;
    /* escape routes (Section VI-A): collision-free EGO trajectories ranked by probability */
    int ne = 0;
    for (long i = 0; i < he; ++i)
        if (hits[i] == 0) escape[ne++] = (int)i;
    for (int u = 1; u < ne; ++u) {               /* insertion sort: descending p, ascending index */
        int cur = escape[u];
        double pc = prob[traj_off[ego] + cur];
        int v = u - 1;
        while (v >= 0) {
            double pv = prob[traj_off[ego] + escape[v]];
            if (pv < pc || (pv == pc && escape[v] > cur)) { escape[v + 1] = escape[v]; --v; }
            else break;
        }
        escape[v + 1] = cur;
    }
    *n_escape = ne;
    free(list);
    free(mass);
    return 0;
}

/* Eq. (normTraj) with the factors of reading R-x: the score of every hypothesis of every object, in
   the generation's order (hypothesis h of object o at traj index traj_off[o] + h uses grid_a[h / n_b] and
   grid_b[h % n_b], or path h % n_b).  Inputs as orc_generate; paths as registered by orc_set_paths. */
int orc_scores(int n_obj, const int *kind, const double *x0, const double *y0, const double *psi0,
               const double *v0, const int *n_a, const int *n_b, const long *grid_off, const double *grids,
               const int *flags, double *out) {
    const double w_acc = 0.5, w_str = 0.5;
    long t = 0;
    for (int o = 0; o < n_obj; ++o) {
        const double *ga = grids + grid_off[o];
        const double *gb = ga + n_a[o];
        for (int ia = 0; ia < n_a[o]; ++ia) {
            for (int ib = 0; ib < n_b[o]; ++ib, ++t) {
                double n_acc, d_str, c_com = 1.0, c_cou = 1.0;
                if (kind[o] == ORC_VEHICLE) {
                    n_acc = 1.0 / (1.0 + fabs(ga[ia]) / 2.0);
                    const double *path = object_path(o, ib);
                    if (!path) {
                        d_str = 1.0 / (1.0 + fabs(gb[ib]) / 0.05);
                    } else {
                        double off[3], nx = -sin(psi0[o]), ny = cos(psi0[o]), o_abs = 0.0, o_max = -INFINITY;
                        for (int k = 0; k < 3; ++k) {
                            off[k] = (path[3 * k] - x0[o]) * nx + (path[3 * k + 1] - y0[o]) * ny;
                            o_abs = fmax(o_abs, fabs(off[k]));
                            o_max = fmax(o_max, off[k]);
                        }
                        d_str = 1.0 / (1.0 + o_abs / 1.75);
                        c_com = 1.0 + (fabs(off[1] - off[0]) + fabs(off[2] - off[1])) / 3.5;
                        c_cou = o_max > 1.75 ? 2.0 : 1.0;
                    }
                } else {
                    n_acc = (flags[o] & ORC_PED_ACCEL_GRID) ? 1.0 / (1.0 + fabs(ga[ia]) / 2.0)
                                                            : 1.0 / (1.0 + fabs(ga[ia] - v0[o]) / 1.0);
                    d_str = 1.0 / (1.0 + fabs(gb[ib]) / 0.5);
                }
                out[t] = (w_acc * n_acc + w_str * d_str) / (c_com * c_cou);
            }
        }
    }
    return 0;
}

/* L1 normalisation of non-negative trajectory weights, per object (Section IV-D.1). -1 if invalid. */
int orc_normalise(int n_obj, const long *traj_off, const double *w, double *prob) {
    for (int o = 0; o < n_obj; ++o) {
        double s = 0.0;
        for (long t = traj_off[o]; t < traj_off[o + 1]; ++t) {
            if (!(w[t] >= 0.0)) return -1;
            s += fabs(w[t]);
        }
        if (!(s > 0.0)) return -1;
        for (long t = traj_off[o]; t < traj_off[o + 1]; ++t) prob[t] = w[t] / s;
    }
    return 0;
}
