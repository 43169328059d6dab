// lanes.cu -- street data processing (Section IV-A) and the controller's paths (Section IV-B.2b), on the
// host: a handful of dividers per vehicle (the paper runs this step on at most four threads), whose
// output feeds mhc_object.paths.
//
// Divider j of a vehicle is the second-degree curve y = a x^2 + b x + c (vehicle frame at t = 0: x ahead,
// y to the left) through its three measured points, solved by Gauss-Jordan elimination with partial
// pivoting.  The vehicle's lane is the pair of adjacent dividers enclosing its position; at each sampling
// instant t (1.0, 1.5, 2.0 s) the reference position is x_t = v0 t, the own lane is sampled at 1/4, 1/2
// and 3/4 of its width and each neighbour present at 1/3 and 2/3 (right to left), and a section passes
// through each sample along the lane's centre-line direction there.  A CO follows one path per sample
// index, the EGO every combination.
#include <cmath>
#include <cstring>

#include "runtime.h"

namespace {

// y = c[0] x^2 + c[1] x + c[2] through (x_r, y_r), r = 0..2; false when the abscissae fix no such curve
bool fit_divider(const float *pts, double c[3]) {
    double m[3][4];
    for (int r = 0; r < 3; ++r) {
        const double x = pts[2 * r], y = pts[2 * r + 1];
        m[r][0] = x * x;
        m[r][1] = x;
        m[r][2] = 1.0;
        m[r][3] = y;
    }
    for (int col = 0; col < 3; ++col) {
        int piv = col;
        for (int r = col + 1; r < 3; ++r)
            if (std::fabs(m[r][col]) > std::fabs(m[piv][col])) piv = r;
        if (!(std::fabs(m[piv][col]) > 1e-12)) return false;
        if (piv != col)
            for (int q = 0; q < 4; ++q) std::swap(m[col][q], m[piv][q]);
        const double d = m[col][col];
        for (int q = 0; q < 4; ++q) m[col][q] /= d;
        for (int r = 0; r < 3; ++r) {
            if (r == col) continue;
            const double f = m[r][col];
            for (int q = 0; q < 4; ++q) m[r][q] -= f * m[col][q];
        }
    }
    for (int q = 0; q < 3; ++q) c[q] = m[q][3];
    return true;
}

}  // namespace

extern "C" int mhc_lane_paths(const float *dividers, int32_t n_dividers, float x0, float y0, float psi0, float v0,
                              int32_t ego, float *paths, int32_t *n_paths) {
    using mhc::host::fail;
    if (!dividers || !n_paths) return fail(MHC_E_INVALID, "dividers and n_paths must be non-NULL");
    if (n_dividers < 2 || n_dividers > 4) return fail(MHC_E_INVALID, "n_dividers must be in [2, 4]");
    for (int q = 0; q < 6 * n_dividers; ++q)
        if (!std::isfinite(dividers[q])) return fail(MHC_E_INVALID, "divider points must be finite");
    if (!std::isfinite(x0) || !std::isfinite(y0) || !std::isfinite(psi0) || !std::isfinite(v0) || v0 < 0.f)
        return fail(MHC_E_INVALID, "the vehicle state must be finite with v0 >= 0");
    double cf[4][3];
    for (int j = 0; j < n_dividers; ++j)
        if (!fit_divider(dividers + 6 * j, cf[j])) return fail(MHC_E_INVALID, "a divider's points fix no curve");
    int own = -1;
    for (int j = 0; j + 1 < n_dividers && own < 0; ++j)
        if (cf[j][2] <= 0.0 && 0.0 <= cf[j + 1][2]) own = j;
    if (own < 0) return fail(MHC_E_INVALID, "no lane encloses the vehicle");
    static const double kTimes[3] = {1.0, 1.5, 2.0};
    double lat[3][7], dir[3][7];
    int m = 0;
    for (int k = 0; k < 3; ++k) {
        const double x = (double)v0 * kTimes[k];
        int q = 0;
        for (int lane = own - 1; lane <= own + 1; ++lane) {      // right neighbour, own lane, left neighbour
            if (lane < 0 || lane + 1 >= n_dividers) continue;
            const double *r = cf[lane], *l = cf[lane + 1];
            const double yr = (r[0] * x + r[1]) * x + r[2], yl = (l[0] * x + l[1]) * x + l[2];
            const double heading = std::atan(((2.0 * r[0] * x + r[1]) + (2.0 * l[0] * x + l[1])) / 2.0);
            const int n = lane == own ? 3 : 2;
            for (int u = 1; u <= n; ++u, ++q) {
                lat[k][q] = yr + (yl - yr) * u / (n + 1);
                dir[k][q] = heading;
            }
        }
        m = q;
    }
    const int count = ego ? m * m * m : m;
    *n_paths = count;
    if (!paths) return MHC_OK;                                   // the count only
    const double c = std::cos((double)psi0), s = std::sin((double)psi0);
    for (int p = 0; p < count; ++p) {
        const int idx[3] = {ego ? p / (m * m) : p, ego ? (p / m) % m : p, ego ? p % m : p};
        for (int k = 0; k < 3; ++k) {
            const double bx = (double)v0 * kTimes[k], by = lat[k][idx[k]];
            float *o = paths + 9 * p + 3 * k;
            o[0] = (float)((double)x0 + c * bx - s * by);
            o[1] = (float)((double)y0 + s * bx + c * by);
            o[2] = (float)((double)psi0 + dir[k][idx[k]]);
        }
    }
    return MHC_OK;
}
