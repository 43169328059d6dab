// api.cu -- host runtime behind the C ABI of mhc.h: scenario validation and layout, the context arena,
// descriptor upload through a ring of mapped pinned staging buffers (read by a copy kernel), and the launch
// sequence of each entry point.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "runtime.h"
#include "prepare.cuh"

using namespace mhc;
using namespace mhc::host;

namespace {
thread_local std::string g_err;
}  // namespace

namespace mhc {
namespace host {

int fail(int code, const std::string &why) {
    g_err = why;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    return fail(MHC_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Speed regimes of a vehicle hypothesis with acceleration acc (Eq. EulerVelocity, readings of the low-speed
// limit and the stop rule): the first sub-steps at which the FP64 speed v_0 + n vdot tau_i reaches or leaves
// 2 m/s and at which the next speed turns negative.  Each predicate is monotone in n; the search starts at
// the real-valued crossing and steps to the exact first sub-step, evaluating the predicate itself, so the
// decision is the FP64 one a full search would take.
Regime speed_regime(float v0f, float acc, int model, int NK, double tau_i_d) {
    const double dv = (double)acc * tau_i_d;
    const double v0 = (double)v0f;
    auto speed = [&](int n) { return v0 + (double)n * dv; };
    auto first = [&](auto pred, double guess) {   // smallest n in [0, NK) with pred(n), NK if none
        int n = !(guess > 0.0) ? 0 : (guess >= (double)NK ? NK : (int)std::ceil(guess));
        while (n > 0 && pred(n - 1)) --n;
        while (n < NK && !pred(n)) ++n;
        return n;
    };
    Regime g{0, 0, NK, 0};
    if (model == MHC_MODEL_KIN) {
        g.low_hi = NK;
    } else if (acc > 0.0f) {
        g.low_hi = first([&](int n) { return speed(n) >= kVMinD; }, (kVMinD - v0) / dv);
    } else if (acc < 0.0f) {
        g.low_lo = first([&](int n) { return speed(n) < kVMinD; }, (kVMinD - v0) / dv);
        g.low_hi = NK;
    } else if (v0 < kVMinD) {
        g.low_hi = NK;
    }
    if (acc < 0.0f) g.n_stop = first([&](int n) { return speed(n + 1) < 0.0; }, -v0 / dv - 1.0);
    return g;
}

// Validates the convex outline of a vehicle (Section IV-C.1: any outline detail) and appends it to `out`
// counter-clockwise with the outward unit normal of each edge; `circ` receives its circumradius about the
// pose point.  Returns an empty string, or the reason it is rejected.
std::string append_outline(const float *v, int n, std::vector<PolyVertex> &out, float &circ) {
    if (n < 3 || n > MHC_MAX_VERTICES) return "n_vertices must be 0 or in [3, 16]";
    if (!v) return "vertices is NULL";
    double x[MHC_MAX_VERTICES], y[MHC_MAX_VERTICES];
    for (int q = 0; q < n; ++q) {
        if (!finite(v[2 * q]) || !finite(v[2 * q + 1])) return "outline vertices must be finite";
        x[q] = v[2 * q];
        y[q] = v[2 * q + 1];
    }
    double area2 = 0.0;
    for (int q = 0; q < n; ++q) area2 += x[q] * y[(q + 1) % n] - x[(q + 1) % n] * y[q];
    if (!(std::fabs(area2) > 0.0)) return "outline has no area";
    if (area2 < 0.0)   // clockwise: reverse
        for (int q = 0; q < n / 2; ++q) { std::swap(x[q], x[n - 1 - q]); std::swap(y[q], y[n - 1 - q]); }
    double turn = 0.0, r2 = 0.0;
    for (int q = 0; q < n; ++q) {
        const int q1 = (q + 1) % n, q2 = (q + 2) % n;
        const double ex = x[q1] - x[q], ey = y[q1] - y[q], fx = x[q2] - x[q1], fy = y[q2] - y[q1];
        const double le = std::hypot(ex, ey), lf = std::hypot(fx, fy);
        if (!(le > 1e-6) || !(lf > 1e-6)) return "outline has repeated vertices";
        const double cr = ex * fy - ey * fx;
        if (!(cr > 1e-9 * le * lf)) return "outline is not strictly convex";
        turn += std::atan2(cr, ex * fx + ey * fy);
        r2 = std::max(r2, x[q] * x[q] + y[q] * y[q]);
    }
    if (std::fabs(turn - 6.283185307179586) > 1e-6) return "outline is not simple (it winds more than once)";
    for (int q = 0; q < n; ++q) {
        const int q1 = (q + 1) % n;
        const double ex = x[q1] - x[q], ey = y[q1] - y[q], le = std::hypot(ex, ey);
        out.push_back(make_float4((float)x[q], (float)y[q], (float)(ey / le), (float)(-ex / le)));
    }
    circ = (float)std::sqrt(r2);
    return std::string();
}

// The rectangle of half extents hl x hw as a counter-clockwise 4-gon (for pairs with an outline).
void append_rectangle(float hl, float hw, std::vector<PolyVertex> &out) {
    out.push_back(make_float4(hl, -hw, 1.f, 0.f));
    out.push_back(make_float4(hl, hw, 0.f, 1.f));
    out.push_back(make_float4(-hl, hw, -1.f, 0.f));
    out.push_back(make_float4(-hl, -hw, 0.f, -1.f));
}

// Validates scenario `si` and appends it to the layout.
int append_scenario(const mhc_scenario *sc, int si, bool batch, Layout &L) {
    char sw[48] = "";
    if (batch) std::snprintf(sw, sizeof sw, "scenario %d: ", si);
    const std::string pre(sw);
    if (sc->n_objects < 1 || sc->n_objects > MHC_MAX_OBJECTS || !sc->objects)
        return fail(MHC_E_INVALID, pre + "n_objects must be in [1, 4096] with a non-NULL objects array");
    if (sc->n_steps < 1 || sc->n_steps > MHC_MAX_STEPS) return fail(MHC_E_INVALID, pre + "n_steps must be in [1, 32767]");
    if (sc->substeps < 1 || (long long)sc->n_steps * sc->substeps >= (1LL << 31))
        return fail(MHC_E_INVALID, pre + "substeps must be >= 1 with n_steps * substeps < 2^31");
    if (!(sc->tau > 0.f) || !finite(sc->tau)) return fail(MHC_E_INVALID, pre + "tau must be positive and finite");
    if (sc->pair_mode != MHC_ALL_PAIRS && sc->pair_mode != MHC_EGO_ONLY) return fail(MHC_E_INVALID, pre + "bad pair_mode");
    if (sc->ego < 0 || sc->ego >= sc->n_objects) return fail(MHC_E_INVALID, pre + "ego out of range");
    if (sc->model != MHC_MODEL_OT && sc->model != MHC_MODEL_KIN) return fail(MHC_E_INVALID, pre + "bad model");
    if (sc->pair_mode == MHC_EGO_ONLY && sc->n_objects < 2) return fail(MHC_E_INVALID, pre + "EGO_ONLY needs 2 objects");
    const int N = sc->n_steps, obj0 = L.n_obj, n_obj_s = sc->n_objects;
    if (L.n_obj + n_obj_s > (1 << 24)) return fail(MHC_E_INVALID, "too many objects in the batch");
    if (N > L.max_steps) L.max_steps = N;
    static const float kDefault[6] = {1500.f, 2500.f, 1.2f, 1.5f, 80000.f, 80000.f};
    // a scenario with any convex outline lists every vehicle's outline (rectangles as 4-gons)
    bool any_outline = false;
    for (int o = 0; o < n_obj_s; ++o) any_outline |= sc->objects[o].n_vertices != 0;
    std::vector<char> outline(n_obj_s, 0);
    for (int o = 0; o < n_obj_s; ++o) {
        const mhc_object &src = sc->objects[o];
        ObjDesc d;
        std::memset(&d, 0, sizeof d);
        auto where = [&]() {   // the message prefix, formatted only on a failure
            char w[80];
            std::snprintf(w, sizeof w, "%sobject %d: ", pre.c_str(), o);
            return std::string(w);
        };
        if (src.kind != MHC_VEHICLE && src.kind != MHC_PEDESTRIAN) return fail(MHC_E_INVALID, where() + "bad kind");
        if (src.n_a < 1 || src.n_b < 1 || !src.grid_a || !src.grid_b)
            return fail(MHC_E_INVALID, where() + "grids must be non-empty and non-NULL");
        if ((long long)src.n_a * src.n_b > (1LL << 30)) return fail(MHC_E_INVALID, where() + "too many hypotheses");
        if (!finite(src.x0) || !finite(src.y0) || !finite(src.psi0) || !finite(src.v0) || !(src.v0 >= 0.f))
            return fail(MHC_E_INVALID, where() + "initial state must be finite with v0 >= 0");
        if (L.grids.size() + (size_t)src.n_a + src.n_b > (size_t)0x7fffffff)
            return fail(MHC_E_INVALID, where() + "grids too large");
        d.kind = src.kind; d.flags = src.flags; d.n_a = src.n_a; d.n_b = src.n_b; d.h = src.n_a * src.n_b;
        d.grid_off = (int)L.grids.size();
        for (int q = 0; q < src.n_a; ++q) {
            if (!finite(src.grid_a[q])) return fail(MHC_E_INVALID, where() + "grid_a not finite");
            if (src.kind == MHC_PEDESTRIAN && !(src.flags & MHC_PED_ACCEL_GRID) && src.grid_a[q] < 0.f)
                return fail(MHC_E_INVALID, where() + "pedestrian speeds must be >= 0");
            L.grids.push_back(src.grid_a[q]);
        }
        for (int q = 0; q < src.n_b; ++q) {
            if (!finite(src.grid_b[q])) return fail(MHC_E_INVALID, where() + "grid_b not finite");
            L.grids.push_back(src.grid_b[q]);
        }
        d.traj_off = L.n_traj;
        d.pose_base = L.n_pose;
        L.n_traj += d.h;
        L.n_pose += (long long)d.h * N;
        d.tile_base = L.n_tiles32;
        d.n_tiles32 = (d.h + kBoundTile - 1) / kBoundTile;
        if ((long long)L.n_tiles32 + d.n_tiles32 > 0x7fffffffLL) return fail(MHC_E_INVALID, "too many hypotheses in the batch");
        L.n_tiles32 += d.n_tiles32;
        d.bounds_base = L.n_bounds;
        L.n_bounds += (long long)d.n_tiles32 * N;
        d.x0 = src.x0; d.y0 = src.y0; d.psi0 = src.psi0; d.v0 = src.v0; d.v_max = src.v_max;
        if (src.kind == MHC_VEHICLE) {
            if (!(src.length > 0.f) || !(src.width > 0.f) || !finite(src.length) || !finite(src.width))
                return fail(MHC_E_INVALID, where() + "vehicle needs positive length and width");
            const float *pp = src.veh_params ? src.veh_params : kDefault;
            for (int q = 0; q < 6; ++q)
                if (!(pp[q] > 0.f) || !finite(pp[q])) return fail(MHC_E_INVALID, where() + "vehicle parameters must be positive");
            d.m = pp[0]; d.Iz = pp[1]; d.lf = pp[2]; d.lr = pp[3]; d.caf = pp[4]; d.car = pp[5];
            d.hl = 0.5f * src.length; d.hw = 0.5f * src.width; d.rad = 0.f;
            d.circ = (float)std::sqrt((double)d.hl * d.hl + (double)d.hw * d.hw);
            if (any_outline) {
                d.poly_off = (int)L.polys.size();
                if (src.n_vertices != 0) {
                    const std::string why = append_outline(src.vertices, src.n_vertices, L.polys, d.circ);
                    if (!why.empty()) return fail(MHC_E_INVALID, where() + why);
                    outline[o] = 1;
                } else {
                    append_rectangle(d.hl, d.hw, L.polys);
                }
                d.n_poly = (int)L.polys.size() - d.poly_off;
            }
        } else {
            if (src.n_vertices != 0) return fail(MHC_E_INVALID, where() + "pedestrians take no outline");
            if (!(src.radius > 0.f) || !finite(src.radius)) return fail(MHC_E_INVALID, where() + "pedestrian needs a positive radius");
            d.rad = src.radius; d.circ = src.radius;
        }
        d.scen = si; d.n_steps = N; d.substeps = sc->substeps; d.model = sc->model; d.tau = sc->tau;
        d.tau_i_d = (double)sc->tau / (double)sc->substeps;
        if (src.kind == MHC_VEHICLE) {
            d.regime_off = (int)L.regimes.size();
            for (int q = 0; q < src.n_a; ++q)
                L.regimes.push_back(speed_regime(src.v0, src.grid_a[q], sc->model, N * sc->substeps, d.tau_i_d));
        }
        d.path_off = -1;
        if (src.paths) {   // path hypotheses (Section IV-B.2b): n_b paths of three sections (x, y, psi)
            if (src.kind != MHC_VEHICLE) return fail(MHC_E_INVALID, where() + "pedestrians take no paths");
            if (L.paths.size() / 9 + (size_t)src.n_b > (size_t)0x7fffffff)
                return fail(MHC_E_INVALID, where() + "too many paths in the batch");
            d.path_off = (int)(L.paths.size() / 9);
            for (long long q = 0; q < 9LL * src.n_b; ++q) {
                if (!finite(src.paths[q])) return fail(MHC_E_INVALID, where() + "path sections must be finite");
                L.paths.push_back(src.paths[q]);
            }
            // the sections switch at t = n tau_i >= 1.0 s and >= 1.5 s, decided in FP64
            auto first_at = [&](double t) {
                long long n = (long long)std::ceil(t / d.tau_i_d);
                while (n > 0 && (double)(n - 1) * d.tau_i_d >= t) --n;
                while ((double)n * d.tau_i_d < t) ++n;
                return (int)std::min<long long>(n, 0x7fffffffLL);
            };
            d.path_n1 = first_at(1.0);
            d.path_n2 = first_at(1.5);
        }
        for (int q = 0; q < d.n_tiles32; ++q) { L.warp_obj.push_back(L.n_obj); L.warp_first.push_back(q * kBoundTile); }
        L.objs.push_back(d);
        ++L.n_obj;
    }
    ScenDesc S;
    std::memset(&S, 0, sizeof S);
    S.ego = obj0 + sc->ego;
    S.n_obj = n_obj_s;
    S.n_steps = N;
    S.h_e = L.objs[S.ego].h;
    S.obj0 = obj0;
    S.e_base = L.h_e;
    S.lsum_base = L.n_lsum;
    S.mass_base = L.n_mass;
    S.step_base = L.n_steps_total;
    S.e_traj = L.objs[S.ego].traj_off;
    L.h_e += S.h_e;
    L.n_lsum += (long long)S.h_e * N * n_obj_s;
    L.n_mass += (long long)S.h_e * n_obj_s;
    L.n_steps_total += N;
    L.entry0.push_back(L.n_entries);
    auto add_pair = [&](int la, int lb) {
        PairDesc p;
        std::memset(&p, 0, sizeof p);
        const int a = obj0 + la, b = obj0 + lb;
        const ObjDesc &A = L.objs[a], &B = L.objs[b];
        p.a = a; p.b = b;
        p.tiles_a = (A.h + kTile - 1) / kTile;
        p.tiles_b = (B.h + kTile - 1) / kTile;
        p.off = L.n_entries;
        p.tile_start = L.n_tiles;
        const double R = (double)A.circ + (double)B.circ;
        p.rc2 = (float)(R * R * (1.0 + 1e-6));
        p.r_cull = (float)(R * (1.0 + 1e-6) + 1e-3);
        p.combo = (A.kind == MHC_VEHICLE ? 0 : 2) + (B.kind == MHC_VEHICLE ? 0 : 1);
        if (outline[la] || outline[lb]) p.combo = p.combo == 0 ? 4 : (p.combo == 1 ? 5 : 6);
        p.poly_a = A.poly_off; p.nv_a = A.n_poly;
        p.poly_b = B.poly_off; p.nv_b = B.n_poly;
        copy_object_fields(p, A, B);
        p.ego_side = la == sc->ego ? 0 : (lb == sc->ego ? 1 : -1);
        p.n_steps = N;
        p.scen = si;
        p.kofs = L.n_kofs;
        p.lsum_base = S.lsum_base;
        p.mass_base = S.mass_base;
        p.hits_base = S.e_base;
        p.n_obj_s = n_obj_s;
        p.co_local = p.ego_side == 0 ? lb : (p.ego_side == 1 ? la : 0);
        p.index = (int)L.pairs.size();
        L.n_entries += (long long)A.h * B.h;
        L.n_tiles += (long long)p.tiles_a * p.tiles_b;
        L.n_kofs += N;
        L.pairs.push_back(p);
    };
    if ((long long)L.pairs.size() + (long long)n_obj_s * (n_obj_s - 1) / 2 > 0x7fffffffLL)
        return fail(MHC_E_INVALID, "too many object pairs in the batch");
    if (sc->pair_mode == MHC_EGO_ONLY) {
        for (int b = 0; b < n_obj_s; ++b) if (b != sc->ego) add_pair(sc->ego, b);
    } else {
        for (int a = 0; a < n_obj_s; ++a) for (int b = a + 1; b < n_obj_s; ++b) add_pair(a, b);
    }
    L.scens.push_back(S);
    L.pair0.push_back((int)L.pairs.size());
    ++L.n_scen;
    if (L.n_tiles > 0x7fffffffLL) return fail(MHC_E_INVALID, "too many collision tiles for one launch");
    return MHC_OK;
}

int build_layout(const mhc_scenario *sc, int n_scen, Layout &L) {
    if (!sc) return fail(MHC_E_INVALID, "scenario is NULL");
    if (n_scen < 1 || n_scen > MHC_MAX_SCENARIOS) return fail(MHC_E_INVALID, "n_scenarios must be in [1, 65536]");
    L = Layout();
    {   // capacities from a first look at the inputs (no reallocation while appending)
        size_t objs = 0, pairs = 0, grids = 0, accs = 0, tiles = 0;
        for (int s = 0; s < n_scen; ++s) {
            const int n = sc[s].n_objects;
            if (n < 1 || n > MHC_MAX_OBJECTS || !sc[s].objects) break;      // reported by the validation
            objs += n;
            pairs += sc[s].pair_mode == MHC_EGO_ONLY ? (size_t)(n - 1) : (size_t)n * (n - 1) / 2;
            for (int o = 0; o < n; ++o) {
                const mhc_object &src = sc[s].objects[o];
                if (src.n_a < 1 || src.n_b < 1 || (long long)src.n_a * src.n_b > (1LL << 30)) continue;
                grids += (size_t)src.n_a + src.n_b;
                accs += (size_t)src.n_a;
                tiles += ((size_t)src.n_a * src.n_b + kBoundTile - 1) / kBoundTile;
            }
        }
        L.objs.reserve(objs);
        L.pairs.reserve(pairs);
        L.grids.reserve(grids);
        L.regimes.reserve(accs);
        L.warp_obj.reserve(tiles);
        L.warp_first.reserve(tiles);
        L.scens.reserve(n_scen);
        L.pair0.reserve(n_scen + 1);
        L.entry0.reserve(n_scen + 1);
    }
    L.pair0.push_back(0);
    for (int s = 0; s < n_scen; ++s)
        if (int r = append_scenario(sc + s, s, n_scen > 1, L)) return r;
    L.entry0.push_back(L.n_entries);
    // collision-grid order: pairs by the distance of their objects' initial positions, closest first (the
    // pairs that stay close longest carry the most active steps and candidates; starting them first keeps
    // them off the end of the launch)
    std::vector<std::pair<float, int>> key(L.pairs.size());
    for (size_t p = 0; p < L.pairs.size(); ++p) {
        const ObjDesc &A = L.objs[L.pairs[p].a], &B = L.objs[L.pairs[p].b];
        const float dx = A.x0 - B.x0, dy = A.y0 - B.y0;
        key[p] = {std::sqrt(dx * dx + dy * dy) - A.circ - B.circ, (int)p};
    }
    std::stable_sort(key.begin(), key.end());
    L.pairs_c.resize(L.pairs.size());
    long long tiles = 0;
    for (size_t q = 0; q < key.size(); ++q) {
        PairDesc d = L.pairs[key[q].second];
        d.tile_start = tiles;
        tiles += (long long)d.tiles_a * d.tiles_b;
        L.pairs_c[q] = d;
    }
    return MHC_OK;
}

int build_layout(const mhc_scenario *sc, Layout &L) { return build_layout(sc, 1, L); }

// Generation warp tasks: a hypothesis is a sequential chain of sub-steps, so with fewer hypotheses than
// warp schedulers (4 per SM) each warp takes fewer of them (down to 4) to occupy every scheduler.
void plan_generation(Layout &L, int n_sm, int mode) {
    L.gen_obj.clear();
    L.gen_first.clear();
    // one warp per hypothesis (parallel in time) for the objects of scenarios with few hypotheses, so that
    // a scenario gets the same poses alone and in any batch
    std::vector<char> scan(L.n_obj, 0);
    for (const ScenDesc &S : L.scens) {
        long long traj = 0;
        for (int o = S.obj0; o < S.obj0 + S.n_obj; ++o) traj += L.objs[o].h;
        const bool sc = mode == 1 || (mode == 2 && traj <= kGenScanMaxTraj);
        for (int o = S.obj0; o < S.obj0 + S.n_obj; ++o) scan[o] = sc && L.objs[o].path_off < 0;   // controller
                                                                     // feedback: a path hypothesis runs in order
    }
    // the warp-per-hypothesis objects as ranges of warps: entry k = (object, its first warp)
    long long seq_traj = 0, warps = 0;
    for (int o = 0; o < L.n_obj; ++o) {
        if (!scan[o]) { seq_traj += L.objs[o].h; continue; }
        L.gen_obj.push_back(o);
        L.gen_first.push_back((int)warps);
        warps += L.objs[o].h;
    }
    L.n_gen_scan = (int)warps;
    L.n_gen_scan_objs = (int)L.gen_obj.size();
    // the others: one thread per hypothesis, `lanes` per warp; with fewer hypotheses than warp schedulers
    // (4 per SM) each warp takes fewer of them (down to 4) to occupy every scheduler (more, smaller warps
    // measured slower on large scenes, where the sub-steps' instructions fill the issue slots)
    const long long schedulers = 4LL * (n_sm > 0 ? n_sm : 152);
    int lanes = 32;
    while (lanes > 4 && (seq_traj + lanes - 1) / lanes < schedulers) lanes >>= 1;
    L.gen_lanes = lanes;
    long long tasks = 0;
    for (int o = 0; o < L.n_obj; ++o)
        if (!scan[o]) tasks += (L.objs[o].h + lanes - 1) / lanes;
    const size_t base = L.gen_obj.size();
    L.gen_obj.resize(base + (size_t)tasks);
    L.gen_first.resize(base + (size_t)tasks);
    int *go = L.gen_obj.data() + base, *gf = L.gen_first.data() + base;
    for (int o = 0; o < L.n_obj; ++o)
        if (!scan[o])
            for (int q = 0; q < L.objs[o].h; q += lanes) { *go++ = o; *gf++ = q; }
    L.n_gen_warps = L.n_gen_scan + (int)tasks;
}

// The step-item layout (collision variant 6) applies while its item list (4 x tiles x steps entries) stays
// small; the list lives in the call's scratch.
bool items_eligible(const Layout &L) {
    return L.n_tiles * 4 <= 0x7fffffffLL && 4 * L.n_tiles * (long long)L.max_steps <= kItemsMax &&
           L.n_entries <= kItemsMaxEntries;
}

// The block-list layout (collision variant 8) applies while its records (128 bytes per 32 x 32 block) stay
// small; they live in the call's scratch.
bool blocklist_eligible(const Layout &L) { return 4 * L.n_tiles <= kBlockListMax; }

// Device scratch each call needs (besides caller buffers).
// 64-bit accumulator words of one assessment
long long acc_words(const Layout &L) {
    const long long np = (long long)L.pairs.size();
    return np + L.n_kofs + np + L.n_kofs + L.h_e + L.n_lsum + L.n_mass + L.n_obj + L.n_steps_total +
           5LL * L.n_scen + 1;
}

Scratch scratch_of(const Layout &L, bool with_weights) {
    Scratch s;
    const size_t gen_tasks = (size_t)L.n_traj + L.objs.size();   // the most generation tasks (a warp each)
    s.desc = align_up(sizeof(ObjDesc) * L.objs.size()) + 2 * align_up(sizeof(PairDesc) * (L.pairs.size() + 1)) +
             align_up(sizeof(ScenDesc) * L.scens.size()) + align_up(sizeof(float) * L.grids.size()) +
             2 * align_up(sizeof(int) * L.warp_obj.size()) + 2 * align_up(sizeof(int) * gen_tasks) +
             align_up(sizeof(Regime) * L.regimes.size()) + align_up(sizeof(PolyVertex) * L.polys.size()) +
             align_up(sizeof(float) * L.paths.size());
    s.bounds = align_up(sizeof(float4) * (size_t)L.n_bounds);
    s.prob = align_up(sizeof(double) * (size_t)L.n_traj) + align_up(sizeof(float) * (size_t)L.n_traj) +
             2 * align_up(sizeof(unsigned long long) * (size_t)L.n_traj);
    s.weights = with_weights ? align_up(sizeof(float) * (size_t)L.n_traj) : 0;
    s.acc_words = acc_words(L);
    s.acc = align_up(8 * (size_t)s.acc_words);
    s.items = items_eligible(L) ? kAlign + align_up(sizeof(StepItem) * (size_t)(4 * L.n_tiles * (long long)L.max_steps)) +
                                      align_up(4 * (size_t)L.n_entries) + align_up(16 * (size_t)L.n_tiles) +
                                      align_up(4 * sizeof(ItemBlock) * (size_t)L.n_tiles)
                                : 0;
    if (blocklist_eligible(L))   // variant 6 or 8 takes the space, never both in one call
        s.items = std::max(s.items, kAlign + align_up(4 * sizeof(ActiveBlock) * (size_t)L.n_tiles));
    s.total = s.desc + s.weights + s.bounds + s.prob + s.acc + s.items;
    return s;
}

cudaEvent_t pooled_event(mhc_ctx *ctx) {
    if (!ctx->ev_pool.empty()) {
        cudaEvent_t e = ctx->ev_pool.back();
        ctx->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Order this call after the context's previous call when it used another stream.
int begin_call(mhc_ctx *ctx, cudaStream_t st) {
    MHC_CUDA(cudaSetDevice(ctx->device));
    if (ctx->has_last && ctx->last_stream != st) MHC_CUDA(cudaStreamWaitEvent(st, ctx->done_ev, 0));
    return MHC_OK;
}

int end_call(mhc_ctx *ctx, cudaStream_t st) {
    MHC_CUDA(cudaEventRecord(ctx->done_ev, st));
    ctx->last_stream = st;
    ctx->has_last = true;
    return MHC_OK;
}

size_t pack_descriptors(const Layout &L, const std::vector<float> *weights, char *host, char *dev, DevDesc &out) {
    constexpr int kParts = 12;
    const std::pair<const void *, size_t> parts[kParts] = {
        {L.objs.data(), sizeof(ObjDesc) * L.objs.size()},
        {L.pairs.data(), sizeof(PairDesc) * L.pairs.size()},
        {L.pairs_c.data(), sizeof(PairDesc) * L.pairs_c.size()},
        {L.scens.data(), sizeof(ScenDesc) * L.scens.size()},
        {L.grids.data(), sizeof(float) * L.grids.size()},
        {L.warp_obj.data(), sizeof(int) * L.warp_obj.size()},
        {L.warp_first.data(), sizeof(int) * L.warp_first.size()},
        {L.gen_obj.data(), sizeof(int) * L.gen_obj.size()},
        {L.gen_first.data(), sizeof(int) * L.gen_first.size()},
        {L.regimes.data(), sizeof(Regime) * L.regimes.size()},
        {L.polys.data(), sizeof(PolyVertex) * L.polys.size()},
        {L.paths.data(), sizeof(float) * L.paths.size()},
    };
    size_t caps[kParts];
    for (int q = 0; q < kParts; ++q) caps[q] = align_up(parts[q].second);
    caps[1] = align_up(sizeof(PairDesc) * (L.pairs.size() + 1));
    caps[2] = align_up(sizeof(PairDesc) * (L.pairs.size() + 1));
    size_t off = 0;
    char *ptrs[kParts + 1];
    for (int q = 0; q < kParts; ++q) {
        if (host && parts[q].second) std::memcpy(host + off, parts[q].first, parts[q].second);
        ptrs[q] = dev + off;
        off += caps[q];
    }
    ptrs[kParts] = dev + off;
    if (weights) {
        if (host && !weights->empty()) std::memcpy(host + off, weights->data(), sizeof(float) * weights->size());
        off += align_up(sizeof(float) * weights->size());
    }
    out.objs = reinterpret_cast<ObjDesc *>(ptrs[0]);
    out.pairs = reinterpret_cast<PairDesc *>(ptrs[1]);
    out.pairs_c = reinterpret_cast<PairDesc *>(ptrs[2]);
    out.scens = reinterpret_cast<ScenDesc *>(ptrs[3]);
    out.grids = reinterpret_cast<float *>(ptrs[4]);
    out.warp_obj = reinterpret_cast<int *>(ptrs[5]);
    out.warp_first = reinterpret_cast<int *>(ptrs[6]);
    out.gen_obj = reinterpret_cast<int *>(ptrs[7]);
    out.gen_first = reinterpret_cast<int *>(ptrs[8]);
    out.regimes = reinterpret_cast<Regime *>(ptrs[9]);
    out.polys = L.polys.empty() ? nullptr : reinterpret_cast<PolyVertex *>(ptrs[10]);
    out.paths = L.paths.empty() ? nullptr : reinterpret_cast<float *>(ptrs[11]);
    out.weights = weights ? reinterpret_cast<float *>(ptrs[kParts]) : nullptr;
    return off;
}

int upload(mhc_ctx *ctx, const Layout &L, const std::vector<float> *weights, char *dev, cudaStream_t st,
           DevDesc &out) {
    const size_t total = pack_descriptors(L, weights, nullptr, dev, out);
    const int s = ctx->slot;
    ctx->slot = (ctx->slot + 1) % kSlots;
    MHC_CUDA(cudaEventSynchronize(ctx->stage_ev[s]));
    if (ctx->stage_cap[s] < total) {
        if (ctx->stage[s]) MHC_CUDA(cudaFreeHost(ctx->stage[s]));
        ctx->stage[s] = ctx->stage_dev[s] = nullptr;
        ctx->stage_cap[s] = 0;
        size_t cap = total < (1u << 20) ? (1u << 20) : total * 2;
        MHC_CUDA(alloc_mapped(cap, &ctx->stage[s], &ctx->stage_dev[s]));
        ctx->stage_cap[s] = cap;
    }
    pack_descriptors(L, weights, ctx->stage[s], dev, out);
    {
        TimedScope ts(ctx, st, MHC_K_GENERATE, 1);
        MHC_CUDA(launch_copy(dev, ctx->stage_dev[s], total, st));   // a kernel: no copy-engine hand-off
    }
    MHC_CUDA(cudaEventRecord(ctx->stage_ev[s], st));
    ctx->h2d = (long long)total;
    ctx->d2h = 0;
    return MHC_OK;
}

int check_ctx(mhc_ctx *ctx) { return ctx ? MHC_OK : fail(MHC_E_INVALID, "context is NULL"); }

// The caller's device arrays at their elements' natural alignment (the kernels read and write whole
// elements; a misaligned one would fault on the device).  Any argument may be NULL (not checked here).
int check_device_arrays(const mhc_poses *p, const int16_t *table, const mhc_risk *r) {
    auto bad = [](const void *q, uintptr_t a) { return q && (reinterpret_cast<uintptr_t>(q) % a) != 0; };
    if (p && (bad(p->x, 4) || bad(p->y, 4) || bad(p->c, 4) || bad(p->s, 4)))
        return fail(MHC_E_INVALID, "pose planes must be 4-byte aligned");
    if (bad(table, 2)) return fail(MHC_E_INVALID, "table must be 2-byte aligned");
    if (r && (bad(r->count, 8) || bad(r->count_k, 8) || bad(r->P, 8) || bad(r->H, 8) || bad(r->naive, 8) ||
              bad(r->cond, 8) || bad(r->indep, 8) || bad(r->hits, 4) || bad(r->attr_obj, 8) ||
              bad(r->attr_step, 8) || bad(r->scalars, 8) || bad(r->escape, 4) || bad(r->n_escape, 4)))
        return fail(MHC_E_INVALID, "risk outputs must be aligned to their element size");
    return MHC_OK;
}

// Validated host weights (ones where a pointer is NULL); empty when all uniform.
int gather_weights(const Layout &L, const float *const *w, std::vector<float> &out) {
    out.clear();
    if (!w) return MHC_OK;
    bool any = false;
    for (int o = 0; o < L.n_obj; ++o) any |= w[o] != nullptr;
    if (!any) return MHC_OK;
    out.resize((size_t)L.n_traj);
    for (int o = 0; o < L.n_obj; ++o) {
        const ObjDesc &d = L.objs[o];
        double sum = 0.0;
        for (int i = 0; i < d.h; ++i) {
            const float v = w[o] ? w[o][i] : 1.0f;
            if (!(v >= 0.f) || !finite(v)) {
                char msg[96];
                std::snprintf(msg, sizeof msg, "object %d: weights must be finite and non-negative", o);
                return fail(MHC_E_INVALID, msg);
            }
            out[(size_t)d.traj_off + i] = v;
            sum += v;
        }
        if (!(sum > 0.0)) {
            char msg[96];
            std::snprintf(msg, sizeof msg, "object %d: weights sum to zero", o);
            return fail(MHC_E_INVALID, msg);
        }
    }
    return MHC_OK;
}

// Risk scratch of one assessment (accumulators + probabilities) carved from the arena.
int make_risk_args(const Layout &L, const DevDesc &D, Bump &bump, const int16_t *table, const mhc_risk *rout,
                   RiskArgs &r) {
    std::memset(&r, 0, sizeof r);
    r.objs = D.objs; r.pairs = D.pairs; r.scens = D.scens;
    r.n_pairs = (int)L.pairs.size(); r.n_obj = L.n_obj; r.n_scen = L.n_scen;
    r.h_e = L.h_e; r.n_kofs = L.n_kofs; r.n_steps_total = L.n_steps_total; r.max_steps = L.max_steps;
    r.n_tiles = L.n_tiles; r.table = table;
    r.weights = D.weights;
    r.prob = static_cast<double *>(bump.take(sizeof(double) * (size_t)L.n_traj));
    r.probf = static_cast<float *>(bump.take(sizeof(float) * (size_t)L.n_traj));
    r.pfix = static_cast<unsigned long long *>(bump.take(sizeof(unsigned long long) * (size_t)L.n_traj));
    r.lfix = static_cast<unsigned long long *>(bump.take(sizeof(unsigned long long) * (size_t)L.n_traj));
    const long long np = (long long)L.pairs.size();
    const long long words = acc_words(L);
    unsigned long long *w = static_cast<unsigned long long *>(bump.take(8 * (size_t)words));
    if (!r.prob || !r.probf || !r.pfix || !r.lfix || !w) return fail(MHC_E_NOMEM, "arena too small for risk scratch");
    RiskScratch &A = r.acc;
    A.base = w; A.n_words = words;
    A.count = w; w += np;
    A.count_k = w; w += L.n_kofs;
    A.P = w; w += np;
    A.H = w; w += L.n_kofs;
    A.hits = w; w += L.h_e;
    A.lsum = w; w += L.n_lsum;
    A.mass = w; w += L.n_mass;
    A.attr_obj = w; w += L.n_obj;
    A.attr_step = w; w += L.n_steps_total;
    A.scalars = reinterpret_cast<double *>(w); w += 4LL * L.n_scen;
    A.n_escape = w; w += L.n_scen;
    A.done = w;
    r.count = reinterpret_cast<long long *>(rout->count);
    r.count_k = reinterpret_cast<long long *>(rout->count_k);
    r.P = rout->P; r.H = rout->H; r.naive = rout->naive; r.cond = rout->cond; r.indep = rout->indep;
    r.hits = rout->hits; r.attr_obj = rout->attr_obj; r.attr_step = rout->attr_step;
    r.scalars = rout->scalars; r.escape = rout->escape; r.n_escape = rout->n_escape;
    return MHC_OK;
}

int log2_floor(long long v) {
    int r = 0;
    while (v > 1) { v >>= 1; ++r; }
    return r;
}

// Collision configuration for a scenario: the forced variant, else the tuned one of its size class, else
// the default (a warp per tile for at least 32 tiles per SM, else a warp per quarter tile).
// The collision layout without tuning.  Large scenes: a warp per tile in step order; small ones, whose
// time is the closest pairs' long step chains: every active step in parallel where the item list fits,
// else a warp per quarter tile.
int default_variant(const mhc_ctx *ctx, const Layout &L) {
    return L.n_tiles >= 32LL * ctx->n_sm ? 4 : 7;
}

void pick_collide_config(const mhc_ctx *ctx, const Layout &L, bool fused, int &variant, int &cull) {
    cull = ctx->cull;
    if (ctx->variant != 0) { variant = ctx->variant; return; }
    const int tl = log2_floor(L.n_tiles), sl = log2_floor(L.max_steps);
    for (const auto &t : ctx->tuned)
        if (t.tiles_log2 == tl && t.steps_log2 == sl && t.fused == (int)fused) {
            variant = t.variant;
            cull = t.cull;
            return;
        }
    variant = default_variant(ctx, L);
}

// Device buffers for the risk outputs of one assessment, carved from the arena.
bool take_risk_outputs(Bump &bump, const Layout &L, mhc_risk &R) {
    const size_t np = L.pairs.size(), nk = L.n_kofs, he = L.h_e, no = L.n_obj, ns = L.n_scen;
    std::memset(&R, 0, sizeof R);
    R.count = static_cast<int64_t *>(bump.take(8 * np));
    R.count_k = static_cast<int64_t *>(bump.take(8 * nk));
    R.P = static_cast<double *>(bump.take(8 * np));
    R.H = static_cast<double *>(bump.take(8 * nk));
    R.naive = static_cast<double *>(bump.take(8 * he));
    R.cond = static_cast<double *>(bump.take(8 * he));
    R.indep = static_cast<double *>(bump.take(8 * he));
    R.hits = static_cast<int32_t *>(bump.take(4 * he));
    R.attr_obj = static_cast<double *>(bump.take(8 * no));
    R.attr_step = static_cast<double *>(bump.take(8 * (size_t)L.n_steps_total));
    R.scalars = static_cast<double *>(bump.take(8 * 4 * ns));
    R.escape = static_cast<int32_t *>(bump.take(4 * he));
    R.n_escape = static_cast<int32_t *>(bump.take(4 * ns));
    return R.count && R.count_k && R.P && R.H && R.naive && R.cond && R.indep && R.hits && R.attr_obj &&
           R.attr_step && R.scalars && R.escape && R.n_escape;
}

// Device bytes of the risk outputs take_risk_outputs carves.
size_t risk_output_bytes(const Layout &L) {
    const size_t np = L.pairs.size(), nk = L.n_kofs, he = L.h_e, no = L.n_obj, ns = L.n_scen;
    return align_up(8 * np) * 2 + align_up(8 * nk) * 2 + align_up(8 * he) * 3 + align_up(4 * he) * 2 +
           align_up(8 * no) + align_up(8 * (size_t)L.n_steps_total) + align_up(32 * ns) + align_up(4 * ns);
}

// Launch sequence.  fused: the collision kernel accumulates the risk terms at each first hit (no second
// pass over the table): prepare -> generate -> fill + bounds -> collide -> ego walk + finish.
int launch_all(mhc_ctx *ctx, const Layout &L, const DevDesc &D, Bump &bump, const mhc_poses *gen_out,
               const mhc_poses *coll_in, int16_t *table, bool risk, const mhc_risk *rout, cudaStream_t st,
               bool fused, bool after_upload) {
    RiskArgs r;
    fused = fused && risk && coll_in;
    if (risk) {
        if (int rc = make_risk_args(L, D, bump, table, rout, r)) return rc;
        r.score = ctx->score;
        r.grids = D.grids;
        r.paths = D.paths;
    }
    // after_kernel: the last operation put on the stream here is one of this sequence's kernels, so the
    // next may be a programmatic dependent launch (not while profiling: event records sit in between)
    bool after_kernel = false;
    auto pdl = [&]() { return after_kernel && !ctx->profile; };
    if (fused && !gen_out) {   // else the preparation runs inside the generation launch
        TimedScope ts(ctx, st, MHC_K_RISK, 1);
        cudaError_t e = launch_risk_prepare(r, st);
        if (e != cudaSuccess) return cuda_fail(e, "risk prepare launch");
        after_kernel = true;
    }
    // the collision configuration decides where the table's -1s are written: by the collision kernel itself
    // (variants 5 on small tables, 6); for large tables by fill CTAs of the generation launch when it is
    // part of the sequence (the HBM-bound fill beside the latency-bound integration); else by the bounds
    // kernel (variants 7, 8 with culling: small tables, where fill CTAs would take residency from the
    // generation warps) or a fill kernel
    int variant = 1, cull = 1;
    if (coll_in) {
        pick_collide_config(ctx, L, fused, variant, cull);
        if (variant == 6 && !items_eligible(L)) variant = 5;
        if (variant == 8 && !blocklist_eligible(L)) variant = 7;
    }
    const bool fill_in_collide = (variant == 5 && L.n_entries <= kFillInCollideMax) || variant == 6;
    const bool fill_in_gen = coll_in && gen_out && !fill_in_collide && L.n_entries > kFillInCollideMax &&
                             !L.gen_obj.empty();
    if (gen_out) {
        GenArgs g;
        g.objs = D.objs; g.regimes = D.regimes; g.grids = D.grids; g.warp_obj = D.gen_obj; g.warp_first = D.gen_first;
        g.n_warps = L.n_gen_warps; g.lanes = L.gen_lanes;
        g.n_scan = L.n_gen_scan;
        g.n_scan_objs = L.n_gen_scan_objs;
        g.gen_blocks = 0;
        g.prep_blocks = 0;
        std::memset(&g.prep, 0, sizeof g.prep);
        if (fused) {
            g.prep = prep_of(r);
            // enough CTAs to zero the accumulators at about 2048 words each (at least one per object,
            // at most two per SM): extra CTAs would only take residency from the generation warps
            const long long words = acc_words(L) + L.h_e;
            long long nb = (words + 2047) / 2048;
            if (nb > 304) nb = 304;
            if (nb < L.n_obj) nb = L.n_obj;
            g.prep_blocks = (int)nb;
        }
        g.paths = D.paths;
        g.x = gen_out->x; g.y = gen_out->y; g.c = gen_out->c; g.s = gen_out->s;
        g.fill = fill_in_gen ? table : nullptr;
        g.n_fill = fill_in_gen ? L.n_entries : 0;
        TimedScope ts(ctx, st, MHC_K_GENERATE, 1);
        cudaError_t e = launch_generate(g, st, after_upload && !ctx->profile);
        if (e != cudaSuccess) return cuda_fail(e, "generation kernel launch");
        after_kernel = true;
    }
    if (coll_in) {
        float4 *bounds = static_cast<float4 *>(bump.take(sizeof(float4) * (size_t)L.n_bounds));
        if (!bounds) return fail(MHC_E_NOMEM, "arena too small for tile bounds");
        // small tables: the quarter-tile layout writes the -1s of its own blocks (one launch less); large ones
        // are filled by the HBM-rate fill kernel (in-kernel 2-byte row stores cost issue slots there)
        const bool fill_in_bounds = !fill_in_gen && (variant == 7 || variant == 8) && cull &&
                                    (long long)L.warp_obj.size() * L.max_steps > 0;
        CollideArgs c{};
        if (variant == 6) {   // the item list and its two counters (zeroed by the bounds kernel, else a memset)
            c.max_items = 4 * L.n_tiles * (long long)L.max_steps;
            c.item_count = static_cast<unsigned long long *>(bump.take(kAlign));
            c.items = static_cast<StepItem *>(bump.take(sizeof(StepItem) * (size_t)c.max_items));
            c.active_count = c.item_count + 1;
            c.first32 = static_cast<int *>(bump.take(sizeof(int) * (size_t)L.n_entries));
            c.active = static_cast<int *>(bump.take(sizeof(int) * (size_t)(4 * L.n_tiles)));
            c.blocks = static_cast<ItemBlock *>(bump.take(sizeof(ItemBlock) * (size_t)(4 * L.n_tiles)));
            if (!c.items || !c.item_count || !c.first32 || !c.active || !c.blocks)
                return fail(MHC_E_NOMEM, "arena too small for the step items");
        }
        if (variant == 8) {   // the block records and their count (zeroed by the bounds kernel, else a memset)
            c.item_count = static_cast<unsigned long long *>(bump.take(kAlign));
            c.active_count = c.item_count + 1;
            c.recs = static_cast<ActiveBlock *>(bump.take(sizeof(ActiveBlock) * (size_t)(4 * L.n_tiles)));
            if (!c.item_count || !c.recs) return fail(MHC_E_NOMEM, "arena too small for the block records");
        }
        bool counts_zeroed = false;
        {
            const bool fill_alone = !fill_in_collide && !fill_in_bounds && !fill_in_gen;
            TimedScope ts(ctx, st, MHC_K_BOUNDS, (cull ? 1 : 0) + (fill_alone ? 1 : 0));
            cudaError_t e = fill_alone ? launch_fill_table(table, L.n_entries, st, pdl()) : cudaSuccess;
            if (e != cudaSuccess) return cuda_fail(e, "table fill launch");
            if (fill_alone && L.n_entries > 0) after_kernel = true;
            if (cull) {
                BoundsArgs b{};
                b.objs = D.objs; b.warp_obj = D.warp_obj; b.warp_first = D.warp_first;
                b.n_warps = (int)L.warp_obj.size(); b.max_steps = L.max_steps; b.x = coll_in->x; b.y = coll_in->y;
                b.bounds = bounds;
                const bool launches = (long long)b.n_warps * b.max_steps > 0;
                if ((variant == 6 || variant == 8) && launches) b.zero_counts = c.item_count;
                if (fill_in_bounds) { b.fill = table; b.n_fill = L.n_entries; }
                e = launch_bounds(b, st, pdl());
                if (e != cudaSuccess) return cuda_fail(e, "bounds kernel launch");
                if (launches) after_kernel = true;
                counts_zeroed = b.zero_counts != nullptr;
            }
        }
        c.objs = D.objs; c.pairs = D.pairs_c; c.n_pairs = (int)L.pairs.size(); c.n_obj = L.n_obj; c.n_tiles = L.n_tiles;
        c.max_steps = L.max_steps; c.cull = cull; c.variant = variant; c.fill_blocks = fill_in_collide;
        c.max_ctas = ctx->collide_max_ctas;
        c.x = coll_in->x; c.y = coll_in->y; c.c = coll_in->c; c.s = coll_in->s;
        c.bounds = bounds; c.polys = D.polys; c.table = table; c.counters = ctx->counters;
        if (fused) {
            c.probf = r.probf;
            c.pfix = r.pfix;
            c.lfix = r.lfix;
            c.acc = r.acc;
        }
        if ((variant == 6 || variant == 8) && !counts_zeroed) {
            MHC_CUDA(cudaMemsetAsync(c.item_count, 0, 2 * sizeof(unsigned long long), st));
            after_kernel = false;
        }
        TimedScope ts(ctx, st, MHC_K_COLLIDE, variant == 6 ? 3 : (variant == 8 ? 2 : 1));
        cudaError_t e = launch_collide(c, st, pdl());
        if (e != cudaSuccess) return cuda_fail(e, "collision kernel launch");
        if (L.n_tiles > 0) after_kernel = true;
    }
    if (risk) {   // fused collision: the walk only; else preparation, table scan and walk
        TimedScope ts(ctx, st, MHC_K_RISK, (fused ? 0 : 2) + risk_tail_launches(r));
        cudaError_t e = fused ? launch_risk_tail(r, st, pdl()) : launch_risk(r, st, true, pdl());
        if (e != cudaSuccess) return cuda_fail(e, "risk kernel launch");
    }
    return MHC_OK;
}

}  // namespace host

// Records the reason of a failure for mhc_last_error() (used by entry points in other files).
void set_last_error(const char *why) { g_err = why ? why : ""; }
}  // namespace mhc

extern "C" {

const char *mhc_status_string(int s) {
    switch (s) {
        case MHC_OK: return "MHC_OK";
        case MHC_PENDING: return "MHC_PENDING";
        case MHC_E_INVALID: return "MHC_E_INVALID";
        case MHC_E_NOMEM: return "MHC_E_NOMEM";
        case MHC_E_CUDA: return "MHC_E_CUDA";
        case MHC_E_TIMEOUT: return "MHC_E_TIMEOUT";
        case MHC_E_BUSY: return "MHC_E_BUSY";
        case MHC_E_NOTFOUND: return "MHC_E_NOTFOUND";
        default: return "MHC_E_UNKNOWN";
    }
}

const char *mhc_last_error(void) { return g_err.c_str(); }

const char *mhc_version(void) { return "mhc 0.1 sm_103a"; }

int mhc_create(mhc_ctx **out, int device, void *arena, size_t arena_bytes) {
    if (!out) return fail(MHC_E_INVALID, "out is NULL");
    *out = nullptr;
    if (arena_bytes < (1u << 20)) return fail(MHC_E_INVALID, "arena_bytes must be at least 1 MiB");
    // the arena holds float4 bounds, 8-byte counters and the 16-byte words of the descriptor copy
    if (reinterpret_cast<uintptr_t>(arena) % kAlign) return fail(MHC_E_INVALID, "arena must be 256-byte aligned");
    int n = 0;
    MHC_CUDA(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) return fail(MHC_E_INVALID, "device out of range");
    MHC_CUDA(cudaSetDevice(device));
    mhc_ctx *c = new mhc_ctx();
    c->device = device;
    c->arena_bytes = arena_bytes;
    if (cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) c->n_sm = 152;
    if (arena) {
        c->arena = static_cast<char *>(arena);
    } else {
        cudaError_t e = cudaMalloc(&c->arena, arena_bytes);
        if (e != cudaSuccess) { delete c; return fail(MHC_E_NOMEM, "cudaMalloc of the arena failed"); }
        c->owns = true;
    }
    for (int s = 0; s < kSlots; ++s) {
        cudaError_t e = cudaEventCreateWithFlags(&c->stage_ev[s], cudaEventDisableTiming);
        if (e != cudaSuccess) { mhc_destroy(c); return cuda_fail(e, "cudaEventCreate"); }
    }
    cudaError_t e = cudaEventCreateWithFlags(&c->done_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) { mhc_destroy(c); return cuda_fail(e, "cudaEventCreate"); }
    c->counters = reinterpret_cast<unsigned long long *>(c->arena);
    e = cudaMemset(c->counters, 0, kReserved);
    if (e != cudaSuccess) { mhc_destroy(c); return cuda_fail(e, "cudaMemset"); }
    *out = c;
    return MHC_OK;
}

void mhc_destroy(mhc_ctx *c) {
    if (!c) return;
    if (c->server) serve_shutdown(c);
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    for (int s = 0; s < kSlots; ++s) {
        if (c->stage_ev[s]) cudaEventDestroy(c->stage_ev[s]);
        if (c->stage[s]) cudaFreeHost(c->stage[s]);
    }
    if (c->out_stage) cudaFreeHost(c->out_stage);
    if (c->done_ev) cudaEventDestroy(c->done_ev);
    for (auto &t : c->timed) { cudaEventDestroy(t.a); cudaEventDestroy(t.b); }
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    if (c->owns && c->arena) cudaFree(c->arena);
    delete c;
}

int mhc_set_option(mhc_ctx *ctx, int option, long long value) {
    if (int r = check_ctx(ctx)) return r;
    if (option == MHC_OPT_CULL) { ctx->cull = value != 0; return MHC_OK; }
    if (option == MHC_OPT_PROFILE) { ctx->profile = value != 0; return MHC_OK; }
    if (option == MHC_OPT_SCORE) { ctx->score = value != 0; return MHC_OK; }
    if (option == MHC_OPT_GEN_SCAN) {
        if (value < 0 || value > 2) return fail(MHC_E_INVALID, "generation layout must be 0, 1 or 2");
        ctx->gen_scan = (int)value;
        return MHC_OK;
    }
    if (option == MHC_OPT_COLLIDE_VARIANT) {
        if (value < 0 || value > kCollideVariants) return fail(MHC_E_INVALID, "collide variant must be 0 to 8");
        ctx->variant = (int)value;
        return MHC_OK;
    }
    return fail(MHC_E_INVALID, "unknown option");
}

int mhc_profile_read(mhc_ctx *ctx, double ms[4], int64_t launches[4], int reset) {
    if (int r = check_ctx(ctx)) return r;
    MHC_CUDA(cudaSetDevice(ctx->device));
    for (auto &t : ctx->timed) {
        MHC_CUDA(cudaEventSynchronize(t.b));
        float v = 0.f;
        MHC_CUDA(cudaEventElapsedTime(&v, t.a, t.b));
        ctx->prof_ms[t.kind] += v;
        ctx->prof_n[t.kind] += t.launches;
        ctx->ev_pool.push_back(t.a);
        ctx->ev_pool.push_back(t.b);
    }
    ctx->timed.clear();
    for (int k = 0; k < MHC_K_COUNT; ++k) {
        if (ms) ms[k] = ctx->prof_ms[k];
        if (launches) launches[k] = ctx->prof_n[k];
        if (reset) { ctx->prof_ms[k] = 0.0; ctx->prof_n[k] = 0; }
    }
    return MHC_OK;
}

int mhc_transfer_bytes(mhc_ctx *ctx, int64_t *h2d, int64_t *d2h) {
    if (int r = check_ctx(ctx)) return r;
    if (h2d) *h2d = ctx->h2d;
    if (d2h) *d2h = ctx->d2h;
    return MHC_OK;
}

int mhc_collision_counters(mhc_ctx *ctx, uint64_t *out, int32_t n_out, int reset, void *stream) {
    if (int r = check_ctx(ctx)) return r;
    if (!out) return fail(MHC_E_INVALID, "out is NULL");
    if (n_out < 1 || n_out > MHC_COUNTER_WORDS) return fail(MHC_E_INVALID, "n_out must be 1 to MHC_COUNTER_WORDS");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    MHC_CUDA(cudaSetDevice(ctx->device));
    MHC_CUDA(cudaMemcpyAsync(out, ctx->counters, n_out * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    MHC_CUDA(cudaStreamSynchronize(st));
    if (reset) {
        MHC_CUDA(cudaMemsetAsync(ctx->counters, 0, MHC_COUNTER_WORDS * sizeof(uint64_t), st));
        MHC_CUDA(cudaStreamSynchronize(st));
    }
    return MHC_OK;
}

int mhc_layout(const mhc_scenario *scen, int64_t *n_traj, int32_t *n_pairs, int64_t *n_entries, int32_t *h_ego,
               size_t *scratch) {
    Layout L;
    if (int r = build_layout(scen, L)) return r;
    if (n_traj) *n_traj = L.n_traj;
    if (n_pairs) *n_pairs = (int32_t)L.pairs.size();
    if (n_entries) *n_entries = L.n_entries;
    if (h_ego) *h_ego = L.h_e;
    if (scratch) *scratch = kReserved + scratch_of(L, true).total;
    return MHC_OK;
}

int mhc_pair_table(const mhc_scenario *scen, int32_t *pair_a, int32_t *pair_b, int64_t *pair_off) {
    Layout L;
    if (int r = build_layout(scen, L)) return r;
    for (size_t p = 0; p < L.pairs.size(); ++p) {
        if (pair_a) pair_a[p] = L.pairs[p].a;
        if (pair_b) pair_b[p] = L.pairs[p].b;
        if (pair_off) pair_off[p] = L.pairs[p].off;
    }
    if (pair_off) pair_off[L.pairs.size()] = L.n_entries;
    return MHC_OK;
}

int mhc_generate_trajectories(mhc_ctx *ctx, const mhc_scenario *scen, const mhc_poses *out, void *stream) {
    if (int r = check_ctx(ctx)) return r;
    if (!out || !out->x || !out->y || !out->c || !out->s) return fail(MHC_E_INVALID, "pose planes must be non-NULL");
    if (int r = check_device_arrays(out, nullptr, nullptr)) return r;
    Layout L;
    if (int r = build_layout(scen, L)) return r;
    plan_generation(L, ctx->n_sm, ctx->gen_scan);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Scratch S = scratch_of(L, false);
    Bump bump{ctx->arena, ctx->arena_bytes, kReserved};
    char *dev = static_cast<char *>(bump.take(S.desc));
    if (!dev) return fail(MHC_E_NOMEM, "arena too small for the descriptors");
    if (int r = begin_call(ctx, st)) return r;
    DevDesc D;
    if (int r = upload(ctx, L, nullptr, dev, st, D)) return r;
    if (int r = launch_all(ctx, L, D, bump, out, nullptr, nullptr, false, nullptr, st, false, true)) return r;
    return end_call(ctx, st);
}

int mhc_detect_collisions(mhc_ctx *ctx, const mhc_scenario *scen, const mhc_poses *poses, int16_t *table,
                          void *stream) {
    if (int r = check_ctx(ctx)) return r;
    if (!poses || !poses->x || !poses->y || !poses->c || !poses->s || !table)
        return fail(MHC_E_INVALID, "poses and table must be non-NULL");
    if (int r = check_device_arrays(poses, table, nullptr)) return r;
    Layout L;
    if (int r = build_layout(scen, L)) return r;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Scratch S = scratch_of(L, false);
    Bump bump{ctx->arena, ctx->arena_bytes, kReserved};
    char *dev = static_cast<char *>(bump.take(S.desc));
    if (!dev) return fail(MHC_E_NOMEM, "arena too small for the descriptors");
    if (int r = begin_call(ctx, st)) return r;
    DevDesc D;
    if (int r = upload(ctx, L, nullptr, dev, st, D)) return r;
    if (int r = launch_all(ctx, L, D, bump, nullptr, poses, table, false, nullptr, st)) return r;
    return end_call(ctx, st);
}

int mhc_assess_risk(mhc_ctx *ctx, const mhc_scenario *scen, const int16_t *table, const float *const *traj_weights,
                    const mhc_risk *out, void *stream) {
    if (int r = check_ctx(ctx)) return r;
    if (!table || !out) return fail(MHC_E_INVALID, "table and out must be non-NULL");
    if (int r = check_device_arrays(nullptr, table, out)) return r;
    Layout L;
    if (int r = build_layout(scen, L)) return r;
    std::vector<float> w;
    if (int r = gather_weights(L, traj_weights, w)) return r;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Scratch S = scratch_of(L, !w.empty());
    Bump bump{ctx->arena, ctx->arena_bytes, kReserved};
    char *dev = static_cast<char *>(bump.take(S.desc + S.weights));
    if (!dev) return fail(MHC_E_NOMEM, "arena too small for the descriptors");
    if (int r = begin_call(ctx, st)) return r;
    DevDesc D;
    if (int r = upload(ctx, L, w.empty() ? nullptr : &w, dev, st, D)) return r;
    if (int r = launch_all(ctx, L, D, bump, nullptr, nullptr, const_cast<int16_t *>(table), true, out, st)) return r;
    return end_call(ctx, st);
}

int mhc_evaluate(mhc_ctx *ctx, const mhc_scenario *scen, const float *const *traj_weights, const mhc_poses *poses,
                 int16_t *table, const mhc_risk *out, void *stream) {
    return evaluate_impl(ctx, scen, 1, traj_weights, poses, table, out, stream);
}

int mhc_autotune(mhc_ctx *ctx, const mhc_scenario *scen, const mhc_poses *poses, int16_t *table, int fused,
                 int32_t *best_variant, int32_t *best_cull, void *stream) {
    return autotune_impl(ctx, scen, 1, poses, table, fused, best_variant, best_cull, stream);
}

}  // extern "C"

namespace mhc {
namespace host {

int evaluate_impl(mhc_ctx *ctx, const mhc_scenario *scen, int n_scen, const float *const *traj_weights,
                  const mhc_poses *poses, int16_t *table, const mhc_risk *out, void *stream) {
    if (int r = check_ctx(ctx)) return r;
    if (!poses || !poses->x || !poses->y || !poses->c || !poses->s || !table || !out)
        return fail(MHC_E_INVALID, "poses, table and out must be non-NULL");
    if (int r = check_device_arrays(poses, table, out)) return r;
    Layout L;
    if (int r = build_layout(scen, n_scen, L)) return r;
    plan_generation(L, ctx->n_sm, ctx->gen_scan);
    std::vector<float> w;
    if (int r = gather_weights(L, traj_weights, w)) return r;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Scratch S = scratch_of(L, !w.empty());
    Bump bump{ctx->arena, ctx->arena_bytes, kReserved};
    char *dev = static_cast<char *>(bump.take(S.desc + S.weights));
    if (!dev) return fail(MHC_E_NOMEM, "arena too small for the descriptors");
    if (int r = begin_call(ctx, st)) return r;
    DevDesc D;
    if (int r = upload(ctx, L, w.empty() ? nullptr : &w, dev, st, D)) return r;
    if (int r = launch_all(ctx, L, D, bump, poses, poses, table, true, out, st, true, true)) return r;
    return end_call(ctx, st);
}

int autotune_impl(mhc_ctx *ctx, const mhc_scenario *scen, int n_scen, const mhc_poses *poses, int16_t *table,
                  int fused, int32_t *best_variant, int32_t *best_cull, void *stream) {
    if (int r = check_ctx(ctx)) return r;
    if (!poses || !poses->x || !poses->y || !poses->c || !poses->s || !table)
        return fail(MHC_E_INVALID, "poses and table must be non-NULL");
    if (int r = check_device_arrays(poses, table, nullptr)) return r;
    Layout L;
    if (int r = build_layout(scen, n_scen, L)) return r;
    plan_generation(L, ctx->n_sm, ctx->gen_scan);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int saved_variant = ctx->variant, saved_cull = ctx->cull;
    const bool saved_profile = ctx->profile;
    double saved_ms[MHC_K_COUNT];
    int64_t saved_n[MHC_K_COUNT];
    if (int r = mhc_profile_read(ctx, saved_ms, saved_n, 1)) return r;   // keep the caller's totals aside
    float best = 1e30f, t_default = 1e30f;
    int bv = 1, bc = 1, rc = MHC_OK;
    // the layout used without tuning (culling on); kept unless another is at least 10 % faster, so that
    // near-ties do not flip the choice from run to run
    const int v_default = default_variant(ctx, L);
    ctx->profile = true;
    for (int cull = 1; cull >= 0 && rc == MHC_OK; --cull) {
        for (int v = 1; v <= kCollideVariants && rc == MHC_OK; ++v) {
            ctx->variant = v;
            ctx->cull = cull;
            double ms[MHC_K_COUNT];
            int64_t n[MHC_K_COUNT];
            for (int rep = 0; rep < 5 && rc == MHC_OK; ++rep) {   // the first run warms up, four count
                if (fused) {
                    Scratch S = scratch_of(L, false);
                    Bump bump{ctx->arena, ctx->arena_bytes, kReserved};
                    char *dev = static_cast<char *>(bump.take(S.desc));
                    mhc_risk R;
                    if (!dev || !take_risk_outputs(bump, L, R)) { rc = fail(MHC_E_NOMEM, "arena too small to autotune"); break; }
                    if ((rc = begin_call(ctx, st))) break;
                    DevDesc D;
                    if ((rc = upload(ctx, L, nullptr, dev, st, D))) break;
                    if ((rc = launch_all(ctx, L, D, bump, poses, poses, table, true, &R, st, true, true))) break;
                    if ((rc = end_call(ctx, st))) break;
                } else {
                    Scratch S = scratch_of(L, false);
                    Bump bump{ctx->arena, ctx->arena_bytes, kReserved};
                    char *dev = static_cast<char *>(bump.take(S.desc));
                    if (!dev) { rc = fail(MHC_E_NOMEM, "arena too small to autotune"); break; }
                    if ((rc = begin_call(ctx, st))) break;
                    DevDesc D;
                    if ((rc = upload(ctx, L, nullptr, dev, st, D))) break;
                    if ((rc = launch_all(ctx, L, D, bump, nullptr, poses, table, false, nullptr, st))) break;
                    if ((rc = end_call(ctx, st))) break;
                }
                if ((rc = mhc_profile_read(ctx, ms, n, rep == 0))) break;
            }
            if (rc != MHC_OK) break;
            // the collision stage as the path runs it: fill / bounds, collision, and (fused) the risk kernels,
            // which carry the table scan when a layout does not fuse it
            const float t = (float)(ms[MHC_K_BOUNDS] + ms[MHC_K_COLLIDE] + (fused ? ms[MHC_K_RISK] : 0.0));
            mhc_profile_read(ctx, nullptr, nullptr, 1);
            if (t < best) { best = t; bv = v; bc = cull; }
            if (v == v_default && cull == 1) t_default = t;
        }
    }
    ctx->variant = saved_variant;
    ctx->cull = saved_cull;
    ctx->profile = saved_profile;
    for (int k = 0; k < MHC_K_COUNT; ++k) { ctx->prof_ms[k] = saved_ms[k]; ctx->prof_n[k] = saved_n[k]; }
    if (rc != MHC_OK) return rc;
    if (best > 0.90f * t_default) { bv = v_default; bc = 1; }
    const int tl = log2_floor(L.n_tiles), sl = log2_floor(L.max_steps);
    bool stored = false;
    for (auto &t : ctx->tuned)
        if (t.tiles_log2 == tl && t.steps_log2 == sl && t.fused == (fused != 0)) { t.variant = bv; t.cull = bc; stored = true; }
    if (!stored) ctx->tuned.push_back({tl, sl, fused != 0, bv, bc});
    if (best_variant) *best_variant = bv;
    if (best_cull) *best_cull = bc;
    return MHC_OK;
}

}  // namespace host
}  // namespace mhc

extern "C" {

int mhc_run_bytes(const mhc_scenario *scen, size_t *bytes) {
    Layout L;
    if (int r = build_layout(scen, L)) return r;
    if (!bytes) return fail(MHC_E_INVALID, "bytes is NULL");
    const size_t poses = 4 * align_up(sizeof(float) * (size_t)L.n_pose);
    const size_t table = align_up(sizeof(int16_t) * (size_t)L.n_entries);
    *bytes = kReserved + scratch_of(L, true).total + poses + table + risk_output_bytes(L);
    return MHC_OK;
}

int mhc_run(mhc_ctx *ctx, const mhc_scenario *scen, const float *const *traj_weights, const mhc_risk *out,
            void *stream) {
    if (int r = check_ctx(ctx)) return r;
    if (!out) return fail(MHC_E_INVALID, "out is NULL");
    Layout L;
    if (int r = build_layout(scen, L)) return r;
    plan_generation(L, ctx->n_sm, ctx->gen_scan);
    std::vector<float> w;
    if (int r = gather_weights(L, traj_weights, w)) return r;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Scratch S = scratch_of(L, !w.empty());
    Bump bump{ctx->arena, ctx->arena_bytes, kReserved};
    char *dev = static_cast<char *>(bump.take(S.desc + S.weights));
    const size_t plane = sizeof(float) * (size_t)L.n_pose;
    mhc_poses P;
    P.x = static_cast<float *>(bump.take(plane));
    P.y = static_cast<float *>(bump.take(plane));
    P.c = static_cast<float *>(bump.take(plane));
    P.s = static_cast<float *>(bump.take(plane));
    int16_t *table = static_cast<int16_t *>(bump.take(sizeof(int16_t) * (size_t)L.n_entries));
    const size_t np = L.pairs.size(), nk = L.n_kofs, he = L.h_e, no = L.n_obj, ns = L.n_scen;
    mhc_risk R;
    const bool outs = take_risk_outputs(bump, L, R);
    if (!dev || !P.x || !P.y || !P.c || !P.s || !table || !outs)
        return fail(MHC_E_NOMEM, "arena too small for mhc_run (see mhc_run_bytes)");
    if (int r = begin_call(ctx, st)) return r;
    DevDesc D;
    if (int r = upload(ctx, L, w.empty() ? nullptr : &w, dev, st, D)) return r;
    if (int r = launch_all(ctx, L, D, bump, &P, &P, table, true, &R, st, true, true)) return r;
    // the outputs are contiguous in the arena: one copy into mapped pinned staging, then to the caller's arrays
    const size_t out_bytes = risk_output_bytes(L);
    if (ctx->out_stage_cap < out_bytes) {
        if (ctx->out_stage) MHC_CUDA(cudaFreeHost(ctx->out_stage));
        ctx->out_stage = ctx->out_stage_dev = nullptr;
        ctx->out_stage_cap = 0;
        const size_t cap = out_bytes < (1u << 20) ? (1u << 20) : 2 * out_bytes;
        MHC_CUDA(alloc_mapped(cap, &ctx->out_stage, &ctx->out_stage_dev));
        ctx->out_stage_cap = cap;
    }
    {
        TimedScope ts(ctx, st, MHC_K_RISK, 1);
        // written into mapped host memory; a dependent of the risk walk, the sequence's last kernel
        MHC_CUDA(launch_copy(ctx->out_stage_dev, R.count, out_bytes, st, !ctx->profile));
    }
    ctx->d2h = (long long)out_bytes;
    if (int r = end_call(ctx, st)) return r;
    MHC_CUDA(cudaStreamSynchronize(st));
    const char *h = static_cast<const char *>(ctx->out_stage);
    auto at = [&](const void *dev_field) { return h + (static_cast<const char *>(dev_field) - reinterpret_cast<const char *>(R.count)); };
    struct Cp { void *dst; const void *src; size_t n; } cps[] = {
        {out->count, R.count, 8 * np}, {out->count_k, R.count_k, 8 * nk}, {out->P, R.P, 8 * np},
        {out->H, R.H, 8 * nk}, {out->naive, R.naive, 8 * he}, {out->cond, R.cond, 8 * he},
        {out->indep, R.indep, 8 * he}, {out->hits, R.hits, 4 * he}, {out->attr_obj, R.attr_obj, 8 * no},
        {out->attr_step, R.attr_step, 8 * (size_t)L.n_steps_total}, {out->scalars, R.scalars, 8 * 4 * ns},
        {out->escape, R.escape, 4 * he}, {out->n_escape, R.n_escape, 4 * ns}};
    for (const Cp &c : cps)
        if (c.dst && c.n) std::memcpy(c.dst, at(c.src), c.n);
    return MHC_OK;
}

}  // extern "C"
