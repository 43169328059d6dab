// static_detect.cu -- mhc_detect_collisions_static: the collision step for callers that cannot allocate.
//
// Some callers must not allocate memory once they are running: safety or real-time controllers whose
// memory plan is fixed at start-up (an allocation may block, implicitly synchronise the device or fail at
// a frame deadline), and plugins hosted by a framework that owns every device allocation.  This entry
// point serves them: it needs no context, calls no cudaMalloc / cudaFree / cudaHostAlloc and no heap
// allocation on the host.  Its scratch -- the scenario descriptors and the per-tile bounding boxes the
// collision kernel culls with -- lives in one file-scope device array of kStaticScratchBytes (8 MiB) that
// every GPU which loads the library holds until the process exits.
//
// In host code `g_scratch` is only a host-side stand-in for the device array, never a device address:
// handing it to a kernel would fault or, where the GPU can reach host memory, silently use the wrong
// memory.  Every call therefore looks the device address up with cudaGetSymbolAddress (with the calling
// thread's current device) and hands that address to the kernels; the lookup is a host query, so a
// context torn down and created again (the array may then sit elsewhere) is picked up by the next call.
// With CUDA's lazy module loading the library's device code, this array included, is loaded into a
// device's context on first use: the first call on each device is the warm-up that loads it (and so
// reserves the 8 MiB), and belongs at start-up.
//
// The descriptors are staged in a static host array that every call rewrites, so a call recorded into a
// CUDA graph would upload whatever a later call left there: a stream in capture is refused.
#include <cmath>
#include <cstdio>
#include <cstring>

#include "../../include/mhc.h"
#include "mhc_internal.cuh"
#include "runtime.h"

namespace mhc {
void set_last_error(const char *why);   // api.cu
}

using namespace mhc;

namespace {

constexpr size_t kStaticScratchBytes = 8u << 20;   // descriptors + tile bounds, per device
constexpr int kMaxObjects = 64;
constexpr int kMaxPairs = kMaxObjects * (kMaxObjects - 1) / 2;
constexpr int kMaxWarps = 16384;                    // 32-hypothesis bound tiles (524,288 hypotheses)
constexpr size_t kAlign = 256;

static __device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];

constexpr size_t kObjBytes = ((sizeof(ObjDesc) * kMaxObjects + kAlign - 1) / kAlign) * kAlign;
constexpr size_t kPairBytes = ((sizeof(PairDesc) * (kMaxPairs + 1) + kAlign - 1) / kAlign) * kAlign;
constexpr size_t kWarpBytes = ((sizeof(int) * kMaxWarps + kAlign - 1) / kAlign) * kAlign;
constexpr size_t kDescBytes = kObjBytes + kPairBytes + 2 * kWarpBytes;

// Host staging of the descriptor blob: static storage, reused by every call (one host thread at a time).
alignas(256) unsigned char h_blob[kDescBytes];

int fail(int code, const char *why) {
    set_last_error(why);
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    char msg[256];
    std::snprintf(msg, sizeof msg, "%s: %s", what, cudaGetErrorString(e));
    return fail(MHC_E_CUDA, msg);
}

// Device address of g_scratch in the calling thread's current context (looked up on every call).
int scratch_address(void **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_scratch)");
    *out = p;
    return MHC_OK;
}

bool finite(float v) { return v == v && v - v == 0.0f; }

}  // namespace

extern "C" int mhc_detect_collisions_static(const mhc_scenario *sc, const mhc_poses *poses, int16_t *table,
                                            void *stream) {
    if (!sc || !sc->objects) return fail(MHC_E_INVALID, "scenario is NULL");
    if (!poses || !poses->x || !poses->y || !poses->c || !poses->s || !table)
        return fail(MHC_E_INVALID, "poses and table must be non-NULL");
    if (int r = mhc::host::check_device_arrays(poses, table, nullptr)) return r;
    if (sc->n_objects < 1 || sc->n_objects > kMaxObjects)
        return fail(MHC_E_INVALID, "the allocation-free entry point takes 1 to 64 objects");
    if (sc->n_steps < 1 || sc->n_steps > MHC_MAX_STEPS) return fail(MHC_E_INVALID, "n_steps must be in [1, 32767]");
    if (sc->pair_mode != MHC_ALL_PAIRS && sc->pair_mode != MHC_EGO_ONLY) return fail(MHC_E_INVALID, "bad pair_mode");
    if (sc->ego < 0 || sc->ego >= sc->n_objects) return fail(MHC_E_INVALID, "ego out of range");
    if (sc->pair_mode == MHC_EGO_ONLY && sc->n_objects < 2) return fail(MHC_E_INVALID, "EGO_ONLY needs 2 objects");

    ObjDesc *objs = reinterpret_cast<ObjDesc *>(h_blob);
    PairDesc *pairs = reinterpret_cast<PairDesc *>(h_blob + kObjBytes);
    int *warp_obj = reinterpret_cast<int *>(h_blob + kObjBytes + kPairBytes);
    int *warp_first = reinterpret_cast<int *>(h_blob + kObjBytes + kPairBytes + kWarpBytes);
    const int N = sc->n_steps;
    long long traj = 0;
    int tiles32 = 0;
    for (int o = 0; o < sc->n_objects; ++o) {
        const mhc_object &src = sc->objects[o];
        ObjDesc &d = objs[o];
        std::memset(&d, 0, sizeof d);
        if (src.kind != MHC_VEHICLE && src.kind != MHC_PEDESTRIAN) return fail(MHC_E_INVALID, "bad object kind");
        if (src.n_vertices != 0)
            return fail(MHC_E_INVALID, "the static entry point takes rectangles only (n_vertices must be 0)");
        if (src.n_a < 1 || src.n_b < 1 || (long long)src.n_a * src.n_b > (1LL << 30))
            return fail(MHC_E_INVALID, "hypothesis grid sizes out of range");
        d.kind = src.kind;
        d.n_a = src.n_a;
        d.n_b = src.n_b;
        d.h = src.n_a * src.n_b;
        d.traj_off = traj;
        d.pose_base = traj * (long long)N;
        d.bounds_base = (long long)tiles32 * N;
        d.n_steps = N;
        traj += d.h;
        d.tile_base = tiles32;
        d.n_tiles32 = (d.h + kBoundTile - 1) / kBoundTile;
        if (tiles32 + d.n_tiles32 > kMaxWarps) return fail(MHC_E_INVALID, "more than 524,288 hypotheses");
        for (int q = 0; q < d.n_tiles32; ++q) {
            warp_obj[tiles32 + q] = o;
            warp_first[tiles32 + q] = q * kBoundTile;
        }
        tiles32 += d.n_tiles32;
        if (src.kind == MHC_VEHICLE) {
            if (!(src.length > 0.f) || !(src.width > 0.f) || !finite(src.length) || !finite(src.width))
                return fail(MHC_E_INVALID, "vehicle needs positive length and width");
            d.hl = 0.5f * src.length;
            d.hw = 0.5f * src.width;
            d.circ = (float)std::sqrt((double)d.hl * d.hl + (double)d.hw * d.hw);
        } else {
            if (!(src.radius > 0.f) || !finite(src.radius)) return fail(MHC_E_INVALID, "pedestrian needs a positive radius");
            d.rad = src.radius;
            d.circ = src.radius;
        }
    }
    int n_pairs = 0;
    long long entries = 0, tiles = 0;
    for (int a = 0; a < sc->n_objects; ++a) {
        for (int b = 0; b < sc->n_objects; ++b) {
            const bool take = sc->pair_mode == MHC_EGO_ONLY ? (a == sc->ego && b != a) : (b > a);
            if (!take) continue;
            PairDesc &p = pairs[n_pairs++];
            std::memset(&p, 0, sizeof p);
            const ObjDesc &A = objs[a], &B = objs[b];
            p.a = a;
            p.b = b;
            p.tiles_a = (A.h + kTile - 1) / kTile;
            p.tiles_b = (B.h + kTile - 1) / kTile;
            p.off = entries;
            p.tile_start = tiles;
            const double R = (double)A.circ + (double)B.circ;
            p.rc2 = (float)(R * R * (1.0 + 1e-6));
            p.r_cull = (float)(R * (1.0 + 1e-6) + 1e-3);
            p.combo = (A.kind == MHC_VEHICLE ? 0 : 2) + (B.kind == MHC_VEHICLE ? 0 : 1);
            p.ego_side = a == sc->ego ? 0 : (b == sc->ego ? 1 : -1);
            p.n_steps = N;
            p.index = n_pairs - 1;
            mhc::host::copy_object_fields(p, A, B);
            entries += (long long)A.h * B.h;
            tiles += (long long)p.tiles_a * p.tiles_b;
        }
    }
    if (tiles > 0x7fffffffLL) return fail(MHC_E_INVALID, "too many collision tiles for one launch");
    const size_t bounds_bytes = sizeof(float4) * (size_t)tiles32 * N;
    if (kDescBytes + bounds_bytes > kStaticScratchBytes) {
        char msg[160];
        std::snprintf(msg, sizeof msg, "scenario needs %zu bytes of static scratch; the limit is %zu bytes",
                      kDescBytes + bounds_bytes, kStaticScratchBytes);
        return fail(MHC_E_INVALID, msg);
    }

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaStreamCaptureStatus capturing = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &capturing);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamIsCapturing");
    if (capturing != cudaStreamCaptureStatusNone)
        return fail(MHC_E_INVALID, "the allocation-free entry point does not run on a stream in capture");
    void *base = nullptr;
    if (int r = scratch_address(&base)) return r;
    unsigned char *dev = static_cast<unsigned char *>(base);
    // Only the used part of each descriptor region is copied.  The source is pageable, so each copy has
    // read h_blob by the time cudaMemcpyAsync returns.
    const size_t parts[4][2] = {{0, sizeof(ObjDesc) * sc->n_objects},
                                {kObjBytes, sizeof(PairDesc) * n_pairs},
                                {kObjBytes + kPairBytes, sizeof(int) * tiles32},
                                {kObjBytes + kPairBytes + kWarpBytes, sizeof(int) * tiles32}};
    for (const auto &part : parts) {
        if (!part[1]) continue;
        e = cudaMemcpyAsync(dev + part[0], h_blob + part[0], part[1], cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(descriptors)");
    }
    const ObjDesc *d_objs = reinterpret_cast<const ObjDesc *>(dev);
    const PairDesc *d_pairs = reinterpret_cast<const PairDesc *>(dev + kObjBytes);
    const int *d_warp_obj = reinterpret_cast<const int *>(dev + kObjBytes + kPairBytes);
    const int *d_warp_first = reinterpret_cast<const int *>(dev + kObjBytes + kPairBytes + kWarpBytes);
    float4 *d_bounds = reinterpret_cast<float4 *>(dev + kDescBytes);

    BoundsArgs b{};
    b.objs = d_objs;
    b.warp_obj = d_warp_obj;
    b.warp_first = d_warp_first;
    b.n_warps = tiles32;
    b.max_steps = N;
    b.x = poses->x;
    b.y = poses->y;
    b.bounds = d_bounds;
    if ((e = launch_fill_table(table, entries, st)) != cudaSuccess) return cuda_fail(e, "table fill launch");
    if ((e = launch_bounds(b, st)) != cudaSuccess) return cuda_fail(e, "bounds kernel launch");
    CollideArgs c{};
    c.objs = d_objs;
    c.pairs = d_pairs;
    c.n_pairs = n_pairs;
    c.n_obj = sc->n_objects;
    c.n_tiles = tiles;
    c.max_steps = N;
    c.cull = 1;
    c.x = poses->x;
    c.y = poses->y;
    c.c = poses->c;
    c.s = poses->s;
    c.bounds = d_bounds;
    c.table = table;
    c.counters = nullptr;
    if ((e = launch_collide(c, st)) != cudaSuccess) return cuda_fail(e, "collision kernel launch");
    return MHC_OK;
}
