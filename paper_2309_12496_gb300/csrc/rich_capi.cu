// rich_capi.cu -- the C ABI (rich.h): context, geometry upload, emission,
// trace and counter read-back. Host code only; every step of the photon
// path itself runs in the kernels of rich_kernels.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "rich_bvh.h"
#include "rich_internal.h"

using namespace rich;

// A counter slot: a trace's counters and, right after them, the photon
// total that trace saw, so one copy reads both.
constexpr size_t kCtrBytes = sizeof(Counters) + sizeof(unsigned long long);
// Default trace block: 512 threads of the 64-register build, two blocks per
// SM (32 warps). Faster than one block of 1024 on the mesh and analytic
// scenes alike (RICH1 -4 %, forward + adjoint -5 %).
constexpr int kDefaultThreads = 512;
static_assert(sizeof(Counters) % 8 == 0, "the photon total follows the counters");

// One step of rich_run_host / rich_run_host_async: where its counters land
// (pinned), the event after its copies, and what its completion copies.
struct RunSlot {
    Counters *h_ctr = nullptr;
    unsigned long long *h_total = nullptr;
    cudaEvent_t ev = nullptr;              // the step's kernels and counters' copy
    cudaEvent_t ev_h2d = nullptr;          // its tracks on the device
    cudaEvent_t ev_copy = nullptr;         // its early hit copy (copy stream)
    void *d_tracks = nullptr;              // its device copy of the host tracks
    size_t d_tracks_bytes = 0;
    bool in_flight = false;
    uint64_t ticket = 0;
    rich_hit *host_hits = nullptr;
    uint64_t host_cap = 0, early = 0;
    const rich_hit *dev_hits = nullptr;
    uint64_t dev_cap = 0;
};

struct rich_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int n_sm = 1;
    std::string err;
    // geometry (one device allocation, sub-allocated)
    bool has_geometry = false;
    void *d_geom = nullptr;
    SceneView sc{};
    int bvh_depth = 0;
    // emission scratch
    int64_t track_cap = 0;
    TrackRec *d_rec = nullptr;
    float4 *d_cs = nullptr;
    TrackFrame *d_frame = nullptr;
    uint32_t *d_counts = nullptr;
    uint64_t *d_offsets = nullptr;
    unsigned long long *d_bsum = nullptr;
    bool has_emission = false;
    int64_t n_tracks = 0;
    // azimuth order of each track's photons (sized from the last photon
    // total the host has seen; an emission that does not fit keeps index
    // order, flagged on the device)
    uint2 *d_perm = nullptr;
    uint64_t perm_cap = 0;
    uint32_t *d_perm_ok = nullptr;
    uint64_t known_total = 0;
    uint32_t key0 = 0, key1 = 0;
    float inv1 = 0.f, span = 0.f;
    int32_t source = RICH_SOURCE_CHERENKOV;   // light source of the last emission
    int32_t spectrum = -1;                    // its CDF table, or -1
    int32_t dispersion = 0;                   // its radiator: 1 dispersive
    float disp_a = 0.f, disp_lambda0 = 0.f;
    std::vector<int32_t> table_kind;          // kinds of the scene's tables (host)
    bool has_dielectric = false;              // the scene refracts (window faces)
    // small device state: counters + photon total
    Counters *d_ctr = nullptr;              // the last trace's counter slot
    unsigned long long *d_total = nullptr; // the last emission's photon total
    // two counter slots, each [Counters | the trace's photon total]: a trace
    // counts into one and zeroes the other for the next trace, so the next
    // trace needs no reset before its launch
    Counters *d_ctr_slot[2] = {nullptr, nullptr};   // slot 0 is the allocation
    int cur_slot = 0;
    bool slot_zeroed[2] = {true, true};
    bool capturing = false;                // inside rich_graph_capture
    // kernel timing (rich_set_timing): events around the kernels of the
    // last rich_emit (0 yield, 1 ordering, 2 end) and rich_trace (3 trace,
    // 4 refinement, 5 end); recorded[k]: event k belongs to the last call
    bool timing = false;
    cudaEvent_t tev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    bool tev_emit = false, tev_trace = false, tev_refine = false;
    // counting build of the trace (rich_trace_work): 6 device tallies
    unsigned long long *d_work = nullptr;
    int graph_slot = 0;
    Counters *h_ctr = nullptr;            // pinned
    unsigned long long *h_total = nullptr; // pinned
    // last trace
    bool traced = false;
    bool last_ext = false;
    uint64_t last_ext_n = 0;
    uint64_t last_capacity = 0;
    // refinement side records, one per storable hit
    RefineRec *d_refine = nullptr;
    uint64_t refine_cap = 0;
    // occupancy per (external, refine, threads, smem), queried once
    std::map<std::tuple<bool, bool, int, int, size_t>, int> occupancy;
    int smem_optin = 48 * 1024;
    // gradient: nominal tiles (host), their frames (device), tilted copies
    std::vector<rich_sphere> nom_spheres;
    void *d_grad_tiles = nullptr;          // groups + tiles + tile duals at theta
    double *d_acc = nullptr;               // 12 FP64 accumulators
    double *h_acc = nullptr;               // pinned
    // captured emit + trace (CUDA graph) and the stream it was captured on
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    cudaStream_t capture_stream = nullptr;
    uint64_t graph_capacity = 0;
    // rich_run_host*: the hit count of the last completed step (sizes the
    // next step's early hit copy), the step slots and their copy streams
    uint64_t run_host_hits = 0;
    RunSlot run_slots[3];                  // [0], [1]: the asynchronous ring; [2]: the
                                           // synchronous call
    uint64_t next_ticket = 1;
    cudaStream_t copy_stream = nullptr;    // device-to-host copies of the steps' hits
    cudaStream_t up_stream = nullptr;      // host-to-device copies of the steps' tracks
    // the last emission left its count scan to the ordering pass
    bool scan_pending = false;
};

static thread_local std::string g_create_error;

namespace rich {
void set_global_error(const std::string &msg) { g_create_error = msg; }
}  // namespace rich

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

rich_status fail(rich_ctx *c, rich_status st, const std::string &msg) {
    if (c) c->err = msg;
    return st;
}

rich_status cuda_fail(rich_ctx *c, cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();
    return fail(c, e == cudaErrorMemoryAllocation ? RICH_ERR_OOM : RICH_ERR_CUDA, m);
}

#define RICH_CUDA(call)                                              \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);     \
    } while (0)

bool finite3(const float *v) {
    return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]);
}

// Tiles sharing one sphere (identical FP32 centre and radius) form a group:
// the sphere quadratic is solved once per group.
bool group_tiles(const rich_sphere *sp, int n, int n_materials,
                 std::vector<DevSphereGroup> &groups, std::vector<DevTile> &tiles,
                 std::string &err) {
    groups.clear();
    tiles.clear();
    std::vector<int> tile_group(n);
    std::vector<std::tuple<float, float, float, float>> spheres;
    for (int i = 0; i < n; ++i) {
        const rich_sphere &s = sp[i];
        if (!finite3(s.center) || !finite3(s.axis) || !finite3(s.e1) || !finite3(s.e2) ||
            !(s.radius > 0.f) || !std::isfinite(s.radius)) {
            err = "sphere tile with non-finite or non-positive values";
            return false;
        }
        if (s.n_edges < 0 || s.n_edges > RICH_SPHERE_MAX_EDGES) {
            err = "sphere tile edges 0..8";
            return false;
        }
        if (s.material < 0 || s.material >= n_materials) {
            err = "sphere material index";
            return false;
        }
        auto key = std::make_tuple(s.center[0], s.center[1], s.center[2], s.radius);
        auto it = std::find(spheres.begin(), spheres.end(), key);
        if (it == spheres.end()) {
            spheres.push_back(key);
            tile_group[i] = (int)spheres.size() - 1;
        } else {
            tile_group[i] = (int)(it - spheres.begin());
        }
    }
    if ((int)spheres.size() > RICH_MAX_GROUPS) {
        err = "more than 16 distinct spheres";
        return false;
    }
    groups.resize(spheres.size());
    for (size_t gi = 0; gi < spheres.size(); ++gi) {
        DevSphereGroup &G = groups[gi];
        G.fcx = std::get<0>(spheres[gi]);
        G.fcy = std::get<1>(spheres[gi]);
        G.fcz = std::get<2>(spheres[gi]);
        const double R = std::get<3>(spheres[gi]);
        G.radius = (float)R;
        G.inv_radius = (float)(1.0 / R);
        G.first = (int)tiles.size();
        for (int i = 0; i < n; ++i) {
            if (tile_group[i] != (int)gi) continue;
            const rich_sphere &s = sp[i];
            DevTile T;
            std::memset(&T, 0, sizeof T);
            T.ax = s.axis[0]; T.ay = s.axis[1]; T.az = s.axis[2]; T.cos_min = s.cos_min;
            T.e1x = s.e1[0]; T.e1y = s.e1[1]; T.e1z = s.e1[2];
            T.inv_radius = (float)(1.0 / (double)s.radius);
            T.e2x = s.e2[0]; T.e2y = s.e2[1]; T.e2z = s.e2[2];
            T.n_edges = s.n_edges;
            T.material = s.material;
            T.group = (int)gi;
            T.prim = i;
            for (int e = 0; e < s.n_edges; ++e)
                for (int k = 0; k < 3; ++k) T.edges[e][k] = s.edges[e][k];
            tiles.push_back(T);
        }
        G.count = (int)tiles.size() - G.first;
    }
    return true;
}

// Rodrigues rotation of v about the unit axis u by phi (FP64).
void rotate(const double u[3], double phi, double v[3]) {
    const double c = std::cos(phi), s = std::sin(phi);
    const double uv = u[0] * v[0] + u[1] * v[1] + u[2] * v[2];
    const double x[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2],
                         u[0] * v[1] - u[1] * v[0]};
    for (int k = 0; k < 3; ++k) v[k] = v[k] * c + x[k] * s + u[k] * uv * (1.0 - c);
}

// Tile i at the parameters theta: rotated about its pole by theta[2i] (about
// its nominal e1) then theta[2i+1] (about its nominal e2) for i < 4, radius
// theta[8], centre = pole - radius * axis.
rich_sphere tile_at_theta(const rich_sphere &s, int i, const double theta[10]) {
    const double R0 = s.radius;
    double P[3], a[3], e1[3], e2[3], u1[3], u2[3];
    for (int k = 0; k < 3; ++k) {
        P[k] = (double)s.center[k] + R0 * s.axis[k];
        a[k] = s.axis[k];
        e1[k] = s.e1[k];
        e2[k] = s.e2[k];
        u1[k] = s.e1[k];
        u2[k] = s.e2[k];
    }
    if (i < 4) {
        for (double *v : {a, e1, e2}) {
            rotate(u1, theta[2 * i], v);
            rotate(u2, theta[2 * i + 1], v);
        }
    }
    rich_sphere t = s;
    const double R = theta[8];
    for (int k = 0; k < 3; ++k) {
        t.center[k] = (float)(P[k] - R * a[k]);
        t.axis[k] = (float)a[k];
        t.e1[k] = (float)e1[k];
        t.e2[k] = (float)e2[k];
    }
    t.radius = (float)R;
    return t;
}

// Centre of tile i at theta with its first derivatives, for the adjoint.
// With a1 = M(e1, alpha) a0 and a = M(e2, beta) a1 (rotations about the
// fixed nominal axes, as tile_at_theta), the derivative of a rotation about
// a fixed unit axis u is u x (rotated vector): da/dbeta = e2 x a and
// da/dalpha = M(e2, beta) (e1 x a1); C = P - R a gives dC = -R da and
// dC/dR = -a. The centre is stored as a double-word, hi + lo per axis.
DevTileDual tile_dual(const rich_sphere &s, int i, const double theta[10]) {
    const double R0 = s.radius, R = theta[8];
    double P[3], a[3], u1[3], u2[3], da_dal[3] = {0, 0, 0}, da_dbe[3] = {0, 0, 0};
    for (int k = 0; k < 3; ++k) {
        P[k] = (double)s.center[k] + R0 * s.axis[k];
        a[k] = s.axis[k];
        u1[k] = s.e1[k];
        u2[k] = s.e2[k];
    }
    auto cross = [](const double x[3], const double y[3], double r[3]) {
        r[0] = x[1] * y[2] - x[2] * y[1];
        r[1] = x[2] * y[0] - x[0] * y[2];
        r[2] = x[0] * y[1] - x[1] * y[0];
    };
    if (i < 4) {
        rotate(u1, theta[2 * i], a);            // a1
        cross(u1, a, da_dal);                   // d a1 / d alpha
        rotate(u2, theta[2 * i + 1], da_dal);
        rotate(u2, theta[2 * i + 1], a);        // a
        cross(u2, a, da_dbe);
    }
    DevTileDual D{};
    for (int k = 0; k < 3; ++k) {
        const double c = P[k] - R * a[k];
        D.c_hi[k] = (float)c;
        D.c_lo[k] = (float)(c - (double)D.c_hi[k]);
        D.dc_dalpha[k] = (float)(-R * da_dal[k]);
        D.dc_dbeta[k] = (float)(-R * da_dbe[k]);
        D.dc_dr[k] = (float)(-a[k]);
    }
    return D;
}

// Device scratch of the gradient: sphere groups and tiles at theta, then
// the tiles' dual centres.
size_t grad_tiles_bytes() {
    return sizeof(DevSphereGroup) * RICH_MAX_GROUPS + sizeof(DevTile) * RICH_MAX_TILES +
           sizeof(DevTileDual) * RICH_MAX_TILES;
}

// A captured graph refers to the context's buffers: drop it before any of
// them is freed or replaced (rich_graph_launch then reports that nothing
// is captured).
void drop_graph(rich_ctx *ctx) {
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    if (ctx->graph) cudaGraphDestroy(ctx->graph);
    ctx->graph_exec = nullptr;
    ctx->graph = nullptr;
}

void free_emission(rich_ctx *ctx) {
    drop_graph(ctx);
    cudaFree(ctx->d_rec);
    cudaFree(ctx->d_cs);
    cudaFree(ctx->d_frame);
    cudaFree(ctx->d_counts);
    cudaFree(ctx->d_offsets);
    cudaFree(ctx->d_bsum);
    ctx->d_rec = nullptr;
    ctx->d_cs = nullptr;
    ctx->d_frame = nullptr;
    ctx->d_counts = nullptr;
    ctx->d_offsets = nullptr;
    ctx->d_bsum = nullptr;
    ctx->track_cap = 0;
}

// The last emission as the kernels see it.
EmitView emit_view(const rich_ctx *ctx) {
    EmitView em{ctx->d_rec, ctx->d_cs, ctx->d_offsets, ctx->d_total, ctx->n_tracks,
                ctx->key0, ctx->key1, ctx->inv1, ctx->span, ctx->d_perm, ctx->d_perm_ok,
                ctx->source, ctx->spectrum, ctx->dispersion, ctx->disp_a, ctx->disp_lambda0,
                ctx->d_frame};
    return em;
}

// Yield, Poisson counts and photon offsets of the tracks into the context's
// scratch (asynchronous).
rich_status emit_core(rich_ctx *ctx, const rich_tracks *t, uint64_t seed, float n_minus_1,
                      float lambda_min, float lambda_max, int32_t source = RICH_SOURCE_CHERENKOV,
                      float yield_per_mm = 0.f, int32_t spectrum = -1, int32_t dispersion = 0,
                      float disp_a = 0.f, float disp_lambda0 = 0.f, bool defer_scan = false) {
    const int64_t n = t->n;
    if (n + 1 > ctx->track_cap) {
        RICH_CUDA(cudaStreamSynchronize(ctx->stream));
        free_emission(ctx);
        const int64_t cap = std::max<int64_t>(n + 1, 1024);
        const int64_t blocks = (cap + yield_block_threads() - 1) / yield_block_threads();
        RICH_CUDA(cudaMalloc(&ctx->d_rec, sizeof(TrackRec) * cap));
        RICH_CUDA(cudaMalloc(&ctx->d_cs, sizeof(float4) * cap));
        RICH_CUDA(cudaMalloc(&ctx->d_frame, sizeof(TrackFrame) * cap));
        RICH_CUDA(cudaMalloc(&ctx->d_counts, sizeof(uint32_t) * cap));
        RICH_CUDA(cudaMalloc(&ctx->d_offsets, sizeof(uint64_t) * (cap + 1)));
        RICH_CUDA(cudaMalloc(&ctx->d_bsum, sizeof(unsigned long long) * (blocks + 1)));
        ctx->track_cap = cap;
    }
    ctx->key0 = (uint32_t)seed;
    ctx->key1 = (uint32_t)(seed >> 32);
    {
        // FP32 spectrum constants, one IEEE operation each
        volatile float l1 = lambda_min, l2 = lambda_max;
        volatile float inv1 = 1.0f / l1;
        volatile float inv2 = 1.0f / l2;
        volatile float span = inv1 - inv2;
        ctx->inv1 = inv1;
        ctx->span = span;
    }
    TracksView tv{n, t->x, t->y, t->z, t->dx, t->dy, t->dz, t->p, t->mass, t->length,
                  t->event, t->id, t->n_fixed};
    if (n == 0) {
        RICH_CUDA(cudaMemsetAsync(ctx->d_total, 0, sizeof(unsigned long long), ctx->stream));
        RICH_CUDA(cudaMemsetAsync(ctx->d_offsets, 0, sizeof(uint64_t), ctx->stream));
    } else {
        RICH_CUDA(launch_yield(tv, (double)n_minus_1, lambda_min, lambda_max, ctx->key0,
                               ctx->key1, ctx->d_rec, ctx->d_cs, ctx->d_counts, ctx->d_bsum,
                               ctx->stream,
                               YieldModel{source == RICH_SOURCE_ISOTROPIC ? (double)yield_per_mm
                                                                          : -1.0,
                                          dispersion, disp_a, disp_lambda0},
                               ctx->d_frame, ctx->d_perm_ok));
        // deferred: the ordering pass (order_photons, which the caller
        // runs next) does the scan
        ctx->scan_pending = defer_scan && n <= kOrderScanMaxTracks;
        if (!ctx->scan_pending)
            RICH_CUDA(launch_offsets(ctx->d_counts, ctx->d_bsum, n, ctx->d_offsets,
                                     ctx->d_total, ctx->stream));
    }
    ctx->n_tracks = n;
    ctx->source = source;
    ctx->spectrum = source == RICH_SOURCE_ISOTROPIC ? spectrum : -1;
    ctx->dispersion = dispersion;
    ctx->disp_a = disp_a;
    ctx->disp_lambda0 = disp_lambda0;
    ctx->has_emission = true;
    return RICH_OK;
}

// Azimuth order of the photons of the last emission. The buffer is sized
// from the largest photon total the host has read (with a margin); an
// emission that does not fit is traced in index order (device flag).
rich_status order_photons(rich_ctx *ctx) {
    const uint64_t want = ctx->known_total + ctx->known_total / 4 + 1024;
    if (ctx->known_total && want > ctx->perm_cap) {
        RICH_CUDA(cudaStreamSynchronize(ctx->stream));
        drop_graph(ctx);
        cudaFree(ctx->d_perm);
        ctx->d_perm = nullptr;
        ctx->perm_cap = 0;
        RICH_CUDA(cudaMalloc(&ctx->d_perm, sizeof(uint2) * want));
        ctx->perm_cap = want;
    }
    const EmitView em = emit_view(ctx);
    if (ctx->n_tracks == 0) {
        ctx->scan_pending = false;
        RICH_CUDA(cudaMemsetAsync(ctx->d_perm_ok, 0, sizeof(uint32_t), ctx->stream));
        return RICH_OK;
    }
    const OrderScan scan{ctx->d_counts, ctx->d_bsum, ctx->d_offsets, ctx->d_total};
    RICH_CUDA(launch_order(em, ctx->d_perm, ctx->perm_cap, ctx->d_perm_ok, ctx->n_sm,
                           ctx->stream, ctx->scan_pending ? &scan : nullptr));
    ctx->scan_pending = false;
    return RICH_OK;
}

}  // namespace

extern "C" {

RICH_API const char *rich_version(void) { return "rich-gb300 0.1 (sm_103a)"; }

RICH_API const char *rich_last_error(rich_ctx *ctx) {
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

RICH_API rich_status rich_create(rich_ctx **out, int device, void *stream) {
    if (!out) {
        g_create_error = "rich_create: out is NULL";
        return RICH_ERR_ARG;
    }
    *out = nullptr;
    int n_dev = 0;
    cudaError_t e = cudaGetDeviceCount(&n_dev);
    if (e != cudaSuccess || device < 0 || device >= n_dev) {
        g_create_error = std::string("rich_create: no CUDA device ") + std::to_string(device) +
                         (e != cudaSuccess ? std::string(" (") + cudaGetErrorString(e) + ")" : "");
        cudaGetLastError();
        return e != cudaSuccess ? RICH_ERR_CUDA : RICH_ERR_ARG;
    }
    rich_ctx *ctx = new rich_ctx();
    ctx->device = device;
    ctx->stream = static_cast<cudaStream_t>(stream);
    DeviceGuard g(device);
    cudaDeviceProp prop;
    if ((e = cudaGetDeviceProperties(&prop, device)) != cudaSuccess ||
        (e = cudaMalloc(&ctx->d_ctr, 2 * kCtrBytes + sizeof(unsigned long long))) != cudaSuccess ||
        (e = cudaMalloc(&ctx->d_perm_ok, sizeof(uint32_t))) != cudaSuccess ||
        (e = cudaMemset(ctx->d_perm_ok, 0, sizeof(uint32_t))) != cudaSuccess ||
        (e = cudaMallocHost(&ctx->h_ctr, kCtrBytes)) != cudaSuccess ||
        (e = cudaMemset(ctx->d_ctr, 0, 2 * kCtrBytes + sizeof(unsigned long long))) !=
            cudaSuccess) {
        g_create_error = std::string("rich_create: ") + cudaGetErrorString(e);
        cudaGetLastError();
        cudaFree(ctx->d_ctr);
        cudaFree(ctx->d_perm_ok);
        cudaFreeHost(ctx->h_ctr);
        delete ctx;
        return e == cudaErrorMemoryAllocation ? RICH_ERR_OOM : RICH_ERR_CUDA;
    }
    // slot k at d_ctr + k kCtrBytes holds the counters and the trace's photon
    // total (one copy reads both); the emission's total follows the slots
    {
        char *base = reinterpret_cast<char *>(ctx->d_ctr);
        ctx->d_ctr_slot[0] = reinterpret_cast<Counters *>(base);
        ctx->d_ctr_slot[1] = reinterpret_cast<Counters *>(base + kCtrBytes);
        ctx->d_total = reinterpret_cast<unsigned long long *>(base + 2 * kCtrBytes);
    }
    ctx->h_total = reinterpret_cast<unsigned long long *>(ctx->h_ctr + 1);
    ctx->n_sm = prop.multiProcessorCount;
    ctx->smem_optin = (int)prop.sharedMemPerBlockOptin;
    *out = ctx;
    return RICH_OK;
}

RICH_API rich_status rich_destroy(rich_ctx *ctx) {
    if (!ctx) return RICH_OK;
    {
        DeviceGuard g(ctx->device);
        cudaStreamSynchronize(ctx->stream);
        // steps never waited for: their copies finish before their buffers go
        if (ctx->up_stream) cudaStreamSynchronize(ctx->up_stream);
        if (ctx->copy_stream) cudaStreamSynchronize(ctx->copy_stream);
        cudaFree(ctx->d_geom);
        cudaFree(ctx->d_refine);
        cudaFree(ctx->d_grad_tiles);
        for (RunSlot &S : ctx->run_slots) {
            cudaFreeHost(S.h_ctr);
            cudaFree(S.d_tracks);
            if (S.ev) cudaEventDestroy(S.ev);
            if (S.ev_h2d) cudaEventDestroy(S.ev_h2d);
            if (S.ev_copy) cudaEventDestroy(S.ev_copy);
        }
        if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
        if (ctx->up_stream) cudaStreamDestroy(ctx->up_stream);
        if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
        if (ctx->graph) cudaGraphDestroy(ctx->graph);
        if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
        cudaFree(ctx->d_acc);
        cudaFreeHost(ctx->h_acc);
        cudaFree(ctx->d_work);
        for (cudaEvent_t &e : ctx->tev)
            if (e) cudaEventDestroy(e);
        free_emission(ctx);
        cudaFree(ctx->d_perm);
        cudaFree(ctx->d_perm_ok);
        cudaFree(ctx->d_ctr_slot[0]);
        cudaFreeHost(ctx->h_ctr);
        cudaGetLastError();
    }
    delete ctx;
    return RICH_OK;
}

RICH_API rich_status rich_set_stream(rich_ctx *ctx, void *stream) {
    if (!ctx) return RICH_ERR_ARG;
    ctx->stream = static_cast<cudaStream_t>(stream);
    return RICH_OK;
}

// ---------------------------------------------------------------- geometry
RICH_API rich_status rich_init_geometry(rich_ctx *ctx, const rich_geometry_desc *g) {
    if (!ctx) return RICH_ERR_ARG;
    if (!g) return fail(ctx, RICH_ERR_ARG, "rich_init_geometry: desc is NULL");
    DeviceGuard guard(ctx->device);
    auto bad = [&](const std::string &m) { return fail(ctx, RICH_ERR_GEOMETRY, "rich_init_geometry: " + m); };
    if (g->n_tables < 0 || g->n_materials < 0 || g->n_spheres < 0 || g->n_rects < 0 ||
        g->n_triangles < 0)
        return bad("negative count");
    if (g->n_tables > RICH_MAX_TABLES) return bad("more than 8 tables");
    if (g->n_materials > RICH_MAX_MATERIALS) return bad("more than 32 materials");
    if (g->n_spheres > RICH_MAX_TILES) return bad("more than 64 sphere tiles");
    if (g->n_rects > RICH_MAX_RECTS) return bad("more than 32 rectangles");
    if ((g->n_tables && !g->tables) || (g->n_materials && !g->materials) ||
        (g->n_spheres && !g->spheres) || (g->n_rects && !g->rects) ||
        (g->n_triangles && (!g->tri_vertices || !g->tri_material)))
        return bad("NULL array with a non-zero count");
    for (int i = 0; i < g->n_tables; ++i) {
        const rich_table &t = g->tables[i];
        if (t.kind < 0 || t.kind > 3) return bad("table kind");
        if (t.kind == RICH_TABLE_CDF) {
            if (t.nbins < 1 || t.nbins > RICH_TABLE_MAX_BINS - 1 || !(t.p1 > 0.f) ||
                !std::isfinite(t.p0) || !std::isfinite(t.p1))
                return bad("spectrum (CDF) table needs 1..63 bins and a positive width");
            if (t.values[0] != 0.f || t.values[t.nbins] != 1.f)
                return bad("spectrum (CDF) table must run from 0 to 1");
            for (int k = 0; k < t.nbins; ++k)
                if (!(t.values[k + 1] >= t.values[k]))
                    return bad("spectrum (CDF) table must be nondecreasing");
        }
        if (t.kind == RICH_TABLE_HIST && (t.nbins < 1 || t.nbins > RICH_TABLE_MAX_BINS || !(t.p1 > 0.f)))
            return bad("histogram table needs 1..64 bins and a positive width");
        if (t.kind == RICH_TABLE_GAUSS && !(t.p2 != 0.f)) return bad("Gaussian table width is 0");
    }
    bool any_smooth = false;
    for (int i = 0; i < g->n_materials; ++i) {
        const rich_material &m = g->materials[i];
        if (m.kind < 0 || m.kind > 3) return bad("material kind");
        if (m.kind != RICH_MAT_ABSORBER && (m.table < 0 || m.table >= g->n_tables))
            return bad("material table index out of range");
        if (m.kind != RICH_MAT_ABSORBER && g->tables[m.table].kind == RICH_TABLE_CDF)
            return bad("a spectrum (CDF) table is not a response table");
        if (m.kind == RICH_MAT_DETECTOR && (m.plane < 0 || m.plane >= RICH_MAX_PLANES))
            return bad("detector plane index must be 0..7");
        if (m.flags & RICH_MAT_SMOOTH) any_smooth = true;
    }
    if (any_smooth && g->n_triangles && !g->tri_normals)
        return bad("smooth material without vertex normals");
    bool any_dielectric = false;
    for (int i = 0; i < g->n_materials; ++i)
        any_dielectric |= g->materials[i].kind == RICH_MAT_DIELECTRIC;
    for (int i = 0; i < g->n_spheres; ++i) {
        const int32_t mi = g->spheres[i].material;
        if (mi >= 0 && mi < g->n_materials && g->materials[mi].kind == RICH_MAT_DIELECTRIC)
            return bad("refracting (dielectric) material on a sphere tile");
    }
    // ---- sphere groups (tiles sharing a sphere)
    std::vector<DevSphereGroup> groups;
    std::vector<DevTile> tiles;
    {
        std::string gerr;
        if (!group_tiles(g->spheres, g->n_spheres, g->n_materials, groups, tiles, gerr))
            return bad(gerr);
    }
    // ---- rectangles and planes
    std::vector<DevRect> rects(g->n_rects);
    int plane_nx[RICH_MAX_PLANES] = {0}, plane_ny[RICH_MAX_PLANES] = {0};
    int n_planes = 0;
    for (int i = 0; i < g->n_rects; ++i) {
        const rich_rect &r = g->rects[i];
        if (!finite3(r.origin) || !finite3(r.u_axis) || !finite3(r.v_axis) || !finite3(r.normal) ||
            !(r.width > 0.f) || !(r.height > 0.f) || !std::isfinite(r.width) || !std::isfinite(r.height))
            return bad("rectangle with non-finite or non-positive values");
        if (r.material < 0 || r.material >= g->n_materials) return bad("rectangle material index");
        const rich_material &m = g->materials[r.material];
        DevRect &R = rects[i];
        std::memset(&R, 0, sizeof R);
        R.ox = r.origin[0]; R.oy = r.origin[1]; R.oz = r.origin[2]; R.w = r.width;
        R.ux = r.u_axis[0]; R.uy = r.u_axis[1]; R.uz = r.u_axis[2]; R.h = r.height;
        R.vx = r.v_axis[0]; R.vy = r.v_axis[1]; R.vz = r.v_axis[2]; R.pitch = r.pitch;
        R.nx = r.normal[0]; R.ny = r.normal[1]; R.nz = r.normal[2];
        R.material = r.material;
        R.gx = r.nx;
        R.gy = r.ny;
        R.plane = m.kind == RICH_MAT_DETECTOR ? m.plane : -1;
        R.prim = g->n_spheres + i;
        if (m.kind == RICH_MAT_DETECTOR) {
            if (r.nx <= 0 || r.ny <= 0 || r.nx > 65535 || r.ny > 65535 || !(r.pitch > 0.f))
                return bad("detector rectangle needs a pixel grid (1..65535) and a pitch");
            const double w = (double)r.nx * r.pitch, h = (double)r.ny * r.pitch;
            if (std::fabs(w - r.width) > 1e-3 * w || std::fabs(h - r.height) > 1e-3 * h)
                return bad("detector rectangle size differs from its pixel grid");
            if (plane_nx[m.plane] && (plane_nx[m.plane] != r.nx || plane_ny[m.plane] != r.ny))
                return bad("one detector plane index used with two grid shapes");
            plane_nx[m.plane] = r.nx;
            plane_ny[m.plane] = r.ny;
            n_planes = std::max(n_planes, m.plane + 1);
        }
    }
    // ---- triangles + BVH
    BvhResult bvh;
    std::string berr;
    const int64_t nt = g->n_triangles;
    for (int64_t i = 0; i < nt; ++i)
        if (g->tri_material[i] < 0 || g->tri_material[i] >= g->n_materials)
            return bad("triangle material index");
    if (!build_bvh(g->tri_vertices, g->tri_surface, nt, bvh, berr)) return bad(berr);
    if (bvh.depth >= RICH_BVH_STACK) return bad("BVH deeper than the traversal stack");
    // structural check: children point strictly forward (traversal ends),
    // leaf ranges stay inside the triangle array
    for (size_t i = 0; i < bvh.nodes.size(); ++i) {
        for (int c : bvh.nodes[i].child) {
            if (c == INT_MIN) continue;       // empty slot
            if (c >= 0) {
                if ((size_t)c <= i || (size_t)c >= bvh.nodes.size()) return bad("BVH child index");
            } else {
                const int code = ~c;
                const int64_t first = code >> 3, count = (code & 7) + 1;
                if (first + count > nt) return bad("BVH leaf range");
            }
        }
    }
    const int prim_base = g->n_spheres + g->n_rects;
    std::vector<DevTri> tris((size_t)nt);
    std::vector<DevTriRef> tri_ref((size_t)nt);
    std::vector<float> normals(any_smooth ? 9 * (size_t)nt : 0);
    auto split = [](double x, float *hl) {
        hl[0] = (float)x;
        hl[1] = (float)(x - (double)hl[0]);
    };
    for (int64_t k = 0; k < nt; ++k) {
        const int src = bvh.leaf_order[(size_t)k];
        const float *v = g->tri_vertices + 9 * (int64_t)src;
        DevTri &T = tris[(size_t)k];
        T.v0x = v[0]; T.v0y = v[1]; T.v0z = v[2];
        T.v1x = v[3]; T.v1y = v[4]; T.v1z = v[5];
        T.v2x = v[6]; T.v2y = v[7]; T.v2z = v[8];
        T.prim = prim_base + src;
        T.material = g->tri_material[src];
        T.pad = bvh.surface_ref[(size_t)k];   // subtree of the triangle's surface
        if (any_smooth) std::memcpy(&normals[9 * (size_t)k], g->tri_normals + 9 * (int64_t)src, 36);
        // refinement constants: the edges are exact in FP64 (differences of
        // FP32 numbers), their products too; one rounding per sum
        const double e1[3] = {(double)v[3] - v[0], (double)v[4] - v[1], (double)v[5] - v[2]};
        const double e2[3] = {(double)v[6] - v[0], (double)v[7] - v[1], (double)v[8] - v[2]};
        const double c[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                             e1[0] * e2[1] - e1[1] * e2[0]};
        const double cl = std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        DevTriRef &Q = tri_ref[(size_t)k];
        std::memset(&Q, 0, sizeof Q);
        for (int a = 0; a < 3; ++a) split(cl > 0.0 ? c[a] / cl : 0.0, Q.ng + 2 * a);
        const double d00 = e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2];
        const double d01 = e1[0] * e2[0] + e1[1] * e2[1] + e1[2] * e2[2];
        const double d11 = e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2];
        const double den = d00 * d11 - d01 * d01;
        split(d00, Q.d00);
        split(d01, Q.d01);
        split(d11, Q.d11);
        split(den != 0.0 ? 1.0 / den : 0.0, Q.inv_den);
    }
    std::vector<DevTable> tables(g->n_tables);
    for (int i = 0; i < g->n_tables; ++i) std::memcpy(&tables[i], &g->tables[i], sizeof(DevTable));
    std::vector<DevMaterial> mats(g->n_materials);
    for (int i = 0; i < g->n_materials; ++i) std::memcpy(&mats[i], &g->materials[i], sizeof(DevMaterial));

    // ---- one device allocation
    auto r256 = [](size_t b) { return (b + 255) & ~size_t(255); };
    size_t sizes[] = {sizeof(DevSphereGroup) * groups.size(), sizeof(DevTile) * tiles.size(),
                      sizeof(DevRect) * rects.size(), sizeof(DevTable) * tables.size(), sizeof(DevMaterial) * mats.size(),
                      sizeof(DevNode) * bvh.nodes.size(), sizeof(DevTri) * tris.size(),
                      sizeof(float) * normals.size(), sizeof(DevTriRef) * tri_ref.size()};
    const void *srcs[] = {groups.data(), tiles.data(), rects.data(), tables.data(), mats.data(), bvh.nodes.data(), tris.data(),
                          normals.data(), tri_ref.data()};
    size_t total = 0, offs[9];
    for (int i = 0; i < 9; ++i) {
        offs[i] = total;
        total += r256(sizes[i]);
    }
    RICH_CUDA(cudaStreamSynchronize(ctx->stream));
    drop_graph(ctx);
    cudaFree(ctx->d_geom);
    ctx->d_geom = nullptr;
    ctx->has_geometry = false;
    void *buf = nullptr;
    RICH_CUDA(cudaMalloc(&buf, std::max<size_t>(total, 256)));
    ctx->d_geom = buf;
    for (int i = 0; i < 9; ++i)
        if (sizes[i]) RICH_CUDA(cudaMemcpy((char *)buf + offs[i], srcs[i], sizes[i], cudaMemcpyHostToDevice));
    SceneView sc{};
    auto at = [&](int i) { return sizes[i] ? (const void *)((char *)buf + offs[i]) : nullptr; };
    sc.groups = (const DevSphereGroup *)at(0);
    sc.tiles = (const DevTile *)at(1);
    sc.rects = (const DevRect *)at(2);
    sc.tables = (const DevTable *)at(3);
    sc.materials = (const DevMaterial *)at(4);
    sc.nodes = (const DevNode *)at(5);
    sc.tris = (const DevTri *)at(6);
    sc.tri_normals = (const float *)at(7);
    sc.tri_ref = (const DevTriRef *)at(8);
    sc.n_groups = (int)groups.size();
    sc.n_tiles = (int)tiles.size();
    sc.n_rects = (int)rects.size();
    sc.n_tables = (int)tables.size();
    sc.n_materials = (int)mats.size();
    sc.n_nodes = (int)bvh.nodes.size();
    sc.n_tris = nt;
    sc.tri_prim_base = prim_base;
    sc.n_planes = n_planes;
    int64_t off = 0;
    for (int p = 0; p < RICH_MAX_PLANES; ++p) {
        sc.plane_offset[p] = off;
        sc.plane_nx[p] = plane_nx[p];
        if (p < n_planes) off += (int64_t)plane_nx[p] * plane_ny[p];
    }
    sc.pixels_per_event = off;
    ctx->sc = sc;
    ctx->bvh_depth = bvh.depth;
    // nominal tiles for the gradient
    ctx->nom_spheres.assign(g->spheres, g->spheres + g->n_spheres);
    cudaFree(ctx->d_grad_tiles);
    ctx->d_grad_tiles = nullptr;
    if (g->n_spheres)
        RICH_CUDA(cudaMalloc(&ctx->d_grad_tiles, grad_tiles_bytes()));
    ctx->has_dielectric = any_dielectric;
    ctx->table_kind.assign(g->n_tables, 0);
    for (int i = 0; i < g->n_tables; ++i) ctx->table_kind[i] = g->tables[i].kind;
    ctx->has_geometry = true;
    return RICH_OK;
}

// ----------------------------------------------------------------- emission
RICH_API rich_status rich_emit(rich_ctx *ctx, const rich_tracks *t,
                               const rich_emit_params *prm, rich_photons *out,
                               uint64_t *n_photons) {
    if (!ctx) return RICH_ERR_ARG;
    if (!t || !prm) return fail(ctx, RICH_ERR_ARG, "rich_emit: tracks or params is NULL");
    if (t->n < 0 || t->n > (int64_t(1) << 31))
        return fail(ctx, RICH_ERR_ARG, "rich_emit: track count out of range");
    if (t->n > 0 && (!t->x || !t->y || !t->z || !t->dx || !t->dy || !t->dz || !t->p ||
                     !t->mass || !t->length || !t->event))
        return fail(ctx, RICH_ERR_ARG, "rich_emit: a required track array is NULL");
    if (!(prm->n_minus_1 >= 0.f) || !std::isfinite(prm->n_minus_1) || !(prm->lambda_min > 0.f) ||
        !(prm->lambda_max > prm->lambda_min) || !std::isfinite(prm->lambda_max))
        return fail(ctx, RICH_ERR_ARG, "rich_emit: need n-1 >= 0 and 0 < lambda_min < lambda_max");
    if (prm->source != RICH_SOURCE_CHERENKOV && prm->source != RICH_SOURCE_ISOTROPIC)
        return fail(ctx, RICH_ERR_ARG, "rich_emit: unknown light source");
    if (prm->source == RICH_SOURCE_ISOTROPIC) {
        if (!(prm->yield_per_mm >= 0.f) || !std::isfinite(prm->yield_per_mm))
            return fail(ctx, RICH_ERR_ARG, "rich_emit: isotropic source needs a finite yield_per_mm >= 0");
        if (prm->spectrum_table >= 0 &&
            (!ctx->has_geometry || prm->spectrum_table >= (int32_t)ctx->table_kind.size() ||
             ctx->table_kind[prm->spectrum_table] != RICH_TABLE_CDF))
            return fail(ctx, RICH_ERR_ARG,
                        "rich_emit: spectrum_table is not a CDF table of the loaded scene");
    }
    if (prm->dispersion != 0 && prm->dispersion != 1)
        return fail(ctx, RICH_ERR_ARG, "rich_emit: dispersion must be 0 or 1");
    if (prm->dispersion) {
        if (prm->source != RICH_SOURCE_CHERENKOV)
            return fail(ctx, RICH_ERR_ARG, "rich_emit: dispersion applies to the Cherenkov source");
        if (!(prm->disp_a > 0.f) || !std::isfinite(prm->disp_a) || !(prm->disp_lambda0 > 0.f) ||
            !(prm->lambda_min > prm->disp_lambda0))
            return fail(ctx, RICH_ERR_ARG,
                        "rich_emit: dispersion needs disp_a > 0 and 0 < disp_lambda0 < lambda_min");
    }
    DeviceGuard guard(ctx->device);
    const bool timed = ctx->timing && !ctx->capturing;
    if (timed) RICH_CUDA(cudaEventRecord(ctx->tev[0], ctx->stream));
    {
        const rich_status st = emit_core(ctx, t, prm->seed, prm->n_minus_1, prm->lambda_min,
                                         prm->lambda_max, prm->source, prm->yield_per_mm,
                                         prm->spectrum_table < 0 ? -1 : prm->spectrum_table,
                                         prm->dispersion, prm->disp_a, prm->disp_lambda0,
                                         /*defer_scan=*/!(n_photons || out));
        if (st != RICH_OK) return st;
    }
    if (n_photons || out) {
        RICH_CUDA(cudaMemcpyAsync(ctx->h_total, ctx->d_total, sizeof(unsigned long long),
                                  cudaMemcpyDeviceToHost, ctx->stream));
        RICH_CUDA(cudaStreamSynchronize(ctx->stream));
        ctx->known_total = std::max<uint64_t>(ctx->known_total, *ctx->h_total);
        if (n_photons) *n_photons = *ctx->h_total;
    }
    if (timed) RICH_CUDA(cudaEventRecord(ctx->tev[1], ctx->stream));
    {
        const rich_status st = order_photons(ctx);
        if (st != RICH_OK) return st;
    }
    if (timed) {
        RICH_CUDA(cudaEventRecord(ctx->tev[2], ctx->stream));
        ctx->tev_emit = true;
    }
    if (out) {
        const uint64_t total = *ctx->h_total;
        if (total > out->capacity)
            return fail(ctx, RICH_ERR_OVERFLOW, "rich_emit: photon capacity " +
                                                    std::to_string(out->capacity) + " < " +
                                                    std::to_string(total));
        if (total && (!out->x || !out->y || !out->z || !out->dx || !out->dy || !out->dz ||
                      !out->lambda || !out->event || !out->track || !out->photon))
            return fail(ctx, RICH_ERR_ARG, "rich_emit: a photon output array is NULL");
        const EmitView em = emit_view(ctx);
        RICH_CUDA(launch_materialize(ctx->sc, em, total, *out, ctx->stream));
        out->n = total;
    }
    return RICH_OK;
}

// -------------------------------------------------------------------- trace
// The counter slot of the next trace: the slot the last trace did not use,
// zeroed by that trace's kernel (else reset here; always inside a graph
// capture, whose replays reuse the captured pointers). next: the slot the
// trace kernel zeroes for the trace after it (none inside a capture).
static rich_status trace_counters(rich_ctx *ctx, Counters **slot, Counters **next) {
    const int s = ctx->cur_slot ^ 1;
    if (!ctx->slot_zeroed[s] || ctx->capturing)
        RICH_CUDA(cudaMemsetAsync(ctx->d_ctr_slot[s], 0, sizeof(Counters), ctx->stream));
    *slot = ctx->d_ctr_slot[s];
    *next = ctx->capturing ? nullptr : ctx->d_ctr_slot[ctx->cur_slot];
    return RICH_OK;
}

// After a trace's launches: its slot is the one rich_hits reads.
static void trace_counters_done(rich_ctx *ctx, bool next_zeroed) {
    const int s = ctx->cur_slot ^ 1;
    ctx->slot_zeroed[s] = false;
    ctx->slot_zeroed[ctx->cur_slot] = next_zeroed;
    ctx->cur_slot = s;
    ctx->d_ctr = ctx->d_ctr_slot[s];
}

// Iterations of the trace blocks' bounded wait for the shared-memory copy of
// the top BVH nodes: the option's value, 2^20 by default, none when negative.
static int32_t trace_wait_limit(int32_t opt) {
    return opt == 0 ? (1 << 20) : (opt < 0 ? 0 : opt);
}

// rich_trace, and its counting build for rich_trace_work (work: the device
// tallies, fused emission with refinement only).
static rich_status trace_impl(rich_ctx *ctx, const rich_photons *in, const rich_trace_opts *o,
                              const rich_outputs *out, unsigned long long *work) {
    if (!ctx) return RICH_ERR_ARG;
    if (!o || !out) return fail(ctx, RICH_ERR_ARG, "rich_trace: opts or outputs is NULL");
    if (!ctx->has_geometry) return fail(ctx, RICH_ERR_STATE, "rich_trace: no geometry");
    if (!in && !ctx->has_emission)
        return fail(ctx, RICH_ERR_STATE, "rich_trace: no photons (call rich_emit first)");
    if (o->precision != RICH_PREC_FP32 && o->precision != RICH_PREC_REFINE64)
        return fail(ctx, RICH_ERR_ARG, "rich_trace: precision");
    if (o->max_bounces < 1 || o->max_bounces > RICH_MAX_BOUNCES || o->max_steps < 1 ||
        o->max_steps > RICH_MAX_STEPS || !(o->t_min >= 0.f))
        return fail(ctx, RICH_ERR_ARG, "rich_trace: max_bounces 1..8, max_steps 1..16, t_min >= 0");
    if (out->hit_capacity && !out->hits)
        return fail(ctx, RICH_ERR_ARG, "rich_trace: hits is NULL with a non-zero capacity");
    if (in && in->n && (!in->x || !in->y || !in->z || !in->dx || !in->dy || !in->dz ||
                        !in->lambda || !in->event || !in->track || !in->photon))
        return fail(ctx, RICH_ERR_ARG, "rich_trace: a photon input array is NULL");
    const int threads = o->block_threads ? o->block_threads : kDefaultThreads;
    if (threads % 32 != 0 || threads < 32 || threads > 1024)
        return fail(ctx, RICH_ERR_ARG, "rich_trace: block_threads must be 32..1024, a multiple of 32");
    const int refill = o->refill_min ? o->refill_min : 32;
    if (refill < 1 || refill > 32) return fail(ctx, RICH_ERR_ARG, "rich_trace: refill_min 1..32");
    const int chunk = o->chunk ? o->chunk : 32;
    if (chunk < 1 || chunk > (1 << 20)) return fail(ctx, RICH_ERR_ARG, "rich_trace: chunk 1..2^20");
    if (o->n_prefilter < 0 || o->n_prefilter > 4)
        return fail(ctx, RICH_ERR_ARG, "rich_trace: n_prefilter 0..4");
    for (int k = 0; k < o->n_prefilter; ++k)
        if (o->prefilter_tables[k] < 0 || o->prefilter_tables[k] >= ctx->sc.n_tables)
            return fail(ctx, RICH_ERR_ARG, "rich_trace: prefilter table index outside the scene's tables");
    for (int k = 0; k < o->n_prefilter; ++k)
        if (ctx->table_kind[o->prefilter_tables[k]] == RICH_TABLE_CDF)
            return fail(ctx, RICH_ERR_ARG, "rich_trace: a spectrum (CDF) table is not a response table");
    if (!in && ctx->spectrum >= 0 &&
        (ctx->spectrum >= (int32_t)ctx->table_kind.size() ||
         ctx->table_kind[ctx->spectrum] != RICH_TABLE_CDF))
        return fail(ctx, RICH_ERR_STATE,
                    "rich_trace: the emission's spectrum table is not in the current scene");
    const int cls = trace_shape_class(threads, o->wide_regs != 0);
    int smem_nodes = o->bvh_smem_nodes;
    if (smem_nodes < 0) smem_nodes = threads > 256 ? 256 : 0;
    if (smem_nodes > ctx->sc.n_nodes) smem_nodes = ctx->sc.n_nodes;
    if (ctx->sc.n_tris == 0) smem_nodes = 0;
    DeviceGuard guard(ctx->device);
    const bool refine = o->precision == RICH_PREC_REFINE64;
    const uint64_t hit_cap = out->hits ? out->hit_capacity : 0;
    if (refine && hit_cap > ctx->refine_cap) {
        RICH_CUDA(cudaStreamSynchronize(ctx->stream));
        drop_graph(ctx);
        cudaFree(ctx->d_refine);
        ctx->d_refine = nullptr;
        ctx->refine_cap = 0;
        RICH_CUDA(cudaMalloc(&ctx->d_refine, sizeof(RefineRec) * hit_cap));
        ctx->refine_cap = hit_cap;
    }
    Counters *ctr = nullptr, *ctr_next = nullptr;
    {
        const rich_status cst = trace_counters(ctx, &ctr, &ctr_next);
        if (cst != RICH_OK) return cst;
    }
    TraceParams p{};
    p.precision = o->precision;
    p.max_bounces = o->max_bounces;
    p.max_steps = o->max_steps;
    p.t_min = o->t_min;
    p.refill_min = refill;
    p.chunk = chunk;
    p.hits = out->hits;
    p.hit_capacity = out->hits ? out->hit_capacity : 0;
    p.pixel_counts = out->pixel_counts;
    p.event_sums = out->event_sums;
    p.n_hist_events = (out->pixel_counts || out->event_sums) ? out->n_hist_events : 0;
    p.fate = out->fate;
    p.fate_capacity = out->fate ? out->fate_capacity : 0;
    p.refine = ctx->d_refine;
    p.smem_nodes = smem_nodes;
    p.wait_limit = trace_wait_limit(o->wait_limit);
    p.n_prefilter = o->n_prefilter;
    for (int k = 0; k < 4; ++k) p.prefilter_tables[k] = k < o->n_prefilter ? o->prefilter_tables[k] : 0;
    LaunchShape shape;
    shape.threads = threads;
    shape.smem = trace_smem_bytes(ctx->sc, smem_nodes, threads, cls);
    shape.cls = cls;
    if (shape.smem > (size_t)ctx->smem_optin)
        return fail(ctx, RICH_ERR_ARG, "rich_trace: staged BVH nodes exceed shared memory");
    int bps = o->blocks_per_sm;
    {
        const auto key = std::make_tuple(in != nullptr, refine, cls, threads, shape.smem);
        auto it = ctx->occupancy.find(key);
        if (it == ctx->occupancy.end())
            it = ctx->occupancy.emplace(key, trace_blocks_per_sm(in != nullptr, refine, cls,
                                                                 threads, shape.smem)).first;
        if (it->second < 1)
            return fail(ctx, RICH_ERR_ARG, "rich_trace: launch shape does not fit on an SM");
        if (!bps || bps > it->second) bps = it->second;
    }
    shape.blocks = std::max(1, bps) * ctx->n_sm;
    if (work) {
        if (in || !refine || !trace_count_shape_ok(cls))
            return fail(ctx, RICH_ERR_ARG,
                        "rich_trace_work: counts the fused-emission trace with refinement in "
                        "the wide (up to 896 threads) or the 1024-thread shape");
        p.work = work;
    }
    EmitView em = emit_view(ctx);
    const bool timed = ctx->timing && !ctx->capturing;
    ctx->tev_trace = ctx->tev_refine = false;
    if (in) {
        em.key0 = (uint32_t)o->seed;
        em.key1 = (uint32_t)(o->seed >> 32);
        ExtView ev{in->n, in->x, in->y, in->z, in->dx, in->dy, in->dz, in->lambda,
                   in->event, in->track, in->photon};
        if (in->n) {
            if (timed) RICH_CUDA(cudaEventRecord(ctx->tev[3], ctx->stream));
            RICH_CUDA(launch_trace(ctx->sc, &em, &ev, p, ctr, ctr_next, shape, ctx->stream));
            if (timed) RICH_CUDA(cudaEventRecord(ctx->tev[4], ctx->stream));
            if (refine)
                RICH_CUDA(launch_refine(ctx->sc, &em, &ev, p, ctr, ctx->n_sm, ctx->stream));
            if (timed) RICH_CUDA(cudaEventRecord(ctx->tev[5], ctx->stream));
            ctx->tev_trace = timed;
            ctx->tev_refine = timed && refine;
        } else {
            ctr_next = nullptr;          // no trace kernel: nothing zeroed
        }
        ctx->last_ext = true;
        ctx->last_ext_n = in->n;
    } else {
        if (timed) RICH_CUDA(cudaEventRecord(ctx->tev[3], ctx->stream));
        if (work)
            RICH_CUDA(launch_trace_count(ctx->sc, em, p, ctr, ctr_next, shape, ctx->stream));
        else
            RICH_CUDA(launch_trace(ctx->sc, &em, nullptr, p, ctr, ctr_next, shape, ctx->stream));
        if (timed) RICH_CUDA(cudaEventRecord(ctx->tev[4], ctx->stream));
        if (refine)
            RICH_CUDA(launch_refine(ctx->sc, &em, nullptr, p, ctr, ctx->n_sm, ctx->stream));
        if (timed) RICH_CUDA(cudaEventRecord(ctx->tev[5], ctx->stream));
        ctx->tev_trace = timed;
        ctx->tev_refine = timed && refine;
        ctx->last_ext = false;
    }
    trace_counters_done(ctx, ctr_next != nullptr);
    ctx->traced = true;
    ctx->last_capacity = p.hit_capacity;
    return RICH_OK;
}

RICH_API rich_status rich_trace(rich_ctx *ctx, const rich_photons *in,
                                const rich_trace_opts *o, const rich_outputs *out) {
    return trace_impl(ctx, in, o, out, nullptr);
}

RICH_API rich_status rich_trace_work(rich_ctx *ctx, const rich_trace_opts *o,
                                     const rich_outputs *out, rich_work *work) {
    if (!ctx) return RICH_ERR_ARG;
    if (!work) return fail(ctx, RICH_ERR_ARG, "rich_trace_work: work is NULL");
    if (ctx->capturing) return fail(ctx, RICH_ERR_STATE, "rich_trace_work: inside a capture");
    DeviceGuard guard(ctx->device);
    if (!ctx->d_work) RICH_CUDA(cudaMalloc(&ctx->d_work, sizeof(unsigned long long) * 6));
    RICH_CUDA(cudaMemsetAsync(ctx->d_work, 0, sizeof(unsigned long long) * 6, ctx->stream));
    const rich_status st = trace_impl(ctx, nullptr, o, out, ctx->d_work);
    if (st != RICH_OK) return st;
    unsigned long long w[6];
    RICH_CUDA(cudaMemcpyAsync(w, ctx->d_work, sizeof w, cudaMemcpyDeviceToHost, ctx->stream));
    uint64_t n_hits = 0;
    rich_stats stats;
    const rich_status hs = rich_hits(ctx, &n_hits, &stats);
    if (hs != RICH_OK && hs != RICH_ERR_OVERFLOW) return hs;
    std::memset(work, 0, sizeof *work);
    work->photons = stats.n_photons - stats.n_fate[RICH_FATE_PREFILTERED];
    work->steps = w[0];
    work->nodes_smem = w[1];
    work->nodes_global = w[2];
    work->tri_tests = w[3];
    work->smooth_normals = w[4];
    work->turns = w[5];
    work->detected = n_hits;
    work->tracks = (uint64_t)ctx->n_tracks;
    work->sphere_groups = ctx->sc.n_groups;
    work->rects = ctx->sc.n_rects;
    return hs;
}

RICH_API rich_status rich_set_timing(rich_ctx *ctx, int on) {
    if (!ctx) return RICH_ERR_ARG;
    DeviceGuard guard(ctx->device);
    if (on && !ctx->tev[0])
        for (cudaEvent_t &e : ctx->tev) RICH_CUDA(cudaEventCreate(&e));
    ctx->timing = on != 0;
    ctx->tev_emit = ctx->tev_trace = ctx->tev_refine = false;
    return RICH_OK;
}

RICH_API rich_status rich_kernel_times(rich_ctx *ctx, rich_kernel_ms *out) {
    if (!ctx) return RICH_ERR_ARG;
    if (!out) return fail(ctx, RICH_ERR_ARG, "rich_kernel_times: out is NULL");
    DeviceGuard guard(ctx->device);
    out->yield = out->order = out->trace = out->refine = -1.f;
    if (ctx->tev_emit) {
        RICH_CUDA(cudaEventSynchronize(ctx->tev[2]));
        RICH_CUDA(cudaEventElapsedTime(&out->yield, ctx->tev[0], ctx->tev[1]));
        RICH_CUDA(cudaEventElapsedTime(&out->order, ctx->tev[1], ctx->tev[2]));
    }
    if (ctx->tev_trace) {
        RICH_CUDA(cudaEventSynchronize(ctx->tev[5]));
        RICH_CUDA(cudaEventElapsedTime(&out->trace, ctx->tev[3], ctx->tev[4]));
        if (ctx->tev_refine)
            RICH_CUDA(cudaEventElapsedTime(&out->refine, ctx->tev[4], ctx->tev[5]));
    }
    return RICH_OK;
}

RICH_API rich_status rich_hits(rich_ctx *ctx, uint64_t *n_hits, rich_stats *stats) {
    if (!ctx) return RICH_ERR_ARG;
    if (!ctx->traced) return fail(ctx, RICH_ERR_STATE, "rich_hits: no trace to report");
    DeviceGuard guard(ctx->device);
    RICH_CUDA(cudaMemcpyAsync(ctx->h_ctr, ctx->d_ctr, kCtrBytes, cudaMemcpyDeviceToHost,
                              ctx->stream));
    RICH_CUDA(cudaStreamSynchronize(ctx->stream));
    if (!ctx->last_ext) ctx->known_total = std::max<uint64_t>(ctx->known_total, *ctx->h_total);
    const Counters &c = *ctx->h_ctr;
    if (n_hits) *n_hits = c.hits;
    if (stats) {
        std::memset(stats, 0, sizeof *stats);
        stats->n_photons = ctx->last_ext ? ctx->last_ext_n : *ctx->h_total;
        stats->n_hits = c.hits;
        for (int k = 0; k < RICH_N_FATES; ++k) stats->n_fate[k] = c.fate[k];
        stats->device_status = c.status;
        stats->photon_order = c.ordered;
    }
    if (c.status != 0)
        return fail(ctx, (rich_status)c.status,
                    "rich_hits: device reported status " + std::to_string(c.status));
    if (c.hits > ctx->last_capacity)
        return fail(ctx, RICH_ERR_OVERFLOW, "rich_hits: " + std::to_string(c.hits) +
                                                " hits for capacity " +
                                                std::to_string(ctx->last_capacity));
    return RICH_OK;
}

RICH_API rich_status rich_trace_grad(rich_ctx *ctx, const rich_tracks *t,
                                     const rich_emit_params *prm, const rich_grad_params *th,
                                     const float *targets, float sigma,
                                     const rich_trace_opts *o, const rich_outputs *out,
                                     double grad[10], double *loss, uint64_t *n_used) {
    if (!ctx) return RICH_ERR_ARG;
    if (!t || !prm || !th || !o || !out || !grad || !loss)
        return fail(ctx, RICH_ERR_ARG, "rich_trace_grad: NULL argument");
    if (!ctx->has_geometry) return fail(ctx, RICH_ERR_STATE, "rich_trace_grad: no geometry");
    if (!targets || !(sigma > 0.f) || !out->hits || out->hit_capacity == 0)
        return fail(ctx, RICH_ERR_ARG,
                    "rich_trace_grad: need targets, sigma > 0 and a hit buffer");
    if (!(th->radius > 0.f) || !(th->n_minus_1 >= 0.f))
        return fail(ctx, RICH_ERR_ARG, "rich_trace_grad: need radius > 0 and n - 1 >= 0");
    if (o->n_prefilter != 0)
        return fail(ctx, RICH_ERR_ARG,
                    "rich_trace_grad: the gradient takes in-flight efficiencies (n_prefilter = 0)");
    if (ctx->has_dielectric)
        return fail(ctx, RICH_ERR_ARG,
                    "rich_trace_grad: the gradient is defined for scenes without refracting faces");
    if (prm->source != RICH_SOURCE_CHERENKOV || prm->dispersion)
        return fail(ctx, RICH_ERR_ARG,
                    "rich_trace_grad: the gradient is defined for the Cherenkov source with a "
                    "constant index");
    for (int k = 0; k < 8; ++k)
        if (!std::isfinite(th->tilt[k]) || std::fabs(th->tilt[k]) > 0.5f)
            return fail(ctx, RICH_ERR_ARG, "rich_trace_grad: tilts must be finite, |tilt| <= 0.5 rad");
    if (t->n > 0 && (!t->x || !t->y || !t->z || !t->dx || !t->dy || !t->dz || !t->p ||
                     !t->mass || !t->length || !t->event))
        return fail(ctx, RICH_ERR_ARG, "rich_trace_grad: a required track array is NULL");
    DeviceGuard guard(ctx->device);
    double theta[10];
    for (int k = 0; k < 8; ++k) theta[k] = th->tilt[k];
    theta[8] = th->radius;
    theta[9] = th->n_minus_1;
    // tiles at theta
    SceneView sv = ctx->sc;
    const DevTileDual *grad_duals = nullptr;
    const int ns = (int)ctx->nom_spheres.size();
    if (ns) {
        std::vector<rich_sphere> at(ns);
        std::vector<DevTileDual> duals(ns);
        for (int i = 0; i < ns; ++i) {
            at[i] = tile_at_theta(ctx->nom_spheres[i], i, theta);
            duals[i] = tile_dual(ctx->nom_spheres[i], i, theta);
        }
        std::vector<DevSphereGroup> groups;
        std::vector<DevTile> tiles;
        std::string gerr;
        if (!group_tiles(at.data(), ns, ctx->sc.n_materials, groups, tiles, gerr))
            return fail(ctx, RICH_ERR_ARG, "rich_trace_grad: " + gerr);
        char *base = static_cast<char *>(ctx->d_grad_tiles);
        RICH_CUDA(cudaMemcpyAsync(base, groups.data(), sizeof(DevSphereGroup) * groups.size(),
                                  cudaMemcpyHostToDevice, ctx->stream));
        char *tb = base + sizeof(DevSphereGroup) * RICH_MAX_GROUPS;
        RICH_CUDA(cudaMemcpyAsync(tb, tiles.data(), sizeof(DevTile) * tiles.size(),
                                  cudaMemcpyHostToDevice, ctx->stream));
        char *db = tb + sizeof(DevTile) * RICH_MAX_TILES;
        RICH_CUDA(cudaMemcpyAsync(db, duals.data(), sizeof(DevTileDual) * ns,
                                  cudaMemcpyHostToDevice, ctx->stream));
        grad_duals = reinterpret_cast<const DevTileDual *>(db);
        sv.groups = reinterpret_cast<const DevSphereGroup *>(base);
        sv.tiles = reinterpret_cast<const DevTile *>(tb);
        sv.n_groups = (int)groups.size();
        // host vectors must outlive the asynchronous copies
        RICH_CUDA(cudaStreamSynchronize(ctx->stream));
    }
    {
        rich_status st = emit_core(ctx, t, prm->seed, th->n_minus_1, prm->lambda_min,
                                   prm->lambda_max, RICH_SOURCE_CHERENKOV, 0.f, -1, 0, 0.f, 0.f,
                                   /*defer_scan=*/true);
        if (st == RICH_OK) st = order_photons(ctx);
        if (st != RICH_OK) return st;
    }
    // forward trace recording each detected photon's reflecting surfaces
    rich_trace_opts fo = *o;
    fo.precision = RICH_PREC_REFINE64;
    const uint64_t hit_cap = out->hit_capacity;
    if (hit_cap > ctx->refine_cap) {
        RICH_CUDA(cudaStreamSynchronize(ctx->stream));
        drop_graph(ctx);
        cudaFree(ctx->d_refine);
        ctx->d_refine = nullptr;
        ctx->refine_cap = 0;
        RICH_CUDA(cudaMalloc(&ctx->d_refine, sizeof(RefineRec) * hit_cap));
        ctx->refine_cap = hit_cap;
    }
    if (!ctx->d_acc) {
        RICH_CUDA(cudaMalloc(&ctx->d_acc, sizeof(double) * 12));
        RICH_CUDA(cudaMallocHost(&ctx->h_acc, sizeof(double) * 12));
    }
    const int threads = fo.block_threads ? fo.block_threads : kDefaultThreads;
    const int cls = trace_shape_class(threads, fo.wide_regs != 0);
    int smem_nodes = fo.bvh_smem_nodes;
    if (smem_nodes < 0) smem_nodes = threads > 256 ? 256 : 0;
    if (smem_nodes > ctx->sc.n_nodes) smem_nodes = ctx->sc.n_nodes;
    if (ctx->sc.n_tris == 0) smem_nodes = 0;
    TraceParams p{};
    p.precision = RICH_PREC_REFINE64;
    p.max_bounces = fo.max_bounces;
    p.max_steps = fo.max_steps;
    p.t_min = fo.t_min;
    p.refill_min = fo.refill_min ? fo.refill_min : 32;
    p.chunk = fo.chunk ? fo.chunk : 32;
    p.hits = out->hits;
    p.hit_capacity = hit_cap;
    p.pixel_counts = out->pixel_counts;
    p.event_sums = nullptr;
    p.n_hist_events = out->pixel_counts ? out->n_hist_events : 0;
    p.fate = out->fate;
    p.fate_capacity = out->fate ? out->fate_capacity : 0;
    p.refine = ctx->d_refine;
    p.smem_nodes = smem_nodes;
    p.wait_limit = trace_wait_limit(fo.wait_limit);
    if (p.max_bounces < 1 || p.max_bounces > RICH_MAX_BOUNCES || p.max_steps < 1 ||
        p.max_steps > RICH_MAX_STEPS || threads % 32 || threads > 1024)
        return fail(ctx, RICH_ERR_ARG, "rich_trace_grad: trace options out of range");
    LaunchShape shape;
    shape.threads = threads;
    shape.cls = cls;
    shape.smem = trace_smem_bytes(sv, smem_nodes, threads, cls);
    const int bps = trace_blocks_per_sm(false, true, cls, threads, shape.smem);
    if (bps < 1) return fail(ctx, RICH_ERR_ARG, "rich_trace_grad: launch shape does not fit");
    shape.blocks = bps * ctx->n_sm;
    Counters *ctr = nullptr, *ctr_next = nullptr;
    {
        const rich_status cst = trace_counters(ctx, &ctr, &ctr_next);
        if (cst != RICH_OK) return cst;
    }
    RICH_CUDA(cudaMemsetAsync(ctx->d_acc, 0, sizeof(double) * 12, ctx->stream));
    const EmitView em = emit_view(ctx);
    RICH_CUDA(launch_trace(sv, &em, nullptr, p, ctr, ctr_next, shape, ctx->stream));
    trace_counters_done(ctx, ctr_next != nullptr);
    GradView gv{};
    gv.tiles = grad_duals;
    gv.n_tiles = ns;
    gv.n_planes = ctx->sc.n_planes;
    for (int k = 0; k < 10; ++k) gv.theta[k] = theta[k];
    gv.targets = reinterpret_cast<const float4 *>(targets);
    gv.sigma = sigma;
    gv.acc = ctx->d_acc;
    gv.tracks = TracksView{t->n, t->x, t->y, t->z, t->dx, t->dy, t->dz, t->p, t->mass,
                           t->length, t->event, t->id, t->n_fixed};
    RICH_CUDA(launch_adjoint(sv, em, p, gv, ctx->d_ctr, ctx->n_sm, ctx->stream));
    RICH_CUDA(cudaMemcpyAsync(ctx->h_acc, ctx->d_acc, sizeof(double) * 12,
                              cudaMemcpyDeviceToHost, ctx->stream));
    RICH_CUDA(cudaMemcpyAsync(ctx->h_ctr, ctx->d_ctr, kCtrBytes, cudaMemcpyDeviceToHost,
                              ctx->stream));
    RICH_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->traced = true;
    ctx->last_ext = false;
    ctx->last_capacity = hit_cap;
    const double used = ctx->h_acc[1];
    const double inv = used > 0 ? 1.0 / used : 0.0;
    *loss = ctx->h_acc[0] * inv;
    for (int k = 0; k < 10; ++k) grad[k] = ctx->h_acc[2 + k] * inv;
    if (n_used) *n_used = (uint64_t)used;
    if (ctx->h_ctr->status)
        return fail(ctx, (rich_status)ctx->h_ctr->status,
                    "rich_trace_grad: device reported status " + std::to_string(ctx->h_ctr->status));
    if (ctx->h_ctr->hits > hit_cap)
        return fail(ctx, RICH_ERR_OVERFLOW,
                    "rich_trace_grad: " + std::to_string(ctx->h_ctr->hits) +
                        " hits for capacity " + std::to_string(hit_cap) +
                        " (hits beyond it are not in the gradient)");
    return RICH_OK;
}

// Enqueues one step from host memory into slot S (see rich_run_host).
static rich_status run_enqueue(rich_ctx *ctx, const char *who, const rich_tracks *ht,
                               const rich_emit_params *prm, const rich_trace_opts *o,
                               const rich_outputs *out, rich_hit *host_hits,
                               uint64_t host_hit_capacity, RunSlot &S) {
    const std::string w(who);
    if (!ht || !prm || !o || !out) return fail(ctx, RICH_ERR_ARG, w + ": NULL argument");
    if (ht->n < 0) return fail(ctx, RICH_ERR_ARG, w + ": negative track count");
    if (host_hit_capacity && !host_hits) return fail(ctx, RICH_ERR_ARG, w + ": host_hits is NULL");
    const size_t n = (size_t)ht->n;
    // the arrays in argument order; NULL optional ones are skipped
    const void *src[12] = {ht->x, ht->y, ht->z, ht->dx, ht->dy, ht->dz, ht->p, ht->mass,
                           ht->length, ht->event, ht->id, ht->n_fixed};
    for (int k = 0; k < 10; ++k)
        if (n && !src[k]) return fail(ctx, RICH_ERR_ARG, w + ": a required track array is NULL");
    if (!S.h_ctr) {
        RICH_CUDA(cudaMallocHost(&S.h_ctr, kCtrBytes));
        S.h_total = reinterpret_cast<unsigned long long *>(S.h_ctr + 1);
        RICH_CUDA(cudaEventCreateWithFlags(&S.ev, cudaEventDisableTiming));
        RICH_CUDA(cudaEventCreateWithFlags(&S.ev_h2d, cudaEventDisableTiming));
        RICH_CUDA(cudaEventCreateWithFlags(&S.ev_copy, cudaEventDisableTiming));
    }
    if (!ctx->copy_stream)
        RICH_CUDA(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
    if (!ctx->up_stream)
        RICH_CUDA(cudaStreamCreateWithFlags(&ctx->up_stream, cudaStreamNonBlocking));
    const size_t field = 4 * n;
    const size_t need = std::max<size_t>(12 * field, 256);
    if (need > S.d_tracks_bytes) {
        // the slot is not in flight: its earlier step has completed
        cudaFree(S.d_tracks);
        S.d_tracks = nullptr;
        S.d_tracks_bytes = 0;
        RICH_CUDA(cudaMalloc(&S.d_tracks, need));
        S.d_tracks_bytes = need;
    }
    char *dbase = static_cast<char *>(S.d_tracks);
    // the tracks travel on the upload stream, so they can move while an
    // earlier step computes (runs of arrays that lie back to back on the
    // host: one copy per run); the step's kernels wait for them
    if (n) {
        int k = 0;
        while (k < 12) {
            if (!src[k]) { ++k; continue; }
            int e = k + 1;
            while (e < 12 && src[e] &&
                   static_cast<const char *>(src[e]) == static_cast<const char *>(src[e - 1]) + field)
                ++e;
            RICH_CUDA(cudaMemcpyAsync(dbase + k * field, src[k], (e - k) * field,
                                      cudaMemcpyHostToDevice, ctx->up_stream));
            k = e;
        }
    }
    RICH_CUDA(cudaEventRecord(S.ev_h2d, ctx->up_stream));
    RICH_CUDA(cudaStreamWaitEvent(ctx->stream, S.ev_h2d, 0));
    auto dev = [&](int k) -> const void * { return src[k] ? dbase + k * field : nullptr; };
    rich_tracks dt;
    dt.n = ht->n;
    dt.x = (const float *)dev(0);
    dt.y = (const float *)dev(1);
    dt.z = (const float *)dev(2);
    dt.dx = (const float *)dev(3);
    dt.dy = (const float *)dev(4);
    dt.dz = (const float *)dev(5);
    dt.p = (const float *)dev(6);
    dt.mass = (const float *)dev(7);
    dt.length = (const float *)dev(8);
    dt.event = (const uint32_t *)dev(9);
    dt.id = (const uint32_t *)dev(10);
    dt.n_fixed = (const uint32_t *)dev(11);
    rich_status st = rich_emit(ctx, &dt, prm, nullptr, nullptr);
    if (st != RICH_OK) return st;
    st = rich_trace(ctx, nullptr, o, out);
    if (st != RICH_OK) return st;
    // the counters on the compute stream (the next step resets them); the
    // early copy of the expected hit records on the copy stream, after the
    // step's kernels (the next step writes another output buffer)
    RICH_CUDA(cudaMemcpyAsync(S.h_ctr, ctx->d_ctr, kCtrBytes, cudaMemcpyDeviceToHost,
                              ctx->stream));
    RICH_CUDA(cudaEventRecord(S.ev, ctx->stream));
    uint64_t early = ctx->run_host_hits ? ctx->run_host_hits + ctx->run_host_hits / 4 : 0;
    early = std::min(early, std::min(host_hit_capacity, out->hit_capacity));
    if (early) {
        RICH_CUDA(cudaStreamWaitEvent(ctx->copy_stream, S.ev, 0));
        RICH_CUDA(cudaMemcpyAsync(host_hits, out->hits, early * sizeof(rich_hit),
                                  cudaMemcpyDeviceToHost, ctx->copy_stream));
    }
    RICH_CUDA(cudaEventRecord(S.ev_copy, ctx->copy_stream));
    S.host_hits = host_hits;
    S.host_cap = host_hit_capacity;
    S.early = early;
    S.dev_hits = out->hits;
    S.dev_cap = out->hit_capacity;
    S.in_flight = true;
    return RICH_OK;
}

// Waits for the step in slot S, reports its counters (as rich_hits) and
// copies the hit records the early copy did not cover.
static rich_status run_complete(rich_ctx *ctx, const char *who, RunSlot &S, uint64_t *n_hits,
                                rich_stats *stats) {
    const std::string w(who);
    S.in_flight = false;
    RICH_CUDA(cudaEventSynchronize(S.ev));
    RICH_CUDA(cudaEventSynchronize(S.ev_copy));
    const Counters &c = *S.h_ctr;
    const uint64_t total = *S.h_total;
    ctx->known_total = std::max<uint64_t>(ctx->known_total, total);
    if (n_hits) *n_hits = c.hits;
    if (stats) {
        std::memset(stats, 0, sizeof *stats);
        stats->n_photons = total;
        stats->n_hits = c.hits;
        for (int k = 0; k < RICH_N_FATES; ++k) stats->n_fate[k] = c.fate[k];
        stats->device_status = c.status;
        stats->photon_order = c.ordered;
    }
    if (c.status != 0)
        return fail(ctx, (rich_status)c.status,
                    w + ": device reported status " + std::to_string(c.status));
    if (c.hits > S.dev_cap)
        return fail(ctx, RICH_ERR_OVERFLOW, w + ": " + std::to_string(c.hits) +
                                                " hits for capacity " + std::to_string(S.dev_cap));
    ctx->run_host_hits = c.hits;
    const uint64_t want = std::min<uint64_t>(c.hits, S.host_cap);
    if (want > S.early) {
        // the step's own output buffer (a later step in flight writes another)
        RICH_CUDA(cudaMemcpyAsync(S.host_hits + S.early, S.dev_hits + S.early,
                                  (want - S.early) * sizeof(rich_hit), cudaMemcpyDeviceToHost,
                                  ctx->copy_stream));
        RICH_CUDA(cudaStreamSynchronize(ctx->copy_stream));
    }
    if (S.host_hits && c.hits > S.host_cap)
        return fail(ctx, RICH_ERR_OVERFLOW, w + ": " + std::to_string(c.hits) +
                                                " hits for a host buffer of " +
                                                std::to_string(S.host_cap));
    return RICH_OK;
}

RICH_API rich_status rich_run_host(rich_ctx *ctx, const rich_tracks *ht,
                                   const rich_emit_params *prm, const rich_trace_opts *o,
                                   const rich_outputs *out, rich_hit *host_hits,
                                   uint64_t host_hit_capacity, uint64_t *n_hits,
                                   rich_stats *stats) {
    if (!ctx) return RICH_ERR_ARG;
    DeviceGuard guard(ctx->device);
    RunSlot &S = ctx->run_slots[2];
    const rich_status st = run_enqueue(ctx, "rich_run_host", ht, prm, o, out, host_hits,
                                       host_hit_capacity, S);
    if (st != RICH_OK) return st;
    return run_complete(ctx, "rich_run_host", S, n_hits, stats);
}

RICH_API rich_status rich_run_host_async(rich_ctx *ctx, const rich_tracks *ht,
                                         const rich_emit_params *prm, const rich_trace_opts *o,
                                         const rich_outputs *out, rich_hit *host_hits,
                                         uint64_t host_hit_capacity, uint64_t *ticket) {
    if (!ctx) return RICH_ERR_ARG;
    if (!ticket) return fail(ctx, RICH_ERR_ARG, "rich_run_host_async: ticket is NULL");
    const uint64_t t = ctx->next_ticket;
    RunSlot &S = ctx->run_slots[t % 2];
    if (S.in_flight)
        return fail(ctx, RICH_ERR_STATE,
                    "rich_run_host_async: two steps are in flight; wait for the older one");
    // the other step in flight still writes its hit records into its own
    // buffers (its trace, its early copy, rich_run_wait's completion copy)
    const RunSlot &other = ctx->run_slots[(t + 1) % 2];
    if (other.in_flight && out && out->hits && out->hits == other.dev_hits)
        return fail(ctx, RICH_ERR_ARG,
                    "rich_run_host_async: out->hits is the hit buffer of the step in flight");
    if (other.in_flight && host_hits && host_hits == other.host_hits)
        return fail(ctx, RICH_ERR_ARG,
                    "rich_run_host_async: host_hits is the host buffer of the step in flight");
    DeviceGuard guard(ctx->device);
    const rich_status st = run_enqueue(ctx, "rich_run_host_async", ht, prm, o, out, host_hits,
                                       host_hit_capacity, S);
    if (st != RICH_OK) return st;
    S.ticket = t;
    ctx->next_ticket = t + 1;
    *ticket = t;
    return RICH_OK;
}

RICH_API rich_status rich_run_wait(rich_ctx *ctx, uint64_t ticket, uint64_t *n_hits,
                                   rich_stats *stats) {
    if (!ctx) return RICH_ERR_ARG;
    RunSlot &S = ctx->run_slots[ticket % 2];
    if (ticket == 0 || !S.in_flight || S.ticket != ticket)
        return fail(ctx, RICH_ERR_STATE, "rich_run_wait: no step in flight with ticket " +
                                             std::to_string(ticket));
    DeviceGuard guard(ctx->device);
    return run_complete(ctx, "rich_run_wait", S, n_hits, stats);
}

RICH_API rich_status rich_graph_capture(rich_ctx *ctx, const rich_tracks *t,
                                        const rich_emit_params *prm,
                                        const rich_trace_opts *o, const rich_outputs *out) {
    if (!ctx) return RICH_ERR_ARG;
    if (!t || !prm || !o || !out)
        return fail(ctx, RICH_ERR_ARG, "rich_graph_capture: NULL argument");
    DeviceGuard guard(ctx->device);
    // warm-up pass: allocates scratch (reading the photon total sizes the
    // azimuth-order buffer) and fills the launch caches so the captured
    // pass makes no allocation and no synchronising call
    uint64_t n_warm = 0;
    rich_status st = rich_emit(ctx, t, prm, nullptr, &n_warm);
    if (st == RICH_OK) st = rich_trace(ctx, nullptr, o, out);
    if (st != RICH_OK) return st;
    RICH_CUDA(cudaStreamSynchronize(ctx->stream));
    if (!ctx->capture_stream)
        RICH_CUDA(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
    if (ctx->graph_exec) {
        cudaGraphExecDestroy(ctx->graph_exec);
        ctx->graph_exec = nullptr;
    }
    if (ctx->graph) {
        cudaGraphDestroy(ctx->graph);
        ctx->graph = nullptr;
    }
    cudaStream_t user = ctx->stream;
    ctx->stream = ctx->capture_stream;
    RICH_CUDA(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    ctx->capturing = true;               // the captured trace resets its own slot
    st = rich_emit(ctx, t, prm, nullptr, nullptr);
    if (st == RICH_OK) st = rich_trace(ctx, nullptr, o, out);
    ctx->capturing = false;
    ctx->graph_slot = ctx->cur_slot;
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
    ctx->stream = user;
    if (st != RICH_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
    ctx->graph = g;
    RICH_CUDA(cudaGraphInstantiate(&ctx->graph_exec, g, 0));
    ctx->graph_capacity = out->hits ? out->hit_capacity : 0;
    return RICH_OK;
}

RICH_API rich_status rich_graph_launch(rich_ctx *ctx) {
    if (!ctx) return RICH_ERR_ARG;
    if (!ctx->graph_exec) return fail(ctx, RICH_ERR_STATE, "rich_graph_launch: nothing captured");
    DeviceGuard guard(ctx->device);
    RICH_CUDA(cudaGraphLaunch(ctx->graph_exec, ctx->stream));
    // the replay counted into the captured slot; the other one is not known
    // to be zero
    ctx->cur_slot = ctx->graph_slot;
    ctx->d_ctr = ctx->d_ctr_slot[ctx->graph_slot];
    ctx->slot_zeroed[ctx->graph_slot] = false;
    ctx->slot_zeroed[ctx->graph_slot ^ 1] = false;
    ctx->traced = true;
    ctx->last_ext = false;
    ctx->last_capacity = ctx->graph_capacity;
    return RICH_OK;
}

RICH_API rich_status rich_philox(rich_ctx *ctx, const uint32_t *counters, uint64_t n,
                                 uint64_t seed, uint32_t *out) {
    if (!ctx) return RICH_ERR_ARG;
    if (n && (!counters || !out)) return fail(ctx, RICH_ERR_ARG, "rich_philox: NULL buffer");
    if ((reinterpret_cast<uintptr_t>(counters) | reinterpret_cast<uintptr_t>(out)) & 15u)
        return fail(ctx, RICH_ERR_ARG, "rich_philox: buffers must be 16-byte aligned");
    DeviceGuard guard(ctx->device);
    RICH_CUDA(launch_philox(counters, n, seed, out, ctx->stream));
    return RICH_OK;
}

}  // extern "C"
