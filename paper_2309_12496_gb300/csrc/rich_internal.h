// rich_internal.h -- layouts shared by the C-ABI host code and the kernels.
//
// Device layout of a scene (built by rich_init_geometry):
//   * sphere groups: tiles sharing one sphere (centre, radius) are grouped so
//     the double-word quadratic is solved once per sphere and the FP32 aperture
//     tests run per tile;
//   * rectangles, response tables and materials: small arrays staged into
//     shared memory by every trace block;
//   * triangles: 48-byte records in BVH leaf order; per-vertex normals in a
//     parallel array; four-wide BVH nodes of 128 bytes holding the four
//     children's boxes by axis.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "rich.h"

#define RICH_MAX_TILES 64
#define RICH_MAX_GROUPS 16
#define RICH_MAX_RECTS 32
#define RICH_MAX_TABLES 8
#define RICH_MAX_MATERIALS 32
#define RICH_MAX_PLANES 8
#define RICH_BVH_STACK 64

namespace rich {

struct DevTable {            // same fields as rich_table
    int32_t kind, nbins;
    float p0, p1, p2, p3;
    float values[RICH_TABLE_MAX_BINS];
};

struct DevMaterial {
    int32_t kind, table, plane, flags;
};

struct DevSphereGroup {      // 32 B
    float fcx, fcy, fcz;     // the FP32 input centre
    float radius, inv_radius;
    int32_t first, count;    // tiles [first, first + count)
    float pad;
};

struct DevTile {             // 160 B
    float ax, ay, az, cos_min;
    float e1x, e1y, e1z, inv_radius;
    float e2x, e2y, e2z;
    int32_t n_edges;
    int32_t material, group, prim, pad;
    float edges[RICH_SPHERE_MAX_EDGES][3];
};

struct DevRect {             // 80 B
    float ox, oy, oz, w;
    float ux, uy, uz, h;
    float vx, vy, vz, pitch;
    float nx, ny, nz;
    int32_t material;
    int32_t gx, gy, plane, prim;
};

struct alignas(16) DevTri {  // 48 B: v0 | v1 | v2 | prim, material, surface
    float v0x, v0y, v0z, v1x;
    float v1y, v1z, v2x, v2y;
    float v2z;
    int32_t prim, material;
    int32_t pad;              // BVH reference (node index or leaf code) of the
                              // subtree holding exactly this triangle's
                              // surface, or 0x7FFFFFFF when it has none
};

struct alignas(16) DevNode { // 128 B: boxes of up to four children (by axis) + refs
    // each box as centre and half extent per axis, rounded outward so that
    // [c - e, c + e] holds the children's bounds; the slab test then forms
    // entry and exit distances as (c - o) / d -+ e / |d| (FP32 multiply-adds)
    // without a min/max per axis to order them
    float cx[4], ex[4];
    float cy[4], ey[4];
    float cz[4], ez[4];
    int32_t child[4];          // >= 0 node, < 0 leaf ~(first << 3 | (count - 1)),
                               // INT_MIN an empty slot (its box is empty too)
    int32_t pad[4];
};

// Per triangle (leaf order), constants of the double-word refinement formed
// once on the host in FP64 and stored as hi + lo pairs: the unit geometric
// normal and, for the barycentrics of the smooth normal, the edge dot
// products d00 = e1.e1, d01 = e1.e2, d11 = e2.e2 and 1 / (d00 d11 - d01^2).
struct alignas(16) DevTriRef { // 64 B
    float ng[6];               // x hi, x lo, y hi, y lo, z hi, z lo
    float d00[2], d01[2], d11[2], inv_den[2];
    float pad[2];
};

struct alignas(16) TrackRec {  // 64 B, written by the yield kernel
    float x, y, z, len;
    float tx, ty, tz, tan_theta;  // unit direction (normalised in double-word) and tan
                                  // theta (constant index) or 1 - beta (FP32,
                                  // dispersive radiator)
    float rx, ry, rz;             // raw input direction
    uint32_t event;
    uint32_t id;
    uint32_t count;
    float disp_span;              // dispersive: FP32 1/lambda_min - 1/lambda_hi
                                  // of the emitting band
    float disp_s2max;             // dispersive: FP32 sin^2 theta(lambda_min)
};

// Emission model of the yield kernel.
struct YieldModel {
    double iso_yield;      // >= 0: isotropic source, photons per mm
    int32_t dispersion;    // 1: dispersive radiator (a, lambda0)
    float disp_a, disp_lambda0;
};

struct SceneView {
    const DevSphereGroup *groups;
    const DevTile *tiles;
    const DevRect *rects;
    const DevTable *tables;
    const DevMaterial *materials;
    const DevNode *nodes;
    const DevTri *tris;
    const float *tri_normals;   // 9 floats per triangle, leaf order, or null
    const DevTriRef *tri_ref;   // per triangle, leaf order
    int32_t n_groups, n_tiles, n_rects, n_tables, n_materials, n_nodes;
    int64_t n_tris;
    int32_t tri_prim_base;
    int32_t n_planes;
    int64_t pixels_per_event;
    int64_t plane_offset[RICH_MAX_PLANES];
    int32_t plane_nx[RICH_MAX_PLANES];
};

struct TracksView {          // device SoA of rich_tracks
    int64_t n;
    const float *x, *y, *z, *dx, *dy, *dz, *p, *mass, *length;
    const uint32_t *event, *id, *n_fixed;
};

// Per track, the double-word frame of the refinement's emission: the unit
// direction t and the orthonormal basis (e1, e2) around it, as (hi, lo)
// pairs per component (written by the yield pass).
struct alignas(16) TrackFrame {  // 80 B
    float t[6], e1[6], e2[6];
    float pad[2];
};

struct EmitView {            // result of rich_emit used by the trace
    const TrackRec *tracks;
    const float4 *cos_sin;    // (cos hi, cos lo, sin hi, sin lo) of the Cherenkov
                              // angle; dispersive radiator: (beta, 1 - beta),
                              // double-words
    const uint64_t *offsets;  // n_tracks + 1
    const unsigned long long *total;
    int64_t n_tracks;
    uint32_t key0, key1;
    float inv1, span;         // FP32 1/lambda_min and 1/lambda_min - 1/lambda_max
    const uint2 *perm;        // per queue entry: (photon index in its track, track
                              // index), each track's photons in azimuth order; entries
                              // of tracks above kOrderMaxPhotons are not written; or null
    const uint32_t *perm_ok;  // device flag: perm covers this emission
    int32_t source;           // RICH_SOURCE_*
    int32_t spectrum;         // isotropic: CDF table index of the scene, or -1
    int32_t dispersion;       // 1: dispersive radiator
    float disp_a, disp_lambda0;
    const TrackFrame *frame;  // per track
};

struct ExtView {             // caller photons
    uint64_t n;
    const float *x, *y, *z, *dx, *dy, *dz, *lambda;
    const uint32_t *event, *track, *photon;
};

struct Counters {            // device, cleared before each trace
    unsigned long long work;
    unsigned long long hits;
    unsigned long long fate[RICH_N_FATES];
    unsigned int status;
    unsigned int ordered;    // 1: photons were taken in azimuth order
};

// Per stored hit, what the refinement pass needs to replay the photon:
// its track (or caller-photon) index, the detector rectangle and the
// sequence of reflecting primitives (triangles by BVH leaf position).
struct RefineRec {             // 40 B
    uint32_t index;
    uint8_t det_rect, n_path;
    uint16_t pad;
    int32_t path[RICH_MAX_BOUNCES];
};

struct TraceParams {
    int32_t precision, max_bounces, max_steps;
    float t_min;
    int32_t refill_min, chunk;
    rich_hit *hits;
    uint64_t hit_capacity;
    uint32_t *pixel_counts;
    double *event_sums;
    uint32_t n_hist_events;
    uint8_t *fate;
    uint64_t fate_capacity;   // entries of fate; photons beyond get none
    RefineRec *refine;        // capacity hit_capacity (refined precision only)
    int32_t smem_nodes;       // BVH nodes [0, smem_nodes) staged in shared memory
    int32_t n_prefilter;      // > 0: efficiencies applied before propagation
    int32_t prefilter_tables[4];
    int32_t wait_limit;       // iterations of the bounded wait for the node copy
    unsigned long long *work; // counting build only: 6 tallies (WorkTally order)
};

// Sphere tile i at the gradient's parameters: centre C = P - R a(alpha_i,
// beta_i) as a double-word (hi + lo per axis) and its derivatives with
// respect to alpha_i, beta_i (zero for i >= 4) and R.
struct DevTileDual {          // 64 B
    float c_hi[3], c_lo[3];
    float dc_dalpha[3], dc_dbeta[3], dc_dr[3];
    float pad;
};

// Gradient of the soft ring chi^2: parameters theta (8 tile tilts, radius of
// curvature, n - 1), ring targets [n_tracks][n_planes] = (cu, cv, r, weight)
// and the FP64 accumulators (loss sum, hits used, 10 gradient sums).
struct GradView {
    const DevTileDual *tiles;
    int32_t n_tiles;
    int32_t n_planes;
    double theta[10];
    const float4 *targets;
    double sigma;
    double *acc;              // 12 doubles
    TracksView tracks;
};

struct LaunchShape {
    int blocks, threads;
    size_t smem;
    int cls;                  // kernel variant class (trace_shape_class)
};

// ---------------------------------------------------------------- launchers
// model.iso_yield >= 0: isotropic source with that mean per mm (the
// Cherenkov angle is not computed); < 0: Cherenkov source, constant index
// n_minus_1 or the dispersive radiator of model.
cudaError_t launch_yield(const TracksView &t, double n_minus_1,
                         double lam_min, double lam_max, uint32_t key0,
                         uint32_t key1, TrackRec *rec, float4 *cs,
                         uint32_t *counts, unsigned long long *block_sums,
                         cudaStream_t s, const YieldModel &model,
                         TrackFrame *frame = nullptr, uint32_t *perm_ok = nullptr);
cudaError_t launch_offsets(const uint32_t *counts,
                           const unsigned long long *block_sums,
                           int64_t n_tracks, uint64_t *offsets,
                           unsigned long long *total, cudaStream_t s);
// Azimuth ordering of each track's photons (the trace takes them in this
// order so a warp's rays are spatially coherent); tracks with more than
// kOrderMaxPhotons photons keep index order.
constexpr uint32_t kOrderMaxPhotons = 16384;
// The ordering pass can also do the scan of the photon counts (offsets and
// total from the yield pass's 256-track group sums; up to 4096 groups),
// which saves the separate scan launch when nothing reads the offsets in
// between.
constexpr int kOrderScanGroups = 4096;
constexpr int64_t kOrderScanMaxTracks = (int64_t)kOrderScanGroups * 256;
struct OrderScan {
    const uint32_t *counts;
    const unsigned long long *group_sums;
    uint64_t *offsets;             // n + 1 entries, written
    unsigned long long *total;     // written
};
cudaError_t launch_order(const EmitView &em, uint2 *perm, uint64_t cap, uint32_t *perm_ok,
                         int n_sm, cudaStream_t s, const OrderScan *scan = nullptr);
cudaError_t launch_materialize(const SceneView &sc, const EmitView &em,
                               uint64_t n, const rich_photons &out,
                               cudaStream_t s);
// counters: the trace's slot (the kernel also stores the photon total right
// after it); next: the slot it zeroes for the next trace, or null.
cudaError_t launch_trace(const SceneView &sc, const EmitView *em,
                         const ExtView *ext, const TraceParams &p,
                         Counters *counters, Counters *next, const LaunchShape &shape,
                         cudaStream_t s);
// The counting build of the trace (fused emission, refinement records; the
// shape classes of more than 256 threads only): p.work receives 6 tallies.
bool trace_count_shape_ok(int cls);
cudaError_t launch_trace_count(const SceneView &sc, const EmitView &em, const TraceParams &p,
                               Counters *counters, Counters *next, const LaunchShape &shape,
                               cudaStream_t s);
cudaError_t launch_refine(const SceneView &sc, const EmitView *em,
                          const ExtView *ext, const TraceParams &p,
                          Counters *counters, int n_sm, cudaStream_t s);
cudaError_t launch_philox(const uint32_t *ctr, uint64_t n, uint64_t seed, uint32_t *out,
                          cudaStream_t s);
cudaError_t launch_adjoint(const SceneView &sc, const EmitView &em, const TraceParams &p,
                           const GradView &gv, Counters *counters, int n_sm,
                           cudaStream_t s);
size_t trace_smem_bytes(const SceneView &sc, int smem_nodes, int threads, int cls);
int trace_shape_class(int threads, bool wide);
int trace_blocks_per_sm(bool ext, bool refine, int cls, int threads, size_t smem);
int yield_block_threads();

}  // namespace rich
