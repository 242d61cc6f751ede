/*
 * rich.h — C ABI of the GB300 Cherenkov-photon propagator.
 *
 * The library propagates Cherenkov photons through a RICH-like optical
 * geometry: photons are emitted along charged tracks at cos(theta) = 1/(n*beta)
 * (paper Sec. 3), carry a wavelength drawn from the Frank-Tamm 1/lambda^2
 * spectrum, are traced through spherical and flat mirrors (analytic surfaces,
 * or triangle meshes behind a BVH, as in the mesh scene of Sec. 4.1), are
 * reflected with a wavelength-dependent reflectivity and accepted by a
 * quantum-efficiency table (the binned efficiencies and accept/reject of
 * Sec. 4.3, applied in flight as proposed in Sec. 6), and are recorded as a
 * list of detector-plane positions relative to the plane's bottom-left corner
 * (Sec. 4.4 and the hit-list detector proposed in Sec. 6) and binned into
 * pixels.
 *
 * Conventions shared by every entry point
 *   - Lengths are millimetres, wavelengths nanometres, momenta GeV/c, masses
 *     GeV/c^2.
 *   - "device" pointers are CUDA global-memory addresses on the context's
 *     device; "host" pointers are ordinary CPU memory. The caller owns every
 *     buffer it passes; the context owns the geometry, the BVH, the response
 *     tables and its own scratch.
 *   - Calls are ordered on the context's CUDA stream and are asynchronous
 *     unless stated otherwise. Entry points that return counts to the host
 *     (rich_emit with a non-NULL count pointer, rich_hits, rich_trace_grad)
 *     synchronise that stream.
 *   - Every entry point returns a rich_status and never throws. The message
 *     of the last failure on a context is available from rich_last_error().
 *     Device-side failures (hit-buffer overflow, a bounded wait that expired)
 *     are recorded in a device status word and reported by the next call
 *     that synchronises (rich_hits).
 *   - Random numbers: every random draw is a Philox4x32-10 output (Salmon et
 *     al., SC'11) with key = (seed_lo, seed_hi) and counter = (block, photon,
 *     track id, event). Results therefore do not depend on launch shape,
 *     batching or sharding. The draw map is:
 *       per photon, block 0: w0 -> position along the track, w1 -> azimuth,
 *                            w2 -> wavelength, w3 -> quantum-efficiency test
 *       per photon, block 1: reflectivity tests at mirror reflections 0..3
 *       per photon, block 2: reflectivity tests at mirror reflections 4..7
 *       per photon, block 3: w0, w1 -> Gaussian smear of the hit (loss only),
 *                            w2 -> cos(theta) of an isotropic photon,
 *                            w3 -> first wavelength test (dispersive radiator)
 *       per photon, blocks 8..39: further wavelength trials (dispersive)
 *       per track (photon = 0xFFFFFFFF), blocks 0,1,...: Poisson sampler
 *     A 32-bit word w maps to the uniform (w >> 8) * 2^-24 in [0, 1).
 */
#ifndef RICH_H
#define RICH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define RICH_API __attribute__((visibility("default")))
#else
#define RICH_API
#endif

/* ------------------------------------------------------------------ status */
typedef enum rich_status {
    RICH_OK = 0,
    RICH_ERR_ARG = 1,       /* invalid argument (NULL, size, out of range)   */
    RICH_ERR_CUDA = 2,      /* a CUDA runtime call failed                    */
    RICH_ERR_OOM = 3,       /* device allocation failed                      */
    RICH_ERR_OVERFLOW = 4,  /* an output buffer was too small (truncated)    */
    RICH_ERR_TIMEOUT = 5,   /* a bounded device wait expired                 */
    RICH_ERR_GEOMETRY = 6,  /* malformed geometry description                */
    RICH_ERR_STATE = 7      /* call out of order (e.g. trace before geometry)*/
} rich_status;

/* ----------------------------------------------------- geometry description */
enum { RICH_TABLE_CONST = 0, RICH_TABLE_GAUSS = 1, RICH_TABLE_HIST = 2, RICH_TABLE_CDF = 3 };
enum { RICH_MAT_MIRROR = 0, RICH_MAT_ABSORBER = 1, RICH_MAT_DETECTOR = 2,
       RICH_MAT_DIELECTRIC = 3 };
enum { RICH_MAT_SMOOTH = 1 }; /* material flag: triangles use vertex normals */

#define RICH_TABLE_MAX_BINS 64
#define RICH_SPHERE_MAX_EDGES 8
#define RICH_MAX_BOUNCES 8   /* mirror reflections per photon (draw map)    */
#define RICH_MAX_STEPS 16    /* surface interactions per photon             */
/* Scene limits checked by rich_init_geometry (RICH_ERR_GEOMETRY beyond):
 * 64 sphere tiles on at most 16 distinct spheres, 32 rectangles, 8 tables,
 * 32 materials, 8 detector planes, 2^27 triangles. */

/* Wavelength response (reflectivity or quantum efficiency), Sec. 4.3.
 *   CONST: P = p0
 *   GAUSS: P = p0 * exp(-((lambda - p1) / p2)^2)
 *   HIST : P = values[clamp(floor((lambda - p0) / p1), 0, nbins - 1)]
 *          (piecewise-constant histogram, e.g. 33 nm bins for QE and 25 nm
 *           bins for reflectivity as in Sec. 4.3)
 *   CDF  : not a response but a binned emission spectrum for the isotropic
 *          source (rich_emit_params): values[0..nbins] is its cumulative
 *          distribution at the bin edges p0 + k*p1 (values[0] = 0,
 *          values[nbins] = 1, nondecreasing, nbins <= 63). A uniform u picks
 *          the bin k with values[k] <= u < values[k+1]; the wavelength is
 *          p0 + p1 * (k + (u - values[k]) / (values[k+1] - values[k])),
 *          each operation rounded in FP32.
 * P is evaluated in FP32. 280 bytes. */
typedef struct rich_table {
    int32_t kind;
    int32_t nbins;
    float p0, p1, p2, p3;
    float values[RICH_TABLE_MAX_BINS];
} rich_table;

/* Surface material. kind: RICH_MAT_*. table: index of the reflectivity
 * (mirror) or quantum-efficiency (detector) table, or of the refractive
 * index (dielectric). plane: detector-plane index for detectors (selects the
 * hit plane and histogram slice), else -1. flags: RICH_MAT_SMOOTH. Mirrors
 * reflect on their front side and absorb on the back; detectors accept on
 * the front and are transparent from the back; absorbers absorb on both
 * sides. A dielectric surface (a window face; rectangles and triangles only)
 * separates the medium in front (index 1) from a medium of index
 * table(lambda) behind it: the photon refracts by Snell's law with
 * eta = n_in / n_out and the geometric normal, or is totally internally
 * reflected when 1 - eta^2 (1 - cos^2 theta_i) < 0; no random draw (an
 * ideal anti-reflection-coated face). A slab is two faces whose normals
 * point away from the glass. */
typedef struct rich_material {
    int32_t kind, table, plane, flags;
} rich_material;

/* Analytic spherical-mirror tile. The sphere has centre `center` and radius
 * `radius`; the tile is the part of the sphere with unit vector
 * w = (p - center) / radius satisfying w . axis >= cos_min and, with
 * x = (p - center) . e1 and y = (p - center) . e2 (mm), every aperture edge
 * edges[j] = (a, b, c) satisfies a*x + b*y <= c. The reflective (front) side
 * is the concave one, facing the centre. 160 bytes. */
typedef struct rich_sphere {
    float center[3];
    float radius;
    float axis[3];
    float cos_min;
    float e1[3];
    int32_t n_edges;
    float e2[3];
    int32_t material;
    float edges[RICH_SPHERE_MAX_EDGES][3];
} rich_sphere;

/* Flat rectangle (flat mirror, absorber or detector plane). A point p is on
 * the rectangle when u = (p - origin) . u_axis lies in [0, width) and
 * v = (p - origin) . v_axis lies in [0, height). The front side is the side
 * `normal` points to (a ray with d . normal < 0 hits the front). Detector
 * rectangles carry an nx x ny pixel grid of pitch `pitch` with origin at the
 * bottom-left corner (Sec. 4.4); width = nx*pitch and height = ny*pitch.
 * 80 bytes. */
typedef struct rich_rect {
    float origin[3];
    float width;
    float u_axis[3];
    float height;
    float v_axis[3];
    float pitch;
    float normal[3];
    int32_t material;
    int32_t nx, ny, reserved0, reserved1;
} rich_rect;

/* Whole scene, all HOST pointers (copied by rich_init_geometry).
 * tri_vertices: n_triangles x 3 vertices x 3 floats. tri_normals: same shape,
 * per-vertex unit normals used by RICH_MAT_SMOOTH materials (may be NULL when
 * no material is smooth). tri_material: n_triangles material indices.
 * tri_surface: n_triangles surface ids (may be NULL: every triangle is a
 * surface of its own). Triangles sharing an id >= 0 form one surface (a
 * mirror segment, a flat mirror, a window face); -1 marks a triangle that is
 * a surface of its own. A photon leaving a surface (after reflecting or
 * refracting on it, or crossing it from behind) does not intersect that
 * surface again at its next step; every analytic sphere tile and rectangle
 * is a surface of its own.
 * Primitive ids: spheres are 0..n_spheres-1, rectangles follow, triangles
 * follow the rectangles (ids used in ties: the lowest id wins). */
typedef struct rich_geometry_desc {
    int32_t n_tables;
    int32_t n_materials;
    int32_t n_spheres;
    int32_t n_rects;
    int64_t n_triangles;
    const rich_table *tables;
    const rich_material *materials;
    const rich_sphere *spheres;
    const rich_rect *rects;
    const float *tri_vertices;
    const float *tri_normals;
    const int32_t *tri_material;
    const int32_t *tri_surface;
} rich_geometry_desc;

/* ------------------------------------------------------------------ inputs */
/* Charged tracks, structure of arrays, all DEVICE pointers of length n,
 * read-only, owned by the caller and kept alive until the rich_trace that
 * consumes this emission has completed on the stream.
 * (x,y,z) track origin; (dx,dy,dz) direction (normalised by the library);
 * p momentum; mass (0 -> beta = 1); length: emission length along the track
 * (0 -> point source); event: event id; id: track id within the event
 * (NULL -> the array index); n_fixed: fixed photon count per track (NULL ->
 * Poisson with the Frank-Tamm mean). */
typedef struct rich_tracks {
    int64_t n;
    const float *x, *y, *z;
    const float *dx, *dy, *dz;
    const float *p, *mass, *length;
    const uint32_t *event;
    const uint32_t *id;
    const uint32_t *n_fixed;
} rich_tracks;

/* Light sources (Sec. 6 names the Cherenkov light of liquid radiators such
 * as water, and scintillation light, as the next sources). */
enum { RICH_SOURCE_CHERENKOV = 0, RICH_SOURCE_ISOTROPIC = 1 };

/* Radiator and spectrum. seed: Philox key. n_minus_1: refractive index
 * minus one (constant, no dispersion). lambda_min/max: emission band (nm).
 * source: RICH_SOURCE_CHERENKOV (the zero default): photons on the cone
 *   cos(theta) = 1/(n beta) around the track, Frank-Tamm mean count and
 *   1/lambda^2 spectrum on [lambda_min, lambda_max].
 *   RICH_SOURCE_ISOTROPIC: photons uniform on the unit sphere (world frame;
 *   cos(theta) from draw block 3 word 2, azimuth from block 0 word 1) from
 *   points uniform along each track, Poisson mean yield_per_mm * length
 *   (or the track's n_fixed), wavelength from the scene's RICH_TABLE_CDF
 *   table `spectrum_table` (>= 0; needs the geometry loaded), or from the
 *   1/lambda^2 law on [lambda_min, lambda_max] when spectrum_table < 0.
 *   n_minus_1 and the track momenta are not used.
 * dispersion (Cherenkov source only): 0 = constant n_minus_1; 1 = the
 *   radiator's index follows n(lambda) - 1 = disp_a / (1/disp_lambda0^2 -
 *   1/lambda^2) (lambda, disp_lambda0 in nm, disp_a in nm^-2; needs
 *   lambda_min > disp_lambda0) and n_minus_1 is not used. Each photon then
 *   has the Cherenkov angle of its own wavelength, cos(theta) =
 *   1/(n(lambda) beta); the track's mean count is the Frank-Tamm integral
 *   2 pi alpha L int sin^2 theta(lambda) dlambda / lambda^2 over the part of
 *   the band where n(lambda) beta > 1 (closed form, FP64); and the
 *   wavelength is drawn by accept/reject: a candidate from the 1/lambda^2 law
 *   on that part of the band is kept with probability
 *   sin^2 theta(lambda) / sin^2 theta(lambda_min), both in FP32. Trial 0
 *   uses draw block 0 word 2 (candidate) and block 3 word 3 (test); trial
 *   t >= 1 uses block 8 + (t-1)/2, words 2((t-1) mod 2) and 2((t-1) mod 2)+1;
 *   after 64 trials the last candidate stands. */
typedef struct rich_emit_params {
    uint64_t seed;
    float n_minus_1;
    float lambda_min;
    float lambda_max;
    float reserved;
    int32_t source;
    float yield_per_mm;
    int32_t spectrum_table;
    int32_t dispersion;
    float disp_a;
    float disp_lambda0;
} rich_emit_params;

/* Materialised photons, structure of arrays of DEVICE pointers (caller
 * owned). rich_emit fills them when asked; rich_trace can consume them, or
 * photons supplied by the caller (e.g. from an external simulation), whose
 * keys (event, track, photon) select their reflectivity/QE random draws.
 * (dx,dy,dz) must be unit vectors. */
typedef struct rich_photons {
    uint64_t n;
    uint64_t capacity;
    float *x, *y, *z;
    float *dx, *dy, *dz;
    float *lambda;
    uint32_t *event, *track, *photon;
} rich_photons;

/* ----------------------------------------------------------------- options */
enum {
    RICH_PREC_FP32 = 0,     /* FP32 trace; the sphere quadratic in double-word
                               FP32 arithmetic (hi + lo, ~48 bits) */
    RICH_PREC_REFINE64 = 1  /* FP32 trace, then the detected photon's recorded
                               surface sequence is replayed in double-word
                               arithmetic (~48 bits, hit positions within
                               ~1e-10 mm of an FP64 replay) to give the hit
                               position and pixel */
};

typedef struct rich_trace_opts {
    uint64_t seed;          /* Philox key of the reflectivity/QE draws of
                               caller-supplied photons (photons from
                               rich_emit use the rich_emit seed)             */
    int32_t precision;      /* RICH_PREC_*                                    */
    int32_t max_bounces;    /* direction changes (mirror reflections and
                               refractions), 1..RICH_MAX_BOUNCES             */
    int32_t max_steps;      /* surface interactions, 1..RICH_MAX_STEPS        */
    float t_min;            /* minimum hit distance after an interaction (mm) */
    /* launch knobs (0 -> default: 512 threads of the 64-register build, two
       blocks per SM, 256 staged top nodes) */
    int32_t block_threads;  /* threads per block, multiple of 32, <= 1024;
                               above 256 the kernel is built for one block
                               per SM (see wide_regs); launched with 512
                               threads or fewer, two such blocks share one  */
    int32_t blocks_per_sm;  /* resident blocks per SM of the persistent grid
                               (0 or above the occupancy limit -> the limit) */
    int32_t refill_min;     /* refill a warp when at least this many lanes are
                               idle (1..32): the compaction interval          */
    int32_t chunk;          /* photons a warp takes from the queue at a time */
    int32_t wide_regs;      /* <= 256 threads: 0 caps the trace kernel at 64
                               registers (four blocks per SM), 1 uncapped;
                               257..896 threads: 1 caps it at 72 registers
                               (the 896-thread build), 0 at 64 (the
                               1024-thread build); > 896 threads: the
                               1024-thread build. Both builds of more than
                               256 threads keep the photon state the BVH
                               walk does not use in shared memory          */
    int32_t bvh_smem_nodes; /* top BVH nodes (128 bytes each) staged in shared
                               memory per block by a TMA bulk copy
                               (-1: default, 256 above 256 threads)         */
    /* Efficiencies applied before propagation (Sec. 4.3: the quantum
     * efficiency and the mirror reflectivities combined into one
     * accept/reject per photon at its wavelength, and rejected photons not
     * propagated). n_prefilter = 0: off (every efficiency is applied in
     * flight). 1..4: the photon enters the trace only if its QE uniform
     * (draw block 0, word 3) is below the FP32 product, taken left to right,
     * of the listed scene tables at its wavelength; it then reflects at
     * every mirror front and is recorded at every detector front without
     * further random tests. Rejected photons get RICH_FATE_PREFILTERED.
     * prefilter_tables: indices into the scene's tables. */
    int32_t n_prefilter;
    int32_t prefilter_tables[4];
    /* Iterations of each block's bounded wait for the TMA copy of the top
     * BVH nodes into shared memory (0: default, 2^20). When the wait runs
     * out the trace records RICH_ERR_TIMEOUT (read by rich_hits), waits
     * again, bounded, for the copy still in flight, and reads every node from
     * global memory instead: results are unchanged. A negative value makes
     * the first wait give up at once (a test of that path). */
    int32_t wait_limit;
} rich_trace_opts;

/* ----------------------------------------------------------------- outputs */
/* One detected photon, 40 bytes. (u, v): position on the detector plane in
 * mm relative to its bottom-left corner; (ix, iy) = floor((u, v) / pitch). */
typedef struct rich_hit {
    uint32_t event, track, photon;
    uint8_t plane;
    uint8_t n_reflections;
    uint16_t reserved;
    uint16_t ix, iy;
    float lambda;
    double u, v;
} rich_hit;

/* Photon fates (optional per-photon output). */
enum {
    RICH_FATE_NONE = 0,
    RICH_FATE_ESCAPED = 1,        /* left the scene                          */
    RICH_FATE_MIRROR_ABSORBED = 2,/* failed the reflectivity test            */
    RICH_FATE_ABSORBED = 3,       /* absorber, or the back of a mirror       */
    RICH_FATE_QE_REJECTED = 4,    /* reached a detector, failed the QE test  */
    RICH_FATE_DETECTED = 5,       /* recorded hit                            */
    RICH_FATE_MAX_BOUNCES = 6,    /* more than max_bounces reflections       */
    RICH_FATE_MAX_STEPS = 7,      /* more than max_steps interactions        */
    RICH_FATE_PREFILTERED = 8     /* failed the efficiencies applied before
                                     propagation (rich_trace_opts.n_prefilter) */
};
#define RICH_N_FATES 9

/* DEVICE output buffers, caller owned.
 * hits: capacity hit_capacity; hits beyond it are counted, not written.
 *   Hits are appended in no particular order (sort by key if needed).
 * pixel_counts: u32 histogram [n_hist_events][sum over planes of ny*nx],
 *   plane slices in plane-index order, row-major (iy, ix); accumulated
 *   (not cleared) by rich_trace; photons with event >= n_hist_events are not
 *   binned. May be NULL.
 * event_sums: FP64 [n_hist_events][n_planes][4] = (hits, sum u, sum v,
 *   sum lambda), accumulated. May be NULL.
 * fate: one byte per photon (RICH_FATE_*) indexed by the photon's global
 *   emission index, fate_capacity entries; photons at or beyond
 *   fate_capacity get no entry (size it from the photon total to have all).
 *   May be NULL. */
typedef struct rich_outputs {
    rich_hit *hits;
    uint64_t hit_capacity;
    uint32_t *pixel_counts;
    double *event_sums;
    uint32_t n_hist_events;
    uint32_t reserved;
    uint8_t *fate;
    uint64_t fate_capacity;
} rich_outputs;

/* Counters of the last rich_trace, read by rich_hits. */
typedef struct rich_stats {
    uint64_t n_photons;      /* photons handed to the trace (with the
                                prefilter on, n_photons - n_fate[8] photons
                                were propagated)                            */
    uint64_t n_hits;         /* detected photons (may exceed hit_capacity)  */
    uint64_t n_fate[RICH_N_FATES]; /* photons per RICH_FATE_* code          */
    uint32_t device_status;  /* RICH_OK or the first device-side error      */
    uint32_t photon_order;   /* 1: the trace took each track's photons in
                                azimuth order (a processing order only;
                                results do not depend on it), 0: index order */
} rich_stats;

typedef struct rich_ctx rich_ctx;

/* ------------------------------------------------------------ entry points */

/* Create a context on CUDA device `device`, ordered on `stream` (a
 * cudaStream_t, or NULL for the legacy default stream). *out receives the
 * handle. Allocates the context's small device state. */
RICH_API rich_status rich_create(rich_ctx **out, int device, void *stream);

/* Release every resource owned by the context (geometry, scratch). Waits for
 * the context's stream. NULL is accepted. */
RICH_API rich_status rich_destroy(rich_ctx *ctx);

/* Change the stream later calls are ordered on. */
RICH_API rich_status rich_set_stream(rich_ctx *ctx, void *stream);

/* Upload a scene (Sec. 4.1: mirrors and detector as separate surfaces with
 * their own materials; Sec. 4.3: wavelength tables). All pointers in `desc`
 * are HOST memory and are copied. Builds the SAH BVH over the triangles on
 * the host and uploads it. Replaces any previous geometry. Returns
 * RICH_ERR_GEOMETRY for inconsistent descriptions (bad indices, non-finite
 * values, pixel grid not matching a detector rectangle). Synchronous. */
RICH_API rich_status rich_init_geometry(rich_ctx *ctx, const rich_geometry_desc *desc);

/* Photon yield and emission (Sec. 3: cos(theta) = 1/(n beta), azimuth
 * uniform; photons are the input of the trace as in Sec. 4.2). For each
 * track computes beta, the Cherenkov angle and the Frank-Tamm mean
 * mu = L * 2*pi*alpha * sin^2(theta) * (1/lambda_min - 1/lambda_max), draws
 * N_t ~ Poisson(mu) (or takes n_fixed), all in double-word FP32 arithmetic
 * (~2^-44 per operation; the dispersive radiator's mean in FP64), and scans
 * the counts into photon offsets kept in the context for the next fused
 * rich_trace.
 * tracks: DEVICE arrays (see rich_tracks). out: if non-NULL, the photons are
 * also materialised into the caller's SoA (RICH_ERR_OVERFLOW if capacity is
 * too small; nothing is written then) and out->n is set on the host after a
 * synchronisation. n_photons: if non-NULL, receives the total photon count
 * (synchronises the stream); if NULL the call stays asynchronous. */
RICH_API rich_status rich_emit(rich_ctx *ctx, const rich_tracks *tracks,
                      const rich_emit_params *params, rich_photons *out,
                      uint64_t *n_photons);

/* Propagate photons through the scene. `in` NULL: the photons of the last
 * rich_emit are generated on the fly inside the trace kernel (fused emission,
 * no photon round trip through memory); otherwise the caller's photons are
 * traced. Mirrors reflect with probability R(lambda) at each reflection;
 * detectors accept with probability QE(lambda) (Sec. 4.3, in flight as in
 * Sec. 6); accepted photons are appended to out->hits and binned. With
 * opts->n_prefilter > 0 the efficiencies are instead applied once per photon
 * before propagation (Sec. 4.3) and only accepted photons are traced.
 * RICH_ERR_ARG for an invalid option (including a prefilter table index
 * outside the scene's tables). Clears the context's counters first;
 * asynchronous. */
RICH_API rich_status rich_trace(rich_ctx *ctx, const rich_photons *in,
                       const rich_trace_opts *opts, const rich_outputs *out);

/* Wait for the last rich_trace and report its counters. n_hits (host, may be
 * NULL) receives the number of detected photons; stats (host, may be NULL)
 * receives all counters. Returns RICH_ERR_OVERFLOW if hits were dropped for
 * lack of capacity (the count still reports every hit), or the device-side
 * error recorded during the trace. */
RICH_API rich_status rich_hits(rich_ctx *ctx, uint64_t *n_hits, rich_stats *stats);

/* ------------------------------------------------------- measurement aids */
/* Kernel timing (the profiling aid of the stage timers the paper used,
 * Sec. 5.1). When on, rich_emit and rich_trace record CUDA events on the
 * context's stream around each of their kernels, and rich_kernel_times
 * reports the durations of the last such calls. Recording an event between
 * two kernels ends the overlap of their programmatic launch, so the kernels'
 * sum can exceed the untimed step by a few microseconds. Calls inside a
 * graph capture are not timed. Off by default. */
typedef struct rich_kernel_ms {
    float yield;    /* per-track yield and Poisson count (and the count scan
                       pass when the emission synchronises)               */
    float order;    /* the ordering pass (with the count scan otherwise)  */
    float trace;    /* the persistent trace kernel                          */
    float refine;   /* the refinement pass; -1 without refinement          */
} rich_kernel_ms;

RICH_API rich_status rich_set_timing(rich_ctx *ctx, int on);

/* Durations (ms, host out) of the kernels of the last timed rich_emit and
 * rich_trace; -1 for a kernel that was not timed. Waits for those events. */
RICH_API rich_status rich_kernel_times(rich_ctx *ctx, rich_kernel_ms *out);

/* Algorithmic work of one trace, counted by the counting build of the trace
 * kernel (the same traversal with per-thread tallies). From these tallies
 * and the sizes of the records the traversal reads (128-byte four-wide BVH
 * nodes, 48-byte triangles, 36-byte vertex normals) follow the FP32
 * operations and the bytes per photon that bound the kernel. */
typedef struct rich_work {
    uint64_t photons;         /* photons that entered the trace            */
    uint64_t steps;           /* nearest-surface queries (bounce steps)    */
    uint64_t nodes_smem;      /* four-wide node tests on nodes staged in
                                 shared memory                             */
    uint64_t nodes_global;    /* node tests on nodes read from global memory */
    uint64_t tri_tests;       /* ray-triangle tests                         */
    uint64_t smooth_normals;  /* vertex-normal blends at smooth-triangle hits */
    uint64_t turns;           /* reflections and refractions               */
    uint64_t detected;        /* hits                                       */
    uint64_t tracks;          /* tracks of the emission                     */
    int32_t sphere_groups;    /* distinct spheres tested at every step      */
    int32_t rects;            /* rectangles tested at every step            */
} rich_work;

/* rich_trace of the last emission (fused photons; precision
 * RICH_PREC_REFINE64; more than 256 block_threads -- the 80- and 64-register
 * shapes, which have a counting build) through the counting build, then
 * the counters (as rich_hits) and the tallies into *work (host).
 * Synchronous; slower than rich_trace (for measurement only). Results
 * (hits, fates, histograms) are those of rich_trace. RICH_ERR_ARG for
 * another form; statuses of rich_hits otherwise (RICH_ERR_OVERFLOW still
 * fills *work). */
RICH_API rich_status rich_trace_work(rich_ctx *ctx, const rich_trace_opts *opts,
                                     const rich_outputs *out, rich_work *work);

/* One step from host memory: the track arrays (HOST pointers; pinned memory
 * makes the copies asynchronous, and arrays that lie back to back in one
 * allocation are copied as one block) are copied into device scratch owned
 * by the context, emitted (rich_emit) and traced with fused photons
 * (rich_trace) into out (device buffers, as for rich_trace), the counters
 * are read (rich_hits) and the first min(n_hits, host_hit_capacity) hit
 * records are copied into host_hits (host memory, pinned for speed). The
 * copy of the hit records is issued before the synchronisation for as many
 * records as the previous call of this context found (plus a quarter), so a
 * step usually synchronises once. Synchronous. n_hits / stats (may be NULL)
 * as for rich_hits. Returns the status of the first step that failed;
 * RICH_ERR_OVERFLOW also when host_hit_capacity is smaller than n_hits (the
 * first host_hit_capacity records are copied). host_hits NULL (capacity 0):
 * no records are copied, only the counters are read. */
RICH_API rich_status rich_run_host(rich_ctx *ctx, const rich_tracks *host_tracks,
                                   const rich_emit_params *params,
                                   const rich_trace_opts *opts, const rich_outputs *out,
                                   rich_hit *host_hits, uint64_t host_hit_capacity,
                                   uint64_t *n_hits, rich_stats *stats);

/* Pipelined form of rich_run_host: enqueues the same step (the track copy,
 * emit, trace, the early copy of the hit records and the counters' copy) on
 * the context's stream and returns at once with *ticket (host) naming it;
 * rich_run_wait completes it. At most two steps are in flight per context
 * (RICH_ERR_STATE for a third), so the host can enqueue step i + 1 while
 * the GPU runs step i. Each step in flight needs its own out buffers and
 * host_hits buffer (rich_run_wait may copy further records from its out):
 * RICH_ERR_ARG, with nothing enqueued, when out->hits or host_hits is the
 * one of the other step in flight. The host track arrays must stay
 * unchanged until the step is waited for. */
RICH_API rich_status rich_run_host_async(rich_ctx *ctx, const rich_tracks *host_tracks,
                                         const rich_emit_params *params,
                                         const rich_trace_opts *opts, const rich_outputs *out,
                                         rich_hit *host_hits, uint64_t host_hit_capacity,
                                         uint64_t *ticket);

/* Completes the pipelined step `ticket`: waits for it, reports its counters
 * (n_hits, stats as for rich_hits; may be NULL) and copies the hit records
 * the early copy did not cover. Statuses as for rich_run_host;
 * RICH_ERR_STATE for a ticket that is not in flight. */
RICH_API rich_status rich_run_wait(rich_ctx *ctx, uint64_t ticket, uint64_t *n_hits,
                                   rich_stats *stats);

/* Batched launch as a CUDA graph: captures rich_emit(tracks, params) +
 * rich_trace(fused photons, opts, out) -- the yield kernel, the count scan
 * and azimuth ordering, the counter reset, the persistent trace launch and
 * the refinement pass -- into
 * one graph owned by the context, after an uncaptured warm-up pass that
 * makes every allocation (the pass is also a full trace: its results are in
 * out). The graph keeps the pointers it was captured with: the caller's
 * track and output buffers must stay valid; replays see their current
 * contents (new track values, same count). Outputs accumulate across
 * replays unless the caller clears them. Replaces any earlier graph.
 * Synchronous. */
RICH_API rich_status rich_graph_capture(rich_ctx *ctx, const rich_tracks *tracks,
                                        const rich_emit_params *params,
                                        const rich_trace_opts *opts,
                                        const rich_outputs *out);

/* Replays the captured graph on the context's stream (asynchronous); read
 * the counters with rich_hits. */
RICH_API rich_status rich_graph_launch(rich_ctx *ctx);

/* Parameters of the gradient (10 scalars).
 *   tilt[2k], tilt[2k+1]: rotation of sphere tile k (k = 0..3, descriptor
 *     order) about the axis through its pole parallel to its nominal e1,
 *     then about the nominal e2 (rad); the pole stays fixed.
 *   radius: radius of curvature of every sphere tile (mm), pole fixed.
 *   n_minus_1: refractive index of the radiator minus one. */
typedef struct rich_grad_params {
    float tilt[8];
    float radius;
    float n_minus_1;
} rich_grad_params;

/* Soft ring chi^2 and its gradient with respect to rich_grad_params (the
 * differentiation of the mirror alignment and of the Cherenkov angle,
 * cos(theta) = 1/(n beta), Sec. 3, through the propagation of Sec. 4). The
 * tracks are emitted with n - 1 = theta->n_minus_1 (emit->n_minus_1 is
 * ignored; seed and band are used) and traced through the scene with its
 * sphere tiles moved to theta; every detected photon is then replayed along
 * its recorded reflecting surfaces (fixed topology, the photon's path
 * recomputed per photon, not stored) in forward mode: double-word values
 * (~48 bits), 10 FP32 tangents. The hit (u, v) is smeared by sigma (g1, g2), a Box-Muller pair
 * from the photon's draw block 3; rho = (|(u~, v~) - (cu, cv)| - r) / sigma
 * and loss = mean rho^2 over the hits whose (track index, plane) target has
 * weight > 0.
 * targets: DEVICE float [n_tracks][n_planes][4] = (cu, cv, r, weight).
 * out: DEVICE outputs of the forward pass; hits must have room for every
 *   hit (RICH_ERR_OVERFLOW otherwise: missing hits are not in the gradient);
 *   pixel_counts optional; event_sums ignored. Hits carry FP64 positions.
 * grad, loss, n_used: HOST results (mean over the hits used). Synchronous.
 * opts->n_prefilter must be 0 (RICH_ERR_ARG otherwise). */
RICH_API rich_status rich_trace_grad(rich_ctx *ctx, const rich_tracks *tracks,
                                     const rich_emit_params *emit,
                                     const rich_grad_params *theta,
                                     const float *targets, float sigma,
                                     const rich_trace_opts *opts,
                                     const rich_outputs *out, double grad[10],
                                     double *loss, uint64_t *n_used);

/* The library's random numbers: Philox4x32-10 (Salmon et al., SC'11) of n
 * counters (DEVICE, n x 4 words, 16-byte aligned) under key = (seed low
 * word, seed high word), written to out (DEVICE, n x 4 words, 16-byte
 * aligned). With counter (block, photon, track id, event) this reproduces
 * any draw of the map above. Asynchronous. */
RICH_API rich_status rich_philox(rich_ctx *ctx, const uint32_t *counters,
                                 uint64_t n, uint64_t seed, uint32_t *out);

/* Per-track photon counts and photon offsets without any device allocation,
 * for callers that cannot allocate device memory: code running under a
 * framework whose own pool allocator owns all of the GPU's memory, or a hook
 * inside a simulation step that must not make the synchronising cudaMalloc /
 * cudaFree calls. (The paper has no counterpart: it is a service of this
 * library.) It computes what rich_emit computes for the trace -- beta, the
 * Cherenkov angle, the Frank-Tamm mean and the keyed Poisson count of every
 * track -- without a context.
 * tracks: DEVICE arrays as for rich_emit, at most 1,048,576 tracks
 *   (RICH_ERR_ARG beyond, nothing launched). params: as for rich_emit.
 * counts: DEVICE, n entries, receives each track's photon count.
 * offsets: DEVICE, n + 1 entries, receives the exclusive prefix sums of the
 *   counts; offsets[n] is the total.
 * stream: cudaStream_t (NULL: legacy default stream); runs on the current
 *   device; asynchronous.
 * Its only scratch is a 32 KiB array in the library's device memory, present
 * on every GPU that loads the library until the process exits. The first
 * call on a device looks up that array's address (make it before any stream
 * capture). All calls share the array: calls whose work overlaps on the GPU
 * (e.g. issued on two streams at once) race and give wrong results. Errors
 * are reported by rich_last_error(NULL). Calls no allocating routine. */
RICH_API rich_status rich_photon_counts_static(const rich_tracks *tracks,
                                               const rich_emit_params *params,
                                               uint32_t *counts, uint64_t *offsets,
                                               void *stream);

/* Message for the last failure on ctx (or of rich_create when ctx is NULL).
 * The string is owned by the library and valid until the next call. */
RICH_API const char *rich_last_error(rich_ctx *ctx);

/* Library version string. */
RICH_API const char *rich_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RICH_H */
