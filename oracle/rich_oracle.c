/*
 * rich_oracle.c -- plain FP64 CPU oracle of the Cherenkov photon propagator.
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg use this file. It shares no code, header, table or helper
 * with the CUDA library: it reads the same binary input records (declared
 * again below) and implements every step itself, slowly and plainly, in
 * double precision, in the order the method takes them:
 *
 *   1. keyed random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
 *      "Parallel random numbers: as easy as 1, 2, 3", SC'11), counter =
 *      (block, photon, track id, event), key = seed;
 *   2. photon yield per track: Cherenkov angle cos(theta) = 1/(n beta)
 *      (paper Sec. 3) and the Frank-Tamm number of photons per unit length
 *      2 pi alpha sin^2(theta) (1/lambda_1 - 1/lambda_2) (textbook), drawn
 *      from a Poisson law (inversion below mean 10, the PTRS transformed
 *      rejection of Hoermann 1993 above);
 *   3. emission: a point uniform along the track segment, azimuth uniform
 *      on the Cherenkov cone (Sec. 3), wavelength from the 1/lambda^2
 *      spectrum by inverting its CDF; photons are thereafter independent
 *      rays as in the photon emitter of Sec. 4.2;
 *   4. nearest intersection with analytic spherical tiles, rectangles and
 *      triangles (Moeller-Trumbore, through a median-split BVH, or brute
 *      force) -- the mirror and detector surfaces of Sec. 4.1;
 *   5. surface response: specular reflection d' = d - 2 (d.n) n with an
 *      accept/reject on the mirror reflectivity, quantum-efficiency
 *      accept/reject at the detector (binned efficiencies, Sec. 4.3, applied
 *      in flight as proposed in Sec. 6), position on the detector plane
 *      relative to its bottom-left corner (Sec. 4.4) and pixel index;
 *   6. hit list, per-pixel counts and per-event sums (Sec. 6: the detector
 *      writes the position of each ray into a list).
 *
 * Variants of these steps:
 *   - efficiencies applied before propagation (Sec. 4.3): one accept/reject
 *     per photon on the product of listed tables at its wavelength, with its
 *     QE uniform; accepted photons then reflect and are recorded without
 *     further tests;
 *   - other light sources (Sec. 6: liquids, scintillation): isotropic
 *     emission along a segment with a yield per mm and a binned spectrum;
 *     water is the Cherenkov source with n = 1.33;
 *   - a dispersive radiator n(lambda): per-photon Cherenkov angle, the
 *     Frank-Tamm integral of sin^2 theta(lambda) as the mean count, and the
 *     wavelength law sin^2 theta(lambda)/lambda^2 by accept/reject;
 *   - refraction at window faces (Snell's law, total internal reflection),
 *     the windows the paper's simplified geometry removed (Sec. 4.1).
 *
 * Precision rules. Geometry runs in FP64 on the FP32 input values promoted
 * exactly. Quantities that decide integers are evaluated in FP32, the
 * precision the propagator itself takes those decisions in: the wavelength
 * (it selects a histogram bin), the response probabilities R(lambda) and
 * QE(lambda) (and their product before propagation) compared with a
 * uniform, and the dispersive radiator's wavelength acceptance. Every photon whose outcome hinges on
 * a decision closer than a margin to its threshold (a point within eps of a
 * surface, aperture, triangle, grid or pixel edge; two surfaces within eps
 * in distance; a uniform within prob_eps of its probability) is flagged as
 * a graze.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Input records (binary layout of the input generator's arrays).           */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t kind, nbins;
    float p0, p1, p2, p3;
    float values[64];
} o_table_in;
typedef struct {
    int32_t kind, table, plane, flags;
} o_material_in;
typedef struct {
    float center[3];
    float radius;
    float axis[3];
    float cos_min;
    float e1[3];
    int32_t n_edges;
    float e2[3];
    int32_t material;
    float edges[8][3];
} o_sphere_in;
typedef struct {
    float origin[3];
    float width;
    float u[3];
    float height;
    float v[3];
    float pitch;
    float normal[3];
    int32_t material;
    int32_t nx, ny, r0, r1;
} o_rect_in;

typedef struct {
    int32_t n_tables, n_materials, n_spheres, n_rects;
    int64_t n_triangles;
    const o_table_in *tables;
    const o_material_in *materials;
    const o_sphere_in *spheres;
    const o_rect_in *rects;
    const float *tri_v;      /* n x 3 x 3 */
    const float *tri_n;      /* n x 3 x 3 or NULL */
    const int32_t *tri_m;    /* n */
    const int32_t *tri_s;    /* n surface ids (>= 0 shared, -1 own) or NULL */
} o_scene_in;

typedef struct {
    int64_t n;
    const float *x, *y, *z, *dx, *dy, *dz, *p, *mass, *length;
    const uint32_t *event, *id, *n_fixed;
} o_tracks_in;

typedef struct {
    uint64_t seed;
    double n_minus_1;
    float lambda_min, lambda_max;
    int32_t max_bounces, max_steps;
    double t_min;
    double eps;        /* geometric graze margin (mm)          */
    double prob_eps;   /* probability graze margin             */
    int32_t use_bvh;
    int32_t n_threads;
    /* Efficiencies applied before propagation (Sec. 4.3): when n_prefilter
     * > 0 a photon is propagated only if its QE uniform is below the product
     * of the listed tables at its wavelength, and is then propagated with
     * the in-flight reflectivity and QE tests switched off. */
    int32_t n_prefilter;
    int32_t prefilter_tables[4];
    /* Light source (Sec. 6 names liquids and scintillation as the next
     * sources): 0 = Cherenkov emission along the track; 1 = isotropic
     * emission along the track (scintillation), yield_per_mm photons per mm
     * on average, wavelength from the `spectrum` CDF table (kind 3) or, when
     * spectrum is NULL, from the 1/lambda^2 law on [lambda_min, lambda_max]. */
    int32_t source;
    float yield_per_mm;
    const void *spectrum;
    /* Dispersive radiator (Cherenkov source): when dispersion = 1 the
     * refractive index follows the single-resonance form
     * n(lambda) - 1 = disp_a / (1/disp_lambda0^2 - 1/lambda^2) (lambda and
     * lambda0 in nm, a in nm^-2) and n_minus_1 is not used. */
    int32_t dispersion;
    float disp_a;
    float disp_lambda0;
} o_params;

/* Per-photon results, arrays indexed by global photon index. Any pointer
 * may be NULL. */
typedef struct {
    uint8_t *fate;
    int32_t *plane;
    int32_t *ix, *iy;
    double *u, *v;
    float *lambda;
    uint8_t *n_refl;
    uint8_t *graze;      /* bit 1 geometry, 2 probability, 4 pixel edge,
                            8 the surface just left was nearer (skip rule) */
    int32_t *path;       /* max_steps primitive ids per photon, -1 padded  */
    double *dir_out;     /* final direction (3 per photon)                 */
    double *pos_out;     /* final position (3 per photon)                  */
    uint32_t *pixel_counts;  /* [n_hist_events][pixels] or NULL            */
    double *event_sums;      /* [n_hist_events][n_planes][4] or NULL       */
    int64_t n_hist_events;
} o_photon_out;

enum { FATE_NONE = 0, FATE_ESCAPED = 1, FATE_MIRROR_ABSORBED = 2,
       FATE_ABSORBED = 3, FATE_QE_REJECTED = 4, FATE_DETECTED = 5,
       FATE_MAX_BOUNCES = 6, FATE_MAX_STEPS = 7, FATE_PREFILTERED = 8 };
enum { TAB_CONST = 0, TAB_GAUSS = 1, TAB_HIST = 2, TAB_CDF = 3 };
enum { SRC_CHERENKOV = 0, SRC_ISOTROPIC = 1 };
enum { MAT_MIRROR = 0, MAT_ABSORBER = 1, MAT_DETECTOR = 2, MAT_DIELECTRIC = 3 };
enum { MAT_SMOOTH = 1 };
enum { PRIM_SPHERE = 0, PRIM_RECT = 1, PRIM_TRI = 2 };

/* ------------------------------------------------------------------------ */
/* Small FP64 vector helpers.                                               */
/* ------------------------------------------------------------------------ */
typedef struct { double x, y, z; } v3;
static v3 mk(double x, double y, double z) { v3 r = {x, y, z}; return r; }
static v3 fromf(const float *a) { return mk(a[0], a[1], a[2]); }
static v3 add(v3 a, v3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static v3 sub(v3 a, v3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static v3 scl(v3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
static double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static v3 cross(v3 a, v3 b) {
    return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z,
              a.x * b.y - a.y * b.x);
}
static double norm(v3 a) { return sqrt(dot(a, a)); }
static v3 unit(v3 a) { return scl(a, 1.0 / norm(a)); }
static double comp(v3 a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }

/* ------------------------------------------------------------------------ */
/* 1. Philox4x32-10 (Salmon et al., SC'11).                                  */
/*    Round: with the two multipliers M0, M1, the products M0*c0 and M1*c2   */
/*    are split into high and low halves; the new counter is                 */
/*    (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)).      */
/*    The key is bumped by the two Weyl constants after each round.          */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void oracle_philox(const uint32_t ctr[4], const uint32_t key[2],
                   uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)PHILOX_M0 * (uint64_t)c[0];
        uint64_t prod1 = (uint64_t)PHILOX_M1 * (uint64_t)c[2];
        uint32_t n0 = (uint32_t)(prod1 >> 32) ^ c[1] ^ k0;
        uint32_t n1 = (uint32_t)prod1;
        uint32_t n2 = (uint32_t)(prod0 >> 32) ^ c[3] ^ k1;
        uint32_t n3 = (uint32_t)prod0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

void oracle_philox_batch(int64_t n, const uint32_t *ctr, const uint32_t *key,
                         uint32_t *out)
{
    for (int64_t i = 0; i < n; ++i)
        oracle_philox(ctr + 4 * i, key, out + 4 * i);
}

static void draw_block(uint64_t seed, uint32_t event, uint32_t track,
                       uint32_t photon, uint32_t block, uint32_t w[4])
{
    uint32_t ctr[4] = {block, photon, track, event};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    oracle_philox(ctr, key, w);
}

/* 24-bit uniform in [0, 1): exactly representable in FP32 and FP64. */
static double u24(uint32_t w) { return (double)(w >> 8) * (1.0 / 16777216.0); }

/* ------------------------------------------------------------------------ */
/* 2. Frank-Tamm yield and the Poisson draw.                                */
/* ------------------------------------------------------------------------ */
#define ALPHA_FS (1.0 / 137.035999)
#define PI_D 3.14159265358979323846

static double track_beta(double p, double m)
{
    if (m == 0.0) return 1.0;
    return p / sqrt(p * p + m * m);
}

/* sin^2 of the Cherenkov angle, cos(theta) = 1/(n beta) (Sec. 3); 0 below
 * threshold. Plain definition. */
static double sin2_theta(double n_minus_1, double beta)
{
    double nb = (1.0 + n_minus_1) * beta;
    if (nb <= 1.0) return 0.0;
    double c = 1.0 / nb;
    return 1.0 - c * c;
}

/* Mean number of photons per mm, charge 1, wavelengths in nm. */
double oracle_yield_per_mm(double n_minus_1, double beta, double lam_min_nm,
                           double lam_max_nm)
{
    double s2 = sin2_theta(n_minus_1, beta);
    double inv = 1.0e6 / lam_min_nm - 1.0e6 / lam_max_nm;   /* 1/mm */
    return 2.0 * PI_D * ALPHA_FS * s2 * inv;
}

/* ---- dispersive radiator ------------------------------------------------
 * 1 - beta written without cancellation: m^2 / (E (E + p)). */
static double one_minus_beta(double p, double m)
{
    if (m == 0.0) return 0.0;
    double E = sqrt(p * p + m * m);
    return m * m / (E * (E + p));
}

/* n(lambda) - 1 of the single-resonance form, FP64, lambda in nm. */
static double disp_n1(const o_params *prm, double lam)
{
    double il0 = 1.0 / (double)prm->disp_lambda0, il = 1.0 / lam;
    return (double)prm->disp_a / ((il0 - il) * (il0 + il));
}

/* Largest inverse wavelength x_t (nm^-1) below which n(x) beta <= 1, i.e.
 * no Cherenkov light: n increases with x = 1/lambda, and n beta = 1 at
 * x_t^2 = 1/lambda0^2 - a beta / (1 - beta). 0 when every x emits. */
static double disp_x_threshold(const o_params *prm, double beta, double omb)
{
    if (omb <= 0.0) return 0.0;
    double il0 = 1.0 / (double)prm->disp_lambda0;
    double u = il0 * il0 - (double)prm->disp_a * beta / omb;
    return u > 0.0 ? sqrt(u) : 0.0;
}

/* Frank-Tamm photons per mm of a dispersive radiator:
 * 2 pi alpha * integral over x = 1/lambda of sin^2 theta(x) =
 * 1 - 1/(n(x) beta)^2, over the part of [1/lambda_max, 1/lambda_min] where
 * n beta > 1. With c = 1/lambda0^2 and q = c + a, 1/n^2 =
 * (1 - a/(q - x^2))^2, so the integrand is (1 - 1/beta^2)
 * + (2a/beta^2)/(q - x^2) - (a^2/beta^2)/(q - x^2)^2, whose antiderivatives
 * are x, atanh(x/sqrt q)/sqrt q and x/(2q(q - x^2)) + atanh(x/sqrt q)/(2 q^1.5). */
static double disp_yield_per_mm(const o_params *prm, double beta, double omb)
{
    double xa = 1.0 / (double)prm->lambda_max, xb = 1.0 / (double)prm->lambda_min;
    double xt = disp_x_threshold(prm, beta, omb);
    if (xt > xa) xa = xt;
    if (!(xb > xa)) return 0.0;
    double il0 = 1.0 / (double)prm->disp_lambda0;
    double a = (double)prm->disp_a, q = il0 * il0 + a, sq = sqrt(q);
    double b2 = beta * beta;
    /* 1 - 1/beta^2 = -(1 - beta)(1 + beta)/beta^2, without cancellation */
    double c0 = -omb * (2.0 - omb) / b2;
#define F1(x) (atanh((x) / sq) / sq)
#define F2(x) ((x) / (2.0 * q * (q - (x) * (x))) + atanh((x) / sq) / (2.0 * q * sq))
    double I = c0 * (xb - xa) + (2.0 * a / b2) * (F1(xb) - F1(xa)) -
               (a * a / b2) * (F2(xb) - F2(xa));
#undef F1
#undef F2
    return 2.0 * PI_D * ALPHA_FS * I * 1.0e6;       /* x in nm^-1 -> per mm */
}

double oracle_disp_yield_per_mm(const o_params *prm, double p, double m)
{
    double omb = one_minus_beta(p, m);
    return disp_yield_per_mm(prm, 1.0 - omb, omb);
}

typedef struct {
    uint64_t seed;
    uint32_t event, track, block;
    int word;
    uint32_t w[4];
} o_stream;

static double stream_next(o_stream *s)
{
    if (s->word == 4) {
        draw_block(s->seed, s->event, s->track, 0xFFFFFFFFu, s->block, s->w);
        s->block++;
        s->word = 0;
    }
    return u24(s->w[s->word++]);
}

/* Poisson(mu): for mu < 10 invert the CDF with one uniform (the smallest k
 * with u < F(k)); otherwise the PTRS transformed-rejection sampler
 * (Hoermann, "The transformed rejection method for generating Poisson
 * random variables", 1993), two uniforms per trial, at most 64 trials
 * (then round(mu)). */
static int64_t poisson_draw(double mu, o_stream *s)
{
    if (!(mu > 0.0)) return 0;
    if (mu < 10.0) {
        double u = stream_next(s);
        double pk = exp(-mu), F = pk;
        int64_t k = 0;
        while (F <= u && k < 1000) {
            k += 1;
            pk *= mu / (double)k;
            F += pk;
        }
        return k;
    }
    double smu = sqrt(mu), lmu = log(mu);
    double b = 0.931 + 2.53 * smu;
    double a = -0.059 + 0.02483 * b;
    double inv_alpha = 1.1239 + 1.1328 / (b - 3.4);
    double v_r = 0.9277 - 3.6224 / (b - 2.0);
    for (int trial = 0; trial < 64; ++trial) {
        double U = stream_next(s) - 0.5;
        double V = stream_next(s);
        double us = 0.5 - fabs(U);
        if (!(us > 0.0)) continue;
        double kd = floor((2.0 * a / us + b) * U + mu + 0.43);
        if (!(kd >= 0.0)) continue;
        if (us >= 0.07 && V <= v_r) return (int64_t)kd;
        if (us < 0.013 && V > us) continue;
        double lhs = log(V) + log(inv_alpha) - log(a / (us * us) + b);
        double rhs = -mu + kd * lmu - lgamma(kd + 1.0);
        if (lhs <= rhs) return (int64_t)kd;
    }
    return (int64_t)floor(mu + 0.5);
}

/* Per-track mean and count. Returns the total photon count. */
int64_t oracle_yield(const o_tracks_in *t, const o_params *prm,
                     uint32_t *n_out, double *mu_out, uint64_t *offsets)
{
    uint64_t total = 0;
    for (int64_t i = 0; i < t->n; ++i) {
        double beta = track_beta(t->p[i], t->mass[i]);
        double omb = one_minus_beta(t->p[i], t->mass[i]);
        double mu = prm->dispersion && prm->source == SRC_CHERENKOV
                        ? (double)t->length[i] * disp_yield_per_mm(prm, 1.0 - omb, omb)
                    : prm->source == SRC_ISOTROPIC
                        ? (double)t->length[i] * (double)prm->yield_per_mm
                        : (double)t->length[i] *
                              oracle_yield_per_mm(prm->n_minus_1, beta,
                                                  prm->lambda_min, prm->lambda_max);
        int64_t k;
        if (t->n_fixed) {
            k = t->n_fixed[i];
        } else {
            o_stream s;
            memset(&s, 0, sizeof s);
            s.seed = prm->seed;
            s.event = t->event[i];
            s.track = t->id ? t->id[i] : (uint32_t)i;
            s.word = 4;
            k = poisson_draw(mu, &s);
        }
        if (n_out) n_out[i] = (uint32_t)k;
        if (mu_out) mu_out[i] = mu;
        if (offsets) offsets[i] = total;
        total += (uint64_t)k;
    }
    if (offsets) offsets[t->n] = total;
    return (int64_t)total;
}

int64_t oracle_poisson(double mu, uint64_t seed, uint32_t event,
                       uint32_t track)
{
    o_stream s;
    memset(&s, 0, sizeof s);
    s.seed = seed; s.event = event; s.track = track; s.word = 4;
    return poisson_draw(mu, &s);
}

/* ------------------------------------------------------------------------ */
/* 3. Emission.                                                             */
/* ------------------------------------------------------------------------ */
/* Wavelength by inverting the CDF of dN/dlambda ~ 1/lambda^2 on
 * [lambda_1, lambda_2]: 1/lambda = 1/lambda_1 - u (1/lambda_1 - 1/lambda_2).
 * Evaluated in FP32, one IEEE operation at a time (it selects table bins). */
static float emit_lambda(float u, float lam1, float lam2)
{
    volatile float inv1 = 1.0f / lam1;
    volatile float inv2 = 1.0f / lam2;
    volatile float span = inv1 - inv2;
    volatile float prod = u * span;
    volatile float inv = inv1 - prod;
    return 1.0f / inv;
}

/* Wavelength from a binned emission spectrum by inverting its CDF: the
 * table holds c_0 = 0 <= c_1 <= ... <= c_n = 1 at the bin edges
 * lambda_0 + k w; the bin is the k with c_k <= u < c_{k+1} and the
 * wavelength is linear inside it. FP32, one IEEE operation at a time (the
 * wavelength selects response-table bins). */
static float spectrum_lambda(const o_table_in *tab, float u)
{
    int k = 0;
    while (k + 1 < tab->nbins && tab->values[k + 1] <= u) ++k;
    volatile float num = u - tab->values[k];
    volatile float den = tab->values[k + 1] - tab->values[k];
    volatile float fr = num / den;
    volatile float kk = (float)k + fr;
    volatile float off = kk * tab->p1;
    volatile float lam = tab->p0 + off;
    return lam;
}

/* Orthonormal basis around a unit vector t (Duff, Burgess, Christensen,
 * Hery, Kensler, Liani, Villemin, "Building an orthonormal basis,
 * revisited", JCGT 6(1), 2017). */
static void basis(v3 t, v3 *e1, v3 *e2)
{
    double s = t.z >= 0.0 ? 1.0 : -1.0;
    double a = -1.0 / (s + t.z);
    double b = t.x * t.y * a;
    *e1 = mk(1.0 + s * t.x * t.x * a, s * b, -s * t.x);
    *e2 = mk(b, s + t.y * t.y * a, -t.y);
}

typedef struct {
    v3 o, d;
    float lambda;
    double u_qe;
    double u_refl[8];
    double u_smear[2];
    int graze;           /* 2: an emission accept/reject within prob_eps */
} o_photon;

/* sin^2 of the Cherenkov angle of the dispersive radiator at lambda, the
 * quantity the wavelength accept/reject compares, in FP32 one IEEE operation
 * at a time from the FP32 inputs: n - 1 = a/((1/l0 - 1/l)(1/l0 + 1/l)),
 * n beta - 1 = (n - 1) - (1 - beta) - (n - 1)(1 - beta), and
 * sin^2 = (n beta - 1)(n beta + 1)/(n beta)^2. */
static float disp_s2_f32(const o_params *prm, float omb, float lam)
{
    volatile float il = 1.0f / lam;
    volatile float il0 = 1.0f / prm->disp_lambda0;
    volatile float d1 = il0 - il;
    volatile float d2 = il0 + il;
    volatile float den = d1 * d2;
    volatile float n1 = prm->disp_a / den;
    volatile float t1 = n1 * omb;
    volatile float t2 = n1 - omb;
    volatile float nb1 = t2 - t1;
    if (!(nb1 > 0.0f)) return 0.0f;
    volatile float tw = 2.0f + nb1;
    volatile float num = nb1 * tw;
    volatile float op = 1.0f + nb1;
    volatile float dd = op * op;
    return num / dd;
}

/* Wavelength of a photon of a dispersive radiator: dN/dlambda is
 * proportional to sin^2 theta(lambda) / lambda^2 (Frank-Tamm), so a
 * candidate from the 1/lambda^2 law on the band where light is emitted,
 * [lambda_min, min(lambda_max, 1/x_t)], is accepted with probability
 * sin^2 theta(lambda) / sin^2 theta(lambda_min) (n, and so sin^2 theta,
 * decrease with lambda). Trial 0 takes block 0 word 2 (candidate) and block
 * 3 word 3 (test); trial t >= 1 takes block 8 + (t-1)/2, words
 * 2((t-1) mod 2) and 2((t-1) mod 2) + 1; after 64 trials the last candidate
 * stands. FP32 decisions as in disp_s2_f32. */
static float disp_lambda(const o_params *prm, uint64_t seed, uint32_t event,
                         uint32_t tid, uint32_t j, const uint32_t w0[4],
                         const uint32_t w3[4], double omb, double xt,
                         int *graze)
{
    float ombf = (float)omb;
    volatile float inv1 = 1.0f / prm->lambda_min;
    volatile float inv2 = 1.0f / prm->lambda_max;
    float xlo = inv2;
    if ((float)xt > xlo) xlo = (float)xt;
    /* the threshold's FP32 rounding decides the band: flag a near tie */
    if (xt > 0.0) {
        float r = (float)xt;
        float nb = xt < (double)r ? nextafterf(r, 0.0f) : nextafterf(r, 2.0f * r);
        double mid = 0.5 * ((double)r + (double)nb);
        if (fabs(xt - mid) < 1e-6 * fabs((double)nb - (double)r)) *graze |= 2;
    }
    volatile float span = inv1 - xlo;
    float s2max = disp_s2_f32(prm, ombf, prm->lambda_min);
    float lam = 0.0f;
    uint32_t w[4];
    for (int t = 0; t < 64; ++t) {
        uint32_t wl, wa;
        if (t == 0) {
            wl = w0[2];
            wa = w3[3];
        } else {
            draw_block(seed, event, tid, j, 8u + (uint32_t)(t - 1) / 2u, w);
            wl = w[2 * ((t - 1) & 1)];
            wa = w[2 * ((t - 1) & 1) + 1];
        }
        volatile float u = (float)u24(wl);
        volatile float prod = u * span;
        volatile float inv = inv1 - prod;
        lam = 1.0f / inv;
        if (!(s2max > 0.0f)) break;
        volatile float s2 = disp_s2_f32(prm, ombf, lam);
        volatile float pa = s2 / s2max;
        double ua = u24(wa);
        if (fabs(ua - (double)pa) < prm->prob_eps) *graze |= 2;
        if (ua < (double)pa) break;
    }
    return lam;
}

/* Photon j of track i. */
static void emit_photon(const o_tracks_in *t, const o_params *prm, int64_t i,
                        uint32_t j, o_photon *ph)
{
    uint32_t event = t->event[i];
    uint32_t tid = t->id ? t->id[i] : (uint32_t)i;
    uint32_t w0[4], w1[4], w2[4], w3[4];
    ph->graze = 0;
    draw_block(prm->seed, event, tid, j, 0, w0);
    draw_block(prm->seed, event, tid, j, 1, w1);
    draw_block(prm->seed, event, tid, j, 2, w2);
    draw_block(prm->seed, event, tid, j, 3, w3);
    v3 dir = unit(mk(t->dx[i], t->dy[i], t->dz[i]));
    double s = u24(w0[0]) * (double)t->length[i];
    ph->o = add(mk(t->x[i], t->y[i], t->z[i]), scl(dir, s));
    double phi = 2.0 * PI_D * u24(w0[1]);
    if (prm->source == SRC_ISOTROPIC && prm->spectrum)
        ph->lambda = spectrum_lambda((const o_table_in *)prm->spectrum,
                                     (float)u24(w0[2]));
    else
        ph->lambda = emit_lambda((float)u24(w0[2]), prm->lambda_min,
                                 prm->lambda_max);
    ph->u_qe = u24(w0[3]);
    for (int k = 0; k < 4; ++k) {
        ph->u_refl[k] = u24(w1[k]);
        ph->u_refl[4 + k] = u24(w2[k]);
    }
    ph->u_smear[0] = u24(w3[0]);
    ph->u_smear[1] = u24(w3[1]);
    if (prm->source == SRC_ISOTROPIC) {
        /* uniform on the unit sphere in the world frame: cos(theta) uniform
         * on [-1, 1] from draw block 3 word 2, azimuth from block 0 word 1 */
        double ct = 1.0 - 2.0 * u24(w3[2]);
        double st = sqrt(fmax(0.0, 1.0 - ct * ct));
        ph->d = mk(st * cos(phi), st * sin(phi), ct);
        return;
    }
    double beta = track_beta(t->p[i], t->mass[i]);
    double nb = (1.0 + prm->n_minus_1) * beta;
    if (prm->dispersion) {
        /* Cherenkov angle at the photon's own wavelength */
        double omb = one_minus_beta(t->p[i], t->mass[i]);
        beta = 1.0 - omb;
        ph->lambda = disp_lambda(prm, prm->seed, event, tid, j, w0, w3, omb,
                                 disp_x_threshold(prm, beta, omb), &ph->graze);
        nb = (1.0 + disp_n1(prm, (double)ph->lambda)) * beta;
    }
    double ct = 1.0 / nb;
    double st = sqrt(fmax(0.0, 1.0 - ct * ct));
    v3 e1, e2;
    basis(dir, &e1, &e2);
    ph->d = add(scl(dir, ct),
                scl(add(scl(e1, cos(phi)), scl(e2, sin(phi))), st));
}

void oracle_emit(const o_tracks_in *t, const o_params *prm, int64_t track,
                 uint32_t photon, double *origin, double *dir, float *lambda)
{
    o_photon ph;
    emit_photon(t, prm, track, photon, &ph);
    origin[0] = ph.o.x; origin[1] = ph.o.y; origin[2] = ph.o.z;
    dir[0] = ph.d.x; dir[1] = ph.d.y; dir[2] = ph.d.z;
    *lambda = ph.lambda;
}

/* ------------------------------------------------------------------------ */
/* Scene in FP64 and the oracle's own BVH (median split on centroids).      */
/* ------------------------------------------------------------------------ */
typedef struct {
    v3 c, axis, e1, e2;
    double R, cos_min;
    int n_edges;
    double edges[8][3];
    int material;
} o_sphere;
typedef struct {
    v3 o, u, v, n;
    double w, h, pitch;
    int nx, ny, material;
} o_rect;
typedef struct {
    v3 v0, v1, v2;
    v3 n0, n1, n2;
    v3 ng;        /* unit geometric normal, (v1-v0)x(v2-v0) */
    int material;
    int surface;  /* surface id (>= 0) shared by the triangles of one mirror
                     segment, flat or window face, or -1 */
} o_tri;
typedef struct {
    double lo[3], hi[3];
    int left, right;   /* internal: children; leaf: left = -1 */
    int first, count;  /* leaf range in the index array */
} o_node;

typedef struct {
    int n_tables, n_materials, n_spheres, n_rects;
    int64_t n_tris;
    o_table_in *tables;
    o_material_in *materials;
    o_sphere *spheres;
    o_rect *rects;
    o_tri *tris;
    o_node *nodes;
    int n_nodes;
    int *order;        /* triangle indices in leaf order */
    int n_planes;
    int64_t *plane_offset;   /* pixel offset of each plane in one event */
    int *plane_nx, *plane_ny;
    int64_t pixels_per_event;
} o_scene;

static void tri_bounds(const o_tri *t, double lo[3], double hi[3])
{
    for (int k = 0; k < 3; ++k) {
        double a = comp(t->v0, k), b = comp(t->v1, k), c = comp(t->v2, k);
        lo[k] = fmin(a, fmin(b, c));
        hi[k] = fmax(a, fmax(b, c));
    }
}

static o_scene *g_sort_scene;
static int g_sort_axis;
static int cmp_centroid(const void *pa, const void *pb)
{
    const o_tri *ta = &g_sort_scene->tris[*(const int *)pa];
    const o_tri *tb = &g_sort_scene->tris[*(const int *)pb];
    double ca = comp(ta->v0, g_sort_axis) + comp(ta->v1, g_sort_axis) +
                comp(ta->v2, g_sort_axis);
    double cb = comp(tb->v0, g_sort_axis) + comp(tb->v1, g_sort_axis) +
                comp(tb->v2, g_sort_axis);
    if (ca < cb) return -1;
    if (ca > cb) return 1;
    return *(const int *)pa - *(const int *)pb;
}

static int build_node(o_scene *s, int first, int count, int leaf_size)
{
    int id = s->n_nodes++;
    o_node *nd = &s->nodes[id];
    for (int k = 0; k < 3; ++k) { nd->lo[k] = INFINITY; nd->hi[k] = -INFINITY; }
    double clo[3] = {INFINITY, INFINITY, INFINITY};
    double chi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = first; i < first + count; ++i) {
        const o_tri *t = &s->tris[s->order[i]];
        double lo[3], hi[3];
        tri_bounds(t, lo, hi);
        for (int k = 0; k < 3; ++k) {
            nd->lo[k] = fmin(nd->lo[k], lo[k]);
            nd->hi[k] = fmax(nd->hi[k], hi[k]);
            double c = (comp(t->v0, k) + comp(t->v1, k) + comp(t->v2, k)) / 3;
            clo[k] = fmin(clo[k], c);
            chi[k] = fmax(chi[k], c);
        }
    }
    if (count <= leaf_size) {
        nd->left = nd->right = -1;
        nd->first = first;
        nd->count = count;
        return id;
    }
    int axis = 0;
    for (int k = 1; k < 3; ++k)
        if (chi[k] - clo[k] > chi[axis] - clo[axis]) axis = k;
    g_sort_scene = s;
    g_sort_axis = axis;
    qsort(s->order + first, (size_t)count, sizeof(int), cmp_centroid);
    int half = count / 2;
    nd->first = first;
    nd->count = 0;
    int l = build_node(s, first, half, leaf_size);
    int r = build_node(s, first + half, count - half, leaf_size);
    s->nodes[id].left = l;
    s->nodes[id].right = r;
    return id;
}

void *oracle_scene_create(const o_scene_in *in, int leaf_size)
{
    o_scene *s = (o_scene *)calloc(1, sizeof(o_scene));
    s->n_tables = in->n_tables;
    s->n_materials = in->n_materials;
    s->n_spheres = in->n_spheres;
    s->n_rects = in->n_rects;
    s->n_tris = in->n_triangles;
    s->tables = (o_table_in *)calloc((size_t)in->n_tables + 1, sizeof(o_table_in));
    memcpy(s->tables, in->tables, sizeof(o_table_in) * (size_t)in->n_tables);
    s->materials = (o_material_in *)calloc((size_t)in->n_materials + 1,
                                           sizeof(o_material_in));
    memcpy(s->materials, in->materials,
           sizeof(o_material_in) * (size_t)in->n_materials);
    s->spheres = (o_sphere *)calloc((size_t)in->n_spheres + 1, sizeof(o_sphere));
    for (int i = 0; i < in->n_spheres; ++i) {
        const o_sphere_in *a = &in->spheres[i];
        o_sphere *b = &s->spheres[i];
        b->c = fromf(a->center);
        b->R = a->radius;
        b->axis = fromf(a->axis);
        b->cos_min = a->cos_min;
        b->e1 = fromf(a->e1);
        b->e2 = fromf(a->e2);
        b->n_edges = a->n_edges;
        for (int j = 0; j < a->n_edges && j < 8; ++j)
            for (int k = 0; k < 3; ++k) b->edges[j][k] = a->edges[j][k];
        b->material = a->material;
    }
    s->rects = (o_rect *)calloc((size_t)in->n_rects + 1, sizeof(o_rect));
    int max_plane = -1;
    for (int i = 0; i < in->n_rects; ++i) {
        const o_rect_in *a = &in->rects[i];
        o_rect *b = &s->rects[i];
        b->o = fromf(a->origin);
        b->u = fromf(a->u);
        b->v = fromf(a->v);
        b->n = fromf(a->normal);
        b->w = a->width;
        b->h = a->height;
        b->pitch = a->pitch;
        b->nx = a->nx;
        b->ny = a->ny;
        b->material = a->material;
        const o_material_in *m = &s->materials[a->material];
        if (m->kind == MAT_DETECTOR && m->plane > max_plane) max_plane = m->plane;
    }
    s->n_planes = max_plane + 1;
    s->plane_offset = (int64_t *)calloc((size_t)s->n_planes + 1, sizeof(int64_t));
    s->plane_nx = (int *)calloc((size_t)s->n_planes + 1, sizeof(int));
    s->plane_ny = (int *)calloc((size_t)s->n_planes + 1, sizeof(int));
    for (int i = 0; i < in->n_rects; ++i) {
        const o_material_in *m = &s->materials[in->rects[i].material];
        if (m->kind == MAT_DETECTOR) {
            s->plane_nx[m->plane] = in->rects[i].nx;
            s->plane_ny[m->plane] = in->rects[i].ny;
        }
    }
    int64_t off = 0;
    for (int p = 0; p < s->n_planes; ++p) {
        s->plane_offset[p] = off;
        off += (int64_t)s->plane_nx[p] * s->plane_ny[p];
    }
    s->pixels_per_event = off;

    s->tris = (o_tri *)calloc((size_t)s->n_tris + 1, sizeof(o_tri));
    for (int64_t i = 0; i < s->n_tris; ++i) {
        const float *v = in->tri_v + 9 * i;
        o_tri *t = &s->tris[i];
        t->v0 = fromf(v);
        t->v1 = fromf(v + 3);
        t->v2 = fromf(v + 6);
        t->ng = unit(cross(sub(t->v1, t->v0), sub(t->v2, t->v0)));
        if (in->tri_n) {
            const float *n = in->tri_n + 9 * i;
            t->n0 = fromf(n);
            t->n1 = fromf(n + 3);
            t->n2 = fromf(n + 6);
        } else {
            t->n0 = t->n1 = t->n2 = t->ng;
        }
        t->material = in->tri_m[i];
        t->surface = in->tri_s ? in->tri_s[i] : -1;
    }
    s->order = (int *)malloc(sizeof(int) * ((size_t)s->n_tris + 1));
    for (int64_t i = 0; i < s->n_tris; ++i) s->order[i] = (int)i;
    s->nodes = (o_node *)calloc(2 * (size_t)s->n_tris + 2, sizeof(o_node));
    s->n_nodes = 0;
    if (s->n_tris > 0)
        build_node(s, 0, (int)s->n_tris, leaf_size > 0 ? leaf_size : 4);
    return s;
}

void oracle_scene_destroy(void *p)
{
    o_scene *s = (o_scene *)p;
    if (!s) return;
    free(s->tables); free(s->materials); free(s->spheres); free(s->rects);
    free(s->tris); free(s->nodes); free(s->order);
    free(s->plane_offset); free(s->plane_nx); free(s->plane_ny);
    free(s);
}

int oracle_scene_n_nodes(void *p) { return ((o_scene *)p)->n_nodes; }
int64_t oracle_scene_pixels_per_event(void *p)
{
    return ((o_scene *)p)->pixels_per_event;
}

/* ------------------------------------------------------------------------ */
/* 4. Intersections.                                                        */
/* ------------------------------------------------------------------------ */
typedef struct {
    double t;
    int prim;          /* global primitive id: spheres, rects, triangles */
    int kind;
    int index;
    int inside;        /* the point lies on the primitive (not beyond an edge) */
    double edge;       /* distance to the primitive's boundary (mm), >= 0 */
    double b1, b2;     /* triangle barycentrics of v1, v2 */
} o_cand;

typedef struct {
    o_cand best;
    int found;
    int graze;
} o_search;

/* Record a candidate: a point on the primitive's surface at distance t,
 * inside or outside its boundary. */
static void consider(o_search *s, const o_cand *c, double eps)
{
    if (c->inside) {
        int better = !s->found || c->t < s->best.t ||
                     (c->t == s->best.t && c->prim < s->best.prim);
        if (better) {
            if (s->found && s->best.t - c->t < eps) s->graze = 1;
            s->best = *c;
            s->found = 1;
        } else if (c->t - s->best.t < eps) {
            s->graze = 1;
        }
    }
}

/* Near misses that would be nearer than the chosen hit make the nearest-hit
 * decision fragile. Evaluated after the search. */
typedef struct {
    double t;
    double edge;
} o_miss;

/* Sphere tile: |o + t d - C| = R, roots of t^2 + 2 b t + c = 0. */
static void isect_sphere(const o_sphere *sp, int prim, v3 o, v3 d,
                         double t_min, double eps, o_search *s, double *near_t)
{
    v3 w = sub(o, sp->c);
    double b = dot(w, d);
    double c = dot(w, w) - sp->R * sp->R;
    double disc = b * b - c;
    if (disc < 0.0) return;
    double sq = sqrt(disc);
    double roots[2] = {-b - sq, -b + sq};
    for (int r = 0; r < 2; ++r) {
        double t = roots[r];
        if (!(t > t_min)) continue;
        v3 p = add(o, scl(d, t));
        v3 pc = sub(p, sp->c);
        double cosang = dot(pc, sp->axis) / sp->R;
        if (cosang > 1.0) cosang = 1.0;
        /* signed margins, positive inside: cap (arc length) and edges */
        int inside = cosang >= sp->cos_min;
        double edge = sp->R * (acos(sp->cos_min) - acos(cosang));
        double x = dot(pc, sp->e1), y = dot(pc, sp->e2);
        for (int j = 0; j < sp->n_edges; ++j) {
            double a = sp->edges[j][0], bb = sp->edges[j][1];
            double lin = a * x + bb * y;
            if (!(lin <= sp->edges[j][2])) inside = 0;
            double m = (sp->edges[j][2] - lin) / sqrt(a * a + bb * bb);
            if (m < edge) edge = m;
        }
        o_cand cd = {t, prim, PRIM_SPHERE, prim, inside, fabs(edge), 0, 0};
        if (!inside && edge > -eps && t < *near_t) *near_t = t;
        consider(s, &cd, eps);
        if (inside) return;   /* nearer root on the tile hides the far one */
    }
}

static void isect_rect(const o_rect *rc, int prim, int index, v3 o, v3 d,
                       double t_min, double eps, o_search *s, double *near_t)
{
    double den = dot(d, rc->n);
    if (den == 0.0) return;
    double t = dot(sub(rc->o, o), rc->n) / den;
    if (!(t > t_min)) return;
    v3 q = sub(add(o, scl(d, t)), rc->o);
    double u = dot(q, rc->u), v = dot(q, rc->v);
    /* half-open extent: 0 <= u < w, 0 <= v < h */
    int inside = u >= 0.0 && u < rc->w && v >= 0.0 && v < rc->h;
    double edge = fmin(fmin(u, rc->w - u), fmin(v, rc->h - v));
    o_cand cd = {t, prim, PRIM_RECT, index, inside, fabs(edge), 0, 0};
    if (!inside && edge > -eps && t < *near_t) *near_t = t;
    consider(s, &cd, eps);
}

/* Moeller-Trumbore ("Fast, minimum storage ray/triangle intersection",
 * 1997) in FP64; the signed distance of the point to the nearest edge line
 * is the smallest barycentric times the matching altitude. */
static void isect_tri(const o_tri *tr, int prim, int index, v3 o, v3 d,
                      double t_min, double eps, o_search *s, double *near_t)
{
    v3 e1 = sub(tr->v1, tr->v0), e2 = sub(tr->v2, tr->v0);
    v3 pv = cross(d, e2);
    double det = dot(e1, pv);
    if (det == 0.0) return;
    double inv = 1.0 / det;
    v3 tv = sub(o, tr->v0);
    double b1 = dot(tv, pv) * inv;
    v3 qv = cross(tv, e1);
    double b2 = dot(d, qv) * inv;
    double t = dot(e2, qv) * inv;
    if (!(t > t_min)) return;
    double b0 = 1.0 - b1 - b2;
    double area2 = norm(cross(e1, e2));
    double h0 = area2 / norm(sub(tr->v2, tr->v1));
    double h1 = area2 / norm(e2);
    double h2 = area2 / norm(e1);
    double edge = fmin(b0 * h0, fmin(b1 * h1, b2 * h2));
    if (edge < -eps) return;
    int inside = b0 >= 0.0 && b1 >= 0.0 && b2 >= 0.0;
    o_cand cd = {t, prim, PRIM_TRI, index, inside, fabs(edge), b1, b2};
    if (!inside && t < *near_t) *near_t = t;
    consider(s, &cd, eps);
}

static int box_hit(const o_node *nd, v3 o, v3 d, double t_max, double pad)
{
    double t0 = 0.0, t1 = t_max;
    for (int k = 0; k < 3; ++k) {
        double ok = comp(o, k), dk = comp(d, k);
        double lo = nd->lo[k] - pad, hi = nd->hi[k] + pad;
        if (dk == 0.0) {
            if (ok < lo || ok > hi) return 0;
            continue;
        }
        double ta = (lo - ok) / dk, tb = (hi - ok) / dk;
        if (ta > tb) { double x = ta; ta = tb; tb = x; }
        if (ta > t0) t0 = ta;
        if (tb < t1) t1 = tb;
        if (t0 > t1) return 0;
    }
    return 1;
}

/* Nearest surface along o + t d, t > t_min. `skip` is the primitive the
 * photon just left: it is not taken as a hit again, and neither is any
 * triangle of the same surface (a photon leaving a mirror segment, a flat
 * mirror or a window face is not intersected with that surface at its next
 * step). For planes that rule is exact. For a concave segment it is an
 * approximation: a photon leaving it close to the tangent plane can meet the
 * same segment again further along the chord. So the skipped primitive and
 * surface are still intersected, into a search of their own, and when one of
 * them would have been the nearest hit (or within eps of it) the decision is
 * flagged (*graze bit 8). Returns 1 and fills *hit if a hit is found; *graze
 * bit 1 is set when the nearest-hit decision is within eps of changing.
 * *skipped_t (may be NULL) receives the distance of the nearest hit on the
 * skipped surface, or INFINITY. */
static int nearest(const o_scene *sc, v3 o, v3 d, int skip, double t_min,
                   double eps, int use_bvh, o_cand *hit, int *graze,
                   double *skipped_t)
{
    o_search s, sk;
    memset(&s, 0, sizeof s);
    memset(&sk, 0, sizeof sk);
    double near_t = INFINITY, sk_near = INFINITY;
    int prim = 0;
    const int tb = sc->n_spheres + sc->n_rects;
    const int skip_surface = (skip >= tb && skip - tb < sc->n_tris)
                                 ? sc->tris[skip - tb].surface : -1;
#define SKIP_TRI(ti) ((tb + (ti)) == skip || \
                      (skip_surface >= 0 && sc->tris[(ti)].surface == skip_surface))
    for (int i = 0; i < sc->n_spheres; ++i, ++prim)
        isect_sphere(&sc->spheres[i], prim, o, d, t_min, eps,
                     prim == skip ? &sk : &s, prim == skip ? &sk_near : &near_t);
    for (int i = 0; i < sc->n_rects; ++i, ++prim)
        isect_rect(&sc->rects[i], prim, i, o, d, t_min, eps,
                   prim == skip ? &sk : &s, prim == skip ? &sk_near : &near_t);
    int tri_base = prim;
    if (sc->n_tris > 0) {
        if (use_bvh) {
            int stack[128];
            int sp = 0;
            stack[sp++] = 0;
            while (sp > 0) {
                const o_node *nd = &sc->nodes[stack[--sp]];
                double tmax = s.found ? s.best.t + 2.0 * eps : INFINITY;
                if (!box_hit(nd, o, d, tmax, 2.0 * eps)) continue;
                if (nd->left < 0) {
                    for (int k = nd->first; k < nd->first + nd->count; ++k) {
                        int ti = sc->order[k];
                        int skipped = SKIP_TRI(ti);
                        isect_tri(&sc->tris[ti], tri_base + ti, ti, o, d, t_min, eps,
                                  skipped ? &sk : &s, skipped ? &sk_near : &near_t);
                    }
                } else {
                    stack[sp++] = nd->left;
                    stack[sp++] = nd->right;
                }
            }
        } else {
            for (int64_t ti = 0; ti < sc->n_tris; ++ti) {
                int skipped = SKIP_TRI(ti);
                isect_tri(&sc->tris[ti], (int)(tri_base + ti), (int)ti, o, d, t_min, eps,
                          skipped ? &sk : &s, skipped ? &sk_near : &near_t);
            }
        }
    }
#undef SKIP_TRI
    *graze = s.graze;
    if (s.found && s.best.edge < eps) *graze = 1;
    if (near_t < INFINITY && (!s.found || near_t < s.best.t + eps)) *graze = 1;
    /* the skip rule decided the hit: the skipped surface (on it, or within
     * eps of its edge) lies nearer than the hit taken */
    double sk_t = sk.found ? sk.best.t : INFINITY;
    if (sk_near < sk_t) sk_t = sk_near;
    if (sk_t < INFINITY && (!s.found || sk_t < s.best.t + eps)) *graze |= 8;
    if (skipped_t) *skipped_t = sk.found ? sk.best.t : INFINITY;
    if (s.found) *hit = s.best;
    return s.found;
}

/* Batch ray cast for the BVH-versus-brute-force pin. */
void oracle_raycast(void *scene, int64_t n, const double *o, const double *d,
                    const int32_t *skip, double t_min, int use_bvh,
                    double *t_out, int32_t *prim_out)
{
    const o_scene *sc = (const o_scene *)scene;
    for (int64_t i = 0; i < n; ++i) {
        o_cand h;
        int g;
        v3 oo = mk(o[3 * i], o[3 * i + 1], o[3 * i + 2]);
        v3 dd = mk(d[3 * i], d[3 * i + 1], d[3 * i + 2]);
        int f = nearest(sc, oo, dd, skip ? skip[i] : -1, t_min, 1e-9, use_bvh,
                        &h, &g, NULL);
        t_out[i] = f ? h.t : INFINITY;
        prim_out[i] = f ? h.prim : -1;
    }
}

/* ------------------------------------------------------------------------ */
/* 5. Surface response.                                                     */
/* ------------------------------------------------------------------------ */
/* Wavelength response P(lambda) in FP32 (Sec. 4.3 binned efficiencies):
 * constant, Gaussian, or piecewise-constant histogram with clamped bins. */
static float table_eval(const o_table_in *t, float lam)
{
    if (t->kind == TAB_CONST) return t->p0;
    if (t->kind == TAB_GAUSS) {
        volatile float dl = lam - t->p1;
        volatile float x = dl / t->p2;
        volatile float x2 = x * x;
        volatile float e = expf(-x2);
        return t->p0 * e;
    }
    volatile float rel = lam - t->p0;
    volatile float q = rel / t->p1;
    float f = floorf(q);
    int b = f < 0.0f ? 0 : (f > (float)(t->nbins - 1) ? t->nbins - 1 : (int)f);
    return t->values[b];
}

float oracle_table_eval(void *scene, int table, float lam)
{
    return table_eval(&((o_scene *)scene)->tables[table], lam);
}

static v3 reflect(v3 d, v3 n)
{
    return sub(d, scl(n, 2.0 * dot(d, n)));
}

/* Reflective-side normal at a hit and the front-side test.
 *   sphere: the concave side faces the centre, n = (C - p)/R;
 *   rect: the given normal; triangle: the unit geometric normal for the
 *   side test, interpolated vertex normals (smooth materials) to reflect. */
static void surface_normals(const o_scene *sc, const o_cand *h, v3 p,
                            v3 *n_geo, v3 *n_shade)
{
    if (h->kind == PRIM_SPHERE) {
        const o_sphere *sp = &sc->spheres[h->index];
        *n_geo = scl(sub(sp->c, p), 1.0 / sp->R);
        *n_shade = unit(*n_geo);
        *n_geo = *n_shade;
    } else if (h->kind == PRIM_RECT) {
        *n_geo = *n_shade = sc->rects[h->index].n;
    } else {
        const o_tri *t = &sc->tris[h->index];
        *n_geo = t->ng;
        const o_material_in *m = &sc->materials[t->material];
        if (m->flags & MAT_SMOOTH) {
            double b0 = 1.0 - h->b1 - h->b2;
            *n_shade = unit(add(add(scl(t->n0, b0), scl(t->n1, h->b1)),
                                scl(t->n2, h->b2)));
        } else {
            *n_shade = t->ng;
        }
    }
}

static int prim_material(const o_scene *sc, const o_cand *h)
{
    if (h->kind == PRIM_SPHERE) return sc->spheres[h->index].material;
    if (h->kind == PRIM_RECT) return sc->rects[h->index].material;
    return sc->tris[h->index].material;
}

/* Ray probe for the pins of the surface geometry: nearest hit of each ray
 * (prim, t; -1 and INFINITY if none), the normals at the hit (geometric, and
 * the one the reflection uses), the graze bits of the nearest-hit decision
 * and the distance of the nearest hit on the skipped surface. */
void oracle_probe(void *scene, int64_t n, const double *o, const double *d,
                  const int32_t *skip, double t_min, double eps, int32_t *prim_out,
                  double *t_out, double *n_geo_out, double *n_shade_out,
                  int32_t *graze_out, double *skipped_t_out)
{
    const o_scene *sc = (const o_scene *)scene;
    for (int64_t i = 0; i < n; ++i) {
        o_cand h;
        int g = 0;
        double st;
        v3 oo = mk(o[3 * i], o[3 * i + 1], o[3 * i + 2]);
        v3 dd = mk(d[3 * i], d[3 * i + 1], d[3 * i + 2]);
        int f = nearest(sc, oo, dd, skip ? skip[i] : -1, t_min, eps, 1, &h, &g, &st);
        v3 ng = mk(0, 0, 0), ns = mk(0, 0, 0);
        if (f) surface_normals(sc, &h, add(oo, scl(dd, h.t)), &ng, &ns);
        prim_out[i] = f ? h.prim : -1;
        t_out[i] = f ? h.t : INFINITY;
        n_geo_out[3 * i] = ng.x; n_geo_out[3 * i + 1] = ng.y; n_geo_out[3 * i + 2] = ng.z;
        n_shade_out[3 * i] = ns.x; n_shade_out[3 * i + 1] = ns.y; n_shade_out[3 * i + 2] = ns.z;
        graze_out[i] = g;
        skipped_t_out[i] = st;
    }
}

typedef struct {
    int fate, plane, ix, iy, n_refl, graze;
    double u, v;
    v3 o, d;
} o_result;

/* Acceptance probability of the efficiencies applied before propagation
 * (Sec. 4.3: "the three efficiencies" -- the detector's quantum efficiency
 * and the reflectivities of the mirrors on the photon's way -- combined in
 * one accept/reject per photon at its wavelength): the product of the
 * listed tables, in FP32, multiplied left to right. */
static float prefilter_prob(const o_scene *sc, const o_params *prm, float lam)
{
    volatile float P = table_eval(&sc->tables[prm->prefilter_tables[0]], lam);
    for (int k = 1; k < prm->n_prefilter; ++k) {
        volatile float f = table_eval(&sc->tables[prm->prefilter_tables[k]], lam);
        P = P * f;
    }
    return P;
}

/* Photon that failed the efficiencies before propagation: not traced. */
static void prefiltered(const o_photon *ph, float P, const o_params *prm,
                        o_result *res)
{
    memset(res, 0, sizeof *res);
    res->plane = -1;
    res->fate = FATE_PREFILTERED;
    res->o = ph->o;
    res->d = ph->d;
    if (fabs(ph->u_qe - (double)P) < prm->prob_eps) res->graze = 2;
}

/* Trace one photon to its fate. With `filtered` set the photon has already
 * passed the efficiencies before propagation (Sec. 4.3): mirrors reflect it
 * and the detector records it without a further random test. */
static void trace_photon(const o_scene *sc, const o_params *prm,
                         const o_photon *ph, o_result *res, int32_t *path,
                         int filtered)
{
    v3 o = ph->o, d = unit(ph->d);
    int skip = -1, n_refl = 0, graze = 0;
    int n_turn = 0;     /* direction changes: reflections and refractions */
    memset(res, 0, sizeof *res);
    res->plane = -1;
    res->fate = FATE_MAX_STEPS;
    for (int k = 0; path && k < prm->max_steps; ++k) path[k] = -1;
    for (int step = 0; step < prm->max_steps; ++step) {
        o_cand h;
        int g = 0;
        if (!nearest(sc, o, d, skip, prm->t_min, prm->eps, prm->use_bvh, &h,
                     &g, NULL)) {
            graze |= (g & 8) | ((g & ~8) ? 1 : 0);
            res->fate = FATE_ESCAPED;
            break;
        }
        graze |= (g & 8) | ((g & ~8) ? 1 : 0);
        if (path) path[step] = h.prim;
        v3 p = add(o, scl(d, h.t));
        v3 n_geo, n_sh;
        surface_normals(sc, &h, p, &n_geo, &n_sh);
        double cosi = dot(d, n_geo);
        if (fabs(cosi) < 1e-9) graze |= 1;
        int front = cosi < 0.0;
        const o_material_in *m = &sc->materials[prim_material(sc, &h)];
        if (m->kind == MAT_ABSORBER) {
            res->fate = FATE_ABSORBED;
            o = p;
            break;
        }
        if (m->kind == MAT_MIRROR) {
            if (!front) { res->fate = FATE_ABSORBED; o = p; break; }
            if (n_turn >= prm->max_bounces) {
                res->fate = FATE_MAX_BOUNCES;
                o = p;
                break;
            }
            if (!filtered) {
                float P = table_eval(&sc->tables[m->table], ph->lambda);
                double u = ph->u_refl[n_refl];
                if (fabs(u - (double)P) < prm->prob_eps) graze |= 2;
                if (!(u < (double)P)) {
                    res->fate = FATE_MIRROR_ABSORBED;
                    o = p;
                    break;
                }
            }
            d = unit(reflect(d, n_sh));
            n_refl++;
            n_turn++;
            o = p;
            skip = h.prim;
            continue;
        }
        if (m->kind == MAT_DIELECTRIC) {
            /* refracting boundary (a window face): the table gives the index
             * n_w(lambda) of the medium behind the surface relative to the
             * one in front. Snell's law with the normal N facing the ray,
             * eta = n_in / n_out: d' = eta d + (eta c1 - sqrt(k)) N,
             * c1 = -d.N, k = 1 - eta^2 (1 - c1^2); total internal
             * reflection when k < 0 */
            if (n_turn >= prm->max_bounces) {
                res->fate = FATE_MAX_BOUNCES;
                o = p;
                break;
            }
            double nw = (double)table_eval(&sc->tables[m->table], ph->lambda);
            double eta = front ? 1.0 / nw : nw;
            v3 N = front ? n_geo : scl(n_geo, -1.0);
            double c1 = -dot(d, N);
            double k = 1.0 - eta * eta * (1.0 - c1 * c1);
            if (fabs(k) < 1e-6) graze |= 1;   /* near the critical angle */
            if (k < 0.0)
                d = unit(reflect(d, N));
            else
                d = unit(add(scl(d, eta), scl(N, eta * c1 - sqrt(k))));
            n_turn++;
            o = p;
            skip = h.prim;
            continue;
        }
        /* detector */
        if (!front) {   /* transparent from behind */
            o = p;
            skip = h.prim;
            continue;
        }
        o = p;
        if (!filtered) {
            float P = table_eval(&sc->tables[m->table], ph->lambda);
            if (fabs(ph->u_qe - (double)P) < prm->prob_eps) graze |= 2;
            if (!(ph->u_qe < (double)P)) {
                res->fate = FATE_QE_REJECTED;
                break;
            }
        }
        const o_rect *rc = &sc->rects[h.index];
        v3 q = sub(p, rc->o);
        double u = dot(q, rc->u), v = dot(q, rc->v);
        int ix = (int)floor(u / rc->pitch), iy = (int)floor(v / rc->pitch);
        if (ix > rc->nx - 1) ix = rc->nx - 1;
        if (iy > rc->ny - 1) iy = rc->ny - 1;
        if (ix < 0) ix = 0;
        if (iy < 0) iy = 0;
        double mu = fmin(u - ix * rc->pitch, (ix + 1) * rc->pitch - u);
        double mv = fmin(v - iy * rc->pitch, (iy + 1) * rc->pitch - v);
        if (fmin(mu, mv) < prm->eps) graze |= 4;
        res->fate = FATE_DETECTED;
        res->plane = m->plane;
        res->ix = ix;
        res->iy = iy;
        res->u = u;
        res->v = v;
        break;
    }
    res->n_refl = n_refl;
    res->graze = graze;
    res->o = o;
    res->d = d;
}

/* ------------------------------------------------------------------------ */
/* 6. Drivers: the photons of a range of tracks, or photons supplied by the */
/*    caller (the photon emitter's vectors of positions and momenta,        */
/*    Sec. 4.2).                                                            */
/* ------------------------------------------------------------------------ */
/* One emitted photon to its fate, with the efficiencies applied before
 * propagation when the parameters list them (Sec. 4.3). */
static void propagate(const o_scene *sc, const o_params *prm, const o_photon *ph,
                      o_result *r, int32_t *path)
{
    int run = 1;
    if (prm->n_prefilter > 0) {
        /* Sec. 4.3: accept/reject on the product of the efficiencies
         * before propagation, with the photon's QE uniform */
        float P = prefilter_prob(sc, prm, ph->lambda);
        if (!(ph->u_qe < (double)P)) {
            prefiltered(ph, P, prm, r);
            if (path) for (int k = 0; k < prm->max_steps; ++k) path[k] = -1;
            run = 0;
        } else if (fabs(ph->u_qe - (double)P) < prm->prob_eps) {
            run = 2;
        }
    }
    if (run) {
        trace_photon(sc, prm, ph, r, path, prm->n_prefilter > 0);
        if (run == 2) r->graze |= 2;
    }
    r->graze |= ph->graze;
}

/* Store the result of photon g (event ev) in the output arrays, count its
 * pixel and add it to its event's sums. */
static void record_photon(const o_scene *sc, const o_photon_out *out, int64_t g,
                          int64_t ev, float lambda, const o_result *r)
{
    if (out->fate) out->fate[g] = (uint8_t)r->fate;
    if (out->plane) out->plane[g] = r->plane;
    if (out->ix) out->ix[g] = r->ix;
    if (out->iy) out->iy[g] = r->iy;
    if (out->u) out->u[g] = r->u;
    if (out->v) out->v[g] = r->v;
    if (out->lambda) out->lambda[g] = lambda;
    if (out->n_refl) out->n_refl[g] = (uint8_t)r->n_refl;
    if (out->graze) out->graze[g] = (uint8_t)r->graze;
    if (out->dir_out) {
        out->dir_out[3 * g] = r->d.x;
        out->dir_out[3 * g + 1] = r->d.y;
        out->dir_out[3 * g + 2] = r->d.z;
    }
    if (out->pos_out) {
        out->pos_out[3 * g] = r->o.x;
        out->pos_out[3 * g + 1] = r->o.y;
        out->pos_out[3 * g + 2] = r->o.z;
    }
    if (r->fate == FATE_DETECTED && ev < out->n_hist_events) {
        if (out->pixel_counts) {
            int64_t idx = ev * sc->pixels_per_event + sc->plane_offset[r->plane] +
                          (int64_t)r->iy * sc->plane_nx[r->plane] + r->ix;
#ifdef _OPENMP
#pragma omp atomic
#endif
            out->pixel_counts[idx] += 1u;
        }
        if (out->event_sums) {
            double *es = out->event_sums + (ev * sc->n_planes + r->plane) * 4;
#ifdef _OPENMP
#pragma omp critical(oracle_sums)
#endif
            {
                es[0] += 1.0;
                es[1] += r->u;
                es[2] += r->v;
                es[3] += (double)lambda;
            }
        }
    }
}

static int check_params(const o_scene *sc, const o_params *prm)
{
    if (prm->max_steps > 16 || prm->max_bounces > 8) return -1;
    if (prm->n_prefilter < 0 || prm->n_prefilter > 4) return -1;
    if (prm->source != SRC_CHERENKOV && prm->source != SRC_ISOTROPIC) return -1;
    for (int k = 0; k < prm->n_prefilter; ++k)
        if (prm->prefilter_tables[k] < 0 || prm->prefilter_tables[k] >= sc->n_tables)
            return -1;
    return 0;
}

/* All photons of tracks [track_begin, track_end), emitted from the tracks. */
int oracle_trace(void *scene, const o_tracks_in *t, const o_params *prm,
                 const uint64_t *offsets, int64_t track_begin,
                 int64_t track_end, const o_photon_out *out)
{
    const o_scene *sc = (const o_scene *)scene;
    if (check_params(sc, prm)) return -1;
    int64_t first = (int64_t)offsets[track_begin];
    int64_t last = (int64_t)offsets[track_end];
#ifdef _OPENMP
    if (prm->n_threads > 0) omp_set_num_threads(prm->n_threads);
#pragma omp parallel for schedule(dynamic, 256)
#endif
    for (int64_t g = first; g < last; ++g) {
        /* track containing photon g: last i with offsets[i] <= g */
        int64_t lo = track_begin, hi = track_end - 1;
        while (lo < hi) {
            int64_t mid = (lo + hi + 1) / 2;
            if ((int64_t)offsets[mid] <= g) lo = mid; else hi = mid - 1;
        }
        uint32_t j = (uint32_t)(g - (int64_t)offsets[lo]);
        o_photon ph;
        emit_photon(t, prm, lo, j, &ph);
        o_result r;
        int32_t *path = out->path ? out->path + g * prm->max_steps : NULL;
        propagate(sc, prm, &ph, &r, path);
        record_photon(sc, out, g, (int64_t)t->event[lo], ph.lambda, &r);
    }
    return 0;
}

/* Photons given by the caller (Sec. 4.2: the emitter takes vectors of
 * positions and momenta): origin (mm) and direction as FP32 triples, the
 * wavelength (nm), and the key (event, track, photon) that selects the
 * photon's reflectivity and QE draws (blocks 0-2 of the draw map, as for an
 * emitted photon with the same key); prm->seed keys the generator. The
 * direction need not be exactly of unit length: it is normalised in FP64.
 * Results are indexed by the photon's position in the arrays. */
int oracle_trace_photons(void *scene, int64_t n, const float *origin, const float *dir,
                         const float *lambda, const uint32_t *event, const uint32_t *track,
                         const uint32_t *photon, const o_params *prm,
                         const o_photon_out *out)
{
    const o_scene *sc = (const o_scene *)scene;
    if (check_params(sc, prm)) return -1;
#ifdef _OPENMP
    if (prm->n_threads > 0) omp_set_num_threads(prm->n_threads);
#pragma omp parallel for schedule(dynamic, 256)
#endif
    for (int64_t g = 0; g < n; ++g) {
        uint32_t w0[4], w1[4], w2[4];
        draw_block(prm->seed, event[g], track[g], photon[g], 0, w0);
        draw_block(prm->seed, event[g], track[g], photon[g], 1, w1);
        draw_block(prm->seed, event[g], track[g], photon[g], 2, w2);
        o_photon ph;
        memset(&ph, 0, sizeof ph);
        ph.o = fromf(origin + 3 * g);
        ph.d = fromf(dir + 3 * g);
        ph.lambda = lambda[g];
        ph.u_qe = u24(w0[3]);
        for (int k = 0; k < 4; ++k) {
            ph.u_refl[k] = u24(w1[k]);
            ph.u_refl[4 + k] = u24(w2[k]);
        }
        o_result r;
        int32_t *path = out->path ? out->path + g * prm->max_steps : NULL;
        propagate(sc, prm, &ph, &r, path);
        record_photon(sc, out, g, (int64_t)event[g], ph.lambda, &r);
    }
    return 0;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* 7. Gradient of the soft ring chi^2 with respect to the mirror tilts, the */
/*    radius of curvature and n - 1 (the differentiation pattern).          */
/*                                                                          */
/* Parameters theta[0..9]: (alpha_k, beta_k) for sphere tiles k = 0..3 --   */
/* rotation of the tile about the axis through its pole P_k = C_k + R a_k   */
/* parallel to its nominal e1 by alpha_k, then about the nominal e2 by      */
/* beta_k (Rodrigues' formula); theta[8] = radius of curvature of every     */
/* sphere tile (pole fixed: C = P - R a); theta[9] = n - 1.                 */
/* Loss over the detected photons whose (track, plane) target has weight    */
/* > 0: the hit (u, v) is smeared by sigma (g1, g2), a Box-Muller pair from */
/* the photon's draw block 3, rho = (|(u~, v~) - (cu, cv)| - r) / sigma and */
/* L = mean rho^2. Derivatives follow the photon's recorded sequence of     */
/* reflecting surfaces (fixed topology: each surface extended past its     */
/* edges), by forward-mode dual numbers with 10 tangents, and separately   */
/* by central finite differences of the same replay.                        */
/* ------------------------------------------------------------------------ */
#define NG 10
typedef struct { double v; double d[NG]; } dn;
typedef struct { dn x, y, z; } dv;

static dn dc(double v) { dn r; r.v = v; memset(r.d, 0, sizeof r.d); return r; }
static dn dadd(dn a, dn b) { for (int k = 0; k < NG; ++k) a.d[k] += b.d[k]; a.v += b.v; return a; }
static dn dsub(dn a, dn b) { for (int k = 0; k < NG; ++k) a.d[k] -= b.d[k]; a.v -= b.v; return a; }
static dn dmul(dn a, dn b)
{
    dn r; r.v = a.v * b.v;
    for (int k = 0; k < NG; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
    return r;
}
static dn dscl(dn a, double s) { for (int k = 0; k < NG; ++k) a.d[k] *= s; a.v *= s; return a; }
static dn ddiv(dn a, dn b)
{
    dn r; r.v = a.v / b.v;
    for (int k = 0; k < NG; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) / b.v;
    return r;
}
static dn dsqrt(dn a)
{
    dn r; r.v = sqrt(a.v);
    for (int k = 0; k < NG; ++k) r.d[k] = a.d[k] / (2.0 * r.v);
    return r;
}
static dn dsin(dn a)
{
    dn r; r.v = sin(a.v); double c = cos(a.v);
    for (int k = 0; k < NG; ++k) r.d[k] = c * a.d[k];
    return r;
}
static dn dcos(dn a)
{
    dn r; r.v = cos(a.v); double s = -sin(a.v);
    for (int k = 0; k < NG; ++k) r.d[k] = s * a.d[k];
    return r;
}
static dv dvc(v3 a) { dv r = {dc(a.x), dc(a.y), dc(a.z)}; return r; }
static dv dvadd(dv a, dv b) { dv r = {dadd(a.x, b.x), dadd(a.y, b.y), dadd(a.z, b.z)}; return r; }
static dv dvsub(dv a, dv b) { dv r = {dsub(a.x, b.x), dsub(a.y, b.y), dsub(a.z, b.z)}; return r; }
static dv dvscl(dv a, dn s) { dv r = {dmul(a.x, s), dmul(a.y, s), dmul(a.z, s)}; return r; }
static dn dvdot(dv a, dv b) { return dadd(dadd(dmul(a.x, b.x), dmul(a.y, b.y)), dmul(a.z, b.z)); }
static dn dvdotc(dv a, v3 b)
{
    return dadd(dadd(dscl(a.x, b.x), dscl(a.y, b.y)), dscl(a.z, b.z));
}
/* u x v with u a fixed vector */
static dv dcrossc(v3 u, dv v)
{
    dv r = {dsub(dscl(v.z, u.y), dscl(v.y, u.z)), dsub(dscl(v.x, u.z), dscl(v.z, u.x)),
            dsub(dscl(v.y, u.x), dscl(v.x, u.y))};
    return r;
}
/* Rodrigues: v cos(phi) + (u x v) sin(phi) + u (u.v)(1 - cos(phi)), u unit */
static dv drot(v3 u, dn phi, dv v)
{
    dn c = dcos(phi), s = dsin(phi);
    dn uv = dvdotc(v, u);
    dn k = dmul(uv, dsub(dc(1.0), c));
    dv a = dvscl(v, c);
    dv b = dvscl(dcrossc(u, v), s);
    dv w = {dmul(dc(u.x), k), dmul(dc(u.y), k), dmul(dc(u.z), k)};
    return dvadd(dvadd(a, b), w);
}

typedef struct {
    dv c, a, e1, e2;
    dn R;
} o_tile_d;

/* Tile k at parameters theta (duals). */
static o_tile_d tile_at(const o_sphere *sp, int k, const dn th[NG])
{
    v3 P = add(sp->c, scl(sp->axis, sp->R));
    dn al = k < 4 ? th[2 * k] : dc(0.0);
    dn be = k < 4 ? th[2 * k + 1] : dc(0.0);
    o_tile_d t;
    t.a = drot(sp->e2, be, drot(sp->e1, al, dvc(sp->axis)));
    t.e1 = drot(sp->e2, be, drot(sp->e1, al, dvc(sp->e1)));
    t.e2 = drot(sp->e2, be, drot(sp->e1, al, dvc(sp->e2)));
    t.R = th[8];
    t.c = dvsub(dvc(P), dvscl(t.a, t.R));
    return t;
}

/* Plain-double transformed copy of the scene's tiles at theta. */
static void tiles_at_theta(const o_scene *nom, const double theta[NG], o_sphere *out)
{
    dn th[NG];
    for (int k = 0; k < NG; ++k) th[k] = dc(theta[k]);
    for (int i = 0; i < nom->n_spheres; ++i) {
        o_tile_d t = tile_at(&nom->spheres[i], i, th);
        out[i] = nom->spheres[i];
        out[i].c = mk(t.c.x.v, t.c.y.v, t.c.z.v);
        out[i].axis = mk(t.a.x.v, t.a.y.v, t.a.z.v);
        out[i].e1 = mk(t.e1.x.v, t.e1.y.v, t.e1.z.v);
        out[i].e2 = mk(t.e2.x.v, t.e2.y.v, t.e2.z.v);
        out[i].R = t.R.v;
    }
}

static dv dreflect(dv d, dv n)
{
    dn k = dscl(dvdot(d, n), 2.0);
    return dvsub(d, dvscl(n, k));
}

/* Replay of one detected photon along its reflecting surfaces with duals.
 * refl: primitive ids of the reflections in order; det: detector rectangle. */
static void replay_dual(const o_scene *nom, const o_tracks_in *t, const o_params *prm,
                        int64_t i, uint32_t j, const int32_t *refl, int n_refl,
                        int det, const dn th[NG], dn *u_out, dn *v_out)
{
    uint32_t event = t->event[i];
    uint32_t tid = t->id ? t->id[i] : (uint32_t)i;
    uint32_t w0[4];
    draw_block(prm->seed, event, tid, j, 0, w0);
    v3 dir = unit(mk(t->dx[i], t->dy[i], t->dz[i]));
    double s = u24(w0[0]) * (double)t->length[i];
    dv o = dvc(add(mk(t->x[i], t->y[i], t->z[i]), scl(dir, s)));
    double phi = 2.0 * PI_D * u24(w0[1]);
    double beta = track_beta(t->p[i], t->mass[i]);
    dn nb = dscl(dadd(dc(1.0), th[9]), beta);
    dn ct = ddiv(dc(1.0), nb);
    dn one_m = dsub(dc(1.0), dmul(ct, ct));
    dn st;
    if (one_m.v > 0.0) {
        st = dsqrt(one_m);
    } else {   /* below threshold: the emission leaves along the track */
        ct = dc(1.0);
        st = dc(0.0);
    }
    v3 e1, e2;
    basis(dir, &e1, &e2);
    v3 tr = add(scl(e1, cos(phi)), scl(e2, sin(phi)));
    dv d = dvadd(dvscl(dvc(dir), ct), dvscl(dvc(tr), st));
    for (int k = 0; k < n_refl; ++k) {
        int prim = refl[k];
        dv n;
        if (prim < nom->n_spheres) {
            o_tile_d tl = tile_at(&nom->spheres[prim], prim, th);
            dv w = dvsub(o, tl.c);
            dn b = dvdot(w, d);
            dn c = dsub(dvdot(w, w), dmul(tl.R, tl.R));
            dn sq = dsqrt(dsub(dmul(b, b), c));
            /* exit root (concave side) in the form free of cancellation */
            dn tt = b.v <= 0.0 ? dsub(sq, b) : ddiv(c, dsub(dscl(b, -1.0), sq));
            o = dvadd(o, dvscl(d, tt));
            n = dvscl(dvsub(tl.c, o), ddiv(dc(1.0), tl.R));
        } else if (prim < nom->n_spheres + nom->n_rects) {
            const o_rect *rc = &nom->rects[prim - nom->n_spheres];
            n = dvc(rc->n);
            dn tt = ddiv(dvdotc(dvsub(dvc(rc->o), o), rc->n), dvdotc(d, rc->n));
            o = dvadd(o, dvscl(d, tt));
        } else {
            const o_tri *tri = &nom->tris[prim - nom->n_spheres - nom->n_rects];
            dn tt = ddiv(dvdotc(dvsub(dvc(tri->v0), o), tri->ng), dvdotc(d, tri->ng));
            o = dvadd(o, dvscl(d, tt));
            const o_material_in *m = &nom->materials[tri->material];
            if (m->flags & MAT_SMOOTH) {
                v3 ea = sub(tri->v1, tri->v0), eb = sub(tri->v2, tri->v0);
                dv q = dvsub(o, dvc(tri->v0));
                double d00 = dot(ea, ea), d01 = dot(ea, eb), d11 = dot(eb, eb);
                dn d20 = dvdotc(q, ea), d21 = dvdotc(q, eb);
                double den = d00 * d11 - d01 * d01;
                dn b1 = dscl(dsub(dscl(d20, d11), dscl(d21, d01)), 1.0 / den);
                dn b2 = dscl(dsub(dscl(d21, d00), dscl(d20, d01)), 1.0 / den);
                dn b0 = dsub(dsub(dc(1.0), b1), b2);
                dv nn = dvadd(dvadd(dvscl(dvc(tri->n0), b0), dvscl(dvc(tri->n1), b1)),
                              dvscl(dvc(tri->n2), b2));
                n = dvscl(nn, ddiv(dc(1.0), dsqrt(dvdot(nn, nn))));
            } else {
                n = dvc(tri->ng);
            }
        }
        d = dreflect(d, n);
        /* keep |d| = 1 exactly as the forward trace renormalises */
        d = dvscl(d, ddiv(dc(1.0), dsqrt(dvdot(d, d))));
    }
    const o_rect *rc = &nom->rects[det];
    dn tt = ddiv(dvdotc(dvsub(dvc(rc->o), o), rc->n), dvdotc(d, rc->n));
    dv q = dvsub(dvadd(o, dvscl(d, tt)), dvc(rc->o));
    *u_out = dvdotc(q, rc->u);
    *v_out = dvdotc(q, rc->v);
}

/* Box-Muller pair from draw block 3 (words 0 and 1). */
static void smear_pair(uint64_t seed, uint32_t event, uint32_t tid, uint32_t j,
                       double *g1, double *g2)
{
    uint32_t w[4];
    draw_block(seed, event, tid, j, 3, w);
    double u1 = ((double)(w[0] >> 8) + 0.5) * (1.0 / 16777216.0);
    double u2 = u24(w[1]);
    double r = sqrt(-2.0 * log(u1));
    *g1 = r * cos(2.0 * PI_D * u2);
    *g2 = r * sin(2.0 * PI_D * u2);
}

/* rho = (|h~ - c| - r) / sigma with dual hit coordinates */
static dn ring_residual(dn u, dn v, double g1, double g2, const float *tg, double sigma)
{
    dn du = dadd(u, dc(sigma * g1 - tg[0]));
    dn dvv = dadd(v, dc(sigma * g2 - tg[1]));
    dn dist = dsqrt(dadd(dmul(du, du), dmul(dvv, dvv)));
    return dscl(dsub(dist, dc(tg[2])), 1.0 / sigma);
}

/* Loss, gradient (dual numbers) and central-difference gradient at theta.
 * targets: [n_tracks][n_planes][4] = (cu, cv, r, weight); hits of a
 * (track, plane) with weight <= 0 are not used. h_angle: step of the tilt
 * differences (rad); h_rel: relative step for R and n - 1. grad_fd may be
 * NULL (no differences). Returns the number of hits used, or -1. */
int64_t oracle_trace_grad(void *scene, const o_tracks_in *t, const o_params *prm_in,
                          const double theta[NG], const float *targets, int n_planes,
                          double sigma, double h_angle, double h_rel, double *loss,
                          double *grad, double *grad_fd)
{
    const o_scene *nom = (const o_scene *)scene;
    if (prm_in->max_steps > 16 || prm_in->max_bounces > 8) return -1;
    o_params prm = *prm_in;
    prm.n_minus_1 = theta[9];
    /* the scene at theta (forward trace decides the topology) */
    o_scene at = *nom;
    at.spheres = (o_sphere *)calloc((size_t)nom->n_spheres + 1, sizeof(o_sphere));
    tiles_at_theta(nom, theta, at.spheres);
    uint64_t *off = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)t->n + 1));
    oracle_yield(t, &prm, NULL, NULL, off);
    int64_t total = (int64_t)off[t->n];
    double hk[NG];
    for (int k = 0; k < NG; ++k) hk[k] = k < 8 ? h_angle : h_rel * fabs(theta[k]);
    double acc_l = 0.0, acc_g[NG] = {0}, acc_fd[NG] = {0};
    int64_t used = 0;
#ifdef _OPENMP
    if (prm.n_threads > 0) omp_set_num_threads(prm.n_threads);
#pragma omp parallel
#endif
    {
        double l_l = 0.0, l_g[NG] = {0}, l_fd[NG] = {0};
        int64_t l_used = 0;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 256)
#endif
        for (int64_t g = 0; g < total; ++g) {
            int64_t lo = 0, hi = t->n - 1;
            while (lo < hi) {
                int64_t mid = (lo + hi + 1) / 2;
                if ((int64_t)off[mid] <= g) lo = mid; else hi = mid - 1;
            }
            uint32_t j = (uint32_t)(g - (int64_t)off[lo]);
            o_photon ph;
            emit_photon(t, &prm, lo, j, &ph);
            int32_t path[16];
            o_result r;
            trace_photon(&at, &prm, &ph, &r, path, 0);
            if (r.fate != FATE_DETECTED) continue;
            const float *tg = targets + ((size_t)lo * n_planes + r.plane) * 4;
            if (!(tg[3] > 0.0f)) continue;
            int32_t refl[16];
            int nr = 0, det = -1;
            for (int s = 0; s < prm.max_steps && path[s] >= 0; ++s) {
                int prim = path[s];
                int mat;
                if (prim < at.n_spheres) mat = at.spheres[prim].material;
                else if (prim < at.n_spheres + at.n_rects) mat = at.rects[prim - at.n_spheres].material;
                else mat = at.tris[prim - at.n_spheres - at.n_rects].material;
                if (at.materials[mat].kind == MAT_MIRROR) refl[nr++] = prim;
                det = prim;
            }
            det -= at.n_spheres;   /* detector rectangle index */
            double g1, g2;
            smear_pair(prm.seed, t->event[lo], t->id ? t->id[lo] : (uint32_t)lo, j, &g1, &g2);
            dn th[NG];
            for (int k = 0; k < NG; ++k) { th[k] = dc(theta[k]); th[k].d[k] = 1.0; }
            dn u, v;
            replay_dual(nom, t, &prm, lo, j, refl, nr, det, th, &u, &v);
            dn rho = ring_residual(u, v, g1, g2, tg, sigma);
            l_l += rho.v * rho.v;
            for (int k = 0; k < NG; ++k) l_g[k] += 2.0 * rho.v * rho.d[k];
            l_used++;
            if (grad_fd) {
                for (int k = 0; k < NG; ++k) {
                    dn tp[NG], tm[NG];
                    for (int q = 0; q < NG; ++q) { tp[q] = dc(theta[q]); tm[q] = dc(theta[q]); }
                    tp[k].v += hk[k];
                    tm[k].v -= hk[k];
                    dn up, vp, um, vm;
                    replay_dual(nom, t, &prm, lo, j, refl, nr, det, tp, &up, &vp);
                    replay_dual(nom, t, &prm, lo, j, refl, nr, det, tm, &um, &vm);
                    double rp = ring_residual(up, vp, g1, g2, tg, sigma).v;
                    double rm = ring_residual(um, vm, g1, g2, tg, sigma).v;
                    l_fd[k] += (rp * rp - rm * rm) / (2.0 * hk[k]);
                }
            }
        }
#ifdef _OPENMP
#pragma omp critical(oracle_grad)
#endif
        {
            acc_l += l_l;
            used += l_used;
            for (int k = 0; k < NG; ++k) { acc_g[k] += l_g[k]; acc_fd[k] += l_fd[k]; }
        }
    }
    double inv = used ? 1.0 / (double)used : 0.0;
    *loss = acc_l * inv;
    for (int k = 0; k < NG; ++k) {
        grad[k] = acc_g[k] * inv;
        if (grad_fd) grad_fd[k] = acc_fd[k] * inv;
    }
    free(off);
    free(at.spheres);
    return used;
}

/* Hits of the forward trace at theta (for ring targets and checks): same as
 * oracle_trace on the transformed scene with n - 1 = theta[9]. */
int oracle_trace_at(void *scene, const o_tracks_in *t, const o_params *prm_in,
                    const double theta[NG], const uint64_t *offsets,
                    const o_photon_out *out)
{
    const o_scene *nom = (const o_scene *)scene;
    o_params prm = *prm_in;
    prm.n_minus_1 = theta[9];
    o_scene at = *nom;
    at.spheres = (o_sphere *)calloc((size_t)nom->n_spheres + 1, sizeof(o_sphere));
    tiles_at_theta(nom, theta, at.spheres);
    int rc = oracle_trace(&at, t, &prm, offsets, 0, t->n, out);
    free(at.spheres);
    return rc;
}

/* Hit position and its derivatives d(u, v)/d(theta_k) of one photon (track
 * i, photon j) at theta. Returns the photon's fate; u, v, du, dv are set
 * when it is detected. */
int oracle_hit_jacobian(void *scene, const o_tracks_in *t, const o_params *prm_in,
                        const double theta[NG], int64_t i, uint32_t j, double *u,
                        double *v, double *du, double *dv_)
{
    const o_scene *nom = (const o_scene *)scene;
    o_params prm = *prm_in;
    prm.n_minus_1 = theta[9];
    o_scene at = *nom;
    at.spheres = (o_sphere *)calloc((size_t)nom->n_spheres + 1, sizeof(o_sphere));
    tiles_at_theta(nom, theta, at.spheres);
    o_photon ph;
    emit_photon(t, &prm, i, j, &ph);
    int32_t path[16];
    o_result r;
    trace_photon(&at, &prm, &ph, &r, path, 0);
    if (r.fate == FATE_DETECTED) {
        int32_t refl[16];
        int nr = 0, det = -1;
        for (int s = 0; s < prm.max_steps && path[s] >= 0; ++s) {
            int prim = path[s];
            int mat;
            if (prim < at.n_spheres) mat = at.spheres[prim].material;
            else if (prim < at.n_spheres + at.n_rects) mat = at.rects[prim - at.n_spheres].material;
            else mat = at.tris[prim - at.n_spheres - at.n_rects].material;
            if (at.materials[mat].kind == MAT_MIRROR) refl[nr++] = prim;
            det = prim;
        }
        dn th[NG];
        for (int k = 0; k < NG; ++k) { th[k] = dc(theta[k]); th[k].d[k] = 1.0; }
        dn uu, vv;
        replay_dual(nom, t, &prm, i, j, refl, nr, det - at.n_spheres, th, &uu, &vv);
        *u = uu.v;
        *v = vv.v;
        for (int k = 0; k < NG; ++k) { du[k] = uu.d[k]; dv_[k] = vv.d[k]; }
    }
    free(at.spheres);
    return r.fate;
}
