// rich_kernels.cu -- sm_103a kernels of the Cherenkov photon propagator.
//
//   k_yield        one thread per track, double-word FP32: beta, Cherenkov angle
//                  (cos theta = 1/(n beta), Sec. 3), Frank-Tamm mean and the
//                  keyed Poisson photon count; block sums of the counts.
//   k_offsets      exclusive scan of the counts into photon offsets
//                  (deterministic two-pass scan: block prefix from the block
//                  sums, then an in-block warp-shuffle scan).
//   k_materialize  optional: photons written out as a structure of arrays
//                  (the "vector of positions and momenta" of Sec. 4.2).
//   k_trace        persistent propagation kernel: warps take chunks of
//                  photons from an atomic queue, generate them in registers
//                  (fused emission), trace them bounce by bounce and refill
//                  idle lanes with new photons (warp-level compaction by
//                  ballot/popc), apply reflectivity and quantum-efficiency
//                  accept/reject in flight (Sec. 4.3 and Sec. 6), append
//                  hits with warp-aggregated atomics and bin them.
#include <climits>
#include <cstdint>
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <utility>
#include <math_constants.h>

#include "rich_device.cuh"
#include "rich_ff.cuh"
#include "rich_log_tables.h"
#include "rich_trig_tables.h"

namespace rich {

constexpr unsigned kFull = 0xFFFFFFFFu;

// The photon state the BVH walk does not use (wavelength, the QE and
// reflectivity words, the keys, indices and counters) kept in per-thread
// shared memory instead of registers, by the two shapes of one block per SM
// (more than 256 threads).
#ifndef RICH_COLD_SMEM
#define RICH_COLD_SMEM 1
#endif
// Threads of the wide 72-register shape class (one block per SM at 896
// threads; with its cold photon state in shared memory it does not spill).
#ifndef RICH_WIDE_THREADS
#define RICH_WIDE_THREADS 896
#endif
constexpr int kYieldThreads = 256;   // tracks per scan group / scan block
constexpr int kYieldBlock = 32;      // threads per yield block: one warp, so
                                     // the per-track chains of a small batch
                                     // spread over as many SMs as possible
constexpr int kYieldLanes = 4;       // lanes per track (parallel Poisson trials)
constexpr double kAlpha = 1.0 / 137.035999;
constexpr double kPi = 3.14159265358979323846;
constexpr ff k2PiAlpha = ffc(2.0 * kPi * kAlpha);

int yield_block_threads() { return kYieldThreads; }

// Programmatic dependent launch: a kernel launched with the programmatic
// stream-serialisation attribute may be scheduled before the kernel ahead of
// it in the stream has ended (once that one has signalled); grid_dep_wait()
// returns when that kernel has completed and its memory is visible. Without
// the attribute both are no-ops. The waits are the hardware's, not spins.
__device__ __forceinline__ void grid_dep_wait() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void grid_dep_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Launch with the programmatic stream-serialisation attribute.
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*kern)(KArgs...), unsigned blocks, unsigned threads,
                              size_t smem, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

__device__ __forceinline__ void set_status(Counters *c, unsigned code) {
    atomicCAS(&c->status, 0u, code);
}

// ================================================================ yield
// Keyed stream of uniforms for the per-track Poisson draw: words x, y, z, w
// of blocks 0, 1, 2, ... with counter (block, 0xFFFFFFFF, track id, event).
struct TrackStream {
    uint32_t event, id, k0, k1, block, word;
    u4 w;
    // the next uniform, in FP32 (exact: 24 bits)
    __device__ float nextf() {
        if (word == 4) {
            w = philox10(block, 0xFFFFFFFFu, id, event, k0, k1);
            ++block;
            word = 0;
        }
        uint32_t v = word == 0 ? w.x : (word == 1 ? w.y : (word == 2 ? w.z : w.w));
        ++word;
        return u24f(v);
    }
};

// FP64 natural logarithm of a positive normal x, table-driven after Tang
// (ACM TOMS 16(4), 1990): x = 2^e m with m in [1, 2); c the centre of the
// 1/128-wide interval of m (its top 7 mantissa bits); r = m (1/c) - 1 with
// one fused multiply-add, |r| < 2^-8; log x = e log 2 + log(1/(1/c)) +
// log(1 + r), the last by its Taylor series to r^7 (truncation < 2^-59
// relative). log 2 is split so e * hi is exact. x = 0 gives -infinity.
__device__ __forceinline__ double log64(double x) {
    if (!(x > 0.0)) return -CUDART_INF;
    constexpr double kLn2Hi = 0x1.62e42fefa3800p-1, kLn2Lo = 0x1.ef35793c76730p-45;
    const long long bits = __double_as_longlong(x);
    const int e = (int)((bits >> 52) & 0x7FF) - 1023;
    const double m = __longlong_as_double((bits & 0x000FFFFFFFFFFFFFLL) | 0x3FF0000000000000LL);
    const int i = (int)((bits >> (52 - kLogTableBits)) & ((1 << kLogTableBits) - 1));
    const double inv_c = __ldg(&g_log_tab[i][0]);
    const double lc_hi = __ldg(&g_log_tab[i][1]), lc_lo = __ldg(&g_log_tab[i][2]);
    const double r = fma(m, inv_c, -1.0);
    double q = fma(r, 1.0 / 7.0, -1.0 / 6.0);           // log(1+r) = r + r^2 q(r)
    q = fma(q, r, 0.2);
    q = fma(q, r, -0.25);
    q = fma(q, r, 1.0 / 3.0);
    q = fma(q, r, -0.5);
    const double ed = (double)e;
    const double hi = fma(ed, kLn2Hi, lc_hi);
    const double lo = fma(ed, kLn2Lo, lc_lo);
    return hi + (r + fma(r * r, q, lo));
}

// ------------------------------------ double-word per-track arithmetic
// The per-track chain of the yield kernel (beta, angle, Frank-Tamm mean,
// Poisson draw) is one dependent sequence per thread. An FP64 instruction
// holds a warp for ~64 cycles on this GPU whatever its active lanes, so the
// chain runs in double-word FP32 arithmetic (rich_ff.cuh, ~2^-44 relative
// per operation against FP64's 2^-53): a count can differ from the FP64
// draw only if a floor or a rejection test lands within ~1e-10 of its
// threshold.

constexpr ff kLn2 = ffc(0.69314718055994530942);

// log of a double-word x with normal hi (2^-126 <= hi < 2^127), table-driven
// as log64 (Tang): x = 2^e m with m in [1, 2) (both parts scaled exactly),
// F the FP32 reciprocal of the centre of m's 1/128-wide interval (top 7
// mantissa bits of hi), r = m F - 1 (|r| < 2^-7); log x = e log 2 - log F +
// log(1 + r), with r - r^2/2 in double-word and the series' tail
// r^3 (1/3 - r/4 + r^2/5 - r^3/6 + r^4/7) in FP32 (below 2^-45). x = 0
// gives -infinity.
__device__ __forceinline__ ff ff_log(ff x) {
    if (!(x.hi > 0.0f)) return {__int_as_float((int)0xff800000), 0.0f};
    const int bits = __float_as_int(x.hi);
    const int e = ((bits >> 23) & 0xFF) - 127;
    const int i = (bits >> (23 - kLogTableBits)) & ((1 << kLogTableBits) - 1);
    const float sc = __int_as_float((127 - e) << 23);           // 2^-e
    const ff m = {x.hi * sc, x.lo * sc};
    const float F = __ldg(&g_log_tab_f[i][0]);
    const ff lc = {__ldg(&g_log_tab_f[i][1]), __ldg(&g_log_tab_f[i][2])};
    const ff r = ff_add(ff_mul(m, F), -1.0f);
    const float z = r.hi;
    const float tail =
        z * z * z * (1.0f / 3.0f - z * (0.25f - z * (0.2f - z * (1.0f / 6.0f - z * (1.0f / 7.0f)))));
    const ff r2 = ff_mul(r, r);
    const ff l1p = ff_add(ff_sub(r, ff{0.5f * r2.hi, 0.5f * r2.lo}), tail);
    const float ef = (float)e;
    const ff el = ff_add(two_prod(ef, kLn2.hi), ef * kLn2.lo);
    return ff_add(ff_add(el, lc), l1p);
}

// e^-x for 0 <= x < 80: x = k log 2 + r, |r| <= log(2)/2 + 2^-20, e^-r by
// its Taylor series (terms 8..12 in FP32, below 6e-9 of the sum; 0..7 in
// double-word Horner steps; truncation below 2^-52), then the exact
// scaling by 2^-k.
__device__ __forceinline__ ff ff_exp_neg(ff x) {
    const float kf = rintf(x.hi * 1.44269504f);
    const ff r = ff_sub(x, ff_add(two_prod(kf, kLn2.hi), kf * kLn2.lo));
    const ff z = ff_neg(r);
    const float zh = z.hi;
    const float q = 1.0f / 40320.0f +
                    zh * (1.0f / 362880.0f +
                          zh * (1.0f / 3628800.0f + zh * (1.0f / 39916800.0f + zh * (1.0f / 479001600.0f))));
    constexpr ff c7 = ffc(1.0 / 5040.0), c6 = ffc(1.0 / 720.0), c5 = ffc(1.0 / 120.0),
                 c4 = ffc(1.0 / 24.0), c3 = ffc(1.0 / 6.0);
    ff s = ff_add(c7, zh * q);
    s = ff_add(ff_mul(s, z), c6);
    s = ff_add(ff_mul(s, z), c5);
    s = ff_add(ff_mul(s, z), c4);
    s = ff_add(ff_mul(s, z), c3);
    s = ff_add(ff_mul(s, z), 0.5f);
    s = ff_add(ff_mul(s, z), 1.0f);
    s = ff_add(ff_mul(s, z), 1.0f);
    const float sc = __int_as_float((127 - (int)kf) << 23);      // 2^-k
    return {s.hi * sc, s.lo * sc};
}

// floor of a double-word as an integer (any magnitude below 2^62). The
// 32-bit conversions take the common case: 64-bit ones issue on the FP64
// pipe on this GPU.
__device__ __forceinline__ int64_t ff_floor_i64(ff a) {
    const float f = floorf(a.hi);
    if (f != a.hi) return (int64_t)__float2int_rz(f);  // |hi| < 2^23, lo cannot cross
    if (fabsf(a.hi) < 1.0e9f) return (int64_t)__float2int_rz(a.hi) + __float2int_rz(floorf(a.lo));
    return (int64_t)a.hi + (int64_t)floorf(a.lo);
}

// an integer (|k| < 2^48) as a double-word, exactly
__device__ __forceinline__ ff ff_from_i64(int64_t k) {
    if (k >= -(1ll << 24) && k <= (1ll << 24)) return ffv(__int2float_rn((int)k));
    const float hi = (float)k;
    return fast_two_sum(hi, (float)(k - (int64_t)hi));
}

// log k! (k >= 0): the table below 2048, Stirling's series above (four
// correction terms in FP32, truncation < 1/(1188 k^9)).
__device__ __forceinline__ ff ff_log_factorial(int64_t k) {
    if (k < kLogFactTable) return {__ldg(&g_logfact_ff[k][0]), __ldg(&g_logfact_ff[k][1])};
    constexpr ff kHalfLog2Pi = ffc(0.91893853320467274178);
    const ff x = ff_from_i64(k + 1);
    const float r = 1.0f / x.hi, r2 = r * r;
    const float series =
        r * (1.0f / 12.0f - r2 * (1.0f / 360.0f - r2 * (1.0f / 1260.0f - r2 * (1.0f / 1680.0f))));
    ff v = ff_mul(ff_add(x, -0.5f), ff_log(x));
    v = ff_sub(v, x);
    v = ff_add(v, kHalfLog2Pi);
    return ff_add(v, series);
}

// Poisson(mu): CDF inversion (smallest k with u < F(k)) below mean 10; the
// PTRS transformed rejection sampler (Hoermann 1993) above, at most 64
// trials, then round(mu); in double-word arithmetic. The rejection test
// log V + log(1/alpha) - log(a/us^2 + b) <= -mu + k log mu - log k! is
// taken as log(V us^2 / (alpha (a + b us^2))) with one logarithm and log k!
// from a table. The uniforms are 24-bit, exact in FP32, as are U, us and
// us^2 (the last as a double-word).
__device__ int64_t poisson_draw(ff mu, TrackStream &s) {
    if (!(mu.hi > 0.0f)) return 0;
    if (ff_lt(mu, ffv(10.0f))) {
        const ff u = ffv(s.nextf());
        ff pk = ff_exp_neg(mu), F = pk;
        int64_t k = 0;
        while (ff_le(F, u) && k < 1000) {
            k += 1;
            pk = ff_mul(pk, ff_div(mu, ffv(__int2float_rn((int)k))));
            F = ff_add(F, pk);
        }
        return k;
    }
    constexpr ff kB0 = ffc(0.931), kB1 = ffc(2.53), kA0 = ffc(-0.059), kA1 = ffc(0.02483),
                 kI0 = ffc(1.1239), kI1 = ffc(1.1328), kI2 = ffc(3.4), kV0 = ffc(0.9277),
                 kV1 = ffc(3.6224), kK = ffc(0.43), kUs0 = ffc(0.07), kUs1 = ffc(0.013);
    const ff smu = ff_sqrt(mu), lmu = ff_log(mu);
    const ff b = ff_add(kB0, ff_mul(kB1, smu));
    const ff a = ff_add(kA0, ff_mul(kA1, b));
    const ff inv_alpha = ff_add(kI0, ff_div(kI1, ff_sub(b, kI2)));
    const ff v_r = ff_sub(kV0, ff_div(kV1, ff_add(b, -2.0f)));
    const ff two_a = {2.0f * a.hi, 2.0f * a.lo};
    const ff mu_k = ff_add(mu, kK);
    for (int trial = 0; trial < 64; ++trial) {
        const float U = s.nextf() - 0.5f;
        const float V = s.nextf();
        const float us = 0.5f - fabsf(U);
        if (!(us > 0.0f)) continue;
        const int64_t k = ff_floor_i64(ff_add(ff_mul(ff_add(ff_div(two_a, ffv(us)), b), U), mu_k));
        if (k < 0) continue;
        if (!ff_lt(ffv(us), kUs0) && ff_le(ffv(V), v_r)) return k;
        if (ff_lt(ffv(us), kUs1) && V > us) continue;
        const ff us2 = two_prod(us, us);
        const ff lhs = ff_log(ff_div(ff_mul(ff_mul(inv_alpha, V), us2), ff_add(ff_mul(b, us2), a)));
        const ff rhs = ff_sub(ff_sub(ff_mul(lmu, ff_from_i64(k)), mu), ff_log_factorial(k));
        if (ff_le(lhs, rhs)) return k;
    }
    return ff_floor_i64(ff_add(mu, 0.5f));
}

// The same sampler with the PTRS trials spread over a group of kYieldLanes
// lanes (one track): in round r, lane `sub` takes trial r kYieldLanes + sub,
// whose uniforms are words 2t and 2t + 1 of the track's stream (block t / 2,
// words x, y for even t and z, w for odd t), and the earliest accepting
// trial of the first round with one wins: the sequential sampler's result,
// with the same uniforms and tests. The group's lanes run the setup and the
// inversion below mean 10 redundantly. grp: the group's lanes in the warp.
__device__ int64_t poisson_draw_group(ff mu, const TrackStream &s0, int sub, unsigned grp) {
    if (!(mu.hi > 0.0f)) return 0;
    if (ff_lt(mu, ffv(10.0f))) {
        TrackStream s = s0;
        return poisson_draw(mu, s);
    }
    constexpr ff kB0 = ffc(0.931), kB1 = ffc(2.53), kA0 = ffc(-0.059), kA1 = ffc(0.02483),
                 kI0 = ffc(1.1239), kI1 = ffc(1.1328), kI2 = ffc(3.4), kV0 = ffc(0.9277),
                 kV1 = ffc(3.6224), kK = ffc(0.43), kUs0 = ffc(0.07), kUs1 = ffc(0.013);
    const ff smu = ff_sqrt(mu), lmu = ff_log(mu);
    const ff b = ff_add(kB0, ff_mul(kB1, smu));
    const ff a = ff_add(kA0, ff_mul(kA1, b));
    const ff inv_alpha = ff_add(kI0, ff_div(kI1, ff_sub(b, kI2)));
    const ff v_r = ff_sub(kV0, ff_div(kV1, ff_add(b, -2.0f)));
    const ff two_a = {2.0f * a.hi, 2.0f * a.lo};
    const ff mu_k = ff_add(mu, kK);
    for (int round = 0; round < 64 / kYieldLanes; ++round) {
        const int trial = round * kYieldLanes + sub;
        const u4 w = philox10((uint32_t)(trial >> 1), 0xFFFFFFFFu, s0.id, s0.event, s0.k0, s0.k1);
        const float U = u24f((trial & 1) ? w.z : w.x) - 0.5f;
        const float V = u24f((trial & 1) ? w.w : w.y);
        const float us = 0.5f - fabsf(U);
        bool accept = false;
        int64_t k = -1;
        if (us > 0.0f) {
            k = ff_floor_i64(ff_add(ff_mul(ff_add(ff_div(two_a, ffv(us)), b), U), mu_k));
            if (k >= 0) {
                if (!ff_lt(ffv(us), kUs0) && ff_le(ffv(V), v_r)) {
                    accept = true;
                } else if (!(ff_lt(ffv(us), kUs1) && V > us)) {
                    const ff us2 = two_prod(us, us);
                    const ff lhs = ff_log(
                        ff_div(ff_mul(ff_mul(inv_alpha, V), us2), ff_add(ff_mul(b, us2), a)));
                    const ff rhs =
                        ff_sub(ff_sub(ff_mul(lmu, ff_from_i64(k)), mu), ff_log_factorial(k));
                    accept = ff_le(lhs, rhs);
                }
            }
        }
        const unsigned acc = __ballot_sync(grp, accept) & grp;
        if (acc) return __shfl_sync(grp, (long long)k, __ffs(acc) - 1);
    }
    return ff_floor_i64(ff_add(mu, 0.5f));
}

// ------------------------------------------------- dispersive radiator
// sin^2 theta of the single-resonance radiator at lambda in FP32, one IEEE
// operation at a time (it decides the wavelength accept/reject):
// n - 1 = a / ((1/l0 - 1/l)(1/l0 + 1/l)), n beta - 1 = (n - 1) - (1 - beta)
// - (n - 1)(1 - beta), sin^2 = (n beta - 1)(n beta + 1) / (n beta)^2.
__device__ __forceinline__ float disp_s2_f32(float a, float il0, float omb, float lam) {
    const float il = __fdiv_rn(1.0f, lam);
    const float den = __fmul_rn(__fsub_rn(il0, il), __fadd_rn(il0, il));
    const float n1 = __fdiv_rn(a, den);
    const float nb1 = __fsub_rn(__fsub_rn(n1, omb), __fmul_rn(n1, omb));
    if (!(nb1 > 0.0f)) return 0.0f;
    const float num = __fmul_rn(nb1, __fadd_rn(2.0f, nb1));
    const float op = __fadd_rn(1.0f, nb1);
    return __fdiv_rn(num, __fmul_rn(op, op));
}

__device__ __forceinline__ double atanh64(double z) {
    return 0.5 * log64(__ddiv_rn(1.0 + z, 1.0 - z));
}

// Frank-Tamm photons per mm of the dispersive radiator (FP64): with
// x = 1/lambda, c = 1/l0^2 and q = c + a, 1/n^2 = (1 - a/(q - x^2))^2, so
// sin^2 theta integrates in closed form over the emitting part
// [max(1/lambda_max, x_t), 1/lambda_min] of the band, x_t^2 = c - a beta /
// (1 - beta) being where n beta = 1. Returns x_t (0: no threshold) too.
__device__ double disp_yield_per_mm(const YieldModel &m, double beta, double omb,
                                   double lam_min, double lam_max, double &xt) {
    const double il0 = 1.0 / (double)m.disp_lambda0, a = (double)m.disp_a;
    xt = 0.0;
    if (omb > 0.0) {
        const double u = il0 * il0 - a * beta / omb;
        if (u > 0.0) xt = sqrt(u);
    }
    double xa = 1.0 / lam_max;
    const double xb = 1.0 / lam_min;
    if (xt > xa) xa = xt;
    if (!(xb > xa)) return 0.0;
    const double q = il0 * il0 + a, sq = sqrt(q), b2 = beta * beta;
    const double c0 = -omb * (2.0 - omb) / b2;              // 1 - 1/beta^2
    const double F1b = atanh64(xb / sq) / sq, F1a = atanh64(xa / sq) / sq;
    const double F2b = xb / (2.0 * q * (q - xb * xb)) + atanh64(xb / sq) / (2.0 * q * sq);
    const double F2a = xa / (2.0 * q * (q - xa * xa)) + atanh64(xa / sq) / (2.0 * q * sq);
    const double I = c0 * (xb - xa) + (2.0 * a / b2) * (F1b - F1a) - (a * a / b2) * (F2b - F2a);
    return 2.0 * kPi * kAlpha * I * 1.0e6;
}

__device__ __forceinline__ void basis_ff(const ff3 &t, ff3 &e1, ff3 &e2);

template <bool RECS>
__global__ void __launch_bounds__(kYieldBlock)
k_yield(TracksView t, ff nm1, ff inv_band, uint32_t key0,
        uint32_t key1, TrackRec *rec, float4 *cs, uint32_t *counts,
        unsigned long long *block_sums, YieldModel model, double lam_min, double lam_max,
        TrackFrame *frame, uint32_t *perm_ok) {
    grid_dep_launch_dependents();        // the ordering pass may be scheduled
    // the ordering pass of this emission ORs its flags into a zeroed word
    if (perm_ok && blockIdx.x == 0 && threadIdx.x == 0) *perm_ok = 0u;
    // kYieldLanes consecutive lanes per track; lane 0 of each group writes
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i = gt / kYieldLanes;
    const int sub = (int)(gt % kYieldLanes);
    const unsigned grp = ((1u << kYieldLanes) - 1u) << ((threadIdx.x & 31) & ~(kYieldLanes - 1));
    uint32_t count = 0;
    if (i < t.n) {
        // every input of the track in one round of loads
        const float p = t.p[i], m = t.mass[i], len = t.length[i];
        const float tx = t.x[i], ty = t.y[i], tz = t.z[i];
        const float fdx = t.dx[i], fdy = t.dy[i], fdz = t.dz[i];
        const uint32_t event = t.event[i];
        const uint32_t id = t.id ? t.id[i] : (uint32_t)i;
        const uint32_t n_fixed = t.n_fixed ? t.n_fixed[i] : 0u;
        const ff pf = ffv(p), mf = ffv(m), lf = ffv(len);     // FP32 inputs, exact
        // 1 - beta = m^2 / (E (E + p)) keeps n*beta - 1 accurate near 1
        const ff E = ff_sqrt(ff_add(ff_mul(pf, pf), ff_mul(mf, mf)));
        const ff omb = mf.hi == 0.0f ? ffv(0.0f) : ff_div(ff_mul(mf, mf), ff_mul(E, ff_add(E, pf)));
        const ff beta = ff_add(ff_neg(omb), 1.0f);
        const ff nbm1 = ff_sub(ff_mul(nm1, beta), omb);
        ff cos_t = ffv(1.0f), sin_t = ffv(0.0f), mu = ffv(0.0f);
        float tan_f = 0.0f, disp_span = 0.0f, disp_s2max = 0.0f;
        float4 cs_out;
        if (model.iso_yield >= 0.0) {
            // isotropic source: mean photons = yield per mm x length
            mu = ff_mul(lf, ff_from_double(model.iso_yield));
        } else if (model.dispersion) {
            // dispersive radiator (FP64): Frank-Tamm integral of sin^2 theta(lambda),
            // and the FP32 band and normaliser of the wavelength accept/reject
            const double p64 = p, m64 = m;
            const double E64 = sqrt(p64 * p64 + m64 * m64);
            const double omb64 = (m64 == 0.0) ? 0.0 : (m64 * m64) / (E64 * (E64 + p64));
            double xt = 0.0;
            mu = ff_from_double((double)len * disp_yield_per_mm(model, 1.0 - omb64, omb64,
                                                                 lam_min, lam_max, xt));
            const float inv1 = __fdiv_rn(1.0f, (float)lam_min);
            const float inv2 = __fdiv_rn(1.0f, (float)lam_max);
            const float xlo = (float)xt > inv2 ? (float)xt : inv2;
            disp_span = __fsub_rn(inv1, xlo);
            tan_f = (float)omb64;                            // stored as 1 - beta
            disp_s2max = disp_s2_f32(model.disp_a, __fdiv_rn(1.0f, model.disp_lambda0),
                                     (float)omb64, (float)lam_min);
            const ff b_ff = ff_from_double(1.0 - omb64), o_ff = ff_from_double(omb64);
            cs_out = make_float4(b_ff.hi, b_ff.lo, o_ff.hi, o_ff.lo);   // (beta, 1 - beta)
        } else if (nbm1.hi > 0.0f) {
            const ff nb = ff_add(nbm1, 1.0f);
            const ff tan_t = ff_sqrt(ff_mul(nbm1, ff_add(nb, 1.0f)));   // (n beta)^2 - 1
            cos_t = ff_div(ffv(1.0f), nb);
            sin_t = ff_mul(tan_t, cos_t);
            tan_f = tan_t.hi;
            mu = ff_mul(ff_mul(lf, ff_mul(sin_t, sin_t)), ff_mul(k2PiAlpha, inv_band));
        }
        if (!model.dispersion) cs_out = make_float4(cos_t.hi, cos_t.lo, sin_t.hi, sin_t.lo);
        if (t.n_fixed) {
            count = n_fixed;
        } else {
            const TrackStream s{event, id, key0, key1, 0u, 4u, {0u, 0u, 0u, 0u}};
            const int64_t k = poisson_draw_group(mu, s, sub, grp);
            count = (uint32_t)(k > 0xFFFFFFF0ll ? 0xFFFFFFF0ll : k);
        }
        if (RECS && sub == 0) {
        // the unit direction, rounded to FP32 from its double-word, and the
        // double-word frame of the refinement's emission
        const ff3 tn = ff3_normalized(ff3v(fdx, fdy, fdz));
        ff3 e1, e2;
        basis_ff(tn, e1, e2);
        frame[i] = TrackFrame{{tn.x.hi, tn.x.lo, tn.y.hi, tn.y.lo, tn.z.hi, tn.z.lo},
                              {e1.x.hi, e1.x.lo, e1.y.hi, e1.y.lo, e1.z.hi, e1.z.lo},
                              {e2.x.hi, e2.x.lo, e2.y.hi, e2.y.lo, e2.z.hi, e2.z.lo},
                              {0.0f, 0.0f}};
        TrackRec r;
        r.x = tx;
        r.y = ty;
        r.z = tz;
        r.len = len;
        r.tx = tn.x.hi;
        r.ty = tn.y.hi;
        r.tz = tn.z.hi;
        r.tan_theta = tan_f;
        r.rx = fdx;
        r.ry = fdy;
        r.rz = fdz;
        r.event = event;
        r.id = id;
        r.count = count;
        r.disp_span = disp_span;
        r.disp_s2max = disp_s2max;
        rec[i] = r;
        cs[i] = cs_out;
        }
        if (sub == 0) counts[i] = count;
    }
    if (sub != 0) count = 0;            // one contribution per track to the sums
    // sum of the counts of this block, added to its 256-track scan group
    // (integer atomics: exact and order independent)
    unsigned long long v = count;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    __shared__ unsigned long long warp_sum[kYieldBlock / 32];
    if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long s = 0;
        for (int w = 0; w < kYieldBlock / 32; ++w) s += warp_sum[w];
        const int64_t first = (int64_t)blockIdx.x * (kYieldBlock / kYieldLanes);  // first track
        if (s) atomicAdd(&block_sums[first / kYieldThreads], s);
    }
}

__global__ void __launch_bounds__(kYieldThreads)
k_offsets(const uint32_t *counts, const unsigned long long *block_sums,
          int64_t n, uint64_t *offsets, unsigned long long *total) {
    __shared__ unsigned long long red[kYieldThreads / 32];
    __shared__ unsigned long long base;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // prefix of the earlier blocks
    unsigned long long acc = 0;
    for (unsigned b = threadIdx.x; b < blockIdx.x; b += blockDim.x) acc += block_sums[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(kFull, acc, o);
    if (lane == 0) red[wid] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long s = 0;
        for (int w = 0; w < kYieldThreads / 32; ++w) s += red[w];
        base = s;
    }
    __syncthreads();
    // in-block exclusive scan
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long c = i < n ? counts[i] : 0ull;
    unsigned long long inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += y;
    }
    __shared__ unsigned long long wsum[kYieldThreads / 32];
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    unsigned long long wpre = 0;
    for (int w = 0; w < wid; ++w) wpre += wsum[w];
    unsigned long long excl = base + wpre + inc - c;
    if (i < n) offsets[i] = excl;
    if (i == n - 1) {
        offsets[n] = excl + c;
        if (total) *total = excl + c;
    }
}

// ============================================================ ordering
// Photons of a track sorted by azimuth bin (the top 5 bits of the azimuth
// draw): photons that leave the track in nearby directions hit nearby
// points of the mirror and, being nearly parallel there, are focused to
// nearby points after it, so a warp that takes consecutive entries traces
// coherent rays at every bounce. Processing order only: every photon keeps
// its own draws and results. One block of kOrderWarps warps per track
// (grid-stride), counting sort in shared memory (the bins of the first
// kOrderBinCache photons kept from the counting pass), order within a bin
// arbitrary.
constexpr int kAzBins = 32;
constexpr int kOrderWarps = 4;
// bins of the first 8192 photons kept (8 KiB): tracks of up to 8192 photons
// draw each azimuth once (5000-photon tracks: 16.9 -> 15.4 us per 200 tracks;
// 8 warps per block were slower on 10^4 tracks)
constexpr uint32_t kOrderBinCache = 8192;

// SCAN: the offsets are not computed yet; each block first forms the
// exclusive prefix of the 256-track group sums in shared memory, and each
// track's warp adds the counts before it in its group and writes its
// offset (block 0 writes offsets[n] and the total).
template <bool SCAN>
__global__ void __launch_bounds__(32 * kOrderWarps) k_order(EmitView em, uint2 *perm,
                                                            uint64_t cap, uint32_t *perm_ok,
                                                            OrderScan scan, bool signal_early) {
    grid_dep_wait();                     // the yield (and scan) pass has ended
    // the trace's prologue may start, when every block orders one track;
    // over many tracks per block the trace's blocks, resident early, slowed
    // the ordering pass (RICH2, 4.9e5 tracks: 45 -> 50 ms per chunk)
    if (signal_early) grid_dep_launch_dependents();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    extern __shared__ unsigned long long s_gpre[];      // SCAN: one entry per group
    __shared__ unsigned long long s_wsum[kOrderWarps];
    __shared__ unsigned long long s_total;
    uint64_t total;
    if (SCAN) {
        // a contiguous segment of groups per thread, then a block scan of
        // the segment sums
        const int ng = (int)((em.n_tracks + kYieldThreads - 1) / kYieldThreads);
        const int per = (ng + (int)blockDim.x - 1) / (int)blockDim.x;
        const int a = min((int)threadIdx.x * per, ng), b = min(a + per, ng);
        unsigned long long seg = 0;
        for (int g = a; g < b; ++g) seg += scan.group_sums[g];
        unsigned long long inc = seg;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(kFull, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) s_wsum[w] = inc;
        __syncthreads();
        unsigned long long run = inc - seg;
        for (int k = 0; k < w; ++k) run += s_wsum[k];
        for (int g = a; g < b; ++g) {
            s_gpre[g] = run;
            run += scan.group_sums[g];
        }
        if (threadIdx.x == blockDim.x - 1) s_total = run;
        __syncthreads();
        total = s_total;
    } else {
        total = *em.total;
    }
    const bool fits = total <= cap;
    // perm_ok (zeroed by the yield pass): bit 0 the entries fit the buffer,
    // bit 1 a track above kOrderMaxPhotons kept index order (its entries are
    // not written)
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (fits) atomicOr(perm_ok, 1u);
        if (SCAN) {
            *scan.total = total;
            scan.offsets[em.n_tracks] = total;
        }
    }
    if (!SCAN && !fits) return;
    // one block per track (grid-stride): the block's warps share the bin
    // histogram, so each lane draws and places only a few photons
    __shared__ uint32_t hist[kAzBins];
    __shared__ uint8_t bins[kOrderBinCache];
    __shared__ unsigned long long s_part[kOrderWarps];
    const int nthreads = (int)blockDim.x;
    for (int64_t t = blockIdx.x; t < em.n_tracks; t += gridDim.x) {   // block-uniform
        uint64_t off, n64;
        if (SCAN) {
            const int64_t g = t / kYieldThreads;
            unsigned long long part = 0;
            for (int64_t i = g * kYieldThreads + threadIdx.x; i < t; i += nthreads)
                part += scan.counts[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(kFull, part, o);
            if (lane == 0) s_part[w] = part;
            __syncthreads();
            off = s_gpre[g];
            for (int k = 0; k < kOrderWarps; ++k) off += s_part[k];
            n64 = scan.counts[t];
            if (threadIdx.x == 0) scan.offsets[t] = off;
        } else {
            off = em.offsets[t];
            n64 = em.offsets[t + 1] - off;
        }
        if (fits && n64 > kOrderMaxPhotons && threadIdx.x == 0) atomicOr(perm_ok, 2u);
        if (fits && n64 != 0 && n64 <= kOrderMaxPhotons) {   // uniform in the block
            const uint32_t n = (uint32_t)n64;
            const uint32_t id = em.tracks[t].id, ev = em.tracks[t].event;
            if (threadIdx.x < kAzBins) hist[threadIdx.x] = 0u;
            __syncthreads();
            for (uint32_t j = threadIdx.x; j < n; j += (uint32_t)nthreads) {
                const uint32_t bin = philox10(0u, j, id, ev, em.key0, em.key1).y >> 27;
                if (j < kOrderBinCache) bins[j] = (uint8_t)bin;
                atomicAdd(&hist[bin], 1u);
            }
            __syncthreads();
            if (w == 0) {
                const uint32_t c = hist[lane];
                uint32_t inc = c;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(kFull, inc, o);
                    if (lane >= o) inc += y;
                }
                hist[lane] = inc - c;                           // bin cursors
            }
            __syncthreads();
            for (uint32_t j = threadIdx.x; j < n; j += (uint32_t)nthreads) {
                const uint32_t bin = j < kOrderBinCache
                                         ? (uint32_t)bins[j]
                                         : philox10(0u, j, id, ev, em.key0, em.key1).y >> 27;
                perm[off + atomicAdd(&hist[bin], 1u)] = make_uint2(j, (uint32_t)t);
            }
        }
        __syncthreads();                 // the shared histogram and bins are reused
    }
}

cudaError_t launch_order(const EmitView &em, uint2 *perm, uint64_t cap, uint32_t *perm_ok,
                         int n_sm, cudaStream_t s, const OrderScan *scan) {
    int64_t blocks = em.n_tracks;                       // one block per track
    if (blocks < 1) blocks = 1;
    const int64_t max_blocks = (int64_t)n_sm * 16;
    if (blocks > max_blocks) blocks = max_blocks;
    const bool early = em.n_tracks <= blocks;
    if (scan) {
        const int64_t groups = (em.n_tracks + kYieldThreads - 1) / kYieldThreads;
        if (groups > kOrderScanGroups) return cudaErrorInvalidValue;
        return launch_pdl(k_order<true>, (unsigned)blocks, 32 * kOrderWarps,
                          sizeof(unsigned long long) * (size_t)groups, s, em, perm, cap, perm_ok,
                          *scan, early);
    }
    return launch_pdl(k_order<false>, (unsigned)blocks, 32 * kOrderWarps, 0, s, em, perm, cap,
                      perm_ok, OrderScan{}, early);
}

// ============================================================== emission
struct Photon {
    f3 o, d;
    float lam;
    uint32_t event, id, j;
    uint32_t track;        // track index (fused) or external photon index
    uint64_t g;            // global photon index
    uint32_t w_qe;
    uint32_t wr0, wr1, wr2, wr3;
    int skip, n_refl, steps;
    int n_turn;            // direction changes: reflections and refractions
    int skip_ref;          // BVH subtree of the surface just left, or kNoSurf
};

// Wavelength from a binned emission spectrum (CDF table): the bin k with
// c_k <= u < c_{k+1}, linear inside it, each operation rounded in FP32.
__device__ __forceinline__ float spectrum_lambda(const DevTable &T, float u) {
    int k = 0;
    while (k + 1 < T.nbins && T.values[k + 1] <= u) ++k;
    const float fr = __fdiv_rn(__fsub_rn(u, T.values[k]), __fsub_rn(T.values[k + 1], T.values[k]));
    return __fadd_rn(T.p0, __fmul_rn(__fadd_rn((float)k, fr), T.p1));
}

// Wavelength of a dispersive-radiator photon: candidates from the 1/lambda^2
// law on the track's emitting band kept with probability
// sin^2 theta(lambda) / sin^2 theta(lambda_min); trial 0 takes block 0 word
// 2 and block 3 word 3, trial t >= 1 block 8 + (t-1)/2; the last of 64
// candidates stands.
__device__ float disp_lambda(const TrackRec &tr, uint32_t j, const EmitView &em, uint32_t wl0,
                             uint32_t wa0) {
    const float il0 = __fdiv_rn(1.0f, em.disp_lambda0);
    const float omb = tr.tan_theta;
    float lam = 0.0f;
    for (int t = 0; t < 64; ++t) {
        uint32_t wl = wl0, wa = wa0;
        if (t > 0) {
            const u4 w = philox10(8u + (uint32_t)(t - 1) / 2u, j, tr.id, tr.event, em.key0,
                                  em.key1);
            const bool hi = ((t - 1) & 1) != 0;
            wl = hi ? w.z : w.x;
            wa = hi ? w.w : w.y;
        }
        lam = __fdiv_rn(1.0f, __fsub_rn(em.inv1, __fmul_rn(u24f(wl), tr.disp_span)));
        if (!(tr.disp_s2max > 0.0f)) break;
        const float pa = __fdiv_rn(disp_s2_f32(em.disp_a, il0, omb, lam), tr.disp_s2max);
        if (u24f(wa) < pa) break;
    }
    return lam;
}

// Wavelength of a fused-emission photon from its draws: the source's binned
// spectrum, the dispersive radiator's law, or the Frank-Tamm 1/lambda^2 law
// on the emission band.
__device__ __forceinline__ float photon_wavelength(const TrackRec &tr, uint32_t j,
                                                   const EmitView &em, const u4 &w0,
                                                   const DevTable *spec) {
    if (spec) return spectrum_lambda(*spec, u24f(w0.z));
    if (em.dispersion) {
        const u4 w3 = philox10(3u, j, tr.id, tr.event, em.key0, em.key1);
        return disp_lambda(tr, j, em, w0.z, w3.w);
    }
    return emit_lambda(u24f(w0.z), em.inv1, em.span);
}

// FP32 tan(theta) of the dispersive radiator at lambda: sqrt((n beta)^2 - 1)
// with n beta - 1 formed without cancellation.
__device__ __forceinline__ float disp_tan_f32(const EmitView &em, float omb, float lam) {
    const float il0 = __fdiv_rn(1.0f, em.disp_lambda0);
    const float il = __fdiv_rn(1.0f, lam);
    const float n1 = em.disp_a / ((il0 - il) * (il0 + il));
    const float nb1 = (n1 - omb) - n1 * omb;
    return sqrtf(fmaxf(0.0f, nb1 * (2.0f + nb1)));
}

// Fused emission of photon j of track tr (Sec. 3 angle, Sec. 4.2 photons as
// independent rays): origin uniform on the segment, azimuth uniform,
// wavelength `lam` from photon_wavelength. The direction is built as
// t + tan(theta) (cos phi e1 + sin phi e2), normalised, so the small
// Cherenkov angle is carried by tan(theta) and not by a cosine near 1;
// a dispersive radiator takes tan(theta) of the photon's own wavelength.
// Isotropic source (the scintillation light named in Sec. 6): the
// direction is uniform on the sphere, cos(theta) = 1 - 2u from draw block 3.
__device__ __forceinline__ void emit_photon(const TrackRec &tr, uint32_t j,
                                            const EmitView &em, const u4 &w0, float lam,
                                            Photon &ph) {
    u4 w1 = philox10(1u, j, tr.id, tr.event, em.key0, em.key1);
    f3 t = mk3(tr.tx, tr.ty, tr.tz);
    float s = u24f(w0.x) * tr.len;
    ph.o = fma3(t, s, mk3(tr.x, tr.y, tr.z));
    float sp, cp;
    sincospif(2.0f * u24f(w0.y), &sp, &cp);
    if (em.source == RICH_SOURCE_ISOTROPIC) {
        const u4 w3 = philox10(3u, j, tr.id, tr.event, em.key0, em.key1);
        const float ct = 1.0f - 2.0f * u24f(w3.z);      // exact
        const float st = sqrtf(fmaxf(0.0f, (1.0f - ct) * (1.0f + ct)));
        ph.d = normalize3(mk3(st * cp, st * sp, ct));
    } else {
        f3 e1, e2;
        basis_f(t, e1, e2);
        f3 r = fma3(e1, cp, e2 * sp);
        const float tan_t = em.dispersion ? disp_tan_f32(em, tr.tan_theta, lam) : tr.tan_theta;
        ph.d = normalize3(fma3(r, tan_t, t));
    }
    ph.lam = lam;
    ph.w_qe = w0.w;
    ph.wr0 = w1.x;
    ph.wr1 = w1.y;
    ph.wr2 = w1.z;
    ph.wr3 = w1.w;
    ph.event = tr.event;
    ph.id = tr.id;
    ph.j = j;
}

__global__ void k_materialize(SceneView sc, EmitView em, uint64_t n, rich_photons out) {
    const DevTable *spec = em.spectrum >= 0 ? sc.tables + em.spectrum : nullptr;
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n;
         g += (uint64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = em.n_tracks - 1;
        while (lo < hi) {
            int64_t mid = (lo + hi + 1) >> 1;
            if (em.offsets[mid] <= g) lo = mid; else hi = mid - 1;
        }
        TrackRec tr = em.tracks[lo];
        Photon ph;
        const uint32_t j = (uint32_t)(g - em.offsets[lo]);
        const u4 w0 = philox10(0u, j, tr.id, tr.event, em.key0, em.key1);
        emit_photon(tr, j, em, w0, photon_wavelength(tr, j, em, w0, spec), ph);
        out.x[g] = ph.o.x;
        out.y[g] = ph.o.y;
        out.z[g] = ph.o.z;
        out.dx[g] = ph.d.x;
        out.dy[g] = ph.d.y;
        out.dz[g] = ph.d.z;
        out.lambda[g] = ph.lam;
        out.event[g] = ph.event;
        out.track[g] = ph.id;
        out.photon[g] = ph.j;
    }
}

// ============================================================ intersection
struct Best {
    float t;
    int prim;     // global primitive id
    int kind;     // 0 tile, 1 rect, 2 triangle
    int idx;      // index into tiles / rects / tris
    float b0, b1, b2;
};

// The small scene tables staged in the trace kernel's dynamic shared memory,
// each addressed by a 32-bit byte offset (a generic 64-bit pointer would
// hold two registers through the bounce loop).
extern __shared__ __align__(128) unsigned char rich_dsmem[];
struct SmemScene {
    uint32_t o_groups, o_tiles, o_rects, o_tables, o_materials;
    int n_groups, n_tiles, n_rects;
    __device__ __forceinline__ const DevSphereGroup *groups() const {
        return reinterpret_cast<const DevSphereGroup *>(rich_dsmem + o_groups);
    }
    __device__ __forceinline__ const DevTile *tiles() const {
        return reinterpret_cast<const DevTile *>(rich_dsmem + o_tiles);
    }
    __device__ __forceinline__ const DevRect *rects() const {
        return reinterpret_cast<const DevRect *>(rich_dsmem + o_rects);
    }
    __device__ __forceinline__ const DevTable *tables() const {
        return reinterpret_cast<const DevTable *>(rich_dsmem + o_tables);
    }
    __device__ __forceinline__ const DevMaterial *materials() const {
        return reinterpret_cast<const DevMaterial *>(rich_dsmem + o_materials);
    }
};

// Tiles: per distinct sphere, the quadratic |w + t d|^2 = R^2 with w = o - C
// in double-word arithmetic (rich_ff.cuh, ~48 bits; precision policy: the
// large-radius discriminant is the one place the trace needs more than
// FP32, and double-words give it at FP32 issue rates), roots by the
// cancellation-free pair (q, c/q); the aperture of each tile is then tested
// in FP32 at the point relative to the centre. The nearer root on any tile
// hides the farther one. Out of line, as sphere_normal: inlined, their
// double-word registers enter the bounce loop's allocation under the
// 64-register cap and slow mesh-only traces by a few per cent.
__device__ __noinline__ void nearest_tiles(const SmemScene &S, f3 o, f3 d,
                                           int skip, float t_min, Best &b) {
    for (int gi = 0; gi < S.n_groups; ++gi) {
        const DevSphereGroup &G = S.groups()[gi];
        // w = o - C exactly (FP32 inputs)
        const ff wx = two_sum(o.x, -G.fcx), wy = two_sum(o.y, -G.fcy),
                 wz = two_sum(o.z, -G.fcz);
        const ff bq = ff_add(ff_add(ff_mul(wx, d.x), ff_mul(wy, d.y)), ff_mul(wz, d.z));
        const ff c = ff_sub(ff_add(ff_add(ff_mul(wx, wx), ff_mul(wy, wy)), ff_mul(wz, wz)),
                            two_prod(G.radius, G.radius));
        const ff disc = ff_sub(ff_mul(bq, bq), c);
        if (disc.hi < 0.0f) continue;
        const ff sq = ff_sqrt(disc);
        const ff q = bq.hi > 0.0f ? ff_neg(ff_add(bq, sq)) : ff_sub(sq, bq);
        const ff r2 = q.hi != 0.0f ? ff_div(c, q) : ffv(0.0f);
        const bool q_first = ff_lt(q, r2);
        const ff t_lo = q_first ? q : r2, t_hi = q_first ? r2 : q;
#pragma unroll
        for (int ri = 0; ri < 2; ++ri) {
            const ff tr = ri == 0 ? t_lo : t_hi;
            // tr > t_min and tr < b.t for the double-word value
            if (!ff_lt(ffv(t_min), tr) || !ff_lt(tr, ffv(b.t))) continue;
            const f3 pc = mk3(ff_add(wx, ff_mul(tr, d.x)).hi, ff_add(wy, ff_mul(tr, d.y)).hi,
                              ff_add(wz, ff_mul(tr, d.z)).hi);
            bool hit = false;
            for (int k = G.first; k < G.first + G.count; ++k) {
                const DevTile &T = S.tiles()[k];
                if (T.prim == skip) continue;
                const float ca = (pc.x * T.ax + pc.y * T.ay + pc.z * T.az) * T.inv_radius;
                if (!(ca >= T.cos_min)) continue;
                const float x = pc.x * T.e1x + pc.y * T.e1y + pc.z * T.e1z;
                const float y = pc.x * T.e2x + pc.y * T.e2y + pc.z * T.e2z;
                bool in = true;
                for (int e = 0; e < T.n_edges; ++e)
                    in = in && (T.edges[e][0] * x + T.edges[e][1] * y <= T.edges[e][2]);
                if (!in) continue;
                b.t = tr.hi;
                b.prim = T.prim;
                b.kind = 0;
                b.idx = k;
                hit = true;
                break;
            }
            if (hit) break;
        }
    }
}

// Inward unit normal (towards the centre) at o + t d on the group's sphere,
// from the double-word point relative to the centre.
__device__ __noinline__ f3 sphere_normal(const DevSphereGroup &G, f3 o, f3 d, float t) {
    const ff3 p = {ff_add(two_sum(o.x, -G.fcx), two_prod(t, d.x)),
                   ff_add(two_sum(o.y, -G.fcy), two_prod(t, d.y)),
                   ff_add(two_sum(o.z, -G.fcz), two_prod(t, d.z))};
    const ff inv = ff_neg(ff_rsqrt(ff3_dot(p, p)));
    return mk3(ff_mul(p.x, inv).hi, ff_mul(p.y, inv).hi, ff_mul(p.z, inv).hi);
}

__device__ __forceinline__ void nearest_rects(const SmemScene &S, f3 o, f3 d,
                                              int skip, float t_min, Best &b) {
    for (int k = 0; k < S.n_rects; ++k) {
        const DevRect &R = S.rects()[k];
        if (R.prim == skip) continue;
        const f3 n = mk3(R.nx, R.ny, R.nz);
        const float den = dot3(d, n);
        if (den == 0.0f) continue;
        const f3 oo = mk3(R.ox, R.oy, R.oz) - o;
        const float t = __fdiv_rn(dot3(oo, n), den);
        if (!(t > t_min) || !(t < b.t)) continue;
        const f3 q = fma3(d, t, mk3(-oo.x, -oo.y, -oo.z));
        const float u = dot3(q, mk3(R.ux, R.uy, R.uz));
        const float v = dot3(q, mk3(R.vx, R.vy, R.vz));
        if (!(u >= 0.0f && u < R.w && v >= 0.0f && v < R.h)) continue;
        b.t = t;
        b.prim = R.prim;
        b.kind = 1;
        b.idx = k;
    }
}

// Watertight ray/triangle test (Woop, Benthin, Wald, JCGT 2(1) 2013):
// translate to the ray origin, shear so the ray is +z, evaluate the three
// 2-D edge functions (products kept unfused so shared edges get exactly
// opposite values; exact FP64 re-evaluation when one is zero), accept both
// windings, distance from the sheared z.
struct Ray {
    f3 o, d, inv;
    float sx, sy, sz;
    int k;              // axes of the watertight test: kx | ky << 2 | kz << 4
    __device__ __forceinline__ int kx() const { return k & 3; }
    __device__ __forceinline__ int ky() const { return (k >> 2) & 3; }
    __device__ __forceinline__ int kz() const { return k >> 4; }
};

__device__ __forceinline__ float pick(float x, float y, float z, int k) {
    return k == 0 ? x : (k == 1 ? y : z);
}

__device__ __forceinline__ Ray make_ray(f3 o, f3 d) {
    Ray r;
    r.o = o;
    r.d = d;
    const float eps = 1e-30f;
    r.inv = mk3(1.0f / (fabsf(d.x) > eps ? d.x : copysignf(eps, d.x)),
                1.0f / (fabsf(d.y) > eps ? d.y : copysignf(eps, d.y)),
                1.0f / (fabsf(d.z) > eps ? d.z : copysignf(eps, d.z)));
    const float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
    int kz = (ax > ay) ? (ax > az ? 0 : 2) : (ay > az ? 1 : 2);
    int kx = kz == 2 ? 0 : kz + 1;
    int ky = kx == 2 ? 0 : kx + 1;
    const float dz = pick(d.x, d.y, d.z, kz);
    if (dz < 0.0f) {
        int tmp = kx;
        kx = ky;
        ky = tmp;
    }
    r.k = kx | ky << 2 | kz << 4;
    r.sx = pick(d.x, d.y, d.z, kx) / dz;
    r.sy = pick(d.x, d.y, d.z, ky) / dz;
    r.sz = 1.0f / dz;
    return r;
}

__device__ __forceinline__ bool watertight(const Ray &r, const DevTri &T,
                                           float t_min, float t_max, float &t,
                                           float &b0, float &b1, float &b2) {
    const float Ax0 = T.v0x - r.o.x, Ay0 = T.v0y - r.o.y, Az0 = T.v0z - r.o.z;
    const float Bx0 = T.v1x - r.o.x, By0 = T.v1y - r.o.y, Bz0 = T.v1z - r.o.z;
    const float Cx0 = T.v2x - r.o.x, Cy0 = T.v2y - r.o.y, Cz0 = T.v2z - r.o.z;
    const int kx = r.kx(), ky = r.ky(), kz = r.kz();
    const float Akz = pick(Ax0, Ay0, Az0, kz), Bkz = pick(Bx0, By0, Bz0, kz),
                Ckz = pick(Cx0, Cy0, Cz0, kz);
    const float Ax = fmaf(-r.sx, Akz, pick(Ax0, Ay0, Az0, kx));
    const float Ay = fmaf(-r.sy, Akz, pick(Ax0, Ay0, Az0, ky));
    const float Bx = fmaf(-r.sx, Bkz, pick(Bx0, By0, Bz0, kx));
    const float By = fmaf(-r.sy, Bkz, pick(Bx0, By0, Bz0, ky));
    const float Cx = fmaf(-r.sx, Ckz, pick(Cx0, Cy0, Cz0, kx));
    const float Cy = fmaf(-r.sy, Ckz, pick(Cx0, Cy0, Cz0, ky));
    float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
    float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
    float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
    if (U == 0.0f || V == 0.0f || W == 0.0f) {
        U = (float)((double)Cx * By - (double)Cy * Bx);
        V = (float)((double)Ax * Cy - (double)Ay * Cx);
        W = (float)((double)Bx * Ay - (double)By * Ax);
    }
    if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f))
        return false;
    const float det = U + V + W;
    if (det == 0.0f) return false;
    const float T_ = fmaf(U, r.sz * Akz, fmaf(V, r.sz * Bkz, W * (r.sz * Ckz)));
    const float rcp = 1.0f / det;
    t = T_ * rcp;
    if (!(t > t_min && t <= t_max)) return false;
    b0 = U * rcp;
    b1 = V * rcp;
    b2 = W * rcp;
    return true;
}

__device__ __forceinline__ DevTri load_tri(const DevTri *p) {
    const float4 *q = reinterpret_cast<const float4 *>(p);
    float4 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2);
    DevTri t;
    t.v0x = a.x; t.v0y = a.y; t.v0z = a.z; t.v1x = a.w;
    t.v1y = b.x; t.v1z = b.y; t.v2x = b.z; t.v2y = b.w;
    t.v2z = c.x;
    t.prim = __float_as_int(c.y);
    t.material = __float_as_int(c.z);
    t.pad = __float_as_int(c.w);
    return t;
}

__device__ __forceinline__ bool slab(const Ray &r, float lx, float ly, float lz,
                                     float hx, float hy, float hz, float tmax,
                                     float &tnear) {
    const float ox = r.o.x * r.inv.x, oy = r.o.y * r.inv.y, oz = r.o.z * r.inv.z;
    const float tx0 = fmaf(lx, r.inv.x, -ox), tx1 = fmaf(hx, r.inv.x, -ox);
    const float ty0 = fmaf(ly, r.inv.y, -oy), ty1 = fmaf(hy, r.inv.y, -oy);
    const float tz0 = fmaf(lz, r.inv.z, -oz), tz1 = fmaf(hz, r.inv.z, -oz);
    const float tn = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)),
                           fmaxf(fminf(tz0, tz1), 0.0f));
    const float tf = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)),
                           fminf(fmaxf(tz0, tz1), tmax));
    tnear = tn;
    // 1 + 2^-20 widening keeps boxes conservative under FP32 rounding
    return tn <= tf * 1.00000095f;
}

// Per-thread tallies of the counting build of the trace (COUNT = true): the
// algorithmic events of the traversal, summed into TraceParams::work at the
// end of the kernel. The production build compiles none of it.
struct WorkTally {
    uint32_t steps;          // nearest-surface queries
    uint32_t nodes_smem;     // four-wide node tests on nodes in shared memory
    uint32_t nodes_global;   // ... on nodes read from global memory
    uint32_t tris;           // ray-triangle tests
    uint32_t normals;        // vertex-normal blends at smooth triangle hits
    uint32_t turns;          // reflections and refractions
};

template <bool COUNT>
__device__ __forceinline__ void leaf_tris(const SceneView &sc, const Ray &r,
                                          int code, int skip, float t_min,
                                          Best &b, WorkTally *w) {
    const int first = code >> 3, count = (code & 7) + 1;
    for (int k = first; k < first + count; ++k) {
        const DevTri T = load_tri(sc.tris + k);
        if (T.prim == skip) continue;
        if constexpr (COUNT) w->tris += 1;
        float t, b0, b1, b2;
        if (!watertight(r, T, t_min, b.t, t, b0, b1, b2)) continue;
        if (t == b.t && T.prim > b.prim) continue;
        b.t = t;
        b.prim = T.prim;
        b.kind = 2;
        b.idx = k;
        if (sc.tri_normals) {
            // the shading step reads this triangle's vertex normals next
            const float *nrm = sc.tri_normals + 9 * (int64_t)k;
            asm volatile("prefetch.global.L1 [%0];" ::"l"(nrm));
            asm volatile("prefetch.global.L1 [%0];" ::"l"(nrm + 8));
        }
        b.b0 = b0;
        b.b1 = b1;
        b.b2 = b2;
    }
}

// Three-input FP32 maximum and minimum (one instruction each on sm_100 and
// later; exact, like two fmaxf / fminf).
__device__ __forceinline__ float max3f(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float min3f(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Box tests of the four children of a four-wide node, axis by axis (the
// node holds centre x, half extent x, centre y, ... of the four children as
// six float4, then the children's references), read through one generic
// load path for shared and global memory. Per axis the slab's entry and
// exit distances are tc -+ e with tc = (c - o) / d and e = half extent /
// |d|: FP32 multiply-adds, no min/max to order them; the axes and the
// clamp to [0, tmax] are combined by three-input min/max. Returns each
// child's entry distance, +infinity for a miss, with the widening of `slab`.
__device__ __forceinline__ void node4_test(const Ray &r, const DevNode *p, float tmax,
                                           int skip_ref, float4 &key, int4 &ch) {
    const float4 *q = reinterpret_cast<const float4 *>(p);
    const float ox = r.o.x * r.inv.x, oy = r.o.y * r.inv.y, oz = r.o.z * r.inv.z;
    const float ax = fabsf(r.inv.x), ay = fabsf(r.inv.y), az = fabsf(r.inv.z);
    float4 tn, tf;
    {
        const float4 c = q[0], e = q[1];
        float t, w;
        t = fmaf(c.x, r.inv.x, -ox); w = e.x * ax; tn.x = t - w; tf.x = t + w;
        t = fmaf(c.y, r.inv.x, -ox); w = e.y * ax; tn.y = t - w; tf.y = t + w;
        t = fmaf(c.z, r.inv.x, -ox); w = e.z * ax; tn.z = t - w; tf.z = t + w;
        t = fmaf(c.w, r.inv.x, -ox); w = e.w * ax; tn.w = t - w; tf.w = t + w;
    }
    {
        const float4 c = q[2], e = q[3];
        float t, w;
        t = fmaf(c.x, r.inv.y, -oy); w = e.x * ay; tn.x = max3f(tn.x, t - w, 0.0f); tf.x = min3f(tf.x, t + w, tmax);
        t = fmaf(c.y, r.inv.y, -oy); w = e.y * ay; tn.y = max3f(tn.y, t - w, 0.0f); tf.y = min3f(tf.y, t + w, tmax);
        t = fmaf(c.z, r.inv.y, -oy); w = e.z * ay; tn.z = max3f(tn.z, t - w, 0.0f); tf.z = min3f(tf.z, t + w, tmax);
        t = fmaf(c.w, r.inv.y, -oy); w = e.w * ay; tn.w = max3f(tn.w, t - w, 0.0f); tf.w = min3f(tf.w, t + w, tmax);
    }
    {
        const float4 c = q[4], e = q[5];
        float t, w;
        t = fmaf(c.x, r.inv.z, -oz); w = e.x * az; tn.x = fmaxf(tn.x, t - w); tf.x = fminf(tf.x, t + w);
        t = fmaf(c.y, r.inv.z, -oz); w = e.y * az; tn.y = fmaxf(tn.y, t - w); tf.y = fminf(tf.y, t + w);
        t = fmaf(c.z, r.inv.z, -oz); w = e.z * az; tn.z = fmaxf(tn.z, t - w); tf.z = fminf(tf.z, t + w);
        t = fmaf(c.w, r.inv.z, -oz); w = e.w * az; tn.w = fmaxf(tn.w, t - w); tf.w = fminf(tf.w, t + w);
    }
    ch = *reinterpret_cast<const int4 *>(q + 6);
    const float kInf = __int_as_float(0x7f800000);
    // 1 + 2^-20 widening keeps boxes conservative under FP32 rounding
    // (the subtree of the surface just left, skip_ref, counts as a miss)
    key.x = tn.x <= tf.x * 1.00000095f && ch.x != skip_ref ? tn.x : kInf;
    key.y = tn.y <= tf.y * 1.00000095f && ch.y != skip_ref ? tn.y : kInf;
    key.z = tn.z <= tf.z * 1.00000095f && ch.z != skip_ref ? tn.z : kInf;
    key.w = tn.w <= tf.w * 1.00000095f && ch.w != skip_ref ? tn.w : kInf;
}

__device__ __forceinline__ void cas_key(float &ka, int &ca, float &kb, int &cb) {
    const bool sw = kb < ka;
    const float k = sw ? kb : ka;
    const int c = sw ? cb : ca;
    kb = sw ? ka : kb;
    cb = sw ? ca : cb;
    ka = k;
    ca = c;
}

constexpr int kNoSurf = 0x7FFFFFFF;   // no surface subtree to skip

// Nearest triangle along the ray: four-wide BVH in the "while-while" order
// of Aila and Laine (HPG 2009): descend inner nodes (nearest child first, the
// other hit children stacked farthest first with their entry distances)
// until a leaf is found, postpone it, and intersect postponed leaves
// together once every active lane holds one, which keeps the lanes of a warp
// on the same kind of work. The top levels of the tree are read from shared
// memory. The subtree `skip_ref` (the surface the photon just left) is never
// entered.
template <bool COUNT>
__device__ void nearest_bvh(const SceneView &sc, const DevNode *snodes, int n_snodes,
                            f3 o, f3 d, int skip, int skip_ref, float t_min, Best &b,
                            Counters *ctr, WorkTally *w) {
    constexpr int kEmpty = INT_MIN;
    const float kInf = __int_as_float(0x7f800000);
    if (skip_ref == 0) return;            // the whole tree is that surface
    const Ray r = make_ray(o, d);
    int2 stack[RICH_BVH_STACK];
    int sp = 0;
    int ref = 0, leaf = kEmpty;
    auto pop = [&]() -> int {
        while (sp > 0) {
            --sp;
            const int2 e = stack[sp];
            if (__int_as_float(e.y) <= b.t) return e.x;
        }
        return kEmpty;
    };
    auto push = [&](int c, float t) {
        if (sp < RICH_BVH_STACK) {
            stack[sp] = make_int2(c, __float_as_int(t));
            ++sp;
        } else {
            set_status(ctr, RICH_ERR_GEOMETRY);
        }
    };
    while (ref != kEmpty || leaf != kEmpty) {
        while (ref >= 0) {
            float4 key;
            int4 ch;
            node4_test(r, ref < n_snodes ? snodes + ref : sc.nodes + ref, b.t, skip_ref, key, ch);
            if constexpr (COUNT) {
                if (ref < n_snodes) w->nodes_smem += 1; else w->nodes_global += 1;
            }
            float k0 = key.x, k1 = key.y, k2 = key.z, k3 = key.w;
            int c0 = ch.x, c1 = ch.y, c2 = ch.z, c3 = ch.w;
            // nearest first: sorting network of the four entry distances
            cas_key(k0, c0, k1, c1);
            cas_key(k2, c2, k3, c3);
            cas_key(k0, c0, k2, c2);
            cas_key(k1, c1, k3, c3);
            cas_key(k1, c1, k2, c2);
            if (k0 == kInf) {
                ref = pop();
            } else {
                if (k3 != kInf) push(c3, k3);
                if (k2 != kInf) push(c2, k2);
                if (k1 != kInf) push(c1, k1);
                ref = c0;
            }
            if (ref < 0 && ref != kEmpty && leaf == kEmpty) {
                leaf = ref;
                ref = pop();
            }
            // scheduling only: leave once every lane still here holds a leaf
            if (!__any_sync(__activemask(), leaf == kEmpty)) break;
        }
        while (leaf != kEmpty) {
            leaf_tris<COUNT>(sc, r, ~leaf, skip, t_min, b, w);
            leaf = kEmpty;
            if (ref < 0 && ref != kEmpty) {
                leaf = ref;
                ref = pop();
            }
        }
    }
}

// ======================================================= refinement replay
// Refinement of a detected photon: the recorded sequence of reflecting
// primitives is replayed in double-word arithmetic (about 48 bits, see
// rich_ff.cuh): emission, each reflection on the same primitive's surface
// extended past its edges, the final plane. All geometry is FP32 input, so
// it enters the replay exactly. Runs in its own pass (k_refine), one thread
// per stored hit, so the warps are converged.
__device__ void replay_ff(const SceneView &sc, ff3 o, ff3 d, const RefineRec &rr, float lam,
                          ff &u, ff &v) {
    for (int k = 0; k < rr.n_path; ++k) {
        const int prim = rr.path[k];
        ff3 n;               // reflective (shading) normal
        ff3 ng;              // geometric unit normal
        int mat;
        if (prim < sc.n_tiles) {
            int ti = 0;
            for (int q = 0; q < sc.n_tiles; ++q)
                if (sc.tiles[q].prim == prim) ti = q;
            const DevSphereGroup &G = sc.groups[sc.tiles[ti].group];
            const ff3 C = ff3v(G.fcx, G.fcy, G.fcz);
            const ff3 w = ff3_sub(o, C);
            const ff bq = ff3_dot(w, d);
            const ff c = ff_sub(ff3_dot(w, w), two_prod(G.radius, G.radius));
            const ff disc = ff_sub(ff_mul(bq, bq), c);
            const ff sq = ff_sqrt(disc);
            // concave (front) side: the exit root -b + sqrt(disc), taken in
            // the form free of cancellation
            const ff t = bq.hi <= 0.0f ? ff_sub(sq, bq) : ff_div(c, ff_sub(ff_neg(bq), sq));
            o = ff3_axpy(t, d, o);
            const ff3 pc = ff3_sub(o, C);
            n = ff3_scale(pc, ff_neg(ff_rsqrt(ff3_dot(pc, pc))));
            ng = n;
            mat = sc.tiles[ti].material;
        } else if (prim < sc.tri_prim_base) {
            const DevRect &R = sc.rects[prim - sc.n_tiles];
            n = ff3v(R.nx, R.ny, R.nz);
            ng = n;
            mat = R.material;
            const ff t = ff_div(ff3_dot(ff3_sub(ff3v(R.ox, R.oy, R.oz), o), n), ff3_dot(d, n));
            o = ff3_axpy(t, d, o);
        } else {
            const int k_tri = prim - sc.tri_prim_base;   // leaf-order index
            const DevTri T = load_tri(sc.tris + k_tri);
            // the triangle's refinement constants (unit normal, barycentric
            // dot products), formed on the host in FP64
            const float4 *Q = reinterpret_cast<const float4 *>(sc.tri_ref + k_tri);
            const float4 q0 = __ldg(Q), q1 = __ldg(Q + 1);
            const ff3 v0 = ff3v(T.v0x, T.v0y, T.v0z);
            ng = {ff{q0.x, q0.y}, ff{q0.z, q0.w}, ff{q1.x, q1.y}};
            const ff t = ff_div(ff3_dot(ff3_sub(v0, o), ng), ff3_dot(d, ng));
            o = ff3_axpy(t, d, o);
            mat = T.material;
            const DevMaterial &M = sc.materials[T.material];
            if ((M.flags & RICH_MAT_SMOOTH) && sc.tri_normals) {
                // barycentrics of the hit in the triangle's plane
                const float4 q2 = __ldg(Q + 2), q3 = __ldg(Q + 3);
                const ff3 e1 = ff3_diff(T.v1x, T.v1y, T.v1z, T.v0x, T.v0y, T.v0z);
                const ff3 e2 = ff3_diff(T.v2x, T.v2y, T.v2z, T.v0x, T.v0y, T.v0z);
                const ff3 q = ff3_sub(o, v0);
                const ff d00 = {q1.z, q1.w}, d01 = {q2.x, q2.y}, d11 = {q2.z, q2.w};
                const ff inv_den = {q3.x, q3.y};
                const ff d20 = ff3_dot(q, e1), d21 = ff3_dot(q, e2);
                const ff b1 = ff_mul(ff_sub(ff_mul(d11, d20), ff_mul(d01, d21)), inv_den);
                const ff b2 = ff_mul(ff_sub(ff_mul(d00, d21), ff_mul(d01, d20)), inv_den);
                const ff b0 = ff_sub(ff_sub(ffv(1.0f), b1), b2);
                const float *N = sc.tri_normals + 9 * (int64_t)k_tri;
                const ff3 m = ff3_add(ff3_add(ff3_scale(ff3v(N[0], N[1], N[2]), b0),
                                              ff3_scale(ff3v(N[3], N[4], N[5]), b1)),
                                      ff3_scale(ff3v(N[6], N[7], N[8]), b2));
                n = ff3_normalized(m);
            } else {
                n = ng;
            }
        }
        if (sc.materials[mat].kind == RICH_MAT_DIELECTRIC) {
            // refraction at a window face (as in the trace), double-word
            const float nw = table_eval(sc.tables[sc.materials[mat].table], lam);
            const bool front = ff3_dot(d, ng).hi < 0.0f;
            const ff3 N = front ? ng : ff3_scale(ng, -1.0f);
            const ff eta = front ? ff_div(ffv(1.0f), ffv(nw)) : ffv(nw);
            const ff c1 = ff_neg(ff3_dot(d, N));
            const ff kk = ff_sub(ffv(1.0f),
                                 ff_mul(ff_mul(eta, eta), ff_sub(ffv(1.0f), ff_mul(c1, c1))));
            if (kk.hi < 0.0f)
                d = ff3_reflect(d, N);
            else
                d = ff3_normalized(ff3_add(ff3_scale(d, eta),
                                           ff3_scale(N, ff_sub(ff_mul(eta, c1), ff_sqrt(kk)))));
            continue;
        }
        // |d| = 1 is kept by the reflection about a unit normal
        d = ff3_reflect(d, n);
    }
    const DevRect &R = sc.rects[rr.det_rect];
    const ff3 nrm = ff3v(R.nx, R.ny, R.nz);
    const ff3 O = ff3v(R.ox, R.oy, R.oz);
    const ff t = ff_div(ff3_dot(ff3_sub(O, o), nrm), ff3_dot(d, nrm));
    const ff3 q = ff3_sub(ff3_axpy(t, d, o), O);
    u = ff3_dot(q, R.ux, R.uy, R.uz);
    v = ff3_dot(q, R.vx, R.vy, R.vz);
}

// Orthonormal basis around a unit double-word vector (the branch-free form
// of Duff et al., JCGT 6(1) 2017, as basis_f).
__device__ __forceinline__ void basis_ff(const ff3 &t, ff3 &e1, ff3 &e2) {
    const float s = t.z.hi >= 0.0f ? 1.0f : -1.0f;
    const ff a = ff_div(ffv(-1.0f), ff_add(t.z, s));
    const ff b = ff_mul(ff_mul(t.x, t.y), a);
    e1 = {ff_add(ff_mul(ff_mul(ff_mul(t.x, t.x), a), s), 1.0f), ff_mul(b, s),
          ff_mul(t.x, -s)};
    e2 = {b, ff_add(ff_mul(ff_mul(t.y, t.y), a), s), ff_neg(t.y)};
}

// sin and cos of 2 pi u for the 24-bit uniform u = k 2^-24 of a draw word,
// double-word (~48 bits) without FP64: with k = 2^16 j + r, 2 pi u = A_j + d,
// A_j = 2 pi j / 256 from a table of (sin, cos) as hi + lo, and
// d = r (2 pi / 2^24) < 2 pi / 256; sin d and cos d by their Taylor series
// (the leading terms in double-word, the rest, below 1e-10, in FP32); then
// the angle-addition formulas.
__device__ __forceinline__ void ff_sincos_2pi(uint32_t w, ff &s, ff &c) {
    const uint32_t k = w >> 8;
    const int j = (int)(k >> 16);
    const float r = (float)(k & 0xFFFFu);
    const ff d = ff_mul(ff{kTwoPi24Hi, kTwoPi24Lo}, r);
    const ff d2 = ff_mul(d, d);
    const float t2 = d2.hi;
    // sin d = d - d^3/6 + d^5/120 - d^7/5040
    const ff d3_6 = ff_mul(ff_mul(d, d2), ff{kSixthHi, kSixthLo});
    const float s_tail = d.hi * t2 * t2 * (1.0f / 120.0f - t2 * (1.0f / 5040.0f));
    const ff sd = ff_add(ff_sub(d, d3_6), s_tail);
    // cos d = 1 - d^2/2 + d^4/24 - d^6/720
    const ff d4_24 = ff_mul(ff_mul(d2, t2), 1.0f / 24.0f);
    const float c_tail = -t2 * t2 * t2 * (1.0f / 720.0f);
    const ff cd = ff_add(ff_add(ff_sub(ffv(1.0f), ff{0.5f * d2.hi, 0.5f * d2.lo}), d4_24), c_tail);
    const float4 T = __ldg(reinterpret_cast<const float4 *>(g_sincos_tab[j]));
    const ff sa{T.x, T.y}, ca{T.z, T.w};
    s = ff_add(ff_mul(sa, cd), ff_mul(ca, sd));
    c = ff_sub(ff_mul(ca, cd), ff_mul(sa, sd));
}

__device__ __forceinline__ ff3 frame_vec(const float *v) {
    return {ff{v[0], v[1]}, ff{v[2], v[3]}, ff{v[4], v[5]}};
}

// Origin, unit track direction (from the track's frame) and (sin, cos) of
// the azimuth of photon j.
__device__ __forceinline__ void emit_start_ff(const TrackRec &tr, const TrackFrame &fr,
                                              uint32_t j, const EmitView &em, ff3 &o, ff3 &t,
                                              ff &sp, ff &cp) {
    const u4 w0 = philox10(0u, j, tr.id, tr.event, em.key0, em.key1);
    t = frame_vec(fr.t);
    const ff s = two_prod(u24f(w0.x), tr.len);      // exact: 24 x 24 bits
    o = ff3_axpy(s, t, ff3v(tr.x, tr.y, tr.z));
    ff_sincos_2pi(w0.y, sp, cp);
}

// Unit direction of the azimuth (cos, sin) in the plane normal to t, from
// the track's basis.
__device__ __forceinline__ ff3 azimuth_dir_ff(const TrackFrame &fr, ff sp, ff cp) {
    const ff3 e1 = frame_vec(fr.e1), e2 = frame_vec(fr.e2);
    return {ff_add(ff_mul(e1.x, cp), ff_mul(e2.x, sp)), ff_add(ff_mul(e1.y, cp), ff_mul(e2.y, sp)),
            ff_add(ff_mul(e1.z, cp), ff_mul(e2.z, sp))};
}

// Emission of photon j of a track with the same draws as emit_photon:
// the track direction normalised, the origin at s = u L along it, the
// azimuth 2 pi u from ff_sincos_2pi, cos and sin of the Cherenkov angle
// from the yield pass (double-words). Isotropic source: cos(theta) =
// 1 - 2u (exact) and sin(theta) = 2 sqrt(u (1 - u)) from the exact product
// u (1 - u).
__device__ void emit_ff(const TrackRec &tr, const TrackFrame &fr, float4 cs, uint32_t j,
                        float lam, const EmitView &em, ff3 &o, ff3 &d) {
    ff3 t;
    ff sp, cp;
    emit_start_ff(tr, fr, j, em, o, t, sp, cp);
    if (em.source == RICH_SOURCE_ISOTROPIC) {
        const u4 w3 = philox10(3u, j, tr.id, tr.event, em.key0, em.key1);
        const float u = u24f(w3.z);
        const ff st = ff_mul(ff_sqrt(two_prod(u, 1.0f - u)), 2.0f);
        d = {ff_mul(st, cp), ff_mul(st, sp), ffv(1.0f - 2.0f * u)};
        return;
    }
    const ff3 r = azimuth_dir_ff(fr, sp, cp);
    ff ct = {cs.x, cs.y}, st = {cs.z, cs.w};
    if (em.dispersion) {
        // dispersive radiator: the angle of the photon's own wavelength, FP64,
        // from 1 - beta (cs.z + cs.w) and n(lambda) - 1
        const double omb = (double)cs.z + (double)cs.w;
        const double il0 = 1.0 / (double)em.disp_lambda0, il = 1.0 / (double)lam;
        const double n1 = (double)em.disp_a / ((il0 - il) * (il0 + il));
        const double nb1 = (n1 - omb) - n1 * omb;
        const double cos_t = 1.0 / (1.0 + nb1);
        ct = ff_from_double(cos_t);
        st = ff_from_double(nb1 > 0.0 ? sqrt(nb1 * (2.0 + nb1)) * cos_t : 0.0);
    }
    d = ff3_normalized({ff_add(ff_mul(t.x, ct), ff_mul(r.x, st)),
                        ff_add(ff_mul(t.y, ct), ff_mul(r.y, st)),
                        ff_add(ff_mul(t.z, ct), ff_mul(r.z, st))});
}

// Pixel of a double-word position: floor(u / pitch), clamped to the grid.
__device__ __forceinline__ void pixel_of_ff(const DevRect &R, ff u, ff v, int &ix, int &iy) {
    const ff p = ffv(R.pitch);
    ix = (int)ff_floor(ff_div(u, p));
    iy = (int)ff_floor(ff_div(v, p));
    ix = ix < 0 ? 0 : (ix >= R.gx ? R.gx - 1 : ix);
    iy = iy < 0 ? 0 : (iy >= R.gy ? R.gy - 1 : iy);
}

__device__ __forceinline__ void bin_hit(const SceneView &sc, const TraceParams &P,
                                        uint32_t event, int plane, int ix, int iy) {
    if (P.pixel_counts && event < P.n_hist_events) {
        const int64_t idx = (int64_t)event * sc.pixels_per_event + sc.plane_offset[plane] +
                            (int64_t)iy * sc.plane_nx[plane] + ix;
        atomicAdd(P.pixel_counts + idx, 1u);
    }
}

constexpr int kSmemKeys = 64;   // event-sum keys a block table holds

// FP32 pixel of an FP32 plane position (the FP32 trace's own binning):
// floor(u / pitch), clamped to the grid.
__device__ __forceinline__ void pixel_of_f32(const DevRect &R, float u, float v, int &ix,
                                             int &iy) {
    ix = (int)floorf(__fdiv_rn(u, R.pitch));
    iy = (int)floorf(__fdiv_rn(v, R.pitch));
    ix = ix < 0 ? 0 : (ix >= R.gx ? R.gx - 1 : ix);
    iy = iy < 0 ? 0 : (iy >= R.gy ? R.gy - 1 : iy);
}

// The block's shared event-sum table: used when the call's keys fit.
__device__ __forceinline__ bool es_table_on(const SceneView &sc, const TraceParams &P) {
    const int64_t n_keys = P.event_sums ? (int64_t)P.n_hist_events * sc.n_planes : 0;
    return n_keys > 0 && n_keys <= kSmemKeys;
}
__device__ __forceinline__ void es_table_flush(const SceneView &sc, const TraceParams &P,
                                               const double *s_es) {
    const int n = (int)P.n_hist_events * sc.n_planes * 4;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        if (s_es[i] != 0.0) atomicAdd(P.event_sums + i, s_es[i]);
}

__device__ __forceinline__ ff shfl_xor_ff(ff a, int o) {
    return {__shfl_xor_sync(0xFFFFFFFFu, a.hi, o), __shfl_xor_sync(0xFFFFFFFFu, a.lo, o)};
}

// Event sums (hits, sum u, sum v, sum lambda) of the lanes of a converged
// warp: for each distinct (event, plane) key among the taking lanes, a
// butterfly sum over the warp in double-word arithmetic (lanes of other keys
// add zero; ~1e-14 relative), then one FP64 atomic per component from the
// key's first lane, so the accumulation over warps is FP64; the hit count
// is the lane count. With few keys (one event, a few planes) the warps of a
// block accumulate in shared memory first, which keeps thousands of warps
// from serialising on the same few global addresses.
// s_es: the block's shared-memory table of the sums (all keys of the call,
// flushed to global memory when the block ends) or null for direct global
// atomics.

__device__ __forceinline__ void add_event_sums(const SceneView &sc, const TraceParams &P,
                                               bool on, uint32_t event, int plane, ff u,
                                               ff v, float lam, double *s_es) {
    const bool take = on && P.event_sums && event < P.n_hist_events;
    unsigned act = __ballot_sync(0xFFFFFFFFu, take);
    const long long key = (long long)event * sc.n_planes + plane;
    const int lane = threadIdx.x & 31;
    while (act) {
        const int leader = __ffs(act) - 1;
        const long long k = __shfl_sync(0xFFFFFFFFu, key, leader);
        const bool mine = take && key == k;
        const unsigned grp = __ballot_sync(0xFFFFFFFFu, mine);
        ff su = mine ? u : ffv(0.0f), sv = mine ? v : ffv(0.0f), sl = ffv(mine ? lam : 0.0f);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            su = ff_add(su, shfl_xor_ff(su, o));
            sv = ff_add(sv, shfl_xor_ff(sv, o));
            sl = ff_add(sl, shfl_xor_ff(sl, o));
        }
        if (lane == leader) {
            double *es = (s_es ? s_es : P.event_sums) + k * 4;
            atomicAdd(es + 0, (double)__popc(grp));
            atomicAdd(es + 1, ff_to_double(su));
            atomicAdd(es + 2, ff_to_double(sv));
            atomicAdd(es + 3, ff_to_double(sl));
        }
        act &= ~grp;
    }
}

// Efficiencies applied before propagation (Sec. 4.3): the FP32 product,
// left to right, of the listed response tables at the photon's wavelength.
__device__ __forceinline__ float prefilter_prob(const SmemScene &S, const TraceParams &P,
                                                float lam) {
    float pr = table_eval(S.tables()[P.prefilter_tables[0]], lam);
    for (int k = 1; k < P.n_prefilter; ++k)
        pr = __fmul_rn(pr, table_eval(S.tables()[P.prefilter_tables[k]], lam));
    return pr;
}

// ================================================================ trace
struct TraceArgs {
    SceneView sc;
    EmitView em;
    ExtView ext;
    TraceParams p;
    Counters *ctr;
    Counters *ctr_next;      // zeroed here for the next trace, or null
};

__device__ __forceinline__ uint32_t refl_word(const Photon &ph, int k,
                                              const EmitView &em) {
    if (k < 4) return k == 0 ? ph.wr0 : (k == 1 ? ph.wr1 : (k == 2 ? ph.wr2 : ph.wr3));
    u4 w = philox10(2u, ph.j, ph.id, ph.event, em.key0, em.key1);
    k -= 4;
    return k == 0 ? w.x : (k == 1 ? w.y : (k == 2 ? w.z : w.w));
}

// Cold photon state in shared memory: the kColdWords words of thread t at
// [t * kColdWords + f]; the stride is odd, so the 32 lanes of a warp fall in
// 32 different banks. Addressed by one 32-bit offset into the dynamic shared
// memory (a generic 64-bit pointer would hold two registers).
enum : int {
    kCLam = 0, kCWqe, kCWr0, kCWr1, kCWr2, kCWr3, kCEvent, kCId, kCJ, kCGlo, kCGhi, kCTrack,
    kCCount,            // n_refl | n_turn << 8 | steps << 16
    kColdWords
};
static_assert(kColdWords % 2 == 1, "an odd stride keeps the lanes in distinct banks");
struct ColdState {
    uint32_t off;       // byte offset of this thread's first word
    __device__ __forceinline__ volatile uint32_t &at(int f) const {
        return reinterpret_cast<volatile uint32_t *>(rich_dsmem + off)[f];
    }
};
__device__ __forceinline__ uint32_t cold_refl_word(const ColdState &c, int k,
                                                   const EmitView &em) {
    if (k < 4) return c.at(kCWr0 + k);
    u4 w = philox10(2u, c.at(kCJ), c.at(kCId), c.at(kCEvent), em.key0, em.key1);
    k -= 4;
    return k == 0 ? w.x : (k == 1 ? w.y : (k == 2 ? w.z : w.w));
}

template <bool EXT, bool REFINE, int THREADS, int MINB, bool COUNT = false>
__global__ void __launch_bounds__(THREADS, MINB)
k_trace(TraceArgs A) {
    extern __shared__ __align__(128) unsigned char smem[];
    const SceneView &sc = A.sc;
    // ---- top BVH levels: one TMA bulk copy into shared memory, completion
    //      tracked by an mbarrier; the wait is bounded and falls back to
    //      global reads (with an error status) if it ever runs out
    __shared__ __align__(8) unsigned long long s_bar;
    const int n_snodes_req = A.p.smem_nodes;
    int n_snodes = n_snodes_req;
    const DevNode *snodes = reinterpret_cast<const DevNode *>(smem);
    const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&s_bar);
    if (n_snodes_req > 0) {
        if (threadIdx.x == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const uint32_t bytes = (uint32_t)n_snodes_req * (uint32_t)sizeof(DevNode);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                         "r"(bytes)
                         : "memory");
            const uint32_t dst = (uint32_t)__cvta_generic_to_shared(smem);
            const char *src = reinterpret_cast<const char *>(sc.nodes);
            for (uint32_t off = 0; off < bytes; off += 32768u) {
                const uint32_t len = bytes - off < 32768u ? bytes - off : 32768u;
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
                    "[%0], [%1], %2, [%3];" ::"r"(dst + off),
                    "l"(src + off), "r"(len), "r"(bar)
                    : "memory");
            }
        }
    }
    const size_t scene_off = ((size_t)n_snodes_req * sizeof(DevNode) + 127) & ~size_t(127);
    // ---- stage the small scene tables into shared memory
    SmemScene S;
    uint32_t cold_off = 0;
    {
        size_t off = scene_off;
        auto carve = [&](size_t bytes) {
            unsigned char *p = smem + off;
            off += (bytes + 15) & ~size_t(15);
            return p;
        };
        auto copy = [&](void *dst, const void *src, size_t bytes) {
            const uint32_t *s = static_cast<const uint32_t *>(src);
            uint32_t *d = static_cast<uint32_t *>(dst);
            for (size_t i = threadIdx.x; i < bytes / 4; i += blockDim.x) d[i] = s[i];
        };
        DevSphereGroup *g = reinterpret_cast<DevSphereGroup *>(carve(sizeof(DevSphereGroup) * sc.n_groups));
        DevTile *t = reinterpret_cast<DevTile *>(carve(sizeof(DevTile) * sc.n_tiles));
        DevRect *r = reinterpret_cast<DevRect *>(carve(sizeof(DevRect) * sc.n_rects));
        DevTable *tb = reinterpret_cast<DevTable *>(carve(sizeof(DevTable) * sc.n_tables));
        DevMaterial *m = reinterpret_cast<DevMaterial *>(carve(sizeof(DevMaterial) * sc.n_materials));
        copy(g, sc.groups, sizeof(DevSphereGroup) * sc.n_groups);
        copy(t, sc.tiles, sizeof(DevTile) * sc.n_tiles);
        copy(r, sc.rects, sizeof(DevRect) * sc.n_rects);
        copy(tb, sc.tables, sizeof(DevTable) * sc.n_tables);
        copy(m, sc.materials, sizeof(DevMaterial) * sc.n_materials);
        auto o32 = [&](const void *q) {
            return (uint32_t)(static_cast<const unsigned char *>(q) - smem);
        };
        S = {o32(g), o32(t), o32(r), o32(tb), o32(m), sc.n_groups, sc.n_tiles, sc.n_rects};
        if (RICH_COLD_SMEM && THREADS > 256)
            cold_off = (uint32_t)(carve(sizeof(uint32_t) * kColdWords * blockDim.x) - smem);
    }
    if (n_snodes_req > 0) {
        auto try_wait = [&]() {
            uint32_t ok;
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
                "selp.u32 %0, 1, 0, p;\n\t}"
                : "=r"(ok)
                : "r"(bar)
                : "memory");
            return ok;
        };
        uint32_t done = 0;
        for (int it = 0; it < A.p.wait_limit && !done; ++it) done = try_wait();
        if (!done) {
            // the wait ran out: record it, read every node from global
            // memory, and wait again (bounded) for the copy still in flight
            // so that it does not land while the block runs on or exits
            set_status(A.ctr, RICH_ERR_TIMEOUT);
            n_snodes = 0;
            for (int it = 0; it < (1 << 20) && !done; ++it) done = try_wait();
        }
    }
    __shared__ unsigned long long s_fate[RICH_N_FATES];
    __shared__ unsigned long long s_hits;
    __shared__ double s_es_tab[kSmemKeys * 4];
    double *const s_es = es_table_on(sc, A.p) ? s_es_tab : nullptr;
    for (int i = threadIdx.x; i < kSmemKeys * 4; i += blockDim.x) s_es_tab[i] = 0.0;
    if (threadIdx.x < RICH_N_FATES) s_fate[threadIdx.x] = 0;
    if (threadIdx.x == 0) s_hits = 0;
    __syncthreads();
    // the emission (offsets, total, order) is complete from here on
    grid_dep_wait();
    if (blockIdx.x == 0) {
        // the photon total beside this trace's counters, and the next
        // trace's counter slot zeroed
        if (threadIdx.x == 0)
            *reinterpret_cast<unsigned long long *>(A.ctr + 1) =
                EXT ? (unsigned long long)A.ext.n : *A.em.total;
        if (A.ctr_next && threadIdx.x < (int)(sizeof(Counters) / sizeof(unsigned long long)))
            reinterpret_cast<unsigned long long *>(A.ctr_next)[threadIdx.x] = 0ull;
    }

    // (No early launch_dependents here: letting the refinement pass's blocks
    // be scheduled while the trace runs slowed the trace by ~5 % on large
    // workloads. The refinement is still launched programmatically, so its
    // launch overlaps the trace's end.)
    const TraceParams &P = A.p;
    const EmitView &em = A.em;
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    const bool has_tri = sc.n_tris > 0;
    // order flags of the emission: bit 0 its queue entries are ordered; the
    // word equal to 1 (no track left in index order) makes every entry hold
    // its photon and track
    const uint32_t order_flags = (!EXT && em.perm) ? *em.perm_ok : 0u;
    const bool ordered = (order_flags & 1u) != 0u;
    const bool entries = order_flags == 1u;
    if (blockIdx.x == 0 && threadIdx.x == 0) A.ctr->ordered = ordered ? 1u : 0u;

    Photon ph;
    bool alive = false;
    int path[RICH_MAX_BOUNCES];
    WorkTally tally{};
    // the shapes of one block per SM (896 threads at 72 registers, 1024 at
    // 64) keep the cold photon state in shared memory (there it removes the
    // bounce loop's spills); the 256-thread shapes keep it in registers
    constexpr bool kColdOn = RICH_COLD_SMEM && THREADS > 256;
    const ColdState cold{cold_off + (uint32_t)threadIdx.x * (uint32_t)(sizeof(uint32_t) * kColdWords)};
#define PH_LAM (kColdOn ? __uint_as_float(cold.at(kCLam)) : ph.lam)
#define PH_WQE (kColdOn ? (uint32_t)cold.at(kCWqe) : ph.w_qe)
#define PH_EVENT (kColdOn ? (uint32_t)cold.at(kCEvent) : ph.event)
#define PH_ID (kColdOn ? (uint32_t)cold.at(kCId) : ph.id)
#define PH_J (kColdOn ? (uint32_t)cold.at(kCJ) : ph.j)
#define PH_G (kColdOn ? (((uint64_t)cold.at(kCGhi) << 32) | cold.at(kCGlo)) : ph.g)
#define PH_TRACK (kColdOn ? (uint32_t)cold.at(kCTrack) : ph.track)
#define PH_NREFL (kColdOn ? (int)(cold.at(kCCount) & 0xFFu) : ph.n_refl)
#define PH_NTURN (kColdOn ? (int)((cold.at(kCCount) >> 8) & 0xFFu) : ph.n_turn)
#define PH_STEPS (kColdOn ? (int)(cold.at(kCCount) >> 16) : ph.steps)
#define PH_REFL_WORD(k) (kColdOn ? cold_refl_word(cold, (k), em) : refl_word(ph, (k), em))
#define PH_ADD_REFL() do { if (kColdOn) cold.at(kCCount) = cold.at(kCCount) + 1u; else ph.n_refl += 1; } while (0)
#define PH_ADD_TURN() do { if (kColdOn) cold.at(kCCount) = cold.at(kCCount) + 0x100u; else ph.n_turn += 1; } while (0)
#define PH_ADD_STEP() do { if (kColdOn) cold.at(kCCount) = cold.at(kCCount) + 0x10000u; else ph.steps += 1; } while (0)
    // the warp's photon pool (next, end, track of next; warp-uniform) lives
    // in shared memory between refills, so that it holds no registers
    // through the bounce loop
    __shared__ unsigned long long s_pool[32][3];
    unsigned long long *const wpool = s_pool[threadIdx.x >> 5];
    if (lane < 3) wpool[lane] = 0ull;
    __syncwarp();
    bool more = true;                       // warp-uniform

    while (true) {
        // ---------------------------------------------------- refill
        unsigned idle = __ballot_sync(kFull, !alive);
        if (more && (__popc(idle) >= P.refill_min || idle == kFull)) {
            uint64_t pool_next = wpool[0], pool_end = wpool[1];
            int64_t pool_track = (int64_t)wpool[2];
            const uint64_t N = EXT ? A.ext.n : (uint64_t)(*em.total);
            const uint64_t chunk = (uint64_t)P.chunk;
            while (idle != 0u && more) {
                if (pool_next >= pool_end) {
                    unsigned long long base = 0;
                    if (lane == 0) base = atomicAdd(&A.ctr->work, (unsigned long long)chunk);
                    base = __shfl_sync(kFull, base, 0);
                    if (base >= N) {
                        more = false;
                        break;
                    }
                    pool_next = base;
                    pool_end = base + chunk < N ? base + chunk : N;
                    // the track of pool_next: found below when a lane needs it
                    pool_track = -1;
                }
                const int rank = __popc(idle & lt_mask);
                const uint64_t avail = pool_end - pool_next;
                const bool take = ((idle >> lane) & 1u) && (uint64_t)rank < avail;
                // when every track was ordered, the queue entry names the
                // photon and its track (no search for the track)
                bool from_entry = false;
                uint32_t j_entry = 0;
                int64_t entry_track = 0;
                if (!EXT && take && entries) {
                    const uint2 e = em.perm[pool_next + (uint64_t)rank];
                    from_entry = true;
                    j_entry = e.x;
                    entry_track = (int64_t)e.y;
                }
                if (!EXT && pool_track < 0 && __any_sync(kFull, take && !from_entry)) {
                    // 32-ary search for the track containing pool_next
                    int64_t lo = 0, hi = em.n_tracks;
                    while (hi - lo > 32) {
                        const int64_t step = (hi - lo + 31) / 32;
                        const int64_t idx = lo + lane * step;
                        const bool ok = idx < hi && em.offsets[idx] <= pool_next;
                        const unsigned m = __ballot_sync(kFull, ok);
                        const int L = 31 - __clz(m);
                        lo = lo + L * step;
                        hi = (lo + step < hi) ? lo + step : hi;
                    }
                    const int64_t idx = lo + lane;
                    const bool ok = idx < hi && em.offsets[idx] <= pool_next;
                    const unsigned m = __ballot_sync(kFull, ok);
                    pool_track = lo + (31 - __clz(m));
                }
                int64_t my_track = from_entry ? entry_track : pool_track;
                bool rejected = false;
                if (take) {
                    const uint64_t g = pool_next + (uint64_t)rank;
                    ph.g = g;
                    ph.skip = -1;
                    ph.skip_ref = kNoSurf;
                    ph.n_refl = 0;
                    ph.n_turn = 0;
                    ph.steps = 0;
                    if (EXT) {
                        ph.track = (uint32_t)g;
                        ph.lam = A.ext.lambda[g];
                        ph.event = A.ext.event[g];
                        ph.id = A.ext.track[g];
                        ph.j = A.ext.photon[g];
                        const u4 w0 = philox10(0u, ph.j, ph.id, ph.event, em.key0, em.key1);
                        ph.w_qe = w0.w;
                        if (P.n_prefilter && !(u24f(w0.w) < prefilter_prob(S, P, ph.lam))) {
                            rejected = true;
                        } else {
                            ph.o = mk3(A.ext.x[g], A.ext.y[g], A.ext.z[g]);
                            ph.d = mk3(A.ext.dx[g], A.ext.dy[g], A.ext.dz[g]);
                            const u4 w1 = philox10(1u, ph.j, ph.id, ph.event, em.key0, em.key1);
                            ph.wr0 = w1.x; ph.wr1 = w1.y; ph.wr2 = w1.z; ph.wr3 = w1.w;
                        }
                    } else {
                        if (!from_entry)
                            while (my_track + 1 < em.n_tracks && em.offsets[my_track + 1] <= g)
                                ++my_track;
                        ph.track = (uint32_t)my_track;
                        const TrackRec tr = em.tracks[my_track];
                        const uint64_t toff = em.offsets[my_track];
                        uint32_t j = from_entry ? j_entry : (uint32_t)(g - toff);
                        // some tracks in index order: the ordered ones' entries
                        if (!from_entry && ordered && em.offsets[my_track + 1] - toff <= kOrderMaxPhotons)
                            j = em.perm[g].x;
                        ph.g = toff + j;
                        const u4 w0 = philox10(0u, j, tr.id, tr.event, em.key0, em.key1);
                        const DevTable *spec = em.spectrum >= 0 ? S.tables() + em.spectrum : nullptr;
                        const float lam = photon_wavelength(tr, j, em, w0, spec);
                        // efficiencies before propagation (Sec. 4.3): only
                        // the wavelength is needed to decide
                        if (P.n_prefilter && !(u24f(w0.w) < prefilter_prob(S, P, lam)))
                            rejected = true;
                        else
                            emit_photon(tr, j, em, w0, lam, ph);
                    }
                    if (rejected) {
                        if (ph.g < P.fate_capacity) P.fate[ph.g] = (uint8_t)RICH_FATE_PREFILTERED;
                    } else {
                        alive = true;
                        if (kColdOn) {
                        cold.at(kCLam) = __float_as_uint(ph.lam);
                        cold.at(kCWqe) = ph.w_qe;
                        cold.at(kCWr0) = ph.wr0;
                        cold.at(kCWr1) = ph.wr1;
                        cold.at(kCWr2) = ph.wr2;
                        cold.at(kCWr3) = ph.wr3;
                        cold.at(kCEvent) = ph.event;
                        cold.at(kCId) = ph.id;
                        cold.at(kCJ) = ph.j;
                        cold.at(kCGlo) = (uint32_t)ph.g;
                        cold.at(kCGhi) = (uint32_t)(ph.g >> 32);
                        cold.at(kCTrack) = ph.track;
                        cold.at(kCCount) = 0u;
                        }
                    }
                }
                const unsigned taken = __ballot_sync(kFull, take);
                const unsigned rej = __ballot_sync(kFull, rejected);
                if (rej && lane == 0)
                    atomicAdd(&s_fate[RICH_FATE_PREFILTERED], (unsigned long long)__popc(rej));
                if (taken) {
                    const int last = 31 - __clz(taken);
                    pool_next += __popc(taken);
                    if (!EXT) pool_track = __shfl_sync(kFull, my_track, last);
                }
                idle &= ~(taken & ~rej);
                if (taken == 0u && pool_next < pool_end) break;  // defensive
            }
            __syncwarp();
            if (lane == 0) {
                wpool[0] = pool_next;
                wpool[1] = pool_end;
                wpool[2] = (unsigned long long)pool_track;
            }
            __syncwarp();
        }
        if (!__any_sync(kFull, alive)) {
            if (!more) break;
            continue;
        }

        // ---------------------------------------------- one bounce step
        int fate = 0;
        int det_rect = -1;
        float hit_u = 0.0f, hit_v = 0.0f;
        if (alive) {
            Best b;
            b.t = 3.0e38f;
            b.prim = -1;
            b.kind = -1;
            b.idx = -1;
            b.b0 = b.b1 = b.b2 = 0.0f;
            if constexpr (COUNT) tally.steps += 1;
            if (S.n_groups) nearest_tiles(S, ph.o, ph.d, ph.skip, P.t_min, b);
            nearest_rects(S, ph.o, ph.d, ph.skip, P.t_min, b);
            if (has_tri)
                nearest_bvh<COUNT>(sc, snodes, n_snodes, ph.o, ph.d, ph.skip, ph.skip_ref,
                                   P.t_min, b, A.ctr, COUNT ? &tally : nullptr);
            if (b.prim < 0) {
                fate = RICH_FATE_ESCAPED;
            } else {
                const f3 p = fma3(ph.d, b.t, ph.o);
                int mat_id;
                bool front;
                f3 n_sh, n_geo;
                int hit_ref = kNoSurf;    // surface subtree of a hit triangle
                if (b.kind == 0) {
                    const DevTile &T = S.tiles()[b.idx];
                    const DevSphereGroup &G = S.groups()[T.group];
                    n_sh = sphere_normal(G, ph.o, ph.d, b.t);
                    n_geo = n_sh;
                    front = dot3(ph.d, n_sh) < 0.0f;
                    mat_id = T.material;
                } else if (b.kind == 1) {
                    const DevRect &R = S.rects()[b.idx];
                    n_sh = mk3(R.nx, R.ny, R.nz);
                    n_geo = n_sh;
                    front = dot3(ph.d, n_sh) < 0.0f;
                    mat_id = R.material;
                } else {
                    const DevTri T = load_tri(sc.tris + b.idx);
                    const f3 e1 = mk3(T.v1x - T.v0x, T.v1y - T.v0y, T.v1z - T.v0z);
                    const f3 e2 = mk3(T.v2x - T.v0x, T.v2y - T.v0y, T.v2z - T.v0z);
                    const f3 ng = cross3(e1, e2);
                    front = dot3(ph.d, ng) < 0.0f;
                    n_geo = normalize3(ng);
                    mat_id = T.material;
                    hit_ref = T.pad;
                    const DevMaterial &M0 = S.materials()[mat_id];
                    if ((M0.flags & RICH_MAT_SMOOTH) && sc.tri_normals) {
                        const float *N3 = sc.tri_normals + 9 * (int64_t)b.idx;
                        const f3 n0 = mk3(__ldg(N3 + 0), __ldg(N3 + 1), __ldg(N3 + 2));
                        const f3 n1 = mk3(__ldg(N3 + 3), __ldg(N3 + 4), __ldg(N3 + 5));
                        const f3 n2 = mk3(__ldg(N3 + 6), __ldg(N3 + 7), __ldg(N3 + 8));
                        n_sh = normalize3(fma3(n0, b.b0, fma3(n1, b.b1, n2 * b.b2)));
                        if constexpr (COUNT) tally.normals += 1;
                    } else {
                        n_sh = n_geo;
                    }
                }
                const DevMaterial &M = S.materials()[mat_id];
                if (M.kind == RICH_MAT_ABSORBER) {
                    fate = RICH_FATE_ABSORBED;
                } else if (M.kind == RICH_MAT_MIRROR) {
                    if (!front) {
                        fate = RICH_FATE_ABSORBED;
                    } else if (PH_NTURN >= P.max_bounces) {
                        fate = RICH_FATE_MAX_BOUNCES;
                    } else {
                        // with the efficiencies applied before propagation
                        // every front-side reflection succeeds
                        const bool pass =
                            P.n_prefilter ||
                            u24f(PH_REFL_WORD(PH_NREFL)) < table_eval(S.tables()[M.table], PH_LAM);
                        if (!pass) {
                            fate = RICH_FATE_MIRROR_ABSORBED;
                        } else {
                            ph.d = normalize3(reflect_f(ph.d, n_sh));
                            if constexpr (COUNT) tally.turns += 1;
                            if (REFINE) path[PH_NTURN] = b.kind == 2 ? sc.tri_prim_base + b.idx : b.prim;
                            PH_ADD_REFL();
                            PH_ADD_TURN();
                            ph.o = p;
                            ph.skip = b.prim;
                            ph.skip_ref = hit_ref;
                        }
                    }
                } else if (M.kind == RICH_MAT_DIELECTRIC) {
                    // window face: Snell's law, eta = n_in / n_out with the
                    // table's index behind the face; total internal
                    // reflection when k < 0
                    if (PH_NTURN >= P.max_bounces) {
                        fate = RICH_FATE_MAX_BOUNCES;
                    } else {
                        const float nw = table_eval(S.tables()[M.table], PH_LAM);
                        const float eta = front ? __fdiv_rn(1.0f, nw) : nw;
                        const f3 N = front ? n_geo : n_geo * -1.0f;
                        const float c1 = -dot3(ph.d, N);
                        const float k = 1.0f - eta * eta * (1.0f - c1 * c1);
                        ph.d = k < 0.0f ? normalize3(reflect_f(ph.d, N))
                                        : normalize3(fma3(N, eta * c1 - sqrtf(k), ph.d * eta));
                        if constexpr (COUNT) tally.turns += 1;
                        if (REFINE) path[PH_NTURN] = b.kind == 2 ? sc.tri_prim_base + b.idx : b.prim;
                        PH_ADD_TURN();
                        ph.o = p;
                        ph.skip = b.prim;
                        ph.skip_ref = hit_ref;
                    }
                } else {  // detector
                    if (!front) {
                        ph.o = p;
                        ph.skip = b.prim;
                        ph.skip_ref = hit_ref;
                    } else {
                        const bool pass =
                            P.n_prefilter || u24f(PH_WQE) < table_eval(S.tables()[M.table], PH_LAM);
                        if (!pass) {
                            fate = RICH_FATE_QE_REJECTED;
                        } else {
                            fate = RICH_FATE_DETECTED;
                            det_rect = b.idx;
                            const DevRect &R = S.rects()[b.idx];
                            const f3 q = p - mk3(R.ox, R.oy, R.oz);
                            hit_u = dot3(q, mk3(R.ux, R.uy, R.uz));
                            hit_v = dot3(q, mk3(R.vx, R.vy, R.vz));
                        }
                    }
                }
                if (fate == 0) {
                    PH_ADD_STEP();
                    if (PH_STEPS >= P.max_steps) fate = RICH_FATE_MAX_STEPS;
                }
            }
        }

        // -------------------------------------------- finished photons
        const bool det = fate == RICH_FATE_DETECTED;
        const unsigned dm = __ballot_sync(kFull, det);
        bool binned_here = false;
        float hu = 0.0f, hv = 0.0f;
        int hplane = 0;
        if (dm) {
            unsigned long long base = 0;
            const int leader = __ffs(dm) - 1;
            if (lane == leader) base = atomicAdd(&A.ctr->hits, (unsigned long long)__popc(dm));
            base = __shfl_sync(kFull, base, leader);
            if (det) {
                const DevRect &R = S.rects()[det_rect];
                hplane = S.materials()[R.material].plane;
                hu = hit_u;
                hv = hit_v;
                const uint64_t slot = base + (uint64_t)__popc(dm & lt_mask);
                const bool stored = slot < P.hit_capacity;
                // refined hits are binned (and their pixel found, in double-word)
                // by the refinement pass; the rest here
                binned_here = !(REFINE && stored);
                int ix = 0, iy = 0;
                if (binned_here) pixel_of_f32(R, hu, hv, ix, iy);
                if (stored) {
                    rich_hit h;
                    h.event = PH_EVENT;
                    h.track = PH_ID;
                    h.photon = PH_J;
                    h.plane = (uint8_t)hplane;
                    h.n_reflections = (uint8_t)PH_NREFL;
                    h.reserved = 0;
                    h.ix = (uint16_t)ix;
                    h.iy = (uint16_t)iy;
                    h.lambda = PH_LAM;
                    h.u = hu;
                    h.v = hv;
                    P.hits[slot] = h;
                    if (REFINE) {
                        RefineRec rr;
                        rr.index = PH_TRACK;
                        rr.det_rect = (uint8_t)det_rect;
                        rr.n_path = (uint8_t)PH_NTURN;
                        rr.pad = 0;
#pragma unroll
                        for (int k = 0; k < RICH_MAX_BOUNCES; ++k) rr.path[k] = path[k];
                        P.refine[slot] = rr;
                    }
                }
                if (binned_here) bin_hit(sc, P, PH_EVENT, hplane, ix, iy);
            }
        }
        add_event_sums(sc, P, binned_here, alive ? PH_EVENT : 0u, hplane, ffv(hu), ffv(hv),
                       alive ? PH_LAM : 0.0f, s_es);
        if (fate != 0) {
            const uint64_t g_fate = PH_G;
            if (g_fate < P.fate_capacity) P.fate[g_fate] = (uint8_t)fate;
            atomicAdd(&s_fate[fate], 1ull);
            alive = false;
        }
    }
    if constexpr (COUNT) {
        atomicAdd(P.work + 0, (unsigned long long)tally.steps);
        atomicAdd(P.work + 1, (unsigned long long)tally.nodes_smem);
        atomicAdd(P.work + 2, (unsigned long long)tally.nodes_global);
        atomicAdd(P.work + 3, (unsigned long long)tally.tris);
        atomicAdd(P.work + 4, (unsigned long long)tally.normals);
        atomicAdd(P.work + 5, (unsigned long long)tally.turns);
    }
    __syncthreads();
    if (threadIdx.x < RICH_N_FATES && s_fate[threadIdx.x])
        atomicAdd(&A.ctr->fate[threadIdx.x], s_fate[threadIdx.x]);
    if (s_es) es_table_flush(sc, P, s_es);
    if (n_snodes_req > 0 && n_snodes == 0) {
        // the copy had not completed: give it a second bounded wait so the
        // block does not retire with a transfer into its shared memory
        uint32_t done = 0;
        for (int it = 0; it < (1 << 20) && !done; ++it) {
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
                "selp.u32 %0, 1, 0, p;\n\t}"
                : "=r"(done)
                : "r"(bar)
                : "memory");
        }
    }
}

// Refinement pass: one thread per stored hit (converged warps). Hits are
// taken in chunks of 32, chunk c by the warp with global index c over a
// warp numbering that runs across the blocks first, so the chunks spread
// evenly over the SMs whatever the hit count.
template <bool EXT>
__global__ void __launch_bounds__(256)
k_refine(SceneView sc, EmitView em, ExtView ext, TraceParams P, Counters *ctr) {
    __shared__ double s_es_tab[kSmemKeys * 4];
    double *const s_es = es_table_on(sc, P) ? s_es_tab : nullptr;
    for (int i = threadIdx.x; i < kSmemKeys * 4; i += blockDim.x) s_es_tab[i] = 0.0;
    __syncthreads();
    grid_dep_wait();                     // the trace has ended
    const uint64_t n_hits = ctr->hits < P.hit_capacity ? ctr->hits : P.hit_capacity;
    const uint64_t n_chunks = (n_hits + 31) / 32;
    const uint64_t n_warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    const int lane = threadIdx.x & 31;
    for (uint64_t c = blockIdx.x + (uint64_t)gridDim.x * (threadIdx.x >> 5); c < n_chunks;
         c += n_warps) {
        const uint64_t i = c * 32 + (uint64_t)lane;
        const bool on = i < n_hits;
        ff uf = ffv(0.0f), vf = ffv(0.0f);
        int plane = 0;
        uint32_t event = 0;
        float lam = 0.0f;
        if (on) {
            rich_hit h = P.hits[i];
            const RefineRec rr = P.refine[i];
            ff3 o, d;
            if (EXT) {
                const uint32_t g = rr.index;
                o = ff3v(ext.x[g], ext.y[g], ext.z[g]);
                d = ff3_normalized(ff3v(ext.dx[g], ext.dy[g], ext.dz[g]));
            } else {
                emit_ff(em.tracks[rr.index], em.frame[rr.index], em.cos_sin[rr.index], h.photon,
                        h.lambda, em, o, d);
            }
            replay_ff(sc, o, d, rr, h.lambda, uf, vf);
            int ix, iy;
            pixel_of_ff(sc.rects[rr.det_rect], uf, vf, ix, iy);
            h.u = ff_to_double(uf);
            h.v = ff_to_double(vf);
            h.ix = (uint16_t)ix;
            h.iy = (uint16_t)iy;
            P.hits[i] = h;
            plane = h.plane;
            event = h.event;
            lam = h.lambda;
            bin_hit(sc, P, event, plane, ix, iy);
        }
        add_event_sums(sc, P, on, event, plane, uf, vf, lam, s_es);
    }
    __syncthreads();
    if (s_es) es_table_flush(sc, P, s_es);
}

cudaError_t launch_refine(const SceneView &sc, const EmitView *em, const ExtView *ext,
                          const TraceParams &p, Counters *counters, int n_sm,
                          cudaStream_t s) {
    if (p.hit_capacity == 0) return cudaSuccess;
    // every block resident at once (two 256-thread blocks per SM)
    uint64_t blocks = (p.hit_capacity + 255) / 256;
    const uint64_t cap = (uint64_t)n_sm * 2;
    if (blocks > cap) blocks = cap;
    if (ext)
        return launch_pdl(k_refine<true>, (unsigned)blocks, 256, 0, s, sc,
                          em ? *em : EmitView{}, *ext, p, counters);
    return launch_pdl(k_refine<false>, (unsigned)blocks, 256, 0, s, sc, *em, ExtView{}, p,
                      counters);
}

// ============================================================== adjoint
// Gradient of the soft ring chi^2 with respect to theta = (tilt alpha_k,
// beta_k of sphere tiles 0..3, radius of curvature, n - 1): every stored hit
// is replayed along its recorded reflecting surfaces (fixed topology) in
// forward mode, with double-word values (the refinement replay's arithmetic,
// see rich_ff.cuh) and FP32 tangents. A photon's position depends on the
// tilts of the tiles its path meets only (one, for a photon of the RICH
// layouts), so a replay carries 4 tangents: slots 0 and 1 the tilts of one
// tile, 2 the radius, 3 n - 1. Forward mode is linear in the seeds: the first
// pass seeds the first tile's tilts, the radius and n - 1, each further tile
// of the path one more pass with its tilts alone.
constexpr int kNG = 4;     // tangents per replay
constexpr int kNP = 10;    // parameters
struct Dm {
    ff v;
    float d[kNG];
};
struct Dm3 {
    Dm x, y, z;
};

__device__ __forceinline__ Dm dm_c(ff v) {
    Dm r;
    r.v = v;
#pragma unroll
    for (int k = 0; k < kNG; ++k) r.d[k] = 0.0f;
    return r;
}
__device__ __forceinline__ Dm dm_add(const Dm &a, const Dm &b) {
    Dm r;
    r.v = ff_add(a.v, b.v);
#pragma unroll
    for (int k = 0; k < kNG; ++k) r.d[k] = a.d[k] + b.d[k];
    return r;
}
__device__ __forceinline__ Dm dm_sub(const Dm &a, const Dm &b) {
    Dm r;
    r.v = ff_sub(a.v, b.v);
#pragma unroll
    for (int k = 0; k < kNG; ++k) r.d[k] = a.d[k] - b.d[k];
    return r;
}
__device__ __forceinline__ Dm dm_addf(const Dm &a, float c) {
    Dm r = a;
    r.v = ff_add(a.v, c);
    return r;
}
__device__ __forceinline__ Dm dm_neg(const Dm &a) {
    Dm r;
    r.v = ff_neg(a.v);
#pragma unroll
    for (int k = 0; k < kNG; ++k) r.d[k] = -a.d[k];
    return r;
}
__device__ __forceinline__ Dm dm_mul(const Dm &a, const Dm &b) {
    Dm r;
    r.v = ff_mul(a.v, b.v);
#pragma unroll
    for (int k = 0; k < kNG; ++k) r.d[k] = fmaf(a.d[k], b.v.hi, a.v.hi * b.d[k]);
    return r;
}
__device__ __forceinline__ Dm dm_scl(const Dm &a, ff s) {
    Dm r;
    r.v = ff_mul(a.v, s);
#pragma unroll
    for (int k = 0; k < kNG; ++k) r.d[k] = a.d[k] * s.hi;
    return r;
}
__device__ __forceinline__ Dm dm_scl(const Dm &a, float s) {
    Dm r;
    r.v = ff_mul(a.v, s);
#pragma unroll
    for (int k = 0; k < kNG; ++k) r.d[k] = a.d[k] * s;
    return r;
}
__device__ __forceinline__ Dm dm_div(const Dm &a, const Dm &b) {
    Dm r;
    r.v = ff_div(a.v, b.v);
    const float ib = 1.0f / b.v.hi;
#pragma unroll
    for (int k = 0; k < kNG; ++k) r.d[k] = (a.d[k] - r.v.hi * b.d[k]) * ib;
    return r;
}
__device__ __forceinline__ Dm dm_divc(const Dm &a, ff c) {
    Dm r;
    r.v = ff_div(a.v, c);
    const float ic = 1.0f / c.hi;
#pragma unroll
    for (int k = 0; k < kNG; ++k) r.d[k] = a.d[k] * ic;
    return r;
}
__device__ __forceinline__ Dm dm_sqrt(const Dm &a) {
    Dm r;
    r.v = ff_sqrt(a.v);
    const float h = r.v.hi > 0.0f ? 0.5f / r.v.hi : 0.0f;
#pragma unroll
    for (int k = 0; k < kNG; ++k) r.d[k] = a.d[k] * h;
    return r;
}
// 1 / sqrt(a), a > 0: d(a^-1/2) = -a^-3/2 da / 2
__device__ __forceinline__ Dm dm_rsqrt(const Dm &a) {
    Dm r;
    r.v = ff_rsqrt(a.v);
    const float h = -0.5f * r.v.hi * r.v.hi * r.v.hi;
#pragma unroll
    for (int k = 0; k < kNG; ++k) r.d[k] = a.d[k] * h;
    return r;
}
__device__ __forceinline__ Dm3 dm3_c(const ff3 &a) { return {dm_c(a.x), dm_c(a.y), dm_c(a.z)}; }
__device__ __forceinline__ Dm3 dm3_sub(const Dm3 &a, const Dm3 &b) {
    return {dm_sub(a.x, b.x), dm_sub(a.y, b.y), dm_sub(a.z, b.z)};
}
// c - a for a constant c
__device__ __forceinline__ Dm3 dm3_csub(const ff3 &c, const Dm3 &a) {
    return {dm_add(dm_neg(a.x), dm_c(c.x)), dm_add(dm_neg(a.y), dm_c(c.y)),
            dm_add(dm_neg(a.z), dm_c(c.z))};
}
__device__ __forceinline__ Dm3 dm3_scl(const Dm3 &a, const Dm &s) {
    return {dm_mul(a.x, s), dm_mul(a.y, s), dm_mul(a.z, s)};
}
// a + s b
__device__ __forceinline__ Dm3 dm3_axpy(const Dm3 &a, const Dm3 &b, const Dm &s) {
    return {dm_add(a.x, dm_mul(b.x, s)), dm_add(a.y, dm_mul(b.y, s)),
            dm_add(a.z, dm_mul(b.z, s))};
}
__device__ __forceinline__ Dm dm3_dot(const Dm3 &a, const Dm3 &b) {
    return dm_add(dm_add(dm_mul(a.x, b.x), dm_mul(a.y, b.y)), dm_mul(a.z, b.z));
}
__device__ __forceinline__ Dm dm3_dotc(const Dm3 &a, const ff3 &b) {
    return dm_add(dm_add(dm_scl(a.x, b.x), dm_scl(a.y, b.y)), dm_scl(a.z, b.z));
}
__device__ __forceinline__ Dm dm3_dotf(const Dm3 &a, float bx, float by, float bz) {
    return dm_add(dm_add(dm_scl(a.x, bx), dm_scl(a.y, by)), dm_scl(a.z, bz));
}
// reflection about the unit normal n, renormalised: the tangent of the
// normal does not keep |d| = 1 to first order by itself
__device__ __forceinline__ Dm3 dm3_reflect_unit(const Dm3 &d, const Dm3 &n) {
    const Dm k = dm_scl(dm3_dot(d, n), -2.0f);
    const Dm3 r = dm3_axpy(d, n, k);
    return dm3_scl(r, dm_rsqrt(dm3_dot(r, r)));
}
// component c of tile centre C(theta) with its tangents: in the tile's own
// tilts when it is the pass's tile (own), in R on the first pass
__device__ __forceinline__ Dm tile_centre(const DevTileDual &T, int c, bool own, bool first) {
    Dm r;
    r.v = {T.c_hi[c], T.c_lo[c]};
    r.d[0] = own ? T.dc_dalpha[c] : 0.0f;
    r.d[1] = own ? T.dc_dbeta[c] : 0.0f;
    r.d[2] = first ? T.dc_dr[c] : 0.0f;
    r.d[3] = 0.0f;
    return r;
}

// pass_tile: the tile (0..3) whose tilts are seeded in slots 0 and 1, or
// -1; first: the radius and n - 1 seeded in slots 2 and 3
__device__ void replay_dual(const SceneView &sc, const GradView &gv, const EmitView &em,
                            const RefineRec &rr, uint32_t j, int pass_tile, bool first,
                            Dm &u_out, Dm &v_out) {
    const TrackRec tr = em.tracks[rr.index];
    const float4 cs = em.cos_sin[rr.index];
    // emission as in the refinement replay; the tangent of the Cherenkov
    // angle in n - 1: cos = 1 / (n beta) gives d cos / dn = -cos / n and
    // d sin / dn = -cos (d cos / dn) / sin
    const TrackFrame fr = em.frame[rr.index];
    ff3 o0, t;
    ff sp, cp;
    emit_start_ff(tr, fr, j, em, o0, t, sp, cp);
    const ff3 r = azimuth_dir_ff(fr, sp, cp);
    const ff ct = {cs.x, cs.y}, st = {cs.z, cs.w};
    const ff3 d0 = ff3_normalized({ff_add(ff_mul(t.x, ct), ff_mul(r.x, st)),
                                   ff_add(ff_mul(t.y, ct), ff_mul(r.y, st)),
                                   ff_add(ff_mul(t.z, ct), ff_mul(r.z, st))});
    const float dct = first ? -ct.hi / (1.0f + (float)gv.theta[9]) : 0.0f;
    const float dst = st.hi > 0.0f ? -ct.hi * dct / st.hi : 0.0f;
    Dm3 o = dm3_c(o0), d = dm3_c(d0);
    d.x.d[3] = t.x.hi * dct + r.x.hi * dst;
    d.y.d[3] = t.y.hi * dct + r.y.hi * dst;
    d.z.d[3] = t.z.hi * dct + r.z.hi * dst;
    Dm R = dm_c(ff_from_double(gv.theta[8]));
    R.d[2] = first ? 1.0f : 0.0f;
    const Dm inv_R = dm_div(dm_c(ffv(1.0f)), R);
    for (int k = 0; k < rr.n_path; ++k) {
        const int prim = rr.path[k];
        Dm3 n;
        if (prim < sc.n_tiles) {
            const DevTileDual &T = gv.tiles[prim];
            const bool own = prim == pass_tile;
            const Dm3 C = {tile_centre(T, 0, own, first), tile_centre(T, 1, own, first),
                           tile_centre(T, 2, own, first)};
            const Dm3 w = dm3_sub(o, C);
            const Dm b = dm3_dot(w, d);
            const Dm c = dm_sub(dm3_dot(w, w), dm_mul(R, R));
            const Dm sq = dm_sqrt(dm_sub(dm_mul(b, b), c));
            // the concave side's exit root, in the form free of cancellation
            const Dm tt = b.v.hi <= 0.0f ? dm_sub(sq, b) : dm_div(c, dm_sub(dm_neg(b), sq));
            o = dm3_axpy(o, d, tt);
            n = dm3_scl(dm3_sub(C, o), inv_R);
        } else if (prim < sc.tri_prim_base) {
            const DevRect &Rc = sc.rects[prim - sc.n_tiles];
            const ff3 nn = ff3v(Rc.nx, Rc.ny, Rc.nz);
            const Dm tt = dm_div(dm3_dotc(dm3_csub(ff3v(Rc.ox, Rc.oy, Rc.oz), o), nn),
                                 dm3_dotc(d, nn));
            o = dm3_axpy(o, d, tt);
            n = dm3_c(nn);
        } else {
            const int k_tri = prim - sc.tri_prim_base;
            const DevTri T = load_tri(sc.tris + k_tri);
            const float4 *Q = reinterpret_cast<const float4 *>(sc.tri_ref + k_tri);
            const float4 q0 = __ldg(Q), q1 = __ldg(Q + 1);
            const ff3 v0 = ff3v(T.v0x, T.v0y, T.v0z);
            const ff3 ng = {ff{q0.x, q0.y}, ff{q0.z, q0.w}, ff{q1.x, q1.y}};
            const Dm tt = dm_div(dm3_dotc(dm3_csub(v0, o), ng), dm3_dotc(d, ng));
            o = dm3_axpy(o, d, tt);
            const DevMaterial &M = sc.materials[T.material];
            if ((M.flags & RICH_MAT_SMOOTH) && sc.tri_normals) {
                const float4 q2 = __ldg(Q + 2), q3 = __ldg(Q + 3);
                const ff3 e1 = ff3_diff(T.v1x, T.v1y, T.v1z, T.v0x, T.v0y, T.v0z);
                const ff3 e2 = ff3_diff(T.v2x, T.v2y, T.v2z, T.v0x, T.v0y, T.v0z);
                const Dm3 q = dm3_sub(o, dm3_c(v0));
                const ff d00 = {q1.z, q1.w}, d01 = {q2.x, q2.y}, d11 = {q2.z, q2.w};
                const ff inv_den = {q3.x, q3.y};
                const Dm d20 = dm3_dotc(q, e1), d21 = dm3_dotc(q, e2);
                const Dm b1 = dm_scl(dm_sub(dm_scl(d20, d11), dm_scl(d21, d01)), inv_den);
                const Dm b2 = dm_scl(dm_sub(dm_scl(d21, d00), dm_scl(d20, d01)), inv_den);
                const Dm b0 = dm_addf(dm_neg(dm_add(b1, b2)), 1.0f);
                const float *N = sc.tri_normals + 9 * (int64_t)k_tri;
                const Dm3 m = {
                    dm_add(dm_add(dm_scl(b0, N[0]), dm_scl(b1, N[3])), dm_scl(b2, N[6])),
                    dm_add(dm_add(dm_scl(b0, N[1]), dm_scl(b1, N[4])), dm_scl(b2, N[7])),
                    dm_add(dm_add(dm_scl(b0, N[2]), dm_scl(b1, N[5])), dm_scl(b2, N[8]))};
                n = dm3_scl(m, dm_rsqrt(dm3_dot(m, m)));
            } else {
                n = dm3_c(ng);
            }
        }
        d = dm3_reflect_unit(d, n);
    }
    const DevRect &Rc = sc.rects[rr.det_rect];
    const ff3 nn = ff3v(Rc.nx, Rc.ny, Rc.nz);
    const ff3 O = ff3v(Rc.ox, Rc.oy, Rc.oz);
    const Dm tt = dm_div(dm3_dotc(dm3_csub(O, o), nn), dm3_dotc(d, nn));
    const Dm3 q = dm3_sub(dm3_axpy(o, d, tt), dm3_c(O));
    u_out = dm3_dotf(q, Rc.ux, Rc.uy, Rc.uz);
    v_out = dm3_dotf(q, Rc.vx, Rc.vy, Rc.vz);
}

// Box-Muller pair of the photon's smear draws (words x, y of draw block 3)
// in FP32: u1 = (k + 1/2) 2^-24 from the leading 24 bits k of x, and
// log u1 as logf(u1) below 1/2 and log1pf(-(1 - u1)) above, where u1 and
// 1 - u1 are both exact in FP32, so -2 log u1 keeps its relative precision
// as u1 approaches 1.
__device__ __forceinline__ void smear_pair_f32(u4 w3, float &g1, float &g2) {
    const uint32_t k = w3.x >> 8;
    const float lg = k < (1u << 23)
                         ? logf((float)(2u * k + 1u) * 0x1p-25f)
                         : log1pf(-(float)(2u * ((1u << 24) - k) - 1u) * 0x1p-25f);
    const float rad = sqrtf(-2.0f * lg);
    float s, c;
    sincospif(2.0f * u24f(w3.y), &s, &c);
    g1 = rad * c;
    g2 = rad * s;
}

constexpr int kAdjThreads = 128;
// three blocks per SM: 163 registers, no spills (12 warps per SM; four
// blocks at 128 registers spill and are no faster)
constexpr int kAdjMinBlocks = 3;

// Sums of the loss and the gradient: double-word FP32 per thread and over
// the block (a warp butterfly, then shared memory; ~2^-44 relative per
// addition), then one FP64 atomic per accumulator per block. On GB300 an
// FP64 instruction holds the SM's FP64 unit for ~64 cycles; summing in FP64
// per hit kept that unit the busiest of the kernel.
__global__ void __launch_bounds__(kAdjThreads, kAdjMinBlocks)
k_adjoint(SceneView sc, EmitView em, TraceParams P, GradView gv, Counters *ctr) {
    const uint64_t n_hits = ctr->hits < P.hit_capacity ? ctr->hits : P.hit_capacity;
    ff acc[1 + kNP];
#pragma unroll
    for (int k = 0; k < 1 + kNP; ++k) acc[k] = ffv(0.0f);
    uint32_t used = 0;
    const ff sg = ff_from_double(gv.sigma);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_hits;
         i += (uint64_t)gridDim.x * blockDim.x) {
        rich_hit h = P.hits[i];
        const RefineRec rr = P.refine[i];
        const float4 tg = gv.targets[(int64_t)rr.index * gv.n_planes + h.plane];
        float g1 = 0.0f, g2 = 0.0f;
        if (tg.w > 0.0f) {
            const u4 w3 = philox10(3u, h.photon, h.track, h.event, em.key0, em.key1);
            smear_pair_f32(w3, g1, g2);
        }
        // the tilted tiles (0..3) the path meets: one replay per tile
        uint32_t rest = 0;
        for (int k = 0; k < rr.n_path; ++k)
            if (rr.path[k] < sc.n_tiles && rr.path[k] < 4) rest |= 1u << rr.path[k];
        bool first = true;
        do {
            const int pass_tile = rest ? __ffs(rest) - 1 : -1;
            rest &= rest - 1u;
            Dm u, v;
            replay_dual(sc, gv, em, rr, h.photon, pass_tile, first, u, v);
            if (first) {
                int ix, iy;
                pixel_of_ff(sc.rects[rr.det_rect], u.v, v.v, ix, iy);
                h.u = ff_to_double(u.v);
                h.v = ff_to_double(v.v);
                h.ix = (uint16_t)ix;
                h.iy = (uint16_t)iy;
                P.hits[i] = h;
                bin_hit(sc, P, h.event, h.plane, ix, iy);
            }
            if (tg.w > 0.0f) {
                const Dm du = dm_addf(dm_addf(u, -tg.x), sg.hi * g1);
                const Dm dv = dm_addf(dm_addf(v, -tg.y), sg.hi * g2);
                const Dm dist = dm_sqrt(dm_add(dm_mul(du, du), dm_mul(dv, dv)));
                const Dm rho = dm_divc(dm_addf(dist, -tg.z), sg);
                if (first) {
                    acc[0] = ff_add(acc[0], ff_mul(rho.v, rho.v));
                    used += 1;
                    acc[1 + 8] = ff_add(acc[1 + 8], ff_mul(rho.v, 2.0f * rho.d[2]));
                    acc[1 + 9] = ff_add(acc[1 + 9], ff_mul(rho.v, 2.0f * rho.d[3]));
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (q == pass_tile) {
                        acc[1 + 2 * q] = ff_add(acc[1 + 2 * q], ff_mul(rho.v, 2.0f * rho.d[0]));
                        acc[2 + 2 * q] = ff_add(acc[2 + 2 * q], ff_mul(rho.v, 2.0f * rho.d[1]));
                    }
                }
            }
            first = false;
        } while (rest);
    }
    // block reduction, one FP64 atomic per accumulator per block
    __shared__ ff red[kAdjThreads / 32][1 + kNP];
    __shared__ uint32_t red_used[kAdjThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 1 + kNP; ++k) {
        ff x = acc[k];
        for (int o = 16; o > 0; o >>= 1) x = ff_add(x, shfl_xor_ff(x, o));
        if (lane == 0) red[wid][k] = x;
    }
    for (int o = 16; o > 0; o >>= 1) used += __shfl_xor_sync(kFull, used, o);
    if (lane == 0) red_used[wid] = used;
    __syncthreads();
    if (threadIdx.x < 2 + kNP) {
        double x = 0.0;
        if (threadIdx.x == 1) {
            uint32_t n = 0;
            for (int w = 0; w < kAdjThreads / 32; ++w) n += red_used[w];
            x = (double)n;
        } else {
            const int k = threadIdx.x == 0 ? 0 : threadIdx.x - 1;
            ff y = ffv(0.0f);
            for (int w = 0; w < kAdjThreads / 32; ++w) y = ff_add(y, red[w][k]);
            x = ff_to_double(y);
        }
        if (x != 0.0) atomicAdd(gv.acc + threadIdx.x, x);
    }
}

cudaError_t launch_adjoint(const SceneView &sc, const EmitView &em, const TraceParams &p,
                           const GradView &gv, Counters *counters, int n_sm,
                           cudaStream_t s) {
    if (p.hit_capacity == 0) return cudaSuccess;
    uint64_t blocks = (p.hit_capacity + kAdjThreads - 1) / kAdjThreads;
    const uint64_t cap = (uint64_t)n_sm * 8;
    if (blocks > cap) blocks = cap;
    k_adjoint<<<(unsigned)blocks, kAdjThreads, 0, s>>>(sc, em, p, gv, counters);
    return cudaGetLastError();
}

// Philox outputs for caller-given counters (reproduction of draws).
__global__ void k_philox(const uint32_t *ctr, uint64_t n, uint32_t k0, uint32_t k1,
                         uint32_t *out) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint4 c = reinterpret_cast<const uint4 *>(ctr)[i];
        const u4 r = philox10(c.x, c.y, c.z, c.w, k0, k1);
        reinterpret_cast<uint4 *>(out)[i] = make_uint4(r.x, r.y, r.z, r.w);
    }
}

cudaError_t launch_philox(const uint32_t *ctr, uint64_t n, uint64_t seed, uint32_t *out,
                          cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    uint64_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_philox<<<(unsigned)blocks, 256, 0, s>>>(ctr, n, (uint32_t)seed, (uint32_t)(seed >> 32), out);
    return cudaGetLastError();
}

// ============================================================== launchers
cudaError_t launch_yield(const TracksView &t, double n_minus_1,
                         double lam_min, double lam_max, uint32_t key0,
                         uint32_t key1, TrackRec *rec, float4 *cs,
                         uint32_t *counts, unsigned long long *block_sums,
                         cudaStream_t s, const YieldModel &model, TrackFrame *frame,
                         uint32_t *perm_ok) {
    if (t.n <= 0) return cudaSuccess;
    const double inv_band_mm = 1.0e6 / lam_min - 1.0e6 / lam_max;
    // the kernel's double-word parameters, split here
    const ff nm1 = ffc(n_minus_1), inv_band = ffc(inv_band_mm);
    const int64_t groups = (t.n + kYieldThreads - 1) / kYieldThreads;
    cudaError_t e = cudaMemsetAsync(block_sums, 0, sizeof(unsigned long long) * groups, s);
    if (e != cudaSuccess) return e;
    const unsigned blocks =
        (unsigned)((t.n * kYieldLanes + kYieldBlock - 1) / kYieldBlock);
    if (rec)
        k_yield<true><<<blocks, kYieldBlock, 0, s>>>(t, nm1, inv_band, key0, key1,
                                                     rec, cs, counts, block_sums, model,
                                                     lam_min, lam_max, frame, perm_ok);
    else
        k_yield<false><<<blocks, kYieldBlock, 0, s>>>(t, nm1, inv_band, key0, key1,
                                                      rec, cs, counts, block_sums, model,
                                                      lam_min, lam_max, nullptr, perm_ok);
    return cudaGetLastError();
}

cudaError_t launch_offsets(const uint32_t *counts,
                           const unsigned long long *block_sums,
                           int64_t n_tracks, uint64_t *offsets,
                           unsigned long long *total, cudaStream_t s) {
    if (n_tracks <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((n_tracks + kYieldThreads - 1) / kYieldThreads);
    k_offsets<<<blocks, kYieldThreads, 0, s>>>(counts, block_sums, n_tracks, offsets, total);
    return cudaGetLastError();
}

cudaError_t launch_materialize(const SceneView &sc, const EmitView &em,
                               uint64_t n, const rich_photons &out,
                               cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    uint64_t blocks = (n + 255) / 256;
    if (blocks > 65535ull * 16) blocks = 65535ull * 16;
    k_materialize<<<(unsigned)blocks, 256, 0, s>>>(sc, em, n, out);
    return cudaGetLastError();
}

enum { kShape256x4 = 0, kShape256x1 = 1, kShape1024 = 2, kShapeWide = 3 };

size_t trace_smem_bytes(const SceneView &sc, int smem_nodes, int threads, int cls) {
    auto r16 = [](size_t b) { return (b + 15) & ~size_t(15); };
    const size_t nodes = ((size_t)smem_nodes * sizeof(DevNode) + 127) & ~size_t(127);
    // the shapes of one block per SM keep their cold photon state here
    const size_t cold = (RICH_COLD_SMEM && (cls == kShapeWide || cls == kShape1024))
                            ? r16(sizeof(uint32_t) * kColdWords * (size_t)threads) : 0;
    return nodes + r16(sizeof(DevSphereGroup) * sc.n_groups) + r16(sizeof(DevTile) * sc.n_tiles) +
           r16(sizeof(DevRect) * sc.n_rects) + r16(sizeof(DevTable) * sc.n_tables) +
           r16(sizeof(DevMaterial) * sc.n_materials) + cold;
}

// Dynamic shared-memory limit of a trace kernel variant: raised to `bytes`
// when it is below, never lowered (the occupancy queries and the launches of
// one variant ask for different sizes; the attribute persists, so a captured
// replay issues no such call).
static cudaError_t ensure_dyn_smem(const void *f, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, size_t> raised;   // per device
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    size_t &r = raised[{dev, f}];
    if (bytes <= r) return cudaSuccess;
    const cudaError_t e =
        cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) r = bytes;
    return e;
}

template <bool EXT, bool REFINE, int THREADS, int MINB, bool COUNT = false>
static cudaError_t launch_trace_t(const TraceArgs &a, const LaunchShape &shape,
                                  cudaStream_t s) {
    auto kern = k_trace<EXT, REFINE, THREADS, MINB, COUNT>;
    if (shape.smem) {
        const cudaError_t e = ensure_dyn_smem((const void *)kern, shape.smem);
        if (e != cudaSuccess) return e;
    }
    // programmatic: the prologue (staging the top BVH levels and the scene
    // tables) may overlap the ordering pass ahead of it
    return launch_pdl(kern, (unsigned)shape.blocks, (unsigned)shape.threads, shape.smem, s, a);
}

// Kernel variants: caller photons or fused emission; refinement side
// records or not; block shape class: up to 256 threads capped at 64
// registers (4 blocks per SM), up to 256 threads uncapped, up to 896
// threads capped at 72 registers, or up to 1024 threads capped at 64 (the
// last two one block per SM, sharing one staged copy of the BVH top, with
// the cold photon state in shared memory).

template <bool EXT, bool REFINE>
static const void *trace_kernel_t(int cls) {
    if (cls == kShape1024) return (const void *)k_trace<EXT, REFINE, 1024, 1>;
    if (cls == kShapeWide) return (const void *)k_trace<EXT, REFINE, RICH_WIDE_THREADS, 1>;
    if (cls == kShape256x1) return (const void *)k_trace<EXT, REFINE, 256, 1>;
    return (const void *)k_trace<EXT, REFINE, 256, 4>;
}

static const void *trace_kernel(bool ext, bool refine, int cls) {
    if (ext) return refine ? trace_kernel_t<true, true>(cls) : trace_kernel_t<true, false>(cls);
    return refine ? trace_kernel_t<false, true>(cls) : trace_kernel_t<false, false>(cls);
}

int trace_shape_class(int threads, bool wide) {
    if (threads > 256) return (wide && threads <= RICH_WIDE_THREADS) ? kShapeWide : kShape1024;
    return wide ? kShape256x1 : kShape256x4;
}

int trace_blocks_per_sm(bool ext, bool refine, int cls, int threads, size_t smem) {
    int n = 0;
    const void *f = trace_kernel(ext, refine, cls);
    if (smem > 0 && ensure_dyn_smem(f, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

template <bool EXT, bool REFINE>
static cudaError_t launch_cls(const TraceArgs &a, const LaunchShape &shape, cudaStream_t s) {
    if (shape.cls == kShape1024) return launch_trace_t<EXT, REFINE, 1024, 1>(a, shape, s);
    if (shape.cls == kShapeWide) return launch_trace_t<EXT, REFINE, RICH_WIDE_THREADS, 1>(a, shape, s);
    if (shape.cls == kShape256x1) return launch_trace_t<EXT, REFINE, 256, 1>(a, shape, s);
    return launch_trace_t<EXT, REFINE, 256, 4>(a, shape, s);
}

cudaError_t launch_trace(const SceneView &sc, const EmitView *em,
                         const ExtView *ext, const TraceParams &p,
                         Counters *counters, Counters *next, const LaunchShape &shape,
                         cudaStream_t s) {
    TraceArgs a;
    a.sc = sc;
    a.em = em ? *em : EmitView{};
    a.ext = ext ? *ext : ExtView{};
    a.p = p;
    a.ctr = counters;
    a.ctr_next = next;
    const bool refine = p.precision == RICH_PREC_REFINE64;
    if (ext) return refine ? launch_cls<true, true>(a, shape, s) : launch_cls<true, false>(a, shape, s);
    return refine ? launch_cls<false, true>(a, shape, s) : launch_cls<false, false>(a, shape, s);
}

// The counting build of the fused-emission trace with refinement records
// (the benchmark's form) in the two shape classes of more than 256 threads
// (72 registers up to 896 threads, 64 registers up to 1024): the same
// traversal, plus per-thread tallies of its work summed into p.work.
bool trace_count_shape_ok(int cls) { return cls == kShapeWide || cls == kShape1024; }

cudaError_t launch_trace_count(const SceneView &sc, const EmitView &em, const TraceParams &p,
                               Counters *counters, Counters *next, const LaunchShape &shape,
                               cudaStream_t s) {
    TraceArgs a;
    a.sc = sc;
    a.em = em;
    a.ext = ExtView{};
    a.p = p;
    a.ctr = counters;
    a.ctr_next = next;
    if (shape.cls == kShapeWide) return launch_trace_t<false, true, RICH_WIDE_THREADS, 1, true>(a, shape, s);
    if (shape.cls == kShape1024) return launch_trace_t<false, true, 1024, 1, true>(a, shape, s);
    return cudaErrorInvalidValue;
}

}  // namespace rich
