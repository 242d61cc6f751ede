// rich_ff.cuh -- double-word ("float-float") arithmetic for the refinement
// replay.
//
// A value is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi) / 2, about 48 significant bits. On this GPU an FP32
// operation issues at 64 times the rate of an FP64 one, so a replay written
// with these building blocks finishes well before the same replay in FP64
// while keeping hit positions within ~1e-10 mm of it.
//
// Building blocks, written from their published definitions:
//   two_sum       Knuth's error-free sum (TAOCP vol. 2, 4.2.2)
//   fast_two_sum  Dekker 1971 (needs |a| >= |b| or a = 0)
//   two_prod      error-free product with one fused multiply-add
//   add / mul / div / sqrt on double-words: the algorithms analysed by
//   Joldes, Muller and Popescu, "Tight and rigorous error bounds for basic
//   building blocks of double-word arithmetic", ACM TOMS 44(2), 2017
//   (accurate DW + DW, DW x FP and DW x DW with FMA, DW / DW), and the
//   one-step Newton corrections s + (x - s^2) / (2 s) for the square root
//   and r + r (1 - x r^2) / 2 for its reciprocal.
// Every FP32 operation is an explicit round-to-nearest intrinsic so the
// compiler cannot contract or reorder the error-free transformations.
#pragma once

#include <cstdint>

namespace rich {

struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ffv(float a) { return {a, 0.0f}; }

// A double constant as a double-word, for constexpr use (evaluated by the
// compiler: no FP64 operation at run time).
__host__ __device__ constexpr ff ffc(double x) {
    return {(float)x, (float)(x - (double)(float)x)};
}

__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float ap = __fsub_rn(s, b);
    const float bp = __fsub_rn(s, ap);
    const float da = __fsub_rn(a, ap);
    const float db = __fsub_rn(b, bp);
    return {s, __fadd_rn(da, db)};
}

__device__ __forceinline__ ff fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float z = __fsub_rn(s, a);
    return {s, __fsub_rn(b, z)};
}

__device__ __forceinline__ ff two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }

// DW + FP
__device__ __forceinline__ ff ff_add(ff x, float y) {
    const ff s = two_sum(x.hi, y);
    return fast_two_sum(s.hi, __fadd_rn(x.lo, s.lo));
}

// DW + DW (the accurate variant: valid for either sign)
__device__ __forceinline__ ff ff_add(ff x, ff y) {
    const ff s = two_sum(x.hi, y.hi);
    const ff t = two_sum(x.lo, y.lo);
    const ff v = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return fast_two_sum(v.hi, __fadd_rn(t.lo, v.lo));
}

__device__ __forceinline__ ff ff_sub(ff x, ff y) { return ff_add(x, ff_neg(y)); }

// DW x FP
__device__ __forceinline__ ff ff_mul(ff x, float y) {
    const ff c = two_prod(x.hi, y);
    return fast_two_sum(c.hi, __fmaf_rn(x.lo, y, c.lo));
}

// DW x DW
__device__ __forceinline__ ff ff_mul(ff x, ff y) {
    const ff c = two_prod(x.hi, y.hi);
    const float t = __fmaf_rn(x.hi, y.lo, __fmul_rn(x.lo, y.lo));
    const float cl = __fadd_rn(c.lo, __fmaf_rn(x.lo, y.hi, t));
    return fast_two_sum(c.hi, cl);
}

// Hardware approximations (a few ulp) of 1/x and 1/sqrt(x): the
// double-word algorithms below start from them and correct the result from
// an error-free remainder, which removes their error to second order.
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
    float r;
    asm("rsqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// DW / DW: FP32 quotient of the leading parts (from an approximate
// reciprocal), then one correction from the remainder x - q y evaluated with
// error-free products: relative error ~2^-44.
__device__ __forceinline__ ff ff_div(ff x, ff y) {
    const float ry = rcp_approx(y.hi);
    const float th = __fmul_rn(x.hi, ry);
    const ff r = ff_mul(y, th);
    const ff p = two_sum(x.hi, -r.hi);
    const float dl = __fadd_rn(__fsub_rn(p.lo, r.lo), x.lo);
    const float d = __fadd_rn(p.hi, dl);
    return fast_two_sum(th, __fmul_rn(d, ry));
}

// sqrt of a DW: s ~ x r with r ~ 1/sqrt(x), then s + (x - s^2) r / 2.
__device__ __forceinline__ ff ff_sqrt(ff x) {
    if (!(x.hi > 0.0f)) return {0.0f, 0.0f};
    const float r = rsqrt_approx(x.hi);
    const float s = __fmul_rn(x.hi, r);
    const ff s2 = two_prod(s, s);
    const float e = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, s2.hi), s2.lo), x.lo);
    return fast_two_sum(s, __fmul_rn(e, __fmul_rn(0.5f, r)));
}

// 1 / sqrt(x), x > 0: one Newton step in double-word from the approximation
__device__ __forceinline__ ff ff_rsqrt(ff x) {
    const float r = rsqrt_approx(x.hi);
    const ff r2 = two_prod(r, r);
    const ff m = ff_mul(x, r2);                 // x r^2 = 1 - e
    const float e = __fsub_rn(__fsub_rn(1.0f, m.hi), m.lo);
    return fast_two_sum(r, __fmul_rn(__fmul_rn(0.5f, r), e));
}

__device__ __forceinline__ ff ff_from_double(double a) {
    const float h = (float)a;
    return {h, (float)(a - (double)h)};
}

__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

// comparisons of normalised double-words
__device__ __forceinline__ bool ff_lt(ff a, ff b) {
    return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}
__device__ __forceinline__ bool ff_le(ff a, ff b) {
    return a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo);
}

// floor of a double-word (the pixel index)
__device__ __forceinline__ float ff_floor(ff a) {
    const float f = floorf(a.hi);
    if (f != a.hi) return f;          // hi not an integer: lo cannot cross it
    return a.lo < 0.0f ? f - 1.0f : f;
}

// ---------------------------------------------------------------- vectors
struct ff3 {
    ff x, y, z;
};

__device__ __forceinline__ ff3 ff3v(float x, float y, float z) {
    return {ffv(x), ffv(y), ffv(z)};
}
__device__ __forceinline__ ff3 ff3_add(ff3 a, ff3 b) {
    return {ff_add(a.x, b.x), ff_add(a.y, b.y), ff_add(a.z, b.z)};
}
__device__ __forceinline__ ff3 ff3_sub(ff3 a, ff3 b) {
    return {ff_sub(a.x, b.x), ff_sub(a.y, b.y), ff_sub(a.z, b.z)};
}
// exact difference of two FP32 points
__device__ __forceinline__ ff3 ff3_diff(float ax, float ay, float az, float bx, float by,
                                        float bz) {
    return {two_sum(ax, -bx), two_sum(ay, -by), two_sum(az, -bz)};
}
__device__ __forceinline__ ff3 ff3_scale(ff3 a, ff s) {
    return {ff_mul(a.x, s), ff_mul(a.y, s), ff_mul(a.z, s)};
}
__device__ __forceinline__ ff3 ff3_scale(ff3 a, float s) {
    return {ff_mul(a.x, s), ff_mul(a.y, s), ff_mul(a.z, s)};
}
// a + s b
__device__ __forceinline__ ff3 ff3_axpy(ff s, ff3 b, ff3 a) {
    return {ff_add(a.x, ff_mul(b.x, s)), ff_add(a.y, ff_mul(b.y, s)),
            ff_add(a.z, ff_mul(b.z, s))};
}
__device__ __forceinline__ ff ff3_dot(ff3 a, ff3 b) {
    return ff_add(ff_add(ff_mul(a.x, b.x), ff_mul(a.y, b.y)), ff_mul(a.z, b.z));
}
__device__ __forceinline__ ff ff3_dot(ff3 a, float bx, float by, float bz) {
    return ff_add(ff_add(ff_mul(a.x, bx), ff_mul(a.y, by)), ff_mul(a.z, bz));
}
__device__ __forceinline__ ff3 ff3_cross(ff3 a, ff3 b) {
    return {ff_sub(ff_mul(a.y, b.z), ff_mul(a.z, b.y)),
            ff_sub(ff_mul(a.z, b.x), ff_mul(a.x, b.z)),
            ff_sub(ff_mul(a.x, b.y), ff_mul(a.y, b.x))};
}
__device__ __forceinline__ ff3 ff3_normalized(ff3 a) {
    return ff3_scale(a, ff_rsqrt(ff3_dot(a, a)));
}
// reflection about the unit normal n: d - 2 (d.n) n
__device__ __forceinline__ ff3 ff3_reflect(ff3 d, ff3 n) {
    const ff k = ff_mul(ff3_dot(d, n), -2.0f);
    return ff3_axpy(k, n, d);
}

}  // namespace rich
