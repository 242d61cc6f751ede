// rich_device.cuh -- device-side data layout and inline math of the photon
// propagator (sm_103a). Included by the kernel translation unit only.
//
// Every function here is the GPU's own statement of a step of the method:
//   * Philox4x32-10 counter-based random numbers (Salmon et al., SC'11);
//   * Cherenkov emission at cos(theta) = 1/(n beta) (paper Sec. 3) with a
//     Frank-Tamm wavelength (1/lambda^2 spectrum);
//   * ray / sphere-tile, ray / rectangle and ray / triangle intersection
//     (the mirror and detector surfaces of Sec. 4.1), the latter with the
//     watertight test of Woop, Benthin and Wald (JCGT 2(1), 2013);
//   * specular reflection and the binned wavelength responses of Sec. 4.3.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "rich_internal.h"

namespace rich {

// ------------------------------------------------------------ small math
struct f3 {
    float x, y, z;
};
__device__ __forceinline__ f3 mk3(float x, float y, float z) { return {x, y, z}; }
__device__ __forceinline__ f3 operator+(f3 a, f3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ f3 operator-(f3 a, f3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ f3 operator*(f3 a, float s) { return {a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ float dot3(f3 a, f3 b) {
    return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z));
}
__device__ __forceinline__ f3 cross3(f3 a, f3 b) {
    return {fmaf(a.y, b.z, -a.z * b.y), fmaf(a.z, b.x, -a.x * b.z),
            fmaf(a.x, b.y, -a.y * b.x)};
}
__device__ __forceinline__ f3 fma3(f3 a, float s, f3 b) {  // a*s + b
    return {fmaf(a.x, s, b.x), fmaf(a.y, s, b.y), fmaf(a.z, s, b.z)};
}
__device__ __forceinline__ f3 normalize3(f3 a) {
    float inv = rsqrtf(dot3(a, a));
    return a * inv;
}

// --------------------------------------------------------------- Philox
// Philox4x32-10: ten rounds of (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2),
// hi(M0*c0) ^ c3 ^ k1, lo(M0*c0)), the key advanced by the Weyl increments
// between rounds. Counter = (block, photon, track id, event).
struct u4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ u4 philox10(uint32_t c0, uint32_t c1, uint32_t c2,
                                        uint32_t c3, uint32_t k0, uint32_t k1) {
    constexpr uint32_t kMulA = 0xD2511F53u, kMulB = 0xCD9E8D57u;
    constexpr uint32_t kWeylA = 0x9E3779B9u, kWeylB = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t hi_a = __umulhi(kMulA, c0), lo_a = kMulA * c0;
        uint32_t hi_b = __umulhi(kMulB, c2), lo_b = kMulB * c2;
        uint32_t n0 = hi_b ^ c1 ^ k0;
        uint32_t n2 = hi_a ^ c3 ^ k1;
        c0 = n0;
        c1 = lo_b;
        c2 = n2;
        c3 = lo_a;
        k0 += kWeylA;
        k1 += kWeylB;
    }
    return {c0, c1, c2, c3};
}

// 24-bit uniform in [0,1), exact in FP32.
__device__ __forceinline__ float u24f(uint32_t w) {
    return __uint2float_rn(w >> 8) * 5.9604644775390625e-8f;
}

// ------------------------------------------------------------ responses
// Wavelength response of Sec. 4.3, one IEEE FP32 operation at a time.
__device__ __forceinline__ float table_eval(const DevTable &t, float lam) {
    if (t.kind == RICH_TABLE_CONST) return t.p0;
    if (t.kind == RICH_TABLE_GAUSS) {
        float dl = __fsub_rn(lam, t.p1);
        float x = __fdiv_rn(dl, t.p2);
        float x2 = __fmul_rn(x, x);
        return __fmul_rn(t.p0, expf(-x2));
    }
    float q = __fdiv_rn(__fsub_rn(lam, t.p0), t.p1);
    float f = floorf(q);
    int b = f < 0.0f ? 0 : (f > (float)(t.nbins - 1) ? t.nbins - 1 : (int)f);
    return t.values[b];
}

// Frank-Tamm wavelength: inverse CDF of 1/lambda^2 on [l1, l2].
__device__ __forceinline__ float emit_lambda(float u, float inv1, float span) {
    return __fdiv_rn(1.0f, __fsub_rn(inv1, __fmul_rn(u, span)));
}

// Orthonormal basis (e1, e2) around the unit vector t (Duff et al., JCGT
// 6(1) 2017, branchless sign form).
__device__ __forceinline__ void basis_f(f3 t, f3 &e1, f3 &e2) {
    float s = copysignf(1.0f, t.z);
    float a = -1.0f / (s + t.z);
    float b = t.x * t.y * a;
    e1 = mk3(fmaf(s * t.x * t.x, a, 1.0f), s * b, -s * t.x);
    e2 = mk3(b, fmaf(t.y * t.y, a, s), -t.y);
}
__device__ __forceinline__ f3 reflect_f(f3 d, f3 n) {
    float k = -2.0f * dot3(d, n);
    return fma3(n, k, d);
}

}  // namespace rich
