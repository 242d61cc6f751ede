// rich_peaks.cu -- throughput microbenchmarks of the units the photon trace
// uses: the FP32 fused multiply-add pipe, the FP32 min/max (ALU) pipe, the
// special-function (MUFU) unit and the L2 cache's read bandwidth. They are
// the denominators of the trace kernel's roofline: the rates a kernel can
// reach on this GPU at its current clocks, measured rather than derived from
// unit counts. Each kernel keeps every SM busy with independent chains (or,
// for L2, with 16-byte loads that bypass L1) and is timed with CUDA events on
// the caller's stream; the best of three runs is reported.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "rich_peaks.h"

namespace {

constexpr int kChains = 8;

// FP32 FMA: kChains independent dependent chains per thread.
__global__ void __launch_bounds__(256) k_peak_ffma(float *sink, int iters, float b, float c) {
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (float)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == 1.2345e-30f) sink[blockIdx.x] = s;     // keeps the chains live
}

// FP32 min/max: each step is one fmaxf and one fminf per chain, against
// bounds the compiler cannot see (two pairs, alternating).
__global__ void __launch_bounds__(256) k_peak_fmnmx(float *sink, int iters, float lo, float hi,
                                                    float lo2, float hi2) {
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (float)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int k = 0; k < kChains; ++k)
                a[k] = (u & 1) ? fminf(fmaxf(a[k], lo2), hi2) : fminf(fmaxf(a[k], lo), hi);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == 1.2345e-30f) sink[blockIdx.x] = s;
}

// MUFU: approximate reciprocal chains, each reciprocal fed through an FMA
// with runtime operands so that no two reciprocals can be folded; the FMA
// pipe runs 8x faster than the special-function unit, so the unit binds.
__global__ void __launch_bounds__(256) k_peak_mufu(float *sink, int iters, float b, float c) {
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1.0f + (float)(threadIdx.x + k) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) {
                float x = fmaf(a[k], b, c);
                asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(a[k]) : "f"(x));
            }
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == 1.2345e-30f) sink[blockIdx.x] = s;
}

// L2 read bandwidth: every thread streams 16-byte loads cached in L2 only
// (ld.global.cg) over a buffer that fits in L2, `reps` times.
__global__ void __launch_bounds__(512) k_peak_l2(const float4 *buf, long long n4, int reps,
                                                 float *sink) {
    float acc = 0.f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (int r = 0; r < reps; ++r) {
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
            float4 v;
            asm volatile("ld.global.cg.v4.f32 {%0, %1, %2, %3}, [%4];"
                         : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                         : "l"(buf + i));
            acc += v.x + v.y + v.z + v.w;
        }
    }
    if (acc == 1.2345e-30f) sink[blockIdx.x] = acc;
}

thread_local std::string g_err;

template <typename F>
bool best_ms(cudaStream_t s, F launch, float &best) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return false;
    launch();                                   // warm-up
    best = 1e30f;
    bool ok = true;
    for (int rep = 0; rep < 3 && ok; ++rep) {
        ok = cudaEventRecord(a, s) == cudaSuccess;
        launch();
        ok = ok && cudaEventRecord(b, s) == cudaSuccess && cudaEventSynchronize(b) == cudaSuccess;
        float ms = 0.f;
        ok = ok && cudaEventElapsedTime(&ms, a, b) == cudaSuccess;
        if (ok) best = std::min(best, ms);
    }
    ok = ok && cudaGetLastError() == cudaSuccess;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ok;
}

}  // namespace

extern "C" RICH_PEAKS_API int rich_measure_peaks(int device, void *stream, rich_peaks *out) {
    if (!out) return 1;
    *out = rich_peaks{};
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) {
        g_err = "rich_measure_peaks: cudaSetDevice failed";
        return 2;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int n_sm = 0;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device);
    float *sink = nullptr;
    float4 *buf = nullptr;
    const long long l2_bytes = 48ll << 20;       // within the 126 MB L2
    int rc = 0;
    if (cudaMalloc(&sink, 1 << 20) != cudaSuccess ||
        cudaMalloc(&buf, (size_t)l2_bytes) != cudaSuccess ||
        cudaMemsetAsync(buf, 0, (size_t)l2_bytes, s) != cudaSuccess) {
        g_err = "rich_measure_peaks: allocation failed";
        rc = 3;
    }
    if (!rc) {
        // 8 blocks of 256 threads per SM: 64 warps, every scheduler full
        const int blocks = n_sm * 8, threads = 256, iters = 4096;
        const double lanes = (double)blocks * threads * iters * 16 * kChains;
        float ms = 0.f;
        bool ok = best_ms(s, [&] { k_peak_ffma<<<blocks, threads, 0, s>>>(sink, iters, 1.0000001f, 1e-7f); }, ms);
        out->fp32_fma_flops = ok ? 2.0 * lanes / (ms * 1e-3) : 0.0;
        ok = ok && best_ms(s, [&] { k_peak_fmnmx<<<blocks, threads, 0, s>>>(sink, iters, -1e30f, 1e30f, -2e30f, 2e30f); }, ms);
        out->fp32_minmax_ops = ok ? 2.0 * lanes / (ms * 1e-3) : 0.0;
        const int mufu_iters = 512;
        const double mufu_lanes = (double)blocks * threads * mufu_iters * 16 * kChains;
        ok = ok && best_ms(s, [&] { k_peak_mufu<<<blocks, threads, 0, s>>>(sink, mufu_iters, 1.0000001f, 1e-7f); }, ms);
        out->mufu_ops = ok ? mufu_lanes / (ms * 1e-3) : 0.0;
        const int reps = 20;
        ok = ok && best_ms(s, [&] {
            k_peak_l2<<<n_sm * 4, 512, 0, s>>>(buf, l2_bytes / 16, reps, sink);
        }, ms);
        out->l2_read_bytes = ok ? (double)l2_bytes * reps / (ms * 1e-3) : 0.0;
        out->n_sm = n_sm;
        int clk_khz = 0;
        cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, device);
        out->sm_clock_mhz_max = clk_khz / 1000.0;
        if (!ok) {
            g_err = std::string("rich_measure_peaks: ") + cudaGetErrorString(cudaGetLastError());
            rc = 2;
        }
    }
    if (buf) cudaFree(buf);
    if (sink) cudaFree(sink);
    cudaSetDevice(prev);
    return rc;
}

extern "C" RICH_PEAKS_API const char *rich_peaks_last_error(void) { return g_err.c_str(); }
