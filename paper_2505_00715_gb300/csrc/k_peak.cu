// Throughput microbenchmarks of the pipes the compression runs on, the
// denominators of its roofline: FP32 fused multiply-add, the special-
// function unit (the four operations of a far-field point pair: reciprocal
// square root, base-2 exponential, sine and cosine) and FP64 fused
// multiply-add.  Every thread runs independent dependency chains long
// enough to hide the pipe latency; the grid fills every SM.
#include "internal.h"
#include "kernels.h"

namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakUnroll = 16;

TD_D float ex2_approx(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 8 independent FMA chains per thread: 8 * kPeakUnroll FMAs per iteration
__global__ void __launch_bounds__(kPeakThreads) k_peak_fma32(float *out, int iters) {
    float a[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) a[c] = 1.0f + 1e-3f * (threadIdx.x + c);
    const float m = 0.999999f, s = 1e-7f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kPeakUnroll; ++u)
#pragma unroll
            for (int c = 0; c < 8; ++c) a[c] = fmaf(a[c], m, s);
    }
    float r = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) r += a[c];
    if (r == 12345.678f) out[blockIdx.x] = r;  // keeps the chains live
}

// 8 independent chains per thread, two of each operation (the sine and
// cosine chains converge, rsqrt(rsqrt(x)) -> 1, x -> 2^-x -> 0.64):
// 8 * kPeakUnroll special-function operations per iteration
__global__ void __launch_bounds__(kPeakThreads) k_peak_sfu(float *out, int iters) {
    float a0 = 0.3f + 1e-4f * threadIdx.x, a1 = a0 + 0.1f;
    float b0 = a0 + 0.2f, b1 = a0 + 0.3f;
    float c0 = a0 + 1.0f, c1 = a0 + 2.0f;
    float d0 = a0, d1 = a0 + 0.5f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kPeakUnroll; ++u) {
            a0 = __sinf(a0);
            a1 = __sinf(a1);
            b0 = __cosf(b0);
            b1 = __cosf(b1);
            c0 = rsqrtf(c0);
            c1 = rsqrtf(c1);
            d0 = ex2_approx(-d0);
            d1 = ex2_approx(-d1);
        }
    }
    const float r = a0 + a1 + b0 + b1 + c0 + c1 + d0 + d1;
    if (r == 12345.678f) out[blockIdx.x] = r;
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_fma64(double *out, int iters) {
    double a[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) a[c] = 1.0 + 1e-3 * (threadIdx.x + c);
    const double m = 0.999999999, s = 1e-12;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kPeakUnroll; ++u)
#pragma unroll
            for (int c = 0; c < 8; ++c) a[c] = fma(a[c], m, s);
    }
    double r = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c) r += a[c];
    if (r == 12345.678) out[blockIdx.x] = r;
}

}  // namespace

// Launches one microbenchmark (what: 0 FP32 FMA, 1 SFU, 2 FP64 FMA) on
// `grid` CTAs; returns the operations it performs (an FMA counts as one).
int td_launch_peak(cudaStream_t st, int what, int grid, int iters, void *out, double *ops) {
    const double per_thread = (double)iters * kPeakUnroll * 8;
    *ops = per_thread * kPeakThreads * grid;
    if (what == 0)
        k_peak_fma32<<<grid, kPeakThreads, 0, st>>>((float *)out, iters);
    else if (what == 1)
        k_peak_sfu<<<grid, kPeakThreads, 0, st>>>((float *)out, iters);
    else
        k_peak_fma64<<<grid, kPeakThreads, 0, st>>>((double *)out, iters);
    return (int)cudaGetLastError();
}
