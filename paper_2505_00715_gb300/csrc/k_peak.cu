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

// FP64 point pairs of the far field (single layer), the inner operation of
// the plain FP64 form: r = |y - x|, exp(-Re(sigma) r), sin and cos of
// Im(sigma) r, weight / r, complex accumulate.  4 independent chains per
// thread, the distance of each chain moving every step so that nothing is
// loop invariant: 4 * kPeakPairUnroll pairs per iteration.
constexpr int kPeakPairUnroll = 2;
__global__ void __launch_bounds__(kPeakThreads) k_peak_pair64(double *out, int iters) {
    double x[4], are[4], aim[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        x[c] = 0.05 + 1e-4 * (threadIdx.x + 64 * c);
        are[c] = aim[c] = 0.0;
    }
    const double sr = 3.7, si = 21.3, y = 0.3, z = 0.2, w = 1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kPeakPairUnroll; ++u)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const double r = sqrt(x[c] * x[c] + y * y + z * z);
                const double ea = exp(-sr * r);
                double sn, cs;
                sincos(si * r, &sn, &cs);
                const double wr = w / r;
                are[c] += wr * ea * cs;
                aim[c] -= wr * ea * sn;
                x[c] += 1e-7;
            }
    }
    double r = 0.0;
#pragma unroll
    for (int c = 0; c < 4; ++c) r += are[c] + aim[c];
    if (r == 12345.678) out[blockIdx.x] = r;
}

}  // namespace

// Launches one microbenchmark (what: 0 FP32 FMA, 1 SFU, 2 FP64 FMA, 3 FP64
// point pairs) on `grid` CTAs; returns the operations it performs (an FMA
// counts as one, a point pair as one).
int td_launch_peak(cudaStream_t st, int what, int grid, int iters, void *out, double *ops) {
    const double per_thread = what == 3 ? (double)iters * kPeakPairUnroll * 4 : (double)iters * kPeakUnroll * 8;
    *ops = per_thread * kPeakThreads * grid;
    if (what == 3)
        k_peak_pair64<<<grid, kPeakThreads, 0, st>>>((double *)out, iters);
    else if (what == 0)
        k_peak_fma32<<<grid, kPeakThreads, 0, st>>>((float *)out, iters);
    else if (what == 1)
        k_peak_sfu<<<grid, kPeakThreads, 0, st>>>((float *)out, iters);
    else
        k_peak_fma64<<<grid, kPeakThreads, 0, st>>>((double *)out, iters);
    return (int)cudaGetLastError();
}
