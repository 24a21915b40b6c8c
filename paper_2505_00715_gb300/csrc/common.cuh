// Device helpers shared by the tdbem kernels: complex arithmetic in FP32 and
// FP64, warp/block reductions, error flags.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define TD_HD __host__ __device__ __forceinline__
#define TD_D __device__ __forceinline__

template <class T>
struct cx {
    T x, y;
};
using c32 = cx<float>;
using c64 = cx<double>;

template <class T> TD_HD cx<T> mk(T a, T b) { return cx<T>{a, b}; }
template <class T> TD_HD cx<T> operator+(cx<T> a, cx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <class T> TD_HD cx<T> operator-(cx<T> a, cx<T> b) { return {a.x - b.x, a.y - b.y}; }
template <class T> TD_HD cx<T> operator*(cx<T> a, cx<T> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <class T> TD_HD cx<T> operator*(T s, cx<T> a) { return {s * a.x, s * a.y}; }
template <class T> TD_HD cx<T> cconj(cx<T> a) { return {a.x, -a.y}; }
template <class T> TD_HD T cabs2(cx<T> a) { return a.x * a.x + a.y * a.y; }
template <class T> TD_HD cx<T> cdiv(cx<T> a, cx<T> b) {
    T d = b.x * b.x + b.y * b.y;
    return {(a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d};
}
// a += b * c
template <class T> TD_HD void cfma(cx<T> &a, cx<T> b, cx<T> c) {
    a.x = fma(b.x, c.x, fma(-b.y, c.y, a.x));
    a.y = fma(b.x, c.y, fma(b.y, c.x, a.y));
}
// a -= b * c
template <class T> TD_HD void cfms(cx<T> &a, cx<T> b, cx<T> c) {
    a.x = fma(-b.x, c.x, fma(b.y, c.y, a.x));
    a.y = fma(-b.x, c.y, fma(-b.y, c.x, a.y));
}
template <class T, class U> TD_HD cx<T> ccast(cx<U> a) { return {(T)a.x, (T)a.y}; }

TD_D double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
TD_D float warp_sum(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// arg-max over (value, index) pairs: larger value wins, ties -> lower index.
struct ArgMax {
    float v;
    int i;
};
struct ArgMaxD {
    double v;
    int i;
};
TD_D bool am_better(double v, int i, double bv, int bi) { return v > bv || (v == bv && i < bi); }
TD_D bool am_better(float v, int i, float bv, int bi) { return v > bv || (v == bv && i < bi); }
template <class AM>
TD_D AM warp_argmax(AM a) {
    for (int o = 16; o > 0; o >>= 1) {
        const auto ov = __shfl_xor_sync(0xffffffffu, a.v, o);
        const int oi = __shfl_xor_sync(0xffffffffu, a.i, o);
        if (am_better(ov, oi, a.v, a.i)) {
            a.v = ov;
            a.i = oi;
        }
    }
    return a;
}

// Pivot key of a complex value: a strictly increasing function of |v|.  In
// FP32 it is |v| itself, formed without squaring (|v|^2 underflows for
// entries below ~1e-19 that are still representable); in FP64 |v|^2.
TD_D float pivot_key(cx<float> v) {
    const float a = fabsf(v.x), b = fabsf(v.y);
    const float hi = fmaxf(a, b), lo = fminf(a, b);
    if (!(hi > 0.f)) return 0.f;
    const float q = __fdividef(lo, hi);
    return hi * sqrtf(fmaf(q, q, 1.f));
}
TD_D double pivot_key(cx<double> v) { return v.x * v.x + v.y * v.y; }
template <class T> struct AmOf;
template <> struct AmOf<float> { using type = ArgMax; };
template <> struct AmOf<double> { using type = ArgMaxD; };

// Block-wide arg-max; `red` is shared scratch of >= 32 entries.  All threads
// receive the result.  Must be called by every thread of the block.
template <class AM>
TD_D AM block_argmax(AM a, AM *red) {
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    a = warp_argmax(a);
    __syncthreads();
    if (lane == 0) red[wid] = a;
    __syncthreads();
    if (wid == 0) {
        AM b = lane < nw ? red[lane] : AM{-1.0, 0x7fffffff};
        b = warp_argmax(b);
        if (lane == 0) red[0] = b;
    }
    __syncthreads();
    AM r = red[0];
    __syncthreads();
    return r;
}

// Block-wide sum of `n` doubles per thread (in place).  `red` >= 32*n doubles.
template <int N>
TD_D void block_sum(double *v, double *red) {
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = warp_sum(v[k]);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < N; ++k) red[k * 32 + wid] = v[k];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < N; ++k) {
            double x = lane < nw ? red[k * 32 + lane] : 0.0;
            x = warp_sum(x);
            if (lane == 0) red[k * 32] = x;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = red[k * 32];
    __syncthreads();
}

// Inner-product accumulator x * conj(y) in the working precision (FP32 in the
// mixed form, FP64 in the FP64 form).  The stopping decisions built on these
// sums are taken in FP64; an FP32 sum of n products carries a relative error
// of about n * 6e-8 of the sum of magnitudes, far below the tolerances
// (1e-4 / 1e-6) the norms are compared against.
template <class T> struct DotAcc {
    T re = 0, im = 0;
    // += x * conj(y)
    TD_D void add(cx<T> x, cx<T> y) {
        re = fma(x.x, y.x, fma(x.y, y.y, re));
        im = fma(x.y, y.x, fma(-x.x, y.y, im));
    }
    TD_D double real() const { return (double)re; }
    TD_D double imag() const { return (double)im; }
    // sums over the 32 lanes of the warp (every lane gets the result)
    TD_D T warp_re() const { return warp_sum(re); }
    TD_D T warp_im() const { return warp_sum(im); }
    TD_D double warp_real() const { return (double)warp_sum(re); }
    TD_D double warp_imag() const { return (double)warp_sum(im); }
};

// Device-side error word: kernels record a code and keep going safely.
enum { TD_DEV_OK = 0, TD_DEV_POOL_OVERFLOW = 1, TD_DEV_BAD_INDEX = 2, TD_DEV_RANK_CAP = 4, TD_DEV_TIMEOUT = 8,
       TD_DEV_FAR_OVERFLOW = 16 };
