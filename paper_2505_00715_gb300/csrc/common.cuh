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
template <class AM>
TD_D AM warp_argmax(AM a) {
    for (int o = 16; o > 0; o >>= 1) {
        double ov = __shfl_xor_sync(0xffffffffu, (double)a.v, o);
        int oi = __shfl_xor_sync(0xffffffffu, a.i, o);
        if (am_better(ov, oi, a.v, a.i)) {
            a.v = (decltype(a.v))ov;
            a.i = oi;
        }
    }
    return a;
}

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

// Compensated ("twice the working precision") accumulation of products of
// FP32 numbers on the FP32 pipe: TwoProd by FMA and TwoSum (Ogita, Rump and
// Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. 2005).  The
// pair (s, c) represents s + c; the result is read out in FP64.  For FP64
// inputs the plain FP64 accumulation is used.
struct F2 {
    float s, c;
};
// (the _rn intrinsics keep the compiler from contracting these steps into FMAs)
TD_D void f2_fma(F2 &a, float x, float y) {
    const float p = __fmul_rn(x, y);
    const float e = fmaf(x, y, -p);
    const float s = __fadd_rn(a.s, p);
    const float z = __fsub_rn(s, a.s);
    const float err = __fadd_rn(__fsub_rn(a.s, __fsub_rn(s, z)), __fsub_rn(p, z));
    a.c = __fadd_rn(a.c, __fadd_rn(err, e));
    a.s = s;
}
// Warp sum of a compensated pair, combined with TwoSum in FP32; read out in FP64.
TD_D double warp_sum_f2(F2 v) {
    for (int o = 16; o > 0; o >>= 1) {
        const float s2 = __shfl_xor_sync(0xffffffffu, v.s, o), c2 = __shfl_xor_sync(0xffffffffu, v.c, o);
        const float s = __fadd_rn(v.s, s2);
        const float z = __fsub_rn(s, v.s);
        const float err = __fadd_rn(__fsub_rn(v.s, __fsub_rn(s, z)), __fsub_rn(s2, z));
        v.c = __fadd_rn(__fadd_rn(v.c, c2), err);
        v.s = s;
    }
    return (double)v.s + (double)v.c;
}

template <class T> struct DotAcc;
template <> struct DotAcc<float> {
    F2 re{0.f, 0.f}, im{0.f, 0.f};
    // += x * conj(y)
    TD_D void add(cx<float> x, cx<float> y) {
        f2_fma(re, x.x, y.x);
        f2_fma(re, x.y, y.y);
        f2_fma(im, x.y, y.x);
        f2_fma(im, -x.x, y.y);
    }
    TD_D double real() const { return (double)re.s + (double)re.c; }
    TD_D double imag() const { return (double)im.s + (double)im.c; }
    // sums over the 32 lanes of the warp (every lane gets the result)
    TD_D double warp_real() const { return warp_sum_f2(re); }
    TD_D double warp_imag() const { return warp_sum_f2(im); }
};
template <> struct DotAcc<double> {
    double re = 0.0, im = 0.0;
    TD_D void add(cx<double> x, cx<double> y) {
        re = fma(x.x, y.x, fma(x.y, y.y, re));
        im = fma(x.y, y.x, fma(-x.x, y.y, im));
    }
    TD_D double real() const { return re; }
    TD_D double imag() const { return im; }
    TD_D double warp_real() const { return warp_sum(re); }
    TD_D double warp_imag() const { return warp_sum(im); }
};

// Device-side error word: kernels record a code and keep going safely.
enum { TD_DEV_OK = 0, TD_DEV_POOL_OVERFLOW = 1, TD_DEV_BAD_INDEX = 2, TD_DEV_RANK_CAP = 4 };
