// 3D-ACA over frequency (Sec. 4, Algorithm 1) for every block of the block
// cluster tree.
//
// Per block, with C^(0) = 0, k_1 = the first unique frequency:
//   H_l = ENTRY(., ., k_l) - C^(l-1)(., ., k_l)        residual face
//   (i_l, j_l) = argmax |H_l|                            pivot
//   f_l[k] = (ENTRY(i_l, j_l, k) - C^(l-1)(i_l, j_l, k)) / H_l[i_l, j_l]
//   stop when ||H_l||_F ||f_l|| <= eps ||C^(l)||_F  (the last term is dropped),
//   ||C^(l)||_F^2 = sum_{d,d'} <H_d, H_d'> <f_d, f_d'>   (eq. norm, FP64),
//   k_{l+1} = argmax |f_l[k]| over frequencies not selected yet.
// Near-field blocks (k_near_aca): dense faces from the precomputed near tensor,
// one CTA per block.  Far-field blocks (k_far_aca): every residual face is
// compressed by ACA with partial pivoting (row fibre at i*, column fibre at
// j*, FP64 norm recursion of the matrix analogue of eq. norm) from entries
// evaluated on the fly; the face is rebuilt to find the pivot and discarded
// (Sec. 4); the frequency tube at the pivot is evaluated with one warp per
// frequency.  Persistent CTAs take far blocks from an atomic work queue
// ordered by decreasing size.
#include <algorithm>
#include <type_traits>

#include "internal.h"
#include "kernels.h"
#include "pair.cuh"

namespace {

constexpr int kMaxNu = 256;

// sum_{c < cn} coef[c] * base[c][idx]: eight independent loads in flight
// per thread (the loop is memory-latency bound otherwise).
template <class T>
TD_D cx<T> coef_sum(const cx<T> *coef, const cx<T> *const *base, int cn, int idx) {
    cx<T> acc[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    int c = 0;
    for (; c + 8 <= cn; c += 8) {
        cx<T> b[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) b[q] = base[c + q][idx];
#pragma unroll
        for (int q = 0; q < 8; ++q) cfma(acc[q & 3], coef[c + q], b[q]);
    }
    for (; c < cn; ++c) cfma(acc[0], coef[c], base[c][idx]);
    return (acc[0] + acc[1]) + (acc[2] + acc[3]);
}
template <class T>
TD_D cx<T> apply_coef(cx<T> v, const cx<T> *coef, const cx<T> *const *base, int cn, int idx) {
    return v - coef_sum(coef, base, cn, idx);
}

// dst[t n + i] = src[t ld + i] for t < k, i < n, by the whole block; the
// index pair of an element is advanced incrementally (one division per thread).
template <class T>
TD_D void copy_cols(cx<T> *dst, const cx<T> *src, int64_t ld, int k, int n) {
    int t = threadIdx.x / n, i = threadIdx.x - (threadIdx.x / n) * n;
    const int dt = blockDim.x / n, di = blockDim.x - (blockDim.x / n) * n;
    for (int e = threadIdx.x; e < k * n; e += blockDim.x) {
        dst[e] = src[(int64_t)t * ld + i];
        t += dt;
        i += di;
        if (i >= n) {
            i -= n;
            ++t;
        }
    }
}

// h = sum_{t < kf} U[t * su + i] V[t * sv + j] with independent accumulators.
template <class T>
TD_D cx<T> lowrank_at(const cx<T> *U, int64_t su, const cx<T> *V, int64_t sv, int kf, int i, int j) {
    cx<T> acc[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    int t = 0;
    for (; t + 4 <= kf; t += 4) {
        cx<T> u[4], w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            u[q] = U[(t + q) * su + i];
            w[q] = V[(t + q) * sv + j];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) cfma(acc[q], u[q], w[q]);
    }
    for (; t < kf; ++t) cfma(acc[0], U[t * su + i], V[t * sv + j]);
    return (acc[0] + acc[1]) + (acc[2] + acc[3]);
}

// ============================================================================
// Near field
// ============================================================================
template <class T>
__global__ void __launch_bounds__(128) k_near_aca(NearArgs a, TensorOut o, AcaParams p,
                                                  cx<T> *scratch, int64_t sper) {
    using AM = typename AmOf<T>::type;
    __shared__ cx<T> s_fl[kMaxNu];
    __shared__ cx<T> s_hd[kMaxNu];
    __shared__ cx<T> s_fk[kMaxNu];
    __shared__ const cx<T> *s_base[kMaxNu];
    __shared__ int s_sel[kMaxNu];
    __shared__ c64 s_g[kMaxNu + 1], s_gf[kMaxNu + 1];  // <H_l, H_d>, <f_l, f_d> for d <= l
    __shared__ AM red[32];
    __shared__ long long s_off;
    __shared__ double s_normC2;
    __shared__ int s_stop, s_knext;
    const int Nu = a.nf;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nwarps = blockDim.x >> 5;
    cx<T> *H = scratch + (int64_t)blockIdx.x * sper;
    cx<T> *fib = (cx<T> *)o.fib;
    cx<T> *pool = (cx<T> *)o.face;
    for (int nb = blockIdx.x; nb < a.nnear; nb += gridDim.x) {
        const int b = a.near_ids[nb];
        const int *bl = a.blocks + 5 * b;
        const int nI = bl[1] - bl[0], nJ = bl[3] - bl[2];
        const int64_t nIJ = (int64_t)nI * nJ;
        const cx<T> *N = (const cx<T> *)a.near + a.noff[nb];
        const int64_t tb = (int64_t)b * Nu;
        for (int kk = tid; kk < Nu; kk += blockDim.x) s_sel[kk] = 0;
        if (tid == 0) s_normC2 = 0.0;
        __syncthreads();
        int l = 0, k = 0, r = -1;
        while (l < Nu) {
            AM am = {-1, 0x7fffffff};
            for (int d = tid; d < l; d += blockDim.x) {
                s_fk[d] = fib[(tb + d) * Nu + k];
                s_base[d] = pool + o.foff[tb + d];
            }
            __syncthreads();
            for (int64_t e = tid; e < nIJ; e += blockDim.x) {
                cx<T> h = apply_coef(N[k * nIJ + e], s_fk, s_base, l, (int)e);
                H[e] = h;
                const auto key = pivot_key(h);
                if (am_better(key, (int)e, am.v, am.i)) am = {key, (int)e};
            }
            am = block_argmax(am, red);
            if (!(am.v > 0)) {
                r = l;
                break;
            }
            const int ep = am.i;
            const cx<T> piv = H[ep];
            for (int d = tid; d < l; d += blockDim.x) s_hd[d] = pool[o.foff[tb + d] + ep];
            __syncthreads();
            for (int kk = tid; kk < Nu; kk += blockDim.x) {
                cx<T> v = N[kk * nIJ + ep];
                for (int d = 0; d < l; ++d) cfms(v, s_hd[d], fib[(tb + d) * Nu + kk]);
                s_fl[kk] = cdiv(v, piv);
            }
            __syncthreads();
            // eq. norm: <H_l, H_d> and <f_l, f_d> for d < l, ||H_l||^2 and
            // ||f_l||^2 at d = l; one warp per term, the recursion in FP64
            for (int d = wid; d <= l; d += nwarps) {
                const cx<T> *Hd = d < l ? pool + o.foff[tb + d] : H;
                DotAcc<T> ah, af;
                for (int64_t e = lane; e < nIJ; e += 32) ah.add(H[e], Hd[e]);
                for (int kk = lane; kk < Nu; kk += 32) af.add(s_fl[kk], d < l ? fib[(tb + d) * Nu + kk] : s_fl[kk]);
                const double hr = ah.warp_real(), hi = ah.warp_imag(), fr = af.warp_real(), fi = af.warp_imag();
                if (lane == 0) {
                    s_g[d] = {hr, hi};
                    s_gf[d] = {fr, fi};
                }
            }
            __syncthreads();
            if (tid == 0) {
                double cross = 0.0;
                for (int d = 0; d < l; ++d) cross += s_g[d].x * s_gf[d].x - s_g[d].y * s_gf[d].y;
                const double hl2 = s_g[l].x, fl2 = s_gf[l].x;
                s_normC2 += 2.0 * cross + hl2 * fl2;
                s_stop = hl2 * fl2 <= p.eps * p.eps * s_normC2;  // ||H_l|| ||f_l|| <= eps ||C||, squared
            }
            __syncthreads();
            if (s_stop) {
                r = l;
                break;
            }
            if (tid == 0) {
                unsigned long long off = atomicAdd(o.face_used, (unsigned long long)nIJ);
                if ((int64_t)(off + nIJ) > o.face_cap) {
                    atomicOr(o.dev_flags, TD_DEV_POOL_OVERFLOW);
                    s_off = -1;
                } else {
                    s_off = (long long)off;
                }
            }
            __syncthreads();
            const long long off = s_off;
            if (off < 0) {
                r = l;
                break;
            }
            for (int64_t e = tid; e < nIJ; e += blockDim.x) pool[off + e] = H[e];
            for (int kk = tid; kk < Nu; kk += blockDim.x) fib[(tb + l) * Nu + kk] = s_fl[kk];
            if (tid == 0) {
                o.kpiv[tb + l] = k;
                o.frank[tb + l] = -1;
                o.foff[tb + l] = off;
                s_sel[k] = 1;
            }
            __syncthreads();
            ++l;
            // next frequency: largest |f_l[k]| among those not selected yet
            if (wid == 0) {
                AM an = {-1, 0x7fffffff};
                for (int kk = lane; kk < Nu; kk += 32) {
                    if (s_sel[kk]) continue;
                    const auto key = pivot_key(s_fl[kk]);
                    if (am_better(key, kk, an.v, an.i)) an = {key, kk};
                }
                an = warp_argmax(an);
                if (lane == 0) s_knext = an.i == 0x7fffffff ? -1 : an.i;
            }
            __syncthreads();
            const int kn = s_knext;
            if (kn < 0) {
                r = l;
                break;
            }
            k = kn;
        }
        if (r < 0) r = l;
        if (tid == 0) o.rank[b] = r;
        __syncthreads();
    }
}

// ============================================================================
// Far field
// ============================================================================
// One point pair (a of the test triangle, b of the trial triangle); fibres and
// tubes are evaluated one entry per warp, the lanes splitting the point pairs.
TD_D c32 point_pair(const MeshDev &m, int op, int ti, int a, int tj, int b, int loc, float sr, float si) {
    const int oa = a * m.nt + ti, ob = b * m.nt + tj;
    const float4 xa = __ldg(&m.qp[2 * oa]), xla = __ldg(&m.qp[2 * oa + 1]);
    const float4 yb = __ldg(&m.qp[2 * ob]), ylb = __ldg(&m.qp[2 * ob + 1]);
    const float dx = (yb.x - xa.x) + (ylb.x - xla.x);
    const float dy = (yb.y - xa.y) + (ylb.y - xla.y);
    const float dz = (yb.z - xa.z) + (ylb.z - xla.z);
    const float r2 = dx * dx + dy * dy + dz * dz;
    const float rinv = rsqrtf(r2), r = r2 * rinv;
    const c32 e = expm_sr(sr, si, r);
    float w = xa.w * yb.w * rinv;
    if (op == TD_SLP) return {w * e.x, w * e.y};
    if (op == TD_DLP) {
        const float4 n = __ldg(&m.nrm4[tj]);  // (x - y).n_y, P1 hat of the trial vertex
        w *= bary7f(b, loc) * -(dx * n.x + dy * n.y + dz * n.z) * rinv * rinv;
    } else {
        const float4 n = __ldg(&m.nrm4[ti]);  // (y - x).n_x
        w *= (dx * n.x + dy * n.y + dz * n.z) * rinv * rinv;
    }
    const float pr = fmaf(sr, r, 1.0f), pi = si * r;
    return {w * (pr * e.x - pi * e.y), w * (pr * e.y + pi * e.x)};
}
TD_D c64 point_pair(const MeshDev &m, int op, int ti, int a, int tj, int b, int loc, double sr, double si) {
    const int oa = a * m.nt + ti, ob = b * m.nt + tj;
    double dx = m.qx[ob] - m.qx[oa], dy = m.qy[ob] - m.qy[oa], dz = m.qz[ob] - m.qz[oa];
    double r = sqrt(dx * dx + dy * dy + dz * dz);
    c64 e = expm_sr(sr, si, r);
    double w = m.qw[oa] * m.qw[ob] / r;
    if (op == TD_SLP) return {w * e.x, w * e.y};
    if (op == TD_DLP)
        w *= bary7d(b, loc) * -(dx * m.n64[tj] + dy * m.n64[m.nt + tj] + dz * m.n64[2 * m.nt + tj]) / (r * r);
    else
        w *= (dx * m.n64[ti] + dy * m.n64[m.nt + ti] + dz * m.n64[2 * m.nt + ti]) / (r * r);
    double pr = 1.0 + sr * r, pi = si * r;
    return {w * (pr * e.x - pi * e.y), w * (pr * e.y + pi * e.x)};
}

// Entry by a group of 8 lanes: lanes 0..6 of the group take test point a =
// lane % 8 against the 7 trial points (lane 7 adds nothing); the group sum
// reaches all 8 lanes.  Every lane of the warp must call it (the shuffles
// stay inside each group); valid = false contributes 0.
template <class T, int OP>
TD_D cx<T> group_entry(const MeshDev &m, int row, int col, T sr, T si, bool valid) {
    const int sub = threadIdx.x & 7;
    cx<T> acc = {0, 0};
    if (valid && sub < 7) {
        if (!TD_P1_TRIAL(OP)) {
            // independent point pairs in flight: 3 + 3 + 1
            cx<T> acc2 = {0, 0}, acc3 = {0, 0};
#pragma unroll 1
            for (int b = 0; b < 6; b += 3) {
                acc = acc + point_pair(m, OP, row, sub, col, b, 0, sr, si);
                acc2 = acc2 + point_pair(m, OP, row, sub, col, b + 1, 0, sr, si);
                acc3 = acc3 + point_pair(m, OP, row, sub, col, b + 2, 0, sr, si);
            }
            acc = acc + point_pair(m, OP, row, sub, col, 6, 0, sr, si) + (acc2 + acc3);
        } else {
            const int p1 = m.v2t_ptr[col + 1];
            for (int p = m.v2t_ptr[col]; p < p1; ++p) {
                const int tj = m.v2t[p], loc = m.v2t_loc[p];
                cx<T> acc2 = {0, 0}, acc3 = {0, 0};
#pragma unroll 1
                for (int b = 0; b < 6; b += 3) {
                    acc = acc + point_pair(m, OP, row, sub, tj, b, loc, sr, si);
                    acc2 = acc2 + point_pair(m, OP, row, sub, tj, b + 1, loc, sr, si);
                    acc3 = acc3 + point_pair(m, OP, row, sub, tj, b + 2, loc, sr, si);
                }
                acc = acc + point_pair(m, OP, row, sub, tj, 6, loc, sr, si) + (acc2 + acc3);
            }
        }
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    const T s = (T)(1.0 / TD_FOUR_PI);
    return cx<T>{acc.x * s, acc.y * s};
}

constexpr int kNCoef = 512;
// blocks up to kDenseS entries also keep the face under construction,
// S = sum_t u_t v_t^T, densely (its rank-1 updates cost |I||J| per ACA step,
// which pays off only for small blocks)
constexpr int kDenseS = 1600;
// Dense-face blocks keep the rebuilt faces H_d of their first terms in the
// CTA's scratch, packed with stride |I||J|: min(kDenseTerms, capacity / |I||J|)
// of them.  The residual fibres
// are then corrected by sum_d f_d[k] H_d[i*, :] (l loads per entry instead of
// one per earlier factor column, k_1 + ... + k_{l-1}), and eq. norm's
// <H_l, H_d> is one pass over the dense faces.  Blocks up to kCdMax entries
// form C(k) = sum_d f_d[k] H_d once per term instead (cheaper when the face
// ranks exceed about |I| / 5).
constexpr int kDenseTerms = 16;
constexpr int kCdMax = 16384;

// accumulation type of the inner products: FP32 in the mixed form
template <class T>
using AccT = T;

// Terms of Algorithm 1 whose Gram matrix <H_d, H_d'> a far-field CTA keeps
// (the norm of the frequency slice C^(l-1)(k_l) is formed from it).
constexpr int kGmax = 24;
// Rounding floor of the mixed form's FP32 residual faces, relative to the
// frequency slice they were subtracted from: the residual of term l is
// A(k_l) - C^(l-1)(k_l) minus the face's own terms, every one stored and
// summed in FP32 (unit roundoff 2^-24, a few hundred terms).  Face ACA steps
// below 2^-20 ||C^(l-1)(k_l)||_F are rounding noise, not residual.
constexpr double kFp32Floor = 9.5367431640625e-07;  // 2^-20

// Fixed shared state of one far-field CTA.
template <class T>
struct FarShared {
    typename AmOf<T>::type red[2][32];  // arg-max scratch, used alternately
    AccT<T> nrow[64], nu[64], nv[64];  // ACA norm terms per step (face rank <= 64)
    double normS2, normC2;
    AccT<T> red3[2][32][3];            // block sums of the dense path, used alternately
    int kstop, stop, knext;
    int idx;
    long long off;
    cx<T> piv;
    cx<T> coef[kNCoef];
    const cx<T> *base[kNCoef];
    cx<T> part[256];  // partial corrections of the thread groups (correct_fibre)
    AccT<T> gre[kGmax][kGmax], gim[kGmax][kGmax];  // <H_d, H_d'> of the block's kept terms
    double floor2;  // mixed form: (2^-20 ||C^(l-1)(k_l)||_F)^2, the face ACA's noise floor (0: none)
};

// Per-frequency arrays of one far-field CTA, carved from dynamic shared memory
// with Nu entries each (Nu + 1 for gf, 2 (Nu + 1) for gH).
template <class T>
struct FarFreq {
    cx<T> *fl, *hd;
    c64 *gf;          // <f_l, f_d> for d < l, |f_l|^2 at d = l
    AccT<T> *gH;      // <H_l, H_d> (re, im) for d <= l
    long long *foff;
    int *sel, *frank;
};

TD_HD size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }
template <class T>
TD_HD size_t far_freq_bytes(int Nu) {
    return align16(sizeof(cx<T>) * Nu) * 2 + align16(sizeof(c64) * (Nu + 1)) +
           align16(sizeof(AccT<T>) * 2 * (Nu + 1)) + align16(sizeof(long long) * Nu) + align16(sizeof(int) * Nu) * 2;
}
template <class T>
TD_D FarFreq<T> far_freq(unsigned char *p, int Nu) {
    FarFreq<T> F;
    F.fl = (cx<T> *)p;
    p += align16(sizeof(cx<T>) * Nu);
    F.hd = (cx<T> *)p;
    p += align16(sizeof(cx<T>) * Nu);
    F.gf = (c64 *)p;
    p += align16(sizeof(c64) * (Nu + 1));
    F.gH = (AccT<T> *)p;
    p += align16(sizeof(AccT<T>) * 2 * (Nu + 1));
    F.foff = (long long *)p;
    p += align16(sizeof(long long) * Nu);
    F.sel = (int *)p;
    p += align16(sizeof(int) * Nu);
    F.frank = (int *)p;
    return F;
}

// coefficient list for the residual of previous terms at a fixed row (mode 0:
// coef f_d[k] U_d[tau][i*], base V_d[tau]) or fixed column (mode 1: coef
// f_d[k] V_d[tau][j*], base U_d[tau]), followed by the current face's own
// terms (u_t[i*], base v_t) / (v_t[j*], base u_t).  Entries [c0, c0+kNCoef).
template <class T>
TD_D int build_coef(FarShared<T> &S, const FarFreq<T> &F, int mode, int fixed, int l, int kf, int k, int Nu,
                    int64_t tb, int nI, int nJ, const cx<T> *pool, const cx<T> *fib, const cx<T> *Uw,
                    const cx<T> *Vw, int maxI, int maxJ, int c0) {
    int total = kf;
    for (int d = 0; d < l; ++d) total += F.frank[d];
    const int cend = min(total, c0 + kNCoef);
    for (int c = c0 + threadIdx.x; c < cend; c += blockDim.x) {
        int rem = c, d = 0;
        while (d < l && rem >= F.frank[d]) {
            rem -= F.frank[d];
            ++d;
        }
        cx<T> cf;
        const cx<T> *bp;
        if (d < l) {
            const cx<T> *Ud = pool + F.foff[d];
            const cx<T> *Vd = Ud + (int64_t)F.frank[d] * nI;
            const cx<T> fk = fib[(tb + d) * Nu + k];
            if (mode == 0) {
                cf = fk * Ud[(int64_t)rem * nI + fixed];
                bp = Vd + (int64_t)rem * nJ;
            } else {
                cf = fk * Vd[(int64_t)rem * nJ + fixed];
                bp = Ud + (int64_t)rem * nI;
            }
        } else {
            if (mode == 0) {
                cf = Uw[(int64_t)rem * maxI + fixed];
                bp = Vw + (int64_t)rem * maxJ;
            } else {
                cf = Vw[(int64_t)rem * maxJ + fixed];
                bp = Uw + (int64_t)rem * maxI;
            }
        }
        S.coef[c - c0] = cf;
        S.base[c - c0] = bp;
    }
    return total;
}

// x[idx] -= sum_{c < cn} S.coef[c] * S.base[c][idx] for idx < n.  Short
// fibres (n < blockDim) split the coefficient list over G thread groups so
// that more loads are in flight, and combine the partial sums through
// shared memory.  Called by every thread of the block.
template <class T>
TD_D void correct_fibre(FarShared<T> &S, cx<T> *x, int n, int cn) {
    const int G = n >= (int)blockDim.x ? 1 : min(16, (int)blockDim.x / n);
    if (G == 1) {
        for (int j = threadIdx.x; j < n; j += blockDim.x) x[j] = x[j] - coef_sum(S.coef, S.base, cn, j);
        return;
    }
    const int per = (cn + G - 1) / G;
    for (int e = threadIdx.x; e < n * G; e += blockDim.x) {
        const int j = e % n, g = e / n, cb = min(cn, g * per), ce = min(cn, cb + per);
        S.part[e] = coef_sum(S.coef + cb, S.base + cb, ce - cb, j);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        cx<T> v = x[j];
        for (int g = 0; g < G; ++g) v = v - S.part[g * n + j];
        x[j] = v;
    }
}

// Block-wide arg-max with one barrier: warp maxima to `red`, then every
// thread reduces the warp maxima itself.  Successive calls must alternate
// between two `red` arrays (a call may start writing while slower threads
// still read the previous one).
template <class AM>
TD_D AM block_argmax_1sync(AM a, AM *red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    a = warp_argmax(a);
    if (lane == 0) red[wid] = a;
    __syncthreads();
    AM r = red[0];
    for (int w = 1; w < nw; ++w)
        if (am_better(red[w].v, red[w].i, r.v, r.i)) r = red[w];
    return r;
}

constexpr int kTI = 16;     // Gram tile width (rows of U / V per stage)
constexpr int kGCh = 32;    // Gram tile height (factor columns per stage)
constexpr int kGOut = 4;    // Gram outputs per thread

// Shared tiles for the Gram sums (dynamic shared memory).
template <class T>
struct GramTiles {
    cx<T> A[64][kTI + 1];      // current face: rows t < kf
    cx<T> B[kGCh][kTI + 1];    // factor columns of the previous terms (and of the face itself)
    const cx<T> *colU[kGCh];   // column descriptors of the current chunk
    const cx<T> *colV[kGCh];
    int colD[kGCh];
};

// Adds v to gH[2 d] (re) / gH[2 d + 1] (im); d < 0: nothing.  Lanes of a warp
// that all carry the same d are summed with shuffles first (the common case:
// the outputs of one warp mostly belong to one term).
template <class A>
TD_D void add_by_term(A *gH, int d, A re, A im) {
    const int d0 = __shfl_sync(0xffffffffu, d, 0);
    if (__all_sync(0xffffffffu, d == d0)) {
        re = warp_sum(re);
        im = warp_sum(im);
        if ((threadIdx.x & 31) == 0 && d0 >= 0) {
            atomicAdd(&gH[2 * d0], re);
            atomicAdd(&gH[2 * d0 + 1], im);
        }
    } else if (d >= 0) {
        atomicAdd(&gH[2 * d], re);
        atomicAdd(&gH[2 * d + 1], im);
    }
}

// eq. norm for the new term l: for every previous term d < l and for d = l,
// gH[d] += sum_{t < kf, tau < k_d} <u_t, U_d[tau]> <v_t, V_d[tau]>, where
// u_t, v_t are the face's ACA factors (Uw, Vw).  The inner products are
// small GEMMs over the rows of U and V, staged through shared-memory tiles;
// each thread owns up to kGOut (t, tau) outputs (t fastest, so that the
// outputs of a warp share a term).  gH must be zero on entry.
template <class T>
TD_D void gram_sums(const FarFreq<T> &F, GramTiles<T> &G, int l, int kf, int nI, int nJ, const cx<T> *pool,
                    const cx<T> *Uw, const cx<T> *Vw, int maxI, int maxJ) {
    using A = AccT<T>;
    const int tid = threadIdx.x;
    int Kprev = 0;
    for (int d = 0; d < l; ++d) Kprev += F.frank[d];
    const int Kall = Kprev + kf;
    const int chmax = max(1, min(kGCh, (kGOut * (int)blockDim.x) / max(kf, 1)));
    for (int g0 = 0; g0 < Kall; g0 += chmax) {
        const int ch = min(chmax, Kall - g0);
        __syncthreads();
        for (int c = tid; c < ch; c += blockDim.x) {
            int d = 0, rem = g0 + c;
            while (d < l && rem >= F.frank[d]) {
                rem -= F.frank[d];
                ++d;
            }
            if (d < l) {
                const cx<T> *Ud = pool + F.foff[d];
                G.colU[c] = Ud + (int64_t)rem * nI;
                G.colV[c] = Ud + (int64_t)F.frank[d] * nI + (int64_t)rem * nJ;
            } else {
                G.colU[c] = Uw + (int64_t)rem * maxI;
                G.colV[c] = Vw + (int64_t)rem * maxJ;
            }
            G.colD[c] = d;
        }
        DotAcc<T> au[kGOut], av[kGOut];
        for (int pass = 0; pass < 2; ++pass) {
            const int n = pass ? nJ : nI;
            const cx<T> *W = pass ? Vw : Uw;
            const int64_t sw = pass ? maxJ : maxI;
            for (int x0 = 0; x0 < n; x0 += kTI) {
                __syncthreads();
                for (int e = tid; e < kf * kTI; e += blockDim.x) {
                    const int t = e / kTI, xx = e % kTI;
                    G.A[t][xx] = x0 + xx < n ? W[t * sw + x0 + xx] : cx<T>{0, 0};
                }
                for (int e = tid; e < ch * kTI; e += blockDim.x) {
                    const int c = e / kTI, xx = e % kTI;
                    const cx<T> *col = pass ? G.colV[c] : G.colU[c];
                    G.B[c][xx] = x0 + xx < n ? col[x0 + xx] : cx<T>{0, 0};
                }
                __syncthreads();
#pragma unroll
                for (int q = 0; q < kGOut; ++q) {
                    const int o = tid + q * blockDim.x;
                    if (o < kf * ch) {
                        const int t = o % kf, c = o / kf;
                        DotAcc<T> &acc = pass ? av[q] : au[q];
#pragma unroll 4
                        for (int xx = 0; xx < kTI; ++xx) acc.add(G.A[t][xx], G.B[c][xx]);
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < kGOut; ++q) {
            const int o = tid + q * blockDim.x;
            const bool has = o < kf * ch;
            const int d = has ? G.colD[o / kf] : -1;
            const A pr = has ? au[q].re * av[q].re - au[q].im * av[q].im : A(0);
            const A pi = has ? au[q].re * av[q].im + au[q].im * av[q].re : A(0);
            add_by_term(F.gH, d, pr, pi);
        }
    }
    __syncthreads();
}

// Asynchronous 8-byte copy global -> shared (zero-filled when !valid; src
// must still be a valid address), commit and wait of copy groups.
TD_D void cp_async8(void *dst, const void *src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(valid ? 8 : 0) : "memory");
}
TD_D void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
TD_D void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Rebuild of a large face H = sum_{t<kf} u_t v_t^T with its arg-max (FP32
// form).  The face is swept in tiles of (NT/16)*4 rows x 64 columns; chunks
// of KC factor columns are staged in shared memory (the Gram tiles' space)
// in two stages, the next chunk's asynchronous copies in flight while the
// current one is multiplied; every thread accumulates a 4 x 4 register tile:
// rows 4*ty .. 4*ty+3 and columns tx, tx+16, tx+32, tx+48 (8 shared loads
// per 16 complex MACs, conflict-free).  Entries are summed over t in the
// same order as the plain rebuild.  Dense-face blocks also store the face to
// Sd.
template <int NT>
struct RebuildTile {
    static constexpr int TI = NT / 16 * 4, TJ = 64, KC = NT <= 128 ? 8 : 4;
};

template <int NT, class AM>
TD_D void rebuild_tiled(void *smem, const c32 *Uw, const c32 *Vw, int64_t maxI, int64_t maxJ, int kf, int nI, int nJ,
                        c32 *Sd, AM &am) {
    constexpr int TI = RebuildTile<NT>::TI, TJ = RebuildTile<NT>::TJ, KC = RebuildTile<NT>::KC;
    constexpr int SSTAGE = KC * (TI + TJ);  // complex values per stage: U chunk [KC][TI], V chunk [KC][TJ]
    c32 *base = reinterpret_cast<c32 *>(smem);
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    for (int i0 = 0; i0 < nI; i0 += TI) {
        for (int j0 = 0; j0 < nJ; j0 += TJ) {
            c32 h[4][4];
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) h[x][y] = c32{0.f, 0.f};
            auto stage = [&](int st, int t0) {
                c32 *u = base + st * SSTAGE, *v = u + KC * TI;
                for (int e = tid; e < KC * TI; e += NT) {
                    const int t = e / TI, x = e - t * TI;
                    const bool ok = t0 + t < kf && i0 + x < nI;
                    cp_async8(u + e, ok ? Uw + (int64_t)(t0 + t) * maxI + i0 + x : Uw, ok);
                }
                for (int e = tid; e < KC * TJ; e += NT) {
                    const int t = e / TJ, y = e - t * TJ;
                    const bool ok = t0 + t < kf && j0 + y < nJ;
                    cp_async8(v + e, ok ? Vw + (int64_t)(t0 + t) * maxJ + j0 + y : Vw, ok);
                }
                cp_async_commit();
            };
            __syncthreads();  // the shared space is free (caller, previous tile)
            if (kf > 0) stage(0, 0);  // (kf = 0: zero face, no copies in flight)
            int st = 0;
            for (int t0 = 0; t0 < kf; t0 += KC, st ^= 1) {
                if (t0 + KC < kf) {
                    stage(st ^ 1, t0 + KC);
                    cp_async_wait<1>();
                } else {
                    cp_async_wait<0>();
                }
                __syncthreads();
                const c32 *su = base + st * SSTAGE, *sv = su + KC * TI;
                const int kc = min(KC, kf - t0);
                for (int t = 0; t < kc; ++t) {
                    c32 u[4], v[4];
#pragma unroll
                    for (int x = 0; x < 4; ++x) u[x] = su[t * TI + 4 * ty + x];
#pragma unroll
                    for (int y = 0; y < 4; ++y) v[y] = sv[t * TJ + tx + 16 * y];
#pragma unroll
                    for (int x = 0; x < 4; ++x)
#pragma unroll
                        for (int y = 0; y < 4; ++y) cfma(h[x][y], u[x], v[y]);
                }
                __syncthreads();  // this stage is refilled two chunks later
            }
#pragma unroll
            for (int x = 0; x < 4; ++x) {
                const int i = i0 + 4 * ty + x;
#pragma unroll
                for (int y = 0; y < 4; ++y) {
                    const int j = j0 + tx + 16 * y;
                    if (i >= nI || j >= nJ) continue;
                    const int e = i * nJ + j;
                    if (Sd) Sd[e] = h[x][y];
                    const auto key = pivot_key(h[x][y]);
                    if (am_better(key, e, am.v, am.i)) am = {key, e};
                }
            }
        }
    }
}

// The tiled rebuild for FP32 faces whose tiles are at least half filled;
// returns false (nothing done) otherwise and in the FP64 form.
template <int NT, class T, class AM>
TD_D bool rebuild_tiled_fp32(void *smem, const cx<T> *Uw, const cx<T> *Vw, int64_t maxI, int64_t maxJ, int kf, int nI,
                             int nJ, cx<T> *Sd, AM &am) {
    if constexpr (std::is_same<T, float>::value) {
        constexpr int TI = RebuildTile<NT>::TI, TJ = RebuildTile<NT>::TJ;
        const int64_t padded = (int64_t)((nI + TI - 1) / TI) * TI * (((nJ + TJ - 1) / TJ) * TJ);
        if (2 * (int64_t)nI * nJ < padded) return false;
        rebuild_tiled<NT>(smem, Uw, Vw, maxI, maxJ, kf, nI, nJ, Sd, am);
        return true;
    } else {
        return false;
    }
}

// sum_{d < l} coef[d] H_d[e] over the dense faces (stride ds), eight
// independent loads in flight.
template <class T>
TD_D cx<T> dense_prev(const cx<T> *Hs, int64_t ds, const cx<T> *coef, int l, int64_t e) {
    cx<T> a4[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    int d = 0;
    for (; d + 8 <= l; d += 8) {
        cx<T> h[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) h[q] = Hs[(int64_t)(d + q) * ds + e];
#pragma unroll
        for (int q = 0; q < 8; ++q) cfma(a4[q & 3], coef[d + q], h[q]);
    }
    for (; d < l; ++d) cfma(a4[d & 3], coef[d], Hs[(int64_t)d * ds + e]);
    return (a4[0] + a4[1]) + (a4[2] + a4[3]);
}

// sum_{t < kf} X[t sx + fixed] Y[t sy + idx]: the current face's own terms at
// a fixed row (X = U, Y = V) or column (X = V, Y = U), eight independent
// pairs of loads in flight.
template <class T>
TD_D cx<T> own_sum(const cx<T> *X, int64_t sx, int fixed, const cx<T> *Y, int64_t sy, int idx, int kf) {
    cx<T> a4[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    int t = 0;
    for (; t + 8 <= kf; t += 8) {
        cx<T> xv[8], yv[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            xv[q] = X[(int64_t)(t + q) * sx + fixed];
            yv[q] = Y[(int64_t)(t + q) * sy + idx];
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) cfma(a4[q & 3], xv[q], yv[q]);
    }
    for (; t < kf; ++t) cfma(a4[t & 3], X[(int64_t)t * sx + fixed], Y[(int64_t)t * sy + idx]);
    return (a4[0] + a4[1]) + (a4[2] + a4[3]);
}

// sum_{i < n} x[i] conj(y[i]) over the lanes of a warp (each lane its part;
// the caller sums over the warp), four pairs of loads in flight per lane.
template <class T>
TD_D DotAcc<T> lane_dot(const cx<T> *x, const cx<T> *y, int n, int lane) {
    DotAcc<T> a, b;
    int i = lane;
    for (; i + 96 < n; i += 128) {
        cx<T> xv[4], yv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            xv[u] = x[i + 32 * u];
            yv[u] = y[i + 32 * u];
        }
        a.add(xv[0], yv[0]);
        b.add(xv[1], yv[1]);
        a.add(xv[2], yv[2]);
        b.add(xv[3], yv[3]);
    }
    for (; i < n; i += 32) a.add(x[i], y[i]);
    a.re += b.re;
    a.im += b.im;
    return a;
}

// eq. norm's <H_l, H_d> for every d <= l (< kDenseTerms) from the dense
// faces: each thread sums its entries for all terms at once, so that every
// face is read once; warp sums are added to gH (zero on entry).
template <class T>
TD_D void dense_grams(const cx<T> *Hs, int l, int64_t nIJ, AccT<T> *gH) {
    DotAcc<T> acc[kDenseTerms];
    const cx<T> *Hl = Hs + (int64_t)l * nIJ;
    const int64_t st = blockDim.x;
    // four entries per thread and pass: four loads in flight per face
    for (int64_t e0 = threadIdx.x; e0 < nIJ; e0 += 4 * st) {
        cx<T> h[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) h[u] = e0 + u * st < nIJ ? Hl[e0 + u * st] : cx<T>{0, 0};
#pragma unroll
        for (int d = 0; d < kDenseTerms; ++d) {
            if (d > l) break;
            cx<T> g[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) g[u] = e0 + u * st < nIJ ? Hs[(int64_t)d * nIJ + e0 + u * st] : cx<T>{0, 0};
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[d].add(h[u], g[u]);
        }
    }
#pragma unroll
    for (int d = 0; d < kDenseTerms; ++d) {
        if (d > l) break;
        const AccT<T> re = acc[d].warp_re(), im = acc[d].warp_im();
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&gH[2 * d], re);
            atomicAdd(&gH[2 * d + 1], im);
        }
    }
}

template <class T, int OP, int NT>
__global__ void __launch_bounds__(NT, 640 / NT) k_far_aca(MeshDev m, FarArgs a, TensorOut o, AcaParams p) {
    static_assert(sizeof(GramTiles<float>) >=
                      2 * RebuildTile<NT>::KC * (RebuildTile<NT>::TI + RebuildTile<NT>::TJ) * sizeof(c32),
                  "both rebuild stages must fit in the Gram tiles' shared memory");
    static_assert(sizeof(GramTiles<T>) >= kDenseS * sizeof(cx<T>), "S of a dense-S face must fit in the Gram tiles");
    using AM = typename AmOf<T>::type;
    using A = AccT<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FarShared<T> &S = *reinterpret_cast<FarShared<T> *>(smem_raw);
    size_t soff = align16(sizeof(FarShared<T>));
    GramTiles<T> *gt = reinterpret_cast<GramTiles<T> *>(smem_raw + soff);
    cx<T> *Ss = reinterpret_cast<cx<T> *>(gt);  // S of dense-S blocks (no Gram tiles needed there)
    soff += align16(sizeof(GramTiles<T>));
    const int Nu = a.nf;
    FarFreq<T> F = far_freq<T>(smem_raw + soff, Nu);
    soff += far_freq_bytes<T>(Nu);
    unsigned int *used = reinterpret_cast<unsigned int *>(smem_raw + soff);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nwarps = blockDim.x >> 5;
    cx<T> *Uw = (cx<T> *)a.scratch + (int64_t)blockIdx.x * a.scratch_per_cta;
    cx<T> *Vw = Uw + (int64_t)p.kcap * a.maxI;
    cx<T> *Hs = Vw + (int64_t)p.kcap * a.maxJ;  // rebuilt faces of dense-face blocks [dense_cap]
    cx<T> *Cd = Hs + a.dense_cap;                // C(k) of the current term [min(dense_cap, kCdMax)]
    const int64_t dcap = a.dense_cap;
    cx<T> *fib = (cx<T> *)o.fib;
    cx<T> *pool = (cx<T> *)o.face;
    long long ev_reg = 0, ev_tube = 0, ev_tests = 0;  // entries; synchronised ACA stopping tests
    for (;;) {
        if (tid == 0) S.idx = (int)atomicAdd(a.counter, 1u);
        __syncthreads();
        const int idx = S.idx;
        __syncthreads();
        const int nitems = a.harvest ? a.nfar * Nu : a.nfar;
        if (idx >= nitems) break;
        const int b = a.far_ids[a.harvest ? idx / Nu : idx];
        const int *bl = a.blocks + 5 * b;
        const int nI = bl[1] - bl[0], nJ = bl[3] - bl[2];
        const int *rows = a.perm_r + bl[0], *cols = a.perm_c + bl[2];
        const int64_t tb = (int64_t)b * Nu;
        const int64_t nIJb = (int64_t)nI * nJ;
        const int nd = (int)min((int64_t)kDenseTerms, dcap / max(nIJb, (int64_t)1));  // dense faces kept
        const bool dense_b = nd > 0;
        const bool cd_b = dense_b && nI * nJ <= kCdMax;         // and C(k) formed once per term
        const bool dense_sb = cd_b && nI * nJ <= kDenseS;       // and the face's own S kept densely
        for (int kk = tid; kk < Nu; kk += blockDim.x) F.sel[kk] = 0;
        if (tid == 0) S.normC2 = 0.0;
        __syncthreads();
        int l = 0, k = a.harvest ? idx % Nu : 0, r = -1;
        while (l < Nu) {
            const T sr = (T)a.sig[2 * k], si = (T)a.sig[2 * k + 1];
            // ------------------------------------------------ ACA of the residual face
            for (int w = tid; w < (nI + 31) / 32; w += blockDim.x) used[w] = 0u;
            // dense-path blocks: C(k) = sum_d f_d[k] H_d from the rebuilt faces, once per
            // term; dense-S blocks also start the face's own approximation S = 0 in shared
            // memory (the Gram tiles' space, unused by these blocks), copied to H_l at the end
            cx<T> *Sd = Hs + (int64_t)l * nIJb;
            // terms past kDenseTerms continue on the factors of the earlier terms
            const bool small = dense_b && l < nd, cdm = cd_b && small, dense_s = dense_sb && small;
            for (int t = tid; t < 64; t += blockDim.x) S.nrow[t] = A(0);
            if (small && !cdm)
                for (int d = tid; d < l; d += blockDim.x) S.coef[d] = fib[(tb + d) * Nu + k];
            if (cdm) {
                for (int e = tid; e < nI * nJ; e += blockDim.x) {
                    cx<T> acc = {0, 0};
                    for (int d = 0; d < l; ++d) cfma(acc, fib[(tb + d) * Nu + k], Hs[(int64_t)d * nIJb + e]);
                    Cd[e] = acc;
                    if (dense_s) Ss[e] = cx<T>{0, 0};
                }
            }
            __syncthreads();
            int kf = 0, istar = 0, par = 0;
            if (tid == 0) {
                S.normS2 = 0.0;
                // mixed form: ||C^(l-1)(k)||_F^2 = sum_{d,d'} f_d[k] conj(f_d'[k]) <H_d, H_d'>
                double c2 = 0.0;
                if (std::is_same<T, float>::value && l <= kGmax) {
                    for (int d = 0; d < l; ++d) {
                        const cx<T> fd = fib[(tb + d) * Nu + k];
                        for (int e = 0; e < l; ++e) {
                            const cx<T> fe = fib[(tb + e) * Nu + k];
                            // Re(fd conj(fe) G[d][e])
                            const double pr = (double)fd.x * fe.x + (double)fd.y * fe.y;
                            const double pi = (double)fd.y * fe.x - (double)fd.x * fe.y;
                            c2 += pr * S.gre[d][e] - pi * S.gim[d][e];
                        }
                    }
                }
                S.floor2 = kFp32Floor * kFp32Floor * fmax(c2, 0.0);
            }
            int pend0 = 0;  // first ACA step whose norm terms are not yet summed
            const int kp = (a.kpred && !a.harvest) ? min(a.kpred[tb + k], p.kcap) : 0;
            bool converged = false;
            int guard = 0;
            if (dense_s) {
                // ---- dense path: R = A(k) - C(k) - S, S = sum_t u_t v_t^T kept densely
                while (kf < p.kcap && guard < nI + p.kcap) {
                    ++guard;
                    // residual row fibre at i*: entry minus C and S, by the group leader
                    AM am = {-1, 0x7fffffff};
                    for (int j0 = wid * 4; j0 < nJ; j0 += nwarps * 4) {
                        const int j = j0 + (lane >> 3);
                        const cx<T> ent = group_entry<T, OP>(m, rows[istar], cols[min(j, nJ - 1)], sr, si, j < nJ);
                        if (j < nJ && (lane & 7) == 0) {
                            const int64_t e = (int64_t)istar * nJ + j;
                            const cx<T> v = ent - Cd[e] - Ss[e];
                            Vw[(int64_t)kf * a.maxJ + j] = v;
                            const auto key = pivot_key(v);
                            if (am_better(key, j, am.v, am.i)) am = {key, j};
                        }
                    }
                    ev_reg += nJ;
                    am = block_argmax_1sync(am, S.red[par]);
                    par ^= 1;
                    if (tid == 0) used[istar >> 5] |= 1u << (istar & 31);
                    if (!(am.v > 0)) {
                        // zero residual row: next unused row, if any
                        __syncthreads();
                        int nxt = -1;
                        for (int i = 0; i < nI; ++i)
                            if (!(used[i >> 5] & (1u << (i & 31)))) {
                                nxt = i;
                                break;
                            }
                        if (nxt < 0) {
                            converged = true;
                            break;
                        }
                        istar = nxt;
                        continue;
                    }
                    const int jstar = am.i;
                    const cx<T> piv = Vw[(int64_t)kf * a.maxJ + jstar];
                    // residual column fibre at j*, divided by the pivot
                    AM am2 = {-1, 0x7fffffff};
                    for (int i0 = wid * 4; i0 < nI; i0 += nwarps * 4) {
                        const int i = i0 + (lane >> 3);
                        const cx<T> ent = group_entry<T, OP>(m, rows[min(i, nI - 1)], cols[jstar], sr, si, i < nI);
                        if (i < nI && (lane & 7) == 0) {
                            const int64_t e = (int64_t)i * nJ + jstar;
                            const cx<T> u = cdiv(ent - Cd[e] - Ss[e], piv);
                            Uw[(int64_t)kf * a.maxI + i] = u;
                            if (i != istar && !(used[i >> 5] & (1u << (i & 31)))) {
                                const auto key = pivot_key(u);
                                if (am_better(key, i, am2.v, am2.i)) am2 = {key, i};
                            }
                        }
                    }
                    ev_reg += nI;
                    am2 = block_argmax_1sync(am2, S.red[par]);
                    par ^= 1;
                    // S += u v^T with ||S||_F^2, |u|^2 and |v|^2: FP32 partial and block sums,
                    // the stopping test in FP64 by each warp's first lane (no FP64 per element)
                    bool stop;
                    {
                        A s2 = 0, uu = 0, vv = 0;
                        const cx<T> *uk = Uw + (int64_t)kf * a.maxI, *vk = Vw + (int64_t)kf * a.maxJ;
                        // (i, j) of e advanced incrementally: no division per element
                        int ie = tid / nJ, je = tid - (tid / nJ) * nJ;
                        const int di = NT / nJ, dj = NT - (NT / nJ) * nJ;
                        for (int e = tid; e < nI * nJ; e += NT) {
                            cx<T> sv = Ss[e];
                            cfma(sv, uk[ie], vk[je]);
                            Ss[e] = sv;
                            s2 += cabs2(sv);
                            ie += di;
                            je += dj;
                            if (je >= nJ) {
                                je -= nJ;
                                ++ie;
                            }
                        }
                        for (int i = tid; i < nI; i += blockDim.x) uu += cabs2(uk[i]);
                        for (int j = tid; j < nJ; j += blockDim.x) vv += cabs2(vk[j]);
                        s2 = warp_sum(s2);
                        uu = warp_sum(uu);
                        vv = warp_sum(vv);
                        if (lane == 0) {
                            S.red3[par][wid][0] = s2;
                            S.red3[par][wid][1] = uu;
                            S.red3[par][wid][2] = vv;
                        }
                        __syncthreads();
                        int st = 0;
                        if (lane == 0) {
                            A t0 = 0, t1 = 0, t2 = 0;
                            for (int w = 0; w < nwarps; ++w) {
                                t0 += S.red3[par][w][0];
                                t1 += S.red3[par][w][1];
                                t2 += S.red3[par][w][2];
                            }
                            // squared test, no FP64 sqrt; the mixed form also stops at its rounding floor
                            st = (double)t1 * (double)t2 <= fmax(p.eps_aca * p.eps_aca * (double)t0, S.floor2);
                        }
                        stop = __shfl_sync(0xffffffffu, st, 0) != 0;
                    }
                    const bool have_next = !(am2.i == 0x7fffffff || am2.v < 0);
                    ++kf;
                    if (stop || !have_next) {
                        converged = true;
                        break;
                    }
                    istar = am2.i;
                }
            } else
            while (kf < p.kcap && guard < nI + p.kcap) {
                ++guard;
                // row fibre at istar: entries first (kept in Vw[kf]), then the
                // residual corrections in chunks
                AM am = {-1, 0x7fffffff};
                int total = 0;
                for (int j0 = wid * 4; j0 < nJ; j0 += nwarps * 4) {  // warp-uniform trip count
                    const int j = j0 + (lane >> 3);
                    const cx<T> v = group_entry<T, OP>(m, rows[istar], cols[min(j, nJ - 1)], sr, si, j < nJ);
                    if (j < nJ && (lane & 7) == 0) Vw[(int64_t)kf * a.maxJ + j] = v;
                }
                ev_reg += nJ;
                if (small) {
                    // previous terms from C(k); the face's own terms by each thread
                    // (u_t[i*] broadcast, v_t[j] coalesced), no coefficient list
                    __syncthreads();
                    for (int j = tid; j < nJ; j += blockDim.x) {
                        const int64_t ep = (int64_t)istar * nJ + j;
                        cx<T> v = Vw[(int64_t)kf * a.maxJ + j] - (cdm ? Cd[ep] : dense_prev(Hs, nIJb, S.coef, l, ep));
                        v = v - own_sum(Uw, (int64_t)a.maxI, istar, Vw, (int64_t)a.maxJ, j, kf);
                        Vw[(int64_t)kf * a.maxJ + j] = v;
                        const auto key = pivot_key(v);
                        if (am_better(key, j, am.v, am.i)) am = {key, j};
                    }
                } else {
                    for (int c0 = 0;; c0 += kNCoef) {
                        __syncthreads();
                        total = build_coef(S, F, 0, istar, l, kf, k, Nu, tb, nI, nJ, pool, fib, Uw, Vw, a.maxI, a.maxJ, c0);
                        __syncthreads();
                        correct_fibre(S, Vw + (int64_t)kf * a.maxJ, nJ, min(kNCoef, total - c0));
                        if (c0 + kNCoef >= total) break;
                    }
                    for (int j = tid; j < nJ; j += blockDim.x) {
                        const auto key = pivot_key(Vw[(int64_t)kf * a.maxJ + j]);
                        if (am_better(key, j, am.v, am.i)) am = {key, j};
                    }
                }
                am = block_argmax_1sync(am, S.red[par]);
                par ^= 1;
                if (tid == 0) used[istar >> 5] |= 1u << (istar & 31);
                __syncthreads();
                if (!(am.v > 0)) {
                    // zero residual row: next unused row, if any
                    int nxt = -1;
                    for (int i = 0; i < nI; ++i)
                        if (!(used[i >> 5] & (1u << (i & 31)))) {
                            nxt = i;
                            break;
                        }
                    if (nxt < 0) {
                        converged = true;
                        break;
                    }
                    istar = nxt;
                    continue;
                }
                const int jstar = am.i;
                const cx<T> piv = Vw[(int64_t)kf * a.maxJ + jstar];
                __syncthreads();
                for (int j = tid; j < nJ; j += blockDim.x) {
                    cx<T> v = Vw[(int64_t)kf * a.maxJ + j];
                    Vw[(int64_t)kf * a.maxJ + j] = cdiv(v, piv);
                }
                // column fibre at jstar
                for (int i0 = wid * 4; i0 < nI; i0 += nwarps * 4) {
                    const int i = i0 + (lane >> 3);
                    const cx<T> v = group_entry<T, OP>(m, rows[min(i, nI - 1)], cols[jstar], sr, si, i < nI);
                    if (i < nI && (lane & 7) == 0) Uw[(int64_t)kf * a.maxI + i] = v;
                }
                ev_reg += nI;
                if (!small) {
                    for (int c0 = 0;; c0 += kNCoef) {
                        __syncthreads();
                        total = build_coef(S, F, 1, jstar, l, kf, k, Nu, tb, nI, nJ, pool, fib, Uw, Vw, a.maxI, a.maxJ, c0);
                        __syncthreads();
                        correct_fibre(S, Uw + (int64_t)kf * a.maxI, nI, min(kNCoef, total - c0));
                        if (c0 + kNCoef >= total) break;
                    }
                }
                __syncthreads();
                AM am2 = {-1, 0x7fffffff};
                for (int i = tid; i < nI; i += blockDim.x) {
                    cx<T> u = Uw[(int64_t)kf * a.maxI + i];
                    if (small) {
                        // previous terms from C(k); the face's own terms by each thread
                        const int64_t ep = (int64_t)i * nJ + jstar;
                        u = u - (cdm ? Cd[ep] : dense_prev(Hs, nIJb, S.coef, l, ep));
                        u = u - own_sum(Vw, (int64_t)a.maxJ, jstar, Uw, (int64_t)a.maxI, i, kf);
                        Uw[(int64_t)kf * a.maxI + i] = u;
                    }
                    if (used[i >> 5] & (1u << (i & 31))) continue;
                    const auto key = pivot_key(u);
                    if (am_better(key, i, am2.v, am2.i)) am2 = {key, i};
                }
                am2 = block_argmax_1sync(am2, S.red[par]);
                par ^= 1;
                // Norm recursion of the ACA (matrix analogue of eq. norm, FP64):
                // ||S_k||^2 = ||S_{k-1}||^2 + 2 Re sum_{t<k} <u_k,u_t><v_k,v_t> + |u_k|^2 |v_k|^2.
                // Steps below the predicted rank kp run without the check; their
                // norms are formed in one batched pass when step kp - 1 is reached
                // and the first step that meets the criterion is taken, exactly as
                // if every step had been checked (the ACA steps themselves do not
                // depend on the check).
                const bool have_next = !(am2.i == 0x7fffffff || am2.v < 0);
                if (kf + 1 < kp && have_next) {
                    ++kf;
                    istar = am2.i;
                    continue;
                }
                for (int t = tid; t <= kf; t += blockDim.x) S.nrow[t] = A(0);
                ++ev_tests;
                __syncthreads();
                {
                    int npairs = 0;
                    for (int t = pend0; t <= kf; ++t) npairs += t + 1;
                    for (int pr = wid; pr < npairs; pr += nwarps) {
                        int t = pend0, rem = pr;
                        while (rem >= t + 1) {
                            rem -= t + 1;
                            ++t;
                        }
                        const int t2 = rem;
                        const DotAcc<T> au = lane_dot(Uw + (int64_t)t * a.maxI, Uw + (int64_t)t2 * a.maxI, nI, lane);
                        const DotAcc<T> av = lane_dot(Vw + (int64_t)t * a.maxJ, Vw + (int64_t)t2 * a.maxJ, nJ, lane);
                        const A ur = au.warp_re(), vr = av.warp_re();
                        if (t2 < t) {
                            const A ui = au.warp_im(), vi = av.warp_im();
                            if (lane == 0) atomicAdd(&S.nrow[t], ur * vr - ui * vi);
                        } else if (lane == 0) {
                            S.nu[t] = ur;
                            S.nv[t] = vr;
                        }
                    }
                }
                __syncthreads();
                if (tid == 0) {
                    double n2 = S.normS2;
                    int kstop = -1;
                    for (int t = pend0; t <= kf; ++t) {
                        const double uu = S.nu[t], vv = S.nv[t];
                        n2 += 2.0 * (double)S.nrow[t] + uu * vv;
                        if (uu * vv <= fmax(p.eps_aca * p.eps_aca * n2, S.floor2)) {
                            kstop = t;
                            break;
                        }
                    }
                    S.normS2 = n2;
                    S.kstop = kstop;
                }
                __syncthreads();
                if (S.kstop >= 0) {
                    kf = S.kstop + 1;
                    converged = true;
                    break;
                }
                ++kf;
                pend0 = kf;
                if (!have_next) {
                    converged = true;
                    break;
                }
                istar = am2.i;
            }
            if (!converged && tid == 0) atomicOr(o.dev_flags, TD_DEV_RANK_CAP);
            if (a.harvest) {  // face-rank harvest: record the ACA rank of the plain face and stop
                if (tid == 0) a.harvest[idx] = converged ? kf : kf + 1;
                r = 0;
                break;
            }
            // ------------------------------------------------ pivot on the rebuilt face
            AM am = {-1, 0x7fffffff};
            const int64_t nIJ = (int64_t)nI * nJ;
            if (dense_s) {
                // dense-S path: the rebuilt face is S itself (stored as H_l)
                for (int e = tid; e < (int)nIJ; e += blockDim.x) {
                    const cx<T> v = Ss[e];
                    Sd[e] = v;
                    const auto key = pivot_key(v);
                    if (am_better(key, e, am.v, am.i)) am = {key, e};
                }
            } else if (rebuild_tiled_fp32<NT>(gt, Uw, Vw, a.maxI, a.maxJ, kf, nI, nJ, small ? Sd : nullptr, am)) {
                // large face: tiled rebuild done
            } else {
                // H = sum_t u_t v_t^T in 2 x 4 register tiles (6 loads per 8 complex MACs);
                // dense-face blocks store it
                const int nIt = (nI + 1) >> 1, nJt = (nJ + 3) >> 2;
                for (int e4 = tid; e4 < nIt * nJt; e4 += blockDim.x) {
                    const int i0 = 2 * (e4 / nJt), j0 = 4 * (e4 - (e4 / nJt) * nJt);
                    const int ni = min(2, nI - i0), nj = min(4, nJ - j0);
                    cx<T> h[2][4];
#pragma unroll
                    for (int x = 0; x < 2; ++x)
#pragma unroll
                        for (int y = 0; y < 4; ++y) h[x][y] = cx<T>{0, 0};
                    for (int t = 0; t < kf; ++t) {
                        const cx<T> *ut = Uw + (int64_t)t * a.maxI + i0, *vt = Vw + (int64_t)t * a.maxJ + j0;
                        cx<T> u[2], v[4];
#pragma unroll
                        for (int x = 0; x < 2; ++x) u[x] = x < ni ? ut[x] : cx<T>{0, 0};
#pragma unroll
                        for (int y = 0; y < 4; ++y) v[y] = y < nj ? vt[y] : cx<T>{0, 0};
#pragma unroll
                        for (int x = 0; x < 2; ++x)
#pragma unroll
                            for (int y = 0; y < 4; ++y) cfma(h[x][y], u[x], v[y]);
                    }
#pragma unroll
                    for (int x = 0; x < 2; ++x)
#pragma unroll
                        for (int y = 0; y < 4; ++y) {
                            if (x >= ni || y >= nj) continue;
                            const int e = (i0 + x) * nJ + j0 + y;
                            if (small) Sd[e] = h[x][y];
                            const auto key = pivot_key(h[x][y]);
                            if (am_better(key, e, am.v, am.i)) am = {key, e};
                        }
                }
            }
            am = block_argmax(am, S.red[0]);
            if (!(am.v > 0) || kf == 0) {
                r = l;
                break;
            }
            const int ip = am.i / nJ, jp = am.i % nJ;
            if (tid == 0) {
                cx<T> h = {0, 0};
                if (small)
                    h = Sd[am.i];
                else
                    for (int t = 0; t < kf; ++t) cfma(h, Uw[(int64_t)t * a.maxI + ip], Vw[(int64_t)t * a.maxJ + jp]);
                S.piv = h;
            }
            // previous faces at the pivot
            for (int d = tid; d < l; d += blockDim.x) {
                if (small) {
                    F.hd[d] = Hs[(int64_t)d * nIJb + am.i];
                } else {
                    const cx<T> *Ud = pool + F.foff[d];
                    const cx<T> *Vd = Ud + (int64_t)F.frank[d] * nI;
                    F.hd[d] = lowrank_at(Ud, (int64_t)nI, Vd, (int64_t)nJ, F.frank[d], ip, jp);
                }
            }
            for (int d = tid; d <= l; d += blockDim.x) F.gH[2 * d] = F.gH[2 * d + 1] = A(0);
            __syncthreads();
            const cx<T> piv = S.piv;
            // tube over all unique frequencies, one warp per frequency
            for (int k0 = wid * 4; k0 < Nu; k0 += nwarps * 4) {
                const int kk = min(k0 + (lane >> 3), Nu - 1);
                cx<T> v = group_entry<T, OP>(m, rows[ip], cols[jp], (T)a.sig[2 * kk], (T)a.sig[2 * kk + 1],
                                             k0 + (lane >> 3) < Nu);
                if (k0 + (lane >> 3) < Nu && (lane & 7) == 0) {
                    for (int d = 0; d < l; ++d) cfms(v, F.hd[d], fib[(tb + d) * Nu + kk]);
                    F.fl[kk] = cdiv(v, piv);
                }
            }
            ev_tube += Nu;
            // eq. norm: <H_l, H_d> for d <= l; dense-face blocks from the dense faces
            // (one pass), others from the factors:
            // sum_{t,tau} <u_t, U_d[tau]> <v_t, V_d[tau]>
            if (small) {
                dense_grams(Hs, l, nIJ, F.gH);
                __syncthreads();
            } else {
                gram_sums(F, *gt, l, kf, nI, nJ, pool, Uw, Vw, a.maxI, a.maxJ);
            }
            // <f_l, f_d> (d < l) and |f_l|^2 (d = l), one warp per term
            for (int d = wid; d <= l; d += nwarps) {
                DotAcc<T> acc;
                for (int kk = lane; kk < Nu; kk += 32) acc.add(F.fl[kk], d < l ? fib[(tb + d) * Nu + kk] : F.fl[kk]);
                const double gr = acc.warp_real(), gi = acc.warp_imag();
                if (lane == 0) F.gf[d] = {gr, gi};
            }
            __syncthreads();
            if (tid == 0) {
                double cross = 0.0;
                for (int d = 0; d < l; ++d) cross += (double)F.gH[2 * d] * F.gf[d].x - (double)F.gH[2 * d + 1] * F.gf[d].y;
                const double hl2 = F.gH[2 * l], fl2 = F.gf[l].x;
                S.normC2 += 2.0 * cross + hl2 * fl2;
                S.stop = fabs(hl2) * fl2 <= p.eps * p.eps * S.normC2;  // ||H_l|| ||f_l|| <= eps ||C||, squared
            }
            __syncthreads();
            if (S.stop) {
                r = l;
                break;
            }
            // ------------------------------------------------ keep term l
            const int64_t need = (int64_t)kf * (nI + nJ);
            if (tid == 0) {
                unsigned long long off = atomicAdd(o.face_used, (unsigned long long)need);
                if ((int64_t)(off + need) > o.face_cap) {
                    // the block is recorded and redone once the pool has grown
                    atomicOr(o.dev_flags, a.redo ? TD_DEV_FAR_OVERFLOW : TD_DEV_POOL_OVERFLOW);
                    if (a.redo) a.redo[atomicAdd(a.redo_count, 1u)] = b;
                    S.off = -1;
                } else {
                    S.off = (long long)off;
                }
            }
            __syncthreads();
            const long long off = S.off;
            if (off < 0) {
                r = l;
                break;
            }
            copy_cols(pool + off, Uw, a.maxI, kf, nI);
            copy_cols(pool + off + (int64_t)kf * nI, Vw, a.maxJ, kf, nJ);
            for (int kk = tid; kk < Nu; kk += blockDim.x) fib[(tb + l) * Nu + kk] = F.fl[kk];
            if (l < kGmax)
                for (int d = tid; d <= l; d += blockDim.x) {
                    // <H_l, H_d> and <H_d, H_l> = conj
                    S.gre[l][d] = F.gH[2 * d];
                    S.gim[l][d] = F.gH[2 * d + 1];
                    S.gre[d][l] = F.gH[2 * d];
                    S.gim[d][l] = -F.gH[2 * d + 1];
                }
            if (tid == 0) {
                o.kpiv[tb + l] = k;
                o.frank[tb + l] = kf;
                o.foff[tb + l] = off;
                F.frank[l] = kf;
                F.foff[l] = off;
                F.sel[k] = 1;
            }
            __syncthreads();
            ++l;
            // next frequency: largest |f_l[k]| among those not selected yet
            if (wid == 0) {
                AM an = {-1, 0x7fffffff};
                for (int kk = lane; kk < Nu; kk += 32) {
                    if (F.sel[kk]) continue;
                    const auto key = pivot_key(F.fl[kk]);
                    if (am_better(key, kk, an.v, an.i)) an = {key, kk};
                }
                an = warp_argmax(an);
                if (lane == 0) S.knext = an.i == 0x7fffffff ? -1 : an.i;
            }
            __syncthreads();
            const int kn = S.knext;
            if (kn < 0) {
                r = l;
                break;
            }
            k = kn;
        }
        if (r < 0) r = l;
        if (tid == 0 && !a.harvest) o.rank[b] = r;
        __syncthreads();
    }
    if (tid == 0 && a.evals) {
        atomicAdd((unsigned long long *)&a.evals[0], (unsigned long long)ev_reg);
        atomicAdd((unsigned long long *)&a.evals[1], (unsigned long long)ev_tube);
        atomicAdd((unsigned long long *)&a.evals[2], (unsigned long long)ev_tests);
    }
}

}  // namespace

namespace {
// The far-field engine's entry evaluation on its own: out[f][r][c] =
// A[rows[r], cols[c]](sig_f) by group_entry, the 8-lane point-pair groups
// with which k_far_aca forms its row and column fibres and its frequency
// tubes (regular 7 x 7 rule, every pair; admissible blocks hold no touching
// pairs).  Four entries per warp; every lane of a warp takes the same number
// of trips, as group_entry's shuffles require.  An index out of range gives
// NaN without any table access.
template <class T, int OP>
__global__ void __launch_bounds__(128) k_fibre_entries(MeshDev m, const double *sig, const int *rows, int64_t nr,
                                                       const int *cols, int64_t nc, int64_t nf, cx<T> *out) {
    const int64_t n = nr * nc * nf;
    const int ncol_max = TD_P1_TRIAL(OP) ? m.nv : m.nt;
    const int64_t stride = ((int64_t)gridDim.x * blockDim.x) >> 3;
    for (int64_t base = ((int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31)) >> 3; base < n; base += stride) {
        const int64_t t = base + ((threadIdx.x & 31) >> 3);
        const int64_t tt = t < n ? t : 0;
        const int64_t c = tt % nc, r = (tt / nc) % nr, f = tt / (nc * nr);
        const int row = rows[r], col = cols[c];
        const bool ok = t < n && row >= 0 && row < m.nt && col >= 0 && col < ncol_max;
        const cx<T> v = group_entry<T, OP>(m, ok ? row : 0, ok ? col : 0, (T)sig[2 * f], (T)sig[2 * f + 1], ok);
        if (t < n && (threadIdx.x & 7) == 0) out[t] = ok ? v : cx<T>{(T)NAN, (T)NAN};
    }
}
}  // namespace

int td_launch_fibre_entries(cudaStream_t st, const MeshDev &m, int op, int prec, const double *sig, const int *rows,
                            int64_t nr, const int *cols, int64_t nc, int64_t nf, void *out, int num_sms) {
    const int64_t n = nr * nc * nf;
    if (n == 0) return 0;
    const int grid = (int)std::min<int64_t>((n + 15) / 16, (int64_t)num_sms * 16);
    if (prec == TDBEM_FP64) {
        if (op == TD_SLP) k_fibre_entries<double, TD_SLP><<<grid, 128, 0, st>>>(m, sig, rows, nr, cols, nc, nf, (c64 *)out);
        else if (op == TD_DLP) k_fibre_entries<double, TD_DLP><<<grid, 128, 0, st>>>(m, sig, rows, nr, cols, nc, nf, (c64 *)out);
        else k_fibre_entries<double, TD_ADLP><<<grid, 128, 0, st>>>(m, sig, rows, nr, cols, nc, nf, (c64 *)out);
    } else {
        if (op == TD_SLP) k_fibre_entries<float, TD_SLP><<<grid, 128, 0, st>>>(m, sig, rows, nr, cols, nc, nf, (c32 *)out);
        else if (op == TD_DLP) k_fibre_entries<float, TD_DLP><<<grid, 128, 0, st>>>(m, sig, rows, nr, cols, nc, nf, (c32 *)out);
        else k_fibre_entries<float, TD_ADLP><<<grid, 128, 0, st>>>(m, sig, rows, nr, cols, nc, nf, (c32 *)out);
    }
    return (int)cudaGetLastError();
}

int td_launch_near_aca(cudaStream_t st, int prec, const NearArgs &a, const TensorOut &o,
                       const AcaParams &p, void *scratch, int64_t sper, int nctas) {
    if (a.nnear == 0) return 0;
    if (prec == TDBEM_FP64)
        k_near_aca<double><<<nctas, 128, 0, st>>>(a, o, p, (c64 *)scratch, sper);
    else
        k_near_aca<float><<<nctas, 128, 0, st>>>(a, o, p, (c32 *)scratch, sper);
    return (int)cudaGetLastError();
}

template <class T, int OP, int NT>
static int launch_far_nt(cudaStream_t st, const MeshDev &m, const FarArgs &a, const TensorOut &o,
                         const AcaParams &p, int nctas) {
    const size_t sm = align16(sizeof(FarShared<T>)) + align16(sizeof(GramTiles<T>)) + far_freq_bytes<T>(a.nf) +
                      sizeof(unsigned int) * ((a.maxI + 31) / 32 + 1);
    cudaError_t e = cudaFuncSetAttribute(k_far_aca<T, OP, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return (int)e;
    k_far_aca<T, OP, NT><<<nctas, NT, sm, st>>>(m, a, o, p);
    return (int)cudaGetLastError();
}

template <class T, int OP>
static int launch_far(cudaStream_t st, const MeshDev &m, const FarArgs &a, const TensorOut &o,
                      const AcaParams &p, int nctas, int nt) {
    if (nt <= 64) return launch_far_nt<T, OP, 64>(st, m, a, o, p, nctas);
    if (nt <= 128) return launch_far_nt<T, OP, 128>(st, m, a, o, p, nctas);
    return launch_far_nt<T, OP, 256>(st, m, a, o, p, nctas);
}

int td_far_dense_terms() { return kDenseTerms; }
int td_far_cd_max() { return kCdMax; }

int td_launch_far_aca(cudaStream_t st, const MeshDev &m, int op, int prec, const FarArgs &a,
                      const TensorOut &o, const AcaParams &p, int nctas, int nt) {
    const int nitems = a.harvest ? a.nfar * a.nf : a.nfar;
    if (nitems == 0) return 0;
    if (prec == TDBEM_FP64)
        return op == TD_SLP   ? launch_far<double, TD_SLP>(st, m, a, o, p, nctas, nt)
               : op == TD_DLP ? launch_far<double, TD_DLP>(st, m, a, o, p, nctas, nt)
                              : launch_far<double, TD_ADLP>(st, m, a, o, p, nctas, nt);
    return op == TD_SLP   ? launch_far<float, TD_SLP>(st, m, a, o, p, nctas, nt)
           : op == TD_DLP ? launch_far<float, TD_DLP>(st, m, a, o, p, nctas, nt)
                          : launch_far<float, TD_ADLP>(st, m, a, o, p, nctas, nt);
}
