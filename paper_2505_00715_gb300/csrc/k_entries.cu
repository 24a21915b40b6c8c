// Entry kernels (Sec. 3; the ENTRY function of Algorithm 1):
//   k_entries_generic : arbitrary rows x cols x frequencies (C-ABI tdbem_entries)
//   (operators: single layer, double layer, adjoint double layer K')
//   k_sing_table      : touching pairs (Sauter-Schwab, FP64) at all unique
//                       frequencies, one warp per pair
//   k_near_entries    : every entry of every near-field block at all unique
//                       frequencies; regular pairs in the block precision with
//                       the quadrature geometry shared across frequencies,
//                       touching pairs read from the table.
#include "internal.h"
#include "kernels.h"
#include "pair.cuh"

namespace {

// ---- generic entries --------------------------------------------------------
// One entry A[row, col](sigma) (sigma = s/c), scaled by 1/(4 pi).
template <class T, int OP>
TD_D cx<T> entry_one(const MeshDev &m, int row, int col, double sr, double si) {
    using R = Reg<T>;
    typename R::Test X;
    load_test(m, row, X);
    cx<T> acc = {0, 0};
    c64 accs = {0.0, 0.0};
    if (!TD_P1_TRIAL(OP)) {
        if (touching_slot(m, row, col) >= 0) {
            c64 o[3] = {};
            pair_singular_f64<OP>(m, row, col, sr, si, o);
            accs = o[0];
        } else {
            cx<T> o[3] = {};
            R::template pair<OP>(X, m, col, (T)sr, (T)si, o);
            acc = o[0];
        }
    } else {
        for (int p = m.v2t_ptr[col]; p < m.v2t_ptr[col + 1]; ++p) {
            int e = m.v2t[p], l = m.v2t_loc[p];
            if (touching_slot(m, row, e) >= 0) {
                c64 o[3] = {};
                pair_singular_f64<TD_DLP>(m, row, e, sr, si, o);
                accs = accs + o[l];
            } else {
                cx<T> o[3] = {};
                R::template pair<TD_DLP>(X, m, e, (T)sr, (T)si, o);
                acc = acc + o[l];
            }
        }
    }
    const double inv4pi = 1.0 / TD_FOUR_PI;
    return cx<T>{(T)(((double)acc.x + accs.x) * inv4pi), (T)(((double)acc.y + accs.y) * inv4pi)};
}

template <class T, int OP>
__global__ void k_entries_generic(MeshDev m, const double *sig, int nq, const int *rows, int64_t nr,
                                  const int *cols, int64_t nc, const int *fidx, int64_t nf,
                                  cx<T> *out) {
    int64_t n = nr * nc * nf;
    const int ncols = TD_P1_TRIAL(OP) ? m.nv : m.nt;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t c = t % nc, r = (t / nc) % nr, f = t / (nc * nr);
        const int k = fidx[f], row = rows[r], col = cols[c];
        if (k < 0 || k >= nq || row < 0 || row >= m.nt || col < 0 || col >= ncols) {
            out[t] = cx<T>{(T)NAN, (T)NAN};  // invalid index: no access, NaN result
            continue;
        }
        out[t] = entry_one<T, OP>(m, row, col, sig[2 * k], sig[2 * k + 1]);
    }
}

// ---- touching-pair table ----------------------------------------------------
// table layout: [slot][nf][3] complex128 (SLP uses component 0), 1/(4 pi) applied.
template <int OP, int FC>
__global__ void k_sing_table(MeshDev m, const int *pti, const int *ptj, int npairs,
                             const double *sig, int nf, c64 *table) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int p = warp; p < npairs; p += nwarps) {
        int ti = pti[p], tj = ptj[p];
        if (OP == TD_SLP && ti > tj) {
            int t = ti;
            ti = tj;
            tj = t;
        }
        SingGeom G;
        classify_pair(m, ti, tj, G);
        const int nq = ss_npoints(G.cls, m.ng);
        const bool zero = (OP != TD_SLP && G.cls == 3) || G.cls == 0;
        for (int f0 = 0; f0 < nf; f0 += FC) {
            c64 acc[FC][3];
#pragma unroll
            for (int j = 0; j < FC; ++j)
                for (int k = 0; k < 3; ++k) acc[j][k] = {0.0, 0.0};
            if (!zero) {
                for (int q = lane; q < nq; q += 32) {
                    double d[3], w, lam[3];
                    ss_point(G, q, m.ng, m.gx, m.gw, d, w, lam);
                    double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                    double base, pre;
                    if (OP == TD_SLP) {
                        base = w / r;
                    } else {
                        base = w * ss_dn<OP>(G, d) / (r * r * r);
                    }
                    (void)pre;
#pragma unroll
                    for (int j = 0; j < FC; ++j) {
                        if (f0 + j < nf) {
                            double sr = sig[2 * (f0 + j)], si = sig[2 * (f0 + j) + 1];
                            c64 e = expm_sr(sr, si, r);
                            if (OP == TD_SLP) {
                                acc[j][0].x += base * e.x;
                                acc[j][0].y += base * e.y;
                            } else {
                                double pr = 1.0 + sr * r, pi = si * r;
                                c64 v = {base * (pr * e.x - pi * e.y), base * (pr * e.y + pi * e.x)};
                                if (OP == TD_ADLP) {
                                    acc[j][0].x += v.x;
                                    acc[j][0].y += v.y;
                                } else {
#pragma unroll
                                    for (int k = 0; k < 3; ++k) {
                                        acc[j][k].x += lam[k] * v.x;
                                        acc[j][k].y += lam[k] * v.y;
                                    }
                                }
                            }
                        }
                    }
                }
            }
            const double inv4pi = 1.0 / TD_FOUR_PI;
#pragma unroll
            for (int j = 0; j < FC; ++j) {
                c64 outv[3];
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    outv[k] = {warp_sum(acc[j][k].x) * inv4pi, warp_sum(acc[j][k].y) * inv4pi};
                if (lane == 0 && f0 + j < nf) {
                    c64 *o = table + ((int64_t)p * nf + f0 + j) * 3;
                    if (!TD_P1_TRIAL(OP)) {
                        o[0] = zero ? c64{0.0, 0.0} : outv[0];
                        o[1] = o[2] = {0.0, 0.0};
                    } else {
                        // parametrisation order -> mesh-local trial vertex
                        c64 z = {0.0, 0.0};
                        o[0] = o[1] = o[2] = z;
                        for (int k = 0; k < 3; ++k) o[G.loc[k]] = zero ? z : outv[k];
                    }
                }
            }
        }
    }
}

// Mixed form of the touching-pair table: the transformed coordinates, the
// Jacobian weights and the chunk sums in the table are FP64; the smooth
// factor e^{-sigma r} (SLP) or e^{-sigma r}(1 + sigma r) (DLP, ADLP) of
// every point and frequency runs on the FP32 special-function path
// (relative error about 3e-7), and each lane's partial sums over its points
// are FP32.  The points of a pair are taken in chunks of 32 P (P per lane,
// held in registers): the FP64 point geometry of a chunk is formed once and
// reused by every frequency, FC frequencies per pass; each pass's lane sums
// are reduced over the warp and added to the pair's table rows.
template <int OP, int FC>
__global__ void k_sing_table_mixed(MeshDev m, const int *pti, const int *ptj, int npairs, const double *sig,
                                   int nf, c64 *table) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    constexpr int NV = TD_P1_TRIAL(OP) ? 3 : 1;
    constexpr int P = TD_P1_TRIAL(OP) ? 8 : 16;  // points per lane and chunk
    // s / c of every frequency in shared memory (nf <= 256, checked by the caller)
    __shared__ float2 s_sig[256];
    for (int k = threadIdx.x; k < nf; k += blockDim.x) s_sig[k] = make_float2((float)sig[2 * k], (float)sig[2 * k + 1]);
    __syncthreads();
    const double inv4pi = 1.0 / TD_FOUR_PI;
    for (int p = warp; p < npairs; p += nwarps) {
        int ti = pti[p], tj = ptj[p];
        if (OP == TD_SLP && ti > tj) {
            int t = ti;
            ti = tj;
            tj = t;
        }
        SingGeom G;
        classify_pair(m, ti, tj, G);
        const int nq = ss_npoints(G.cls, m.ng);
        const bool zero = (OP != TD_SLP && G.cls == 3) || G.cls == 0;
        c64 *o = table + (int64_t)p * nf * 3;
        for (int e = lane; e < nf * 3; e += 32) o[e] = c64{0.0, 0.0};
        __syncwarp();
        if (zero) continue;
        for (int q0 = 0; q0 < nq; q0 += 32 * P) {
            // the transformed point and the difference x - y in FP64 (no
            // cancellation near the singularity); |d|^2 is exact to FP64
            // rounding, so the square root, the division and the rest run in
            // FP32 at FP32 relative accuracy
            float rf[P], bf[P], lf[P][NV];
#pragma unroll
            for (int i = 0; i < P; ++i) {
                const int q = q0 + 32 * i + lane;
                rf[i] = 1.0f;
                bf[i] = 0.0f;
#pragma unroll
                for (int k = 0; k < NV; ++k) lf[i][k] = 0.0f;
                if (q < nq) {
                    double d[3], w, lam[3];
                    ss_point(G, q, m.ng, m.gx, m.gw, d, w, lam);
                    const float r2 = (float)(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                    const float rinv = rsqrtf(r2);
                    rf[i] = r2 * rinv;
                    bf[i] = OP == TD_SLP ? (float)w * rinv : (float)w * (float)ss_dn<OP>(G, d) * rinv * rinv * rinv;
#pragma unroll
                    for (int k = 0; k < NV; ++k) lf[i][k] = TD_P1_TRIAL(OP) ? (float)lam[k] : 1.0f;
                }
            }
            for (int f0 = 0; f0 < nf; f0 += FC) {
                c32 acc[FC][NV];
#pragma unroll
                for (int j = 0; j < FC; ++j)
#pragma unroll
                    for (int k = 0; k < NV; ++k) acc[j][k] = {0.f, 0.f};
#pragma unroll
                for (int i = 0; i < P; ++i) {
#pragma unroll
                    for (int j = 0; j < FC; ++j) {
                        const float2 sgj = s_sig[min(f0 + j, nf - 1)];
                        const c32 e = expm_sr(sgj.x, sgj.y, rf[i]);
                        c32 v;
                        if (OP == TD_SLP) {
                            v = {bf[i] * e.x, bf[i] * e.y};
                        } else {
                            const float pr = fmaf(sgj.x, rf[i], 1.0f), pi = sgj.y * rf[i];
                            v = {bf[i] * (pr * e.x - pi * e.y), bf[i] * (pr * e.y + pi * e.x)};
                        }
#pragma unroll
                        for (int k = 0; k < NV; ++k) {
                            acc[j][k].x = fmaf(lf[i][k], v.x, acc[j][k].x);
                            acc[j][k].y = fmaf(lf[i][k], v.y, acc[j][k].y);
                        }
                    }
                }
                // lane sums over the warp in FP32, chunk sums into the FP64 table
#pragma unroll
                for (int j = 0; j < FC; ++j) {
#pragma unroll
                    for (int k = 0; k < NV; ++k) {
                        const float sx = warp_sum(acc[j][k].x), sy = warp_sum(acc[j][k].y);
                        if (lane == 0 && f0 + j < nf) {
                            c64 &t = o[(int64_t)(f0 + j) * 3 + (TD_P1_TRIAL(OP) ? G.loc[k] : 0)];
                            t.x += (double)sx * inv4pi;
                            t.y += (double)sy * inv4pi;
                        }
                    }
                }
            }
        }
    }
}

// ---- near-field dense entries -------------------------------------------------
// Regular pair at FC frequencies with the geometry computed once per point
// pair (test triangle in registers, trial points streamed from the tables).
template <int OP, int FC>
TD_D void pair_multi(const TestF &X, const MeshDev &m, int tj, const float *sg, int nfc, c32 *acc, int loc) {
    // signed kernel normal: -n_y (DLP) or +n_x (ADLP), multiplied by d = y - x
    float nx = 0.f, ny = 0.f, nz = 0.f;
    if (OP == TD_DLP) {
        nx = -m.n32[tj];
        ny = -m.n32[m.nt + tj];
        nz = -m.n32[2 * m.nt + tj];
    } else if (OP == TD_ADLP) {
        nx = X.nx;
        ny = X.ny;
        nz = X.nz;
    }
#pragma unroll 1
    for (int b = 0; b < 7; ++b) {
        const int ob = b * m.nt + tj;
        const float yxh = m.qxh[ob], yyh = m.qyh[ob], yzh = m.qzh[ob];
        const float yxl = m.qxl[ob], yyl = m.qyl[ob], yzl = m.qzl[ob];
        const float wyb = m.qw32[ob] * (OP == TD_DLP ? bary7f(b, loc) : 1.0f);
#pragma unroll
        for (int a = 0; a < 7; ++a) {
            const float dx = (yxh - X.xh[a]) + (yxl - X.xl[a]);
            const float dy = (yyh - X.yh[a]) + (yyl - X.yl[a]);
            const float dz = (yzh - X.zh[a]) + (yzl - X.zl[a]);
            const float r2 = dx * dx + dy * dy + dz * dz;
            const float rinv = rsqrtf(r2);
            const float r = r2 * rinv;
            float w = X.w[a] * wyb * rinv;
            if (OP != TD_SLP) w *= (dx * nx + dy * ny + dz * nz) * rinv * rinv;
#pragma unroll
            for (int j = 0; j < FC; ++j) {
                if (j < nfc) {
                    const float sr = sg[2 * j], si = sg[2 * j + 1];
                    const c32 e = expm_sr(sr, si, r);
                    if (OP == TD_SLP) {
                        acc[j].x = fmaf(w, e.x, acc[j].x);
                        acc[j].y = fmaf(w, e.y, acc[j].y);
                    } else {
                        const float pr = fmaf(sr, r, 1.0f), pi = si * r;
                        acc[j].x = fmaf(w, pr * e.x - pi * e.y, acc[j].x);
                        acc[j].y = fmaf(w, pr * e.y + pi * e.x, acc[j].y);
                    }
                }
            }
        }
    }
}

template <int OP, int FC>
TD_D void pair_multi(const TestD &X, const MeshDev &m, int tj, const double *sg, int nfc, c64 *acc, int loc) {
    double nx = 0.0, ny = 0.0, nz = 0.0;  // signed kernel normal, as in the FP32 version
    if (OP == TD_DLP) {
        nx = -m.n64[tj];
        ny = -m.n64[m.nt + tj];
        nz = -m.n64[2 * m.nt + tj];
    } else if (OP == TD_ADLP) {
        nx = X.nx;
        ny = X.ny;
        nz = X.nz;
    }
#pragma unroll 1
    for (int b = 0; b < 7; ++b) {
        const int ob = b * m.nt + tj;
        const double yx = m.qx[ob], yy = m.qy[ob], yz = m.qz[ob];
        const double wyb = m.qw[ob] * (OP == TD_DLP ? bary7d(b, loc) : 1.0);
#pragma unroll 1
        for (int a = 0; a < 7; ++a) {
            const double dx = yx - X.x[a], dy = yy - X.y[a], dz = yz - X.z[a];
            const double r = sqrt(dx * dx + dy * dy + dz * dz);
            double w = X.w[a] * wyb / r;
            if (OP != TD_SLP) w *= (dx * nx + dy * ny + dz * nz) / (r * r);
#pragma unroll
            for (int j = 0; j < FC; ++j) {
                if (j < nfc) {
                    const double sr = sg[2 * j], si = sg[2 * j + 1];
                    const c64 e = expm_sr(sr, si, r);
                    if (OP == TD_SLP) {
                        acc[j].x += w * e.x;
                        acc[j].y += w * e.y;
                    } else {
                        const double pr = 1.0 + sr * r, pi = si * r;
                        acc[j].x += w * (pr * e.x - pi * e.y);
                        acc[j].y += w * (pr * e.y + pi * e.x);
                    }
                }
            }
        }
    }
}

// near[noff[b] + (k * nI + i) * nJ + j] for every near block b (list nb_idx),
// all nf unique frequencies.  Entry e of the flattened list belongs to the
// near block found by binary search in the prefix `eprefix` (entries per block).
template <class T, int OP, int FC>
__global__ void __launch_bounds__(128) k_near_entries(MeshDev m, NearArgs a, const c64 *table) {
    __shared__ T sg[2 * 256];
    const int nf = a.nf;  // <= 256 (checked by the caller)
    for (int i = threadIdx.x; i < 2 * nf; i += blockDim.x) sg[i] = (T)a.sig[i];
    __syncthreads();
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < a.nentries;
         t += (int64_t)gridDim.x * blockDim.x) {
        // block lookup
        int lo = 0, hi = a.nnear - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (a.eprefix[mid] <= t) lo = mid; else hi = mid - 1;
        }
        const int nb = lo;
        const int32_t *bl = a.blocks + 5 * a.near_ids[nb];
        const int nI = bl[1] - bl[0], nJ = bl[3] - bl[2];
        const int64_t loc_e = t - a.eprefix[nb];
        const int i = (int)(loc_e / nJ), j = (int)(loc_e % nJ);
        const int row = a.perm_r[bl[0] + i], col = a.perm_c[bl[2] + j];
        cx<T> *dst = (cx<T> *)a.near + a.noff[nb] + (int64_t)i * nJ + j;
        const int64_t fstride = (int64_t)nI * nJ;
        typename Reg<T>::Test X;
        load_test(m, row, X);
        const int nsup = TD_P1_TRIAL(OP) ? m.v2t_ptr[col + 1] - m.v2t_ptr[col] : 1;
        for (int f0 = 0; f0 < nf; f0 += FC) {
            const int nfc = min(FC, nf - f0);
            cx<T> acc[FC];
#pragma unroll
            for (int jj = 0; jj < FC; ++jj) acc[jj] = {0, 0};
            c64 sing[FC];
#pragma unroll
            for (int jj = 0; jj < FC; ++jj) sing[jj] = {0.0, 0.0};
            for (int sidx = 0; sidx < nsup; ++sidx) {
                int e, l;
                if (!TD_P1_TRIAL(OP)) {
                    e = col;
                    l = 0;
                } else {
                    int p = m.v2t_ptr[col] + sidx;
                    e = m.v2t[p];
                    l = m.v2t_loc[p];
                }
                int slot = touching_slot(m, row, e);
                if (slot >= 0) {
#pragma unroll
                    for (int jj = 0; jj < FC; ++jj)
                        if (jj < nfc) sing[jj] = sing[jj] + table[((int64_t)slot * nf + f0 + jj) * 3 + l];
                } else {
                    pair_multi<OP, FC>(X, m, e, sg + 2 * f0, nfc, acc, l);
                }
            }
            const T inv4pi = (T)(1.0 / TD_FOUR_PI);
#pragma unroll
            for (int jj = 0; jj < FC; ++jj)
                if (jj < nfc)
                    dst[(int64_t)(f0 + jj) * fstride] =
                        cx<T>{(T)(acc[jj].x * inv4pi + (T)sing[jj].x), (T)(acc[jj].y * inv4pi + (T)sing[jj].y)};
        }
    }
}

}  // namespace

// ---- launchers ----------------------------------------------------------------
int td_launch_entries(cudaStream_t st, const MeshDev &m, int op, int prec, const double *sig, int nq,
                      const int *rows, int64_t nr, const int *cols, int64_t nc, const int *fidx,
                      int64_t nf, void *out) {
    int64_t n = nr * nc * nf;
    if (n == 0) return 0;
    int grid = (int)std::min<int64_t>((n + 127) / 128, 152 * 16);
    if (prec == TDBEM_FP64) {
        if (op == TD_SLP)
            k_entries_generic<double, TD_SLP><<<grid, 128, 0, st>>>(m, sig, nq, rows, nr, cols, nc, fidx, nf, (c64 *)out);
        else if (op == TD_DLP)
            k_entries_generic<double, TD_DLP><<<grid, 128, 0, st>>>(m, sig, nq, rows, nr, cols, nc, fidx, nf, (c64 *)out);
        else
            k_entries_generic<double, TD_ADLP><<<grid, 128, 0, st>>>(m, sig, nq, rows, nr, cols, nc, fidx, nf, (c64 *)out);
    } else {
        if (op == TD_SLP)
            k_entries_generic<float, TD_SLP><<<grid, 128, 0, st>>>(m, sig, nq, rows, nr, cols, nc, fidx, nf, (c32 *)out);
        else if (op == TD_DLP)
            k_entries_generic<float, TD_DLP><<<grid, 128, 0, st>>>(m, sig, nq, rows, nr, cols, nc, fidx, nf, (c32 *)out);
        else
            k_entries_generic<float, TD_ADLP><<<grid, 128, 0, st>>>(m, sig, nq, rows, nr, cols, nc, fidx, nf, (c32 *)out);
    }
    return (int)cudaGetLastError();
}

// Frequencies per pass of the mixed-form kernels, selected by the tuning
// variant (0 = default): touching-pair table (single layer / double layer /
// adjoint double layer: one value per pair and frequency like the single
// layer) and near-field tensor.
constexpr int kSingFcSlp[3] = {4, 8, 16};
constexpr int kSingFcDlp[3] = {2, 4, 8};
constexpr int kNearFc[3] = {8, 4, 16};
int td_sing_fc(int op, int variant) { return op == TD_DLP ? kSingFcDlp[variant % 3] : kSingFcSlp[variant % 3]; }
int td_near_fc(int variant) { return kNearFc[variant % 3]; }

int td_launch_sing_table(cudaStream_t st, const MeshDev &m, int op, int prec, const int *pti, const int *ptj,
                         int npairs, const double *sig, int nf, c64 *table, int num_sms, int variant) {
    if (npairs == 0) return 0;
    if (nf > 256) return (int)cudaErrorInvalidValue;  // the frequencies are staged in shared memory
    int grid = std::min((npairs + 3) / 4, num_sms * 8);
    if (prec == TDBEM_MIXED) {
        const int v = variant % 3;
        if (op == TD_SLP) {
            if (v == 1) k_sing_table_mixed<TD_SLP, 8><<<grid, 128, 0, st>>>(m, pti, ptj, npairs, sig, nf, table);
            else if (v == 2) k_sing_table_mixed<TD_SLP, 16><<<grid, 128, 0, st>>>(m, pti, ptj, npairs, sig, nf, table);
            else k_sing_table_mixed<TD_SLP, 4><<<grid, 128, 0, st>>>(m, pti, ptj, npairs, sig, nf, table);
        } else if (op == TD_DLP) {
            if (v == 1) k_sing_table_mixed<TD_DLP, 4><<<grid, 128, 0, st>>>(m, pti, ptj, npairs, sig, nf, table);
            else if (v == 2) k_sing_table_mixed<TD_DLP, 8><<<grid, 128, 0, st>>>(m, pti, ptj, npairs, sig, nf, table);
            else k_sing_table_mixed<TD_DLP, 2><<<grid, 128, 0, st>>>(m, pti, ptj, npairs, sig, nf, table);
        } else {
            if (v == 1) k_sing_table_mixed<TD_ADLP, 8><<<grid, 128, 0, st>>>(m, pti, ptj, npairs, sig, nf, table);
            else if (v == 2) k_sing_table_mixed<TD_ADLP, 16><<<grid, 128, 0, st>>>(m, pti, ptj, npairs, sig, nf, table);
            else k_sing_table_mixed<TD_ADLP, 4><<<grid, 128, 0, st>>>(m, pti, ptj, npairs, sig, nf, table);
        }
        return (int)cudaGetLastError();
    }
    if (op == TD_SLP)
        k_sing_table<TD_SLP, 8><<<grid, 128, 0, st>>>(m, pti, ptj, npairs, sig, nf, table);
    else if (op == TD_DLP)
        k_sing_table<TD_DLP, 4><<<grid, 128, 0, st>>>(m, pti, ptj, npairs, sig, nf, table);
    else
        k_sing_table<TD_ADLP, 4><<<grid, 128, 0, st>>>(m, pti, ptj, npairs, sig, nf, table);
    return (int)cudaGetLastError();
}

int td_launch_near_entries(cudaStream_t st, const MeshDev &m, int op, int prec, const NearArgs &a,
                           const c64 *table, int num_sms, int variant) {
    if (a.nentries == 0) return 0;
    int grid = (int)std::min<int64_t>((a.nentries + 127) / 128, (int64_t)num_sms * 16);
    if (prec == TDBEM_FP64) {
        if (op == TD_SLP) k_near_entries<double, TD_SLP, 4><<<grid, 128, 0, st>>>(m, a, table);
        else if (op == TD_DLP) k_near_entries<double, TD_DLP, 4><<<grid, 128, 0, st>>>(m, a, table);
        else k_near_entries<double, TD_ADLP, 4><<<grid, 128, 0, st>>>(m, a, table);
    } else {
        const int v = variant % 3;
        if (op == TD_SLP) {
            if (v == 1) k_near_entries<float, TD_SLP, 4><<<grid, 128, 0, st>>>(m, a, table);
            else if (v == 2) k_near_entries<float, TD_SLP, 16><<<grid, 128, 0, st>>>(m, a, table);
            else k_near_entries<float, TD_SLP, 8><<<grid, 128, 0, st>>>(m, a, table);
        } else if (op == TD_DLP) {
            if (v == 1) k_near_entries<float, TD_DLP, 4><<<grid, 128, 0, st>>>(m, a, table);
            else if (v == 2) k_near_entries<float, TD_DLP, 16><<<grid, 128, 0, st>>>(m, a, table);
            else k_near_entries<float, TD_DLP, 8><<<grid, 128, 0, st>>>(m, a, table);
        } else {
            if (v == 1) k_near_entries<float, TD_ADLP, 4><<<grid, 128, 0, st>>>(m, a, table);
            else if (v == 2) k_near_entries<float, TD_ADLP, 16><<<grid, 128, 0, st>>>(m, a, table);
            else k_near_entries<float, TD_ADLP, 8><<<grid, 128, 0, st>>>(m, a, table);
        }
    }
    return (int)cudaGetLastError();
}
