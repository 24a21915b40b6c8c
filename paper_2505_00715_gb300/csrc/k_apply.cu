// Compressed multi-frequency apply (eq. product):
//   y = sum_{l < NQ} A(s_l) W_l = sum_b sum_d [ H_d z1_d + conj(H_d) z2_d ]_I,
//   z1_d = sum_{l: s_l = s_u}       f_d[u] W_l[J],
//   z2_d = sum_{l: s_l = conj(s_u)} conj(f_d[u]) W_l[J],
// using A(conj s) = conj A(s) for the conjugate half of the frequency set.
// Far faces H_d = U_d V_d^T are applied as U_d (V_d^T z1) + conj(U_d) (V_d^H z2).
// One CTA per block: the block's W columns are streamed tile by tile (TJ
// columns, all NQ frequencies) through shared memory, the frequency
// contraction of every term is done on the tile, then contracted with the
// face (near) or V (far); results are added to y with atomics.
#include "internal.h"
#include "kernels.h"

namespace {

template <class T>
TD_D void atomic_add_c(cx<T> *p, cx<T> v) {
    atomicAdd(&p->x, v.x);
    atomicAdd(&p->y, v.y);
}

// dynamic shared memory layout (complex T units):
//   Wt [NQ][TJ][nrhs] | z [RC][2][TJ][nrhs] | acc: near [nI][nrhs] or far [sumk][2][nrhs]
template <class T>
__global__ void __launch_bounds__(256) k_apply(ApplyArgs a, TensorOut o, int TJ, int RC) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T> *sm = reinterpret_cast<cx<T> *>(smem_raw);
    const int NQ = a.single_f >= 0 ? 1 : a.NQ;
    const int nrhs = a.nrhs, Nu = a.Nu;
    const cx<T> *W = (const cx<T> *)a.W;
    cx<T> *y = (cx<T> *)a.y;
    const cx<T> *fib = (const cx<T> *)o.fib;
    const cx<T> *pool = (const cx<T> *)o.face;
    cx<T> *Wt = sm;
    cx<T> *z = Wt + (int64_t)NQ * TJ * nrhs;
    cx<T> *acc = z + (int64_t)RC * 2 * TJ * nrhs;
    cx<T> *fq_s = acc + a.acc_max;                                   // [RC][NQ]
    int *sg_s = reinterpret_cast<int *>(fq_s + (int64_t)RC * NQ);    // [NQ]
    const int tid = threadIdx.x;
    for (int b = blockIdx.x; b < a.nb; b += gridDim.x) {
        const int *bl = a.blocks + 5 * b;
        const int nI = bl[1] - bl[0], nJ = bl[3] - bl[2];
        const bool far = bl[4] != 0;
        const int r = o.rank[b];
        const int64_t tb = (int64_t)b * Nu;
        for (int d0 = 0; d0 < r; d0 += RC) {
            const int rc = min(RC, r - d0);
            // accumulator size for this chunk
            int sumk = 0;
            if (far)
                for (int d = d0; d < d0 + rc; ++d) sumk += o.frank[tb + d];
            const int nacc = far ? sumk * 2 * nrhs : nI * nrhs;
            for (int e = tid; e < nacc; e += blockDim.x) acc[e] = {0, 0};
            // fibre value per point of the frequency list (conjugated for the
            // conjugate half) and the half it belongs to
            for (int e = tid; e < rc * NQ; e += blockDim.x) {
                const int q = e % NQ, dd = e / NQ;
                const int mp = a.qmap[a.single_f >= 0 ? a.single_f : q];
                const cx<T> fv = fib[(tb + d0 + dd) * Nu + (mp > 0 ? mp - 1 : -mp - 1)];
                fq_s[e] = mp > 0 ? fv : cconj(fv);
                if (dd == 0) sg_s[q] = mp > 0 ? 1 : -1;
            }
            for (int j0 = 0; j0 < nJ; j0 += TJ) {
                const int tj = min(TJ, nJ - j0);
                __syncthreads();
                for (int e = tid; e < NQ * tj * nrhs; e += blockDim.x) {
                    const int c = e % nrhs, jj = (e / nrhs) % tj, q = e / (nrhs * tj);
                    const int64_t col = a.perm_c[bl[2] + j0 + jj];
                    Wt[((int64_t)q * TJ + jj) * nrhs + c] = W[((int64_t)q * a.ncols + col) * nrhs + c];
                }
                __syncthreads();
                // frequency contraction of the tile for the chunk's terms; the
                // per-point fibre coefficients were staged in shared memory
                for (int e = tid; e < rc * tj * nrhs; e += blockDim.x) {
                    const int c = e % nrhs, jj = (e / nrhs) % tj, dd = e / (nrhs * tj);
                    const cx<T> *fq = fq_s + (int64_t)dd * NQ;
                    cx<T> z1 = {0, 0}, z2 = {0, 0};
#pragma unroll 4
                    for (int q = 0; q < NQ; ++q) {
                        const cx<T> w = Wt[((int64_t)q * TJ + jj) * nrhs + c];
                        if (sg_s[q] > 0) cfma(z1, fq[q], w);
                        else cfma(z2, fq[q], w);
                    }
                    z[(((int64_t)dd * 2 + 0) * TJ + jj) * nrhs + c] = z1;
                    z[(((int64_t)dd * 2 + 1) * TJ + jj) * nrhs + c] = z2;
                }
                __syncthreads();
                if (!far) {
                    for (int e = tid; e < nI * nrhs; e += blockDim.x) {
                        const int c = e % nrhs, i = e / nrhs;
                        cx<T> s = acc[e];
                        for (int dd = 0; dd < rc; ++dd) {
                            const cx<T> *H = pool + o.foff[tb + d0 + dd] + (int64_t)i * nJ + j0;
                            for (int jj = 0; jj < tj; ++jj) {
                                const cx<T> h = H[jj];
                                cfma(s, h, z[(((int64_t)dd * 2 + 0) * TJ + jj) * nrhs + c]);
                                cfma(s, cconj(h), z[(((int64_t)dd * 2 + 1) * TJ + jj) * nrhs + c]);
                            }
                        }
                        acc[e] = s;
                    }
                } else {
                    // acc[(tau, p, c)] += sum_j V[tau][j] z_p[j][c]  (p = 1 uses conj V)
                    for (int e = tid; e < sumk * nrhs; e += blockDim.x) {
                        const int c = e % nrhs;
                        int t = e / nrhs, dd = 0;
                        while (t >= o.frank[tb + d0 + dd]) {
                            t -= o.frank[tb + d0 + dd];
                            ++dd;
                        }
                        const int kd = o.frank[tb + d0 + dd];
                        const cx<T> *V = pool + o.foff[tb + d0 + dd] + (int64_t)kd * nI + (int64_t)t * nJ + j0;
                        cx<T> s1 = acc[(e / nrhs) * 2 * nrhs + c], s2 = acc[(e / nrhs) * 2 * nrhs + nrhs + c];
                        for (int jj = 0; jj < tj; ++jj) {
                            const cx<T> v = V[jj];
                            cfma(s1, v, z[(((int64_t)dd * 2 + 0) * TJ + jj) * nrhs + c]);
                            cfma(s2, cconj(v), z[(((int64_t)dd * 2 + 1) * TJ + jj) * nrhs + c]);
                        }
                        acc[(e / nrhs) * 2 * nrhs + c] = s1;
                        acc[(e / nrhs) * 2 * nrhs + nrhs + c] = s2;
                    }
                }
            }
            __syncthreads();
            if (!far) {
                for (int e = tid; e < nI * nrhs; e += blockDim.x) {
                    const int c = e % nrhs, i = e / nrhs;
                    atomic_add_c(y + (int64_t)a.perm_r[bl[0] + i] * nrhs + c, acc[e]);
                }
            } else {
                for (int e = tid; e < nI * nrhs; e += blockDim.x) {
                    const int c = e % nrhs, i = e / nrhs;
                    cx<T> s = {0, 0};
                    int base = 0;
                    for (int dd = 0; dd < rc; ++dd) {
                        const int kd = o.frank[tb + d0 + dd];
                        const cx<T> *U = pool + o.foff[tb + d0 + dd];
                        for (int t = 0; t < kd; ++t) {
                            const cx<T> u = U[(int64_t)t * nI + i];
                            cfma(s, u, acc[(int64_t)(base + t) * 2 * nrhs + c]);
                            cfma(s, cconj(u), acc[(int64_t)(base + t) * 2 * nrhs + nrhs + c]);
                        }
                        base += kd;
                    }
                    atomic_add_c(y + (int64_t)a.perm_r[bl[0] + i] * nrhs + c, s);
                }
            }
            __syncthreads();
        }
    }
}

// Second phase of the tensor-core apply.  The frequency contraction
// z_(b,d,p) = sum_l f_d(l) W_l[J] is already in Z (k_zgemm.cu); Z rows of a
// block are (term d, half p) at zbase[b] + (rpt d + p) nJ nrhs.
//   k_apply_t: one warp per far term: T_p = V_d^T z_p (p = 1: conj V_d),
//              16 ranks at a time in registers, lanes over (half, rhs);
//   k_apply_y: one CTA per block, one thread per output (row, rhs), all
//              terms accumulated in registers: far y_I += U_d T1 + conj(U_d) T2,
//              near y_I += H_d z1 + conj(H_d) z2; one atomic add per output
//              and block.  No shared memory and no barriers in either kernel.
__global__ void __launch_bounds__(256) k_apply_t(ApplyZArgs a, TensorOut o) {
    const int nrhs = a.nrhs, Nu = a.Nu, rpt = a.rpt, lane = threadIdx.x & 31;
    const c32 *pool = (const c32 *)o.face;
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwt = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t it = gw; it < a.nft; it += nwt) {
        const int2 bd = a.ftab[it];
        const int *bl = a.blocks + 5 * bd.x;
        const int nI = bl[1] - bl[0], nJ = bl[3] - bl[2];
        const int64_t tb = (int64_t)bd.x * Nu + bd.y;
        const int kd = o.frank[tb];
        const c32 *V = pool + o.foff[tb] + (int64_t)kd * nI;
        const int64_t L = (int64_t)nJ * nrhs;
        const c32 *z1 = a.Z + a.zbase[bd.x] + (int64_t)rpt * bd.y * L;
        c32 *Tout = a.T + a.toff[tb];
        for (int pc = lane; pc < rpt * nrhs; pc += 32) {
            const int p = pc / nrhs, c = pc - p * nrhs;
            const c32 *z = z1 + p * L + c;
            for (int t0 = 0; t0 < kd; t0 += 16) {
                const int nt = min(16, kd - t0);
                c32 acc[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) acc[q] = c32{0.f, 0.f};
                for (int j = 0; j < nJ; ++j) {
                    const c32 zj = z[(int64_t)j * nrhs];
#pragma unroll
                    for (int q = 0; q < 16; ++q)
                        if (q < nt) {
                            const c32 v = V[(int64_t)(t0 + q) * nJ + j];
                            cfma(acc[q], p ? cconj(v) : v, zj);
                        }
                }
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    if (q < nt) Tout[((int64_t)p * kd + t0 + q) * nrhs + c] = acc[q];
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_apply_y(ApplyZArgs a, TensorOut o) {
    // each thread: one row i and four consecutive right-hand sides (face
    // loads shared by the four)
    const int nrhs = a.nrhs, Nu = a.Nu, rpt = a.rpt;
    const int nc4 = (nrhs + 3) >> 2;
    const c32 *pool = (const c32 *)o.face;
    for (int b = blockIdx.x; b < a.nb; b += gridDim.x) {
        const int *bl = a.blocks + 5 * b;
        const int nI = bl[1] - bl[0], nJ = bl[3] - bl[2];
        const bool far = bl[4] != 0;
        const int r = o.rank[b];
        if (r == 0 || a.zbase[b] < 0) continue;
        const int64_t tb = (int64_t)b * Nu, L = (int64_t)nJ * nrhs;
        for (int e = threadIdx.x; e < nI * nc4; e += blockDim.x) {
            const int i = e / nc4, c0 = 4 * (e - i * nc4), nc = min(4, nrhs - c0);
            c32 acc[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = c32{0.f, 0.f};
            for (int d = 0; d < r; ++d) {
                const c32 *X1, *X2, *M;
                int K;
                int64_t ms;
                if (far) {
                    K = o.frank[tb + d];
                    M = pool + o.foff[tb + d] + i;  // U[t][i], stride nI
                    ms = nI;
                    X1 = a.T + a.toff[tb + d] + c0;
                    X2 = X1 + (int64_t)K * nrhs;
                } else {
                    K = nJ;
                    M = pool + o.foff[tb + d] + (int64_t)i * nJ;  // H[i][j], stride 1
                    ms = 1;
                    X1 = a.Z + a.zbase[b] + (int64_t)rpt * d * L + c0;
                    X2 = X1 + L;
                }
                // face entries four at a time, loaded before use (the loop is bound by
                // the latency of these loads from HBM)
                int t = 0;
                for (; t + 4 <= K; t += 4) {
                    c32 mv[4];
#pragma unroll
                    for (int s = 0; s < 4; ++s) mv[s] = M[(int64_t)(t + s) * ms];
#pragma unroll
                    for (int s = 0; s < 4; ++s) {
                        const c32 mc = cconj(mv[s]);
                        const c32 *x1 = X1 + (int64_t)(t + s) * nrhs, *x2 = X2 + (int64_t)(t + s) * nrhs;
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            if (q >= nc) continue;
                            cfma(acc[q], mv[s], x1[q]);
                            if (rpt == 2) cfma(acc[q], mc, x2[q]);
                        }
                    }
                }
                for (; t < K; ++t) {
                    const c32 mv = M[(int64_t)t * ms], mc = cconj(mv);
                    const c32 *x1 = X1 + (int64_t)t * nrhs, *x2 = X2 + (int64_t)t * nrhs;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if (q >= nc) continue;
                        cfma(acc[q], mv, x1[q]);
                        if (rpt == 2) cfma(acc[q], mc, x2[q]);
                    }
                }
            }
            c32 *yr = a.y + (int64_t)a.perm_r[bl[0] + i] * nrhs + c0;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (q < nc) atomic_add_c(yr + q, acc[q]);
        }
    }
}

template <class T>
__global__ void k_tensor_entries(TensorOut o, const int *blocks, int nb, int64_t nrows, int64_t ncols,
                                 int nq, const int *inv_r, const int *inv_c, const int *qmap,
                                 const int *rows, const int *cols, const int *fidx, int64_t count,
                                 cx<T> *out) {
    const cx<T> *fib = (const cx<T> *)o.fib;
    const cx<T> *pool = (const cx<T> *)o.face;
    const int Nu = o.Nu;
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < count;
         n += (int64_t)gridDim.x * blockDim.x) {
        if (rows[n] < 0 || rows[n] >= nrows || cols[n] < 0 || cols[n] >= ncols || fidx[n] < 0 || fidx[n] >= nq) {
            out[n] = cx<T>{(T)NAN, (T)NAN};  // invalid index: no access, NaN result
            continue;
        }
        const int pi = inv_r[rows[n]], pj = inv_c[cols[n]];
        const int mp = qmap[fidx[n]];
        const int u = mp > 0 ? mp - 1 : -mp - 1;
        cx<T> v = {0, 0};
        for (int b = 0; b < nb; ++b) {
            const int *bl = blocks + 5 * b;
            if (pi < bl[0] || pi >= bl[1] || pj < bl[2] || pj >= bl[3]) continue;
            const int nI = bl[1] - bl[0], nJ = bl[3] - bl[2];
            const int i = pi - bl[0], j = pj - bl[2];
            const int64_t tb = (int64_t)b * Nu;
            for (int d = 0; d < o.rank[b]; ++d) {
                const cx<T> *F = pool + o.foff[tb + d];
                cx<T> h = {0, 0};
                const int kd = o.frank[tb + d];
                if (kd < 0)
                    h = F[(int64_t)i * nJ + j];
                else
                    for (int t = 0; t < kd; ++t) cfma(h, F[(int64_t)t * nI + i], F[(int64_t)kd * nI + (int64_t)t * nJ + j]);
                cfma(v, h, fib[(tb + d) * Nu + u]);
            }
            break;
        }
        out[n] = mp > 0 ? v : cconj(v);
    }
}

}  // namespace

int td_launch_apply(cudaStream_t st, int prec, const ApplyArgs &a, const TensorOut &o, int num_sms) {
    const int NQ = a.single_f >= 0 ? 1 : a.NQ;
    const size_t es = prec == TDBEM_FP64 ? 16 : 8;
    const int budget = 160 * 1024;
    // W tile: NQ x TJ x nrhs; z: RC x 2 x TJ x nrhs; acc: max(nI, 2*sumk) x nrhs
    int TJ = (int)std::max<int64_t>(1, std::min<int64_t>(32, (budget / 2) / ((int64_t)NQ * a.nrhs * es)));
    const int RC = 4;
    const int64_t acc_max = (int64_t)std::max(2 * RC * a.kcap, a.max_near_rows) * a.nrhs;
    auto smem = [&](int tj) {
        return ((int64_t)NQ * tj * a.nrhs + (int64_t)RC * 2 * tj * a.nrhs + acc_max + (int64_t)RC * NQ) * es +
               sizeof(int) * NQ;
    };
    size_t sm = smem(TJ);
    while (sm > (size_t)(200 * 1024) && TJ > 1) {
        TJ /= 2;
        sm = smem(TJ);
    }
    ApplyArgs aa = a;
    aa.acc_max = acc_max;
    if (sm > (size_t)(220 * 1024)) return (int)cudaErrorInvalidConfiguration;
    const int grid = std::min(a.nb, num_sms * 4);
    cudaError_t e;
    if (prec == TDBEM_FP64) {
        e = cudaFuncSetAttribute(k_apply<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return (int)e;
        k_apply<double><<<grid, 256, sm, st>>>(aa, o, TJ, RC);
    } else {
        e = cudaFuncSetAttribute(k_apply<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return (int)e;
        k_apply<float><<<grid, 256, sm, st>>>(aa, o, TJ, RC);
    }
    return (int)cudaGetLastError();
}

int td_launch_apply_z(cudaStream_t st, const ApplyZArgs &a, const TensorOut &o, int num_sms) {
    if (a.nft > 0) {
        const int grid = (int)std::min<int64_t>(((int64_t)a.nft * 32 + 255) / 256, (int64_t)num_sms * 8);
        k_apply_t<<<grid, 256, 0, st>>>(a, o);
    }
    const int grid = std::min(a.nb, num_sms * 8);
    k_apply_y<<<grid, 256, 0, st>>>(a, o);
    return (int)cudaGetLastError();
}

int td_launch_tensor_entries(cudaStream_t st, int prec, const TensorOut &o, const int *blocks,
                             int nb, int64_t nrows, int64_t ncols, int nq, const int *inv_r,
                             const int *inv_c, const int *qmap,
                             const int *rows, const int *cols, const int *fidx, int64_t count,
                             void *out) {
    if (count == 0) return 0;
    const int grid = (int)std::min<int64_t>((count + 127) / 128, 4096);
    if (prec == TDBEM_FP64)
        k_tensor_entries<double><<<grid, 128, 0, st>>>(o, blocks, nb, nrows, ncols, nq, inv_r, inv_c, qmap, rows, cols, fidx, count, (c64 *)out);
    else
        k_tensor_entries<float><<<grid, 128, 0, st>>>(o, blocks, nb, nrows, ncols, nq, inv_r, inv_c, qmap, rows, cols, fidx, count, (c32 *)out);
    return (int)cudaGetLastError();
}
