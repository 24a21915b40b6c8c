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
// block are (term d, half p) at zbase[b] + p zpstride[b] + d nJ nrhs.  Both face
// stages are small complex GEMMs out[m][(p, c)] = sum_k A_p[m][k] B[k][(p, c)]
// with A_1 = conj(A_0) for the conjugate half, tiled through shared memory:
//   stage 0 (one CTA per far term):  T_p = V_d^T z_p, m = tau < k_d, k = j < |J|,
//            A = V_d (row-major), written to T;
//   stage 1 (one CTA per block):      y_I += sum_d U_d T_(d,1) + conj(U_d) T_(d,2)
//            (far; m = i, k = (d, tau), A = U_d^T, column-major) or
//            y_I += sum_d H_d z_(d,1) + conj(H_d) z_(d,2) (near; k = (d, j),
//            A = H_d row-major); both halves summed before one atomic add
//            per output.
// Tiles: 64 rows x (rpt nrhs) columns, k in chunks of 32; 16 x CG threads,
// every thread holds a 4 x CPT register tile (rows 4 ty .. 4 ty + 3,
// columns tx + CG q, tx < CG).
constexpr int kFM = 64, kFK = 32, kFPad = 65;

struct FaceSmem {
    c32 A[kFK][kFPad];  // A[k][m] (m contiguous)
};

template <int CG, int CPT>
__global__ void __launch_bounds__(16 * CG) k_apply_faces(ApplyZArgs a, TensorOut o, int stage) {
    constexpr int NT = 16 * CG;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FaceSmem &F = *reinterpret_cast<FaceSmem *>(smem_raw);
    c32 *Bs = reinterpret_cast<c32 *>(smem_raw + sizeof(FaceSmem));  // [kFK][ncol]
    const int nrhs = a.nrhs, Nu = a.Nu, rpt = a.rpt, ncol = rpt * nrhs;
    const c32 *pool = (const c32 *)o.face;
    const int tid = threadIdx.x, tx = tid % CG, ty = tid / CG;
    // columns of this thread and their half; both halves of one right-hand side
    // sit in the same thread (q and q + CPT / 2) when 2 nrhs = CG CPT
    bool conj_q[CPT];
#pragma unroll
    for (int q = 0; q < CPT; ++q) conj_q[q] = tx + CG * q >= nrhs;
    const bool pair_halves = CPT >= 2 && rpt == 2 && 2 * nrhs == CG * CPT;
    const int64_t njobs = stage == 0 ? a.nft : a.nb;
    for (int64_t job = blockIdx.x; job < njobs; job += gridDim.x) {
        int b, d0, d1, M;
        if (stage == 0) {
            const int2 bd = a.ftab[job];
            b = bd.x;
            d0 = bd.y;
            d1 = bd.y + 1;
        } else {
            b = (int)job;
            d0 = 0;
            d1 = o.rank[b];
            if (d1 == 0 || a.zbase[b] < 0) continue;
        }
        const int *bl = a.blocks + 5 * b;
        const int nI = bl[1] - bl[0], nJ = bl[3] - bl[2];
        const bool far = bl[4] != 0;
        const int64_t tb = (int64_t)b * Nu, L = (int64_t)nJ * nrhs;
        M = stage == 0 ? o.frank[tb + d0] : nI;
        for (int m0 = 0; m0 < M; m0 += kFM) {
            c32 acc[4][CPT];
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int q = 0; q < CPT; ++q) acc[x][q] = c32{0.f, 0.f};
            for (int d = d0; d < d1; ++d) {
                const int kd = o.frank[tb + d];
                const c32 *face = pool + o.foff[tb + d];
                // A operand, its layout and length; B operand rows (p = 0 / 1)
                const c32 *Ab;
                int64_t lda;
                bool acol;
                int K;
                const c32 *B0;
                int64_t bstride;  // B[k][(p, c)] = B0[p * bstride + k * nrhs + c]
                if (stage == 0) {
                    Ab = face + (int64_t)kd * nI;  // V[tau][j]
                    lda = nJ;
                    acol = false;
                    K = nJ;
                    B0 = a.Z + a.zbase[b] + (int64_t)d * L;
                    bstride = a.zpstride[b];
                } else if (far) {
                    Ab = face;  // U[tau][i]: A[i][tau] column-major
                    lda = nI;
                    acol = true;
                    K = kd;
                    B0 = a.T + a.toff[tb + d];
                    bstride = (int64_t)kd * nrhs;
                } else {
                    Ab = face;  // H[i][j]
                    lda = nJ;
                    acol = false;
                    K = nJ;
                    B0 = a.Z + a.zbase[b] + (int64_t)d * L;
                    bstride = a.zpstride[b];
                }
                for (int k0 = 0; k0 < K; k0 += kFK) {
                    const int kc = min(kFK, K - k0), mc = min(kFM, M - m0);
                    __syncthreads();
                    if (acol) {
                        for (int e = tid; e < kFK * kFM; e += NT) {
                            const int kk = e / kFM, mm = e - kk * kFM;
                            F.A[kk][mm] = (kk < kc && mm < mc) ? Ab[(int64_t)(k0 + kk) * lda + m0 + mm] : c32{0.f, 0.f};
                        }
                    } else {
                        for (int e = tid; e < kFK * kFM; e += NT) {
                            const int mm = e / kFK, kk = e - mm * kFK;
                            F.A[kk][mm] = (kk < kc && mm < mc) ? Ab[(int64_t)(m0 + mm) * lda + k0 + kk] : c32{0.f, 0.f};
                        }
                    }
                    for (int e = tid; e < kFK * ncol; e += NT) {
                        const int kk = e / ncol, n = e - kk * ncol, p = n / nrhs, c = n - p * nrhs;
                        Bs[e] = kk < kc ? B0[p * bstride + (int64_t)(k0 + kk) * nrhs + c] : c32{0.f, 0.f};
                    }
                    __syncthreads();
#pragma unroll 4
                    for (int kk = 0; kk < kFK; ++kk) {
                        c32 av[4], bv[CPT];
#pragma unroll
                        for (int x = 0; x < 4; ++x) av[x] = F.A[kk][4 * ty + x];
#pragma unroll
                        for (int q = 0; q < CPT; ++q) {
                            const int n = tx + CG * q;
                            bv[q] = n < ncol ? Bs[kk * ncol + n] : c32{0.f, 0.f};
                        }
#pragma unroll
                        for (int x = 0; x < 4; ++x)
#pragma unroll
                            for (int q = 0; q < CPT; ++q) {
                                // conjugate half: conj(a) b
                                const float ay = conj_q[q] ? -av[x].y : av[x].y;
                                acc[x][q].x = fmaf(av[x].x, bv[q].x, fmaf(-ay, bv[q].y, acc[x][q].x));
                                acc[x][q].y = fmaf(av[x].x, bv[q].y, fmaf(ay, bv[q].x, acc[x][q].y));
                            }
                    }
                }
            }
            // ---- output
#pragma unroll
            for (int x = 0; x < 4; ++x) {
                const int m = m0 + 4 * ty + x;
                if (m >= M) continue;
                if (stage == 0) {
                    const int kd = M;
                    c32 *Tout = a.T + a.toff[tb + d0];
#pragma unroll
                    for (int q = 0; q < CPT; ++q) {
                        const int n = tx + CG * q;
                        if (n >= ncol) continue;
                        const int p = n / nrhs, c = n - p * nrhs;
                        Tout[((int64_t)p * kd + m) * nrhs + c] = acc[x][q];
                    }
                } else {
                    c32 *yr = a.y + (int64_t)a.perm_r[bl[0] + m] * nrhs;
                    if (pair_halves) {
#pragma unroll
                        for (int q = 0; q < CPT / 2; ++q) {
                            const int c = tx + CG * q;
                            if (c < nrhs) atomic_add_c(yr + c, acc[x][q] + acc[x][q + CPT / 2]);
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < CPT; ++q) {
                            const int n = tx + CG * q;
                            if (n < ncol) atomic_add_c(yr + n % nrhs, acc[x][q]);
                        }
                    }
                }
            }
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

template <int CG, int CPT>
static int launch_faces(cudaStream_t st, const ApplyZArgs &a, const TensorOut &o, int stage, int grid) {
    const size_t sm = sizeof(FaceSmem) + sizeof(c32) * kFK * a.rpt * a.nrhs;
    cudaError_t e = cudaFuncSetAttribute(k_apply_faces<CG, CPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return (int)e;
    k_apply_faces<CG, CPT><<<grid, 16 * CG, sm, st>>>(a, o, stage);
    return (int)cudaGetLastError();
}

int td_launch_apply_z(cudaStream_t st, const ApplyZArgs &a, const TensorOut &o, int num_sms) {
    const int ncol = a.rpt * a.nrhs;
    auto run = [&](int stage, int grid) {
        // 8 x 4 or 16 x 4 threads' register tiles of 4 x 4 complex outputs
        // (ncol <= 64); 16 column groups of 8 columns beyond
        if (ncol <= 16) return launch_faces<8, 2>(st, a, o, stage, grid);
        if (ncol <= 32) return launch_faces<8, 4>(st, a, o, stage, grid);
        if (ncol <= 64) return launch_faces<16, 4>(st, a, o, stage, grid);
        return launch_faces<16, 8>(st, a, o, stage, grid);
    };
    int e = 0;
    if (a.nft > 0) e = run(0, (int)std::min<int64_t>(a.nft, (int64_t)num_sms * 32));
    if (!e && a.nb > 0) e = run(1, std::min(a.nb, num_sms * 32));
    return e;
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
