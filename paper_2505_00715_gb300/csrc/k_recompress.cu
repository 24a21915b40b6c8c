// Recompression of low-rank faces by QR and SVD (Sec. 4, the H-matrix
// variant: the ACA factors of a face are recompressed to the rank the
// tolerance needs).  A face H = U V^T (U: nI x k, V: nJ x k, k <= 64):
//
//   U = Q_U R_U, V = Q_V R_V        (Householder QR, Q_U = H_0 H_1 .. H_{k-1})
//   M = R_U R_V^T = W S Z^H         (one-sided Jacobi SVD: M Z = W S)
//   H = (Q_U W S) (Q_V conj(Z))^T,  truncated to the k' largest singular
//   values with sum_{i >= k'} s_i^2 <= eps^2 sum_i s_i^2,
//
// so U' = Q_U (M Z)[:, :k'] and V' = Q_V conj(Z)[:, :k'].  One CTA of 256
// threads per face: the factors are copied to per-CTA scratch, reduced there
// to their reflectors, and the new factors are written into the face's slot
// (they take k'(nI + nJ) <= k(nI + nJ) values).  Working precision: FP32 in
// the mixed form (backward stable: singular values resolved to ~1e-7 of the
// largest), FP64 in the FP64 form.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"
#include "kernels.h"

namespace {

constexpr int kRcMax = 64;       // largest face rank
constexpr int kRcLd = kRcMax + 1;  // padded leading dimension of the k x k matrices
constexpr int kRcThreads = 256;

template <class T> struct RcEps;
template <> struct RcEps<float> { static constexpr float v = 1e-7f; };
template <> struct RcEps<double> { static constexpr double v = 1e-15; };

// Householder QR of the n x k matrix A (column c at A + c * ld) in place:
// column j keeps the reflector v_j below and on the diagonal (H_j = I -
// tau_j v_j v_j^H), beta_j = R[j][j]; R[j][c] (c > j) stays in A[c][j].
template <class T>
TD_D void house_qr(cx<T> *A, int64_t ld, int n, int k, cx<T> *beta, T *tau, T *red) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = kRcThreads / 32;
    for (int j = 0; j < k; ++j) {
        cx<T> *x = A + (int64_t)j * ld;
        T s = 0;
        for (int i = j + tid; i < n; i += kRcThreads) s += x[i].x * x[i].x + x[i].y * x[i].y;
        s = warp_sum(s);
        if (lane == 0) red[wid] = s;
        __syncthreads();
        if (tid == 0) {
            T a2 = 0;
            for (int w = 0; w < nw; ++w) a2 += red[w];
            const T alpha = sqrt(a2);
            const cx<T> x0 = j < n ? x[j] : cx<T>{0, 0};
            const T ax0 = sqrt(x0.x * x0.x + x0.y * x0.y);
            if (alpha == (T)0) {
                beta[j] = cx<T>{0, 0};
                tau[j] = 0;
            } else {
                const cx<T> ph = ax0 > (T)0 ? cx<T>{x0.x / ax0, x0.y / ax0} : cx<T>{1, 0};
                const cx<T> b = cx<T>{-ph.x * alpha, -ph.y * alpha};
                beta[j] = b;
                tau[j] = (T)1 / (alpha * (alpha + ax0));
                x[j] = x0 - b;  // v_j = x - beta e_j
            }
        }
        __syncthreads();
        const T tj = tau[j];
        if (tj != (T)0) {
            for (int c = j + 1 + wid; c < k; c += nw) {
                cx<T> *y = A + (int64_t)c * ld;
                cx<T> d = {0, 0};
                for (int i = j + lane; i < n; i += 32) cfma(d, cconj(x[i]), y[i]);
                d.x = warp_sum(d.x);
                d.y = warp_sum(d.y);
                const cx<T> f = {tj * d.x, tj * d.y};
                for (int i = j + lane; i < n; i += 32) cfms(y[i], f, x[i]);
            }
        }
        __syncthreads();
    }
}

// y <- Q y for y of length n (Q = H_0 .. H_{k-1} from house_qr), by one warp.
template <class T>
TD_D void apply_q_warp(const cx<T> *A, int64_t ld, int n, int k, const T *tau, cx<T> *y) {
    const int lane = threadIdx.x & 31;
    for (int j = k - 1; j >= 0; --j) {
        const T tj = tau[j];
        if (tj == (T)0) continue;
        const cx<T> *v = A + (int64_t)j * ld;
        cx<T> d = {0, 0};
        for (int i = j + lane; i < n; i += 32) cfma(d, cconj(v[i]), y[i]);
        d.x = warp_sum(d.x);
        d.y = warp_sum(d.y);
        const cx<T> f = {tj * d.x, tj * d.y};
        __syncwarp();
        for (int i = j + lane; i < n; i += 32) cfms(y[i], f, v[i]);
        __syncwarp();
    }
}

struct RcJob {
    int nI, nJ, k, pad;
    int64_t off;  // face offset (complex units): U [k][nI] then V [k][nJ]
    int64_t kout; // where the new rank goes (index into the rank array)
};

template <class T>
__global__ void __launch_bounds__(kRcThreads) k_recompress(const RcJob *jobs, int njobs, cx<T> *pool, int *ranks,
                                                           cx<T> *scratch, int maxI, int maxJ, double eps) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T> *Ms = reinterpret_cast<cx<T> *>(smem_raw);  // M columns [kRcMax][kRcLd]
    cx<T> *Zs = Ms + kRcMax * kRcLd;                    // Z columns
    cx<T> *bu = Zs + kRcMax * kRcLd, *bv = bu + kRcMax;
    T *tu = reinterpret_cast<T *>(bv + kRcMax), *tv = tu + kRcMax, *sig = tv + kRcMax, *red = sig + kRcMax;
    int *perm = reinterpret_cast<int *>(red + 32);
    int *flag = perm + kRcMax;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = kRcThreads / 32;
    cx<T> *QU = scratch + (int64_t)blockIdx.x * kRcMax * ((int64_t)maxI + maxJ);
    cx<T> *QV = QU + (int64_t)kRcMax * maxI;
    const int64_t ldv = maxJ;
    for (int jb = blockIdx.x; jb < njobs; jb += gridDim.x) {
        const RcJob J = jobs[jb];
        const int nI = J.nI, nJ = J.nJ, k = J.k;
        cx<T> *U = pool + J.off, *V = U + (int64_t)k * nI;
        __syncthreads();
        for (int64_t e = tid; e < (int64_t)k * nI; e += kRcThreads) QU[(e / nI) * maxI + e % nI] = U[e];
        for (int64_t e = tid; e < (int64_t)k * nJ; e += kRcThreads) QV[(e / nJ) * ldv + e % nJ] = V[e];
        __syncthreads();
        house_qr(QU, maxI, nI, k, bu, tu, red);
        house_qr(QV, ldv, nJ, k, bv, tv, red);
        // M = R_U R_V^T (column b of M at Ms + b kRcLd), Z = I
        for (int e = tid; e < kRcMax * kRcMax; e += kRcThreads) {
            const int a = e % kRcMax, b = e / kRcMax;
            cx<T> m = {0, 0};
            // (R_U has min(k, nI) nonzero rows, R_V min(k, nJ))
            if (a < k && b < k && a < nI && b < nJ) {
                for (int c = max(a, b); c < k; ++c) {
                    const cx<T> ru = c == a ? bu[a] : QU[(int64_t)c * maxI + a];
                    const cx<T> rv = c == b ? bv[b] : QV[(int64_t)c * ldv + b];
                    cfma(m, ru, rv);
                }
            }
            Ms[b * kRcLd + a] = m;
            Zs[b * kRcLd + a] = cx<T>{(T)(a == b ? 1 : 0), 0};
        }
        __syncthreads();
        // one-sided Jacobi on the columns of M (round-robin pairs, rotations
        // accumulated in Z), until a sweep rotates nothing
        const int kk = k + (k & 1);
        for (int sweep = 0; sweep < 30; ++sweep) {
            if (tid == 0) *flag = 0;
            __syncthreads();
            for (int r = 0; r + 1 < kk; ++r) {
                for (int pi = wid; pi < kk / 2; pi += nw) {
                    const int s0 = pi, s1 = kk - 1 - pi;
                    const int p = s0 == 0 ? 0 : 1 + (s0 - 1 + r) % (kk - 1);
                    const int q = 1 + (s1 - 1 + r) % (kk - 1);
                    if (p >= k || q >= k) continue;
                    cx<T> *mp = Ms + p * kRcLd, *mq = Ms + q * kRcLd;
                    T al = 0, be = 0;
                    cx<T> g = {0, 0};
                    for (int a = lane; a < k; a += 32) {
                        al += mp[a].x * mp[a].x + mp[a].y * mp[a].y;
                        be += mq[a].x * mq[a].x + mq[a].y * mq[a].y;
                        cfma(g, cconj(mp[a]), mq[a]);
                    }
                    al = warp_sum(al);
                    be = warp_sum(be);
                    g.x = warp_sum(g.x);
                    g.y = warp_sum(g.y);
                    const T ag = sqrt(g.x * g.x + g.y * g.y);
                    if (!(ag > RcEps<T>::v * sqrt(al * be))) continue;
                    // columns p, q <- [c m_p - s e^{-i phi} m_q, s e^{i phi} m_p + c m_q]
                    const T zeta = (be - al) / (2 * ag);
                    const T t = (zeta >= 0 ? (T)1 : (T)-1) / (fabs(zeta) + sqrt((T)1 + zeta * zeta));
                    const T cs = (T)1 / sqrt((T)1 + t * t), sn = cs * t;
                    const cx<T> e = {g.x / ag, g.y / ag};  // e^{i phi}
                    const cx<T> sp = {sn * e.x, sn * e.y}, sm = {sn * e.x, -sn * e.y};
                    cx<T> *zp = Zs + p * kRcLd, *zq = Zs + q * kRcLd;
                    for (int a = lane; a < k; a += 32) {
                        const cx<T> x = mp[a], y = mq[a];
                        mp[a] = cx<T>{cs * x.x, cs * x.y} - sm * y;
                        mq[a] = sp * x + cx<T>{cs * y.x, cs * y.y};
                        const cx<T> u = zp[a], w = zq[a];
                        zp[a] = cx<T>{cs * u.x, cs * u.y} - sm * w;
                        zq[a] = sp * u + cx<T>{cs * w.x, cs * w.y};
                    }
                    if (lane == 0) *flag = 1;
                }
                __syncthreads();
            }
            if (*flag == 0) break;
            __syncthreads();
        }
        // singular values, order, truncation
        for (int c = wid; c < k; c += nw) {
            T s2 = 0;
            for (int a = lane; a < k; a += 32) s2 += Ms[c * kRcLd + a].x * Ms[c * kRcLd + a].x + Ms[c * kRcLd + a].y * Ms[c * kRcLd + a].y;
            s2 = warp_sum(s2);
            if (lane == 0) sig[c] = s2;
        }
        __syncthreads();
        if (tid == 0) {
            for (int c = 0; c < k; ++c) perm[c] = c;
            for (int a = 0; a < k; ++a)
                for (int b = a + 1; b < k; ++b)
                    if (sig[perm[b]] > sig[perm[a]]) {
                        const int t = perm[a];
                        perm[a] = perm[b];
                        perm[b] = t;
                    }
            double tot = 0.0, tail = 0.0;
            for (int c = 0; c < k; ++c) tot += (double)sig[c];
            int kn = k;
            while (kn > 1 && tail + (double)sig[perm[kn - 1]] <= eps * eps * tot) {
                tail += (double)sig[perm[kn - 1]];
                --kn;
            }
            flag[1] = kn;
        }
        __syncthreads();
        const int kn = flag[1];
        // U' row c = Q_U (M Z)[:, perm[c]], V' row c = Q_V conj(Z)[:, perm[c]]
        cx<T> *Un = U, *Vn = U + (int64_t)kn * nI;
        for (int c = wid; c < 2 * kn; c += nw) {
            const bool isv = c >= kn;
            const int cc = isv ? c - kn : c, src = perm[cc];
            const int n = isv ? nJ : nI;
            cx<T> *y = isv ? Vn + (int64_t)cc * nJ : Un + (int64_t)cc * nI;
            const cx<T> *col = (isv ? Zs : Ms) + src * kRcLd;
            for (int i = lane; i < n; i += 32) y[i] = i < k ? (isv ? cconj(col[i]) : col[i]) : cx<T>{0, 0};
            __syncwarp();
            if (isv)
                apply_q_warp(QV, ldv, nJ, k, tv, y);
            else
                apply_q_warp(QU, maxI, nI, k, tu, y);
        }
        if (tid == 0) ranks[J.kout] = kn;
        __syncthreads();
    }
}

// Copies the faces of a pool into a compacted pool: src offset, dst offset, size.
template <class T>
__global__ void k_pool_gather(const int64_t *moves, int nmoves, const cx<T> *src, cx<T> *dst) {
    for (int mv = blockIdx.x; mv < nmoves; mv += gridDim.x) {
        const int64_t so = moves[3 * mv], dof = moves[3 * mv + 1], n = moves[3 * mv + 2];
        for (int64_t e = threadIdx.x; e < n; e += blockDim.x) dst[dof + e] = src[so + e];
    }
}

}  // namespace

size_t td_recompress_smem(int prec) {
    const size_t es = prec == TDBEM_FP64 ? sizeof(c64) : sizeof(c32), rs = prec == TDBEM_FP64 ? 8 : 4;
    return es * (2 * kRcMax * kRcLd + 2 * kRcMax) + rs * (3 * kRcMax + 32) + sizeof(int) * (kRcMax + 2) + 64;
}

// jobs: device [njobs] {nI, nJ, k, 0, off, kout}; scratch: nctas x 64 (maxI + maxJ)
int td_launch_recompress(cudaStream_t st, int prec, const void *jobs, int njobs, void *pool, int *ranks,
                         void *scratch, int maxI, int maxJ, double eps, int nctas) {
    if (njobs == 0) return 0;
    const size_t sm = td_recompress_smem(prec);
    cudaError_t e;
    if (prec == TDBEM_FP64) {
        e = cudaFuncSetAttribute(k_recompress<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return (int)e;
        k_recompress<double><<<nctas, kRcThreads, sm, st>>>((const RcJob *)jobs, njobs, (c64 *)pool, ranks,
                                                           (c64 *)scratch, maxI, maxJ, eps);
    } else {
        e = cudaFuncSetAttribute(k_recompress<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return (int)e;
        k_recompress<float><<<nctas, kRcThreads, sm, st>>>((const RcJob *)jobs, njobs, (c32 *)pool, ranks,
                                                          (c32 *)scratch, maxI, maxJ, eps);
    }
    return (int)cudaGetLastError();
}

int td_launch_pool_gather(cudaStream_t st, int prec, const int64_t *moves, int nmoves, const void *src, void *dst,
                          int num_sms) {
    if (nmoves == 0) return 0;
    const int grid = std::min(nmoves, num_sms * 8);
    if (prec == TDBEM_FP64)
        k_pool_gather<double><<<grid, 256, 0, st>>>(moves, nmoves, (const c64 *)src, (c64 *)dst);
    else
        k_pool_gather<float><<<grid, 256, 0, st>>>(moves, nmoves, (const c32 *)src, (c32 *)dst);
    return (int)cudaGetLastError();
}

int td_recompress_job_bytes() { return (int)sizeof(RcJob); }

// ============================================================================
// C-ABI: recompression of a compressed tensor's far faces, and of one face
// ============================================================================
namespace {

struct HostJob {
    int nI, nJ, k, pad;
    int64_t off, kout;
};
static_assert(sizeof(HostJob) == sizeof(RcJob), "job layout");

template <class P>
int rc_alloc(tdbem_ctx *ctx, P **p, size_t bytes, std::vector<void *> &g) {
    *p = nullptr;
    if (cudaMalloc((void **)p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
        cudaGetLastError();
        return td_fail(ctx, TDBEM_ERR_OOM, "recompression: device allocation of %zu bytes failed", bytes);
    }
    g.push_back((void *)*p);
    return TDBEM_OK;
}

struct Frees {
    std::vector<void *> p;
    ~Frees() {
        for (void *q : p) cudaFree(q);
    }
};

}  // namespace

extern "C" int tdbem_tensor_recompress(tdbem_tensor_t t, double eps) {
    if (!t) return TDBEM_ERR_ARG;
    tdbem_ctx *ctx = t->ctx;
    cudaGetLastError();
    if (!(eps > 0.0) || !(eps < 1.0)) return td_fail(ctx, TDBEM_ERR_ARG, "tdbem_tensor_recompress: need 0 < eps < 1");
    cudaStream_t st = ctx->stream;
    const int64_t nb = t->nblocks, Nu = t->Nu;
    const size_t es = t->prec == TDBEM_FP64 ? sizeof(c64) : sizeof(c32);
    std::vector<int32_t> frank((size_t)nb * Nu);
    std::vector<int64_t> foff((size_t)nb * Nu);
    TD_CUDA(ctx, cudaStreamSynchronize(st));
    TD_CUDA(ctx, cudaMemcpy(frank.data(), t->dfrank, sizeof(int32_t) * frank.size(), cudaMemcpyDeviceToHost));
    TD_CUDA(ctx, cudaMemcpy(foff.data(), t->dfoff, sizeof(int64_t) * foff.size(), cudaMemcpyDeviceToHost));
    std::vector<HostJob> jobs;
    int maxI = 1, maxJ = 1;
    for (int64_t b = 0; b < nb; ++b) {
        const int32_t *bl = &t->blocks[5 * b];
        if (!bl[4]) continue;
        for (int d = 0; d < t->rank[b]; ++d) {
            const int k = frank[b * Nu + d];
            if (k <= 1) continue;
            HostJob j{bl[1] - bl[0], bl[3] - bl[2], k, 0, foff[b * Nu + d], b * Nu + d};
            jobs.push_back(j);
            maxI = std::max(maxI, j.nI);
            maxJ = std::max(maxJ, j.nJ);
        }
    }
    Frees g;
    if (!jobs.empty()) {
        const int nctas = std::min<int>((int)jobs.size(), ctx->num_sms * 2);
        void *djobs, *scr;
        int rc;
        if ((rc = rc_alloc(ctx, &djobs, sizeof(HostJob) * jobs.size(), g.p)) ||
            (rc = rc_alloc(ctx, &scr, es * (size_t)nctas * kRcMax * ((size_t)maxI + maxJ), g.p)))
            return rc;
        TD_CUDA(ctx, cudaMemcpyAsync(djobs, jobs.data(), sizeof(HostJob) * jobs.size(), cudaMemcpyHostToDevice, st));
        const int e = td_launch_recompress(st, t->prec, djobs, (int)jobs.size(), t->dface, t->dfrank, scr, maxI, maxJ,
                                           eps, nctas);
        if (e) return td_fail(ctx, TDBEM_ERR_CUDA, "recompression kernel failed: %s", cudaGetErrorString((cudaError_t)e));
        TD_CUDA(ctx, cudaStreamSynchronize(st));
        TD_CUDA(ctx, cudaMemcpy(frank.data(), t->dfrank, sizeof(int32_t) * frank.size(), cudaMemcpyDeviceToHost));
    }
    // compaction: every face moves to its place in a pool of the exact size
    std::vector<int64_t> moves, noff(foff);
    int64_t used = 0;
    for (int64_t b = 0; b < nb; ++b) {
        const int32_t *bl = &t->blocks[5 * b];
        const int64_t nI = bl[1] - bl[0], nJ = bl[3] - bl[2];
        for (int d = 0; d < t->rank[b]; ++d) {
            const int k = frank[b * Nu + d];
            const int64_t n = k < 0 ? nI * nJ : (int64_t)k * (nI + nJ);
            moves.push_back(foff[b * Nu + d]);
            moves.push_back(used);
            moves.push_back(n);
            noff[b * Nu + d] = used;
            used += n;
        }
    }
    void *npool = nullptr, *dmoves = nullptr;
    if (cudaMalloc(&npool, es * (size_t)std::max<int64_t>(used, 1)) != cudaSuccess) {
        cudaGetLastError();
        return td_fail(ctx, TDBEM_ERR_OOM, "recompression: compacted pool allocation failed");
    }
    int rc = rc_alloc(ctx, &dmoves, sizeof(int64_t) * std::max<size_t>(moves.size(), 1), g.p);
    if (rc) {
        cudaFree(npool);
        return rc;
    }
    if (cudaMemcpyAsync(dmoves, moves.data(), sizeof(int64_t) * moves.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        td_launch_pool_gather(st, t->prec, (const int64_t *)dmoves, (int)(moves.size() / 3), t->dface, npool,
                              ctx->num_sms) ||
        cudaMemcpyAsync(t->dfoff, noff.data(), sizeof(int64_t) * noff.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(t->dface_used, &used, sizeof(int64_t), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaFree(npool);
        return td_fail(ctx, TDBEM_ERR_CUDA, "recompression: pool compaction failed");
    }
    cudaFree(t->dface);
    *std::find(t->owned.begin(), t->owned.end(), t->dface) = npool;
    t->dface = npool;
    t->face_cap = std::max<int64_t>(used, 1);
    // statistics and the apply plan (rebuilt for the new ranks on the next apply)
    tdbem_stats &s = t->stats;
    s.stored_complex = 0;
    s.sum_face_rank = 0;
    for (int64_t b = 0; b < nb; ++b) {
        const int32_t *bl = &t->blocks[5 * b];
        const int64_t nI = bl[1] - bl[0], nJ = bl[3] - bl[2];
        t->frank_sum[b] = 0;
        for (int d = 0; d < t->rank[b]; ++d) {
            const int k = frank[b * Nu + d];
            s.stored_complex += Nu + (k < 0 ? nI * nJ : (int64_t)k * (nI + nJ));
            if (k > 0) {
                s.sum_face_rank += k;
                t->frank_sum[b] += k;
            }
        }
    }
    if (t->plan_mem) cudaFree(t->plan_mem);
    if (t->plan_Z) cudaFree(t->plan_Z);
    t->plan_mem = t->plan_Z = nullptr;
    t->plan_nrhs = 0;
    return TDBEM_OK;
}

extern "C" int tdbem_lowrank_recompress(tdbem_ctx_t ctx, int32_t prec, int32_t nI, int32_t nJ, int32_t k, const void *U,
                                        const void *V, double eps, void *Uout, void *Vout, int32_t *kout) {
    if (!ctx) return TDBEM_ERR_ARG;
    cudaGetLastError();
    if ((prec != TDBEM_FP64 && prec != TDBEM_MIXED) || nI < 1 || nJ < 1 || k < 1 || k > kRcMax || !U || !V || !Uout ||
        !Vout || !kout || !(eps > 0.0) || !(eps < 1.0))
        return td_fail(ctx, TDBEM_ERR_ARG, "tdbem_lowrank_recompress: need 1 <= k <= 64, 0 < eps < 1, non-NULL buffers");
    const size_t es = prec == TDBEM_FP64 ? sizeof(c64) : sizeof(c32);
    cudaStream_t st = ctx->stream;
    Frees g;
    char *pool;
    int *dk;
    void *djobs, *scr;
    int rc;
    if ((rc = rc_alloc(ctx, &pool, es * (size_t)k * (nI + nJ), g.p)) || (rc = rc_alloc(ctx, &dk, sizeof(int), g.p)) ||
        (rc = rc_alloc(ctx, &djobs, sizeof(HostJob), g.p)) ||
        (rc = rc_alloc(ctx, &scr, es * kRcMax * ((size_t)nI + nJ), g.p)))
        return rc;
    const HostJob j{nI, nJ, k, 0, 0, 0};
    TD_CUDA(ctx, cudaMemcpyAsync(pool, U, es * (size_t)k * nI, cudaMemcpyDeviceToDevice, st));
    TD_CUDA(ctx, cudaMemcpyAsync(pool + es * (size_t)k * nI, V, es * (size_t)k * nJ, cudaMemcpyDeviceToDevice, st));
    TD_CUDA(ctx, cudaMemcpyAsync(djobs, &j, sizeof j, cudaMemcpyHostToDevice, st));
    const int e = td_launch_recompress(st, prec, djobs, 1, pool, dk, scr, nI, nJ, eps, 1);
    if (e) return td_fail(ctx, TDBEM_ERR_CUDA, "recompression kernel failed: %s", cudaGetErrorString((cudaError_t)e));
    int kn = 0;
    TD_CUDA(ctx, cudaMemcpyAsync(&kn, dk, sizeof(int), cudaMemcpyDeviceToHost, st));
    TD_CUDA(ctx, cudaStreamSynchronize(st));
    TD_CUDA(ctx, cudaMemcpyAsync(Uout, pool, es * (size_t)kn * nI, cudaMemcpyDeviceToDevice, st));
    TD_CUDA(ctx, cudaMemcpyAsync(Vout, pool + es * (size_t)kn * nI, es * (size_t)kn * nJ, cudaMemcpyDeviceToDevice, st));
    TD_CUDA(ctx, cudaStreamSynchronize(st));
    *kout = kn;
    return TDBEM_OK;
}
