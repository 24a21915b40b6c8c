// Per-frequency solve on the compressed tensor and persistence of tensors
// and models.
//
// tdbem_solve: restarted GMRES (Arnoldi with modified Gram-Schmidt, Givens
// rotations) for A(s_l) x = b, one Krylov space per right-hand side, all
// right-hand sides advanced together so that every operator application is
// one call of the single-frequency apply (y = sum_d f_d[l] H_d x, eq. product
// at one frequency).  Inner products are accumulated in FP64.
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"
#include "kernels.h"
#include "mlp.h"

namespace {

// out[c] += sum_i conj(a[i][c]) b[i][c]  (FP64 accumulation), M rows, n columns
template <class T>
__global__ void k_dot_cols(const cx<T> *a, const cx<T> *b, int64_t M, int n, double *out) {
    __shared__ double red[2][32];
    const int c = blockIdx.y;
    double re = 0.0, im = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        const cx<T> x = a[i * n + c], y = b[i * n + c];
        re += (double)x.x * y.x + (double)x.y * y.y;
        im += (double)x.x * y.y - (double)x.y * y.x;
    }
    re = warp_sum(re);
    im = warp_sum(im);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][wid] = re;
        red[1][wid] = im;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sr = 0.0, si = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            sr += red[0][w];
            si += red[1][w];
        }
        atomicAdd(&out[2 * c], sr);
        atomicAdd(&out[2 * c + 1], si);
    }
}

// y[i][c] = beta * y[i][c] + alpha[c] * x[i][c]  (alpha as interleaved doubles;
// y is not read when beta == 0, so it may start uninitialised)
template <class T>
__global__ void k_axpby_cols(cx<T> *y, const cx<T> *x, const double *alpha, double beta, int64_t M, int n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < M * n; e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e % n);
        const cx<T> a = {(T)alpha[2 * c], (T)alpha[2 * c + 1]};
        cx<T> v = {(T)0, (T)0};
        if (beta != 0.0) v = {(T)(beta * y[e].x), (T)(beta * y[e].y)};
        if (x) cfma(v, a, x[e]);
        y[e] = v;
    }
}

template <class T>
struct Ops {
    cudaStream_t st;
    int64_t M;
    int n;
    double *dtmp;  // [2 n]
    int sms;
    int dot(const cx<T> *a, const cx<T> *b, std::vector<std::complex<double>> &out) {
        cudaMemsetAsync(dtmp, 0, sizeof(double) * 2 * n, st);
        dim3 grid((unsigned)std::min<int64_t>((M + 255) / 256, sms * 2), n);
        k_dot_cols<T><<<grid, 256, 0, st>>>(a, b, M, n, dtmp);
        out.resize(n);
        if (cudaMemcpyAsync(out.data(), dtmp, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return TDBEM_ERR_CUDA;
        return TDBEM_OK;
    }
    // y = beta y + alpha x
    int axpby(cx<T> *y, const cx<T> *x, const std::vector<std::complex<double>> &alpha, double beta) {
        cudaMemcpyAsync(dtmp, alpha.data(), sizeof(double) * 2 * n, cudaMemcpyHostToDevice, st);
        const int grid = (int)std::min<int64_t>((M * n + 255) / 256, sms * 8);
        k_axpby_cols<T><<<grid, 256, 0, st>>>(y, x, dtmp, beta, M, n);
        return cudaGetLastError() == cudaSuccess ? TDBEM_OK : TDBEM_ERR_CUDA;
    }
};

template <class T>
int gmres(tdbem_tensor *t, int fidx, const cx<T> *b, int n, cx<T> *x, double tol, int maxit, int m, int *iters,
          double *relres) {
    tdbem_ctx *ctx = t->ctx;
    const int64_t M = t->nrows;
    std::vector<void *> owned;
    auto cleanup = [&]() {
        for (void *p : owned) cudaFree(p);
    };
    cx<T> *V = nullptr, *w = nullptr, *r = nullptr;
    double *dtmp = nullptr;
    if (cudaMalloc(&V, sizeof(cx<T>) * M * n * (m + 1)) != cudaSuccess) return TDBEM_ERR_OOM;
    owned.push_back(V);
    if (cudaMalloc(&w, sizeof(cx<T>) * M * n) != cudaSuccess || (owned.push_back(w), false) ||
        cudaMalloc(&r, sizeof(cx<T>) * M * n) != cudaSuccess || (owned.push_back(r), false) ||
        cudaMalloc(&dtmp, sizeof(double) * 2 * n) != cudaSuccess) {
        cleanup();
        cudaGetLastError();
        return TDBEM_ERR_OOM;
    }
    owned.push_back(dtmp);
    Ops<T> ops{ctx->stream, M, n, dtmp, ctx->num_sms};
    using C = std::complex<double>;
    std::vector<C> one(n, C(1.0, 0.0)), mone(n, C(-1.0, 0.0)), tmp;
    int rc = TDBEM_OK;
    // x = 0, ||b||
    cudaMemsetAsync(x, 0, sizeof(cx<T>) * M * n, ctx->stream);
    std::vector<double> bnorm(n);
    if ((rc = ops.dot(b, b, tmp))) {
        cleanup();
        return rc;
    }
    for (int c = 0; c < n; ++c) bnorm[c] = std::sqrt(std::max(tmp[c].real(), 1e-300));
    int it = 0;
    std::vector<double> res(n, 1.0);
    bool done = false;
    while (!done && it < maxit) {
        // r = b - A x
        if ((rc = tdbem_apply_freq(t, fidx, x, n, w))) break;
        cudaMemcpyAsync(r, b, sizeof(cx<T>) * M * n, cudaMemcpyDeviceToDevice, ctx->stream);
        if ((rc = ops.axpby(r, w, mone, 1.0))) break;
        if ((rc = ops.dot(r, r, tmp))) break;
        std::vector<double> beta(n);
        done = true;
        for (int c = 0; c < n; ++c) {
            beta[c] = std::sqrt(std::max(tmp[c].real(), 0.0));
            res[c] = beta[c] / bnorm[c];
            if (res[c] > tol) done = false;
        }
        if (done) break;
        // V0 = r / beta
        std::vector<C> inv(n);
        for (int c = 0; c < n; ++c) inv[c] = C(beta[c] > 0 ? 1.0 / beta[c] : 0.0, 0.0);
        if ((rc = ops.axpby(V, r, inv, 0.0))) break;
        std::vector<std::vector<C>> H(n, std::vector<C>((m + 1) * m, C(0, 0)));
        std::vector<std::vector<C>> cs(n, std::vector<C>(m)), sn(n, std::vector<C>(m));
        std::vector<std::vector<C>> g(n, std::vector<C>(m + 1, C(0, 0)));
        for (int c = 0; c < n; ++c) g[c][0] = beta[c];
        int j = 0;
        for (; j < m && it < maxit; ++j, ++it) {
            cx<T> *Vj = V + (int64_t)j * M * n, *Vn = V + (int64_t)(j + 1) * M * n;
            if ((rc = tdbem_apply_freq(t, fidx, Vj, n, w))) break;
            for (int i = 0; i <= j; ++i) {
                const cx<T> *Vi = V + (int64_t)i * M * n;
                if ((rc = ops.dot(Vi, w, tmp))) break;
                std::vector<C> neg(n);
                for (int c = 0; c < n; ++c) {
                    H[c][i * m + j] = tmp[c];
                    neg[c] = -tmp[c];
                }
                if ((rc = ops.axpby(w, Vi, neg, 1.0))) break;
            }
            if (rc) break;
            if ((rc = ops.dot(w, w, tmp))) break;
            std::vector<C> inv2(n);
            bool all = true;
            for (int c = 0; c < n; ++c) {
                const double h = std::sqrt(std::max(tmp[c].real(), 0.0));
                H[c][(j + 1) * m + j] = h;
                inv2[c] = C(h > 0 ? 1.0 / h : 0.0, 0.0);
                // Givens rotations on column j
                for (int i = 0; i < j; ++i) {
                    const C a = H[c][i * m + j], bb = H[c][(i + 1) * m + j];
                    H[c][i * m + j] = std::conj(cs[c][i]) * a + std::conj(sn[c][i]) * bb;
                    H[c][(i + 1) * m + j] = -sn[c][i] * a + cs[c][i] * bb;
                }
                const C a = H[c][j * m + j], bb = H[c][(j + 1) * m + j];
                const double den = std::sqrt(std::norm(a) + std::norm(bb));
                if (den > 0) {
                    cs[c][j] = a / den;
                    sn[c][j] = bb / den;
                } else {
                    cs[c][j] = 1.0;
                    sn[c][j] = 0.0;
                }
                H[c][j * m + j] = std::conj(cs[c][j]) * a + std::conj(sn[c][j]) * bb;
                H[c][(j + 1) * m + j] = 0.0;
                const C gj = g[c][j];
                g[c][j] = std::conj(cs[c][j]) * gj;
                g[c][j + 1] = -sn[c][j] * gj;
                res[c] = std::abs(g[c][j + 1]) / bnorm[c];
                if (res[c] > tol) all = false;
            }
            if ((rc = ops.axpby(Vn, w, inv2, 0.0))) break;
            if (all) {
                ++j;
                ++it;
                break;
            }
        }
        if (rc) break;
        // x += V y with H y = g (upper triangular, per column)
        const int kk = j;
        for (int c = 0; c < n; ++c) {
            std::vector<C> yv(kk);
            for (int i = kk - 1; i >= 0; --i) {
                C s = g[c][i];
                for (int l = i + 1; l < kk; ++l) s -= H[c][i * m + l] * yv[l];
                yv[i] = std::abs(H[c][i * m + i]) > 0 ? s / H[c][i * m + i] : C(0, 0);
            }
            g[c].assign(yv.begin(), yv.end());
        }
        for (int i = 0; i < kk && !rc; ++i) {
            std::vector<C> yi(n);
            for (int c = 0; c < n; ++c) yi[c] = g[c][i];
            rc = ops.axpby(x, V + (int64_t)i * M * n, yi, 1.0);
        }
        if (rc) break;
    }
    if (!rc && !done) {
        // explicit final residual (when the loop ended by the true residual
        // test, res holds the explicit residuals of the final x already; a
        // second product would differ from it by the rounding of the apply)
        if (!(rc = tdbem_apply_freq(t, fidx, x, n, w))) {
            cudaMemcpyAsync(r, b, sizeof(cx<T>) * M * n, cudaMemcpyDeviceToDevice, ctx->stream);
            if (!(rc = ops.axpby(r, w, mone, 1.0)) && !(rc = ops.dot(r, r, tmp)))
                for (int c = 0; c < n; ++c) res[c] = std::sqrt(std::max(tmp[c].real(), 0.0)) / bnorm[c];
        }
    }
    cudaStreamSynchronize(ctx->stream);
    cleanup();
    if (iters) *iters = it;
    if (relres)
        for (int c = 0; c < n; ++c) relres[c] = res[c];
    if (rc) return rc;
    for (int c = 0; c < n; ++c)
        if (!(res[c] <= tol * 1.0000001)) return TDBEM_ERR_NOT_CONVERGED;
    return TDBEM_OK;
}

// ---- binary files ------------------------------------------------------------
const char kTensorMagic[8] = {'T', 'D', 'B', 'E', 'M', 'T', '0', '1'};
const char kModelMagic[8] = {'T', 'D', 'B', 'E', 'M', 'M', '0', '1'};

bool wr(FILE *f, const void *p, size_t n) { return n == 0 || fwrite(p, 1, n, f) == n; }
bool rd(FILE *f, void *p, size_t n) { return n == 0 || fread(p, 1, n, f) == n; }

template <class V>
bool wr_dev(FILE *f, const V *d, size_t count) {
    std::vector<V> h(count);
    if (count && cudaMemcpy(h.data(), d, sizeof(V) * count, cudaMemcpyDeviceToHost) != cudaSuccess) return false;
    return wr(f, h.data(), sizeof(V) * count);
}
template <class V>
bool rd_dev(FILE *f, V *d, size_t count) {
    std::vector<V> h(count);
    if (!rd(f, h.data(), sizeof(V) * count)) return false;
    return count == 0 || cudaMemcpy(d, h.data(), sizeof(V) * count, cudaMemcpyHostToDevice) == cudaSuccess;
}

}  // namespace

extern "C" int tdbem_solve(tdbem_tensor_t t, int32_t fidx, const void *b, int32_t nrhs, void *x, double tol,
                           int32_t maxit, int32_t restart, int32_t *iters, double *relres) {
    if (!t) return TDBEM_ERR_ARG;
    tdbem_ctx *ctx = t->ctx;
    cudaGetLastError();
    if (t->nrows != t->ncols) return td_fail(ctx, TDBEM_ERR_ARG, "tdbem_solve needs a square operator (SLP)");
    if (!b || !x || nrhs < 1 || nrhs > 64 || fidx < 0 || fidx >= t->NQ || !(tol > 0.0) || maxit < 1)
        return td_fail(ctx, TDBEM_ERR_ARG, "tdbem_solve: bad arguments");
    const int m = restart > 0 ? std::min(restart, 200) : 30;
    int rc = t->prec == TDBEM_FP64 ? gmres<double>(t, fidx, (const c64 *)b, nrhs, (c64 *)x, tol, maxit, m, iters, relres)
                                   : gmres<float>(t, fidx, (const c32 *)b, nrhs, (c32 *)x, tol, maxit, m, iters, relres);
    if (rc == TDBEM_ERR_NOT_CONVERGED) return td_fail(ctx, rc, "GMRES did not reach the tolerance in %d iterations", maxit);
    if (rc) return td_fail(ctx, rc, "tdbem_solve failed");
    return TDBEM_OK;
}

extern "C" int tdbem_tensor_save(tdbem_tensor_t t, const char *path) {
    if (!t || !path) return TDBEM_ERR_ARG;
    tdbem_ctx *ctx = t->ctx;
    TD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    FILE *f = fopen(path, "wb");
    if (!f) return td_fail(ctx, TDBEM_ERR_ARG, "cannot open %s for writing", path);
    int64_t used = 0;
    cudaMemcpy(&used, t->dface_used, sizeof(int64_t), cudaMemcpyDeviceToHost);
    const size_t es = t->prec == TDBEM_FP64 ? sizeof(c64) : sizeof(c32);
    const int32_t hdr_i[8] = {t->op, t->prec, t->ng, t->Nu, t->NQ, t->kcap, t->max_near_rows, 0};
    const int64_t hdr_l[4] = {t->nrows, t->ncols, t->nblocks, used};
    bool ok = wr(f, kTensorMagic, 8) && wr(f, hdr_i, sizeof hdr_i) && wr(f, hdr_l, sizeof hdr_l) && wr(f, &t->c, sizeof(double)) &&
              wr(f, &t->stats, sizeof t->stats) && wr(f, t->blocks.data(), sizeof(int32_t) * 5 * t->nblocks) &&
              wr(f, t->rank.data(), sizeof(int32_t) * t->nblocks) && wr(f, t->frank_sum.data(), sizeof(int32_t) * t->nblocks) &&
              wr_dev(f, t->dperm_r, t->nrows) && wr_dev(f, t->dperm_c, t->ncols) && wr_dev(f, t->dinv_r, t->nrows) &&
              wr_dev(f, t->dinv_c, t->ncols) && wr_dev(f, t->drank, t->nblocks) && wr_dev(f, t->dkpiv, t->nblocks * t->Nu) &&
              wr_dev(f, t->dfrank, t->nblocks * t->Nu) && wr_dev(f, t->dfoff, t->nblocks * t->Nu) &&
              wr_dev(f, t->dpartner, t->NQ) && wr_dev(f, (const char *)t->dfib, es * t->nblocks * t->Nu * t->Nu) &&
              wr_dev(f, (const char *)t->dface, es * used);
    fclose(f);
    return ok ? TDBEM_OK : td_fail(ctx, TDBEM_ERR_CUDA, "writing %s failed", path);
}

extern "C" int tdbem_tensor_info(tdbem_tensor_t t, int32_t *op, int32_t *prec, int64_t *nrows, int64_t *ncols,
                                 int32_t *NQ, int32_t *Nu) {
    if (!t) return TDBEM_ERR_ARG;
    if (op) *op = t->op;
    if (prec) *prec = t->prec;
    if (nrows) *nrows = t->nrows;
    if (ncols) *ncols = t->ncols;
    if (NQ) *NQ = t->NQ;
    if (Nu) *Nu = t->Nu;
    return TDBEM_OK;
}

extern "C" int tdbem_tensor_load(tdbem_ctx_t ctx, const char *path, tdbem_tensor_t *out) {
    if (!ctx || !path || !out) return TDBEM_ERR_ARG;
    *out = nullptr;
    FILE *f = fopen(path, "rb");
    if (!f) return td_fail(ctx, TDBEM_ERR_ARG, "cannot open %s", path);
    char magic[8];
    int32_t hi[8];
    int64_t hl[4];
    tdbem_tensor *t = new (std::nothrow) tdbem_tensor();
    bool ok = t && rd(f, magic, 8) && !memcmp(magic, kTensorMagic, 8) && rd(f, hi, sizeof hi) && rd(f, hl, sizeof hl);
    if (!ok) {
        fclose(f);
        delete t;
        return td_fail(ctx, TDBEM_ERR_ARG, "%s is not a tensor file of this version", path);
    }
    // sizes must be plausible and account for the file's length exactly
    {
        const int64_t nb = hl[2], nr = hl[0], nc = hl[1], used = hl[3];
        const int Nu = hi[3], NQ = hi[4];
        const bool sane = (hi[0] == TDBEM_SLP || hi[0] == TDBEM_DLP || hi[0] == TDBEM_ADLP) && (hi[1] == TDBEM_FP64 || hi[1] == TDBEM_MIXED) &&
                          Nu >= 1 && Nu <= 256 && NQ >= Nu && NQ <= (1 << 20) && nb >= 1 && nb < (1LL << 31) &&
                          nr >= 1 && nr < (1LL << 31) && nc >= 1 && nc < (1LL << 31) && used >= 0 && used < (1LL << 40);
        const long here = ftell(f);
        const int64_t es = hi[1] == TDBEM_FP64 ? 16 : 8;
        const int64_t expect = here + 8 + (int64_t)sizeof(tdbem_stats) + 4 * (7 * nb) + 4 * (2 * nr + 2 * nc) +
                               4 * nb * (1 + 2 * (int64_t)Nu) + 8 * nb * Nu + 4 * (int64_t)NQ +
                               es * (nb * Nu * Nu + used);
        bool size_ok = false;
        if (sane && here > 0 && fseek(f, 0, SEEK_END) == 0) {
            size_ok = ftell(f) == expect;
            fseek(f, here, SEEK_SET);
        }
        if (!sane || !size_ok) {
            fclose(f);
            delete t;
            return td_fail(ctx, TDBEM_ERR_ARG, "%s: header sizes do not match the file", path);
        }
    }
    t->ctx = ctx;
    t->op = hi[0];
    t->prec = hi[1];
    t->ng = hi[2];
    t->Nu = hi[3];
    t->NQ = hi[4];
    t->kcap = hi[5];
    t->max_near_rows = hi[6];
    t->nrows = hl[0];
    t->ncols = hl[1];
    t->nblocks = hl[2];
    const int64_t used = hl[3], nb = t->nblocks;
    const size_t es = t->prec == TDBEM_FP64 ? sizeof(c64) : sizeof(c32);
    t->blocks.resize(5 * nb);
    t->rank.resize(nb);
    t->frank_sum.resize(nb);
    auto alloc = [&](void **p, size_t bytes) {
        if (cudaMalloc(p, std::max<size_t>(bytes, 1)) != cudaSuccess) return false;
        t->owned.push_back(*p);
        return true;
    };
    ok = rd(f, &t->c, sizeof(double)) && rd(f, &t->stats, sizeof t->stats) &&
         rd(f, t->blocks.data(), sizeof(int32_t) * 5 * nb) && rd(f, t->rank.data(), sizeof(int32_t) * nb) &&
         rd(f, t->frank_sum.data(), sizeof(int32_t) * nb) && alloc((void **)&t->dblocks, sizeof(int32_t) * 5 * nb) &&
         alloc((void **)&t->dperm_r, sizeof(int32_t) * t->nrows) && alloc((void **)&t->dperm_c, sizeof(int32_t) * t->ncols) &&
         alloc((void **)&t->dinv_r, sizeof(int32_t) * t->nrows) && alloc((void **)&t->dinv_c, sizeof(int32_t) * t->ncols) &&
         alloc((void **)&t->drank, sizeof(int32_t) * nb) && alloc((void **)&t->dkpiv, sizeof(int32_t) * nb * t->Nu) &&
         alloc((void **)&t->dfrank, sizeof(int32_t) * nb * t->Nu) && alloc((void **)&t->dfoff, sizeof(int64_t) * nb * t->Nu) &&
         alloc((void **)&t->dpartner, sizeof(int32_t) * (t->NQ + 1)) && alloc(&t->dfib, es * nb * t->Nu * t->Nu) &&
         alloc(&t->dface, es * used) && alloc((void **)&t->dface_used, sizeof(int64_t) * 2) &&
         cudaMemcpy(t->dblocks, t->blocks.data(), sizeof(int32_t) * 5 * nb, cudaMemcpyHostToDevice) == cudaSuccess &&
         rd_dev(f, t->dperm_r, t->nrows) && rd_dev(f, t->dperm_c, t->ncols) && rd_dev(f, t->dinv_r, t->nrows) &&
         rd_dev(f, t->dinv_c, t->ncols) && rd_dev(f, t->drank, nb) && rd_dev(f, t->dkpiv, nb * t->Nu) &&
         rd_dev(f, t->dfrank, nb * t->Nu) && rd_dev(f, t->dfoff, nb * t->Nu) && rd_dev(f, t->dpartner, t->NQ) &&
         rd_dev(f, (char *)t->dfib, es * nb * t->Nu * t->Nu) && rd_dev(f, (char *)t->dface, es * used) &&
         cudaMemcpy(t->dface_used, &used, sizeof(int64_t), cudaMemcpyHostToDevice) == cudaSuccess;
    fclose(f);
    if (!ok) {
        cudaGetLastError();
        for (void *p : t->owned) cudaFree(p);
        delete t;
        return td_fail(ctx, TDBEM_ERR_ARG, "reading %s failed", path);
    }
    t->face_cap = used;
    *out = t;
    return TDBEM_OK;
}

extern "C" int tdbem_model_save(tdbem_model_t m, const char *path) {
    if (!m || !path) return TDBEM_ERR_ARG;
    std::vector<float> p(TD_MLP_NPARAMS);
    int rc = tdbem_model_get_params(m, p.data());
    if (rc) return rc;
    FILE *f = fopen(path, "wb");
    if (!f) return TDBEM_ERR_ARG;
    const int32_t n = TD_MLP_NPARAMS;
    const bool ok = wr(f, kModelMagic, 8) && wr(f, &n, sizeof n) && wr(f, p.data(), sizeof(float) * n);
    fclose(f);
    return ok ? TDBEM_OK : TDBEM_ERR_ARG;
}

extern "C" int tdbem_model_load(tdbem_ctx_t ctx, const char *path, tdbem_model_t *out) {
    if (!ctx || !path || !out) return TDBEM_ERR_ARG;
    *out = nullptr;
    FILE *f = fopen(path, "rb");
    if (!f) return td_fail(ctx, TDBEM_ERR_ARG, "cannot open %s", path);
    char magic[8];
    int32_t n = 0;
    std::vector<float> p(TD_MLP_NPARAMS);
    const bool ok = rd(f, magic, 8) && !memcmp(magic, kModelMagic, 8) && rd(f, &n, sizeof n) && n == TD_MLP_NPARAMS &&
                    rd(f, p.data(), sizeof(float) * n);
    fclose(f);
    if (!ok) return td_fail(ctx, TDBEM_ERR_ARG, "%s is not a model file of this version", path);
    int rc = tdbem_model_create(ctx, 0, out);
    if (rc) return rc;
    return tdbem_model_set_params(*out, p.data());
}
