// Learned rank predictor (C-ABI part): block features, face-rank harvest,
// training loop, inference and the presizing table used by the compressor.
//
// Features of a far block (I, J) at frequency s (dimensionless, so that
// meshes of different size and wave speed share one model):
//   log(diam_I / dist), log(diam_J / dist), log(dist / h), min(diam)/dist,
//   log(1 + Re(s) dist / c), log(1 + |Im(s)| dist / c),
// with h the mean edge length of the mesh, diam the box diagonal and dist
// the box distance of the two clusters (the quantities of eq. admissible).
// Target: the rank bin of the ACA of the plain face A(., ., s) at eps_aca.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <random>

#include "internal.h"
#include "kernels.h"
#include "mlp.h"
#include "pair.cuh"

static const int kBinUpper[TDBEM_NBINS] = {1, 2, 3, 4, 6, 8, 10, 12, 16, 20, 24, 32, 40, 48, 64, 1 << 30};

extern "C" int tdbem_rank_bin(int32_t rank) {
    for (int b = 0; b < TDBEM_NBINS; ++b)
        if (rank <= kBinUpper[b]) return b;
    return TDBEM_NBINS - 1;
}

// lower edge of a bin: the rank the compressor may run without checks
static int bin_lower(int b) { return b == 0 ? 1 : kBinUpper[b - 1] + 1; }

struct tdbem_model {
    tdbem_ctx *ctx = nullptr;
    float *P = nullptr, *m = nullptr, *v = nullptr, *G = nullptr, *loss = nullptr;  // device
    void *Pb = nullptr;                                                             // BF16 copy
    int step = 0;
    bool bf16_stale = true;
    void *pbuf = nullptr;  // presizing buffers (grown on demand)
    size_t pbytes = 0;
};

namespace {

int model_bf16(tdbem_model *M) {
    if (!M->bf16_stale) return TDBEM_OK;
    if (td_mlp_to_bf16(M->ctx->stream, M->P, M->Pb)) return td_fail(M->ctx, TDBEM_ERR_CUDA, "bf16 conversion failed");
    M->bf16_stale = false;
    return TDBEM_OK;
}

const ClusterNode *find_node(const HostTree &t, int32_t b, int32_t e) {
    // clusters are nested ranges; walk from the root
    int32_t id = 0;
    for (;;) {
        const ClusterNode &n = t.nodes[id];
        if (n.begin == b && n.end == e) return &n;
        if (n.son0 < 0) return nullptr;
        id = (b < t.nodes[n.son0].end) ? n.son0 : n.son1;
    }
}

double diag(const ClusterNode &a) {
    double s = 0.0;
    for (int k = 0; k < 3; ++k) s += (a.box[3 + k] - a.box[k]) * (a.box[3 + k] - a.box[k]);
    return std::sqrt(s);
}

double gap(const ClusterNode &a, const ClusterNode &b) {
    double s = 0.0;
    for (int k = 0; k < 3; ++k) {
        double g = std::max(0.0, std::max(b.box[k] - a.box[3 + k], a.box[k] - b.box[3 + k]));
        s += g * g;
    }
    return std::sqrt(s);
}

}  // namespace

// Host features [far.size() * Nu][6] for the far blocks listed in `far`.
void td_block_features(const tdbem_tree *t, const std::vector<int32_t> &blocks, const tdbem_mesh *m,
                       const tdbem_freqs *f, double c, const std::vector<int32_t> &far, std::vector<float> &x) {
    double h = 0.0;
    for (int64_t e = 0; e < m->nt; ++e)
        for (int k = 0; k < 3; ++k) {
            const double *a = &m->verts[3 * m->tris[3 * e + k]], *b = &m->verts[3 * m->tris[3 * e + (k + 1) % 3]];
            h += std::sqrt((a[0] - b[0]) * (a[0] - b[0]) + (a[1] - b[1]) * (a[1] - b[1]) + (a[2] - b[2]) * (a[2] - b[2]));
        }
    h /= (3.0 * m->nt);
    const int Nu = f->Nu;
    x.assign(far.size() * Nu * TD_MLP_NFEAT, 0.0f);
    for (size_t n = 0; n < far.size(); ++n) {
        const int32_t *bl = &blocks[5 * far[n]];
        const ClusterNode *A = find_node(t->side[0], bl[0], bl[1]), *B = find_node(t->side[1], bl[2], bl[3]);
        const double da = A ? diag(*A) : 0.0, db = B ? diag(*B) : 0.0;
        const double ds = (A && B) ? std::max(gap(*A, *B), 1e-300) : 1.0;
        for (int u = 0; u < Nu; ++u) {
            const double sr = f->s[2 * f->uidx[u]], si = f->s[2 * f->uidx[u] + 1];
            float *o = &x[(n * Nu + u) * TD_MLP_NFEAT];
            o[0] = (float)std::log(std::max(da, 1e-300) / ds);
            o[1] = (float)std::log(std::max(db, 1e-300) / ds);
            o[2] = (float)std::log(ds / h);
            o[3] = (float)(std::min(da, db) / ds);
            o[4] = (float)std::log1p(std::max(0.0, sr) * ds / c);
            o[5] = (float)std::log1p(std::fabs(si) * ds / c);
        }
    }
}

// Predicted first trip counts per (block id, unique frequency) for the far
// blocks, written to the device array dkpred [nb][Nu] (entries of other
// blocks untouched); per far block the predicted cost len * sum kp^2 and
// ks = max_u min(kp, kcap) (face-pool presizing).  The block features are
// formed on the host (7652 blocks: a fraction of a millisecond), the
// frequency features and the MLP on the device.
int td_predict_kpred(tdbem_model *M, const tdbem_tree *t, const std::vector<int32_t> &blocks, const tdbem_mesh *m,
                     const tdbem_freqs *f, double c, const std::vector<int32_t> &far, int kcap, int32_t *dkpred,
                     std::vector<double> &cost, std::vector<int32_t> &ks) {
    tdbem_ctx *ctx = M->ctx;
    const int Nu = f->Nu;
    const int nfar = (int)far.size();
    cost.assign(nfar, 0.0);
    ks.assign(nfar, 0);
    if (nfar == 0) return TDBEM_OK;
    double h = 0.0;
    for (int64_t e = 0; e < m->nt; ++e)
        for (int k = 0; k < 3; ++k) {
            const double *a = &m->verts[3 * m->tris[3 * e + k]], *b = &m->verts[3 * m->tris[3 * e + (k + 1) % 3]];
            h += std::sqrt((a[0] - b[0]) * (a[0] - b[0]) + (a[1] - b[1]) * (a[1] - b[1]) + (a[2] - b[2]) * (a[2] - b[2]));
        }
    h /= (3.0 * m->nt);
    // host staging: bfeat [nfar][5] | ffeat [Nu][2] | far [nfar] | len [nfar] (4-byte words)
    const size_t nw = (size_t)nfar * 5 + (size_t)Nu * 2 + (size_t)nfar * 2;
    std::vector<uint32_t> host(nw);
    float *bf = reinterpret_cast<float *>(host.data());
    float *ff = bf + (size_t)nfar * 5;
    int32_t *hfar = reinterpret_cast<int32_t *>(ff + (size_t)Nu * 2);
    int32_t *hlen = hfar + nfar;
    for (int q = 0; q < nfar; ++q) {
        const int32_t *bl = &blocks[5 * far[q]];
        const ClusterNode *A = find_node(t->side[0], bl[0], bl[1]), *B = find_node(t->side[1], bl[2], bl[3]);
        const double da = A ? diag(*A) : 0.0, db = B ? diag(*B) : 0.0;
        const double ds = (A && B) ? std::max(gap(*A, *B), 1e-300) : 1.0;
        float *o = bf + (size_t)q * 5;
        o[0] = (float)std::log(std::max(da, 1e-300) / ds);
        o[1] = (float)std::log(std::max(db, 1e-300) / ds);
        o[2] = (float)std::log(ds / h);
        o[3] = (float)(std::min(da, db) / ds);
        o[4] = (float)ds;
        hfar[q] = far[q];
        hlen[q] = (bl[1] - bl[0]) + (bl[3] - bl[2]);
    }
    for (int u = 0; u < Nu; ++u) {
        ff[2 * u] = (float)(f->s[2 * f->uidx[u]] / c);
        ff[2 * u + 1] = (float)(std::fabs(f->s[2 * f->uidx[u] + 1]) / c);
    }
    // device buffers (kept by the model, grown when needed): staging + ks [nfar] + cost [nfar]
    const size_t need = sizeof(uint32_t) * (nw + 2 * (size_t)nfar);
    if (need > M->pbytes) {
        if (M->pbuf) cudaFree(M->pbuf);
        M->pbuf = nullptr;
        M->pbytes = 0;
        if (cudaMalloc(&M->pbuf, need) != cudaSuccess) {
            cudaGetLastError();
            return td_fail(ctx, TDBEM_ERR_OOM, "predictor buffers");
        }
        M->pbytes = need;
    }
    int rc = model_bf16(M);
    if (rc) return rc;
    uint32_t *dev = (uint32_t *)M->pbuf;
    const float *dbf = (const float *)dev;
    const float *dff = dbf + (size_t)nfar * 5;
    const int32_t *dfar = (const int32_t *)(dff + (size_t)Nu * 2);
    const int32_t *dlen = dfar + nfar;
    int32_t *dks = (int32_t *)(dlen + nfar);
    float *dcost = (float *)(dks + nfar);
    std::vector<float> hcost(nfar);
    if (cudaMemcpyAsync(dev, host.data(), sizeof(uint32_t) * nw, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess ||
        cudaMemsetAsync(dks, 0, sizeof(int32_t) * 2 * nfar, ctx->stream) != cudaSuccess ||
        td_mlp_presize(ctx->stream, M->Pb, dbf, dff, nfar, Nu, dfar, dlen, kcap, dkpred, dks, dcost, ctx->num_sms) ||
        cudaMemcpyAsync(ks.data(), dks, sizeof(int32_t) * nfar, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
        cudaMemcpyAsync(hcost.data(), dcost, sizeof(float) * nfar, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
        cudaStreamSynchronize(ctx->stream) != cudaSuccess)
        return td_fail(ctx, TDBEM_ERR_CUDA, "predictor presizing failed");
    for (int q = 0; q < nfar; ++q) cost[q] = hcost[q];
    return TDBEM_OK;
}

extern "C" int tdbem_model_create(tdbem_ctx_t ctx, uint64_t seed, tdbem_model_t *out) {
    if (!ctx || !out) return TDBEM_ERR_ARG;
    *out = nullptr;
    tdbem_model *M = new (std::nothrow) tdbem_model();
    if (!M) return TDBEM_ERR_OOM;
    M->ctx = ctx;
    float *base = nullptr;
    if (cudaMalloc(&base, sizeof(float) * (4 * TD_MLP_NPARAMS + 8) + sizeof(uint16_t) * TD_MLP_NPARAMS) != cudaSuccess) {
        cudaGetLastError();
        delete M;
        return td_fail(ctx, TDBEM_ERR_OOM, "model allocation failed");
    }
    M->P = base;
    M->m = base + TD_MLP_NPARAMS;
    M->v = base + 2 * TD_MLP_NPARAMS;
    M->G = base + 3 * TD_MLP_NPARAMS;
    M->loss = base + 4 * TD_MLP_NPARAMS;
    M->Pb = base + 4 * TD_MLP_NPARAMS + 8;
    cudaMemsetAsync(M->m, 0, sizeof(float) * 2 * TD_MLP_NPARAMS, ctx->stream);
    if (td_mlp_init(ctx->stream, M->P, seed)) {
        cudaFree(base);
        delete M;
        return td_fail(ctx, TDBEM_ERR_CUDA, "model init kernel failed");
    }
    *out = M;
    return TDBEM_OK;
}

extern "C" int tdbem_model_destroy(tdbem_model_t M) {
    if (M) {
        cudaFree(M->P);
        if (M->pbuf) cudaFree(M->pbuf);
        delete M;
    }
    return TDBEM_OK;
}

extern "C" int tdbem_model_get_params(tdbem_model_t M, float *host) {
    if (!M || !host) return TDBEM_ERR_ARG;
    TD_CUDA(M->ctx, cudaMemcpyAsync(host, M->P, sizeof(float) * TD_MLP_NPARAMS, cudaMemcpyDeviceToHost, M->ctx->stream));
    TD_CUDA(M->ctx, cudaStreamSynchronize(M->ctx->stream));
    return TDBEM_OK;
}

extern "C" int tdbem_model_set_params(tdbem_model_t M, const float *host) {
    if (!M || !host) return TDBEM_ERR_ARG;
    TD_CUDA(M->ctx, cudaMemcpyAsync(M->P, host, sizeof(float) * TD_MLP_NPARAMS, cudaMemcpyHostToDevice, M->ctx->stream));
    TD_CUDA(M->ctx, cudaMemsetAsync(M->m, 0, sizeof(float) * 2 * TD_MLP_NPARAMS, M->ctx->stream));
    TD_CUDA(M->ctx, cudaStreamSynchronize(M->ctx->stream));
    M->step = 0;
    M->bf16_stale = true;
    return TDBEM_OK;
}

extern "C" int tdbem_model_loss_grad(tdbem_model_t M, const float *x, const int32_t *labels, int64_t n, float *grad,
                                     float *loss) {
    if (!M || n < 1 || !x || !labels || !grad || !loss) return TDBEM_ERR_ARG;
    cudaGetLastError();
    if (td_mlp_grad(M->ctx->stream, M->P, x, labels, n, grad, loss, M->ctx->num_sms))
        return td_fail(M->ctx, TDBEM_ERR_CUDA, "gradient kernel failed");
    return TDBEM_OK;
}

extern "C" int tdbem_model_adam_step(tdbem_model_t M, const float *grad, double lr, int32_t t) {
    if (!M || !grad || t < 1) return TDBEM_ERR_ARG;
    if (td_mlp_adam(M->ctx->stream, M->P, grad, M->m, M->v, (float)lr, 0.9f, 0.999f, 1e-8f, t))
        return td_fail(M->ctx, TDBEM_ERR_CUDA, "adam kernel failed");
    M->bf16_stale = true;
    return TDBEM_OK;
}

extern "C" int tdbem_model_train(tdbem_model_t M, const float *x, const int32_t *labels, int64_t n, int32_t epochs,
                                 int32_t batch, double lr, uint64_t seed, double *final_loss) {
    if (!M || !x || !labels || n < 1 || epochs < 1 || batch < 1) return TDBEM_ERR_ARG;
    tdbem_ctx *ctx = M->ctx;
    cudaGetLastError();
    // shuffle once (seeded) into private copies, then sweep contiguous batches
    std::vector<float> hx(n * TD_MLP_NFEAT);
    std::vector<int32_t> hl(n);
    TD_CUDA(ctx, cudaMemcpyAsync(hx.data(), x, sizeof(float) * hx.size(), cudaMemcpyDeviceToHost, ctx->stream));
    TD_CUDA(ctx, cudaMemcpyAsync(hl.data(), labels, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, ctx->stream));
    TD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    std::vector<int64_t> perm(n);
    for (int64_t k = 0; k < n; ++k) perm[k] = k;
    std::mt19937_64 rng(seed);
    std::shuffle(perm.begin(), perm.end(), rng);
    std::vector<float> sx(hx.size());
    std::vector<int32_t> sl(n);
    for (int64_t k = 0; k < n; ++k) {
        std::memcpy(&sx[k * TD_MLP_NFEAT], &hx[perm[k] * TD_MLP_NFEAT], sizeof(float) * TD_MLP_NFEAT);
        sl[k] = hl[perm[k]];
    }
    float *dx = nullptr;
    int32_t *dl = nullptr;
    if (cudaMalloc(&dx, sizeof(float) * sx.size()) != cudaSuccess || cudaMalloc(&dl, sizeof(int32_t) * n) != cudaSuccess) {
        cudaFree(dx);
        return td_fail(ctx, TDBEM_ERR_OOM, "training buffers");
    }
    cudaMemcpyAsync(dx, sx.data(), sizeof(float) * sx.size(), cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(dl, sl.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, ctx->stream);
    int rc = TDBEM_OK;
    for (int ep = 0; ep < epochs && !rc; ++ep)
        for (int64_t b0 = 0; b0 < n && !rc; b0 += batch) {
            const int64_t nb = std::min<int64_t>(batch, n - b0);
            if (td_mlp_grad(ctx->stream, M->P, dx + b0 * TD_MLP_NFEAT, dl + b0, nb, M->G, M->loss, ctx->num_sms) ||
                td_mlp_adam(ctx->stream, M->P, M->G, M->m, M->v, (float)lr, 0.9f, 0.999f, 1e-8f, ++M->step))
                rc = td_fail(ctx, TDBEM_ERR_CUDA, "training kernels failed");
        }
    if (!rc && final_loss) {
        // loss over the whole set with the final weights
        if (td_mlp_grad(ctx->stream, M->P, dx, dl, n, M->G, M->loss, ctx->num_sms)) {
            rc = td_fail(ctx, TDBEM_ERR_CUDA, "loss kernel failed");
        } else {
            float hloss = 0.0f;
            cudaMemcpyAsync(&hloss, M->loss, sizeof(float), cudaMemcpyDeviceToHost, ctx->stream);
            cudaStreamSynchronize(ctx->stream);
            *final_loss = hloss;
        }
    }
    cudaStreamSynchronize(ctx->stream);
    cudaFree(dx);
    cudaFree(dl);
    M->bf16_stale = true;
    return rc;
}

extern "C" int tdbem_model_predict(tdbem_model_t M, const float *x, int64_t n, int32_t *bins, float *logits) {
    if (!M || n < 0 || (n > 0 && !x)) return TDBEM_ERR_ARG;
    cudaGetLastError();
    int rc = model_bf16(M);
    if (rc) return rc;
    if (td_mlp_predict(M->ctx->stream, M->Pb, x, n, bins, logits, M->ctx->num_sms))
        return td_fail(M->ctx, TDBEM_ERR_CUDA, "predict kernel failed");
    return TDBEM_OK;
}
