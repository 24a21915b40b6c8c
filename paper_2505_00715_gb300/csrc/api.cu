// C-ABI of the tdbem library (include/tdbem.h): handles, argument checks,
// device tables, and the orchestration of the compression phases
// (touching-pair table -> near-field entries -> near 3D-ACA -> far 3D-ACA),
// each a single persistent launch, captured together in a CUDA graph.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>

#include "internal.h"
#include "kernels.h"
#include "pair.cuh"

int td_fail(tdbem_ctx *ctx, int code, const char *fmt, ...) {
    if (code == TDBEM_ERR_CUDA || code == TDBEM_ERR_OOM) cudaGetLastError();  // clear non-sticky errors
    if (ctx) {
        char buf[1024];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return code;
}

namespace {

double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

template <class T>
int dalloc(tdbem_ctx *ctx, T **p, size_t count, std::vector<void *> *owned = nullptr) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, sizeof(T) * count);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return td_fail(ctx, TDBEM_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", sizeof(T) * count,
                       cudaGetErrorString(e));
    }
    if (owned) owned->push_back((void *)*p);
    return TDBEM_OK;
}

template <class T>
int upload(tdbem_ctx *ctx, T *dst, const T *src, size_t count) {
    if (count == 0) return TDBEM_OK;
    TD_CUDA(ctx, cudaMemcpyAsync(dst, src, sizeof(T) * count, cudaMemcpyHostToDevice, ctx->stream));
    return TDBEM_OK;
}

// terms of Algorithm 1 per far block assumed when the face pool is presized
// from predicted face ranks (the far blocks of the benchmark meshes take 7-9
// on average, at most 16)
constexpr int64_t kTermsEst = 8;

struct Guard {
    // frees transient device buffers at scope exit (or earlier, by release())
    std::vector<void *> p;
    void release() {
        for (void *q : p) cudaFree(q);
        p.clear();
    }
    ~Guard() { release(); }
};

}  // namespace

MeshDev td_mesh_dev(const tdbem_mesh *m, int ng, const double *gx, const double *gw, const int *tp_slot) {
    MeshDev d{};
    d.nt = (int)m->nt;
    d.nv = (int)m->nv;
    d.qxh = m->qxh;
    d.qyh = m->qyh;
    d.qzh = m->qzh;
    d.qxl = m->qxl;
    d.qyl = m->qyl;
    d.qzl = m->qzl;
    d.qw32 = m->qw32;
    d.n32 = m->n32;
    d.qp = (const float4 *)m->qp;
    d.nrm4 = (const float4 *)m->nrm4;
    d.qx = m->qx;
    d.qy = m->qy;
    d.qz = m->qz;
    d.qw = m->qw;
    d.n64 = m->n64;
    d.verts = m->dverts;
    d.tris = m->dtris;
    d.area = m->darea;
    d.v2t_ptr = m->dv2t_ptr;
    d.v2t = m->dv2t;
    d.v2t_loc = (const signed char *)m->dv2t_loc;
    d.tp_ptr = m->dtp_ptr;
    d.tp_tri = m->dtp_tri;
    d.tp_slot = tp_slot;
    d.ng = ng;
    d.gx = gx;
    d.gw = gw;
    return d;
}

int td_check_op(tdbem_ctx *ctx, const tdbem_op *op) {
    if (!op) return td_fail(ctx, TDBEM_ERR_ARG, "op is NULL");
    if (op->op != TDBEM_SLP && op->op != TDBEM_DLP && op->op != TDBEM_ADLP)
        return td_fail(ctx, TDBEM_ERR_ARG, "unknown operator %d", op->op);
    if (op->prec != TDBEM_FP64 && op->prec != TDBEM_MIXED) return td_fail(ctx, TDBEM_ERR_ARG, "unknown precision %d", op->prec);
    if (!(op->c > 0.0) || !std::isfinite(op->c)) return td_fail(ctx, TDBEM_ERR_ARG, "wave speed must be > 0");
    if (op->ng < 1 || op->ng > 16) return td_fail(ctx, TDBEM_ERR_ARG, "ng must be in 1..16");
    return TDBEM_OK;
}

namespace {

// Gauss nodes and touching-pair slots for one operator (device, owned by caller)
int prepare_sing(tdbem_ctx *ctx, const tdbem_mesh *m, int op, int ng, std::vector<void *> &owned,
                 double **gx, double **gw, int **tp_slot, int **pti, int **ptj, int *npairs) {
    double hx[32], hw[32];
    td_gauss01(ng, hx, hw);
    int rc;
    if ((rc = dalloc(ctx, gx, 64, &owned))) return rc;
    *gw = *gx + 32;
    if ((rc = upload(ctx, *gx, hx, ng)) || (rc = upload(ctx, *gw, hw, ng))) return rc;
    const int64_t np = m->tp_tri.size();
    std::vector<int32_t> slot(np, -1), ti, tj;
    for (int64_t i = 0; i < m->nt; ++i)
        for (int32_t p = m->tp_ptr[i]; p < m->tp_ptr[i + 1]; ++p) {
            const int32_t j = m->tp_tri[p];
            if (op != TDBEM_SLP || i <= j) {  // the single layer is symmetric: unordered pairs
                slot[p] = (int32_t)ti.size();
                ti.push_back((int32_t)i);
                tj.push_back(j);
            }
        }
    if (op == TDBEM_SLP)
        for (int64_t i = 0; i < m->nt; ++i)
            for (int32_t p = m->tp_ptr[i]; p < m->tp_ptr[i + 1]; ++p) {
                const int32_t j = m->tp_tri[p];
                if (i > j) {
                    const int32_t *b = m->tp_tri.data() + m->tp_ptr[j], *e = m->tp_tri.data() + m->tp_ptr[j + 1];
                    const int32_t *f = std::lower_bound(b, e, (int32_t)i);
                    slot[p] = slot[f - m->tp_tri.data()];
                }
            }
    *npairs = (int)ti.size();
    if ((rc = dalloc(ctx, tp_slot, np, &owned)) || (rc = dalloc(ctx, pti, ti.size(), &owned)) ||
        (rc = dalloc(ctx, ptj, tj.size(), &owned)))
        return rc;
    if ((rc = upload(ctx, *tp_slot, slot.data(), np)) || (rc = upload(ctx, *pti, ti.data(), ti.size())) ||
        (rc = upload(ctx, *ptj, tj.data(), tj.size())))
        return rc;
    return TDBEM_OK;
}

}  // namespace

// ============================================================================
// context
// ============================================================================
extern "C" int tdbem_ctx_create(int device, void *stream, tdbem_ctx_t *out) {
    if (!out) return TDBEM_ERR_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return TDBEM_ERR_CUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return TDBEM_ERR_CUDA;
    tdbem_ctx *c = new (std::nothrow) tdbem_ctx();
    if (!c) return TDBEM_ERR_OOM;
    c->device = device;
    c->stream = (cudaStream_t)stream;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    // graphs cannot be captured on the legacy default stream: capture on a
    // private stream and launch the instantiated graph on the caller's stream
    if (cudaStreamCreateWithFlags(&c->capture, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return TDBEM_ERR_CUDA;
    }
    if (td_noalloc_setup(device) != TDBEM_OK || cudaMalloc(&c->dflags, sizeof(int)) != cudaSuccess ||
        cudaMemset(c->dflags, 0, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        cudaStreamDestroy(c->capture);
        delete c;
        return TDBEM_ERR_CUDA;
    }
    *out = c;
    return TDBEM_OK;
}

extern "C" int tdbem_ctx_destroy(tdbem_ctx_t ctx) {
    if (ctx && ctx->capture) cudaStreamDestroy(ctx->capture);
    if (ctx && ctx->dflags) cudaFree(ctx->dflags);
    delete ctx;
    return TDBEM_OK;
}

extern "C" const char *tdbem_last_error(tdbem_ctx_t ctx) { return ctx ? ctx->err.c_str() : "no context"; }

extern "C" int tdbem_ctx_set_near_batch(tdbem_ctx_t ctx, int64_t bytes) {
    if (!ctx) return TDBEM_ERR_ARG;
    if (bytes <= 0) return td_fail(ctx, TDBEM_ERR_ARG, "near batch size must be > 0");
    ctx->near_batch_bytes = bytes;
    return TDBEM_OK;
}

extern "C" int tdbem_measure_peak(tdbem_ctx_t ctx, int32_t what, double *ops_per_s) {
    if (!ctx || !ops_per_s || what < 0 || what > 3) return TDBEM_ERR_ARG;
    const int grid = ctx->num_sms * 8;
    const int iters = what == 3 ? 128 : what == 2 ? 64 : 2048;
    double *out = nullptr;
    int rc = dalloc(ctx, &out, (size_t)grid);
    if (rc) return rc;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double ops = 0.0;
    int lr = td_launch_peak(ctx->stream, what, grid, iters, out, &ops);  // warm-up
    cudaEventRecord(e0, ctx->stream);
    lr |= td_launch_peak(ctx->stream, what, grid, iters, out, &ops);
    cudaEventRecord(e1, ctx->stream);
    const cudaError_t se = cudaStreamSynchronize(ctx->stream);
    float ms = 0.0f;
    const bool timed = se == cudaSuccess && !lr && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.0f;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (!timed) return td_fail(ctx, TDBEM_ERR_CUDA, "peak microbenchmark failed: %s", cudaGetErrorString(se));
    *ops_per_s = ops / (ms * 1e-3);
    return TDBEM_OK;
}

extern "C" int tdbem_ctx_set_wait_limit(tdbem_ctx_t ctx, int64_t polls) {
    if (!ctx) return TDBEM_ERR_ARG;
    if (polls < 0 || polls > INT32_MAX) return td_fail(ctx, TDBEM_ERR_ARG, "wait limit must be in 0..2^31-1");
    ctx->wait_polls = (uint32_t)polls;
    return TDBEM_OK;
}

extern "C" int tdbem_ctx_set_pool_scale(tdbem_ctx_t ctx, double scale) {
    if (!ctx) return TDBEM_ERR_ARG;
    if (!(scale > 0.0)) return td_fail(ctx, TDBEM_ERR_ARG, "pool scale must be > 0");
    ctx->pool_scale = scale;
    return TDBEM_OK;
}

extern "C" int tdbem_ctx_sync(tdbem_ctx_t ctx) {
    if (!ctx) return TDBEM_ERR_ARG;
    TD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    int fl = 0;
    TD_CUDA(ctx, cudaMemcpy(&fl, ctx->dflags, sizeof(int), cudaMemcpyDeviceToHost));
    if (fl & TD_DEV_TIMEOUT) {
        cudaMemset(ctx->dflags, 0, sizeof(int));
        return td_fail(ctx, TDBEM_ERR_CUDA, "a tensor-core wait of an earlier call gave up (its result is invalid)");
    }
    return TDBEM_OK;
}

// ============================================================================
// mesh
// ============================================================================
extern "C" int tdbem_mesh_create(tdbem_ctx_t ctx, const double *verts, int64_t nv, const int32_t *tris,
                                 int64_t nt, tdbem_mesh_t *out) {
    if (!ctx || !out || !verts || !tris || nv < 3 || nt < 1 || nt > (1 << 30) || nv > (1 << 30))
        return td_fail(ctx, TDBEM_ERR_ARG, "tdbem_mesh_create: bad arguments");
    *out = nullptr;
    for (int64_t k = 0; k < 3 * nv; ++k)
        if (!std::isfinite(verts[k])) return td_fail(ctx, TDBEM_ERR_ARG, "non-finite vertex coordinate at %lld", (long long)k);
    for (int64_t k = 0; k < 3 * nt; ++k)
        if (tris[k] < 0 || tris[k] >= nv) return td_fail(ctx, TDBEM_ERR_ARG, "triangle index out of range at %lld", (long long)k);
    tdbem_mesh *m = new (std::nothrow) tdbem_mesh();
    if (!m) return td_fail(ctx, TDBEM_ERR_OOM, "host allocation failed");
    m->ctx = ctx;
    m->nv = nv;
    m->nt = nt;
    m->verts.assign(verts, verts + 3 * nv);
    m->tris.assign(tris, tris + 3 * nt);
    m->area.resize(nt);
    std::vector<double> nrm(3 * nt);
    for (int64_t e = 0; e < nt; ++e) {
        const double *a = verts + 3 * tris[3 * e], *b = verts + 3 * tris[3 * e + 1], *c = verts + 3 * tris[3 * e + 2];
        const double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
        const double v[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
        const double n[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
        const double len = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        if (!(len > 0.0)) {
            delete m;
            return td_fail(ctx, TDBEM_ERR_ARG, "degenerate triangle %lld", (long long)e);
        }
        m->area[e] = 0.5 * len;
        for (int k = 0; k < 3; ++k) nrm[k * nt + e] = n[k] / len;
    }
    td_mesh_adjacency(m);
    // 7-point tables [7][nt]
    double bary[7][3], w7[7];
    td_rule7(bary, w7);
    std::vector<double> q(3 * 7 * nt), qw(7 * nt);
    std::vector<float> qh(3 * 7 * nt), ql(3 * 7 * nt), qw32(7 * nt), n32(3 * nt);
    for (int64_t e = 0; e < nt; ++e)
        for (int p = 0; p < 7; ++p) {
            for (int c = 0; c < 3; ++c) {
                double x = 0.0;
                for (int k = 0; k < 3; ++k) x += bary[p][k] * verts[3 * tris[3 * e + k] + c];
                const int64_t o = ((int64_t)c * 7 + p) * nt + e;
                q[o] = x;
                qh[o] = (float)x;
                ql[o] = (float)(x - (double)qh[o]);
            }
            qw[p * nt + e] = w7[p] * m->area[e];
            qw32[p * nt + e] = (float)qw[p * nt + e];
        }
    for (int64_t k = 0; k < 3 * nt; ++k) n32[k] = (float)nrm[k];
    // 16-byte packs: (hi xyz, weight) and (lo xyz, 0) per point, (normal, 0) per triangle
    std::vector<float> qp(8 * 7 * (size_t)nt), nrm4(4 * (size_t)nt, 0.f);
    for (int64_t e = 0; e < nt; ++e) {
        for (int p = 0; p < 7; ++p) {
            float *o = &qp[8 * ((size_t)p * nt + e)];
            for (int c = 0; c < 3; ++c) {
                o[c] = qh[((int64_t)c * 7 + p) * nt + e];
                o[4 + c] = ql[((int64_t)c * 7 + p) * nt + e];
            }
            o[3] = qw32[p * nt + e];
            o[7] = 0.f;
        }
        for (int c = 0; c < 3; ++c) nrm4[4 * e + c] = n32[c * nt + e];
    }
    // one device allocation for every table
    const size_t n7 = 7 * (size_t)nt;
    size_t bytes = sizeof(double) * (3 * n7 + n7 + 3 * nt + 3 * nv + nt) + sizeof(float) * (6 * n7 + n7 + 3 * nt) +
                   sizeof(float) * (8 * n7 + 4 * nt) + 64 +
                   sizeof(int32_t) * (3 * nt + (nv + 1) + 3 * nt + (nt + 1) + m->tp_tri.size()) + 3 * nt + 256;
    char *base = nullptr;
    if (cudaMalloc((void **)&base, bytes) != cudaSuccess) {
        cudaGetLastError();
        delete m;
        return td_fail(ctx, TDBEM_ERR_OOM, "device allocation of %zu bytes for the mesh tables failed", bytes);
    }
    m->dev_block = base;
    size_t off = 0;
    auto take = [&](size_t b) {
        char *p = base + off;
        off += (b + 15) & ~(size_t)15;
        return p;
    };
    m->qx = (double *)take(sizeof(double) * n7);
    m->qy = (double *)take(sizeof(double) * n7);
    m->qz = (double *)take(sizeof(double) * n7);
    m->qw = (double *)take(sizeof(double) * n7);
    m->n64 = (double *)take(sizeof(double) * 3 * nt);
    m->dverts = (double *)take(sizeof(double) * 3 * nv);
    m->darea = (double *)take(sizeof(double) * nt);
    m->qxh = (float *)take(sizeof(float) * n7);
    m->qyh = (float *)take(sizeof(float) * n7);
    m->qzh = (float *)take(sizeof(float) * n7);
    m->qxl = (float *)take(sizeof(float) * n7);
    m->qyl = (float *)take(sizeof(float) * n7);
    m->qzl = (float *)take(sizeof(float) * n7);
    m->qw32 = (float *)take(sizeof(float) * n7);
    m->n32 = (float *)take(sizeof(float) * 3 * nt);
    m->qp = take(sizeof(float) * 8 * n7);
    m->nrm4 = take(sizeof(float) * 4 * nt);
    m->dtris = (int32_t *)take(sizeof(int32_t) * 3 * nt);
    m->dv2t_ptr = (int32_t *)take(sizeof(int32_t) * (nv + 1));
    m->dv2t = (int32_t *)take(sizeof(int32_t) * 3 * nt);
    m->dtp_ptr = (int32_t *)take(sizeof(int32_t) * (nt + 1));
    m->dtp_tri = (int32_t *)take(sizeof(int32_t) * std::max<size_t>(1, m->tp_tri.size()));
    m->dv2t_loc = (int8_t *)take(3 * nt);
    int rc = TDBEM_OK;
    if ((rc = upload(ctx, m->qx, q.data(), n7)) || (rc = upload(ctx, m->qy, q.data() + n7, n7)) ||
        (rc = upload(ctx, m->qz, q.data() + 2 * n7, n7)) || (rc = upload(ctx, m->qw, qw.data(), n7)) ||
        (rc = upload(ctx, m->n64, nrm.data(), 3 * nt)) || (rc = upload(ctx, m->dverts, verts, 3 * nv)) ||
        (rc = upload(ctx, m->darea, m->area.data(), nt)) || (rc = upload(ctx, m->qxh, qh.data(), n7)) ||
        (rc = upload(ctx, m->qyh, qh.data() + n7, n7)) || (rc = upload(ctx, m->qzh, qh.data() + 2 * n7, n7)) ||
        (rc = upload(ctx, m->qxl, ql.data(), n7)) || (rc = upload(ctx, m->qyl, ql.data() + n7, n7)) ||
        (rc = upload(ctx, m->qzl, ql.data() + 2 * n7, n7)) || (rc = upload(ctx, m->qw32, qw32.data(), n7)) ||
        (rc = upload(ctx, m->n32, n32.data(), 3 * nt)) || (rc = upload(ctx, m->dtris, tris, 3 * nt)) ||
        (rc = upload(ctx, (float *)m->qp, qp.data(), 8 * n7)) || (rc = upload(ctx, (float *)m->nrm4, nrm4.data(), 4 * nt)) ||
        (rc = upload(ctx, m->dv2t_ptr, m->v2t_ptr.data(), nv + 1)) || (rc = upload(ctx, m->dv2t, m->v2t.data(), 3 * nt)) ||
        (rc = upload(ctx, m->dtp_ptr, m->tp_ptr.data(), nt + 1)) ||
        (rc = upload(ctx, m->dtp_tri, m->tp_tri.data(), m->tp_tri.size())) ||
        (rc = upload(ctx, m->dv2t_loc, m->v2t_loc.data(), 3 * nt))) {
        cudaFree(base);
        delete m;
        return rc;
    }
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        cudaFree(base);
        delete m;
        return td_fail(ctx, TDBEM_ERR_CUDA, "mesh upload failed");
    }
    *out = m;
    return TDBEM_OK;
}

extern "C" int tdbem_mesh_destroy(tdbem_mesh_t m) {
    if (!m) return TDBEM_OK;
    cudaFree(m->dev_block);
    delete m;
    return TDBEM_OK;
}

extern "C" int64_t tdbem_mesh_ndof(tdbem_mesh_t m, int32_t basis) {
    if (!m) return -1;
    return basis == TDBEM_P1 ? m->nv : m->nt;
}

// ============================================================================
// frequencies
// ============================================================================
// Radius factor of the gCQ contour (App. A, as read here): the gCQ steps
// (eq. gCQ_xn) need a contour around every pole 1/(dt lambda_i(A)) of the
// Runge-Kutta resolvents (I - dt s A)^{-1}, i.e. rho >= 1 / min_i |lambda_i|,
// and the stages of the N steps grow along it like max|R(dt_min s)|^N, R the
// stability function, which must stay bounded (1e4) for the quadrature sums
// to keep their digits.  Implicit Euler: |R| = 1 on the circle of rho = 1
// (the contour as printed).  2-stage Radau IIA, R(z) = (1 + z/3) / (1 - 2z/3 +
// z^2/6): rho starts at sqrt(6) and grows by 5 % until the bound holds on 4096
// points of the circle z = rho (1 + e^{i theta}).
double td_gcq_radius(int rk, int nsteps) {
    if (rk != TDBEM_RADAU2) return 1.0;
    const double two_pi = 6.283185307179586476925286766559;
    double rho = std::sqrt(6.0);
    for (int it = 0; it < 400; ++it) {
        double mx = 0.0;
        for (int j = 1; j < 4096; ++j) {
            const double th = two_pi * j / 4096.0;
            const std::complex<double> z = rho * std::complex<double>(1.0 + std::cos(th), std::sin(th));
            const std::complex<double> R = (1.0 + z / 3.0) / (1.0 - 2.0 * z / 3.0 + z * z / 6.0);
            mx = std::max(mx, std::abs(R));
        }
        if (std::max(nsteps, 1) * std::log(mx) <= std::log(1e4)) return rho;
        rho *= 1.05;
    }
    return rho;
}

namespace {
int finish_freqs(tdbem_ctx *ctx, tdbem_freqs *f) {
    TD_CUDA(ctx, cudaMemcpyAsync(f->s.data(), f->ds, sizeof(double) * 2 * f->NQ, cudaMemcpyDeviceToHost, ctx->stream));
    TD_CUDA(ctx, cudaMemcpyAsync(f->w.data(), f->dw, sizeof(double) * 2 * f->NQ, cudaMemcpyDeviceToHost, ctx->stream));
    TD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    // conjugate pairing: BDF2 k <-> N-k (k = 0 and N/2 are real);
    // gCQ l <-> NQ-1-l (no real points for even NQ)
    const int NQ = f->NQ;
    f->unique.assign(NQ, 0);
    f->uidx.clear();
    for (int k = 0; k < NQ; ++k) {
        int partner = f->kind == 0 ? (NQ - k) % NQ : NQ - 1 - k;
        if (f->kind == 2) {
            // explicit points: the partner is the point equal to conj(s_k), if any
            partner = k;
            const double re = f->s[2 * k], im = f->s[2 * k + 1], tol = 1e-12 * std::hypot(re, im);
            if (im != 0.0)
                for (int p = 0; p < NQ; ++p)
                    if (p != k && std::fabs(f->s[2 * p] - re) <= tol && std::fabs(f->s[2 * p + 1] + im) <= tol &&
                        f->unique[p] == 0) {
                        partner = p;
                        break;
                    }
            if (f->unique[k] != 0) continue;  // already the conjugate of an earlier point
            const int rep = (int)f->uidx.size();
            f->uidx.push_back(k);
            f->unique[k] = rep + 1;
            if (partner != k) f->unique[partner] = -(rep + 1);
            continue;
        }
        if (partner < k) continue;  // assigned as conjugate below
        const int rep = (int)f->uidx.size();
        f->uidx.push_back(k);
        f->unique[k] = rep + 1;
        if (partner != k) f->unique[partner] = -(rep + 1);
    }
    f->Nu = (int)f->uidx.size();
    return TDBEM_OK;
}
}  // namespace

extern "C" int tdbem_freqs_cq_bdf2(tdbem_ctx_t ctx, int32_t N, double dt, double lambda, tdbem_freqs_t *out) {
    cudaGetLastError();  // errors of earlier unrelated calls are not ours to report
    if (!ctx || !out || N < 1 || N > 65536 || !(dt > 0.0) || !std::isfinite(dt) || lambda >= 1.0)
        return td_fail(ctx, TDBEM_ERR_ARG, "tdbem_freqs_cq_bdf2: need N >= 1, dt > 0, lambda < 1");
    *out = nullptr;
    if (lambda <= 0.0) lambda = std::pow(1e-8, 1.0 / (2.0 * N));
    tdbem_freqs *f = new (std::nothrow) tdbem_freqs();
    if (!f) return TDBEM_ERR_OOM;
    f->ctx = ctx;
    f->NQ = N;
    f->kind = 0;
    f->s.assign(2 * N, 0.0);
    f->w.assign(2 * N, 0.0);
    int rc;
    if ((rc = dalloc(ctx, &f->ds, 4 * (size_t)N))) {
        delete f;
        return rc;
    }
    f->dw = f->ds + 2 * N;
    cudaMemsetAsync(f->dw, 0, sizeof(double) * 2 * N, ctx->stream);
    if (td_launch_bdf2(ctx->stream, N, dt, lambda, f->ds) || (rc = finish_freqs(ctx, f))) {
        cudaFree(f->ds);
        delete f;
        return rc ? rc : td_fail(ctx, TDBEM_ERR_CUDA, "BDF2 frequency kernel failed");
    }
    *out = f;
    return TDBEM_OK;
}

extern "C" int tdbem_freqs_gcq(tdbem_ctx_t ctx, const double *dts, int32_t N, int32_t rk, int32_t NQ, double rho_in,
                               tdbem_freqs_t *out) {
    cudaGetLastError();  // errors of earlier unrelated calls are not ours to report
    if (!ctx || !out || !dts || N < 1 || NQ < 2 || NQ % 2 || NQ > 65536 || (rk != TDBEM_EULER && rk != TDBEM_RADAU2) ||
        !std::isfinite(rho_in))
        return td_fail(ctx, TDBEM_ERR_ARG, "tdbem_freqs_gcq: need N >= 1 steps, even NQ >= 2, rk EULER|RADAU2");
    *out = nullptr;
    double dt_min = dts[0], dt_max = dts[0];
    for (int32_t n = 0; n < N; ++n) {
        if (!(dts[n] > 0.0) || !std::isfinite(dts[n]))
            return td_fail(ctx, TDBEM_ERR_ARG, "tdbem_freqs_gcq: step %d is not a finite positive number", n);
        dt_min = std::min(dt_min, dts[n]);
        dt_max = std::max(dt_max, dts[n]);
    }
    double q = dt_max / dt_min;
    if (rk == TDBEM_RADAU2) q *= 5.0;  // |lambda_1(A)| = |lambda_2(A)| for 2-stage Radau IIA
    if (q < 1.01) q = 1.01;            // App. A: q = 1 gives k = 0; lift it slightly
    tdbem_freqs *f = new (std::nothrow) tdbem_freqs();
    if (!f) return TDBEM_ERR_OOM;
    f->ctx = ctx;
    f->NQ = NQ;
    f->kind = 1;
    f->dts.assign(dts, dts + N);
    f->s.assign(2 * NQ, 0.0);
    f->w.assign(2 * NQ, 0.0);
    int rc;
    if ((rc = dalloc(ctx, &f->ds, 4 * (size_t)NQ))) {
        delete f;
        return rc;
    }
    f->dw = f->ds + 2 * NQ;
    // the contour is built for dt_min / rho (td_gcq_radius): a circle through 0
    // and 2 rho / dt_min around every resolvent pole of the steps
    const double rho = rho_in > 0.0 ? rho_in : td_gcq_radius(rk, N);
    f->rho = rho;
    if (td_launch_gcq(ctx->stream, NQ, dt_min / rho, q, f->ds, f->dw) || (rc = finish_freqs(ctx, f))) {
        cudaFree(f->ds);
        delete f;
        return rc ? rc : td_fail(ctx, TDBEM_ERR_CUDA, "gCQ frequency kernel failed");
    }
    *out = f;
    return TDBEM_OK;
}

extern "C" int tdbem_freqs_points(tdbem_ctx_t ctx, const double *s, const double *w, int32_t NQ, tdbem_freqs_t *out) {
    cudaGetLastError();
    if (!ctx || !out || !s || NQ < 1 || NQ > 65536)
        return td_fail(ctx, TDBEM_ERR_ARG, "tdbem_freqs_points: need 1 <= NQ <= 65536 points");
    *out = nullptr;
    for (int k = 0; k < 2 * NQ; ++k)
        if (!std::isfinite(s[k]) || (w && !std::isfinite(w[k])))
            return td_fail(ctx, TDBEM_ERR_ARG, "tdbem_freqs_points: non-finite value at %d", k);
    for (int k = 0; k < NQ; ++k)
        if (!(s[2 * k] > 0.0)) return td_fail(ctx, TDBEM_ERR_ARG, "tdbem_freqs_points: Re(s_%d) must be > 0", k);
    tdbem_freqs *f = new (std::nothrow) tdbem_freqs();
    if (!f) return TDBEM_ERR_OOM;
    f->ctx = ctx;
    f->NQ = NQ;
    f->kind = 2;
    f->s.assign(s, s + 2 * NQ);
    f->w.assign(2 * NQ, 0.0);
    if (w) f->w.assign(w, w + 2 * NQ);
    int rc;
    if ((rc = dalloc(ctx, &f->ds, 4 * (size_t)NQ))) {
        delete f;
        return rc;
    }
    f->dw = f->ds + 2 * NQ;
    if ((rc = upload(ctx, f->ds, f->s.data(), 2 * NQ)) || (rc = upload(ctx, f->dw, f->w.data(), 2 * NQ)) ||
        (rc = finish_freqs(ctx, f))) {
        cudaFree(f->ds);
        delete f;
        return rc;
    }
    *out = f;
    return TDBEM_OK;
}

extern "C" int tdbem_freqs_get(tdbem_freqs_t f, double *s, double *w, int32_t *NQ, int32_t *Nu, int32_t *unique) {
    if (!f) return TDBEM_ERR_ARG;
    if (s) std::memcpy(s, f->s.data(), sizeof(double) * 2 * f->NQ);
    if (w) std::memcpy(w, f->w.data(), sizeof(double) * 2 * f->NQ);
    if (NQ) *NQ = f->NQ;
    if (Nu) *Nu = f->Nu;
    if (unique) std::memcpy(unique, f->unique.data(), sizeof(int32_t) * f->NQ);
    return TDBEM_OK;
}

extern "C" int tdbem_freqs_steps(tdbem_freqs_t f, double *dts, int32_t *N) {
    if (!f) return TDBEM_ERR_ARG;
    if (dts && !f->dts.empty()) std::memcpy(dts, f->dts.data(), sizeof(double) * f->dts.size());
    if (N) *N = (int32_t)f->dts.size();
    return TDBEM_OK;
}

extern "C" int tdbem_freqs_destroy(tdbem_freqs_t f) {
    if (!f) return TDBEM_OK;
    cudaFree(f->ds);
    delete f;
    return TDBEM_OK;
}

// ============================================================================
// tree
// ============================================================================
extern "C" int tdbem_tree_build(tdbem_mesh_t mesh, int32_t row_basis, int32_t col_basis, int32_t leaf, double eta,
                                tdbem_tree_t *out) {
    if (!mesh || !out) return TDBEM_ERR_ARG;
    tdbem_ctx *ctx = mesh->ctx;
    *out = nullptr;
    if (leaf < 1 || !(eta > 0.0) || !std::isfinite(eta) || (row_basis != TDBEM_P0 && row_basis != TDBEM_P1) ||
        (col_basis != TDBEM_P0 && col_basis != TDBEM_P1))
        return td_fail(ctx, TDBEM_ERR_ARG, "tdbem_tree_build: need leaf >= 1, eta > 0, basis P0|P1");
    tdbem_tree *t = new (std::nothrow) tdbem_tree();
    if (!t) return TDBEM_ERR_OOM;
    t->mesh = mesh;
    t->leaf = leaf;
    t->eta = eta;
    td_plan_tree(mesh, row_basis, leaf, t->side[0]);
    if (col_basis == row_basis)
        t->side[1] = t->side[0];  // the same DOF points give the same tree
    else
        td_plan_tree(mesh, col_basis, leaf, t->side[1]);
    td_plan_blocks(t->side[0], t->side[1], eta, t->blocks);
    *out = t;
    return TDBEM_OK;
}

extern "C" int tdbem_tree_export(tdbem_tree_t t, int32_t *pr, int32_t *pc, int64_t *nb, int32_t *blocks) {
    if (!t) return TDBEM_ERR_ARG;
    if (pr) std::memcpy(pr, t->side[0].perm.data(), sizeof(int32_t) * t->side[0].n);
    if (pc) std::memcpy(pc, t->side[1].perm.data(), sizeof(int32_t) * t->side[1].n);
    if (nb) *nb = (int64_t)t->blocks.size() / 5;
    if (blocks) std::memcpy(blocks, t->blocks.data(), sizeof(int32_t) * t->blocks.size());
    return TDBEM_OK;
}

extern "C" int tdbem_tree_destroy(tdbem_tree_t t) {
    delete t;
    return TDBEM_OK;
}

// ============================================================================
// entries
// ============================================================================
extern "C" int tdbem_entries(tdbem_mesh_t mesh, const tdbem_op *op, tdbem_freqs_t f, const int32_t *rows, int64_t nr,
                             const int32_t *cols, int64_t nc, const int32_t *fidx, int64_t nf, void *out) {
    cudaGetLastError();  // errors of earlier unrelated calls are not ours to report
    if (!mesh || !f) return TDBEM_ERR_ARG;
    tdbem_ctx *ctx = mesh->ctx;
    int rc = td_check_op(ctx, op);
    if (rc) return rc;
    if (nr < 0 || nc < 0 || nf < 0 || (nr * nc * nf > 0 && (!rows || !cols || !fidx || !out)))
        return td_fail(ctx, TDBEM_ERR_ARG, "tdbem_entries: bad sizes or NULL pointers");
    if (nr * nc * nf == 0) return TDBEM_OK;
    Guard g;
    double *gx, *gw, *sig;
    int *tp_slot, *pti, *ptj, np;
    if ((rc = prepare_sing(ctx, mesh, op->op, op->ng, g.p, &gx, &gw, &tp_slot, &pti, &ptj, &np))) return rc;
    std::vector<double> hs(2 * f->NQ);
    for (int k = 0; k < 2 * f->NQ; ++k) hs[k] = f->s[k] / op->c;
    if ((rc = dalloc(ctx, &sig, hs.size(), &g.p)) || (rc = upload(ctx, sig, hs.data(), hs.size()))) return rc;
    MeshDev md = td_mesh_dev(mesh, op->ng, gx, gw, tp_slot);
    if (td_launch_entries(ctx->stream, md, op->op, op->prec, sig, f->NQ, rows, nr, cols, nc, fidx, nf, out))
        return td_fail(ctx, TDBEM_ERR_CUDA, "entry kernel launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    TD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));  // transient buffers are freed on return
    return TDBEM_OK;
}

extern "C" int tdbem_entries_path(tdbem_mesh_t mesh, const tdbem_op *op, tdbem_freqs_t f, const int32_t *rows,
                                  int64_t nr, const int32_t *cols, int64_t nc, const int32_t *fidx, int64_t nf,
                                  int32_t path, void *out) {
    if (path == TDBEM_PATH_GENERIC) return tdbem_entries(mesh, op, f, rows, nr, cols, nc, fidx, nf, out);
    cudaGetLastError();  // errors of earlier unrelated calls are not ours to report
    if (!mesh || !f) return TDBEM_ERR_ARG;
    tdbem_ctx *ctx = mesh->ctx;
    int rc = td_check_op(ctx, op);
    if (rc) return rc;
    if (path != TDBEM_PATH_NEAR && path != TDBEM_PATH_FIBRE)
        return td_fail(ctx, TDBEM_ERR_ARG, "tdbem_entries_path: unknown path %d", path);
    if (nr < 0 || nc < 0 || nf < 0 || (nr * nc * nf > 0 && (!rows || !cols || !fidx || !out)))
        return td_fail(ctx, TDBEM_ERR_ARG, "tdbem_entries_path: bad sizes or NULL pointers");
    if (nr * nc * nf == 0) return TDBEM_OK;
    if (path == TDBEM_PATH_NEAR && (nf > 256 || nr * nc > INT32_MAX))
        return td_fail(ctx, TDBEM_ERR_ARG, "tdbem_entries_path: the near-field path takes at most 256 frequencies "
                                           "and 2^31 - 1 entries per frequency");
    // the index arrays are checked on the host (the near-field kernels read
    // the tables at them without bounds checks, as inside tdbem_compress)
    std::vector<int32_t> hr(nr), hc(nc), hf(nf);
    TD_CUDA(ctx, cudaMemcpyAsync(hr.data(), rows, sizeof(int32_t) * nr, cudaMemcpyDeviceToHost, ctx->stream));
    TD_CUDA(ctx, cudaMemcpyAsync(hc.data(), cols, sizeof(int32_t) * nc, cudaMemcpyDeviceToHost, ctx->stream));
    TD_CUDA(ctx, cudaMemcpyAsync(hf.data(), fidx, sizeof(int32_t) * nf, cudaMemcpyDeviceToHost, ctx->stream));
    TD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    const int64_t ncol_max = op->op == TDBEM_DLP ? mesh->nv : mesh->nt;
    for (int32_t v : hr)
        if (v < 0 || v >= mesh->nt) return td_fail(ctx, TDBEM_ERR_ARG, "tdbem_entries_path: row %d out of range", v);
    for (int32_t v : hc)
        if (v < 0 || v >= ncol_max) return td_fail(ctx, TDBEM_ERR_ARG, "tdbem_entries_path: column %d out of range", v);
    for (int32_t v : hf)
        if (v < 0 || v >= f->NQ) return td_fail(ctx, TDBEM_ERR_ARG, "tdbem_entries_path: frequency %d out of range", v);
    std::vector<double> hs(2 * nf);
    for (int64_t q = 0; q < nf; ++q) {
        hs[2 * q] = f->s[2 * hf[q]] / op->c;
        hs[2 * q + 1] = f->s[2 * hf[q] + 1] / op->c;
    }
    Guard g;
    double *sig;
    if ((rc = dalloc(ctx, &sig, hs.size(), &g.p)) || (rc = upload(ctx, sig, hs.data(), hs.size()))) return rc;
    int lrc = 0;
    if (path == TDBEM_PATH_FIBRE) {
        MeshDev md = td_mesh_dev(mesh, op->ng, nullptr, nullptr, nullptr);  // regular rule only
        lrc = td_launch_fibre_entries(ctx->stream, md, op->op, op->prec, sig, rows, nr, cols, nc, nf, out, ctx->num_sms);
    } else {
        // the compression's near-field phases on one block rows x cols: the
        // touching-pair table of the mesh, then the dense near tensor
        // [nf][nr][nc] written straight into out
        double *gx, *gw;
        int *tp_slot, *pti, *ptj, np;
        if ((rc = prepare_sing(ctx, mesh, op->op, op->ng, g.p, &gx, &gw, &tp_slot, &pti, &ptj, &np))) return rc;
        c64 *table;
        int32_t *blk;
        int64_t *pre;
        if ((rc = dalloc(ctx, &table, (size_t)std::max(np, 1) * nf * 3, &g.p)) || (rc = dalloc(ctx, &blk, 8, &g.p)) ||
            (rc = dalloc(ctx, &pre, 2, &g.p)))
            return rc;
        const int32_t hb[8] = {0, (int32_t)nr, 0, (int32_t)nc, 0, 0, 0, 0};  // block, then near_ids = {0}
        const int64_t hp[2] = {0, 0};                                        // eprefix, noff
        if ((rc = upload(ctx, blk, hb, 8)) || (rc = upload(ctx, pre, hp, 2))) return rc;
        MeshDev md = td_mesh_dev(mesh, op->ng, gx, gw, tp_slot);
        lrc = td_launch_sing_table(ctx->stream, md, op->op, op->prec, pti, ptj, np, sig, (int)nf, table, ctx->num_sms);
        NearArgs na{};
        na.nf = (int)nf;
        na.sig = sig;
        na.nnear = 1;
        na.near_ids = blk + 5;
        na.eprefix = pre;
        na.noff = pre + 1;
        na.blocks = blk;
        na.perm_r = rows;
        na.perm_c = cols;
        na.nentries = nr * nc;
        na.near = out;
        if (!lrc) lrc = td_launch_near_entries(ctx->stream, md, op->op, op->prec, na, table, ctx->num_sms);
    }
    if (lrc) return td_fail(ctx, TDBEM_ERR_CUDA, "entry kernel launch failed: %s", cudaGetErrorString((cudaError_t)lrc));
    TD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));  // transient buffers are freed on return
    return TDBEM_OK;
}

// ============================================================================
// compression
// ============================================================================
namespace {

void free_tensor(tdbem_tensor *t) {
    if (!t) return;
    for (void *p : t->owned) cudaFree(p);
    if (t->plan_mem) cudaFree(t->plan_mem);
    if (t->plan_Z) cudaFree(t->plan_Z);
    delete t;
}

TensorOut tensor_out(const tdbem_tensor *t, int *flags) {
    TensorOut o{};
    o.Nu = t->Nu;
    o.rank = t->drank;
    o.kpiv = t->dkpiv;
    o.frank = t->dfrank;
    o.foff = t->dfoff;
    o.fib = t->dfib;
    o.face = t->dface;
    o.face_cap = t->face_cap;
    o.face_used = (unsigned long long *)t->dface_used;
    o.dev_flags = flags;
    return o;
}

}  // namespace

extern "C" int tdbem_compress(tdbem_ctx_t ctx, tdbem_mesh_t mesh, const tdbem_op *op, tdbem_freqs_t f,
                              tdbem_tree_t tree, const tdbem_aca_cfg *cfg, tdbem_tensor_t *out) {
    cudaGetLastError();  // errors of earlier unrelated calls are not ours to report
    if (!ctx || !mesh || !f || !tree || !cfg || !out) return td_fail(ctx, TDBEM_ERR_ARG, "tdbem_compress: NULL argument");
    *out = nullptr;
    int rc = td_check_op(ctx, op);
    if (rc) return rc;
    if (tree->mesh != mesh) return td_fail(ctx, TDBEM_ERR_ARG, "tree was built on another mesh");
    if (tree->side[0].basis != TDBEM_P0 || tree->side[1].basis != (op->op == TDBEM_DLP ? TDBEM_P1 : TDBEM_P0))
        return td_fail(ctx, TDBEM_ERR_ARG, "tree bases do not match the operator (SLP: P0 x P0, DLP: P0 x P1)");
    if (!(cfg->eps > 0.0) || !(cfg->eps_aca > 0.0)) return td_fail(ctx, TDBEM_ERR_ARG, "eps and eps_aca must be > 0");
    if (f->Nu > 256) return td_fail(ctx, TDBEM_ERR_ARG, "at most 256 unique frequencies are supported");
    const double t0 = now_ms();
    const int Nu = f->Nu;
    const int kcap = cfg->max_face_rank > 0 ? std::min(cfg->max_face_rank, 64) : 64;  // tiles hold <= 64 rows
    tdbem_tensor *T = new (std::nothrow) tdbem_tensor();
    if (!T) return TDBEM_ERR_OOM;
    T->ctx = ctx;
    T->mesh = mesh;
    T->freqs = f;
    T->op = op->op;
    T->prec = op->prec;
    T->c = op->c;
    T->ng = op->ng;
    T->nrows = tree->side[0].n;
    T->ncols = tree->side[1].n;
    T->Nu = Nu;
    T->NQ = f->NQ;
    const int pf = op->prec == TDBEM_MIXED ? 1 : 0;
    // compression partition: the tree's blocks, with far blocks that would
    // outlast the rest of the persistent far phase split into sub-blocks
    if (cfg->flags & 4)
        T->blocks = tree->blocks;
    else
        td_balance_partition(tree->side[0], tree->side[1], tree->blocks, (int64_t)ctx->num_sms * ctx->far_cps[pf],
                             T->blocks);
    const int64_t nb = (int64_t)T->blocks.size() / 5;
    T->nblocks = nb;
    const size_t es = op->prec == TDBEM_FP64 ? sizeof(c64) : sizeof(c32);
    auto fail = [&](int code) {
        free_tensor(T);
        return code;
    };
    // ---- plan: near/far lists, offsets
    std::vector<int32_t> near_ids, far_ids;
    std::vector<int64_t> eprefix, noff;
    int64_t nent = 0, ntens = 0, maxIJ = 1, sum_far_len = 0;
    int maxI = 1, maxJ = 1, max_near_rows = 1;
    for (int64_t b = 0; b < nb; ++b) {
        const int32_t *bl = &T->blocks[5 * b];
        const int nI = bl[1] - bl[0], nJ = bl[3] - bl[2];
        if (bl[4]) {
            far_ids.push_back((int32_t)b);
            maxI = std::max(maxI, nI);
            maxJ = std::max(maxJ, nJ);
            sum_far_len += nI + nJ;
        } else {
            near_ids.push_back((int32_t)b);
            eprefix.push_back(nent);
            noff.push_back(ntens);
            nent += (int64_t)nI * nJ;
            ntens += (int64_t)nI * nJ * Nu;
            maxIJ = std::max<int64_t>(maxIJ, (int64_t)nI * nJ);
            max_near_rows = std::max(max_near_rows, nI);
        }
    }
    // The near tensor [Nu][nI][nJ] per near block is formed and compressed in
    // batches of consecutive near blocks of at most ctx->near_batch_bytes (one
    // batch when it fits); every batch reuses one buffer.  eprefix / noff
    // become offsets within the batch.
    std::vector<int> nbatch(1, 0);
    std::vector<int64_t> batch_nent;
    int64_t max_batch_tens = 1;
    {
        const int64_t budget = std::max<int64_t>(1, ctx->near_batch_bytes / (int64_t)es);
        const int nn = (int)near_ids.size();
        int64_t acc = 0;
        for (int q = 0; q < nn; ++q) {
            const int64_t next_e = q + 1 < nn ? eprefix[q + 1] : nent;
            const int64_t sz = (next_e - eprefix[q]) * Nu;
            if (acc > 0 && acc + sz > budget) {
                nbatch.push_back(q);
                acc = 0;
            }
            acc += sz;
        }
        nbatch.push_back(nn);
        for (size_t bt = 0; bt + 1 < nbatch.size(); ++bt) {
            const int q0 = nbatch[bt], q1 = nbatch[bt + 1];
            if (q0 >= q1) continue;
            const int64_t e0 = eprefix[q0], t0b = noff[q0];
            const int64_t e1 = q1 < nn ? eprefix[q1] : nent, t1b = q1 < nn ? noff[q1] : ntens;
            batch_nent.push_back(e1 - e0);
            max_batch_tens = std::max(max_batch_tens, t1b - t0b);
            for (int q = q0; q < q1; ++q) {
                eprefix[q] -= e0;
                noff[q] -= t0b;
            }
        }
    }
    std::sort(far_ids.begin(), far_ids.end(), [&](int32_t x, int32_t y) {
        const int32_t *a = &T->blocks[5 * x], *b = &T->blocks[5 * y];
        const int64_t sa = (int64_t)(a[1] - a[0]) * (a[3] - a[2]), sb = (int64_t)(b[1] - b[0]) * (b[3] - b[2]);
        return sa != sb ? sa > sb : x < y;
    });
    // learned presizing: predicted face ranks order the far blocks by cost,
    // size the face pool and set the first unchecked ACA steps
    int64_t pred_far_cap = -1;
    int32_t *dkpred = nullptr;
    Guard gk;
    if (cfg->model) {
        std::vector<double> cost;
        std::vector<int32_t> ks;
        if ((rc = dalloc(ctx, &dkpred, nb * Nu, &gk.p))) return fail(rc);
        if ((rc = td_predict_kpred(cfg->model, tree, T->blocks, mesh, f, op->c, far_ids, kcap, dkpred, cost, ks))) return fail(rc);
        std::vector<size_t> order(far_ids.size());
        for (size_t q = 0; q < order.size(); ++q) order[q] = q;
        std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return cost[x] > cost[y]; });
        std::vector<int32_t> sorted(far_ids.size());
        pred_far_cap = 0;
        for (size_t q = 0; q < order.size(); ++q) {
            sorted[q] = far_ids[order[q]];
            const int32_t *bl = &T->blocks[5 * sorted[q]];
            // about kTermsEst terms of Algorithm 1 per block, each with the block's
            // mean predicted face rank (the lower edge of the predicted bin)
            pred_far_cap += (int64_t)((bl[1] - bl[0]) + (bl[3] - bl[2])) * ((ks[order[q]] + Nu - 1) / Nu) * kTermsEst;
        }
        far_ids.swap(sorted);
    }
    T->kcap = kcap;
    T->max_near_rows = max_near_rows;
    // ---- persistent device data of the tensor
    std::vector<int32_t> inv_r(T->nrows), inv_c(T->ncols);
    for (int64_t k = 0; k < T->nrows; ++k) inv_r[tree->side[0].perm[k]] = (int32_t)k;
    for (int64_t k = 0; k < T->ncols; ++k) inv_c[tree->side[1].perm[k]] = (int32_t)k;
    if ((rc = dalloc(ctx, &T->dblocks, 5 * nb, &T->owned)) || (rc = dalloc(ctx, &T->dperm_r, T->nrows, &T->owned)) ||
        (rc = dalloc(ctx, &T->dperm_c, T->ncols, &T->owned)) || (rc = dalloc(ctx, &T->dinv_r, T->nrows, &T->owned)) ||
        (rc = dalloc(ctx, &T->dinv_c, T->ncols, &T->owned)) || (rc = dalloc(ctx, &T->drank, nb, &T->owned)) ||
        (rc = dalloc(ctx, &T->dkpiv, nb * Nu, &T->owned)) || (rc = dalloc(ctx, &T->dfrank, nb * Nu, &T->owned)) ||
        (rc = dalloc(ctx, &T->dfoff, nb * Nu, &T->owned)) || (rc = dalloc(ctx, &T->dpartner, f->NQ + 1, &T->owned)) ||
        (rc = dalloc(ctx, &T->dface_used, 2, &T->owned)))
        return fail(rc);
    char *fib = nullptr;
    if ((rc = dalloc(ctx, &fib, es * nb * Nu * Nu, &T->owned))) return fail(rc);
    T->dfib = fib;
    if ((rc = upload(ctx, T->dblocks, T->blocks.data(), 5 * nb)) ||
        (rc = upload(ctx, T->dperm_r, tree->side[0].perm.data(), T->nrows)) ||
        (rc = upload(ctx, T->dperm_c, tree->side[1].perm.data(), T->ncols)) ||
        (rc = upload(ctx, T->dinv_r, inv_r.data(), T->nrows)) || (rc = upload(ctx, T->dinv_c, inv_c.data(), T->ncols)) ||
        (rc = upload(ctx, T->dpartner, f->unique.data(), f->NQ)))
        return fail(rc);
    // ---- transient buffers
    Guard g;
    double *gx, *gw, *sig;
    int *tp_slot, *pti, *ptj, npairs;
    if ((rc = prepare_sing(ctx, mesh, op->op, op->ng, g.p, &gx, &gw, &tp_slot, &pti, &ptj, &npairs))) return fail(rc);
    std::vector<double> hs(2 * Nu);
    for (int u = 0; u < Nu; ++u) {
        hs[2 * u] = f->s[2 * f->uidx[u]] / op->c;
        hs[2 * u + 1] = f->s[2 * f->uidx[u] + 1] / op->c;
    }
    c64 *table;
    char *nearbuf, *scr_near, *scr_far;
    int32_t *dnear_ids, *dfar_ids, *flags, *redo_a, *redo_b;
    unsigned int *redo_count;
    int64_t *deprefix, *dnoff, *evals;
    unsigned int *counter;
    const int nctas_near = std::min<int64_t>(std::max<int64_t>(1, (int64_t)near_ids.size()), (int64_t)ctx->num_sms * 8);
    const int nctas_far = std::min<int64_t>(std::max<int64_t>(1, (int64_t)far_ids.size()), (int64_t)ctx->num_sms * ctx->far_cps[pf]);
    // dense faces of far blocks (up to td_far_dense_terms per block, packed)
    // in dense_cap entries per CTA, within a scratch budget of 35 % of the
    // free device memory, 8 to 80 GB
    int64_t dense_cap = 0;
    for (int32_t b : far_ids) {
        const int32_t *bl = &T->blocks[5 * b];
        dense_cap = std::max<int64_t>(dense_cap, (int64_t)td_far_dense_terms() * (bl[1] - bl[0]) * (bl[3] - bl[2]));
    }
    {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) cudaGetLastError();
        const int64_t budget = std::min<int64_t>((int64_t)80 << 30, std::max<int64_t>((int64_t)8 << 30, (int64_t)(0.35 * (double)fr)));
        dense_cap = std::min<int64_t>(dense_cap, budget / ((int64_t)es * std::max(1, nctas_far)));
        if (cfg->flags & 2) dense_cap = 0;  // low-rank evaluation for every far block
    }
    const int64_t sper_far = (int64_t)kcap * (maxI + maxJ) + dense_cap + std::min<int64_t>(dense_cap, td_far_cd_max());
    if ((rc = dalloc(ctx, &sig, 2 * Nu, &g.p)) || (rc = upload(ctx, sig, hs.data(), hs.size())) ||
        (rc = dalloc(ctx, &table, (size_t)npairs * Nu * 3, &g.p)) || (rc = dalloc(ctx, &nearbuf, es * max_batch_tens, &g.p)) ||
        (rc = dalloc(ctx, &scr_near, es * maxIJ * nctas_near, &g.p)) ||
        (rc = dalloc(ctx, &scr_far, es * sper_far * nctas_far, &g.p)) ||
        (rc = dalloc(ctx, &dnear_ids, near_ids.size(), &g.p)) || (rc = dalloc(ctx, &dfar_ids, far_ids.size(), &g.p)) ||
        (rc = dalloc(ctx, &deprefix, eprefix.size(), &g.p)) || (rc = dalloc(ctx, &dnoff, noff.size(), &g.p)) ||
        (rc = dalloc(ctx, &flags, 4, &g.p)) || (rc = dalloc(ctx, &evals, 4, &g.p)) || (rc = dalloc(ctx, &counter, 4, &g.p)) ||
        (rc = dalloc(ctx, &redo_a, far_ids.size(), &g.p)) || (rc = dalloc(ctx, &redo_b, far_ids.size(), &g.p)) ||
        (rc = dalloc(ctx, &redo_count, 4, &g.p)))
        return fail(rc);
    if ((rc = upload(ctx, dnear_ids, near_ids.data(), near_ids.size())) ||
        (rc = upload(ctx, dfar_ids, far_ids.data(), far_ids.size())) ||
        (rc = upload(ctx, deprefix, eprefix.data(), eprefix.size())) || (rc = upload(ctx, dnoff, noff.data(), noff.size())))
        return fail(rc);
    MeshDev md = td_mesh_dev(mesh, op->ng, gx, gw, tp_slot);
    NearArgs na{};
    na.nf = Nu;
    na.sig = sig;
    na.nnear = (int)near_ids.size();
    na.near_ids = dnear_ids;
    na.eprefix = deprefix;
    na.noff = dnoff;
    na.blocks = T->dblocks;
    na.perm_r = T->dperm_r;
    na.perm_c = T->dperm_c;
    na.nentries = nent;
    na.near = nearbuf;
    AcaParams ap{cfg->eps, cfg->eps_aca, kcap};
    FarArgs fa{};
    fa.nfar = (int)far_ids.size();
    fa.far_ids = dfar_ids;
    fa.blocks = T->dblocks;
    fa.perm_r = T->dperm_r;
    fa.perm_c = T->dperm_c;
    fa.sig = sig;
    fa.nf = Nu;
    fa.maxI = maxI;
    fa.maxJ = maxJ;
    fa.scratch = scr_far;
    fa.scratch_per_cta = sper_far;
    fa.dense_cap = dense_cap;
    fa.counter = counter;
    fa.evals = evals;
    fa.redo = redo_a;
    fa.redo_count = redo_count;
    const double t_plan = now_ms();
    // face pool: every near term fits (r <= Nu), far terms get a generous
    // estimate; on overflow the far phase is rerun with a larger pool.
    // face pool: near terms reserved for min(Nu, max(16, Nu / 4)) terms per
    // near block, far terms from the predicted ranks or a generous estimate;
    // on overflow the phases are rerun with a pool twice as large.
    const int64_t near_res = nent * std::min<int64_t>(Nu, std::max<int64_t>(16, Nu / 4));
    // need: the size the attempt must have; cap: the size it asks for first
    // (more where the device has room: the pool is trimmed after the phases)
    auto device_room = [&]() {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) cudaGetLastError();
        return std::max<int64_t>(0, ((int64_t)(0.85 * (double)fr) - ((int64_t)2 << 30)) / (int64_t)es);
    };
    const double far_est = (double)(pred_far_cap >= 0 ? pred_far_cap + pred_far_cap / 2 : sum_far_len * 256);
    // an estimate beyond the device's room starts from the room (a pool that
    // fills up grows where it can)
    int64_t need = std::min(near_res + (int64_t)(ctx->pool_scale * far_est) + 1024,
                            std::max<int64_t>(near_res + 1024, device_room()));
    // a size-based bound asks for up to twice itself where the device has room;
    // a presize from predicted ranks asks for itself (a pool that fills up grows)
    int64_t cap = pred_far_cap >= 0 ? need : std::max(need, std::min(2 * need, device_room()));
    const int64_t pool_first = cap;
    if (dkpred) fa.kpred = dkpred;
    cudaEvent_t ev[5];
    for (int k = 0; k < 5; ++k) cudaEventCreate(&ev[k]);
    int hflags = 0;
    long long hev[3] = {0, 0, 0};
    float ms_redo = 0.0f;  // far blocks redone after the pool grew
    int st_redo = 0;
    int64_t nlaunch = 0;  // kernel launches (graph nodes included)
    for (int attempt = 0; attempt < 4; ++attempt) {
        if (T->dface) {
            cudaFree(T->dface);
            T->owned.erase(std::find(T->owned.begin(), T->owned.end(), T->dface));
            T->dface = nullptr;
        }
        char *face = nullptr;
        while ((rc = dalloc(ctx, &face, es * cap, &T->owned)) && cap > need) cap = std::max(need, cap - cap / 4);
        if (rc) {
            for (int k = 0; k < 5; ++k) cudaEventDestroy(ev[k]);
            return fail(rc);
        }
        T->dface = face;
        T->face_cap = cap;
        TensorOut o = tensor_out(T, flags);
        // One captured graph per phase (touching table, near entries, near
        // 3D-ACA, far 3D-ACA), launched back to back on the caller's stream
        // with timing events between them.
        const bool use_graph = !(cfg->flags & 1);
        int lrc = 0;
        cudaError_t ge = cudaSuccess;
        for (int ph = 0; ph < 4 && !lrc && ge == cudaSuccess; ++ph) {
            cudaStream_t ls = use_graph ? ctx->capture : ctx->stream;
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            if (ph == 0) cudaEventRecord(ev[0], ctx->stream);
            if (use_graph) {
                ge = cudaStreamBeginCapture(ls, cudaStreamCaptureModeRelaxed);
                if (ge != cudaSuccess) break;
            }
            if (ph == 0) {
                cudaMemsetAsync(T->dface_used, 0, sizeof(int64_t) * 2, ls);
                cudaMemsetAsync(flags, 0, sizeof(int32_t) * 4, ls);
                cudaMemsetAsync(evals, 0, sizeof(int64_t) * 4, ls);
                cudaMemsetAsync(counter, 0, sizeof(unsigned int) * 4, ls);
                cudaMemsetAsync(redo_count, 0, sizeof(unsigned int) * 4, ls);
                cudaMemsetAsync(T->drank, 0, sizeof(int32_t) * nb, ls);
                lrc |= td_launch_sing_table(ls, md, op->op, op->prec, pti, ptj, npairs, sig, Nu, table, ctx->num_sms,
                                            ctx->sing_var);
                nlaunch += npairs > 0;
            } else if (ph == 1 || ph == 2) {
                // one batch: entries (phase 1) and 3D-ACA (phase 2); several: both per
                // batch in phase 1
                const int nbt = (int)batch_nent.size();
                for (int bt = 0; bt < nbt; ++bt) {
                    NearArgs nab = na;
                    const int q0 = nbatch[bt];
                    nab.nnear = nbatch[bt + 1] - q0;
                    nab.near_ids = dnear_ids + q0;
                    nab.eprefix = deprefix + q0;
                    nab.noff = dnoff + q0;
                    nab.nentries = batch_nent[bt];
                    const int nct = std::min(nctas_near, nab.nnear);
                    if (ph == 1) {
                        lrc |= td_launch_near_entries(ls, md, op->op, op->prec, nab, table, ctx->num_sms,
                                                      ctx->near_var);
                        nlaunch += nab.nentries > 0;
                    }
                    if ((ph == 2 && nbt == 1) || (ph == 1 && nbt > 1)) {
                        lrc |= td_launch_near_aca(ls, op->prec, nab, o, ap, scr_near, maxIJ, nct);
                        nlaunch += nab.nnear > 0;
                    }
                }
            } else {
                lrc |= td_launch_far_aca(ls, md, op->op, op->prec, fa, o, ap, nctas_far, ctx->far_nt[pf]);
                nlaunch += fa.nfar > 0;
            }
            if (use_graph) {
                ge = cudaStreamEndCapture(ls, &graph);
                if (ge == cudaSuccess && !lrc) ge = cudaGraphInstantiate(&exec, graph, 0);
                if (ge == cudaSuccess && !lrc) ge = cudaGraphLaunch(exec, ctx->stream);
                if (exec) cudaGraphExecDestroy(exec);  // destruction is deferred until the launch completes
                if (graph) cudaGraphDestroy(graph);
            }
            cudaEventRecord(ev[ph + 1], ctx->stream);
        }
        if (ge != cudaSuccess || lrc) {
            for (int k = 0; k < 5; ++k) cudaEventDestroy(ev[k]);
            return fail(td_fail(ctx, TDBEM_ERR_CUDA, "compression launch failed: %s (launch status %d)",
                                cudaGetErrorString(ge), lrc));
        }
        cudaError_t se = cudaStreamSynchronize(ctx->stream);
        if (se != cudaSuccess) {
            for (int k = 0; k < 5; ++k) cudaEventDestroy(ev[k]);
            return fail(td_fail(ctx, TDBEM_ERR_CUDA, "compression kernels failed: %s", cudaGetErrorString(se)));
        }
        cudaMemcpy(&hflags, flags, sizeof(int), cudaMemcpyDeviceToHost);
        // far blocks stopped by a full pool (and no near block): grow the pool
        // keeping its contents, and redo only those blocks
        int32_t *rec = fa.redo, *nxt = fa.redo == redo_a ? redo_b : redo_a;  // records of the last launch / next
        for (int round = 0; round < 4 && !(hflags & TD_DEV_POOL_OVERFLOW) && (hflags & TD_DEV_FAR_OVERFLOW);
             ++round) {
            unsigned int nredo = 0;
            cudaMemcpy(&nredo, redo_count, sizeof nredo, cudaMemcpyDeviceToHost);
            // the old pool is held during the copy: grow within the room left
            const int64_t room = device_room();
            int64_t gneed = std::min(2 * cap, room), gcap = std::max(gneed, room);
            if (gneed <= cap) {
                for (int k = 0; k < 5; ++k) cudaEventDestroy(ev[k]);
                return fail(td_fail(ctx, TDBEM_ERR_OOM, "face pool full and no device memory left to grow it"));
            }
            char *bigger = nullptr;
            int grc;
            while ((grc = dalloc(ctx, &bigger, es * gcap)) && gcap > gneed) gcap = std::max(gneed, gcap - gcap / 4);
            if (grc) {
                for (int k = 0; k < 5; ++k) cudaEventDestroy(ev[k]);
                return fail(grc);
            }
            // every stored face lies below the old capacity
            const int64_t used = cap;
            if (cudaMemcpy(bigger, T->dface, es * cap, cudaMemcpyDeviceToDevice) != cudaSuccess ||
                cudaMemcpy(T->dface_used, &used, sizeof used, cudaMemcpyHostToDevice) != cudaSuccess) {
                cudaFree(bigger);
                for (int k = 0; k < 5; ++k) cudaEventDestroy(ev[k]);
                return fail(td_fail(ctx, TDBEM_ERR_CUDA, "growing the face pool failed"));
            }
            cudaFree(T->dface);
            *std::find(T->owned.begin(), T->owned.end(), T->dface) = bigger;
            T->dface = bigger;
            T->face_cap = cap = gcap;
            cudaMemsetAsync(flags, 0, sizeof(int32_t) * 4, ctx->stream);
            cudaMemsetAsync(counter, 0, sizeof(unsigned int) * 4, ctx->stream);
            cudaMemsetAsync(redo_count, 0, sizeof(unsigned int) * 4, ctx->stream);
            FarArgs fr = fa;
            fr.nfar = (int)nredo;
            fr.far_ids = rec;
            fr.redo = nxt;
            TensorOut o2 = tensor_out(T, flags);
            cudaEvent_t r0, r1;
            cudaEventCreate(&r0);
            cudaEventCreate(&r1);
            cudaEventRecord(r0, ctx->stream);
            const int lr = td_launch_far_aca(ctx->stream, md, op->op, op->prec, fr, o2, ap,
                                             std::min<int>(nctas_far, (int)nredo), ctx->far_nt[pf]);
            ++nlaunch;
            cudaEventRecord(r1, ctx->stream);
            const cudaError_t re = cudaStreamSynchronize(ctx->stream);
            float mr = 0.0f;
            if (cudaEventElapsedTime(&mr, r0, r1) == cudaSuccess) ms_redo += mr;
            cudaEventDestroy(r0);
            cudaEventDestroy(r1);
            if (lr || re != cudaSuccess) {
                for (int k = 0; k < 5; ++k) cudaEventDestroy(ev[k]);
                return fail(td_fail(ctx, TDBEM_ERR_CUDA, "far-field redo failed: %s", cudaGetErrorString(re)));
            }
            cudaMemcpy(&hflags, flags, sizeof(int), cudaMemcpyDeviceToHost);
            std::swap(rec, nxt);
            ++st_redo;
        }
        cudaMemcpy(hev, evals, sizeof hev, cudaMemcpyDeviceToHost);
        if (!(hflags & (TD_DEV_POOL_OVERFLOW | TD_DEV_FAR_OVERFLOW))) break;
        // grow to twice the pool or to the device memory left (less a reserve
        // for the apply plan), whichever is larger; the pool is trimmed below
        cudaFree(T->dface);
        T->owned.erase(std::find(T->owned.begin(), T->owned.end(), T->dface));
        T->dface = nullptr;
        const int64_t room = device_room();
        if (std::min(2 * cap, room) <= cap) {
            for (int k = 0; k < 5; ++k) cudaEventDestroy(ev[k]);
            return fail(td_fail(ctx, TDBEM_ERR_OOM, "face pool full and no device memory left to grow it"));
        }
        need = std::min(2 * cap, room);
        cap = std::max(need, room);
        ++st_redo;
    }
    if (hflags & (TD_DEV_POOL_OVERFLOW | TD_DEV_FAR_OVERFLOW)) {
        for (int k = 0; k < 5; ++k) cudaEventDestroy(ev[k]);
        return fail(td_fail(ctx, TDBEM_ERR_CAPACITY, "face pool overflow after retries"));
    }
    float ms[4] = {0, 0, 0, 0};
    for (int k = 0; k < 4; ++k)
        if (cudaEventElapsedTime(&ms[k], ev[k], ev[k + 1]) != cudaSuccess) {
            cudaGetLastError();
            ms[k] = -1.0f;
        }
    for (int k = 0; k < 5; ++k) cudaEventDestroy(ev[k]);
    // trim the face pool to the stored faces when more than 4 GB would stay
    // unused (after the transient buffers are returned)
    g.release();
    gk.release();
    {
        int64_t used = 0;
        if (cudaMemcpy(&used, T->dface_used, sizeof(int64_t), cudaMemcpyDeviceToHost) != cudaSuccess)
            return fail(td_fail(ctx, TDBEM_ERR_CUDA, "reading the face pool size failed"));
        if ((T->face_cap - used) * (int64_t)es > ((int64_t)4 << 30)) {
            char *tight = nullptr;
            if (cudaMalloc((void **)&tight, es * std::max<int64_t>(used, 1)) == cudaSuccess) {
                if (used > 0 && cudaMemcpy(tight, T->dface, es * used, cudaMemcpyDeviceToDevice) != cudaSuccess) {
                    cudaFree(tight);
                    return fail(td_fail(ctx, TDBEM_ERR_CUDA, "trimming the face pool failed"));
                }
                cudaFree(T->dface);
                *std::find(T->owned.begin(), T->owned.end(), T->dface) = tight;
                T->dface = tight;
                T->face_cap = std::max<int64_t>(used, 1);
            } else {
                cudaGetLastError();
            }
        }
    }
    // ---- host copies of the per-block results and statistics
    T->rank.resize(nb);
    std::vector<int32_t> frank(nb * Nu);
    if (cudaMemcpy(T->rank.data(), T->drank, sizeof(int32_t) * nb, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(frank.data(), T->dfrank, sizeof(int32_t) * nb * Nu, cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(td_fail(ctx, TDBEM_ERR_CUDA, "reading the block results failed"));
    tdbem_stats &st = T->stats;
    std::memset(&st, 0, sizeof st);
    st.nblocks = nb;
    st.nnear = (int64_t)near_ids.size();
    st.nfar = (int64_t)far_ids.size();
    T->frank_sum.assign(nb, 0);
    for (int64_t b = 0; b < nb; ++b) {
        const int32_t *bl = &T->blocks[5 * b];
        const int nI = bl[1] - bl[0], nJ = bl[3] - bl[2];
        st.sum_rank += T->rank[b];
        st.max_rank = std::max<int64_t>(st.max_rank, T->rank[b]);
        for (int d = 0; d < T->rank[b]; ++d) {
            const int kf = frank[b * Nu + d];
            st.stored_complex += Nu + (kf < 0 ? (int64_t)nI * nJ : (int64_t)kf * (nI + nJ));
            if (kf > 0) {
                st.sum_face_rank += kf;
                T->frank_sum[b] += kf;
            }
        }
    }
    st.dense_complex = T->nrows * T->ncols * (int64_t)Nu;
    st.entries_regular = nent * Nu + hev[0];
    st.entries_tube = hev[1];
    st.aca_tests = hev[2];
    st.pairs_singular = (int64_t)npairs * Nu;
    st.ms_plan = t_plan - t0;
    st.ms_singular = ms[0];
    st.ms_near = ms[1] + ms[2];
    st.ms_far = ms[3] + ms_redo;
    st.pool_growths = st_redo;
    st.launches = nlaunch;
    st.pool_first = pool_first;
    st.ms_total = now_ms() - t0;
    if (hflags & TD_DEV_RANK_CAP)
        td_fail(ctx, TDBEM_OK, "note: some far faces reached the rank cap %d", kcap);
    *out = T;
    return TDBEM_OK;
}

extern "C" int tdbem_tensor_stats(tdbem_tensor_t t, tdbem_stats *st) {
    if (!t || !st) return TDBEM_ERR_ARG;
    *st = t->stats;
    return TDBEM_OK;
}

extern "C" int tdbem_tensor_partition(tdbem_tensor_t t, int64_t *nb, int32_t *blocks) {
    if (!t) return TDBEM_ERR_ARG;
    if (nb) *nb = t->nblocks;
    if (blocks) std::memcpy(blocks, t->blocks.data(), sizeof(int32_t) * 5 * t->nblocks);
    return TDBEM_OK;
}

extern "C" int tdbem_tensor_blocks(tdbem_tensor_t t, int32_t *rank, int32_t *face_rank_sum, int32_t *kpiv) {
    if (!t) return TDBEM_ERR_ARG;
    if (rank) std::memcpy(rank, t->rank.data(), sizeof(int32_t) * t->nblocks);
    if (face_rank_sum) std::memcpy(face_rank_sum, t->frank_sum.data(), sizeof(int32_t) * t->nblocks);
    if (kpiv) {
        std::vector<int32_t> k(t->nblocks * t->Nu);
        TD_CUDA(t->ctx, cudaMemcpy(k.data(), t->dkpiv, sizeof(int32_t) * k.size(), cudaMemcpyDeviceToHost));
        for (int64_t b = 0; b < t->nblocks; ++b)
            for (int d = 0; d <= t->Nu; ++d)
                kpiv[b * (t->Nu + 1) + d] = d < t->rank[b] ? k[b * t->Nu + d] : -1;
    }
    return TDBEM_OK;
}

extern "C" int tdbem_tensor_entries(tdbem_tensor_t t, const int32_t *rows, const int32_t *cols, const int32_t *fidx,
                                    int64_t count, void *out) {
    if (!t) return TDBEM_ERR_ARG;
    if (count < 0 || (count > 0 && (!rows || !cols || !fidx || !out)))
        return td_fail(t->ctx, TDBEM_ERR_ARG, "tdbem_tensor_entries: bad arguments");
    TensorOut o = tensor_out(t, nullptr);
    if (td_launch_tensor_entries(t->ctx->stream, t->prec, o, t->dblocks, (int)t->nblocks, t->nrows, t->ncols,
                                 t->NQ, t->dinv_r, t->dinv_c,
                                 t->dpartner, rows, cols, fidx, count, out))
        return td_fail(t->ctx, TDBEM_ERR_CUDA, "tensor entry kernel failed");
    return TDBEM_OK;
}

extern "C" int tdbem_tensor_destroy(tdbem_tensor_t t) {
    if (t) {
        if (t->dy_host) cudaFree(t->dy_host);
        free_tensor(t);
    }
    return TDBEM_OK;
}

// ============================================================================
// apply
// ============================================================================
namespace {
// Plan of the tensor-core apply for nrhs right-hand sides: the Z rows
// (block, term, half) grouped by column cluster, half 0 first (each half's
// rows block by block, term by term), the tile jobs of the GEMM (a tile holds
// rows of one half and contracts over that half's frequencies), the
// frequency order of the contraction, and each block's first Z row and
// half-1 offset.  Host work O(nblocks * rank + jobs).
int build_apply_plan(tdbem_tensor *t, int nrhs) {
    tdbem_ctx *ctx = t->ctx;
    if (t->plan_nrhs == nrhs) return TDBEM_OK;
    std::vector<int32_t> qmap(t->NQ);
    TD_CUDA(ctx, cudaMemcpy(qmap.data(), t->dpartner, sizeof(int32_t) * t->NQ, cudaMemcpyDeviceToHost));
    int rpt = 1;
    for (int q = 0; q < t->NQ; ++q)
        if (qmap[q] < 0) rpt = 2;
    // contraction order: the frequencies of half 0, then the conjugate half
    std::vector<int32_t> lperm;
    for (int q = 0; q < t->NQ; ++q)
        if (qmap[q] > 0) lperm.push_back(q);
    const int nq0 = (int)lperm.size();
    for (int q = 0; q < t->NQ; ++q)
        if (qmap[q] <= 0) lperm.push_back(q);
    const int64_t nb = t->nblocks;
    std::vector<ZGroup> groups;
    std::vector<std::vector<int32_t>> gblocks;
    std::vector<int64_t> zbase(nb, -1), zpstride(nb, 0), brow(nb, -1);
    std::vector<int> bgroup(nb, -1);
    std::map<std::pair<int, int>, int> gid;
    for (int64_t b = 0; b < nb; ++b) {
        const int r = t->rank[b];
        if (r <= 0) continue;
        const int32_t *bl = &t->blocks[5 * b];
        auto key = std::make_pair(bl[2], bl[3]);
        auto it = gid.find(key);
        int g;
        if (it == gid.end()) {
            g = (int)groups.size();
            gid[key] = g;
            ZGroup zg{};
            zg.J0 = bl[2];
            zg.nJ = bl[3] - bl[2];
            groups.push_back(zg);
            gblocks.emplace_back();
        } else {
            g = it->second;
        }
        bgroup[b] = g;
        brow[b] = groups[g].Mh;  // first half-0 row of the block within its group
        groups[g].Mh += r;
        gblocks[g].push_back((int32_t)b);
    }
    std::vector<int2> rowtab;
    std::vector<ZJob> jobs;
    int64_t zsize = 0;
    const int TM = td_zgemm_tile_rows(), TN = td_zgemm_tile_cols();
    for (size_t g = 0; g < groups.size(); ++g) {
        ZGroup &zg = groups[g];
        zg.row0 = (int)rowtab.size();
        zg.M = rpt * zg.Mh;
        zg.L = zg.nJ * nrhs;
        zg.zoff = zsize;
        zsize += (int64_t)zg.M * zg.L;
        for (int p = 0; p < rpt; ++p)
            for (int32_t b : gblocks[g])
                for (int d = 0; d < t->rank[b]; ++d) rowtab.push_back(make_int2((int)b, 2 * d + p));
        for (int p = 0; p < rpt; ++p)
            for (int m0 = p * zg.Mh; m0 < (p + 1) * zg.Mh; m0 += TM)
                for (int n0 = 0; n0 < zg.L; n0 += TN) jobs.push_back(ZJob{(int)g, m0, n0, rpt == 2 ? p + 1 : 0});
    }
    for (int64_t b = 0; b < nb; ++b)
        if (bgroup[b] >= 0) {
            const ZGroup &zg = groups[bgroup[b]];
            zbase[b] = zg.zoff + brow[b] * zg.L;
            zpstride[b] = (int64_t)zg.Mh * zg.L;
        }
    // far terms and their T offsets (k_d from the device copy of the face ranks)
    std::vector<int32_t> frank((size_t)nb * t->Nu);
    TD_CUDA(ctx, cudaMemcpy(frank.data(), t->dfrank, sizeof(int32_t) * frank.size(), cudaMemcpyDeviceToHost));
    std::vector<int2> ftab;
    std::vector<int64_t> toff((size_t)nb * t->Nu, -1);
    int64_t tsize = 0;
    for (int64_t b = 0; b < nb; ++b) {
        if (!t->blocks[5 * b + 4]) continue;
        for (int d = 0; d < t->rank[b]; ++d) {
            const int kd = frank[(size_t)b * t->Nu + d];
            ftab.push_back(make_int2((int)b, d));
            toff[(size_t)b * t->Nu + d] = tsize;
            tsize += (int64_t)rpt * std::max(kd, 0) * nrhs;
        }
    }
    if (jobs.size() > (size_t)INT32_MAX || rowtab.size() > (size_t)INT32_MAX)
        return td_fail(ctx, TDBEM_ERR_ARG, "apply plan too large");
    if (t->plan_mem || t->plan_Z) TD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));  // an earlier apply may still read them
    if (t->plan_mem) cudaFree(t->plan_mem);
    if (t->plan_Z) cudaFree(t->plan_Z);
    t->plan_mem = t->plan_Z = nullptr;
    t->plan_nrhs = 0;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t off[9];
    off[0] = 0;
    off[1] = off[0] + al(sizeof(ZGroup) * groups.size());
    off[2] = off[1] + al(sizeof(int2) * rowtab.size());
    off[3] = off[2] + al(sizeof(ZJob) * jobs.size());
    off[4] = off[3] + al(sizeof(int64_t) * nb);
    off[5] = off[4] + al(sizeof(int2) * ftab.size());
    off[6] = off[5] + al(sizeof(int64_t) * toff.size());
    off[7] = off[6] + al(sizeof(int64_t) * nb);
    off[8] = off[7] + al(sizeof(int32_t) * lperm.size());
    // plan_Z: Z | T | packed coefficient rows Fp | packed weights Wk, each
    // segment starting on a 32-value (256-byte) boundary
    const int nq1 = t->NQ - nq0;
    auto r32 = [](int64_t x) { return (x + 31) & ~(int64_t)31; };
    const int KW0 = (int)r32(nq0), KW1 = (int)r32(nq1), FW = std::max(KW0, KW1), WS = KW0 + KW1;
    const int64_t z_al = r32(std::max<int64_t>(zsize, 1)), t_al = r32(tsize);
    const int64_t fp_size = (int64_t)rowtab.size() * FW, wk_size = t->ncols * nrhs * WS;
    char *mem = nullptr;
    if (cudaMalloc(&mem, std::max<size_t>(off[8], 256)) != cudaSuccess ||
        cudaMalloc(&t->plan_Z, sizeof(c32) * (z_al + t_al + fp_size + wk_size)) != cudaSuccess) {
        cudaGetLastError();
        if (mem) cudaFree(mem);
        t->plan_Z = nullptr;
        return td_fail(ctx, TDBEM_ERR_OOM, "apply plan: device allocation of %lld complex values failed", (long long)zsize);
    }
    t->plan_mem = mem;
    TD_CUDA(ctx, cudaMemcpy(mem + off[0], groups.data(), sizeof(ZGroup) * groups.size(), cudaMemcpyHostToDevice));
    TD_CUDA(ctx, cudaMemcpy(mem + off[1], rowtab.data(), sizeof(int2) * rowtab.size(), cudaMemcpyHostToDevice));
    TD_CUDA(ctx, cudaMemcpy(mem + off[2], jobs.data(), sizeof(ZJob) * jobs.size(), cudaMemcpyHostToDevice));
    TD_CUDA(ctx, cudaMemcpy(mem + off[3], zbase.data(), sizeof(int64_t) * nb, cudaMemcpyHostToDevice));
    TD_CUDA(ctx, cudaMemcpy(mem + off[4], ftab.data(), sizeof(int2) * ftab.size(), cudaMemcpyHostToDevice));
    TD_CUDA(ctx, cudaMemcpy(mem + off[5], toff.data(), sizeof(int64_t) * toff.size(), cudaMemcpyHostToDevice));
    TD_CUDA(ctx, cudaMemcpy(mem + off[6], zpstride.data(), sizeof(int64_t) * nb, cudaMemcpyHostToDevice));
    TD_CUDA(ctx, cudaMemcpy(mem + off[7], lperm.data(), sizeof(int32_t) * lperm.size(), cudaMemcpyHostToDevice));
    for (int k = 0; k < 8; ++k) t->plan_off[k] = off[k];
    t->plan_nft = (int)ftab.size();
    t->plan_tz = z_al;  // T follows Z in plan_Z
    t->plan_fp = z_al + t_al;
    t->plan_wk = z_al + t_al + fp_size;
    t->plan_fw = FW;
    t->plan_kw0 = KW0;
    t->plan_kw1 = KW1;
    if (td_launch_pack_fibres(ctx->stream, (const int2 *)(mem + off[1]), (int64_t)rowtab.size(), t->dpartner,
                              (const int *)(mem + off[7]), nq0, nq1, (const c32 *)t->dfib, t->Nu,
                              (c32 *)t->plan_Z + t->plan_fp, FW, ctx->num_sms))
        return td_fail(ctx, TDBEM_ERR_CUDA, "apply plan: packing the coefficients failed");
    t->plan_rpt = rpt;
    t->plan_nq0 = nq0;
    t->plan_njobs = (int)jobs.size();
    t->plan_maxI = t->plan_maxJ = 1;
    for (int64_t b = 0; b < nb; ++b) {
        t->plan_maxI = std::max(t->plan_maxI, t->blocks[5 * b + 1] - t->blocks[5 * b]);
        t->plan_maxJ = std::max(t->plan_maxJ, t->blocks[5 * b + 3] - t->blocks[5 * b + 2]);
    }
    t->plan_nrhs = nrhs;
    return TDBEM_OK;
}

// Weighted apply of the mixed form on the tensor cores: Z = frequency
// contraction (split-BF16 tcgen05 GEMM per column cluster), then the faces.
int apply_tc(tdbem_tensor *t, const void *W, int nrhs, void *y) {
    tdbem_ctx *ctx = t->ctx;
    int rc = build_apply_plan(t, nrhs);
    if (rc) return rc;
    char *mem = (char *)t->plan_mem;
    const ZGroup *groups = (const ZGroup *)(mem + t->plan_off[0]);
    const ZJob *jobs = (const ZJob *)(mem + t->plan_off[2]);
    const int64_t *zbase = (const int64_t *)(mem + t->plan_off[3]);
    const int nq1 = t->NQ - t->plan_nq0, WS = t->plan_kw0 + t->plan_kw1;
    c32 *Wk = (c32 *)t->plan_Z + t->plan_wk;
    int e = td_launch_pack_weights(ctx->stream, (const c32 *)W, t->dperm_c, (const int *)(mem + t->plan_off[7]),
                                   t->ncols, nrhs, t->plan_nq0, nq1, t->plan_kw0, t->plan_kw1, Wk, ctx->num_sms);
    if (!e)
        e = td_launch_zgemm_apply(ctx->stream, groups, (const c32 *)t->plan_Z + t->plan_fp, t->plan_fw, Wk, WS,
                                  t->plan_kw0, t->plan_nq0, nq1, (c32 *)t->plan_Z, nrhs, jobs, t->plan_njobs,
                                  ctx->dflags, ctx->wait_polls, ctx->num_sms);
    if (e) return td_fail(ctx, TDBEM_ERR_CUDA, "tensor-core contraction failed: %s", cudaGetErrorString((cudaError_t)e));
    ApplyZArgs a{};
    a.nb = (int)t->nblocks;
    a.blocks = t->dblocks;
    a.perm_r = t->dperm_r;
    a.Nu = t->Nu;
    a.nrhs = nrhs;
    a.rpt = t->plan_rpt;
    a.zbase = zbase;
    a.zpstride = (const int64_t *)(mem + t->plan_off[6]);
    a.Z = (const c32 *)t->plan_Z;
    a.y = (c32 *)y;
    a.nft = t->plan_nft;
    a.ftab = (const int2 *)(mem + t->plan_off[4]);
    a.toff = (const int64_t *)(mem + t->plan_off[5]);
    a.T = (c32 *)t->plan_Z + t->plan_tz;
    e = td_launch_apply_z(ctx->stream, a, tensor_out(t, nullptr), ctx->num_sms);
    if (e) return td_fail(ctx, TDBEM_ERR_CUDA, "face apply kernel failed: %s", cudaGetErrorString((cudaError_t)e));
    return TDBEM_OK;
}

int apply_impl(tdbem_tensor *t, const void *W, int nrhs, void *y, int single_f) {
    cudaGetLastError();
    tdbem_ctx *ctx = t->ctx;
    if (nrhs < 1 || nrhs > 64 || !W || !y) return td_fail(ctx, TDBEM_ERR_ARG, "apply: need 1 <= nrhs <= 64 and non-NULL buffers");
    const size_t es = t->prec == TDBEM_FP64 ? sizeof(c64) : sizeof(c32);
    TD_CUDA(ctx, cudaMemsetAsync(y, 0, es * t->nrows * nrhs, ctx->stream));
    if (t->prec == TDBEM_MIXED && single_f < 0) return apply_tc(t, W, nrhs, y);
    ApplyArgs a{};
    a.nb = (int)t->nblocks;
    a.blocks = t->dblocks;
    a.perm_r = t->dperm_r;
    a.perm_c = t->dperm_c;
    a.Nu = t->Nu;
    a.NQ = t->NQ;
    a.qmap = t->dpartner;
    a.W = W;
    a.nrhs = nrhs;
    a.ncols = t->ncols;
    a.y = y;
    a.single_f = single_f;
    a.kcap = t->kcap;
    a.max_near_rows = t->max_near_rows;
    TensorOut o = tensor_out(t, nullptr);
    int e = td_launch_apply(ctx->stream, t->prec, a, o, ctx->num_sms);
    if (e) return td_fail(ctx, TDBEM_ERR_CUDA, "apply kernel failed: %s", cudaGetErrorString((cudaError_t)e));
    return TDBEM_OK;
}
}  // namespace

extern "C" int tdbem_apply_weighted(tdbem_tensor_t t, const void *W, int32_t nrhs, void *y) {
    if (!t) return TDBEM_ERR_ARG;
    return apply_impl(t, W, nrhs, y, -1);
}

extern "C" int tdbem_apply_freq(tdbem_tensor_t t, int32_t fidx, const void *x, int32_t nrhs, void *y) {
    if (!t) return TDBEM_ERR_ARG;
    if (fidx < 0 || fidx >= t->NQ) return td_fail(t->ctx, TDBEM_ERR_ARG, "frequency index out of range");
    return apply_impl(t, x, nrhs, y, fidx);
}

extern "C" int tdbem_apply_weighted_host(tdbem_tensor_t t, const void *W_host, int32_t nrhs, void *y_host) {
    if (!t || !W_host || !y_host || nrhs < 1 || nrhs > 64) return TDBEM_ERR_ARG;
    tdbem_ctx *ctx = t->ctx;
    const size_t es = t->prec == TDBEM_FP64 ? sizeof(c64) : sizeof(c32);
    const size_t wb = es * t->NQ * t->ncols * nrhs, yb = es * t->nrows * nrhs;
    if (wb + yb > t->host_buf_bytes) {
        if (t->dy_host) cudaFree(t->dy_host);
        t->dy_host = nullptr;
        t->host_buf_bytes = 0;
        char *p;
        int rc = dalloc(ctx, &p, wb + yb);
        if (rc) return rc;
        t->dy_host = p;
        t->host_buf_bytes = wb + yb;
    }
    char *dW = (char *)t->dy_host, *dy = dW + wb;
    TD_CUDA(ctx, cudaMemcpyAsync(dW, W_host, wb, cudaMemcpyHostToDevice, ctx->stream));
    int rc = apply_impl(t, dW, nrhs, dy, -1);
    if (rc) return rc;
    TD_CUDA(ctx, cudaMemcpyAsync(y_host, dy, yb, cudaMemcpyDeviceToHost, ctx->stream));
    TD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return TDBEM_OK;
}

// ============================================================================
// face-rank harvest (training samples of the rank predictor)
// ============================================================================
extern "C" int tdbem_harvest(tdbem_ctx_t ctx, tdbem_mesh_t mesh, const tdbem_op *op, tdbem_freqs_t f, tdbem_tree_t tree,
                             const tdbem_aca_cfg *cfg, float *feats, int32_t *ranks, int64_t capacity, int64_t *count) {
    if (!ctx || !mesh || !f || !tree || !cfg || !count) return td_fail(ctx, TDBEM_ERR_ARG, "tdbem_harvest: NULL argument");
    cudaGetLastError();
    int rc = td_check_op(ctx, op);
    if (rc) return rc;
    if (tree->mesh != mesh || tree->side[0].basis != TDBEM_P0 ||
        tree->side[1].basis != (op->op == TDBEM_DLP ? TDBEM_P1 : TDBEM_P0))
        return td_fail(ctx, TDBEM_ERR_ARG, "tree does not match mesh and operator");
    if (f->Nu > 256) return td_fail(ctx, TDBEM_ERR_ARG, "at most 256 unique frequencies are supported");
    const int Nu = f->Nu;
    std::vector<int32_t> far_ids;
    int maxI = 1, maxJ = 1;
    const int64_t nb = (int64_t)tree->blocks.size() / 5;
    for (int64_t b = 0; b < nb; ++b) {
        const int32_t *bl = &tree->blocks[5 * b];
        if (!bl[4]) continue;
        far_ids.push_back((int32_t)b);
        maxI = std::max(maxI, bl[1] - bl[0]);
        maxJ = std::max(maxJ, bl[3] - bl[2]);
    }
    *count = (int64_t)far_ids.size() * Nu;
    if (!feats || !ranks) return TDBEM_OK;
    if (capacity < *count) return td_fail(ctx, TDBEM_ERR_ARG, "capacity %lld < %lld samples", (long long)capacity, (long long)*count);
    if (*count == 0) return TDBEM_OK;
    std::vector<float> x;
    td_block_features(tree, tree->blocks, mesh, f, op->c, far_ids, x);
    if ((rc = upload(ctx, feats, x.data(), x.size()))) return rc;
    const int kcap = cfg->max_face_rank > 0 ? std::min(cfg->max_face_rank, 64) : 64;
    Guard g;
    int32_t *dblocks, *dpr, *dpc, *dfar, *flags, *drank;
    double *sig;
    char *scr;
    unsigned int *counter;
    std::vector<double> hs(2 * Nu);
    for (int u = 0; u < Nu; ++u) {
        hs[2 * u] = f->s[2 * f->uidx[u]] / op->c;
        hs[2 * u + 1] = f->s[2 * f->uidx[u] + 1] / op->c;
    }
    const size_t es = op->prec == TDBEM_FP64 ? sizeof(c64) : sizeof(c32);
    const int pf = op->prec == TDBEM_MIXED ? 1 : 0;
    const int nctas = std::min<int64_t>(*count, (int64_t)ctx->num_sms * ctx->far_cps[pf]);
    const int64_t sper = (int64_t)kcap * (maxI + maxJ);
    if ((rc = dalloc(ctx, &dblocks, 5 * nb, &g.p)) || (rc = dalloc(ctx, &dpr, tree->side[0].n, &g.p)) ||
        (rc = dalloc(ctx, &dpc, tree->side[1].n, &g.p)) || (rc = dalloc(ctx, &dfar, far_ids.size(), &g.p)) ||
        (rc = dalloc(ctx, &flags, 4, &g.p)) || (rc = dalloc(ctx, &drank, nb, &g.p)) || (rc = dalloc(ctx, &sig, 2 * Nu, &g.p)) ||
        (rc = dalloc(ctx, &scr, es * sper * nctas, &g.p)) || (rc = dalloc(ctx, &counter, 4, &g.p)))
        return rc;
    if ((rc = upload(ctx, dblocks, tree->blocks.data(), 5 * nb)) || (rc = upload(ctx, dpr, tree->side[0].perm.data(), tree->side[0].n)) ||
        (rc = upload(ctx, dpc, tree->side[1].perm.data(), tree->side[1].n)) ||
        (rc = upload(ctx, dfar, far_ids.data(), far_ids.size())) || (rc = upload(ctx, sig, hs.data(), hs.size())))
        return rc;
    cudaMemsetAsync(flags, 0, sizeof(int32_t) * 4, ctx->stream);
    cudaMemsetAsync(counter, 0, sizeof(unsigned int) * 4, ctx->stream);
    MeshDev md = td_mesh_dev(mesh, op->ng, nullptr, nullptr, nullptr);  // far blocks have no touching pairs
    FarArgs fa{};
    fa.nfar = (int)far_ids.size();
    fa.far_ids = dfar;
    fa.blocks = dblocks;
    fa.perm_r = dpr;
    fa.perm_c = dpc;
    fa.sig = sig;
    fa.nf = Nu;
    fa.maxI = maxI;
    fa.maxJ = maxJ;
    fa.scratch = scr;
    fa.scratch_per_cta = sper;
    fa.counter = counter;
    fa.harvest = ranks;
    TensorOut o{};
    o.Nu = Nu;
    o.rank = drank;
    o.dev_flags = flags;
    AcaParams ap{cfg->eps, cfg->eps_aca, kcap};
    if (td_launch_far_aca(ctx->stream, md, op->op, op->prec, fa, o, ap, nctas, ctx->far_nt[pf]))
        return td_fail(ctx, TDBEM_ERR_CUDA, "harvest kernel launch failed");
    TD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return TDBEM_OK;
}

// ============================================================================
// autotuner of the far-field launch shape
// ============================================================================
extern "C" int tdbem_autotune(tdbem_ctx_t ctx, tdbem_mesh_t mesh, const tdbem_op *op, tdbem_freqs_t f,
                              tdbem_tree_t tree, const tdbem_aca_cfg *cfg, int32_t *chosen) {
    if (!ctx || !op) return TDBEM_ERR_ARG;
    const int pf = op->prec == TDBEM_MIXED ? 1 : 0;
    // times a complete compression (the first of two runs warms up) and
    // returns its statistics
    auto run = [&](tdbem_stats &st) {
        for (int rep = 0; rep < 2; ++rep) {
            tdbem_tensor_t X = nullptr;
            const int rc = tdbem_compress(ctx, mesh, op, f, tree, cfg, &X);
            if (rc) return rc;
            if (rep == 1) st = X->stats;
            tdbem_tensor_destroy(X);
        }
        return (int)TDBEM_OK;
    };
    // 1. far phase: threads per CTA x resident CTAs per SM (CTAs beyond what the
    // registers and shared memory of an SM hold start only when resident ones
    // exit, i.e. once the work queue is empty)
    static const int cand[][2] = {{256, 2}, {128, 4}, {128, 5}, {64, 8}, {64, 10}, {64, 16}};
    double best = 1e300;
    int bnt = ctx->far_nt[pf], bcps = ctx->far_cps[pf];
    for (const auto &c : cand) {
        ctx->far_nt[pf] = c[0];
        ctx->far_cps[pf] = c[1];
        tdbem_stats st{};
        const int rc = run(st);
        if (rc) {
            ctx->far_nt[pf] = bnt;
            ctx->far_cps[pf] = bcps;
            return rc;
        }
        if (st.ms_far < best) {
            best = st.ms_far;
            bnt = c[0];
            bcps = c[1];
        }
    }
    ctx->far_nt[pf] = bnt;
    ctx->far_cps[pf] = bcps;
    // 2. mixed form: frequencies per pass of the touching-pair table and of the
    // near-field tensor kernel (register tiles of FC frequencies), each phase
    // timed on its own from the same compressions
    int bsing = ctx->sing_var, bnear = ctx->near_var;
    if (pf) {
        double ts = 1e300, tn = 1e300;
        for (int v = 0; v < 3; ++v) {
            ctx->sing_var = ctx->near_var = v;
            tdbem_stats st{};
            const int rc = run(st);
            if (rc) {
                ctx->sing_var = bsing;
                ctx->near_var = bnear;
                return rc;
            }
            if (st.ms_singular < ts) {
                ts = st.ms_singular;
                bsing = v;
            }
            if (st.ms_near < tn) {
                tn = st.ms_near;
                bnear = v;
            }
        }
        ctx->sing_var = bsing;
        ctx->near_var = bnear;
    }
    if (chosen) {
        chosen[0] = bnt;
        chosen[1] = bcps;
        chosen[2] = pf ? td_sing_fc(op->op, bsing) : 0;
        chosen[3] = pf ? td_near_fc(bnear) : 0;
    }
    return TDBEM_OK;
}

// ============================================================================
// tensor-core complex GEMM (the engine of the weighted apply)
// ============================================================================
extern "C" int tdbem_zgemm(tdbem_ctx_t ctx, int32_t M, int32_t N, int32_t K, const void *A, int64_t lda,
                           const void *B, int64_t ldb, void *D, int64_t ldd) {
    if (!ctx) return TDBEM_ERR_ARG;
    cudaGetLastError();
    if (M < 0 || N < 0 || K < 0 || (M * (int64_t)N > 0 && (!D || (K > 0 && (!A || !B)))) || lda < K || ldb < N ||
        ldd < N)
        return td_fail(ctx, TDBEM_ERR_ARG, "tdbem_zgemm: bad sizes or NULL pointers");
    if ((int64_t)M * N == 0) return TDBEM_OK;
    if (K == 0) {
        for (int m = 0; m < M; ++m)
            TD_CUDA(ctx, cudaMemsetAsync((c32 *)D + (int64_t)m * ldd, 0, sizeof(c32) * N, ctx->stream));
        return tdbem_ctx_sync(ctx);
    }
    const int TM = td_zgemm_tile_rows(), TN = td_zgemm_tile_cols();
    std::vector<ZJob> jobs;
    for (int m0 = 0; m0 < M; m0 += TM)
        for (int n0 = 0; n0 < N; n0 += TN) jobs.push_back(ZJob{0, m0, n0, 0});
    ZJob *dj = nullptr;
    if (cudaMalloc(&dj, sizeof(ZJob) * jobs.size()) != cudaSuccess) {
        cudaGetLastError();
        return td_fail(ctx, TDBEM_ERR_OOM, "tdbem_zgemm: job list allocation failed");
    }
    int rc = TDBEM_OK;
    if (cudaMemcpyAsync(dj, jobs.data(), sizeof(ZJob) * jobs.size(), cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess)
        rc = td_fail(ctx, TDBEM_ERR_CUDA, "tdbem_zgemm: upload failed");
    if (!rc) {
        int e = td_launch_zgemm_dense(ctx->stream, (const c32 *)A, lda, (const c32 *)B, ldb, (c32 *)D, ldd, M, N, K,
                                      dj, (int)jobs.size(), ctx->dflags, ctx->wait_polls, ctx->num_sms);
        if (e) rc = td_fail(ctx, TDBEM_ERR_CUDA, "tdbem_zgemm: launch failed: %s", cudaGetErrorString((cudaError_t)e));
    }
    if (!rc) rc = tdbem_ctx_sync(ctx);
    cudaFree(dj);
    return rc;
}
