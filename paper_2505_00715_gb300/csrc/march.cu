// gCQ time marching (Sec. 3 "Temporal discretisation", eqs. gCQ_xn and
// gcq_formula; App. A) of the direct Dirichlet problem of Sec. 2 in its
// Galerkin form with piecewise constant test functions:
//
//   V * q = (1/2 M + K) * g,   M[i][v] = int_{tau_i} phi_v (P0 x P1 mass),
//
// g the Dirichlet data (P1 nodal values), q the Neumann data (P0).  Step n
// (size dt_n, Runge-Kutta matrix A with b^T A^{-1} = (0, .., 1)):
//
//   x_{n-1}(s_l) = (I - dt_{n-1} s_l A)^{-1} (last(x_{n-2}(s_l)) 1 + dt_{n-1} A q_{n-1})
//   W_l          = -w_l last(x_{n-1}(s_l)) (I - dt_n s_l A)^{-1} 1
//   V((dt_n A)^{-1}) q_n = 1/2 M g_n + K((dt_n A)^{-1}) g_n + sum_l K(s_l) W_l[g] - sum_l V(s_l) W_l[q]
//
// with w_l the positively oriented Cauchy weights of the contour (so that
// -w_l are the weights omega_l of eq. gcq_formula).  The operator at the
// matrix argument acts through the eigen-decomposition (dt A)^{-1} = P
// diag(mu_k) P^{-1} over the stage index: every mu_k = 1/(dt lambda_k) is a
// point of the step tensors' frequency set.  The history sums are the
// multi-frequency apply (tdbem_apply_weighted) over the contour tensors, the
// step operators the single-frequency apply and GMRES (tdbem_apply_freq,
// tdbem_solve) over the step tensors.  The states x(s_l) of q and g are kept
// in FP64 for the unique contour points (x(conj s) = conj x(s) for real
// data); every arithmetic step runs in the kernels below.
#include <algorithm>
#include <cmath>
#include <complex>
#include <new>
#include <vector>

#include "internal.h"
#include "kernels.h"

namespace {

using zc = std::complex<double>;

// Runge-Kutta matrix (m <= 2) passed by value to the kernels.
struct RkMat {
    int m;
    double a[2][2];
};

// x = (I - h s A)^{-1} v for m <= 2 (Cramer's rule), complex s.
TD_D void rk_solve(const RkMat &A, c64 hs, const c64 *v, c64 *x) {
    if (A.m == 1) {
        const c64 d = {1.0 - hs.x * A.a[0][0], -hs.y * A.a[0][0]};
        x[0] = cdiv(v[0], d);
        return;
    }
    // M = I - hs A
    c64 M[2][2];
    for (int i = 0; i < 2; ++i)
        for (int k = 0; k < 2; ++k) M[i][k] = c64{(i == k ? 1.0 : 0.0) - hs.x * A.a[i][k], -hs.y * A.a[i][k]};
    const c64 det = M[0][0] * M[1][1] - M[0][1] * M[1][0];
    x[0] = cdiv(M[1][1] * v[0] - M[0][1] * v[1], det);
    x[1] = cdiv(M[0][0] * v[1] - M[1][0] * v[0], det);
}

// States of one data series at the unique contour points:
// X[u][j][i][r] <- (I - dtp s_u A)^{-1} (X[u][j][m-1][r] 1 + dtp A D[j][.][r])
__global__ void k_march_advance(c64 *X, const double *D, const double *sq, const int *uidx, int Nu, int64_t n,
                                int nrhs, double dtp, RkMat A) {
    const int m = A.m;
    const int64_t total = (int64_t)Nu * n * nrhs;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(t % nrhs);
        const int64_t j = (t / nrhs) % n;
        const int u = (int)(t / ((int64_t)nrhs * n));
        const int l = uidx[u];
        const c64 hs = {dtp * sq[2 * l], dtp * sq[2 * l + 1]};
        c64 *x = X + ((int64_t)u * n + j) * m * nrhs;
        const c64 xend = x[(int64_t)(m - 1) * nrhs + r];
        c64 v[2], y[2];
        for (int i = 0; i < m; ++i) {
            double ad = 0.0;
            for (int k = 0; k < m; ++k) ad += A.a[i][k] * D[(j * m + k) * nrhs + r];
            v[i] = c64{xend.x + dtp * ad, xend.y};
        }
        rk_solve(A, hs, v, y);
        for (int i = 0; i < m; ++i) x[(int64_t)i * nrhs + r] = y[i];
    }
}

// W[l][j][i nrhs + r] = -w_l last(x(s_l))[j][r] ((I - dt s_l A)^{-1} 1)_i for
// every contour point l (conjugate points from their representative).
template <class T>
__global__ void k_march_weights(const c64 *X, const double *sq, const double *wq, const int *qmap, int NQ, int64_t n,
                                int nrhs, double dt, RkMat A, cx<T> *W) {
    const int m = A.m;
    const int64_t total = (int64_t)NQ * n * nrhs;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(t % nrhs);
        const int64_t j = (t / nrhs) % n;
        const int l = (int)(t / ((int64_t)nrhs * n));
        const int q = qmap[l];
        const int u = (q > 0 ? q : -q) - 1;
        c64 xe = X[(((int64_t)u * n + j) * m + (m - 1)) * nrhs + r];
        if (q < 0) xe = cconj(xe);
        const c64 hs = {dt * sq[2 * l], dt * sq[2 * l + 1]};
        const c64 one[2] = {{1.0, 0.0}, {1.0, 0.0}};
        c64 r1[2];
        rk_solve(A, hs, one, r1);
        const c64 wl = {-wq[2 * l], -wq[2 * l + 1]};
        const c64 c = wl * xe;
        for (int i = 0; i < m; ++i) {
            const c64 v = c * r1[i];
            W[((int64_t)l * n + j) * m * nrhs + (int64_t)i * nrhs + r] = cx<T>{(T)v.x, (T)v.y};
        }
    }
}

// out[i][c] = 1/2 (|tau_i| / 3) sum_{v in tau_i} g[v][c]   (P0 x P1 mass, halved)
template <class T>
__global__ void k_march_mass(const double *g, const int *tris, const double *area, int64_t nt, int ncol, cx<T> *out) {
    const int64_t total = nt * ncol;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(t % ncol);
        const int64_t i = t / ncol;
        const double s = g[(int64_t)tris[3 * i] * ncol + c] + g[(int64_t)tris[3 * i + 1] * ncol + c] +
                         g[(int64_t)tris[3 * i + 2] * ncol + c];
        out[t] = cx<T>{(T)(area[i] * s / 6.0), (T)0};
    }
}

// out[j][r] = sum_i coef_i in[j][i][r]: stage data to one eigen-coordinate
// (real input) ...
template <class T>
__global__ void k_stage_to_eig_real(const double *in, int64_t n, int m, int nrhs, c64 c0, c64 c1, cx<T> *out) {
    const int64_t total = n * nrhs;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(t % nrhs);
        const int64_t j = t / nrhs;
        const double a = in[(j * m) * nrhs + r];
        c64 v = {c0.x * a, c0.y * a};
        if (m > 1) {
            const double b = in[(j * m + 1) * nrhs + r];
            v = v + c64{c1.x * b, c1.y * b};
        }
        out[t] = cx<T>{(T)v.x, (T)v.y};
    }
}

// acc[j][i][r] += coef_i y[j][r]  (eigen-coordinate back to stage data)
template <class T>
__global__ void k_stage_from_eig(const cx<T> *y, int64_t n, int m, int nrhs, c64 c0, c64 c1, cx<T> *acc) {
    const int64_t total = n * nrhs;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(t % nrhs);
        const int64_t j = t / nrhs;
        const c64 v = {(double)y[t].x, (double)y[t].y};
        for (int i = 0; i < m; ++i) {
            const c64 c = i == 0 ? c0 : c1;
            const c64 p = c * v;
            cx<T> &a = acc[(j * m + i) * nrhs + r];
            a = cx<T>{(T)((double)a.x + p.x), (T)((double)a.y + p.y)};
        }
    }
}

// rhs = a + b - c, keeping the real part (the data of the physical problem
// are real; the conjugate-symmetric contour sums are real up to rounding)
template <class T>
__global__ void k_march_rhs(const cx<T> *a, const cx<T> *b, const cx<T> *c, int64_t total, double *out) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        double v = (double)a[t].x;
        if (b) v += (double)b[t].x;
        if (c) v -= (double)c[t].x;
        out[t] = v;
    }
}

// q[j][i][r] = Re sum_k P[i][k] qt_k[j][r]; qt_1 = conj(qt_0) when the step
// eigenvalues are a conjugate pair (conj_pair), else qt_1 given
template <class T>
__global__ void k_march_q(const cx<T> *qt0, const cx<T> *qt1, int64_t n, int m, int nrhs, c64 p00, c64 p01, c64 p10,
                          c64 p11, int conj_pair, double *q) {
    const int64_t total = n * nrhs;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(t % nrhs);
        const int64_t j = t / nrhs;
        const c64 a = {(double)qt0[t].x, (double)qt0[t].y};
        if (m == 1) {
            q[j * nrhs + r] = (p00 * a).x;
            continue;
        }
        c64 b = conj_pair ? cconj(a) : c64{(double)qt1[t].x, (double)qt1[t].y};
        q[(j * 2) * nrhs + r] = (p00 * a + p01 * b).x;
        q[(j * 2 + 1) * nrhs + r] = (p10 * a + p11 * b).x;
    }
}

int grid_for(int64_t n, int sms) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8)); }

// Butcher matrix, its eigenvalues and eigenvectors (P columns), P^{-1}.
struct RkData {
    RkMat A;
    zc lam[2], P[2][2], Pi[2][2];
};

RkData rk_data(int rk) {
    RkData d{};
    if (rk == TDBEM_RADAU2) {
        d.A.m = 2;
        d.A.a[0][0] = 5.0 / 12.0;
        d.A.a[0][1] = -1.0 / 12.0;
        d.A.a[1][0] = 3.0 / 4.0;
        d.A.a[1][1] = 1.0 / 4.0;
        const double tr = d.A.a[0][0] + d.A.a[1][1];
        const double det = d.A.a[0][0] * d.A.a[1][1] - d.A.a[0][1] * d.A.a[1][0];
        const zc disc = std::sqrt(zc(tr * tr - 4.0 * det, 0.0));
        d.lam[0] = 0.5 * (tr + disc);
        d.lam[1] = 0.5 * (tr - disc);
        for (int k = 0; k < 2; ++k) {  // (A - lam I) v = 0 -> v = (a01, lam - a00)
            d.P[0][k] = d.A.a[0][1];
            d.P[1][k] = d.lam[k] - d.A.a[0][0];
        }
        const zc dp = d.P[0][0] * d.P[1][1] - d.P[0][1] * d.P[1][0];
        d.Pi[0][0] = d.P[1][1] / dp;
        d.Pi[0][1] = -d.P[0][1] / dp;
        d.Pi[1][0] = -d.P[1][0] / dp;
        d.Pi[1][1] = d.P[0][0] / dp;
    } else {
        d.A.m = 1;
        d.A.a[0][0] = 1.0;
        d.lam[0] = 1.0;
        d.P[0][0] = d.Pi[0][0] = 1.0;
    }
    return d;
}

c64 to_c64(zc z) { return c64{z.real(), z.imag()}; }

}  // namespace

struct tdbem_march {
    tdbem_ctx *ctx = nullptr;
    tdbem_tensor *V = nullptr, *K = nullptr, *Vs = nullptr, *Ks = nullptr;
    int rk = 0, m = 1, nrhs = 1, N = 0, n = 0, NQ = 0, Nu = 0;
    int64_t nt = 0, nv = 0;
    size_t es = 8;
    const int *mesh_tris = nullptr;          // device tables of the mesh
    const double *mesh_area = nullptr;
    std::vector<double> dts;
    RkData R{};
    std::vector<void *> mem;
    c64 *Xq = nullptr, *Xg = nullptr;        // states at the unique contour points [Nu][n][m][nrhs]
    double *Qp = nullptr, *Gp = nullptr;     // previous stage data [n][m][nrhs]
    int *qmap = nullptr, *uidx = nullptr;    // contour unique map [NQ], representatives [Nu]
    void *Wq = nullptr, *Wg = nullptr;       // [NQ][n][m nrhs] in the tensors' precision
    void *Hq = nullptr, *Hg = nullptr;       // history sums [nt][m nrhs]
    void *R1 = nullptr;                      // 1/2 M g + K(B) g [nt][m nrhs]
    void *E1 = nullptr, *E2 = nullptr, *E3 = nullptr;  // eigen-coordinate buffers [max(nt, nv)][nrhs] x 3
    double *rhs = nullptr;                   // real right-hand side [nt][m][nrhs]
    ~tdbem_march() {
        for (void *p : mem) cudaFree(p);
    }
};

namespace {

template <class P>
int mk(tdbem_march *M, P **p, size_t bytes) {
    *p = nullptr;
    if (cudaMalloc((void **)p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
        cudaGetLastError();
        return td_fail(M->ctx, TDBEM_ERR_OOM, "tdbem_march: device allocation of %zu bytes failed", bytes);
    }
    M->mem.push_back((void *)*p);
    return TDBEM_OK;
}

// index of the point mu in the frequency set of tensor t (full list), or -1
int find_point(const tdbem_tensor *t, zc mu) {
    const tdbem_freqs *f = t->freqs;
    if (!f) return -1;
    for (int k = 0; k < f->NQ; ++k) {
        const zc s(f->s[2 * k], f->s[2 * k + 1]);
        if (std::abs(s - mu) <= 1e-10 * std::abs(mu)) return k;
    }
    return -1;
}

template <class T>
int march_step_t(tdbem_march *M, const double *g, double *q, double tol, int maxit, int *iters) {
    tdbem_ctx *ctx = M->ctx;
    cudaStream_t st = ctx->stream;
    const int sms = ctx->num_sms;
    const int m = M->m, nrhs = M->nrhs, mr = m * nrhs;
    const int64_t nt = M->nt, nv = M->nv;
    const double dt = M->dts[M->n];
    const tdbem_freqs *fc = M->V->freqs;
    cx<T> *Hq = (cx<T> *)M->Hq, *Hg = (cx<T> *)M->Hg, *R1 = (cx<T> *)M->R1;
    cx<T> *E1 = (cx<T> *)M->E1, *E2 = (cx<T> *)M->E2, *E3 = (cx<T> *)M->E3;
    int rc;
    bool hist = M->n > 0;
    if (hist) {
        const double dtp = M->dts[M->n - 1];
        k_march_advance<<<grid_for((int64_t)M->Nu * nt * nrhs, sms), 256, 0, st>>>(M->Xq, M->Qp, fc->ds, M->uidx, M->Nu,
                                                                                 nt, nrhs, dtp, M->R.A);
        k_march_advance<<<grid_for((int64_t)M->Nu * nv * nrhs, sms), 256, 0, st>>>(M->Xg, M->Gp, fc->ds, M->uidx, M->Nu,
                                                                                 nv, nrhs, dtp, M->R.A);
        k_march_weights<T><<<grid_for((int64_t)M->NQ * nt * nrhs, sms), 256, 0, st>>>(
            M->Xq, fc->ds, fc->dw, M->qmap, M->NQ, nt, nrhs, dt, M->R.A, (cx<T> *)M->Wq);
        k_march_weights<T><<<grid_for((int64_t)M->NQ * nv * nrhs, sms), 256, 0, st>>>(
            M->Xg, fc->ds, fc->dw, M->qmap, M->NQ, nv, nrhs, dt, M->R.A, (cx<T> *)M->Wg);
        if (cudaPeekAtLastError() != cudaSuccess)
            return td_fail(ctx, TDBEM_ERR_CUDA, "tdbem_march_step: state kernels failed: %s",
                           cudaGetErrorString(cudaGetLastError()));
        if ((rc = tdbem_apply_weighted(M->V, M->Wq, mr, Hq)) || (rc = tdbem_apply_weighted(M->K, M->Wg, mr, Hg))) return rc;
    }
    // R1 = 1/2 M g + K((dt A)^{-1}) g
    k_march_mass<T><<<grid_for(nt * mr, sms), 256, 0, st>>>(g, M->mesh_tris, M->mesh_area, nt, mr, R1);
    zc mu[2];
    int idxK[2], idxV[2];
    for (int k = 0; k < m; ++k) {
        mu[k] = 1.0 / (dt * M->R.lam[k]);
        idxK[k] = find_point(M->Ks, mu[k]);
        idxV[k] = find_point(M->Vs, mu[k]);
        if (idxK[k] < 0 || idxV[k] < 0)
            return td_fail(ctx, TDBEM_ERR_ARG, "tdbem_march_step: the step tensors' frequency set lacks 1/(dt lambda) "
                                               "= %g%+gi of step %d", mu[k].real(), mu[k].imag(), M->n);
    }
    for (int k = 0; k < m; ++k) {
        k_stage_to_eig_real<T><<<grid_for(nv * nrhs, sms), 256, 0, st>>>(g, nv, m, nrhs, to_c64(M->R.Pi[k][0]),
                                                                        to_c64(m > 1 ? M->R.Pi[k][1] : zc(0.0)), E1);
        if ((rc = tdbem_apply_freq(M->Ks, idxK[k], E1, nrhs, E2))) return rc;
        k_stage_from_eig<T><<<grid_for(nt * nrhs, sms), 256, 0, st>>>(E2, nt, m, nrhs, to_c64(M->R.P[0][k]),
                                                                     to_c64(m > 1 ? M->R.P[1][k] : zc(0.0)), R1);
    }
    k_march_rhs<T><<<grid_for(nt * mr, sms), 256, 0, st>>>(R1, hist ? Hg : nullptr, hist ? Hq : nullptr, nt * mr, M->rhs);
    // V((dt A)^{-1}) q = rhs through the eigen-coordinates; for a conjugate pair
    // of step eigenvalues (real data) the second solution is the conjugate of the first
    const bool conj_pair = m == 2 && std::abs(mu[1] - std::conj(mu[0])) <= 1e-12 * std::abs(mu[0]);
    int it_total = 0;
    cx<T> *qt[2] = {E2, E3};
    for (int k = 0; k < (conj_pair ? 1 : m); ++k) {
        k_stage_to_eig_real<T><<<grid_for(nt * nrhs, sms), 256, 0, st>>>(M->rhs, nt, m, nrhs, to_c64(M->R.Pi[k][0]),
                                                                        to_c64(m > 1 ? M->R.Pi[k][1] : zc(0.0)), E1);
        int it = 0;
        rc = tdbem_solve(M->Vs, idxV[k], E1, nrhs, qt[k], tol, maxit, 0, &it, nullptr);
        it_total += it;
        if (rc) return rc;
    }
    k_march_q<T><<<grid_for(nt * nrhs, sms), 256, 0, st>>>(
        qt[0], qt[1], nt, m, nrhs, to_c64(M->R.P[0][0]), to_c64(m > 1 ? M->R.P[0][1] : zc(0.0)),
        to_c64(m > 1 ? M->R.P[1][0] : zc(0.0)), to_c64(m > 1 ? M->R.P[1][1] : zc(0.0)), conj_pair ? 1 : 0, q);
    // the stage data of this step become the previous data of the next one
    TD_CUDA(ctx, cudaMemcpyAsync(M->Qp, q, sizeof(double) * nt * mr, cudaMemcpyDeviceToDevice, st));
    TD_CUDA(ctx, cudaMemcpyAsync(M->Gp, g, sizeof(double) * nv * mr, cudaMemcpyDeviceToDevice, st));
    TD_CUDA(ctx, cudaStreamSynchronize(st));
    if (iters) *iters = it_total;
    ++M->n;
    return TDBEM_OK;
}

}  // namespace

extern "C" int tdbem_march_step_points(const double *dts, int32_t N, int32_t rk, double *s, int32_t *count) {
    if (!dts || N < 1 || !count || (rk != TDBEM_EULER && rk != TDBEM_RADAU2)) return TDBEM_ERR_ARG;
    const RkData R = rk_data(rk);
    std::vector<zc> pts;
    for (int n = 0; n < N; ++n) {
        if (!(dts[n] > 0.0) || !std::isfinite(dts[n])) return TDBEM_ERR_ARG;
        for (int k = 0; k < R.A.m; ++k) {
            const zc mu = 1.0 / (dts[n] * R.lam[k]);
            bool seen = false;
            for (const zc &p : pts) seen = seen || std::abs(p - mu) <= 1e-12 * std::abs(mu);
            if (!seen) pts.push_back(mu);
        }
    }
    if (s)
        for (size_t k = 0; k < pts.size(); ++k) {
            s[2 * k] = pts[k].real();
            s[2 * k + 1] = pts[k].imag();
        }
    *count = (int32_t)pts.size();
    return TDBEM_OK;
}

extern "C" int tdbem_march_create(tdbem_tensor_t V, tdbem_tensor_t K, tdbem_tensor_t Vs, tdbem_tensor_t Ks,
                                  const double *dts, int32_t N, int32_t rk, int32_t nrhs, tdbem_march_t *out) {
    if (!V || !K || !Vs || !Ks || !out) return TDBEM_ERR_ARG;
    tdbem_ctx *ctx = V->ctx;
    *out = nullptr;
    if (!dts || N < 1 || (rk != TDBEM_EULER && rk != TDBEM_RADAU2) || nrhs < 1)
        return td_fail(ctx, TDBEM_ERR_ARG, "tdbem_march_create: need N >= 1 steps, rk EULER|RADAU2, nrhs >= 1");
    const RkData R = rk_data(rk);
    if (R.A.m * nrhs > 64) return td_fail(ctx, TDBEM_ERR_ARG, "tdbem_march_create: stages x nrhs must be <= 64");
    if (V->op != TDBEM_SLP || Vs->op != TDBEM_SLP || K->op != TDBEM_DLP || Ks->op != TDBEM_DLP)
        return td_fail(ctx, TDBEM_ERR_ARG, "tdbem_march_create: V, Vstep must be single-layer and K, Kstep "
                                           "double-layer tensors");
    if (V->prec != K->prec || V->prec != Vs->prec || V->prec != Ks->prec || V->mesh != K->mesh ||
        V->mesh != Vs->mesh || V->mesh != Ks->mesh || V->c != K->c || V->c != Vs->c || V->c != Ks->c)
        return td_fail(ctx, TDBEM_ERR_ARG, "tdbem_march_create: the four tensors need one mesh, precision and wave "
                                           "speed");
    if (!V->freqs || V->freqs != K->freqs || V->freqs->kind != 1 || !Vs->freqs || !Ks->freqs)
        return td_fail(ctx, TDBEM_ERR_ARG, "tdbem_march_create: V and K must be compressed over one gCQ contour, "
                                           "Vstep and Kstep over a frequency set");
    for (int n = 0; n < N; ++n)
        if (!(dts[n] > 0.0) || !std::isfinite(dts[n])) return td_fail(ctx, TDBEM_ERR_ARG, "tdbem_march_create: bad step %d", n);
    tdbem_march *M = new (std::nothrow) tdbem_march();
    if (!M) return TDBEM_ERR_OOM;
    M->ctx = ctx;
    M->V = V;
    M->K = K;
    M->Vs = Vs;
    M->Ks = Ks;
    M->rk = rk;
    M->R = R;
    M->m = R.A.m;
    M->nrhs = nrhs;
    M->N = N;
    M->dts.assign(dts, dts + N);
    M->nt = V->nrows;
    M->nv = K->ncols;
    M->NQ = V->freqs->NQ;
    M->Nu = V->freqs->Nu;
    M->es = V->prec == TDBEM_FP64 ? sizeof(c64) : sizeof(c32);
    M->mesh_tris = V->mesh->dtris;
    M->mesh_area = V->mesh->darea;
    const int mr = M->m * nrhs;
    const int64_t nmax = std::max(M->nt, M->nv);
    int rc;
    if ((rc = mk(M, &M->Xq, sizeof(c64) * M->Nu * M->nt * mr)) || (rc = mk(M, &M->Xg, sizeof(c64) * M->Nu * M->nv * mr)) ||
        (rc = mk(M, &M->Qp, sizeof(double) * M->nt * mr)) || (rc = mk(M, &M->Gp, sizeof(double) * M->nv * mr)) ||
        (rc = mk(M, &M->qmap, sizeof(int) * M->NQ)) || (rc = mk(M, &M->uidx, sizeof(int) * M->Nu)) ||
        (rc = mk(M, &M->Wq, M->es * M->NQ * M->nt * mr)) || (rc = mk(M, &M->Wg, M->es * M->NQ * M->nv * mr)) ||
        (rc = mk(M, &M->Hq, M->es * M->nt * mr)) || (rc = mk(M, &M->Hg, M->es * M->nt * mr)) ||
        (rc = mk(M, &M->R1, M->es * M->nt * mr)) || (rc = mk(M, &M->E1, M->es * nmax * nrhs)) ||
        (rc = mk(M, &M->E2, M->es * nmax * nrhs)) || (rc = mk(M, &M->E3, M->es * nmax * nrhs)) ||
        (rc = mk(M, &M->rhs, sizeof(double) * M->nt * mr))) {
        delete M;
        return rc;
    }
    cudaStream_t st = ctx->stream;
    if (cudaMemsetAsync(M->Xq, 0, sizeof(c64) * M->Nu * M->nt * mr, st) != cudaSuccess ||
        cudaMemsetAsync(M->Xg, 0, sizeof(c64) * M->Nu * M->nv * mr, st) != cudaSuccess ||
        cudaMemcpyAsync(M->qmap, V->freqs->unique.data(), sizeof(int) * M->NQ, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(M->uidx, V->freqs->uidx.data(), sizeof(int) * M->Nu, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        delete M;
        return td_fail(ctx, TDBEM_ERR_CUDA, "tdbem_march_create: initialisation failed");
    }
    *out = M;
    return TDBEM_OK;
}

extern "C" int tdbem_march_step(tdbem_march_t M, const double *g, double *q, double tol, int32_t maxit, int32_t *iters) {
    if (!M) return TDBEM_ERR_ARG;
    cudaGetLastError();
    if (!g || !q || !(tol > 0.0) || maxit < 1)
        return td_fail(M->ctx, TDBEM_ERR_ARG, "tdbem_march_step: need device g, q, tol > 0, maxit >= 1");
    if (M->n >= M->N) return td_fail(M->ctx, TDBEM_ERR_ARG, "tdbem_march_step: all %d steps are done", M->N);
    return M->es == sizeof(c64) ? march_step_t<double>(M, g, q, tol, maxit, iters)
                                : march_step_t<float>(M, g, q, tol, maxit, iters);
}

extern "C" int tdbem_march_destroy(tdbem_march_t M) {
    delete M;
    return TDBEM_OK;
}
