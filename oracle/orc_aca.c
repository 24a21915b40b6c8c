/*
 * Oracle (test infrastructure only): ACA, 3D-ACA and the compressed apply.
 *
 * Sec. 4: the operator tensor C (rows x cols x frequencies) is approximated
 * per block of the block cluster tree by a sum of outer products
 * C^(l) = sum_d H_d (x) f_d  (eq. outerProd), built by Algorithm 1:
 *   l = 0, k_1 = first frequency;
 *   repeat: l += 1;
 *     H_l = ENTRY(., ., k_l) - C^(l-1)(., ., k_l)          (the residual face)
 *     (i_l, j_l) = argmax |H_l|
 *     f_l[k] = (ENTRY(i_l, j_l, k) - C^(l-1)(i_l, j_l, k)) / H_l[i_l, j_l]
 *     C^(l) = C^(l-1) + H_l (x) f_l
 *     k_{l+1} = argmax_k |f_l[k]|
 *   until ||H_l||_F ||f_l||_2 <= eps ||C^(l)||_F;  r = l - 1,
 * with ||C^(l)||_F^2 = sum_{d,d'} <H_d, H_d'> <f_d, f_d'> (eq. norm),
 * <A, B> = sum A conj(B).  Near-field blocks use dense residual faces; far
 * field blocks compress each residual face by ACA with partial pivoting to
 * eps_aca, rebuild it densely to find the pivot and discard the dense copy
 * (Sec. 4, last paragraphs before eq. product).  The apply follows eq.
 * product: sum_l A(s_l) W_l = sum_d H_d (sum_l f_d[l] W_l).
 *
 * Readings: ties in every argmax go to the lowest (row-major) index; the
 * next frequency k_{l+1} is the argmax of |f_l| over frequencies not yet
 * selected (f_l[k_l] = 1 by construction, so the unrestricted argmax would
 * mostly return k_l, whose residual face is zero, and end the loop early —
 * partial pivoting as in matrix ACA); when every frequency has been selected
 * the approximation interpolates all faces and the loop ends keeping all
 * terms; the first row of the ACA is the block's first row; a residual row
 * that is exactly zero is skipped for the next unused row; the ACA stops when
 * ||u_k|| ||v_k|| <= eps_aca ||S_k||_F (S_k the current approximation, norm
 * by the matrix analogue of eq. norm) or at rank min(|I|, |J|); Algorithm 1
 * also stops when a residual face is exactly zero.
 */
#define _POSIX_C_SOURCE 200809L /* clock_gettime */
#include <time.h>
#include "orc.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

const int32_t *orc_tree_perm(const orc_tree *T, int side);
const int32_t *orc_tree_blocks(const orc_tree *T);
int64_t orc_mesh_ndof(const orc_mesh *m, int basis);

/* ---- a tensor source: ENTRY(i, j, k) ----------------------------------- */
typedef struct {
    int nI, nJ, nK;
    /* BEM source */
    const orc_mesh *mesh;
    int op, ng;
    double c;
    const double *s;
    const int32_t *rows, *cols;
    /* explicit dense source t[k][i][j] */
    const double *dense;
    int64_t evals;
} src3;

static cplx src_at(src3 *S, int i, int j, int k) {
    S->evals++;
    if (S->dense) {
        const double *p = S->dense + 2 * (((int64_t)k * S->nI + i) * S->nJ + j);
        return p[0] + I * p[1];
    }
    double o[2];
    orc_entry(S->mesh, S->op, S->rows[i], S->cols[j], S->s[2 * k], S->s[2 * k + 1], S->c, S->ng,
              o);
    return o[0] + I * o[1];
}

/* ---- faces --------------------------------------------------------------- */
typedef struct {
    int rank;  /* -1: dense */
    cplx *H;   /* dense [nI][nJ] */
    cplx *U;   /* [nI][rank] */
    cplx *V;   /* [nJ][rank] */
} face;

static cplx face_at(const face *F, int nJ, int i, int j) {
    if (F->rank < 0) return F->H[(int64_t)i * nJ + j];
    cplx a = 0.0;
    for (int t = 0; t < F->rank; ++t) a += F->U[(int64_t)i * F->rank + t] * F->V[(int64_t)j * F->rank + t];
    return a;
}

static void face_free(face *F) {
    free(F->H);
    free(F->U);
    free(F->V);
    memset(F, 0, sizeof *F);
}

/* residual of the 3D approximation at frequency k: R(i,j) = ENTRY - C^(l)(i,j,k) */
typedef struct {
    src3 *S;
    const face *faces;
    const cplx *f; /* [l][nK] */
    int l, k;
} resid;

static cplx resid_at(resid *R, int i, int j) {
    cplx a = src_at(R->S, i, j, R->k);
    for (int d = 0; d < R->l; ++d) a -= R->f[(int64_t)d * R->S->nK + R->k] * face_at(&R->faces[d], R->S->nJ, i, j);
    return a;
}

/* ACA with partial pivoting on R; writes F (low rank). */
static void aca(resid *R, int nI, int nJ, double eps, int kmax, face *F) {
    cplx *U = malloc(sizeof(cplx) * (int64_t)nI * kmax);
    cplx *V = malloc(sizeof(cplx) * (int64_t)nJ * kmax);
    cplx *row = malloc(sizeof(cplx) * nJ), *col = malloc(sizeof(cplx) * nI);
    char *used = calloc(nI, 1);
    double norm2 = 0.0;
    int k = 0, istar = 0;
    while (k < kmax) {
        for (int j = 0; j < nJ; ++j) {
            cplx a = resid_at(R, istar, j);
            for (int t = 0; t < k; ++t) a -= U[(int64_t)t * nI + istar] * V[(int64_t)t * nJ + j];
            row[j] = a;
        }
        used[istar] = 1;
        int jstar = 0;
        for (int j = 1; j < nJ; ++j)
            if (cabs(row[j]) > cabs(row[jstar])) jstar = j;
        if (cabs(row[jstar]) == 0.0) {
            int nxt = -1;
            for (int i = 0; i < nI; ++i)
                if (!used[i]) {
                    nxt = i;
                    break;
                }
            if (nxt < 0) break;
            istar = nxt;
            continue;
        }
        cplx piv = row[jstar];
        for (int j = 0; j < nJ; ++j) V[(int64_t)k * nJ + j] = row[j] / piv;
        for (int i = 0; i < nI; ++i) {
            cplx a = resid_at(R, i, jstar);
            for (int t = 0; t < k; ++t) a -= U[(int64_t)t * nI + i] * V[(int64_t)t * nJ + jstar];
            col[i] = a;
            U[(int64_t)k * nI + i] = a;
        }
        /* ||S_k||^2 = ||S_{k-1}||^2 + 2 Re sum_t <u_k,u_t><v_k,v_t> + |u_k|^2 |v_k|^2 */
        double nu = 0.0, nv = 0.0;
        for (int i = 0; i < nI; ++i) nu += creal(col[i] * conj(col[i]));
        for (int j = 0; j < nJ; ++j) nv += creal(V[(int64_t)k * nJ + j] * conj(V[(int64_t)k * nJ + j]));
        double cross = 0.0;
        for (int t = 0; t < k; ++t) {
            cplx gu = 0.0, gv = 0.0;
            for (int i = 0; i < nI; ++i) gu += U[(int64_t)k * nI + i] * conj(U[(int64_t)t * nI + i]);
            for (int j = 0; j < nJ; ++j) gv += V[(int64_t)k * nJ + j] * conj(V[(int64_t)t * nJ + j]);
            cross += creal(gu * gv);
        }
        norm2 += 2.0 * cross + nu * nv;
        k++;
        if (sqrt(nu * nv) <= eps * sqrt(norm2)) break;
        int nxt = -1;
        for (int i = 0; i < nI; ++i)
            if (!used[i] && (nxt < 0 || cabs(col[i]) > cabs(col[nxt]))) nxt = i;
        if (nxt < 0) break;
        istar = nxt;
    }
    /* store as U[i][t], V[j][t] */
    F->rank = k;
    F->H = NULL;
    F->U = malloc(sizeof(cplx) * (int64_t)nI * (k ? k : 1));
    F->V = malloc(sizeof(cplx) * (int64_t)nJ * (k ? k : 1));
    for (int t = 0; t < k; ++t) {
        for (int i = 0; i < nI; ++i) F->U[(int64_t)i * k + t] = U[(int64_t)t * nI + i];
        for (int j = 0; j < nJ; ++j) F->V[(int64_t)j * k + t] = V[(int64_t)t * nJ + j];
    }
    free(U);
    free(V);
    free(row);
    free(col);
    free(used);
}

/* Algorithm 1 on source S.  near: dense faces; otherwise ACA faces at eps_aca.
 * Fills faces[0..r), f[r][nK], kpiv[r]; returns r. */
static int aca3d(src3 *S, int near, double eps, double eps_aca, int rmax, face *faces, cplx *f,
                 int32_t *kpiv) {
    const int nI = S->nI, nJ = S->nJ, nK = S->nK;
    int lmax = nK + 1;
    if (rmax > 0 && rmax < lmax) lmax = rmax;
    face *tf = calloc(lmax, sizeof(face));
    cplx *tfib = calloc((int64_t)lmax * nK, sizeof(cplx));
    int32_t *tk = calloc(lmax, sizeof(int32_t));
    cplx *dense = malloc(sizeof(cplx) * (int64_t)nI * nJ);
    cplx *gramH = calloc((int64_t)lmax * lmax, sizeof(cplx));
    cplx *gramF = calloc((int64_t)lmax * lmax, sizeof(cplx));
    double normC2 = 0.0;
    int l = 0, k = 0, r = -1;
    while (l < lmax) {
        resid R = {S, tf, tfib, l, k};
        face F = {0};
        if (near) {
            F.rank = -1;
            F.H = malloc(sizeof(cplx) * (int64_t)nI * nJ);
            for (int i = 0; i < nI; ++i)
                for (int j = 0; j < nJ; ++j) F.H[(int64_t)i * nJ + j] = resid_at(&R, i, j);
        } else {
            int kmax = nI < nJ ? nI : nJ;
            aca(&R, nI, nJ, eps_aca, kmax, &F);
        }
        /* dense rebuild for the pivot search */
        int ip = 0, jp = 0;
        double best = -1.0;
        for (int i = 0; i < nI; ++i)
            for (int j = 0; j < nJ; ++j) {
                cplx h = face_at(&F, nJ, i, j);
                dense[(int64_t)i * nJ + j] = h;
                if (cabs(h) > best) {
                    best = cabs(h);
                    ip = i;
                    jp = j;
                }
            }
        if (best == 0.0) { /* zero residual face: nothing left to add */
            face_free(&F);
            r = l;
            break;
        }
        cplx piv = dense[(int64_t)ip * nJ + jp];
        cplx *fl = tfib + (int64_t)l * nK;
        for (int kk = 0; kk < nK; ++kk) {
            cplx a = src_at(S, ip, jp, kk);
            for (int d = 0; d < l; ++d) a -= face_at(&tf[d], nJ, ip, jp) * tfib[(int64_t)d * nK + kk];
            fl[kk] = a / piv;
        }
        /* Gram entries <H_l, H_d> and <f_l, f_d> for d <= l (eq. norm) */
        for (int d = 0; d <= l; ++d) {
            cplx gh = 0.0, gf = 0.0;
            for (int i = 0; i < nI; ++i)
                for (int j = 0; j < nJ; ++j)
                    gh += dense[(int64_t)i * nJ + j] *
                          conj(d == l ? dense[(int64_t)i * nJ + j] : face_at(&tf[d], nJ, i, j));
            for (int kk = 0; kk < nK; ++kk) gf += fl[kk] * conj(tfib[(int64_t)d * nK + kk]);
            gramH[(int64_t)l * lmax + d] = gh;
            gramF[(int64_t)l * lmax + d] = gf;
        }
        double cross = 0.0;
        for (int d = 0; d < l; ++d)
            cross += creal(gramH[(int64_t)l * lmax + d] * gramF[(int64_t)l * lmax + d]);
        double hl2 = creal(gramH[(int64_t)l * lmax + l]), fl2 = creal(gramF[(int64_t)l * lmax + l]);
        normC2 += 2.0 * cross + hl2 * fl2;
        tf[l] = F;
        tk[l] = k;
        l++;
        if (sqrt(hl2 * fl2) <= eps * sqrt(normC2)) {
            r = l - 1;
            break;
        }
        /* next frequency: largest |f_l[k]| among frequencies not selected yet */
        int kn = -1;
        for (int kk = 0; kk < nK; ++kk) {
            int used = 0;
            for (int d = 0; d < l; ++d) used |= (tk[d] == kk);
            if (!used && (kn < 0 || cabs(fl[kk]) > cabs(fl[kn]))) kn = kk;
        }
        if (kn < 0) break; /* every frequency selected: the approximation is exact */
        k = kn;
    }
    if (r < 0) r = l;
    for (int d = 0; d < l; ++d) {
        if (d < r) {
            faces[d] = tf[d];
            memcpy(f + (int64_t)d * nK, tfib + (int64_t)d * nK, sizeof(cplx) * nK);
            kpiv[d] = tk[d];
        } else {
            face_free(&tf[d]);
        }
    }
    free(tf);
    free(tfib);
    free(tk);
    free(dense);
    free(gramH);
    free(gramF);
    return r;
}

/* ---- explicit-tensor entry points (used by the exactness pins) ---------- */
int orc_aca_dense(const double *a, int nI, int nJ, double eps, int kmax, double *U, double *V) {
    src3 S = {0};
    S.nI = nI;
    S.nJ = nJ;
    S.nK = 1;
    S.dense = a;
    resid R = {&S, NULL, NULL, 0, 0};
    face F;
    aca(&R, nI, nJ, eps, kmax, &F);
    for (int i = 0; i < nI; ++i)
        for (int t = 0; t < F.rank; ++t) {
            U[2 * ((int64_t)i * kmax + t)] = creal(F.U[(int64_t)i * F.rank + t]);
            U[2 * ((int64_t)i * kmax + t) + 1] = cimag(F.U[(int64_t)i * F.rank + t]);
        }
    for (int j = 0; j < nJ; ++j)
        for (int t = 0; t < F.rank; ++t) {
            V[2 * ((int64_t)j * kmax + t)] = creal(F.V[(int64_t)j * F.rank + t]);
            V[2 * ((int64_t)j * kmax + t) + 1] = cimag(F.V[(int64_t)j * F.rank + t]);
        }
    int r = F.rank;
    face_free(&F);
    return r;
}

static int aca3d_explicit(const double *t, int nI, int nJ, int nK, int near, double eps,
                          double eps_aca, int rmax, int32_t *kpiv, double *H, double *f,
                          int32_t *face_rank) {
    src3 S = {0};
    S.nI = nI;
    S.nJ = nJ;
    S.nK = nK;
    S.dense = t;
    face *faces = calloc(nK + 1, sizeof(face));
    cplx *fib = calloc((int64_t)(nK + 1) * nK, sizeof(cplx));
    int32_t *kp = calloc(nK + 1, sizeof(int32_t));
    int r = aca3d(&S, near, eps, eps_aca, 0, faces, fib, kp);
    int nout = r < rmax ? r : rmax;
    for (int d = 0; d < nout; ++d) {
        kpiv[d] = kp[d];
        if (face_rank) face_rank[d] = faces[d].rank;
        for (int i = 0; i < nI; ++i)
            for (int j = 0; j < nJ; ++j) {
                cplx h = face_at(&faces[d], nJ, i, j);
                int64_t o = ((int64_t)d * nI + i) * nJ + j;
                H[2 * o] = creal(h);
                H[2 * o + 1] = cimag(h);
            }
        for (int kk = 0; kk < nK; ++kk) {
            f[2 * ((int64_t)d * nK + kk)] = creal(fib[(int64_t)d * nK + kk]);
            f[2 * ((int64_t)d * nK + kk) + 1] = cimag(fib[(int64_t)d * nK + kk]);
        }
    }
    for (int d = 0; d < r; ++d) face_free(&faces[d]);
    free(faces);
    free(fib);
    free(kp);
    return r;
}

int orc_aca3d_dense(const double *t, int nI, int nJ, int nK, double eps, int rmax, int32_t *kpiv,
                    double *H, double *f) {
    return aca3d_explicit(t, nI, nJ, nK, 1, eps, 0.0, rmax, kpiv, H, f, NULL);
}

int orc_aca3d_dense_acaface(const double *t, int nI, int nJ, int nK, double eps, double eps_aca,
                            int rmax, int32_t *kpiv, double *H, double *f, int32_t *face_rank) {
    return aca3d_explicit(t, nI, nJ, nK, 0, eps, eps_aca, rmax, kpiv, H, f, face_rank);
}

/* ---- compressed BEM operator tensor ------------------------------------- */
typedef struct {
    int32_t i0, i1, j0, j1, far, r;
    face *faces;
    cplx *f; /* [r][nf] */
    int64_t evals;
    double secs; /* wall time of this block's compression (instrumentation only) */
} blockc;

struct orc_tensor {
    int64_t nrows, ncols;
    int nf;
    int64_t nb;
    blockc *b;
    int32_t *perm_r, *perm_c, *inv_r, *inv_c;
};

/* wall-clock seconds (timing of the blocks only; no part of the method) */
static double orc_wtime(void) {
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

orc_tensor *orc_compress(const orc_mesh *m, int op, double c, int ng, const double *s, int nf,
                         const orc_tree *t, double eps, double eps_aca, int nthreads,
                         int block_stride, const uint8_t *block_mask) {
    orc_tensor *x = calloc(1, sizeof *x);
    x->nrows = orc_mesh_ndof(m, ORC_P0);
    x->ncols = orc_mesh_ndof(m, op == ORC_DLP ? ORC_P1 : ORC_P0);
    x->nf = nf;
    x->nb = orc_tree_nblocks(t);
    x->b = calloc(x->nb, sizeof(blockc));
    x->perm_r = malloc(sizeof(int32_t) * x->nrows);
    x->perm_c = malloc(sizeof(int32_t) * x->ncols);
    memcpy(x->perm_r, orc_tree_perm(t, 0), sizeof(int32_t) * x->nrows);
    memcpy(x->perm_c, orc_tree_perm(t, 1), sizeof(int32_t) * x->ncols);
    x->inv_r = malloc(sizeof(int32_t) * x->nrows);
    x->inv_c = malloc(sizeof(int32_t) * x->ncols);
    for (int64_t k = 0; k < x->nrows; ++k) x->inv_r[x->perm_r[k]] = (int32_t)k;
    for (int64_t k = 0; k < x->ncols; ++k) x->inv_c[x->perm_c[k]] = (int32_t)k;
    const int32_t *bl = orc_tree_blocks(t);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t b = 0; b < x->nb; ++b) {
        blockc *B = &x->b[b];
        B->i0 = bl[5 * b];
        B->i1 = bl[5 * b + 1];
        B->j0 = bl[5 * b + 2];
        B->j1 = bl[5 * b + 3];
        B->far = bl[5 * b + 4];
        if ((block_stride > 1 && b % block_stride != 0) || (block_mask && !block_mask[b])) {
            B->r = 0;
            continue;
        }
        const double t_start = orc_wtime();
        src3 S = {0};
        S.nI = B->i1 - B->i0;
        S.nJ = B->j1 - B->j0;
        S.nK = nf;
        S.mesh = m;
        S.op = op;
        S.ng = ng;
        S.c = c;
        S.s = s;
        S.rows = x->perm_r + B->i0;
        S.cols = x->perm_c + B->j0;
        face *faces = calloc(nf + 1, sizeof(face));
        cplx *fib = calloc((int64_t)(nf + 1) * nf, sizeof(cplx));
        int32_t *kp = calloc(nf + 1, sizeof(int32_t));
        B->r = aca3d(&S, !B->far, eps, eps_aca, 0, faces, fib, kp);
        B->faces = faces;
        B->f = fib;
        B->evals = S.evals;
        B->secs = orc_wtime() - t_start;
        free(kp);
    }
    return x;
}

void orc_tensor_free(orc_tensor *x) {
    if (!x) return;
    for (int64_t b = 0; b < x->nb; ++b) {
        for (int d = 0; d < x->b[b].r; ++d) face_free(&x->b[b].faces[d]);
        free(x->b[b].faces);
        free(x->b[b].f);
    }
    free(x->b);
    free(x->perm_r);
    free(x->perm_c);
    free(x->inv_r);
    free(x->inv_c);
    free(x);
}

void orc_tensor_stats(const orc_tensor *x, double *st) {
    double nfar = 0, sumr = 0, maxr = 0, stored = 0, evals = 0, sumk = 0, secs = 0;
    for (int64_t b = 0; b < x->nb; ++b) {
        const blockc *B = &x->b[b];
        int nI = B->i1 - B->i0, nJ = B->j1 - B->j0;
        nfar += B->far;
        sumr += B->r;
        if (B->r > maxr) maxr = B->r;
        evals += (double)B->evals;
        secs += B->secs;
        for (int d = 0; d < B->r; ++d) {
            stored += x->nf;
            if (B->faces[d].rank < 0)
                stored += (double)nI * nJ;
            else {
                stored += (double)B->faces[d].rank * (nI + nJ);
                sumk += B->faces[d].rank;
            }
        }
    }
    st[0] = (double)x->nb;
    st[1] = nfar;
    st[2] = sumr;
    st[3] = maxr;
    st[4] = stored;
    st[5] = (double)x->nrows * (double)x->ncols * x->nf;
    st[6] = evals;
    st[7] = sumk;
    st[8] = secs;
}

void orc_tensor_block_ranks(const orc_tensor *x, int32_t *r, int32_t *kface) {
    for (int64_t b = 0; b < x->nb; ++b) {
        r[b] = x->b[b].r;
        int s = 0;
        for (int d = 0; d < x->b[b].r; ++d) s += x->b[b].faces[d].rank > 0 ? x->b[b].faces[d].rank : 0;
        if (kface) kface[b] = s;
    }
}

void orc_tensor_entry(const orc_tensor *x, int64_t row, int64_t col, int f, double *out) {
    int32_t pi = x->inv_r[row], pj = x->inv_c[col];
    cplx a = 0.0;
    for (int64_t b = 0; b < x->nb; ++b) {
        const blockc *B = &x->b[b];
        if (pi < B->i0 || pi >= B->i1 || pj < B->j0 || pj >= B->j1) continue;
        int nJ = B->j1 - B->j0;
        for (int d = 0; d < B->r; ++d)
            a += face_at(&B->faces[d], nJ, pi - B->i0, pj - B->j0) * B->f[(int64_t)d * x->nf + f];
        break;
    }
    out[0] = creal(a);
    out[1] = cimag(a);
}

void orc_tensor_apply(const orc_tensor *x, const double *W, int nrhs, double *y) {
    const int nf = x->nf;
    cplx *yy = calloc((size_t)x->nrows * nrhs, sizeof(cplx));
    for (int64_t b = 0; b < x->nb; ++b) {
        const blockc *B = &x->b[b];
        int nI = B->i1 - B->i0, nJ = B->j1 - B->j0;
        cplx *z = malloc(sizeof(cplx) * (int64_t)nJ * nrhs);
        for (int d = 0; d < B->r; ++d) {
            /* inner sum of eq. product: z = sum_l f_d[l] W_l restricted to J */
            for (int j = 0; j < nJ; ++j)
                for (int q = 0; q < nrhs; ++q) {
                    cplx a = 0.0;
                    int64_t col = x->perm_c[B->j0 + j];
                    for (int l = 0; l < nf; ++l) {
                        const double *w = W + 2 * (((int64_t)l * x->ncols + col) * nrhs + q);
                        a += B->f[(int64_t)d * nf + l] * (w[0] + I * w[1]);
                    }
                    z[(int64_t)j * nrhs + q] = a;
                }
            /* outer product: y_I += H_d z */
            for (int i = 0; i < nI; ++i) {
                int64_t row = x->perm_r[B->i0 + i];
                for (int j = 0; j < nJ; ++j) {
                    cplx h = face_at(&B->faces[d], nJ, i, j);
                    for (int q = 0; q < nrhs; ++q) yy[row * nrhs + q] += h * z[(int64_t)j * nrhs + q];
                }
            }
        }
        free(z);
    }
    for (int64_t k = 0; k < x->nrows * nrhs; ++k) {
        y[2 * k] = creal(yy[k]);
        y[2 * k + 1] = cimag(yy[k]);
    }
    free(yy);
}

void orc_dense_apply_rows(const orc_mesh *m, int op, double c, int ng, const double *s, int nf,
                          const int32_t *rows, int64_t nr, const double *W, int nrhs, double *y,
                          int nthreads) {
    int64_t ncols = orc_mesh_ndof(m, op == ORC_DLP ? ORC_P1 : ORC_P0);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t r = 0; r < nr; ++r) {
        cplx *acc = calloc(nrhs, sizeof(cplx));
        for (int l = 0; l < nf; ++l)
            for (int64_t j = 0; j < ncols; ++j) {
                double a[2];
                orc_entry(m, op, rows[r], j, s[2 * l], s[2 * l + 1], c, ng, a);
                cplx av = a[0] + I * a[1];
                for (int q = 0; q < nrhs; ++q) {
                    const double *w = W + 2 * (((int64_t)l * ncols + j) * nrhs + q);
                    acc[q] += av * (w[0] + I * w[1]);
                }
            }
        for (int q = 0; q < nrhs; ++q) {
            y[2 * (r * nrhs + q)] = creal(acc[q]);
            y[2 * (r * nrhs + q) + 1] = cimag(acc[q]);
        }
        free(acc);
    }
}
