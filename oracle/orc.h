/*
 * Oracle for the time-domain BEM tensor path of
 *   M. Schanz, V. Lakshmi Keshava, H. De Gersem,
 *   "Comparison of H-matrix- and FMM-based 3D-ACA for a time-domain boundary
 *    element method" (arXiv 2505.00715).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, FP64 CPU restatement of
 * the method, written to check the CUDA library against.  It shares no code,
 * header, table or constant generator with the library under
 * paper_2505_00715_gb300/, and nothing in that library may include, link or
 * call it.  Only tests, the smoke check and the bench's CPU-baseline leg use it.
 *
 * Conventions (all FP64):
 *   - complex numbers cross this interface as interleaved (re, im) doubles;
 *   - triangles are vertex-index triples, counter-clockwise seen from outside,
 *     so (v1-v0)x(v2-v0) points out of the domain (Sec. 2, outward normal n);
 *   - operators: ORC_SLP = single layer V, Galerkin P0 test x P0 trial;
 *                ORC_DLP = double layer K, Galerkin P0 test x P1 trial;
 *                ORC_ADLP = adjoint double layer K', Galerkin P0 test x P0
 *                trial (the conormal derivative at x of the single layer)
 *     (Sec. 2 eqs. slp/dlp/adlp, Sec. 3 spaces X_D = P1, X_N = P0);
 *   - Laplace-domain kernel exp(-s r / c) / (4 pi r) (fundamental solution of
 *     Sec. 2 transformed to the Laplace domain, Sec. 3 "Temporal
 *     discretisation").
 *
 * Functions with no independent pin are marked "parity unpinned" where they
 * are declared.  Every other function is checked by tests/test_oracle_*.py
 * against closed forms, library routines, brute force or invariants.
 */
#ifndef ORC_H
#define ORC_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_SLP = 0, ORC_DLP = 1, ORC_ADLP = 2 };
enum { ORC_P0 = 0, ORC_P1 = 1 };

typedef struct orc_mesh orc_mesh;

/* Mesh with per-triangle area and unit normal and the vertex -> triangle
 * incidence used for P1 supports.  Returns NULL on a degenerate triangle or
 * an out-of-range index. */
orc_mesh *orc_mesh_new(const double *verts, int64_t nv, const int32_t *tris, int64_t nt);
void orc_mesh_free(orc_mesh *m);
int64_t orc_mesh_ndof(const orc_mesh *m, int basis);

/* ---- quadrature (Sec. 3 "Spatial discretisation", last paragraph) ---- */
/* 7-point degree-5 triangle rule: barycentric points and weights summing to 1. */
void orc_rule7(double *bary /*[7][3]*/, double *w /*[7]*/);
/* n-point Gauss-Legendre rule on [0,1] (Newton iteration on P_n). */
int orc_gauss01(int n, double *x, double *w);

/* Pair integral over test triangle ti and trial triangle tj at frequency s:
 *   SLP: out[0]      = int_ti int_tj  exp(-s r/c)/(4 pi r)
 *   DLP: out[m], m<3 = int_ti int_tj  phi_m(y) d/dn_y [exp(-s r/c)/(4 pi r)]
 *        where phi_m is the P1 hat of tj's m-th vertex restricted to tj;
 *   ADLP: out[0]     = int_ti int_tj  d/dn_x [exp(-s r/c)/(4 pi r)]
 *        (n_x the normal of ti).
 * Touching pairs (identical / common edge / common vertex) use the
 * regularising coordinate transforms of Sauter and Schwab with an ng-point
 * Gauss-Legendre rule in every transformed variable; other pairs the 7x7 rule.
 * SLP pairs are integrated in the order (lower index, higher index), so the
 * single-layer matrix is symmetric exactly.
 * Returns the pair class: 0 regular, 1 vertex, 2 edge, 3 identical. */
int orc_pair(const orc_mesh *m, int op, int64_t ti, int64_t tj, double s_re, double s_im,
             double c, int ng, double *out_re_im /*[2*3]*/);
/* Forced-regular variant (7x7 rule even for touching pairs), used by tests. */
void orc_pair_regular(const orc_mesh *m, int op, int64_t ti, int64_t tj, double s_re,
                      double s_im, double c, double *out_re_im);

/* Matrix entry A[row, col](s) of the Galerkin operator (sum over the trial
 * support for P1 columns). */
void orc_entry(const orc_mesh *m, int op, int64_t row, int64_t col, double s_re, double s_im,
               double c, int ng, double *out_re_im /*[2]*/);
/* Batch: out[f][r][c] (complex, interleaved) for rows x cols x freqs. */
void orc_entries(const orc_mesh *m, int op, const int32_t *rows, int64_t nr,
                 const int32_t *cols, int64_t nc, const double *s /*[2*nf]*/, int64_t nf,
                 double c, int ng, double *out);

/* Magnitude sums out[f][r][c] (real): the quadrature of orc_entries with
 * every term replaced by a bound of its modulus, |exp(-s r/c)|/(4 pi r) for
 * the single layer and |exp(-s r/c)(1 + s r/c)|/(4 pi r^2) for the double
 * layer and its adjoint (|(x - y).n| <= |x - y|; a flat panel with itself
 * contributes 0, as to the entry).  A floating-point evaluation of an entry
 * can only be accurate relative to this sum: rounding in each term is
 * relative to its bound, and the terms may cancel.  For the single layer at
 * real s every term is positive and the sum equals |entry|. */
void orc_entries_mag(const orc_mesh *m, int op, const int32_t *rows, int64_t nr,
                     const int32_t *cols, int64_t nc, const double *s /*[2*nf]*/, int64_t nf,
                     double c, int ng, double *out);

/* ---- frequency sets (App. A; BDF2 CQ) ---- */
/* BDF2 convolution quadrature: s_k = delta(lambda e^{2 pi i k/N})/dt,
 * delta(z) = (1-z) + (1-z)^2/2, k = 0..N-1.  lambda <= 0 picks
 * (1e-8)^(1/(2N)). */
int orc_freqs_bdf2(int N, double dt, double lambda, double *s /*[2N]*/);
/* Complete elliptic integral of the first kind, parameter m = k^2 (AGM). */
double orc_ellipk(double m);
/* Jacobi sn, cn, dn of real argument u, parameter m (descending Landen/AGM). */
void orc_ellipj(double u, double m, double *sn, double *cn, double *dn);
/* Jacobi sn, cn, dn of complex argument (addition formulas with the
 * complementary parameter), interleaved outputs. */
void orc_ellipj_complex(double u, double v, double m, double *sn, double *cn, double *dn);
/* gCQ contour points and weights (App. A): rk = 0 implicit Euler, 1 Radau IIA
 * (2 stages), for nsteps steps in [dt_min, dt_max].  The circle passes through
 * 0 and 2 rho / dt_min with rho = rho_in if rho_in > 0 (rho_in = 1: App. A as
 * printed), else rho = orc_gcq_radius(rk, nsteps), which encloses every
 * resolvent pole 1/(dt lambda_i(A)) and keeps max |R(dt_min s)|^nsteps <= 1e4
 * along the circle (rho = 1 for implicit Euler).  s, w: [2*NQ];
 * the weights are those of the positively oriented Cauchy integral.  info
 * (nullable) [5]: q, k, K(k^2), K'(k^2), rho.  Returns 0, or 1 if q had to be
 * lifted off the q = 1 degeneracy. */
double orc_gcq_radius(int rk, int nsteps);
int orc_freqs_gcq(double dt_min, double dt_max, int rk, int nsteps, double rho_in, int NQ, double *s,
                  double *w, double *info);

/* ---- cluster tree and block cluster tree (Sec. 4, eq. admissible) ---- */
typedef struct orc_tree orc_tree;
/* rows: test basis (P0); cols: trial basis (P0 or P1). */
orc_tree *orc_tree_build(const orc_mesh *m, int row_basis, int col_basis, int leaf, double eta);
void orc_tree_free(orc_tree *t);
int64_t orc_tree_nblocks(const orc_tree *t);
/* perm_rows[k] = DOF at permuted position k; blocks[b] = {i0,i1,j0,j1,far}
 * (half-open ranges in permuted numbering), in depth-first order. */
void orc_tree_export(const orc_tree *t, int32_t *perm_rows, int32_t *perm_cols, int32_t *blocks);
/* cluster count and per-cluster data {begin,end,son0,son1} + bbox[6] (rows). */
int64_t orc_tree_nclusters(const orc_tree *t, int side);
void orc_tree_clusters(const orc_tree *t, int side, int32_t *nodes /*[n][4]*/, double *bbox /*[n][6]*/);

/* ---- ACA and 3D-ACA (Sec. 4, eq. norm, Algorithm 1) ---- */
/* Matrix ACA with partial pivoting on an explicit dense complex matrix
 * a[nI][nJ]; outputs U[nI][kmax], V[nJ][kmax] (a ~ U V^T), returns rank. */
int orc_aca_dense(const double *a, int nI, int nJ, double eps, int kmax, double *U, double *V);
/* 3D-ACA on an explicit dense complex tensor t[nK][nI][nJ] with dense faces
 * (the near-field form of Algorithm 1).  Outputs up to rmax terms: kpiv[r],
 * H[r][nI][nJ], f[r][nK].  Returns r. */
int orc_aca3d_dense(const double *t, int nI, int nJ, int nK, double eps, int rmax, int32_t *kpiv,
                    double *H, double *f);
/* 3D-ACA on an explicit dense tensor where every face is itself compressed
 * by matrix ACA to eps_aca (the far-field form).  Same outputs (faces are
 * returned rebuilt densely). */
int orc_aca3d_dense_acaface(const double *t, int nI, int nJ, int nK, double eps, double eps_aca,
                            int rmax, int32_t *kpiv, double *H, double *f, int32_t *face_rank);

/* Compressed operator tensor of a BEM operator over a frequency list.
 * block_stride > 1 compresses only every block_stride-th block, and a
 * non-NULL block_mask [nblocks] only the blocks with a non-zero mask byte
 * (bounded samples for timing; the others are left empty). */
typedef struct orc_tensor orc_tensor;
orc_tensor *orc_compress(const orc_mesh *m, int op, double c, int ng, const double *s, int nf,
                         const orc_tree *t, double eps, double eps_aca, int nthreads,
                         int block_stride, const uint8_t *block_mask);
void orc_tensor_free(orc_tensor *x);
/* stats[9]: nblocks, nfar, sum ranks, max rank, stored complex entries,
 * dense complex entries (nrows*ncols*nf), entries evaluated, sum face ranks,
 * summed wall-clock seconds of the blocks' compressions (timing only) */
void orc_tensor_stats(const orc_tensor *x, double *stats);
/* per block: rank r_b and for far blocks the sum of face ranks. */
void orc_tensor_block_ranks(const orc_tensor *x, int32_t *r, int32_t *kface);
/* Rebuilt entry of block-compressed tensor at (row, col, freq) (original
 * numbering; conjugate frequencies are not mirrored here). */
void orc_tensor_entry(const orc_tensor *x, int64_t row, int64_t col, int f, double *out);
/* y[nrows][nrhs] = sum_f A(s_f) W_f, W: [nf][ncols][nrhs] complex (eq. product). */
void orc_tensor_apply(const orc_tensor *x, const double *W, int nrhs, double *y);
/* Dense FP64 apply restricted to the listed rows: y[nr][nrhs] =
 * sum_f sum_j A(s_f)[row, j] W_f[j]. */
void orc_dense_apply_rows(const orc_mesh *m, int op, double c, int ng, const double *s, int nf,
                          const int32_t *rows, int64_t nr, const double *W, int nrhs, double *y,
                          int nthreads);

/* ---- rank-predictor MLP (6 -> 64 -> 64 -> 16, GELU) ---- */
/* params layout: W1[64][6] b1[64] W2[64][64] b2[64] W3[16][64] b3[16]. */
int orc_mlp_nparams(void);
/* logits[n][16]; returns nothing. */
void orc_mlp_forward(const double *params, const double *x, int64_t n, double *logits);
/* mean softmax cross-entropy over n samples; grad (nullable) has the params layout. */
double orc_mlp_loss_grad(const double *params, const double *x, const int32_t *label, int64_t n,
                         double *grad);
/* One Adam step (beta1, beta2, eps, lr) with step counter t (1-based). */
void orc_adam_step(double *params, const double *grad, double *m, double *v, int64_t np,
                   double lr, double beta1, double beta2, double eps, int t);

#ifdef __cplusplus
}
#endif
#endif
