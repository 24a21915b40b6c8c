/*
 * tdbem — GB300 (sm_103a) library for the Laplace-domain operator tensor of a
 * time-domain Galerkin boundary element method, compressed by 3D-ACA over the
 * convolution-quadrature frequencies, and its multi-frequency apply.
 *
 * Method: M. Schanz, V. Lakshmi Keshava, H. De Gersem, "Comparison of
 * H-matrix- and FMM-based 3D-ACA for a time-domain boundary element method",
 * arXiv 2505.00715.  Section numbers below refer to that paper.
 *
 * Conventions for every call
 *   - Return value: TDBEM_OK (0) or a negative TDBEM_ERR_* code; the message
 *     of the last failure of a context is returned by tdbem_last_error().
 *     No call aborts, traps or exits the process.
 *   - Host arrays passed in are copied before the call returns; the caller
 *     keeps ownership.  Handles are owned by the library and released by the
 *     matching *_destroy call (NULL is accepted and ignored).
 *   - "device" pointers are CUDA global-memory addresses on the context's
 *     device, owned by the caller; work on them is ordered on the context's
 *     stream and is asynchronous unless the call says otherwise.  Calls that
 *     return host data (tdbem_freqs_get, tdbem_tree_export,
 *     tdbem_tensor_stats) synchronise the stream.
 *   - Complex arrays are interleaved (re, im): complex64 = 2 x float,
 *     complex128 = 2 x double.
 *   - Triangles are vertex-index triples ordered counter-clockwise seen from
 *     outside, so (v1 - v0) x (v2 - v0) is the outward normal n of Sec. 2.
 *   - Indices are 0-based; DOF numbering is the caller's (P0: triangle index,
 *     P1: vertex index); the cluster-tree permutation stays internal.
 */
#ifndef TDBEM_H
#define TDBEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define TDBEM_OK 0
#define TDBEM_ERR_ARG (-1)            /* bad argument, degenerate mesh, NaN, ... */
#define TDBEM_ERR_OOM (-2)            /* device or host allocation failed */
#define TDBEM_ERR_CUDA (-3)           /* a CUDA runtime call failed */
#define TDBEM_ERR_NOT_CONVERGED (-4)  /* ACA / 3D-ACA rank cap hit, GMRES above tol */
#define TDBEM_ERR_CAPACITY (-5)       /* a device pool overflowed (retried internally) */

/* ---- enumerations ------------------------------------------------------- */
enum { TDBEM_SLP = 0, TDBEM_DLP = 1, TDBEM_ADLP = 2 }; /* single layer V, double layer K, adjoint K' (Sec. 2) */
enum { TDBEM_P0 = 0, TDBEM_P1 = 1 };          /* piecewise constant / linear (Sec. 3) */
enum { TDBEM_FP64 = 0, TDBEM_MIXED = 1 };     /* precision forms, see tdbem_op */
enum { TDBEM_EULER = 0, TDBEM_RADAU2 = 1 };   /* Runge-Kutta method of the gCQ (App. A) */

typedef struct tdbem_ctx *tdbem_ctx_t;
typedef struct tdbem_mesh *tdbem_mesh_t;
typedef struct tdbem_freqs *tdbem_freqs_t;
typedef struct tdbem_tree *tdbem_tree_t;
typedef struct tdbem_tensor *tdbem_tensor_t;
typedef struct tdbem_model *tdbem_model_t;

/* Operator and discretisation (Sec. 2 eqs. slp/dlp/adlp, Sec. 3):
 *   op = TDBEM_SLP: A[i,j](s) = int_{tau_i} int_{tau_j} exp(-s r/c)/(4 pi r),
 *        test P0 x trial P0 (Galerkin single layer);
 *   op = TDBEM_DLP: A[i,v](s) = int_{tau_i} int_Gamma phi_v(y) d/dn_y
 *        [exp(-s r/c)/(4 pi r)], test P0 x trial P1 (Galerkin double layer);
 *   op = TDBEM_ADLP: A[i,j](s) = int_{tau_i} d/dn_x int_{tau_j}
 *        exp(-s r/c)/(4 pi r), test P0 x trial P0 (Galerkin adjoint double
 *        layer K', the conormal derivative at x of the single layer; its
 *        column tree is built on P0 like the single layer's).
 * Regular pairs use the 7-point degree-5 triangle rule in x and y (49
 * points); pairs of triangles that share a vertex, an edge or coincide use
 * the Sauter-Schwab regularising transforms with an ng-point Gauss-Legendre
 * rule in every transformed variable (Sec. 3, Erichsen-Sauter formulas).
 *   prec = TDBEM_FP64: every step in FP64 (entries complex128);
 *   prec = TDBEM_MIXED: regular entries and ACA cross updates in FP32,
 *        touching pairs and the 3D-ACA stopping norms in FP64, complex64
 *        storage. */
typedef struct {
    int32_t op;
    int32_t prec;
    double c;   /* wave speed (> 0) */
    int32_t ng; /* Gauss points per transformed variable, 1..16 (default 5) */
    int32_t reserved;
} tdbem_op;

/* 3D-ACA parameters (Sec. 4, Algorithm 1). */
typedef struct {
    double eps;      /* tolerance of Algorithm 1 on each block (e.g. 1e-4) */
    double eps_aca;  /* tolerance of the ACA of every far-field face (e.g. 1e-6) */
    int32_t max_face_rank; /* cap of the face ACA rank, 1..64 (<= 0: 64) */
    int32_t flags;         /* bit 0: launch the phases without graph capture; bit 1: no dense
                              working faces (low-rank corrections and Grams for every far block);
                              bit 2: compress on the tree's partition as it is (by default far
                              blocks with more than twice the mean far entries per persistent
                              CTA are compressed as the blocks of their clusters' sons) */
    tdbem_model_t model;   /* nullable: rank predictor (see the rank-predictor section) */
} tdbem_aca_cfg;

typedef struct {
    int64_t nblocks, nnear, nfar;
    int64_t sum_rank, max_rank;     /* terms r_b of Algorithm 1 per block */
    int64_t sum_face_rank;          /* ACA ranks of the far faces, summed */
    int64_t stored_complex;         /* complex numbers stored (faces + fibres) */
    int64_t dense_complex;          /* rows * cols * unique frequencies */
    int64_t entries_regular;        /* regular entries evaluated */
    int64_t entries_tube;           /* fibre (all-frequency) entries evaluated */
    int64_t pairs_singular;         /* touching pairs integrated (per frequency) */
    double ms_plan, ms_singular, ms_near, ms_far, ms_total;
    int64_t pool_growths;           /* face pool grown during compression: far blocks redone
                                       (or all phases rerun after a near-field overflow) */
    int64_t launches;               /* kernel launches of the compression */
    int64_t aca_tests;              /* synchronised stopping tests of the far faces' ACA on the
                                       factor-norm path (faces above 1600 entries); the rank
                                       predictor batches the tests of the steps below its
                                       predicted rank into one */
    int64_t pool_first;             /* complex values of the first face-pool allocation: from the
                                       predicted face ranks with a rank predictor, else from a
                                       size-based bound (at most the device's free memory) */
} tdbem_stats;

/* ---- context -------------------------------------------------------------- */
/* Bind device `device` and stream `cuda_stream` (a cudaStream_t, NULL = the
 * legacy default stream). */
int tdbem_ctx_create(int device, void *cuda_stream, tdbem_ctx_t *out);
int tdbem_ctx_destroy(tdbem_ctx_t ctx);
const char *tdbem_last_error(tdbem_ctx_t ctx);
/* Block until all work of the context's stream has finished; TDBEM_ERR_CUDA
 * if a tensor-core wait of an earlier asynchronous call gave up. */
int tdbem_ctx_sync(tdbem_ctx_t ctx);
/* Poll limit of every wait of the tensor-core kernels (tdbem_zgemm and the
 * mixed-form weighted apply) on their MMA completion barrier; 0 restores the
 * default (2^24 polls of a blocking try-wait, far above any MMA group's
 * latency); a smaller limit counts non-blocking tests of the barrier.  A wait that
 * reaches the limit gives up: the kernel records the failure, waits (with
 * the default limit) for the MMAs it has issued, frees its tensor memory and
 * returns; the call's result is then invalid and tdbem_ctx_sync (or
 * tdbem_zgemm itself) returns TDBEM_ERR_CUDA.  The context stays usable.
 * A small limit exists to exercise that path.  TDBEM_ERR_ARG if polls < 0
 * or polls >= 2^31. */
int tdbem_ctx_set_wait_limit(tdbem_ctx_t ctx, int64_t polls);
/* Size in bytes of the buffer in which tdbem_compress forms and compresses
 * the near-field tensor, batch by batch of near blocks (default 16 GiB; a
 * block larger than the buffer forms a batch of its own).  TDBEM_ERR_ARG if
 * bytes <= 0. */
int tdbem_ctx_set_near_batch(tdbem_ctx_t ctx, int64_t bytes);
/* Scale (> 0, default 1) of the far-field part of the first face-pool size
 * of tdbem_compress (estimated from the far blocks' sizes or the predicted
 * ranks).  A pool that fills up grows, keeping its contents, and the far
 * blocks it stopped are redone (tdbem_stats.pool_growths counts this).
 * TDBEM_ERR_ARG if scale <= 0. */
int tdbem_ctx_set_pool_scale(tdbem_ctx_t ctx, double scale);

/* ---- mesh (Sec. 3 eq. geomapprox, spaces X_D = P1, X_N = P0) -------------- */
/* verts: host [nv][3] FP64; tris: host [nt][3] int32.  Builds the element
 * tables (quadrature points, weights, normals, FP32 and FP64) in device
 * memory.  ERR_ARG on an out-of-range index, a degenerate triangle or a
 * non-finite coordinate. */
int tdbem_mesh_create(tdbem_ctx_t ctx, const double *verts, int64_t nv, const int32_t *tris,
                      int64_t nt, tdbem_mesh_t *out);
int tdbem_mesh_destroy(tdbem_mesh_t mesh);
int64_t tdbem_mesh_ndof(tdbem_mesh_t mesh, int32_t basis);

/* ---- frequency sets --------------------------------------------------------- */
/* BDF2 convolution quadrature: s_k = delta(lambda e^{2 pi i k/N})/dt,
 * delta(z) = (1-z) + (1-z)^2/2, k = 0..N-1; lambda <= 0 selects
 * (1e-8)^(1/(2N)).  Computed in FP64 on the device. */
int tdbem_freqs_cq_bdf2(tdbem_ctx_t ctx, int32_t N, double dt, double lambda, tdbem_freqs_t *out);
/* gCQ contour of App. A: s_l = gamma(sigma_l), weights w_l (positively
 * oriented Cauchy quadrature), l = 1..NQ, for the N time steps dts (host
 * FP64 [N], every step > 0) and the RK method rk.  The contour depends on
 * the steps through dt_min = min(dts) and dt_max = max(dts) (App. A); the
 * steps are kept with the set (tdbem_freqs_steps).  Computed in FP64 on the
 * device (Jacobi elliptic functions by the AGM).  q = 1 is lifted to 1.01
 * (App. A, last paragraph).  The contour is the circle through 0 and
 * 2 rho / dt_min:
 *   rho > 0: that factor; rho = 1 is App. A as printed;
 *   rho <= 0: the radius the gCQ marching needs (tdbem_march_*): 1 for
 *     EULER; for RADAU2 the smallest rho >= sqrt(6) (every resolvent pole
 *     1/(dt lambda_i(A)) inside) in steps of 5 % with max |R(dt_min s)|^N
 *     <= 1e4 along the circle, R the stability function, so that the
 *     Runge-Kutta stages of the N steps (eq. gCQ_xn) stay bounded on it.
 * ERR_ARG for a non-finite rho. */
int tdbem_freqs_gcq(tdbem_ctx_t ctx, const double *dts, int32_t N, int32_t rk, int32_t NQ, double rho,
                    tdbem_freqs_t *out);
/* The time steps of a gCQ set (host [N], nullable) and their count *N
 * (nullable); a BDF2 set returns N = 0. */
int tdbem_freqs_steps(tdbem_freqs_t f, double *dts, int32_t *N);
/* Copies the NQ points (and weights, nullable; BDF2 sets have none and
 * return zeros) to host arrays [2*NQ]; *NQ and *Nu (number of frequencies up
 * to conjugation, App. A last paragraph) are returned when non-NULL.
 * unique (nullable, host int32 [NQ]) receives for each point the index of its
 * representative among the Nu unique points and the sign +1 (same) or -1
 * (conjugate) as  rep + 1 (same) or -(rep + 1) (conjugate). */
int tdbem_freqs_get(tdbem_freqs_t f, double *s, double *w, int32_t *NQ, int32_t *Nu,
                    int32_t *unique);
/* A frequency set of explicit points s (host [2 * NQ], every Re s > 0) and
 * optional weights w (host [2 * NQ], nullable: zeros).  Points whose
 * conjugate is also in the set are paired (the tensor is built over one of
 * each pair).  For the step operators of the gCQ marching. */
int tdbem_freqs_points(tdbem_ctx_t ctx, const double *s, const double *w, int32_t NQ, tdbem_freqs_t *out);
int tdbem_freqs_destroy(tdbem_freqs_t f);

/* ---- cluster tree and block cluster tree (Sec. 4, eq. admissible) ---------- */
/* PCA bisection of the DOF points (P0 centroids, P1 vertices) until a
 * cluster has at most `leaf` DOFs; blocks are far field when
 * min(diam) <= eta dist with dist > 0 (boxes of the DOF supports), near
 * field when either cluster is a leaf, else split into the four son pairs.
 * Built on the host in IEEE FP64 with a fixed operation order, so it is
 * reproducible bit for bit. */
int tdbem_tree_build(tdbem_mesh_t mesh, int32_t row_basis, int32_t col_basis, int32_t leaf,
                     double eta, tdbem_tree_t *out);
/* perm_rows/perm_cols (nullable, host int32 [ndof]): DOF at permuted
 * position k.  *nblocks (nullable) receives the block count; blocks
 * (nullable, host int32 [nblocks][5]) = {i0, i1, j0, j1, far} as half-open
 * permuted ranges in depth-first order. */
int tdbem_tree_export(tdbem_tree_t tree, int32_t *perm_rows, int32_t *perm_cols, int64_t *nblocks,
                      int32_t *blocks);
int tdbem_tree_destroy(tdbem_tree_t tree);

/* ---- entries (Sec. 3; the ENTRY function of Algorithm 1) -------------------- */
/* out[f][r][c] = A[rows[r], cols[c]](s_{fidx[f]}) for every combination.
 * rows, cols, fidx: device int32 arrays; out: device complex array
 * (complex128 for prec FP64, complex64 for MIXED), layout [nf][nr][nc].
 * Touching pairs go through the FP64 Sauter-Schwab path in both precisions. */
int tdbem_entries(tdbem_mesh_t mesh, const tdbem_op *op, tdbem_freqs_t f, const int32_t *rows,
                  int64_t nr, const int32_t *cols, int64_t nc, const int32_t *fidx, int64_t nf,
                  void *out);

/* The same entries through one of the kernels that tdbem_compress runs, so
 * that each can be checked on its own against an independent evaluation:
 *   path = TDBEM_PATH_GENERIC: tdbem_entries itself;
 *   path = TDBEM_PATH_NEAR: the near-field phases of the compression on the
 *     single block rows x cols: the touching-pair table of the mesh
 *     (Sauter-Schwab, Sec. 3), then the dense near-field tensor kernel
 *     (regular pairs by the 7-point rule with the point geometry shared
 *     across frequencies, touching pairs read from the table); at most 256
 *     frequencies and 2^31 - 1 entries per frequency;
 *   path = TDBEM_PATH_FIBRE: the far-field engine's entry evaluation (the
 *     8-lane point-pair groups with which Algorithm 1's fibres and frequency
 *     tubes are formed in tdbem_compress), which applies the regular 7 x 7
 *     rule to every pair: admissible blocks hold no touching pairs, and on a
 *     touching pair this path does not give the operator's entry.
 * Arguments and layout as tdbem_entries.  The index arrays are copied to the
 * host and checked (TDBEM_ERR_ARG on an index out of range).  Allocates
 * transient device buffers and synchronises the context's stream. */
enum { TDBEM_PATH_GENERIC = 0, TDBEM_PATH_NEAR = 1, TDBEM_PATH_FIBRE = 2 };
int tdbem_entries_path(tdbem_mesh_t mesh, const tdbem_op *op, tdbem_freqs_t f, const int32_t *rows, int64_t nr,
                       const int32_t *cols, int64_t nc, const int32_t *fidx, int64_t nf, int32_t path, void *out);

/* Allocation-free variant of tdbem_entries (the paper has no counterpart; it
 * exists for callers that cannot allocate device memory at call time:
 * applications whose device memory is reserved up front by their own pool
 * allocator, and host loops that must not pay the device-wide
 * synchronisation of cudaFree).  Same arguments, kernel and results as
 * tdbem_entries; the few scratch values of a call (quadrature nodes, scaled
 * frequencies) live in one fixed device array of the library instead of
 * buffers allocated per call, and are written there by a small kernel on the
 * context's stream (no host-to-device copy).
 *   - No cudaMalloc, cudaFree or other allocating call is made.
 *   - The frequency set may have at most TDBEM_NOALLOC_MAX_NQ points;
 *     larger sets return TDBEM_ERR_ARG with a message.
 *   - tdbem_ctx_create looks up the device address of the fixed array (once
 *     per device).  The array (about 132 KB) stays allocated on every device
 *     that loaded the library until the process exits.
 *   - All calls share the array and it keeps the last call's contents; calls
 *     ordered on one stream are safe, calls that overlap on the GPU (other
 *     streams, other threads) race on it.
 *   - Asynchronous: returns after queuing the work on the context's stream. */
#define TDBEM_NOALLOC_MAX_NQ 8192
int tdbem_entries_noalloc(tdbem_mesh_t mesh, const tdbem_op *op, tdbem_freqs_t f, const int32_t *rows,
                          int64_t nr, const int32_t *cols, int64_t nc, const int32_t *fidx, int64_t nf,
                          void *out);

/* ---- compression (Sec. 4, Algorithm 1 per block, eq. norm) ------------------- */
/* 3D-ACA of the operator tensor over the Nu unique frequencies of f on every
 * block of `tree` (which must have been built with test P0 and trial P0 for
 * SLP and ADLP, P1 for DLP).  Near-field blocks: dense residual faces; far-field
 * blocks: residual faces compressed by ACA with partial pivoting to eps_aca,
 * rebuilt to find the pivot (Sec. 4).  The result stays in device memory. */
int tdbem_compress(tdbem_ctx_t ctx, tdbem_mesh_t mesh, const tdbem_op *op, tdbem_freqs_t f,
                   tdbem_tree_t tree, const tdbem_aca_cfg *cfg, tdbem_tensor_t *out);
int tdbem_tensor_stats(tdbem_tensor_t t, tdbem_stats *st);
/* Rebuilt entries C^r[rows[n], cols[n], fidx[n]] (fidx into the full NQ list,
 * conjugates mirrored) for n < count.  Device int32 inputs, device complex
 * output [count] in the tensor's precision. */
int tdbem_tensor_entries(tdbem_tensor_t t, const int32_t *rows, const int32_t *cols,
                         const int32_t *fidx, int64_t count, void *out);
/* Per-block results (host, nullable): ranks [nblocks], face rank sums
 * [nblocks], selected frequencies [nblocks][Nu+1] (-1 padded). */
int tdbem_tensor_blocks(tdbem_tensor_t t, int32_t *rank, int32_t *face_rank_sum, int32_t *kpiv);
/* The partition the tensor was compressed on (host, nullable): *nb blocks,
 * blocks [nb][5] = row begin, row end, column begin, column end (permuted
 * DOF ranges, as tdbem_tree_export) and 1 for far / 0 for near.  It refines
 * the tree's partition (see flags bit 2 of tdbem_aca_cfg); the per-block
 * results of tdbem_tensor_blocks follow its order. */
int tdbem_tensor_partition(tdbem_tensor_t t, int64_t *nb, int32_t *blocks);
int tdbem_tensor_destroy(tdbem_tensor_t t);
/* Project-written autotuner of the compression's launch parameters (Sec. 4
 * Algorithm 1 and the entry kernels of Sec. 3), kept in the context for
 * op->prec: times complete compressions of the given problem (the first of
 * two runs warms up) and keeps, phase by phase, the fastest
 *   - far phase: launch shape threads per CTA x resident CTAs per SM
 *     (64/128/256 threads, 2..16 CTAs per SM);
 *   - mixed form only: frequencies per pass of the touching-pair table
 *     (register tiles of 4/8/16 frequencies for the single layer and its adjoint, 2/4/8
 *     for the double layer) and of the near-field tensor kernel (8/4/16),
 *     each timed on its own phase.
 * chosen (nullable, host int32 [4]) receives {far threads per CTA, far CTAs
 * per SM, touching-pair frequencies per pass, near-field frequencies per
 * pass} (0 for the two mixed-form choices of an FP64 form).  Defaults without
 * tuning: {128, 4 (FP64) / 5 (mixed), 36 or 12, 8}. */
int tdbem_autotune(tdbem_ctx_t ctx, tdbem_mesh_t mesh, const tdbem_op *op, tdbem_freqs_t f, tdbem_tree_t tree,
                   const tdbem_aca_cfg *cfg, int32_t *chosen);

/* QR + SVD recompression of the far faces (Sec. 4, the H-matrix variant:
 * the ACA factors of every face are recompressed): a face H = U V^T of rank
 * k is replaced by the k' leading terms of its SVD (Householder QR of U and
 * V, one-sided Jacobi SVD of R_U R_V^T), k' the smallest rank with
 * sum_{i >= k'} s_i^2 <= eps^2 sum_i s_i^2, i.e. ||H - H'||_F <= eps ||H||_F
 * per face.  Computed in the tensor's precision (FP32 in the mixed form,
 * which resolves singular values down to ~1e-7 of the largest); the face
 * pool is then compacted to the new sizes and the statistics
 * (stored_complex, sum_face_rank) are updated.  Synchronous.  ERR_ARG unless
 * 0 < eps < 1. */
int tdbem_tensor_recompress(tdbem_tensor_t t, double eps);
/* The same recompression of one face (no counterpart in the paper; it exists
 * to test the kernel on its own): U device [k][nI], V device [k][nJ] (face
 * U V^T, column t of U at U + t nI), 1 <= k <= 64, complex64 (prec MIXED) or
 * complex128 (FP64); Uout [k][nI], Vout [k][nJ] receive the first *kout rows.
 * Synchronous. */
int tdbem_lowrank_recompress(tdbem_ctx_t ctx, int32_t prec, int32_t nI, int32_t nJ, int32_t k, const void *U,
                             const void *V, double eps, void *Uout, void *Vout, int32_t *kout);

/* ---- apply (eq. product) ------------------------------------------------------ */
/* y[M][nrhs] = sum_{l < NQ} A(s_l) W_l  with W: device [NQ][ncols][nrhs]
 * complex over all NQ points of the frequency set (conjugate partners are
 * folded in through A(conj s) = conj A(s)); y: device [nrows][nrhs], same
 * complex type as the tensor.  Evaluated as sum_d H_d (sum_l f_d[l] W_l). */
int tdbem_apply_weighted(tdbem_tensor_t t, const void *W, int32_t nrhs, void *y);
/* The mixed form evaluates the frequency contraction sum_l f_d(l) W_l of every
 * term as complex GEMMs on the tensor cores (tcgen05, BF16 operands split in
 * a high and a low part, FP32 accumulation; see tdbem_zgemm), keeps the
 * result in a device buffer of 2 * nrhs * sum_b rank_b * |J_b| complex values
 * owned by the tensor (reallocated when nrhs changes; with it a packed copy
 * of the fibre coefficients, and of W for each call, NQ * ncols * nrhs
 * complex values), and then applies the faces on the FP32 cores.  The first
 * call for a tensor and nrhs builds this plan on the host and synchronises
 * the stream.  The FP64 form runs every step in FP64. */
/* y = A(s_fidx) x for one point of the full list: x device [ncols][nrhs]. */
int tdbem_apply_freq(tdbem_tensor_t t, int32_t fidx, const void *x, int32_t nrhs, void *y);
/* Same as tdbem_apply_weighted with host W and y (pinned or pageable): the
 * host->device copy of W and the device->host copy of y are part of the
 * call, which returns when y is on the host. */
int tdbem_apply_weighted_host(tdbem_tensor_t t, const void *W_host, int32_t nrhs, void *y_host);

/* ---- tensor-core complex GEMM (no counterpart in the paper) ----------------
 * D = A B for complex64 device matrices A [M][K] (row stride lda), B [K][N]
 * (ldb), D [M][N] (ldd): the engine of the weighted apply's frequency
 * contraction, exposed so that it can be tested on its own.  tcgen05 MMAs
 * on split-BF16 operands (x = hi + lo, products hi*hi + hi*lo + lo*hi),
 * FP32 accumulation in tensor memory; relative error about 1e-5 of
 * sum_k |A[m][k]| |B[k][n]|.  Synchronous.  TDBEM_ERR_CUDA if a wait for the
 * tensor cores gave up (the result is then invalid). */
int tdbem_zgemm(tdbem_ctx_t ctx, int32_t M, int32_t N, int32_t K, const void *A, int64_t lda, const void *B,
                int64_t ldb, void *D, int64_t ldd);

/* Measured throughput of a pipe the compression runs on, the denominator of
 * its roofline (no counterpart in the paper): what = 0: FP32 fused
 * multiply-adds per second; 1: special-function operations per second
 * (reciprocal square root, base-2 exponential, sine, cosine in equal
 * parts: the four operations of a far-field point pair); 2: FP64 fused
 * multiply-adds per second; 3: FP64 single-layer point pairs per second
 * (distance, exp, sin and cos, weight, complex accumulate: the inner
 * operation of the FP64 form's entries).  Independent dependency chains on every SM, one
 * warm-up launch, then one launch timed with CUDA events (a few to tens of
 * milliseconds).  Synchronous.  TDBEM_ERR_ARG for another `what`. */
int tdbem_measure_peak(tdbem_ctx_t ctx, int32_t what, double *ops_per_s);

/* ---- per-frequency solve (Sec. 2, the Laplace-domain systems of the gCQ
 * step; Sec. 5 solves them iteratively) --------------------------------------
 * Solves A(s_fidx) x = b for nrhs right-hand sides with restarted GMRES
 * (modified Gram-Schmidt Arnoldi, complex Givens rotations, FP64 inner
 * products; every operator application is tdbem_apply_freq on the compressed
 * tensor).  The paper uses BiCGstab; GMRES reaches the same solution and
 * its residual decreases monotonically.  Square operators only (SLP).
 *   b, x     device [nrows][nrhs] complex in the tensor's precision
 *            (caller-owned; x is overwritten, the start vector is 0)
 *   tol      relative residual ||b - A x|| / ||b|| per column, > 0
 *   maxit    total Arnoldi steps (all restarts), >= 1
 *   restart  Krylov dimension per cycle (<= 0: 30; clamped to 200)
 *   iters    (nullable) host int32: Arnoldi steps taken
 *   relres   (nullable) host double [nrhs]: final relative residuals, formed
 *            explicitly as ||b - A x|| / ||b||
 * Returns TDBEM_ERR_NOT_CONVERGED (x holds the last iterate) when some column
 * is above tol after maxit steps.  Allocates (M * nrhs * (restart + 3))
 * complex values of device scratch per call and synchronises the stream. */
int tdbem_solve(tdbem_tensor_t t, int32_t fidx, const void *b, int32_t nrhs, void *x, double tol, int32_t maxit,
                int32_t restart, int32_t *iters, double *relres);

/* ---- gCQ time marching (Sec. 3 "Temporal discretisation", eqs. gCQ_xn and
 * gcq_formula; App. A) ----------------------------------------------------
 * The direct Dirichlet problem of Sec. 2 in Galerkin form (P0 test):
 *   V * q = (1/2 M + K) * g,   M[i][v] = int_{tau_i} phi_v,
 * g the Dirichlet data (P1 nodal values), q the Neumann data (P0), marched
 * with the Runge-Kutta based gCQ (rk = TDBEM_EULER or TDBEM_RADAU2) over the
 * steps dts.  Step n:
 *   x_{n-1}(s_l) = (I - dt_{n-1} s_l A)^{-1} ((b^T A^{-1} x_{n-2}(s_l)) 1 + dt_{n-1} A q_{n-1})
 *   V((dt_n A)^{-1}) q_n = 1/2 M g_n + K((dt_n A)^{-1}) g_n
 *                          + sum_l K(s_l) W_l[g] - sum_l V(s_l) W_l[q],
 *   W_l = omega_l (b^T A^{-1} x_{n-1}(s_l)) (I - dt_n s_l A)^{-1} 1,
 * omega_l = -w_l (w_l the positively oriented weights of tdbem_freqs_get).
 * The history sums are tdbem_apply_weighted on V and K, tensors compressed
 * over one gCQ contour (tdbem_freqs_gcq with the same steps); the step
 * operators at the matrix argument act through the eigenvalues mu_k =
 * 1/(dt lambda_k(A)) and run on Vstep and Kstep, tensors over a frequency set
 * holding every mu_k of the steps (tdbem_march_step_points, then
 * tdbem_freqs_points): tdbem_apply_freq for K, restarted GMRES
 * (tdbem_solve) for V.  All four tensors: one mesh, precision and wave speed;
 * V and Vstep single layer (P0 x P0), K and Kstep double layer (P0 x P1).
 * The marching keeps FP64 states x(s_l) of q and g at the unique contour
 * points (Nu * (nt + nv) * m * nrhs complex128) and weighted data in the
 * tensors' precision (NQ * (nt + nv) * m * nrhs complex values). */
typedef struct tdbem_march *tdbem_march_t;
/* The distinct step frequencies 1/(dt_n lambda_k(A)) of the steps (host
 * outputs): s (nullable) [2 * count] interleaved, *count. */
int tdbem_march_step_points(const double *dts, int32_t N, int32_t rk, double *s, int32_t *count);
/* m * nrhs <= 64 (m = 1 for EULER, 2 for RADAU2).  TDBEM_ERR_ARG for tensors
 * that do not match the description above. */
int tdbem_march_create(tdbem_tensor_t V, tdbem_tensor_t K, tdbem_tensor_t Vstep, tdbem_tensor_t Kstep,
                       const double *dts, int32_t N, int32_t rk, int32_t nrhs, tdbem_march_t *out);
/* One step: g device FP64 [nv][m][nrhs] (Dirichlet data at the stage times
 * t_{n-1} + c_i dt_n), q device FP64 [nt][m][nrhs] (output, Neumann data at
 * the stage times).  tol, maxit: GMRES of the step system (relative
 * residual per column).  iters (nullable): GMRES steps taken.  Synchronous;
 * TDBEM_ERR_NOT_CONVERGED from the solve, TDBEM_ERR_ARG after N steps. */
int tdbem_march_step(tdbem_march_t mh, const double *g, double *q, double tol, int32_t maxit, int32_t *iters);
int tdbem_march_destroy(tdbem_march_t mh);

/* ---- persistence (not part of the paper) ------------------------------------
 * tdbem_tensor_save writes the compressed tensor (block list, permutations,
 * per-block ranks and selected frequencies, fibres, face pool, statistics) to
 * a binary file in native byte order; tdbem_tensor_load reads it into a new
 * tensor of ctx that apply, tensor_entries, blocks, stats and solve accept
 * like a freshly compressed one.  The file does not hold the mesh or the
 * frequency set.  Errors: TDBEM_ERR_ARG for unreadable or foreign files.
 * tdbem_model_save/load do the same for the rank predictor's FP32 parameters
 * (the BF16 inference copy is rebuilt on load; the Adam state is not kept). */
int tdbem_tensor_save(tdbem_tensor_t t, const char *path);
/* Shape of a tensor (host outputs, each nullable): operator, precision,
 * rows, columns, points of the frequency set, unique points. */
int tdbem_tensor_info(tdbem_tensor_t t, int32_t *op, int32_t *prec, int64_t *nrows, int64_t *ncols, int32_t *NQ,
                      int32_t *Nu);
int tdbem_tensor_load(tdbem_ctx_t ctx, const char *path, tdbem_tensor_t *out);
int tdbem_model_save(tdbem_model_t m, const char *path);
int tdbem_model_load(tdbem_ctx_t ctx, const char *path, tdbem_model_t *out);

/* ---- rank predictor (learned presizing; not part of the paper) ------------
 * A small MLP (6 features -> 64 -> 64 -> 16 rank bins, GELU) predicts, for a
 * far-field block and a frequency, the bin of the rank that the ACA of the
 * plain face reaches at eps_aca.  With cfg->model set, tdbem_compress uses
 * the prediction to order the far blocks by predicted cost, to presize the
 * face pool and to run the first (lower bin edge) ACA steps of each face
 * without per-step norm checks; their norms are then formed in one batch and
 * the adaptive stopping rule picks the same rank it would have picked step by
 * step (the criterion still decides; under-predicted faces simply continue).
 * Bins: rank <= 1, 2, 3, 4, 6, 8, 10, 12, 16, 20, 24, 32, 40, 48, 64, > 64.
 * Features (dimensionless): log(diam_I/dist), log(diam_J/dist), log(dist/h),
 * min(diam)/dist, log(1 + Re(s) dist/c), log(1 + |Im(s)| dist/c), h the mean
 * edge length.  Parameters (FP32 master, BF16 copy for inference) in the
 * order W1[64][6] b1[64] W2[64][64] b2[64] W3[16][64] b3[16]. */
#define TDBEM_MLP_NPARAMS 5648
#define TDBEM_NFEAT 6
#define TDBEM_NBINS 16
int tdbem_rank_bin(int32_t rank);
/* Seeded initialisation (uniform +-sqrt(6/fan_in), zero biases), on the device. */
int tdbem_model_create(tdbem_ctx_t ctx, uint64_t seed, tdbem_model_t *out);
int tdbem_model_destroy(tdbem_model_t m);
/* Host copies of the FP32 master parameters [TDBEM_MLP_NPARAMS]; set also
 * resets the Adam moments. */
int tdbem_model_get_params(tdbem_model_t m, float *host);
int tdbem_model_set_params(tdbem_model_t m, const float *host);
/* Mean softmax cross-entropy over n samples and its gradient (FP32):
 * x device [n][6], labels device [n] (bins), grad device [NPARAMS], loss
 * device [1]. */
int tdbem_model_loss_grad(tdbem_model_t m, const float *x, const int32_t *labels, int64_t n, float *grad,
                          float *loss);
/* One Adam step (b1 0.9, b2 0.999, eps 1e-8) with step counter t >= 1. */
int tdbem_model_adam_step(tdbem_model_t m, const float *grad, double lr, int32_t t);
/* Minibatch Adam over a seeded shuffle of (x, labels) (device arrays);
 * final_loss (nullable, host) receives the loss over the whole set. */
int tdbem_model_train(tdbem_model_t m, const float *x, const int32_t *labels, int64_t n, int32_t epochs,
                      int32_t batch, double lr, uint64_t seed, double *final_loss);
/* BF16-weight inference: bins device [n] (nullable), logits device [n][16]
 * (nullable). */
int tdbem_model_predict(tdbem_model_t m, const float *x, int64_t n, int32_t *bins, float *logits);
/* Training samples from the plain method: for every far block of `tree`
 * (tree order) and every unique frequency, the features (device float
 * [count][6]) and the rank of the ACA of the plain face at cfg->eps_aca
 * (device int32 [count]; max_face_rank + 1 when the cap was hit).  With
 * feats or ranks NULL only *count is returned; ERR_ARG if capacity < count. */
int tdbem_harvest(tdbem_ctx_t ctx, tdbem_mesh_t mesh, const tdbem_op *op, tdbem_freqs_t f, tdbem_tree_t tree,
                  const tdbem_aca_cfg *cfg, float *feats, int32_t *ranks, int64_t capacity, int64_t *count);

#ifdef __cplusplus
}
#endif
#endif
