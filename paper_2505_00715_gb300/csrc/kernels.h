// Kernel launch interfaces shared by the C-ABI layer and the kernel files.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

struct MeshDev;

struct NearArgs {
    int nf;                  // unique frequencies
    const double *sig;       // [2*nf] sigma = s / c
    int nnear;
    const int *near_ids;     // block index of near block n
    const int64_t *eprefix;  // [nnear] prefix of nI*nJ
    const int64_t *noff;     // [nnear] offset (complex units) into `near`, layout [nf][nI][nJ]
    const int *blocks;       // [nb][5]
    const int *perm_r, *perm_c;
    int64_t nentries;
    void *near;
};

// Output arrays of the compressed tensor (fixed slots per block and term).
struct TensorOut {
    int Nu;
    int *rank;          // [nb]
    int *kpiv;          // [nb][Nu]
    int *frank;         // [nb][Nu] face rank (-1 dense)
    int64_t *foff;      // [nb][Nu] offset of the face in the pool (complex units)
    void *fib;          // [nb][Nu][Nu] complex
    void *face;         // pool
    int64_t face_cap;
    unsigned long long *face_used;
    int *dev_flags;     // TD_DEV_* bits
};

struct AcaParams {
    double eps, eps_aca;
    int kcap;           // face-rank cap
};

struct FarArgs {
    int nfar;
    const int *far_ids;     // block ids, processing order
    const int *blocks;
    const int *perm_r, *perm_c;
    const double *sig;      // [2*Nu]
    int nf;
    int maxI, maxJ;
    void *scratch;          // per-CTA workspace: U [kcap][maxI], V [kcap][maxJ], the rebuilt
                            // dense faces of the first min(td_far_dense_terms(),
                            // dense_cap / |I||J|) terms [dense_cap], the correction C(k)
                            // [min(dense_cap, td_far_cd_max())]
    int64_t scratch_per_cta;  // complex units
    unsigned int *counter;  // work queue head
    int64_t *evals;         // [3] regular, tube entries evaluated; ACA stopping tests of the
                            // low-rank-norm faces (one per synchronised test round)
    int *harvest;           // non-null: record face-ACA ranks per (far block, frequency), [nfar][Nu]
    const int *kpred;       // nullable: predicted face rank per (block id, frequency) [nb][Nu]
    int64_t dense_cap;      // complex entries of dense faces per CTA (0: none)
    int *redo;              // nullable: ids of blocks stopped by a full face pool [nfar]
    unsigned int *redo_count;
};

// k_peak.cu: throughput microbenchmark (what: 0 FP32 FMA, 1 special-function
// unit, 2 FP64 FMA); *ops = operations performed by the launch
int td_launch_peak(cudaStream_t st, int what, int grid, int iters, void *out, double *ops);
int td_launch_entries(cudaStream_t st, const MeshDev &m, int op, int prec, const double *sig, int nq,
                      const int *rows, int64_t nr, const int *cols, int64_t nc, const int *fidx,
                      int64_t nf, void *out);
// variant: tuning choice of the mixed form's frequencies per pass (0 = default;
// td_sing_fc / td_near_fc give the values)
int td_launch_sing_table(cudaStream_t st, const MeshDev &m, int op, int prec, const int *pti, const int *ptj,
                         int npairs, const double *sig, int nf, c64 *table, int num_sms, int variant = 0);
int td_launch_near_entries(cudaStream_t st, const MeshDev &m, int op, int prec, const NearArgs &a,
                           const c64 *table, int num_sms, int variant = 0);
int td_sing_fc(int op, int variant);
int td_near_fc(int variant);
int td_launch_near_aca(cudaStream_t st, int prec, const NearArgs &a, const TensorOut &o,
                       const AcaParams &p, void *scratch, int64_t scratch_per_cta, int nctas);
// Dense faces a far-field CTA keeps per block at most, and the largest block
// that forms C(k) once per term (the scratch of a CTA holds dense_cap entries
// of packed dense faces and min(dense_cap, td_far_cd_max()) for C(k)).
int td_far_dense_terms();
int td_far_cd_max();
int td_launch_far_aca(cudaStream_t st, const MeshDev &m, int op, int prec, const FarArgs &a,
                      const TensorOut &o, const AcaParams &p, int nctas, int nt);
// k_aca.cu: entries by the far-field engine's point-pair groups (fibres, tubes)
int td_launch_fibre_entries(cudaStream_t st, const MeshDev &m, int op, int prec, const double *sig, const int *rows,
                            int64_t nr, const int *cols, int64_t nc, int64_t nf, void *out, int num_sms);
int td_launch_bdf2(cudaStream_t st, int N, double dt, double lam, double *ds);
int td_launch_gcq(cudaStream_t st, int NQ, double dt_min, double q, double *ds, double *dw);

struct ApplyArgs {
    int nb;
    const int *blocks;
    const int *perm_r, *perm_c;
    int Nu, NQ;
    const int *qmap;       // [NQ] unique map (rep+1 or -(rep+1))
    const void *W;         // [NQ][ncols][nrhs]
    int nrhs;
    int64_t ncols;
    void *y;               // [nrows][nrhs]
    int single_f;          // >= 0: apply one frequency only (W is x [ncols][nrhs])
    int kcap;              // largest far face rank
    int max_near_rows;     // largest row count of a near block
    int64_t acc_max;       // accumulator size (complex units), set by the launcher
};
int td_launch_apply(cudaStream_t st, int prec, const ApplyArgs &a, const TensorOut &o, int num_sms);

// ---- tensor-core complex GEMM (k_zgemm.cu) and the apply built on it ----
// max_polls: poll limit of each tensor-core wait (0: the default); a wait that
// gives up sets TD_DEV_TIMEOUT in *err, lets its MMAs finish and returns
struct ZJob {               // one output tile
    int g, m0, n0;          // group, first row, first complex column
    int half;               // K range: 0 every frequency, 1 the first nq0 (half 0), 2 the rest
};
struct ZGroup {             // rows (block, term, half) that share a column cluster
    int J0, nJ;             // column cluster (permuted column range)
    int row0, M;            // first entry in the row table, number of rows
    int64_t zoff;           // offset of the group's first Z row (complex units)
    int L, Mh;              // Z row length = nJ * nrhs; rows of half 0 (the half-1 rows follow)
};
int td_launch_zgemm_dense(cudaStream_t st, const c32 *A, int64_t lda, const c32 *B, int64_t ldb, c32 *D, int64_t ldd,
                          int M, int N, int K, const ZJob *jobs, int njobs, int *err, uint32_t max_polls,
                          int num_sms);
// Operands of the apply contraction, packed so that a tile's 8 consecutive
// frequencies of a row are 64 contiguous bytes.  Frequency order lperm: the
// nq0 frequencies of half 0 first, then the nq1 of the conjugate half; each
// half padded with zeros to KW0 / KW1 (multiples of 32) values.
//   Fp[r][k'] (row stride FW = max(KW0, KW1)): Z row r = (block, term, half p)
//     -> its coefficient at frequency lperm[(p ? nq0 : 0) + k'] (conjugated for
//     p = 1), once per apply plan;
//   Wk[j' nrhs + c][hoff_p + k'] (row stride WS = KW0 + KW1, hoff_1 = KW0):
//     W[lperm[(p ? nq0 : 0) + k']][perm_c[j']][c], once per apply.
int td_launch_pack_fibres(cudaStream_t st, const int2 *rowtab, int64_t nrows, const int *qmap, const int *lperm,
                          int nq0, int nq1, const c32 *fib, int Nu, c32 *Fp, int FW, int num_sms);
int td_launch_pack_weights(cudaStream_t st, const c32 *W, const int *perm_c, const int *lperm, int64_t ncols,
                           int nrhs, int nq0, int nq1, int KW0, int KW1, c32 *Wk, int num_sms);
int td_launch_zgemm_apply(cudaStream_t st, const ZGroup *groups, const c32 *Fp, int FW, const c32 *Wk, int WS,
                          int hoff1, int nq0, int nq1, c32 *Z, int nrhs, const ZJob *jobs, int njobs, int *err,
                          uint32_t max_polls, int num_sms);
int td_zgemm_tile_rows();
int td_zgemm_tile_cols();

// second phase of the tensor-core apply: y += faces x Z (k_apply.cu)
struct ApplyZArgs {
    int nb;
    const int *blocks;
    const int *perm_r;
    int Nu, nrhs, rpt;      // rpt: Z rows per term (2 with a conjugate half, else 1)
    const int64_t *zbase;   // [nb] Z offset of the block's row (term 0, half 0) (-1: rank 0);
                            // row (d, p) at zbase + p zpstride + d nJ nrhs
    const int64_t *zpstride;  // [nb] offset between a block's half-0 and half-1 rows
    const c32 *Z;
    c32 *y;
    // far terms: T = V_d^T z1 and V_d^H z2, at toff[b Nu + d] + (p k_d + tau) nrhs + c
    int nft;                // number of far terms
    const int2 *ftab;       // (block, term) of every far term
    const int64_t *toff;    // [nb][Nu]
    c32 *T;
};
int td_launch_apply_z(cudaStream_t st, const ApplyZArgs &a, const TensorOut &o, int num_sms);
int td_launch_tensor_entries(cudaStream_t st, int prec, const TensorOut &o, const int *blocks,
                             int nb, int64_t nrows, int64_t ncols, int nq, const int *inv_r,
                             const int *inv_c, const int *qmap,
                             const int *rows, const int *cols, const int *fidx, int64_t count,
                             void *out);
