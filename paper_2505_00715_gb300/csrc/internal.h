// Internal host-side structures of the tdbem library (not part of the C-ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/tdbem.h"

struct tdbem_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t capture = nullptr;  // side stream used only to capture graphs
    // launch shape of the far-field kernel per precision form [FP64, MIXED]:
    // threads per CTA and CTAs per SM (set by tdbem_autotune)
    int far_nt[2] = {128, 128};
    int far_cps[2] = {4, 5};
    // tuning variants of the mixed form's touching-pair table and near-field
    // tensor kernels (frequencies per pass; 0 = default), set by tdbem_autotune
    int sing_var = 0, near_var = 0;
    int64_t near_batch_bytes = (int64_t)16 << 30;  // buffer of the batched near-field tensor
    double pool_scale = 1.0;                       // far part of the first face-pool size
    std::string err;
    int num_sms = 0;
    int *dflags = nullptr;  // device status word of asynchronous kernels (TD_DEV_* bits)
    uint32_t wait_polls = 0;  // poll limit of the tensor-core waits (0: the kernels' default)
};

// Host-side planner output for the cluster trees and the block list.
struct ClusterNode {
    int32_t begin, end, son0, son1;
    double box[6];
};

struct HostTree {
    int basis = 0;
    int64_t n = 0;
    std::vector<int32_t> perm;
    std::vector<ClusterNode> nodes;
};

struct tdbem_tree {
    tdbem_mesh *mesh = nullptr;
    HostTree side[2];
    std::vector<int32_t> blocks;  // [nb][5]
    int leaf = 0;
    double eta = 0.0;
};

struct tdbem_mesh {
    tdbem_ctx *ctx = nullptr;
    int64_t nv = 0, nt = 0;
    std::vector<double> verts;
    std::vector<int32_t> tris;
    std::vector<double> area;
    // vertex -> triangle incidence (P1 supports)
    std::vector<int32_t> v2t_ptr, v2t;
    std::vector<int8_t> v2t_loc;
    // touching triangles per triangle (sorted by triangle index)
    std::vector<int32_t> tp_ptr, tp_tri;
    // device tables
    float *qxh = nullptr, *qyh, *qzh, *qxl, *qyl, *qzl, *qw32, *n32;
    void *qp = nullptr, *nrm4 = nullptr;  // float4 packs of the FP32 tables (see MeshDev)
    double *qx = nullptr, *qy, *qz, *qw, *n64, *dverts, *darea;
    int32_t *dtris = nullptr, *dv2t_ptr = nullptr, *dv2t = nullptr;
    int8_t *dv2t_loc = nullptr;
    int32_t *dtp_ptr = nullptr, *dtp_tri = nullptr;
    void *dev_block = nullptr;  // one allocation holding all tables
};

struct tdbem_freqs {
    tdbem_ctx *ctx = nullptr;
    int32_t NQ = 0, Nu = 0;
    std::vector<double> s, w;     // [2*NQ] host copies
    std::vector<int32_t> unique;  // per point: rep+1 or -(rep+1)
    std::vector<int32_t> uidx;    // unique representative -> point index
    double *ds = nullptr;         // device [2*NQ]
    double *dw = nullptr;
    int kind = 0;                 // 0 BDF2, 1 gCQ, 2 explicit points
    std::vector<double> dts;      // gCQ: the time steps the contour was built for
    double rho = 1.0;             // gCQ: radius factor of the contour (td_gcq_radius)
};

// Compressed tensor (device pools + host copies of the small metadata).
struct tdbem_tensor {
    tdbem_ctx *ctx = nullptr;
    tdbem_mesh *mesh = nullptr;
    tdbem_freqs *freqs = nullptr;
    int op = 0, prec = 0;
    double c = 1.0;
    int ng = 5;
    int64_t nrows = 0, ncols = 0;
    int Nu = 0, NQ = 0;
    int64_t nblocks = 0;
    int32_t *dblocks = nullptr;     // [nb][5] permuted ranges
    int32_t *dperm_r = nullptr, *dperm_c = nullptr;   // position -> DOF
    int32_t *dinv_r = nullptr, *dinv_c = nullptr;     // DOF -> position
    // per block: number of terms, per term (fixed slots [nb][Nu]): selected
    // frequency, face rank (-1 dense), face offset (complex units)
    int32_t *drank = nullptr, *dkpiv = nullptr, *dfrank = nullptr;
    int64_t *dfoff = nullptr;
    void *dfib = nullptr;           // fibres [nb][Nu][Nu] complex
    void *dface = nullptr;          // face pool (complex)
    int64_t face_cap = 0;
    int64_t *dface_used = nullptr;
    // host copies (filled by compress)
    std::vector<int32_t> blocks;
    std::vector<int32_t> rank, frank_sum;
    tdbem_stats stats{};
    std::vector<void *> owned;      // device allocations to free
    int32_t *dpartner = nullptr;    // [NQ] unique-map of the frequency set
    int kcap = 64;                  // face-rank cap used by the compression
    int max_near_rows = 1;
    void *dy_host = nullptr;        // staging buffers of tdbem_apply_weighted_host
    // plan of the tensor-core weighted apply (mixed form), rebuilt when nrhs
    // changes: groups | row table | jobs | per-block Z offsets, and Z itself
    int plan_nrhs = 0, plan_rpt = 1, plan_njobs = 0, plan_maxI = 1, plan_maxJ = 1;
    void *plan_mem = nullptr, *plan_Z = nullptr;
    size_t plan_off[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int plan_nq0 = 0;
    // packed contraction operands inside plan_Z (complex offsets), their row
    // strides and half widths (see td_launch_pack_fibres / _weights)
    int64_t plan_fp = 0, plan_wk = 0;
    int plan_fw = 0, plan_kw0 = 0, plan_kw1 = 0;
    int plan_nft = 0;
    int64_t plan_tz = 0;
    size_t host_buf_bytes = 0;
};

// helpers (api.cu)
int td_fail(tdbem_ctx *ctx, int code, const char *fmt, ...);
#define TD_CUDA(ctx, call)                                                                   \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return td_fail((ctx), TDBEM_ERR_CUDA, "%s: %s (%s:%d)", #call,                   \
                           cudaGetErrorString(e_), __FILE__, __LINE__);                      \
    } while (0)

// api.cu: argument check of an operator description, and the device view of
// a mesh's tables (Gauss-Legendre rule gx/gw and touching-pair slots as given)
struct MeshDev;
int td_check_op(tdbem_ctx *ctx, const tdbem_op *op);
MeshDev td_mesh_dev(const tdbem_mesh *m, int ng, const double *gx, const double *gw, const int *tp_slot);
// noalloc.cu: device address of the allocation-free entry point's scratch on
// the current device `device` (once per device, cached)
int td_noalloc_setup(int device);

// api.cu: radius factor of the gCQ contour for nsteps steps of method rk
double td_gcq_radius(int rk, int nsteps);

// planner.cpp
void td_plan_tree(const tdbem_mesh *m, int basis, int leaf, HostTree &t);
void td_plan_blocks(const HostTree &rows, const HostTree &cols, double eta,
                    std::vector<int32_t> &blocks);
void td_mesh_adjacency(tdbem_mesh *m);
int td_gauss01(int n, double *x, double *w);
void td_rule7(double bary[7][3], double w[7]);

// planner.cpp: the tree's partition with far blocks above twice the mean far
// work of one of nctas persistent CTAs split into their sons' blocks
void td_balance_partition(const HostTree &R, const HostTree &C, const std::vector<int32_t> &blocks, int64_t nctas,
                          std::vector<int32_t> &out);

// model.cu (blocks: a partition of the tree's clusters, [nb][5])
struct tdbem_model;
void td_block_features(const tdbem_tree *t, const std::vector<int32_t> &blocks, const tdbem_mesh *m,
                       const tdbem_freqs *f, double c, const std::vector<int32_t> &far, std::vector<float> &x);
int td_predict_kpred(tdbem_model *M, const tdbem_tree *t, const std::vector<int32_t> &blocks, const tdbem_mesh *m,
                     const tdbem_freqs *f, double c, const std::vector<int32_t> &far, int kcap, int32_t *dkpred,
                     std::vector<double> &cost, std::vector<int32_t> &ks);
