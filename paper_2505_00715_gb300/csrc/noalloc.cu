// tdbem_entries_noalloc: the entry kernel of tdbem_entries without any device
// allocation (include/tdbem.h).
//
// tdbem_entries allocates a few small device buffers on every call (the
// Gauss-Legendre nodes of the touching-pair rule, the frequencies divided by
// the wave speed, the touching-pair slot table) and frees them before it
// returns.  Some callers cannot allocate device memory at that point: code
// running while a stream is being captured into a CUDA graph (cudaMalloc and
// cudaFree are not capturable), applications whose device memory is fully
// reserved up front by their own pool allocator, and hosts that must not pay
// the implicit synchronisation of cudaFree.  This variant keeps that scratch
// in one fixed array in device memory, declared below, and never calls
// cudaMalloc, cudaFree or any allocating routine.
#include <algorithm>
#include <mutex>

#include "internal.h"
#include "kernels.h"
#include "pair.cuh"

// Scratch of the allocation-free entry point: 64 Gauss-Legendre values
// (nodes then weights, 32 each) followed by 2 * TDBEM_NOALLOC_MAX_NQ doubles of
// scaled frequencies.  Every GPU that loads the library holds it (about
// 132 KB) until the process exits.  All calls share it and it keeps the
// contents of the last call; nothing in it needs to start at zero, since each
// call writes every element it reads.
static __device__ __align__(256) double g_noalloc_scratch[64 + 2 * TDBEM_NOALLOC_MAX_NQ];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on `device` (looked up once per device
// with that device current; the host-side symbol is not a device address).
int scratch_address(int device, double **out) {
    if (device < 0 || device >= kMaxDevices) return TDBEM_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[device]) {
        int cur = -1;
        if (cudaGetDevice(&cur) != cudaSuccess) return TDBEM_ERR_CUDA;
        if (cur != device && cudaSetDevice(device) != cudaSuccess) return TDBEM_ERR_CUDA;
        double *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress((void **)&p, g_noalloc_scratch);
        if (cur != device) cudaSetDevice(cur);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return TDBEM_ERR_CUDA;
        }
        g_scratch_addr[device] = p;
    }
    *out = g_scratch_addr[device];
    return TDBEM_OK;
}

}  // namespace

extern "C" int tdbem_entries_noalloc(tdbem_mesh_t mesh, const tdbem_op *op, tdbem_freqs_t f, const int32_t *rows,
                                     int64_t nr, const int32_t *cols, int64_t nc, const int32_t *fidx, int64_t nf,
                                     void *out) {
    cudaGetLastError();  // errors of earlier unrelated calls are not ours to report
    if (!mesh || !f || !op) return TDBEM_ERR_ARG;
    tdbem_ctx *ctx = mesh->ctx;
    if ((op->op != TDBEM_SLP && op->op != TDBEM_DLP) || (op->prec != TDBEM_FP64 && op->prec != TDBEM_MIXED) ||
        !(op->c > 0.0) || op->ng < 1 || op->ng > 16)
        return td_fail(ctx, TDBEM_ERR_ARG, "tdbem_entries_noalloc: bad operator description");
    if (nr < 0 || nc < 0 || nf < 0 || (nr * nc * nf > 0 && (!rows || !cols || !fidx || !out)))
        return td_fail(ctx, TDBEM_ERR_ARG, "tdbem_entries_noalloc: bad sizes or NULL pointers");
    if (f->NQ > TDBEM_NOALLOC_MAX_NQ)
        return td_fail(ctx, TDBEM_ERR_ARG,
                       "tdbem_entries_noalloc: the frequency set has %d points; the fixed scratch holds at most %d",
                       f->NQ, TDBEM_NOALLOC_MAX_NQ);
    if (nr * nc * nf == 0) return TDBEM_OK;
    double *scratch = nullptr;
    int rc = scratch_address(ctx->device, &scratch);
    if (rc) return td_fail(ctx, rc, "tdbem_entries_noalloc: could not resolve the scratch address");
    // fill the scratch from small host stack buffers (copies from pageable
    // host memory are staged before cudaMemcpyAsync returns, and are ordered
    // after the earlier work of the stream, so a previous call on the same
    // stream has finished reading the scratch)
    double nodes[64] = {0.0};
    td_gauss01(op->ng, nodes, nodes + 32);
    TD_CUDA(ctx, cudaMemcpyAsync(scratch, nodes, sizeof(nodes), cudaMemcpyHostToDevice, ctx->stream));
    double *sig = scratch + 64;
    for (int k0 = 0; k0 < 2 * f->NQ; k0 += 128) {
        const int n = std::min(128, 2 * f->NQ - k0);
        double chunk[128];
        for (int k = 0; k < n; ++k) chunk[k] = f->s[k0 + k] / op->c;
        TD_CUDA(ctx, cudaMemcpyAsync(sig + k0, chunk, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream));
    }
    // the same mesh tables as tdbem_entries; the generic kernel only asks
    // whether two triangles touch, which the touching list itself answers
    MeshDev m{};
    m.nt = (int)mesh->nt;
    m.nv = (int)mesh->nv;
    m.qxh = mesh->qxh;
    m.qyh = mesh->qyh;
    m.qzh = mesh->qzh;
    m.qxl = mesh->qxl;
    m.qyl = mesh->qyl;
    m.qzl = mesh->qzl;
    m.qw32 = mesh->qw32;
    m.n32 = mesh->n32;
    m.qp = (const float4 *)mesh->qp;
    m.nrm4 = (const float4 *)mesh->nrm4;
    m.qx = mesh->qx;
    m.qy = mesh->qy;
    m.qz = mesh->qz;
    m.qw = mesh->qw;
    m.n64 = mesh->n64;
    m.verts = mesh->dverts;
    m.tris = mesh->dtris;
    m.area = mesh->darea;
    m.v2t_ptr = mesh->dv2t_ptr;
    m.v2t = mesh->dv2t;
    m.v2t_loc = (const signed char *)mesh->dv2t_loc;
    m.tp_ptr = mesh->dtp_ptr;
    m.tp_tri = mesh->dtp_tri;
    m.tp_slot = mesh->dtp_tri;  // non-negative entries: "touching" is all the kernel reads
    m.ng = op->ng;
    m.gx = scratch;
    m.gw = scratch + 32;
    if (td_launch_entries(ctx->stream, m, op->op, op->prec, sig, f->NQ, rows, nr, cols, nc, fidx, nf, out))
        return td_fail(ctx, TDBEM_ERR_CUDA, "tdbem_entries_noalloc: kernel launch failed");
    return TDBEM_OK;
}
