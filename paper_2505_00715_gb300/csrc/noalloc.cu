// tdbem_entries_noalloc: the entry kernel of tdbem_entries without any device
// allocation (include/tdbem.h).  The paper has no counterpart.
//
// tdbem_entries allocates a few small device buffers on every call (the
// Gauss-Legendre nodes of the touching-pair rule, the frequencies divided by
// the wave speed, the touching-pair slot table) and frees them before it
// returns.  Some callers cannot allocate device memory at that point:
// applications whose device memory is reserved up front by their own pool
// allocator (a cudaMalloc would fail or steal from the pool), and hosts that
// must not pay the device-wide synchronisation of cudaFree inside a loop.
// This variant keeps that scratch in one fixed array in device memory,
// declared below, fills it on the device (no host-to-device copy of per-call
// data) and never calls cudaMalloc, cudaFree or any allocating routine.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "internal.h"
#include "kernels.h"
#include "pair.cuh"

// Scratch of the allocation-free entry point: 64 Gauss-Legendre values
// (nodes then weights, 32 each) followed by 2 * TDBEM_NOALLOC_MAX_NQ doubles of
// scaled frequencies.  Every GPU that loads the library holds it (about
// 132 KB) until the process exits.  All calls share it and it keeps the
// contents of the last call; nothing in it needs to start at zero, since each
// call writes every element it reads before reading it.
static __device__ __align__(256) double g_noalloc_scratch[64 + 2 * TDBEM_NOALLOC_MAX_NQ];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double *g_scratch_addr[kMaxDevices] = {};

// Fills the scratch for one call: the ng-point Gauss-Legendre rule on [0, 1]
// (Newton iteration on the three-term Legendre recurrence from the usual
// cosine first guess, one thread per node) and sig[k] = s[k] / c for every
// point of the frequency set.  One block.
__global__ void k_noalloc_fill(double *scratch, int ng, const double *s, int n2, double inv_c) {
    const int t = threadIdx.x;
    if (t < ng) {
        const double pi = 3.141592653589793238462643383279502884;
        double z = cos(pi * (t + 0.75) / (ng + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double pm = 1.0, p = z;
            for (int k = 2; k <= ng; ++k) {
                const double pn = ((2 * k - 1) * z * p - (k - 1) * pm) / k;
                pm = p;
                p = pn;
            }
            if (ng == 1) pm = 1.0;
            dp = ng * (z * p - pm) / (z * z - 1.0);
            const double step = p / dp;
            z -= step;
            if (fabs(step) < 1e-16) break;
        }
        // derivative at the converged node
        double pm = 1.0, p = z;
        for (int k = 2; k <= ng; ++k) {
            const double pn = ((2 * k - 1) * z * p - (k - 1) * pm) / k;
            pm = p;
            p = pn;
        }
        if (ng == 1) pm = 1.0;
        dp = ng * (z * p - pm) / (z * z - 1.0);
        scratch[t] = 0.5 * (1.0 - z);
        scratch[32 + t] = 1.0 / ((1.0 - z * z) * dp * dp);
    }
    for (int k = t; k < n2; k += blockDim.x) scratch[64 + k] = s[k] * inv_c;
}

}  // namespace

// Resolves the device address of the scratch array on `device`, which must be
// the current device (the host-side name of the array is not a device
// address).  Called once per device by tdbem_ctx_create; later calls return
// the cached address.
int td_noalloc_setup(int device) {
    if (device < 0 || device >= kMaxDevices) return TDBEM_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (g_scratch_addr[device]) return TDBEM_OK;
    double *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress((void **)&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return TDBEM_ERR_CUDA;
    }
    g_scratch_addr[device] = p;
    return TDBEM_OK;
}

extern "C" int tdbem_entries_noalloc(tdbem_mesh_t mesh, const tdbem_op *op, tdbem_freqs_t f, const int32_t *rows,
                                     int64_t nr, const int32_t *cols, int64_t nc, const int32_t *fidx, int64_t nf,
                                     void *out) {
    cudaGetLastError();  // errors of earlier unrelated calls are not ours to report
    if (!mesh || !f) return TDBEM_ERR_ARG;
    tdbem_ctx *ctx = mesh->ctx;
    int rc = td_check_op(ctx, op);
    if (rc) return rc;
    if (nr < 0 || nc < 0 || nf < 0 || (nr * nc * nf > 0 && (!rows || !cols || !fidx || !out)))
        return td_fail(ctx, TDBEM_ERR_ARG, "tdbem_entries_noalloc: bad sizes or NULL pointers");
    if (f->NQ > TDBEM_NOALLOC_MAX_NQ)
        return td_fail(ctx, TDBEM_ERR_ARG,
                       "tdbem_entries_noalloc: the frequency set has %d points; the fixed scratch holds at most %d",
                       f->NQ, TDBEM_NOALLOC_MAX_NQ);
    if (nr * nc * nf == 0) return TDBEM_OK;
    double *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (ctx->device >= 0 && ctx->device < kMaxDevices) scratch = g_scratch_addr[ctx->device];
    }
    if (!scratch)
        return td_fail(ctx, TDBEM_ERR_CUDA, "tdbem_entries_noalloc: the scratch address of device %d is not known "
                                            "(tdbem_ctx_create could not resolve it)", ctx->device);
    // the scratch is written on the context's stream, after the earlier work
    // of that stream (so a previous call on the same stream has finished
    // reading it) and before the entry kernel reads it
    k_noalloc_fill<<<1, 256, 0, ctx->stream>>>(scratch, op->ng, f->ds, 2 * f->NQ, 1.0 / op->c);
    if (cudaPeekAtLastError() != cudaSuccess)
        return td_fail(ctx, TDBEM_ERR_CUDA, "tdbem_entries_noalloc: scratch kernel launch failed: %s",
                       cudaGetErrorString(cudaGetLastError()));
    // the mesh tables of tdbem_entries; the generic kernel only asks whether
    // two triangles touch (a non-negative slot), which the touching list's own
    // triangle indices answer without the slot table
    MeshDev m = td_mesh_dev(mesh, op->ng, scratch, scratch + 32, mesh->dtp_tri);
    if (td_launch_entries(ctx->stream, m, op->op, op->prec, scratch + 64, f->NQ, rows, nr, cols, nc, fidx, nf, out))
        return td_fail(ctx, TDBEM_ERR_CUDA, "tdbem_entries_noalloc: kernel launch failed");
    return TDBEM_OK;
}
