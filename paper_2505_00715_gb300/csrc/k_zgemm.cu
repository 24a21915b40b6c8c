// Complex GEMM on the tensor cores (tcgen05, BF16 operands split in two,
// FP32 accumulation in tensor memory):
//
//   D[m][n] = sum_k A[m][k] B[k][n]      (complex64 in and out)
//
// Real embedding: per chunk of kTK complex k, the real K axis holds the real
// parts (first kTK) and then the imaginary parts of A; the real N axis holds
// re / im of every complex column (interleaved, so that a row of D in tensor
// memory is a complex64 row):
//   A_r[m][k']      = Re A[m][k']           A_r[m][kTK + k'] = Im A[m][k']
//   B_r[2n][k']     = Re B[k'][n]           B_r[2n][kTK + k'] = -Im B[k'][n]
//   B_r[2n+1][k']   = Im B[k'][n]           B_r[2n+1][kTK + k'] = Re B[k'][n]
// so that D_r = A_r B_r^T has D_r[m][2n] = Re D[m][n], D_r[m][2n+1] = Im D[m][n].
// Split BF16: x = hi + lo with hi = bf16(x), lo = bf16(x - hi); the product
// is taken as hi*hi + hi*lo + lo*hi (the lo*lo term, ~2^-16 relative, is
// dropped), which keeps about 16 mantissa bits of every product.
//
// A tile is 128 complex rows (the 128 TMEM lanes) x 128 complex columns
// (256 FP32 TMEM columns); K is consumed in chunks of 32 complex values
// (64 real = 4 MMAs of K = 16 per split term).  Two CTAs of 256 threads per
// SM (the operand tiles take 96 KB of shared memory and 256 TMEM columns per
// CTA), so that one CTA's operand loads overlap the other's MMAs; tiles are
// taken from a job list in a persistent loop.  Used by the weighted apply (the
// frequency contraction of eq. product) and exposed for testing as
// tdbem_zgemm.
#include <cuda_bf16.h>

#include "internal.h"
#include "kernels.h"
#include "tc.cuh"

namespace {

constexpr int kTM = 128;                       // complex rows per tile
constexpr int kTN = 128;                       // complex columns per tile
constexpr int kTK = 32;                        // complex K per chunk
constexpr int kKS = 2 * kTK / 16;              // MMA K-steps (16 real K each) per chunk
constexpr int kThreads = 256;
constexpr int kABytes = kTM * 2 * kTK * 2;     // one split part of A: 16 KB
constexpr int kBBytes = 2 * kTN * 2 * kTK * 2; // one split part of B: 32 KB
constexpr int kSmemBytes = 2 * kABytes + 2 * kBBytes + 1024 + 64;
constexpr uint32_t kTmemCols = 256;
constexpr uint32_t kMaxPolls = 1u << 24;  // default poll limit of a tensor-core wait

struct SplitPack {
    uint4 hi, lo;
};
// 8 real values -> 8 BF16 hi parts and 8 BF16 lo parts (16 bytes each)
TD_D SplitPack split8(const float *v) {
    __nv_bfloat16 h[8], l[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        h[e] = __float2bfloat16_rn(v[e]);
        l[e] = __float2bfloat16_rn(v[e] - __bfloat162float(h[e]));
    }
    SplitPack p;
    p.hi = *reinterpret_cast<const uint4 *>(h);
    p.lo = *reinterpret_cast<const uint4 *>(l);
    return p;
}

// Dense operands (tdbem_zgemm): A [M][K] lda, B [K][N] ldb, D [M][N] ldd.
struct DenseOps {
    const c32 *A, *B;
    c32 *D;
    int64_t lda, ldb, ldd;
    int M, N;
    // 8 consecutive k of row m of A / column n of B; entries k >= kend are 0
    TD_D void a8(const ZJob &, int m, int k, int kend, c32 *x) const {
        const c32 *p = A + (int64_t)m * lda;
#pragma unroll
        for (int e = 0; e < 8; ++e) x[e] = k + e < kend ? p[k + e] : c32{0.f, 0.f};
    }
    TD_D void b8(const ZJob &, int k, int kend, int n, c32 *x) const {
#pragma unroll
        for (int e = 0; e < 8; ++e) x[e] = k + e < kend ? B[(int64_t)(k + e) * ldb + n] : c32{0.f, 0.f};
    }
    TD_D int rows(const ZJob &j) const { return min(kTM, M - j.m0); }
    TD_D int cols(const ZJob &j) const { return min(kTN, N - j.n0); }
    TD_D c32 *drow(const ZJob &, int m) const { return D + (int64_t)m * ldd; }
    TD_D void krange(const ZJob &, int K, int &kb, int &ke) const {
        kb = 0;
        ke = K;
    }
};

// Frequency contraction of the apply: rows (block b, term d, half p) of a
// column-cluster group g, columns (j, c) of W[l][perm_c[J0 + j]][c].
//   A[(b,d,p)][l] = f_d(l) if l belongs to half p (p = 1: conjugate half,
//                   coefficient conj(f_d[u])), else 0
//   Z[(b,d,p)][(j,c)] = sum_l A[(b,d,p)][l] W[l][J0 + j][c]
// The rows of a group are ordered half 0 then half 1, and a tile of one half
// contracts over that half's frequencies only (the other half's coefficients
// are zero).  Both operands come packed (td_launch_pack_fibres / _weights):
// the 8 frequencies of a load item are 64 contiguous bytes, read as four
// 16-byte loads; the zero padding of each half covers the last chunk.
struct ApplyOps {
    const ZGroup *groups;
    const c32 *Fp;        // packed coefficient rows, stride FW
    const c32 *Wk;        // packed weights, stride WS
    c32 *Z;
    int FW, WS, hoff1, nq0, nq1, nrhs;
    TD_D static void load8(const c32 *p, c32 *x) {
        const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float4 v = q[e];
            x[2 * e] = c32{v.x, v.y};
            x[2 * e + 1] = c32{v.z, v.w};
        }
    }
    TD_D void a8(const ZJob &j, int m, int k, int, c32 *x) const {
        load8(Fp + (int64_t)(groups[j.g].row0 + m) * FW + k, x);
    }
    TD_D void b8(const ZJob &j, int k, int, int n, c32 *x) const {
        const ZGroup &g = groups[j.g];
        load8(Wk + ((int64_t)g.J0 * nrhs + n) * WS + (j.half == 2 ? hoff1 : 0) + k, x);
    }
    TD_D int rows(const ZJob &j) const { return min(kTM, (j.half == 1 ? groups[j.g].Mh : groups[j.g].M) - j.m0); }
    TD_D int cols(const ZJob &j) const { return min(kTN, groups[j.g].L - j.n0); }
    TD_D c32 *drow(const ZJob &j, int m) const {
        const ZGroup &g = groups[j.g];
        return Z + g.zoff + (int64_t)m * g.L;
    }
    // the frequencies of the tile's half, in packed (local) numbering
    TD_D void krange(const ZJob &j, int, int &kb, int &ke) const {
        kb = 0;
        ke = j.half == 2 ? nq1 : nq0;
    }
};

template <class Ops>
__global__ void __launch_bounds__(kThreads, 2) k_zgemm(Ops ops, const ZJob *jobs, int njobs, int K, int *err,
                                                        uint32_t max_polls) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // 1024-byte aligned operand region
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *Ah = base, *Al = base + kABytes, *Bh = base + 2 * kABytes, *Bl = Bh + kBBytes;
    uint64_t *bar = reinterpret_cast<uint64_t *>(Bl + kBBytes);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) tmem_alloc(tslot, kTmemCols);
    if (tid == 0) mbar_init(bar, 1);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t idesc = idesc_bf16_f32(kTM, 2 * kTN);
    uint32_t phase = 0;
    bool failed = false;
    for (int jb = blockIdx.x; jb < njobs && !failed; jb += gridDim.x) {
        const ZJob job = jobs[jb];
        const int mr = ops.rows(job), nc = ops.cols(job);
        int kb, ke;
        ops.krange(job, K, kb, ke);
        for (int k0 = kb; k0 < ke && !failed; k0 += kTK) {
            const int kc = min(kTK, ke - k0);
            // ---- A tile.  Real item it -> (kstep s, row group g, core matrix kh, row
            // rr), its 16 bytes at byte offset 16 * it of the canonical layout.  One
            // complex item (8 consecutive complex k of one row) gives the real item of
            // its real parts (real k < kTK) and the one of its imaginary parts (real
            // k + kTK, kTK / 16 ksteps = kTK * 16 items further): each value is loaded
            // once.  Two complex items per thread and pass, loads issued first.
            constexpr int kAItems = kTM * kTK / 8, kAImag = kTK * 16;
            for (int c0 = tid; c0 < kAItems; c0 += 2 * kThreads) {
                c32 x[2][8];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int ci = c0 + u * kThreads;
                    const int rr = ci & 7, kh = (ci >> 3) & 1, g = (ci >> 4) & 15, sk = ci >> 8;
                    const int r = g * 8 + rr, k = sk * 16 + kh * 8;  // complex k of the first element
                    if (ci < kAItems && r < mr) {
                        ops.a8(job, job.m0 + r, k0 + k, k0 + kc, x[u]);
                    } else {
#pragma unroll
                        for (int e = 0; e < 8; ++e) x[u][e] = c32{0.f, 0.f};
                    }
                }
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int ci = c0 + u * kThreads;
                    if (ci >= kAItems) continue;
                    float v[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) v[e] = x[u][e].x;
                    SplitPack p = split8(v);
                    *reinterpret_cast<uint4 *>(Ah + 16 * ci) = p.hi;
                    *reinterpret_cast<uint4 *>(Al + 16 * ci) = p.lo;
#pragma unroll
                    for (int e = 0; e < 8; ++e) v[e] = x[u][e].y;
                    p = split8(v);
                    *reinterpret_cast<uint4 *>(Ah + 16 * (ci + kAImag)) = p.hi;
                    *reinterpret_cast<uint4 *>(Al + 16 * (ci + kAImag)) = p.lo;
                }
            }
            // ---- B tile: 2 kTN real rows (re / im row of every complex column).
            // Real item it -> (kstep s = it >> 9, row group g, kh, row rr).  One
            // complex item (8 consecutive k of complex column n) gives four real
            // items: rows 2n / 2n + 1 (rr = 2 (n & 3), + 1) in the first K half
            // (Re B, Im B) and in the second (-Im B, Re B, kTK / 16 ksteps further).
            constexpr int kBItems = kTN * kTK / 8, kBSecond = kTK * 32;
            for (int c0 = tid; c0 < kBItems; c0 += 2 * kThreads) {
                c32 x[2][8];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int ci = c0 + u * kThreads;
                    const int n4 = ci & 3, kh = (ci >> 2) & 1, g = (ci >> 3) & 31, sk = ci >> 8;
                    const int n = g * 4 + n4, k = sk * 16 + kh * 8;
                    if (ci < kBItems && n < nc) {
                        ops.b8(job, k0 + k, k0 + kc, job.n0 + n, x[u]);
                    } else {
#pragma unroll
                        for (int e = 0; e < 8; ++e) x[u][e] = c32{0.f, 0.f};
                    }
                }
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int ci = c0 + u * kThreads;
                    if (ci >= kBItems) continue;
                    const int n4 = ci & 3, kh = (ci >> 2) & 1, g = (ci >> 3) & 31, sk = ci >> 8;
                    const int it = sk * 512 + g * 16 + kh * 8 + 2 * n4;
                    float v[8];
                    SplitPack p;
#pragma unroll
                    for (int e = 0; e < 8; ++e) v[e] = x[u][e].x;  // row 2n, first half; row 2n + 1, second
                    p = split8(v);
                    *reinterpret_cast<uint4 *>(Bh + 16 * it) = p.hi;
                    *reinterpret_cast<uint4 *>(Bl + 16 * it) = p.lo;
                    *reinterpret_cast<uint4 *>(Bh + 16 * (it + kBSecond + 1)) = p.hi;
                    *reinterpret_cast<uint4 *>(Bl + 16 * (it + kBSecond + 1)) = p.lo;
#pragma unroll
                    for (int e = 0; e < 8; ++e) v[e] = x[u][e].y;  // row 2n + 1, first half
                    p = split8(v);
                    *reinterpret_cast<uint4 *>(Bh + 16 * (it + 1)) = p.hi;
                    *reinterpret_cast<uint4 *>(Bl + 16 * (it + 1)) = p.lo;
#pragma unroll
                    for (int e = 0; e < 8; ++e) v[e] = -x[u][e].y;  // row 2n, second half
                    p = split8(v);
                    *reinterpret_cast<uint4 *>(Bh + 16 * (it + kBSecond)) = p.hi;
                    *reinterpret_cast<uint4 *>(Bl + 16 * (it + kBSecond)) = p.lo;
                }
            }
            fence_async_shared();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
                const uint32_t ah = smem_u32(Ah), al = smem_u32(Al), bh = smem_u32(Bh), bl = smem_u32(Bl);
#pragma unroll 1
                for (int s = 0; s < kKS; ++s) {
                    const uint64_t dah = smem_desc(ah + s * 4096, 128, 256), dal = smem_desc(al + s * 4096, 128, 256);
                    const uint64_t dbh = smem_desc(bh + s * 8192, 128, 256), dbl = smem_desc(bl + s * 8192, 128, 256);
                    tc_mma_bf16(tmem, dah, dbh, idesc, (k0 > kb || s > 0) ? 1u : 0u);
                    tc_mma_bf16(tmem, dah, dbl, idesc, 1u);
                    tc_mma_bf16(tmem, dal, dbh, idesc, 1u);
                }
                tc_commit(bar);
            }
            // a limit below the default counts non-blocking tests (a blocking
            // try_wait may itself wait until the MMAs are done)
            const bool ok = max_polls < kMaxPolls ? mbar_test(bar, phase, max_polls) : mbar_wait(bar, phase, max_polls);
            phase ^= 1u;
            failed = __syncthreads_or(!ok) != 0;
            tc_fence_after();
        }
        if (failed) break;
        // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 (tile rows),
        // real columns 128 (w / 4) .. +127
        const int q = warp & 3, h = warp >> 2;
        const int r = 32 * q + lane;
        c32 *drow = r < mr ? ops.drow(job, job.m0 + r) : nullptr;
#pragma unroll 1
        for (int c16 = 0; c16 < 8; ++c16) {
            const int col = 128 * h + 16 * c16;  // real column of the first value
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)col, v);
            const int n0 = col >> 1;  // complex column
            if (drow) {
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    if (n0 + e < nc) drow[job.n0 + n0 + e] = c32{v[2 * e], v[2 * e + 1]};
            }
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }
    if (failed && tid == 0) atomicOr(err, TD_DEV_TIMEOUT);
    if (failed) mbar_wait(bar, phase ^ 1u, kMaxPolls);  // let a late MMA group finish before freeing TMEM
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

template <class Ops>
int launch_zgemm(cudaStream_t st, const Ops &ops, const ZJob *jobs, int njobs, int K, int *err, uint32_t max_polls,
                 int num_sms) {
    if (njobs == 0) return 0;
    cudaError_t e = cudaFuncSetAttribute(k_zgemm<Ops>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return (int)e;
    const int grid = std::min(njobs, 2 * num_sms);  // two CTAs per SM
    k_zgemm<Ops><<<grid, kThreads, kSmemBytes, st>>>(ops, jobs, njobs, K, err, max_polls ? max_polls : kMaxPolls);
    return (int)cudaGetLastError();
}

}  // namespace

int td_launch_zgemm_dense(cudaStream_t st, const c32 *A, int64_t lda, const c32 *B, int64_t ldb, c32 *D, int64_t ldd,
                          int M, int N, int K, const ZJob *jobs, int njobs, int *err, uint32_t max_polls,
                          int num_sms) {
    DenseOps ops{A, B, D, lda, ldb, ldd, M, N};
    return launch_zgemm(st, ops, jobs, njobs, K, err, max_polls, num_sms);
}

int td_launch_zgemm_apply(cudaStream_t st, const ZGroup *groups, const c32 *Fp, int FW, const c32 *Wk, int WS,
                          int hoff1, int nq0, int nq1, c32 *Z, int nrhs, const ZJob *jobs, int njobs, int *err,
                          uint32_t max_polls, int num_sms) {
    ApplyOps ops{groups, Fp, Wk, Z, FW, WS, hoff1, nq0, nq1, nrhs};
    return launch_zgemm(st, ops, jobs, njobs, nq0 + nq1, err, max_polls, num_sms);
}

namespace {
__global__ void k_pack_fibres(const int2 *rowtab, int64_t nrows, const int *qmap, const int *lperm, int nq0,
                              int nq1, const c32 *fib, int Nu, c32 *Fp, int FW) {
    const int64_t n = nrows * FW;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / FW;
        const int k = (int)(e - r * FW);
        const int2 rt = rowtab[r];
        const int p = rt.y & 1, d = rt.y >> 1;
        c32 v = {0.f, 0.f};
        if (k < (p ? nq1 : nq0)) {
            const int mp = qmap[lperm[(p ? nq0 : 0) + k]];  // > 0 in half 0, < 0 in half 1
            const c32 f = fib[((int64_t)rt.x * Nu + d) * Nu + (mp > 0 ? mp - 1 : -mp - 1)];
            v = p ? cconj(f) : f;
        }
        Fp[e] = v;
    }
}

// 32 frequencies x 32 columns (j', c) per tile, transposed through shared
// memory: W rows read and Wk rows written 256 bytes at a time.
__global__ void __launch_bounds__(256) k_pack_weights(const c32 *W, const int *perm_c, const int *lperm,
                                                      int64_t ncols, int nrhs, int nq0, int nq1, int KW0, int KW1,
                                                      c32 *Wk) {
    __shared__ c32 tile[32][33];
    const int64_t ncolr = ncols * nrhs;
    const int WS = KW0 + KW1, nkt0 = KW0 / 32, nkt = nkt0 + KW1 / 32;
    const int64_t nnt = (ncolr + 31) / 32;
    for (int64_t job = blockIdx.x; job < nnt * nkt; job += gridDim.x) {
        const int kt = (int)(job % nkt);
        const int64_t nt = job / nkt;
        const int p = kt >= nkt0 ? 1 : 0;
        const int k0 = (p ? kt - nkt0 : kt) * 32, nqp = p ? nq1 : nq0, kb = p ? nq0 : 0, hoff = p ? KW0 : 0;
        __syncthreads();
        for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
            const int kk = e >> 5, nn = e & 31;
            const int64_t n = nt * 32 + nn;
            const int k = k0 + kk;
            c32 v = {0.f, 0.f};
            if (n < ncolr && k < nqp) {
                const int64_t jp = n / nrhs;
                const int c = (int)(n - jp * nrhs);
                v = W[((int64_t)lperm[kb + k] * ncols + perm_c[jp]) * nrhs + c];
            }
            tile[kk][nn] = v;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
            const int nn = e >> 5, kk = e & 31;
            const int64_t n = nt * 32 + nn;
            if (n < ncolr) Wk[n * WS + hoff + k0 + kk] = tile[kk][nn];
        }
    }
}
}  // namespace

int td_launch_pack_fibres(cudaStream_t st, const int2 *rowtab, int64_t nrows, const int *qmap, const int *lperm,
                          int nq0, int nq1, const c32 *fib, int Nu, c32 *Fp, int FW, int num_sms) {
    if (nrows == 0) return 0;
    const int grid = (int)std::min<int64_t>((nrows * FW + 255) / 256, (int64_t)num_sms * 16);
    k_pack_fibres<<<grid, 256, 0, st>>>(rowtab, nrows, qmap, lperm, nq0, nq1, fib, Nu, Fp, FW);
    return (int)cudaGetLastError();
}

int td_launch_pack_weights(cudaStream_t st, const c32 *W, const int *perm_c, const int *lperm, int64_t ncols,
                           int nrhs, int nq0, int nq1, int KW0, int KW1, c32 *Wk, int num_sms) {
    const int64_t jobs = ((ncols * nrhs + 31) / 32) * ((KW0 + KW1) / 32);
    if (jobs == 0) return 0;
    const int grid = (int)std::min<int64_t>(jobs, (int64_t)num_sms * 8);
    k_pack_weights<<<grid, 256, 0, st>>>(W, perm_c, lperm, ncols, nrhs, nq0, nq1, KW0, KW1, Wk);
    return (int)cudaGetLastError();
}

int td_zgemm_tile_rows() { return kTM; }
int td_zgemm_tile_cols() { return kTN; }
