// Rank-predictor MLP: 6 features -> 64 -> 64 -> 16 rank bins, GELU hidden
// activations (x Phi(x), erf form), softmax cross-entropy, Adam.
//
// Parameter layout (FP32 master copy, same order for gradients):
//   W1[64][6] b1[64] W2[64][64] b2[64] W3[16][64] b3[16]
// Inference uses a BF16 copy of the weights with FP32 accumulation; training
// runs forward and backward in FP32 from the master copy.  One thread per
// sample; weights live in shared memory; gradients are reduced per CTA in
// shared memory and then added to the global gradient.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"

#include "internal.h"
#include "mlp.h"

namespace {

constexpr int NIN = 6, NH = 64, NOUT = 16;
constexpr int OW1 = 0, OB1 = OW1 + NH * NIN, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH,
              OB3 = OW3 + NOUT * NH, NP = OB3 + NOUT;
static_assert(NP == TD_MLP_NPARAMS, "parameter count");

TD_D float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
TD_D float gelu_d(float x) {
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

__global__ void k_to_bf16(const float *p, __nv_bfloat16 *q, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) q[i] = __float2bfloat16(p[i]);
}

// Forward pass of one sample from weights in shared memory; returns the arg-max bin.
TD_D int mlp_forward_bin(const float *w, const float *in, float *logits) {
    float h1[NH], h2[NH];
    for (int o = 0; o < NH; ++o) {
        float a = w[OB1 + o];
#pragma unroll
        for (int i = 0; i < NIN; ++i) a = fmaf(w[OW1 + o * NIN + i], in[i], a);
        h1[o] = gelu(a);
    }
    for (int o = 0; o < NH; ++o) {
        float a = w[OB2 + o];
        for (int i = 0; i < NH; ++i) a = fmaf(w[OW2 + o * NH + i], h1[i], a);
        h2[o] = gelu(a);
    }
    int best = 0;
    float bv = -INFINITY;
    for (int o = 0; o < NOUT; ++o) {
        float a = w[OB3 + o];
        for (int i = 0; i < NH; ++i) a = fmaf(w[OW3 + o * NH + i], h2[i], a);
        if (logits) logits[o] = a;
        if (a > bv) {
            bv = a;
            best = o;
        }
    }
    return best;
}

// lower edges of the rank bins (the first ACA steps the compressor may run unchecked)
__constant__ int c_bin_lower[NOUT] = {1, 2, 3, 4, 5, 7, 9, 11, 13, 17, 21, 25, 33, 41, 49, 65};

// Presizing of the far blocks: sample s = (far block q, unique frequency u);
// the two frequency features are formed here from the block distance and
// s/c.  Writes the predicted first trip count kp to kpred[far[q] Nu + u],
// adds min(kp, kcap) to ks[q] (the block's predicted face ranks summed over
// the frequencies) and len[q] kp^2 to cost[q].
__global__ void __launch_bounds__(128) k_mlp_presize(const __nv_bfloat16 *P, const float *bfeat, const float *ffeat,
                                                     int nfar, int Nu, const int *far, const int *len, int kcap,
                                                     int *kpred, int *ks, float *cost) {
    __shared__ float w[NP];
    for (int i = threadIdx.x; i < NP; i += blockDim.x) w[i] = __bfloat162float(P[i]);
    __syncthreads();
    const int64_t n = (int64_t)nfar * Nu;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const int q = (int)(s / Nu), u = (int)(s - (s / Nu) * Nu);
        const float *b = bfeat + (int64_t)q * 5;
        float in[NIN] = {b[0], b[1], b[2], b[3], log1pf(fmaxf(0.f, ffeat[2 * u]) * b[4]),
                         log1pf(ffeat[2 * u + 1] * b[4])};
        const int kp = c_bin_lower[mlp_forward_bin(w, in, nullptr)];
        kpred[(int64_t)far[q] * Nu + u] = kp;
        atomicAdd(&ks[q], min(kp, kcap));
        atomicAdd(&cost[q], (float)len[q] * (float)kp * (float)kp);
    }
}

// Inference: bins[n] = argmax logits (BF16 weights, FP32 accumulation).
__global__ void __launch_bounds__(128) k_mlp_predict(const __nv_bfloat16 *P, const float *x, int64_t n,
                                                     int *bins, float *logits) {
    __shared__ float w[NP];
    for (int i = threadIdx.x; i < NP; i += blockDim.x) w[i] = __bfloat162float(P[i]);
    __syncthreads();
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        float in[NIN], h1[NH], h2[NH];
#pragma unroll
        for (int i = 0; i < NIN; ++i) in[i] = x[s * NIN + i];
        for (int o = 0; o < NH; ++o) {
            float a = w[OB1 + o];
#pragma unroll
            for (int i = 0; i < NIN; ++i) a = fmaf(w[OW1 + o * NIN + i], in[i], a);
            h1[o] = gelu(a);
        }
        for (int o = 0; o < NH; ++o) {
            float a = w[OB2 + o];
            for (int i = 0; i < NH; ++i) a = fmaf(w[OW2 + o * NH + i], h1[i], a);
            h2[o] = gelu(a);
        }
        int best = 0;
        float bv = -INFINITY;
        for (int o = 0; o < NOUT; ++o) {
            float a = w[OB3 + o];
            for (int i = 0; i < NH; ++i) a = fmaf(w[OW3 + o * NH + i], h2[i], a);
            if (logits) logits[s * NOUT + o] = a;
            if (a > bv) {
                bv = a;
                best = o;
            }
        }
        if (bins) bins[s] = best;
    }
}

// Mean softmax cross-entropy and its gradient (FP32).  grad and loss must be
// zeroed by the caller; every CTA adds its partial sums.  Per-sample
// contributions are summed over the warp with shuffles before one shared
// atomic per warp, then once per CTA into global memory.
TD_D float wsum(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(128) k_mlp_grad(const float *P, const float *x, const int *label, int64_t n,
                                                  float *grad, float *loss) {
    __shared__ float w[NP];
    __shared__ float g[NP];
    __shared__ float sl;
    for (int i = threadIdx.x; i < NP; i += blockDim.x) {
        w[i] = P[i];
        g[i] = 0.0f;
    }
    if (threadIdx.x == 0) sl = 0.0f;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const float inv_n = 1.0f / (float)n;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t iters = (n + stride - 1) / stride;
    for (int64_t it = 0; it < iters; ++it) {
        const int64_t s = it * stride + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
        const bool valid = s < n;
        float in[NIN], z1[NH], h1[NH], z2[NH], h2[NH], lg[NOUT];
#pragma unroll
        for (int i = 0; i < NIN; ++i) in[i] = valid ? x[s * NIN + i] : 0.0f;
        for (int o = 0; o < NH; ++o) {
            float a = w[OB1 + o];
#pragma unroll
            for (int i = 0; i < NIN; ++i) a = fmaf(w[OW1 + o * NIN + i], in[i], a);
            z1[o] = a;
            h1[o] = gelu(a);
        }
        for (int o = 0; o < NH; ++o) {
            float a = w[OB2 + o];
            for (int i = 0; i < NH; ++i) a = fmaf(w[OW2 + o * NH + i], h1[i], a);
            z2[o] = a;
            h2[o] = gelu(a);
        }
        float mx = -INFINITY;
        for (int o = 0; o < NOUT; ++o) {
            float a = w[OB3 + o];
            for (int i = 0; i < NH; ++i) a = fmaf(w[OW3 + o * NH + i], h2[i], a);
            lg[o] = a;
            mx = fmaxf(mx, a);
        }
        float se = 0.0f;
        for (int o = 0; o < NOUT; ++o) se += expf(lg[o] - mx);
        const int lab = valid ? label[s] : 0;
        const float ls = wsum(valid ? (logf(se) + mx - lg[lab]) * inv_n : 0.0f);
        if (lane == 0) atomicAdd(&sl, ls);
        // backward: d loss / d logits = (softmax - onehot) / n
        float d3[NOUT];
        for (int o = 0; o < NOUT; ++o) d3[o] = valid ? (expf(lg[o] - mx) / se - (o == lab ? 1.0f : 0.0f)) * inv_n : 0.0f;
        for (int o = 0; o < NOUT; ++o) {
            const float b = wsum(d3[o]);
            if (lane == 0) atomicAdd(&g[OB3 + o], b);
            for (int i = 0; i < NH; ++i) {
                const float v = wsum(d3[o] * h2[i]);
                if (lane == 0) atomicAdd(&g[OW3 + o * NH + i], v);
            }
        }
        float d2[NH];
        for (int i = 0; i < NH; ++i) {
            float a = 0.0f;
            for (int o = 0; o < NOUT; ++o) a = fmaf(w[OW3 + o * NH + i], d3[o], a);
            d2[i] = a * gelu_d(z2[i]);
        }
        for (int o = 0; o < NH; ++o) {
            const float b = wsum(d2[o]);
            if (lane == 0) atomicAdd(&g[OB2 + o], b);
            for (int i = 0; i < NH; ++i) {
                const float v = wsum(d2[o] * h1[i]);
                if (lane == 0) atomicAdd(&g[OW2 + o * NH + i], v);
            }
        }
        for (int i = 0; i < NH; ++i) {
            float a = 0.0f;
            for (int o = 0; o < NH; ++o) a = fmaf(w[OW2 + o * NH + i], d2[o], a);
            const float d1 = a * gelu_d(z1[i]);
            const float b = wsum(d1);
            if (lane == 0) atomicAdd(&g[OB1 + i], b);
#pragma unroll
            for (int k = 0; k < NIN; ++k) {
                const float v = wsum(d1 * in[k]);
                if (lane == 0) atomicAdd(&g[OW1 + i * NIN + k], v);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NP; i += blockDim.x) atomicAdd(&grad[i], g[i]);
    if (threadIdx.x == 0) atomicAdd(loss, sl);
}

// Adam: m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
// p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
__global__ void k_adam(float *P, const float *G, float *m, float *v, int n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = G[i];
    const float mi = b1 * m[i] + (1.0f - b1) * g;
    const float vi = b2 * v[i] + (1.0f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Seeded initialisation (counter-based hash -> uniform in [-a, a] with a =
// sqrt(6 / fan_in) per layer, biases zero).
TD_D uint32_t mix32(uint64_t z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return (uint32_t)((z ^ (z >> 31)) >> 32);
}
__global__ void k_mlp_init(float *P, uint64_t seed) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NP) return;
    float fan = 0.0f;
    if (i < OB1) fan = NIN;
    else if (i >= OW2 && i < OB2) fan = NH;
    else if (i >= OW3 && i < OB3) fan = NH;
    if (fan == 0.0f) {
        P[i] = 0.0f;
        return;
    }
    const float u = (mix32(seed * 1000003ull + (uint64_t)i) + 0.5f) * (1.0f / 4294967296.0f);
    P[i] = (2.0f * u - 1.0f) * sqrtf(6.0f / fan);
}

}  // namespace

int td_mlp_init(cudaStream_t st, float *P, uint64_t seed) {
    k_mlp_init<<<(NP + 255) / 256, 256, 0, st>>>(P, seed);
    return (int)cudaGetLastError();
}

int td_mlp_to_bf16(cudaStream_t st, const float *P, void *Pb) {
    k_to_bf16<<<(NP + 255) / 256, 256, 0, st>>>(P, (__nv_bfloat16 *)Pb, NP);
    return (int)cudaGetLastError();
}

int td_mlp_predict(cudaStream_t st, const void *Pb, const float *x, int64_t n, int *bins, float *logits,
                   int num_sms) {
    if (n <= 0) return 0;
    const int grid = (int)std::min<int64_t>((n + 127) / 128, (int64_t)num_sms * 8);
    k_mlp_predict<<<grid, 128, 0, st>>>((const __nv_bfloat16 *)Pb, x, n, bins, logits);
    return (int)cudaGetLastError();
}

int td_mlp_presize(cudaStream_t st, const void *Pb, const float *bfeat, const float *ffeat, int nfar, int Nu,
                   const int *far, const int *len, int kcap, int *kpred, int *ks, float *cost, int num_sms) {
    if (nfar <= 0) return 0;
    const int64_t n = (int64_t)nfar * Nu;
    const int grid = (int)std::min<int64_t>((n + 127) / 128, (int64_t)num_sms * 8);
    k_mlp_presize<<<grid, 128, 0, st>>>((const __nv_bfloat16 *)Pb, bfeat, ffeat, nfar, Nu, far, len, kcap, kpred, ks,
                                        cost);
    return (int)cudaGetLastError();
}

int td_mlp_grad(cudaStream_t st, const float *P, const float *x, const int *label, int64_t n, float *grad,
                float *loss, int num_sms) {
    cudaMemsetAsync(grad, 0, sizeof(float) * NP, st);
    cudaMemsetAsync(loss, 0, sizeof(float), st);
    if (n <= 0) return (int)cudaGetLastError();
    const int grid = (int)std::min<int64_t>((n + 127) / 128, (int64_t)num_sms * 4);
    k_mlp_grad<<<grid, 128, 0, st>>>(P, x, label, n, grad, loss);
    return (int)cudaGetLastError();
}

int td_mlp_adam(cudaStream_t st, float *P, const float *G, float *m, float *v, float lr, float b1, float b2,
                float eps, int t) {
    const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
    k_adam<<<(NP + 255) / 256, 256, 0, st>>>(P, G, m, v, NP, lr, b1, b2, eps, c1, c2);
    return (int)cudaGetLastError();
}
