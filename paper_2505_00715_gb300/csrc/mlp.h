// Rank-predictor MLP kernels (k_mlp.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define TD_MLP_NPARAMS (6 * 64 + 64 + 64 * 64 + 64 + 16 * 64 + 16)
#define TD_MLP_NBINS 16
#define TD_MLP_NFEAT 6

int td_mlp_init(cudaStream_t st, float *P, uint64_t seed);
int td_mlp_to_bf16(cudaStream_t st, const float *P, void *Pb);
int td_mlp_predict(cudaStream_t st, const void *Pb, const float *x, int64_t n, int *bins, float *logits,
                   int num_sms);
int td_mlp_presize(cudaStream_t st, const void *Pb, const float *bfeat, const float *ffeat, int nfar, int Nu,
                   const int *far, const int *len, int kcap, int *kpred, int *ks, float *cost, int num_sms);
int td_mlp_grad(cudaStream_t st, const float *P, const float *x, const int *label, int64_t n, float *grad,
                float *loss, int num_sms);
int td_mlp_adam(cudaStream_t st, float *P, const float *G, float *m, float *v, float lr, float b1, float b2,
                float eps, int t);
