/*
 * Oracle (test infrastructure only): the rank-predictor MLP in FP64.
 *
 * The network is not part of the paper; it is the learned presizing step of
 * the GPU library (6 features -> 64 -> 64 -> 16 rank bins, GELU hidden
 * activations, softmax cross-entropy, Adam).  This plain restatement is used
 * to check the library's forward, backward and optimiser kernels; it is itself
 * pinned against central finite differences.
 *
 * GELU(x) = x Phi(x) = x (1 + erf(x / sqrt 2)) / 2,
 * GELU'(x) = Phi(x) + x phi(x), phi(x) = exp(-x^2/2) / sqrt(2 pi).
 * Adam: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 *       p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
 */
#include "orc.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

enum { NIN = 6, NH = 64, NOUT = 16 };
enum {
    OFF_W1 = 0,
    OFF_B1 = OFF_W1 + NH * NIN,
    OFF_W2 = OFF_B1 + NH,
    OFF_B2 = OFF_W2 + NH * NH,
    OFF_W3 = OFF_B2 + NH,
    OFF_B3 = OFF_W3 + NOUT * NH,
    NPARAM = OFF_B3 + NOUT
};

int orc_mlp_nparams(void) { return NPARAM; }

static double gelu(double x) { return 0.5 * x * (1.0 + erf(x / sqrt(2.0))); }
static double gelu_d(double x) {
    return 0.5 * (1.0 + erf(x / sqrt(2.0))) + x * exp(-0.5 * x * x) / sqrt(2.0 * acos(-1.0));
}

/* forward pass of one sample; keeps pre-activations for the backward pass */
static void fwd1(const double *P, const double *x, double *z1, double *h1, double *z2, double *h2,
                 double *lg) {
    for (int o = 0; o < NH; ++o) {
        double a = P[OFF_B1 + o];
        for (int i = 0; i < NIN; ++i) a += P[OFF_W1 + o * NIN + i] * x[i];
        z1[o] = a;
        h1[o] = gelu(a);
    }
    for (int o = 0; o < NH; ++o) {
        double a = P[OFF_B2 + o];
        for (int i = 0; i < NH; ++i) a += P[OFF_W2 + o * NH + i] * h1[i];
        z2[o] = a;
        h2[o] = gelu(a);
    }
    for (int o = 0; o < NOUT; ++o) {
        double a = P[OFF_B3 + o];
        for (int i = 0; i < NH; ++i) a += P[OFF_W3 + o * NH + i] * h2[i];
        lg[o] = a;
    }
}

void orc_mlp_forward(const double *P, const double *x, int64_t n, double *logits) {
    double z1[NH], h1[NH], z2[NH], h2[NH];
    for (int64_t k = 0; k < n; ++k) fwd1(P, x + NIN * k, z1, h1, z2, h2, logits + NOUT * k);
}

double orc_mlp_loss_grad(const double *P, const double *x, const int32_t *label, int64_t n,
                         double *G) {
    double z1[NH], h1[NH], z2[NH], h2[NH], lg[NOUT], p[NOUT], d3[NOUT], d2[NH], d1[NH];
    if (G) memset(G, 0, sizeof(double) * NPARAM);
    double loss = 0.0;
    for (int64_t k = 0; k < n; ++k) {
        const double *xi = x + NIN * k;
        fwd1(P, xi, z1, h1, z2, h2, lg);
        double mx = lg[0];
        for (int o = 1; o < NOUT; ++o) mx = lg[o] > mx ? lg[o] : mx;
        double se = 0.0;
        for (int o = 0; o < NOUT; ++o) {
            p[o] = exp(lg[o] - mx);
            se += p[o];
        }
        for (int o = 0; o < NOUT; ++o) p[o] /= se;
        loss += -(lg[label[k]] - mx - log(se));
        if (!G) continue;
        /* d loss / d logits = softmax - onehot, averaged over n */
        for (int o = 0; o < NOUT; ++o) d3[o] = (p[o] - (o == label[k] ? 1.0 : 0.0)) / (double)n;
        for (int o = 0; o < NOUT; ++o) {
            G[OFF_B3 + o] += d3[o];
            for (int i = 0; i < NH; ++i) G[OFF_W3 + o * NH + i] += d3[o] * h2[i];
        }
        for (int i = 0; i < NH; ++i) {
            double a = 0.0;
            for (int o = 0; o < NOUT; ++o) a += P[OFF_W3 + o * NH + i] * d3[o];
            d2[i] = a * gelu_d(z2[i]);
        }
        for (int o = 0; o < NH; ++o) {
            G[OFF_B2 + o] += d2[o];
            for (int i = 0; i < NH; ++i) G[OFF_W2 + o * NH + i] += d2[o] * h1[i];
        }
        for (int i = 0; i < NH; ++i) {
            double a = 0.0;
            for (int o = 0; o < NH; ++o) a += P[OFF_W2 + o * NH + i] * d2[o];
            d1[i] = a * gelu_d(z1[i]);
        }
        for (int o = 0; o < NH; ++o) {
            G[OFF_B1 + o] += d1[o];
            for (int i = 0; i < NIN; ++i) G[OFF_W1 + o * NIN + i] += d1[o] * xi[i];
        }
    }
    return loss / (double)n;
}

void orc_adam_step(double *P, const double *G, double *m, double *v, int64_t np, double lr,
                   double b1, double b2, double eps, int t) {
    double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
    for (int64_t k = 0; k < np; ++k) {
        m[k] = b1 * m[k] + (1.0 - b1) * G[k];
        v[k] = b2 * v[k] + (1.0 - b2) * G[k] * G[k];
        P[k] -= lr * (m[k] / c1) / (sqrt(v[k] / c2) + eps);
    }
}
