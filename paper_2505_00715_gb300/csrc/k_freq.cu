// Frequency sets in FP64 on the device.
//
// BDF2 convolution quadrature: s_k = delta(lambda e^{2 pi i k/N}) / dt with
// delta(z) = (1 - z) + (1 - z)^2 / 2.
//
// Generalised CQ contour (App. A): s_l = gamma(sigma_l),
//   sigma_l = -K + (l - 1/2) 4K / N_Q + i K'/2,
//   gamma(sig)  = (sqrt(2q-1) (1/k + sn)/(1/k - sn) - 1) / (dt_min (q - 1)),
//   gamma'(sig) = sqrt(2q-1) / (dt_min (q - 1)) * 2 cn dn / (k (1/k - sn)^2),
//   k = (q - sqrt(2q-1)) / (q + sqrt(2q-1)), sn/cn/dn and K, K' at parameter
//   m = k^2; weights of the positively oriented Cauchy quadrature
//   w_l = -(4K / N_Q) gamma'(sigma_l) / (2 pi i) (the sigma path runs
//   clockwise).  K by the arithmetic-geometric mean, sn/cn/dn of real
//   argument by the descending Landen sequence, complex argument by the
//   addition formulas with the complementary parameter (Abramowitz-Stegun
//   16.4, 16.21).  The caller passes dt_min / rho (td_gcq_radius), so that
//   the circle through 0 and 2 rho / dt_min encloses every resolvent pole
//   1/(dt lambda_i(A)) of the steps.
#include "common.cuh"
#include "internal.h"

namespace {

__device__ double agm_K(double m) {
    double a = 1.0, b = sqrt(1.0 - m);
    for (int it = 0; it < 64; ++it) {
        if (fabs(a - b) <= 1e-16 * a) break;
        double an = 0.5 * (a + b);
        b = sqrt(a * b);
        a = an;
    }
    return 3.141592653589793238462643383279502884 / (2.0 * a);
}

__device__ void jac_real(double u, double m, double &sn, double &cn, double &dn) {
    if (m < 1e-300) {
        sincos(u, &sn, &cn);
        dn = 1.0;
        return;
    }
    double a[40], c[40];
    a[0] = 1.0;
    c[0] = sqrt(m);
    double b = sqrt(1.0 - m);
    int n = 0;
    while (n < 38 && fabs(c[n]) > 1e-16) {
        double an = 0.5 * (a[n] + b);
        c[n + 1] = 0.5 * (a[n] - b);
        b = sqrt(a[n] * b);
        a[n + 1] = an;
        ++n;
    }
    double phi = ldexp(a[n] * u, n), prev = phi;
    for (int k = n; k >= 1; --k) {
        prev = phi;
        phi = 0.5 * (phi + asin(c[k] * sin(phi) / a[k]));
    }
    sincos(phi, &sn, &cn);
    dn = n >= 1 ? cn / cos(prev - phi) : sqrt(1.0 - m * sn * sn);
}

__global__ void k_bdf2(int N, double dt, double lam, double *s) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    double sn, cs;
    sincospi(2.0 * k / N, &sn, &cs);
    c64 z = {lam * cs, lam * sn};
    c64 om = {1.0 - z.x, -z.y};
    c64 d = om + 0.5 * (om * om);
    s[2 * k] = d.x / dt;
    s[2 * k + 1] = d.y / dt;
}

__global__ void k_gcq(int NQ, double dt_min, double q, double *s, double *w) {
    int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= NQ) return;
    const double r = sqrt(2.0 * q - 1.0);
    const double k = (q - r) / (q + r);
    const double m = k * k;
    const double K = agm_K(m), Kp = agm_K(1.0 - m);
    const double u = -K + (l + 0.5) * 4.0 * K / NQ, v = 0.5 * Kp;
    double s0, c0, d0, s1, c1, d1;
    jac_real(u, m, s0, c0, d0);
    jac_real(v, 1.0 - m, s1, c1, d1);
    const double D = c1 * c1 + m * s0 * s0 * s1 * s1;
    const c64 sn = {s0 * d1 / D, c0 * d0 * s1 * c1 / D};
    const c64 cn = {c0 * c1 / D, -s0 * d0 * s1 * d1 / D};
    const c64 dn = {d0 * c1 * d1 / D, -m * s0 * c0 * s1 / D};
    const double sc = 1.0 / (dt_min * (q - 1.0));
    const c64 ik = {1.0 / k, 0.0};
    const c64 g = sc * (r * cdiv(ik + sn, ik - sn) - c64{1.0, 0.0});
    const c64 den = k * ((ik - sn) * (ik - sn));
    const c64 gp = (sc * r * 2.0) * cdiv(cn * dn, den);
    // -(4K/NQ) gp / (2 pi i) = (4K/NQ) gp * i / (2 pi)
    const double f = 4.0 * K / NQ / (2.0 * 3.141592653589793238462643383279502884);
    s[2 * l] = g.x;
    s[2 * l + 1] = g.y;
    w[2 * l] = -f * gp.y;
    w[2 * l + 1] = f * gp.x;
}

}  // namespace

int td_launch_bdf2(cudaStream_t st, int N, double dt, double lam, double *ds) {
    k_bdf2<<<(N + 127) / 128, 128, 0, st>>>(N, dt, lam, ds);
    return (int)cudaGetLastError();
}

int td_launch_gcq(cudaStream_t st, int NQ, double dt_min, double q, double *ds, double *dw) {
    k_gcq<<<(NQ + 127) / 128, 128, 0, st>>>(NQ, dt_min, q, ds, dw);
    return (int)cudaGetLastError();
}
