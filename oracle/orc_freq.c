/*
 * Oracle (test infrastructure only): frequency sets.
 *
 * BDF2 convolution quadrature (Lubich): the Laplace-domain points are
 * s_k = delta(zeta_k)/dt, zeta_k = lambda e^{2 pi i k/N}, with the BDF2
 * generating function delta(z) = (1 - z) + (1 - z)^2 / 2.
 *
 * Generalised CQ contour of App. A: s_l = gamma(sigma_l) with
 *   gamma(sig)  = (sqrt(2q-1) (1/k + sn)/(1/k - sn) - 1) / (dt_min (q-1)),
 *   gamma'(sig) = sqrt(2q-1)/(dt_min (q-1)) * 2 cn dn / (k (1/k - sn)^2),
 *   sigma_l = -K + (l - 1/2) 4K/N_Q + i K'/2,  l = 1..N_Q,
 *   k = (q - sqrt(2q-1)) / (q + sqrt(2q-1)),
 *   q = 5 dt_max max|lambda(A)| / (dt_min min|lambda(A)|)  (factor 5 dropped
 *       for implicit Euler, whose stability eigenvalue is 1),
 * with sn, cn, dn and K, K' taken at parameter m = k^2 (K' = K(1 - m), the
 * complementary integral).  The weight prefactor of App. A is garbled in the
 * source; it is read as the trapezoidal rule for the positively oriented
 * Cauchy integral (1/(2 pi i)) \oint ds over the sigma-period 4K.  As sigma
 * runs from -K to 3K the image runs clockwise around the circle through 0 and
 * 2/dt_min, hence  w_l = -(4K/N_Q) gamma'(sigma_l) / (2 pi i).
 */
#include "orc.h"

#include <complex.h>
#include <math.h>

typedef double complex cplx;

int orc_freqs_bdf2(int N, double dt, double lambda, double *s) {
    if (N < 1 || !(dt > 0.0)) return -1;
    if (lambda <= 0.0) lambda = pow(1e-8, 1.0 / (2.0 * N));
    const double pi = acos(-1.0);
    for (int k = 0; k < N; ++k) {
        cplx z = lambda * cexp(I * (2.0 * pi * k / N));
        cplx d = (1.0 - z) + 0.5 * (1.0 - z) * (1.0 - z);
        cplx sk = d / dt;
        s[2 * k] = creal(sk);
        s[2 * k + 1] = cimag(sk);
    }
    return 0;
}

/* K(m) = pi / (2 AGM(1, sqrt(1 - m))). */
double orc_ellipk(double m) {
    if (!(m < 1.0)) return INFINITY;
    double a = 1.0, b = sqrt(1.0 - m);
    for (int it = 0; it < 64 && fabs(a - b) > 1e-16 * a; ++it) {
        double an = 0.5 * (a + b);
        b = sqrt(a * b);
        a = an;
    }
    return acos(-1.0) / (2.0 * a);
}

/* Descending Landen / AGM scheme (Abramowitz and Stegun 16.4):
 * a_0 = 1, b_0 = sqrt(1-m), c_0 = sqrt(m); a_n, b_n, c_n by the AGM;
 * phi_N = 2^N a_N u; phi_{n-1} = (phi_n + asin(c_n sin(phi_n) / a_n)) / 2;
 * sn = sin phi_0, cn = cos phi_0, dn = cos phi_0 / cos(phi_1 - phi_0). */
void orc_ellipj(double u, double m, double *sn, double *cn, double *dn) {
    if (m < 1e-300) {
        *sn = sin(u);
        *cn = cos(u);
        *dn = 1.0;
        return;
    }
    if (m >= 1.0) {
        *sn = tanh(u);
        *cn = 1.0 / cosh(u);
        *dn = *cn;
        return;
    }
    double a[40], c[40];
    a[0] = 1.0;
    double b = sqrt(1.0 - m);
    c[0] = sqrt(m);
    int n = 0;
    while (fabs(c[n]) > 1e-16 && n < 38) {
        double an = 0.5 * (a[n] + b);
        c[n + 1] = 0.5 * (a[n] - b);
        b = sqrt(a[n] * b);
        a[n + 1] = an;
        n++;
    }
    double phi = ldexp(a[n] * u, n);
    double phi_next = phi;
    for (int k = n; k >= 1; --k) {
        phi_next = phi;
        phi = 0.5 * (phi + asin(c[k] * sin(phi) / a[k]));
    }
    *sn = sin(phi);
    *cn = cos(phi);
    *dn = (n >= 1) ? cos(phi) / cos(phi_next - phi) : sqrt(1.0 - m * (*sn) * (*sn));
}

/* Addition formulas with the complementary parameter (A and S 16.21.1-4):
 * with s, c, d = sn, cn, dn(u | m) and s1, c1, d1 = sn, cn, dn(v | 1-m),
 * D = c1^2 + m s^2 s1^2,
 *   sn(u+iv) = (s d1 + i c d s1 c1) / D
 *   cn(u+iv) = (c c1 - i s d s1 d1) / D
 *   dn(u+iv) = (d c1 d1 - i m s c s1) / D. */
void orc_ellipj_complex(double u, double v, double m, double *sn, double *cn, double *dn) {
    double s, c, d, s1, c1, d1;
    orc_ellipj(u, m, &s, &c, &d);
    orc_ellipj(v, 1.0 - m, &s1, &c1, &d1);
    double D = c1 * c1 + m * s * s * s1 * s1;
    sn[0] = s * d1 / D;
    sn[1] = c * d * s1 * c1 / D;
    cn[0] = c * c1 / D;
    cn[1] = -s * d * s1 * d1 / D;
    dn[0] = d * c1 * d1 / D;
    dn[1] = -m * s * c * s1 / D;
}

/* Stability function of the Runge-Kutta method, R(z) = 1 + z b^T (I - z A)^{-1} 1:
 * implicit Euler 1/(1 - z); 2-stage Radau IIA (1 + z/3)/(1 - 2z/3 + z^2/6). */
static cplx rk_stability(int rk, cplx z) {
    if (rk == 1) return (1.0 + z / 3.0) / (1.0 - 2.0 * z / 3.0 + z * z / 6.0);
    return 1.0 / (1.0 - z);
}

/* Radius factor rho of the contour (the circle through 0 and 2 rho / dt_min):
 * the gCQ steps (eq. gCQ_xn) need a contour that encloses every resolvent pole
 * 1/(dt lambda_i(A)), which takes rho > 1 / (2 min_i Re lambda_i) and holds
 * for rho = 1 / min_i |lambda_i|; and the Runge-Kutta stages of the N steps
 * grow along the contour like max |R(dt_min s)|^N, which must stay bounded
 * (<= 1e4 here) for the quadrature sums not to cancel away in FP64.  For
 * implicit Euler |R| = 1 on the circle of rho = 1 (the printed contour);
 * for Radau IIA rho grows from sqrt(6) in steps of 5 % until the bound holds
 * on 4096 points of the circle. */
double orc_gcq_radius(int rk, int nsteps) {
    if (rk != 1) return 1.0;
    const double pi = acos(-1.0);
    double rho = sqrt(6.0);
    for (int it = 0; it < 400; ++it) {
        double mx = 0.0;
        for (int j = 1; j < 4096; ++j) {
            cplx z = rho * (1.0 + cexp(I * (2.0 * pi * j / 4096.0)));
            double a = cabs(rk_stability(rk, z));
            if (a > mx) mx = a;
        }
        if ((double)(nsteps > 1 ? nsteps : 1) * log(mx) <= log(1e4)) return rho;
        rho *= 1.05;
    }
    return rho;
}

int orc_freqs_gcq(double dt_min, double dt_max, int rk, int nsteps, double rho_in, int NQ, double *s,
                  double *w, double *info) {
    if (!(dt_min > 0.0) || !(dt_max >= dt_min) || NQ < 2) return -1;
    double q = dt_max / dt_min;
    if (rk == 1) q *= 5.0; /* Radau IIA, 2 stages: |lambda_1| = |lambda_2| */
    int lifted = 0;
    if (q < 1.01) { /* q = 1 makes k = 0 (App. A, last paragraph): lift it */
        q = 1.01;
        lifted = 1;
    }
    const double rho = rho_in > 0.0 ? rho_in : orc_gcq_radius(rk, nsteps);
    const double pi = acos(-1.0);
    double r = sqrt(2.0 * q - 1.0);
    double k = (q - r) / (q + r);
    double m = k * k;
    double K = orc_ellipk(m), Kp = orc_ellipk(1.0 - m);
    /* Reading of App. A: gamma and gamma' take dt_min / rho (orc_gcq_radius);
     * with dt_min as printed the circle misses the Radau IIA poles
     * (2 -/+ i sqrt(2))/dt of steps below 1.5 dt_min. */
    double scale = rho / (dt_min * (q - 1.0));
    for (int l = 1; l <= NQ; ++l) {
        double u = -K + (l - 0.5) * 4.0 * K / NQ, v = 0.5 * Kp;
        double snr[2], cnr[2], dnr[2];
        orc_ellipj_complex(u, v, m, snr, cnr, dnr);
        cplx sn = snr[0] + I * snr[1], cn = cnr[0] + I * cnr[1], dn = dnr[0] + I * dnr[1];
        cplx g = scale * (r * (1.0 / k + sn) / (1.0 / k - sn) - 1.0);
        cplx gp = scale * r * 2.0 * cn * dn / (k * (1.0 / k - sn) * (1.0 / k - sn));
        cplx wl = -(4.0 * K / NQ) * gp / (2.0 * pi * I);
        s[2 * (l - 1)] = creal(g);
        s[2 * (l - 1) + 1] = cimag(g);
        if (w) {
            w[2 * (l - 1)] = creal(wl);
            w[2 * (l - 1) + 1] = cimag(wl);
        }
    }
    if (info) {
        info[0] = q;
        info[1] = k;
        info[2] = K;
        info[3] = Kp;
        info[4] = rho;
    }
    return lifted;
}
