// Galerkin pair integrals of the Laplace-domain layer operators on flat
// triangles (Sec. 2 eqs. slp/dlp, Sec. 3 "Spatial discretisation").
//
//   SLP:  int_x int_y exp(-s r/c) / (4 pi r)                      (P0 x P0)
//   DLP:  int_x int_y phi_m(y) exp(-s r/c)(1 + s r/c)(x-y).n_y / (4 pi r^3)
//         for the three P1 hats phi_m of the trial triangle         (P0 x P1)
//   ADLP: int_x int_y exp(-s r/c)(1 + s r/c)(y-x).n_x / (4 pi r^3)
//         (K', eq. adlp: the conormal derivative at x)              (P0 x P0)
//
// Regular pairs: 7-point degree-5 rule in x and in y.  FP32 form: the
// quadrature-point coordinates are split into hi + lo floats so that the
// difference y - x keeps FP32 relative accuracy for close pairs.
// Touching pairs (identical, common edge, common vertex): Sauter-Schwab
// regularising transforms in FP64 with ng Gauss-Legendre points per variable:
//   identical: z = yh - xh in six sectors, z = xi (e_a + eta (e_b - e_a)),
//              weight xi (1 - xi)^2 / 2 (P0 x P0: kernel depends on z only);
//   edge:      (u, p, q) = (yh1 - xh1, xh2, yh2) on six cone triangles,
//              weight xi^2 e1 |det| (1 - xi), trial point at mid t-range;
//   vertex:    larger of xh1, yh1 is xi, weight xi^3 e1, two regions.
// The parametrisation of a triangle (P0, P1, P2) is
// chi(xh) = P0 + xh1 (P1 - P0) + xh2 (P2 - P1) on {0 <= xh2 <= xh1 <= 1}.
#pragma once
#include "common.cuh"

#define TD_FOUR_PI 12.566370614359172953850573533118
#define TD_INV_FOUR_PI_F 0.079577471545947667884f

enum { TD_SLP = 0, TD_DLP = 1, TD_ADLP = 2 };
// The double layer's trial space is P1 (a column is a vertex and its
// triangles); the single layer and the adjoint double layer have P0 columns.
#define TD_P1_TRIAL(OP) ((OP) == TD_DLP)

struct MeshDev {
    int nt, nv;
    // FP32 7-point tables, layout [7][nt]: hi/lo coordinates, weight*area
    const float *qxh, *qyh, *qzh, *qxl, *qyl, *qzl, *qw32;
    const float *n32;  // [3][nt] unit normals
    // the same FP32 tables packed for 16-byte loads: qp[2 (p nt + e)] =
    // (x_hi, y_hi, z_hi, weight*area), qp[2 (p nt + e) + 1] = (x_lo, y_lo,
    // z_lo, 0); nrm4[e] = (n_x, n_y, n_z, 0)
    const float4 *qp, *nrm4;
    // FP64 7-point tables [7][nt] and normals [3][nt]
    const double *qx, *qy, *qz, *qw, *n64;
    const double *verts;  // [nv][3]
    const int *tris;      // [nt][3]
    const double *area;   // [nt]
    const int *v2t_ptr, *v2t;      // P1 supports: triangles around a vertex
    const signed char *v2t_loc;    // local index of the vertex in that triangle
    const int *tp_ptr, *tp_tri, *tp_slot;  // touching triangles per triangle (sorted)
    int ng;
    const double *gx, *gw;  // Gauss-Legendre on [0,1]
};

// Barycentric coordinates of the 7 rule points: the centroid, the orbit
// (a, a, 1-2a) and the orbit (b, b, 1-2b), a, b = (6 -/+ sqrt 15)/21, in the
// order (a,a,1-2a), (a,1-2a,a), (1-2a,a,a), then the same for b.
#define TD_R7A 0.10128650732345633880098736191512
#define TD_R7A1 0.79742698535308732239802527616975
#define TD_R7B 0.47014206410511508977044120951345
#define TD_R7B1 0.05971587178976982045911758097311
TD_HD double bary7d(int b, int k) {
    if (b == 0) return 1.0 / 3.0;
    const int odd = 2 - (b - 1) % 3;
    const bool orb_a = b <= 3;
    return k == odd ? (orb_a ? TD_R7A1 : TD_R7B1) : (orb_a ? TD_R7A : TD_R7B);
}
TD_HD float bary7f(int b, int k) {
    if (b == 0) return 1.0f / 3.0f;
    const int odd = 2 - (b - 1) % 3;
    const bool orb_a = b <= 3;
    return k == odd ? (orb_a ? (float)TD_R7A1 : (float)TD_R7B1) : (orb_a ? (float)TD_R7A : (float)TD_R7B);
}

// ---------------------------------------------------------------------------
// Regular pairs.  The test triangle's 7 points are held in registers (the
// loop over them is fully unrolled); the trial triangle's points are read
// one at a time from the [7][nt] tables (coalesced when threads take
// different trial triangles, broadcast when they share one).
// ---------------------------------------------------------------------------
struct TestF {
    float xh[7], yh[7], zh[7], xl[7], yl[7], zl[7], w[7];
    float nx, ny, nz;  // unit normal of the test triangle (adjoint double layer)
};

TD_D void load_test(const MeshDev &m, int t, TestF &T) {
#pragma unroll
    for (int q = 0; q < 7; ++q) {
        const int o = q * m.nt + t;
        T.xh[q] = m.qxh[o];
        T.yh[q] = m.qyh[o];
        T.zh[q] = m.qzh[o];
        T.xl[q] = m.qxl[o];
        T.yl[q] = m.qyl[o];
        T.zl[q] = m.qzl[o];
        T.w[q] = m.qw32[o];
    }
    T.nx = m.n32[t];
    T.ny = m.n32[m.nt + t];
    T.nz = m.n32[2 * m.nt + t];
}

// e^{-sigma r} = e^{-sr r} (cos(si r) - i sin(si r)) for sigma = (sr, si), FP32
// on the special-function unit:
//   exponent: e^{-x} = 2^{t}, t = -x log2(e) formed as a rounded product plus
//     its FMA-recovered rounding error and the low part of log2(e), then
//     2^{t_hi} (1 + t_lo ln 2);
//   phase: Cody-Waite additive reduction y - k 2pi with k the nearest integer
//     to y / 2pi (formed by adding and subtracting 1.5 * 2^23, which rounds
//     to an integer in round-to-nearest for |y / 2pi| < 2^22, on the FMA pipe
//     instead of a separate rounding instruction) and 2pi split into a float
//     head and tail (two FMAs), then the SFU sin/cos, whose absolute error is
//     below 4e-7 on [-pi, pi].
// The power of two is the SFU's ex2 with subnormal results flushed to zero
// (values below 1.2e-38, far below the entries' resolution).
#define TD_L2E_HI 1.44269502162933349609375f
#define TD_L2E_LO 1.92596298909109e-08f
#define TD_LN2_F 0.693147180559945309417f
#define TD_2PI_HI 6.28318548202514648438f
#define TD_2PI_LO (-1.7484556025237907e-07f)
#define TD_INV_2PI_F 0.159154943091895335769f
TD_D float ex2_ftz(float t) {
    float v;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(v) : "f"(t));
    return v;
}
TD_D c32 expm_sr(float sr, float si, float r) {
    const float x = sr * r;
    const float th = -x * TD_L2E_HI;
    const float tl = fmaf(-x, TD_L2E_HI, -th) - x * TD_L2E_LO;
    const float ea = ex2_ftz(th) * fmaf(tl, TD_LN2_F, 1.0f);
    const float y = si * r;
    const float k = __fsub_rn(__fadd_rn(y * TD_INV_2PI_F, 12582912.0f), 12582912.0f);
    float yr = fmaf(-k, TD_2PI_HI, y);
    yr = fmaf(-k, TD_2PI_LO, yr);
    float sn, cs;
    __sincosf(yr, &sn, &cs);
    return {ea * cs, -ea * sn};
}

// out (SLP: out[0]; DLP: out[0..2] per trial-local vertex) += pair integral
// over test X and trial triangle tj, sigma = s / c.  Unscaled by 1/(4 pi).
template <int OP>
TD_D void pair_f32(const TestF &X, const MeshDev &m, int tj, float sr, float si, c32 *out) {
    // kernel normal: the trial normal with -d.n (DLP) or the test normal with +d.n (ADLP)
    float nx = 0.f, ny = 0.f, nz = 0.f;
    if (OP == TD_DLP) {
        nx = -m.n32[tj];
        ny = -m.n32[m.nt + tj];
        nz = -m.n32[2 * m.nt + tj];
    } else if (OP == TD_ADLP) {
        nx = X.nx;
        ny = X.ny;
        nz = X.nz;
    }
#pragma unroll 1
    for (int b = 0; b < 7; ++b) {
        const int ob = b * m.nt + tj;
        const float yxh = m.qxh[ob], yyh = m.qyh[ob], yzh = m.qzh[ob];
        const float yxl = m.qxl[ob], yyl = m.qyl[ob], yzl = m.qzl[ob];
        const float wy = m.qw32[ob];
        c32 acc = {0.f, 0.f};
#pragma unroll
        for (int a = 0; a < 7; ++a) {
            const float dx = (yxh - X.xh[a]) + (yxl - X.xl[a]);
            const float dy = (yyh - X.yh[a]) + (yyl - X.yl[a]);
            const float dz = (yzh - X.zh[a]) + (yzl - X.zl[a]);
            const float r2 = dx * dx + dy * dy + dz * dz;
            const float rinv = rsqrtf(r2);
            const float r = r2 * rinv;
            const c32 e = expm_sr(sr, si, r);
            if (OP == TD_SLP) {
                const float w = X.w[a] * rinv;
                acc.x = fmaf(w, e.x, acc.x);
                acc.y = fmaf(w, e.y, acc.y);
            } else {
                // (1 + sigma r) e^{-sigma r} (d.n) / r^3, n signed as above
                const float dn = dx * nx + dy * ny + dz * nz;
                const float w = X.w[a] * dn * rinv * rinv * rinv;
                const float pr = fmaf(sr, r, 1.0f), pi = si * r;
                acc.x = fmaf(w, pr * e.x - pi * e.y, acc.x);
                acc.y = fmaf(w, pr * e.y + pi * e.x, acc.y);
            }
        }
        if (!TD_P1_TRIAL(OP)) {
            out[0].x = fmaf(wy, acc.x, out[0].x);
            out[0].y = fmaf(wy, acc.y, out[0].y);
        } else {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float f = wy * bary7f(b, k);
                out[k].x = fmaf(f, acc.x, out[k].x);
                out[k].y = fmaf(f, acc.y, out[k].y);
            }
        }
    }
}

struct TestD {
    double x[7], y[7], z[7], w[7];
    double nx, ny, nz;  // unit normal of the test triangle (adjoint double layer)
};

TD_D void load_test(const MeshDev &m, int t, TestD &T) {
#pragma unroll
    for (int q = 0; q < 7; ++q) {
        const int o = q * m.nt + t;
        T.x[q] = m.qx[o];
        T.y[q] = m.qy[o];
        T.z[q] = m.qz[o];
        T.w[q] = m.qw[o];
    }
    T.nx = m.n64[t];
    T.ny = m.n64[m.nt + t];
    T.nz = m.n64[2 * m.nt + t];
}

TD_D c64 expm_sr(double sr, double si, double r) {
    double ea = exp(-sr * r);
    double sn, cs;
    sincos(si * r, &sn, &cs);
    return {ea * cs, -ea * sn};
}

template <int OP>
TD_D void pair_f64(const TestD &X, const MeshDev &m, int tj, double sr, double si, c64 *out) {
    double nx = 0.0, ny = 0.0, nz = 0.0;  // signed kernel normal, as in pair_f32
    if (OP == TD_DLP) {
        nx = -m.n64[tj];
        ny = -m.n64[m.nt + tj];
        nz = -m.n64[2 * m.nt + tj];
    } else if (OP == TD_ADLP) {
        nx = X.nx;
        ny = X.ny;
        nz = X.nz;
    }
#pragma unroll 1
    for (int b = 0; b < 7; ++b) {
        const int ob = b * m.nt + tj;
        const double yx = m.qx[ob], yy = m.qy[ob], yz = m.qz[ob], wy = m.qw[ob];
        c64 acc = {0.0, 0.0};
#pragma unroll
        for (int a = 0; a < 7; ++a) {
            const double dx = yx - X.x[a], dy = yy - X.y[a], dz = yz - X.z[a];
            const double r = sqrt(dx * dx + dy * dy + dz * dz);
            const c64 e = expm_sr(sr, si, r);
            if (OP == TD_SLP) {
                const double w = X.w[a] / r;
                acc.x += w * e.x;
                acc.y += w * e.y;
            } else {
                const double dn = dx * nx + dy * ny + dz * nz;
                const double w = X.w[a] * dn / (r * r * r);
                const double pr = 1.0 + sr * r, pi = si * r;
                acc.x += w * (pr * e.x - pi * e.y);
                acc.y += w * (pr * e.y + pi * e.x);
            }
        }
        if (!TD_P1_TRIAL(OP)) {
            out[0].x += wy * acc.x;
            out[0].y += wy * acc.y;
        } else {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const double f = wy * bary7d(b, k);
                out[k].x += f * acc.x;
                out[k].y += f * acc.y;
            }
        }
    }
}

// Precision dispatch used by the kernels.
template <class T> struct Reg;
template <> struct Reg<float> {
    using Test = TestF;
    template <int OP> TD_D static void pair(const Test &X, const MeshDev &m, int tj, float sr, float si, c32 *o) {
        pair_f32<OP>(X, m, tj, sr, si, o);
    }
};
template <> struct Reg<double> {
    using Test = TestD;
    template <int OP> TD_D static void pair(const Test &X, const MeshDev &m, int tj, double sr, double si, c64 *o) {
        pair_f64<OP>(X, m, tj, sr, si, o);
    }
};

// ---------------------------------------------------------------------------
// Touching pairs: classification and Sauter-Schwab quadrature points (FP64)
// ---------------------------------------------------------------------------
struct SingGeom {
    int cls;           // 3 identical, 2 edge, 1 vertex, 0 none
    double P[3][3];    // test parametrisation vertices
    double Q[3][3];    // trial parametrisation vertices
    int loc[3];        // mesh-local index of trial parametrisation vertex k
    double g;          // Jacobian factor (2|ti|)(2|tj|)
    double ny[3];      // trial unit normal
    double nx[3];      // test unit normal
};

// Shared vertices of ti and tj decide the class; the parametrisations follow
// the order described at the top of this file:
//   identical: both in mesh order; edge: shared vertices in increasing local
//   index of ti, then the remaining vertex; vertex: the shared vertex then the
//   next two in each triangle's own cyclic order.
TD_D int classify_pair(const MeshDev &m, int ti, int tj, SingGeom &G) {
    const int *A = m.tris + 3 * ti, *B = m.tris + 3 * tj;
    int a[3] = {A[0], A[1], A[2]}, b[3] = {B[0], B[1], B[2]};
    int ia[3], ib[3], ns = 0;
#pragma unroll
    for (int x = 0; x < 3; ++x)
#pragma unroll
        for (int y = 0; y < 3; ++y)
            if (a[x] == b[y]) {
                ia[ns] = x;
                ib[ns] = y;
                ns++;
            }
    G.cls = ns;
    if (ns == 0) return 0;
    int la[3], lb[3];
    if (ns == 3) {
        for (int k = 0; k < 3; ++k) la[k] = lb[k] = k;
    } else if (ns == 2) {
        la[0] = ia[0];
        la[1] = ia[1];
        la[2] = 3 - ia[0] - ia[1];
        lb[0] = ib[0];
        lb[1] = ib[1];
        lb[2] = 3 - ib[0] - ib[1];
    } else {
        for (int k = 0; k < 3; ++k) {
            la[k] = (ia[0] + k) % 3;
            lb[k] = (ib[0] + k) % 3;
        }
    }
    for (int k = 0; k < 3; ++k) {
        G.loc[k] = lb[k];
        for (int c = 0; c < 3; ++c) {
            G.P[k][c] = m.verts[3 * a[la[k]] + c];
            G.Q[k][c] = m.verts[3 * b[lb[k]] + c];
        }
    }
    G.g = 4.0 * m.area[ti] * m.area[tj];
    G.ny[0] = m.n64[tj];
    G.ny[1] = m.n64[m.nt + tj];
    G.ny[2] = m.n64[2 * m.nt + tj];
    G.nx[0] = m.n64[ti];
    G.nx[1] = m.n64[m.nt + ti];
    G.nx[2] = m.n64[2 * m.nt + ti];
    return ns;
}

TD_HD int ss_npoints(int cls, int ng) {
    int n2 = ng * ng;
    return cls == 3 ? 6 * n2 : cls == 2 ? 6 * n2 * ng : cls == 1 ? 2 * n2 * n2 : 0;
}

// Quadrature point q of the transformed integral: difference vector d = y - x,
// weight (including the Jacobian factor g) and trial barycentric weights lam
// (parametrisation order; use G.loc to map to mesh-local vertices).
TD_D void ss_point(const SingGeom &G, int q, int ng, const double *gx, const double *gw,
                   double d[3], double &wgt, double lam[3]) {
    if (G.cls == 3) {
        // six sectors of the z-plane, rays e_a, e_b with |det| = 1
        const double SA[6][2] = {{1, 0}, {1, 1}, {0, 1}, {-1, 0}, {-1, -1}, {0, -1}};
        const double SB[6][2] = {{1, 1}, {0, 1}, {-1, 0}, {-1, -1}, {0, -1}, {1, 0}};
        int sct = q / (ng * ng), a = (q / ng) % ng, b = q % ng;
        double xi = gx[a], eta = gx[b];
        double z1 = SA[sct][0] + eta * (SB[sct][0] - SA[sct][0]);
        double z2 = SA[sct][1] + eta * (SB[sct][1] - SA[sct][1]);
        for (int k = 0; k < 3; ++k)
            d[k] = xi * (z1 * (G.P[1][k] - G.P[0][k]) + z2 * (G.P[2][k] - G.P[1][k]));
        wgt = gw[a] * gw[b] * xi * (1.0 - xi) * (1.0 - xi) * 0.5 * G.g;
        lam[0] = lam[1] = lam[2] = 0.0;  // identical pairs only occur for P0 x P0
    } else if (G.cls == 2) {
        // cone triangles (u, p, q) with vertices on l(u,p,q) = 1
        const double V[6][3][3] = {
            {{0, 1, 0}, {1, 0, 0}, {1, 0, 1}},  {{0, 1, 0}, {1, 0, 1}, {0, 1, 1}},
            {{0, 0, 1}, {1, 0, 1}, {0, 1, 1}},  {{0, 1, 0}, {0, 1, 1}, {-1, 1, 0}},
            {{-1, 0, 0}, {0, 0, 1}, {0, 1, 1}}, {{-1, 0, 0}, {0, 1, 1}, {-1, 1, 0}}};
        int n3 = ng * ng * ng;
        int tr = q / n3, r = q % n3, a = r / (ng * ng), b = (r / ng) % ng, c = r % ng;
        double xi = gx[a], e1 = gx[b], e2 = gx[c];
        double w3[3];
        for (int k = 0; k < 3; ++k)
            w3[k] = xi * (V[tr][0][k] + e1 * (V[tr][1][k] - V[tr][0][k]) +
                          e1 * e2 * (V[tr][2][k] - V[tr][1][k]));
        double u = w3[0], p = w3[1], qq = w3[2];
        for (int k = 0; k < 3; ++k)
            d[k] = u * (G.P[1][k] - G.P[0][k]) + qq * (G.Q[2][k] - G.Q[1][k]) -
                   p * (G.P[2][k] - G.P[1][k]);
        // |det| is 1 for all six cone triangles
        wgt = gw[a] * gw[b] * gw[c] * xi * xi * e1 * (1.0 - xi) * G.g;
        double tlo = p > qq - u ? p : qq - u;
        double thi = u > 0.0 ? 1.0 - u : 1.0;
        double tm = 0.5 * (tlo + thi);
        double y1 = tm + u, y2 = qq;
        lam[0] = 1.0 - y1;
        lam[1] = y1 - y2;
        lam[2] = y2;
    } else {
        int n4 = ng * ng * ng * ng;
        int reg = q / n4, r = q % n4;
        int a = r / (ng * ng * ng), b = (r / (ng * ng)) % ng, c = (r / ng) % ng, e = r % ng;
        double xi = gx[a], w = gx[b], e1 = gx[c], e2 = gx[e];
        double x1, x2, y1, y2;
        if (reg == 0) {
            x1 = xi;
            x2 = xi * w;
            y1 = xi * e1;
            y2 = xi * e1 * e2;
        } else {
            y1 = xi;
            y2 = xi * w;
            x1 = xi * e1;
            x2 = xi * e1 * e2;
        }
        for (int k = 0; k < 3; ++k)
            d[k] = y1 * (G.Q[1][k] - G.Q[0][k]) + y2 * (G.Q[2][k] - G.Q[1][k]) -
                   x1 * (G.P[1][k] - G.P[0][k]) - x2 * (G.P[2][k] - G.P[1][k]);
        wgt = gw[a] * gw[b] * gw[c] * gw[e] * xi * xi * xi * e1 * G.g;
        lam[0] = 1.0 - y1;
        lam[1] = y1 - y2;
        lam[2] = y2;
    }
}

// Signed normal factor of the double-layer kernels at difference d = y - x:
// (x - y).n_y (DLP) or (y - x).n_x (ADLP).
template <int OP>
TD_HD double ss_dn(const SingGeom &G, const double d[3]) {
    return OP == TD_DLP ? -(d[0] * G.ny[0] + d[1] * G.ny[1] + d[2] * G.ny[2])
                        : d[0] * G.nx[0] + d[1] * G.nx[1] + d[2] * G.nx[2];
}

// Kernel value times weight at one transformed point, accumulated into out
// (mesh-local trial vertex order for DLP).  sigma = s / c.
template <int OP>
TD_D void ss_accum(const SingGeom &G, const double d[3], double wgt, const double lam[3],
                   double sr, double si, c64 *out) {
    double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    c64 e = expm_sr(sr, si, r);
    if (OP == TD_SLP) {
        double w = wgt / r;
        out[0].x += w * e.x;
        out[0].y += w * e.y;
    } else {
        double dn = ss_dn<OP>(G, d);
        double w = wgt * dn / (r * r * r);
        double pr = 1.0 + sr * r, pi = si * r;
        c64 v = {w * (pr * e.x - pi * e.y), w * (pr * e.y + pi * e.x)};
        if (OP == TD_ADLP) {
            out[0].x += v.x;
            out[0].y += v.y;
        } else {
            for (int k = 0; k < 3; ++k) {
                out[G.loc[k]].x += lam[k] * v.x;
                out[G.loc[k]].y += lam[k] * v.y;
            }
        }
    }
}

// Whole touching-pair integral by one thread (used by the generic entry
// kernel; the compressor uses the warp-parallel table kernel instead).
// Returns the class; out is unscaled by 1/(4 pi).
template <int OP>
TD_D int pair_singular_f64(const MeshDev &m, int ti, int tj, double sr, double si, c64 *out) {
    if (OP == TD_SLP && ti > tj) {
        int t = ti;
        ti = tj;
        tj = t;
    }
    SingGeom G;
    if (classify_pair(m, ti, tj, G) == 0) return 0;
    if (OP != TD_SLP && G.cls == 3) return 3;  // flat panel: (x - y).n = 0
    int nq = ss_npoints(G.cls, m.ng);
    for (int q = 0; q < nq; ++q) {
        double d[3], w, lam[3];
        ss_point(G, q, m.ng, m.gx, m.gw, d, w, lam);
        ss_accum<OP>(G, d, w, lam, sr, si, out);
    }
    return G.cls;
}

// Index of tj in ti's touching list, or -1.
TD_D int touching_slot(const MeshDev &m, int ti, int tj) {
    for (int p = m.tp_ptr[ti]; p < m.tp_ptr[ti + 1]; ++p)
        if (m.tp_tri[p] == tj) return m.tp_slot[p];
    return -1;
}
