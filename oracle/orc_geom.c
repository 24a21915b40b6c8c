/*
 * Oracle (test infrastructure only): mesh, quadrature and Galerkin entries.
 *
 * Sec. 2: single layer V with kernel U^(r, s) = exp(-s r/c)/(4 pi r) and
 * double layer K with kernel gamma_{1,y} U^ = exp(-s r/c)(1 + s r/c)
 * (x-y).n_y / (4 pi r^3) (the normal derivative of U^ in y, outward n).
 * Sec. 3 "Spatial discretisation": flat triangles, P0 discontinuous and P1
 * continuous bases, Galerkin double integrals; regular pairs with a Gauss
 * rule, weakly singular pairs with the Erichsen-Sauter formulas, i.e. the
 * regularising coordinate transforms of Sauter and Schwab, written out below
 * from their derivation for flat panels.
 */
#include "orc.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

struct orc_mesh {
    int64_t nv, nt;
    double *v;      /* [nv][3] */
    int32_t *t;     /* [nt][3] */
    double *area;   /* [nt] */
    double *nrm;    /* [nt][3] unit normal */
    int64_t *v2t_ptr; /* CSR vertex -> triangles */
    int32_t *v2t;
    int8_t *v2t_loc; /* local index of the vertex in that triangle */
};

static void sub3(const double *a, const double *b, double *o) {
    o[0] = a[0] - b[0];
    o[1] = a[1] - b[1];
    o[2] = a[2] - b[2];
}
static void cross3(const double *a, const double *b, double *o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double *a, const double *b) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

orc_mesh *orc_mesh_new(const double *verts, int64_t nv, const int32_t *tris, int64_t nt) {
    if (nv <= 0 || nt <= 0) return NULL;
    for (int64_t e = 0; e < 3 * nt; ++e)
        if (tris[e] < 0 || tris[e] >= nv) return NULL;
    orc_mesh *m = calloc(1, sizeof *m);
    m->nv = nv;
    m->nt = nt;
    m->v = malloc(sizeof(double) * 3 * nv);
    memcpy(m->v, verts, sizeof(double) * 3 * nv);
    m->t = malloc(sizeof(int32_t) * 3 * nt);
    memcpy(m->t, tris, sizeof(int32_t) * 3 * nt);
    m->area = malloc(sizeof(double) * nt);
    m->nrm = malloc(sizeof(double) * 3 * nt);
    for (int64_t e = 0; e < nt; ++e) {
        const double *a = m->v + 3 * m->t[3 * e], *b = m->v + 3 * m->t[3 * e + 1],
                     *c = m->v + 3 * m->t[3 * e + 2];
        double ab[3], ac[3], n[3];
        sub3(b, a, ab);
        sub3(c, a, ac);
        cross3(ab, ac, n);
        double len = sqrt(dot3(n, n));
        if (!(len > 0.0) || !isfinite(len)) {
            orc_mesh_free(m);
            return NULL;
        }
        m->area[e] = 0.5 * len;
        for (int k = 0; k < 3; ++k) m->nrm[3 * e + k] = n[k] / len;
    }
    m->v2t_ptr = calloc(nv + 1, sizeof(int64_t));
    for (int64_t e = 0; e < 3 * nt; ++e) m->v2t_ptr[tris[e] + 1]++;
    for (int64_t v = 0; v < nv; ++v) m->v2t_ptr[v + 1] += m->v2t_ptr[v];
    m->v2t = malloc(sizeof(int32_t) * 3 * nt);
    m->v2t_loc = malloc(3 * nt);
    int64_t *fill = calloc(nv, sizeof(int64_t));
    for (int64_t e = 0; e < nt; ++e)
        for (int k = 0; k < 3; ++k) {
            int32_t v = tris[3 * e + k];
            int64_t p = m->v2t_ptr[v] + fill[v]++;
            m->v2t[p] = (int32_t)e;
            m->v2t_loc[p] = (int8_t)k;
        }
    free(fill);
    return m;
}

void orc_mesh_free(orc_mesh *m) {
    if (!m) return;
    free(m->v);
    free(m->t);
    free(m->area);
    free(m->nrm);
    free(m->v2t_ptr);
    free(m->v2t);
    free(m->v2t_loc);
    free(m);
}

int64_t orc_mesh_ndof(const orc_mesh *m, int basis) { return basis == ORC_P1 ? m->nv : m->nt; }

void orc_mesh_view(const orc_mesh *m, int64_t *nv, int64_t *nt, const double **v,
                   const int32_t **t) {
    *nv = m->nv;
    *nt = m->nt;
    *v = m->v;
    *t = m->t;
}

/* ------------------------------------------------------------------------ */
/* Quadrature rules                                                          */
/* ------------------------------------------------------------------------ */

/* Radon's 7-point rule, exact for polynomials of degree 5 on a triangle:
 * the centroid, an orbit of three points a,a,1-2a near the vertices and an
 * orbit b,b,1-2b near the edge midpoints, a,b = (6 -/+ sqrt 15)/21. */
void orc_rule7(double *bary, double *w) {
    const double r15 = sqrt(15.0);
    const double a = (6.0 - r15) / 21.0, b = (6.0 + r15) / 21.0;
    const double wa = (155.0 - r15) / 1200.0, wb = (155.0 + r15) / 1200.0;
    double pts[7][3] = {{1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0},
                        {a, a, 1.0 - 2.0 * a},
                        {a, 1.0 - 2.0 * a, a},
                        {1.0 - 2.0 * a, a, a},
                        {b, b, 1.0 - 2.0 * b},
                        {b, 1.0 - 2.0 * b, b},
                        {1.0 - 2.0 * b, b, b}};
    double ww[7] = {9.0 / 40.0, wa, wa, wa, wb, wb, wb};
    memcpy(bary, pts, sizeof pts);
    memcpy(w, ww, sizeof ww);
}

/* Gauss-Legendre on [-1,1] by Newton iteration on the three-term recurrence
 * (P_k = ((2k-1) z P_{k-1} - (k-1) P_{k-2}) / k), mapped to [0,1]:
 * node (1 - z)/2, weight 1/((1 - z^2) P_n'(z)^2). */
static void legendre(int n, double z, double *pn, double *dpn) {
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
    }
    if (n == 1) p0 = 1.0;
    *pn = p1;
    *dpn = n * (z * p1 - p0) / (z * z - 1.0);
}

int orc_gauss01(int n, double *x, double *w) {
    if (n < 1 || n > 64) return -1;
    const double pi = acos(-1.0);
    for (int i = 0; i < n; ++i) {
        double z = cos(pi * (i + 0.75) / (n + 0.5)), pn, dp;
        for (int it = 0; it < 100; ++it) {
            legendre(n, z, &pn, &dp);
            double dz = pn / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        legendre(n, z, &pn, &dp);
        x[i] = 0.5 * (1.0 - z);
        w[i] = 1.0 / ((1.0 - z * z) * dp * dp);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Kernels                                                                   */
/* ------------------------------------------------------------------------ */

static const double FOUR_PI = 12.566370614359172953850573533118;

/* SLP kernel exp(-s r/c)/(4 pi r); d = y - x, sc = s/c. */
static cplx k_slp(const double *d, cplx sc) {
    double r = sqrt(dot3(d, d));
    return cexp(-sc * r) / (FOUR_PI * r);
}
/* DLP kernel exp(-s r/c)(1 + s r/c)(x-y).n_y/(4 pi r^3); d = y - x, sc = s/c. */
static cplx k_dlp(const double *d, const double *ny, cplx sc) {
    double r = sqrt(dot3(d, d));
    return cexp(-sc * r) * (1.0 + sc * r) * (-dot3(d, ny)) / (FOUR_PI * r * r * r);
}
/* Adjoint double-layer kernel d/dn_x exp(-s r/c)/(4 pi r) =
 * exp(-s r/c)(1 + s r/c)(y-x).n_x/(4 pi r^3); d = y - x, sc = s/c. */
static cplx k_adlp(const double *d, const double *nx, cplx sc) {
    double r = sqrt(dot3(d, d));
    return cexp(-sc * r) * (1.0 + sc * r) * dot3(d, nx) / (FOUR_PI * r * r * r);
}
/* Modulus bounds of the kernels (for the magnitude sums, see orc_entries_mag):
 * |exp(-s r/c)| / (4 pi r), and |exp(-s r/c)(1 + s r/c)| r / (4 pi r^3), the
 * double layer with |(x-y).n_y| replaced by its bound |x - y|. */
static double k_slp_mag(const double *d, cplx sc) {
    double r = sqrt(dot3(d, d));
    return exp(-creal(sc) * r) / (FOUR_PI * r);
}
static double k_dlp_mag(const double *d, cplx sc) {
    double r = sqrt(dot3(d, d));
    return cabs(cexp(-sc * r) * (1.0 + sc * r)) / (FOUR_PI * r * r);
}

/* ------------------------------------------------------------------------ */
/* Pair classification and parametrisation                                   */
/* ------------------------------------------------------------------------ */

/* Parametrisation chi(xh) = P0 + xh1 (P1 - P0) + xh2 (P2 - P1) over the
 * reference triangle {0 <= xh2 <= xh1 <= 1}; its barycentric coordinates are
 * (1 - xh1, xh1 - xh2, xh2) and its Jacobian is twice the area. */
typedef struct {
    double P[3][3];
    int loc[3]; /* mesh-local index of parametrisation vertex k */
} param_tri;

static void set_param(const orc_mesh *m, int64_t e, int k0, param_tri *pt) {
    for (int k = 0; k < 3; ++k) {
        int l = (k0 + k) % 3;
        pt->loc[k] = l;
        memcpy(pt->P[k], m->v + 3 * m->t[3 * e + l], sizeof(double) * 3);
    }
}

/* Count shared vertices; build the parametrisations the transforms expect:
 *   identical: both in mesh order;
 *   edge: P0, P1 = shared vertices in increasing local index of ti, P2 = the
 *         remaining vertex of each triangle;
 *   vertex: P0 = shared vertex, P1, P2 the next vertices in each triangle's
 *           own cyclic order. */
static int classify(const orc_mesh *m, int64_t ti, int64_t tj, param_tri *a, param_tri *b) {
    const int32_t *A = m->t + 3 * ti, *B = m->t + 3 * tj;
    int ia[3], ib[3], ns = 0;
    for (int x = 0; x < 3; ++x)
        for (int y = 0; y < 3; ++y)
            if (A[x] == B[y]) {
                ia[ns] = x;
                ib[ns] = y;
                ns++;
            }
    if (ns == 3) {
        set_param(m, ti, 0, a);
        set_param(m, tj, 0, b);
        return 3;
    }
    if (ns == 2) {
        /* ia[] is ascending by construction of the loops */
        int rem_a = 3 - ia[0] - ia[1], rem_b = 3 - ib[0] - ib[1];
        int la[3] = {ia[0], ia[1], rem_a}, lb[3] = {ib[0], ib[1], rem_b};
        for (int k = 0; k < 3; ++k) {
            a->loc[k] = la[k];
            b->loc[k] = lb[k];
            memcpy(a->P[k], m->v + 3 * A[la[k]], sizeof(double) * 3);
            memcpy(b->P[k], m->v + 3 * B[lb[k]], sizeof(double) * 3);
        }
        return 2;
    }
    if (ns == 1) {
        set_param(m, ti, ia[0], a);
        set_param(m, tj, ib[0], b);
        return 1;
    }
    return 0;
}

/* chi(xh) */
static void chi(const param_tri *p, double x1, double x2, double *o) {
    for (int k = 0; k < 3; ++k)
        o[k] = p->P[0][k] + x1 * (p->P[1][k] - p->P[0][k]) + x2 * (p->P[2][k] - p->P[1][k]);
}

/* Accumulate weight * kernel * basis into out[3] (mesh-local trial vertex).
 * For SLP and ADLP only out[0] is used; nn is the trial normal (DLP) or the
 * test normal (ADLP). */
static void accum(int op, int mag, const double *d, const double *nn, cplx sc, double wgt,
                  const param_tri *pb, double y1, double y2, cplx *out) {
    if (op == ORC_SLP) {
        out[0] += mag ? wgt * k_slp_mag(d, sc) : wgt * k_slp(d, sc);
    } else if (op == ORC_ADLP) {
        out[0] += mag ? wgt * k_dlp_mag(d, sc) : wgt * k_adlp(d, nn, sc);
    } else {
        const double *ny = nn;
        cplx k = mag ? wgt * k_dlp_mag(d, sc) : wgt * k_dlp(d, ny, sc);
        double lam[3] = {1.0 - y1, y1 - y2, y2};
        for (int q = 0; q < 3; ++q) out[pb->loc[q]] += k * lam[q];
    }
}

/* ---- identical panels -------------------------------------------------- */
/* With z = yh - xh the x-domain for fixed z is a copy of the reference
 * triangle scaled by 1 - l(z), l a piecewise linear gauge.  The z-plane
 * splits into six sectors bounded by the rays below; in each, z = xi (e_a +
 * eta (e_b - e_a)) with |det(e_a, e_b)| = 1 and dz = xi dxi deta.  For P0 x
 * P0 the kernel depends on z only, so the x-integral is the area 1/2 times
 * (1 - xi)^2. */
static const double SECT[6][2][2] = {{{1, 0}, {1, 1}},   {{1, 1}, {0, 1}},
                                     {{0, 1}, {-1, 0}},  {{-1, 0}, {-1, -1}},
                                     {{-1, -1}, {0, -1}}, {{0, -1}, {1, 0}}};

static void pair_identical(const orc_mesh *m, int op, int mag, int64_t ti, const param_tri *pa,
                           cplx sc, int ng, const double *gx, const double *gw, cplx *out) {
    (void)op;
    double g = 2.0 * m->area[ti];
    double e1[3], e2[3];
    sub3(pa->P[1], pa->P[0], e1);
    sub3(pa->P[2], pa->P[1], e2);
    cplx acc = 0.0;
    for (int sct = 0; sct < 6; ++sct)
        for (int a = 0; a < ng; ++a)
            for (int b = 0; b < ng; ++b) {
                double xi = gx[a], eta = gx[b];
                double z1 = SECT[sct][0][0] + eta * (SECT[sct][1][0] - SECT[sct][0][0]);
                double z2 = SECT[sct][0][1] + eta * (SECT[sct][1][1] - SECT[sct][0][1]);
                double d[3];
                for (int k = 0; k < 3; ++k) d[k] = xi * (z1 * e1[k] + z2 * e2[k]);
                double wgt = gw[a] * gw[b] * xi * (1.0 - xi) * (1.0 - xi) * 0.5;
                acc += mag ? wgt * k_slp_mag(d, sc) : wgt * k_slp(d, sc);
            }
    out[0] += g * g * acc;
}

/* ---- common edge --------------------------------------------------------- */
/* Shared edge P0P1 in both parametrisations.  With u = yh1 - xh1, p = xh2,
 * q = yh2 the difference y - x = u(P1-P0) + q(P2'-P1) - p(P2-P1) does not
 * depend on t = xh1, whose range has length L = 1 - l(u,p,q),
 * l = max(0,u) + max(p, q-u).  The cone {l <= 1} is the union of the six
 * triangles below (vertices on l = 1) scaled by xi; a point is
 * xi (V0 + e1 (V1-V0) + e1 e2 (V2-V1)) with volume element xi^2 e1 |det|. */
static const double EDGE_TRI[6][3][3] = {
    {{0, 1, 0}, {1, 0, 0}, {1, 0, 1}},   {{0, 1, 0}, {1, 0, 1}, {0, 1, 1}},
    {{0, 0, 1}, {1, 0, 1}, {0, 1, 1}},   {{0, 1, 0}, {0, 1, 1}, {-1, 1, 0}},
    {{-1, 0, 0}, {0, 0, 1}, {0, 1, 1}},  {{-1, 0, 0}, {0, 1, 1}, {-1, 1, 0}}};

static double det3(const double a[3], const double b[3], const double c[3]) {
    return a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) +
           a[2] * (b[0] * c[1] - b[1] * c[0]);
}

static void pair_edge(const orc_mesh *m, int op, int mag, int64_t ti, int64_t tj, const param_tri *pa,
                      const param_tri *pb, cplx sc, int ng, const double *gx, const double *gw,
                      cplx *out) {
    double g = 4.0 * m->area[ti] * m->area[tj];
    const double *ny = m->nrm + 3 * (op == ORC_ADLP ? ti : tj);
    double eu[3], ep[3], eq[3];
    sub3(pa->P[1], pa->P[0], eu);
    sub3(pa->P[2], pa->P[1], ep);
    sub3(pb->P[2], pb->P[1], eq);
    cplx acc[3] = {0, 0, 0};
    for (int tr = 0; tr < 6; ++tr) {
        const double *V0 = EDGE_TRI[tr][0], *V1 = EDGE_TRI[tr][1], *V2 = EDGE_TRI[tr][2];
        double dt = fabs(det3(V0, V1, V2));
        for (int a = 0; a < ng; ++a)
            for (int b = 0; b < ng; ++b)
                for (int cidx = 0; cidx < ng; ++cidx) {
                    double xi = gx[a], e1 = gx[b], e2 = gx[cidx];
                    double w3[3];
                    for (int k = 0; k < 3; ++k)
                        w3[k] = xi * (V0[k] + e1 * (V1[k] - V0[k]) + e1 * e2 * (V2[k] - V1[k]));
                    double u = w3[0], p = w3[1], q = w3[2];
                    double d[3];
                    for (int k = 0; k < 3; ++k) d[k] = u * eu[k] + q * eq[k] - p * ep[k];
                    double wgt = gw[a] * gw[b] * gw[cidx] * xi * xi * e1 * dt * (1.0 - xi);
                    /* trial point for the P1 weights: midpoint of the t-range */
                    double tlo = p > q - u ? p : q - u;
                    double thi = u > 0.0 ? 1.0 - u : 1.0;
                    double tm = 0.5 * (tlo + thi);
                    accum(op, mag, d, ny, sc, wgt, pb, tm + u, q, acc);
                }
    }
    for (int k = 0; k < 3; ++k) out[k] += g * acc[k];
}

/* ---- common vertex --------------------------------------------------------- */
/* Shared vertex P0.  Split on which of xh1, yh1 is larger; the larger one is
 * xi and the other triangle is the Duffy image of the unit square scaled by
 * xi: xh = xi (1, w), yh = xi (e1, e1 e2) (and swapped), weight xi^3 e1. */
static void pair_vertex(const orc_mesh *m, int op, int mag, int64_t ti, int64_t tj, const param_tri *pa,
                        const param_tri *pb, cplx sc, int ng, const double *gx, const double *gw,
                        cplx *out) {
    double g = 4.0 * m->area[ti] * m->area[tj];
    const double *ny = m->nrm + 3 * (op == ORC_ADLP ? ti : tj);
    cplx acc[3] = {0, 0, 0};
    for (int reg = 0; reg < 2; ++reg)
        for (int a = 0; a < ng; ++a)
            for (int b = 0; b < ng; ++b)
                for (int cidx = 0; cidx < ng; ++cidx)
                    for (int dd = 0; dd < ng; ++dd) {
                        double xi = gx[a], w = gx[b], e1 = gx[cidx], e2 = gx[dd];
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
                        double x[3], y[3], d[3];
                        chi(pa, x1, x2, x);
                        chi(pb, y1, y2, y);
                        sub3(y, x, d);
                        double wgt = gw[a] * gw[b] * gw[cidx] * gw[dd] * xi * xi * xi * e1;
                        accum(op, mag, d, ny, sc, wgt, pb, y1, y2, acc);
                    }
    for (int k = 0; k < 3; ++k) out[k] += g * acc[k];
}

/* ---- regular pairs: 7 x 7 rule --------------------------------------------- */
static void pair_regular(const orc_mesh *m, int op, int mag, int64_t ti, int64_t tj, cplx sc, cplx *out) {
    double bary[7][3], w[7];
    orc_rule7(&bary[0][0], w);
    const double *ny = m->nrm + 3 * tj, *nx = m->nrm + 3 * ti;
    const int32_t *A = m->t + 3 * ti, *B = m->t + 3 * tj;
    double scale = m->area[ti] * m->area[tj];
    for (int a = 0; a < 7; ++a) {
        double x[3] = {0, 0, 0};
        for (int k = 0; k < 3; ++k)
            for (int c = 0; c < 3; ++c) x[c] += bary[a][k] * m->v[3 * A[k] + c];
        for (int b = 0; b < 7; ++b) {
            double y[3] = {0, 0, 0}, d[3];
            for (int k = 0; k < 3; ++k)
                for (int c = 0; c < 3; ++c) y[c] += bary[b][k] * m->v[3 * B[k] + c];
            sub3(y, x, d);
            double wgt = w[a] * w[b] * scale;
            if (op == ORC_SLP) {
                out[0] += mag ? wgt * k_slp_mag(d, sc) : wgt * k_slp(d, sc);
            } else if (op == ORC_ADLP) {
                out[0] += mag ? wgt * k_dlp_mag(d, sc) : wgt * k_adlp(d, nx, sc);
            } else {
                cplx k = mag ? wgt * k_dlp_mag(d, sc) : wgt * k_dlp(d, ny, sc);
                for (int q = 0; q < 3; ++q) out[q] += k * bary[b][q];
            }
        }
    }
}

void orc_pair_regular(const orc_mesh *m, int op, int64_t ti, int64_t tj, double s_re,
                      double s_im, double c, double *o) {
    cplx out[3] = {0, 0, 0};
    pair_regular(m, op, 0, ti, tj, (s_re + I * s_im) / c, out);
    for (int k = 0; k < 3; ++k) {
        o[2 * k] = creal(out[k]);
        o[2 * k + 1] = cimag(out[k]);
    }
}

/* Pair integral (mag = 0) or its magnitude sum (mag = 1) into out[3]. */
static int pair_any(const orc_mesh *m, int op, int mag, int64_t ti, int64_t tj, cplx sc, int ng, cplx *out) {
    /* the Galerkin single layer is symmetric: integrate each unordered pair
     * once, in the order (lower index, higher index) */
    if (op == ORC_SLP && ti > tj) {
        int64_t t = ti;
        ti = tj;
        tj = t;
    }
    param_tri pa, pb;
    int cls = classify(m, ti, tj, &pa, &pb);
    double gx[64], gw[64];
    if (cls > 0 && orc_gauss01(ng, gx, gw) != 0) return -1;
    switch (cls) {
    case 3:
        /* flat panel: (x - y).n = 0, the double layer and its adjoint vanish identically */
        if (op == ORC_SLP) pair_identical(m, op, mag, ti, &pa, sc, ng, gx, gw, out);
        break;
    case 2: pair_edge(m, op, mag, ti, tj, &pa, &pb, sc, ng, gx, gw, out); break;
    case 1: pair_vertex(m, op, mag, ti, tj, &pa, &pb, sc, ng, gx, gw, out); break;
    default: pair_regular(m, op, mag, ti, tj, sc, out); break;
    }
    return cls;
}

int orc_pair(const orc_mesh *m, int op, int64_t ti, int64_t tj, double s_re, double s_im,
             double c, int ng, double *o) {
    cplx out[3] = {0, 0, 0};
    int cls = pair_any(m, op, 0, ti, tj, (s_re + I * s_im) / c, ng, out);
    for (int k = 0; k < 3; ++k) {
        o[2 * k] = creal(out[k]);
        o[2 * k + 1] = cimag(out[k]);
    }
    return cls;
}

void orc_entry(const orc_mesh *m, int op, int64_t row, int64_t col, double s_re, double s_im,
               double c, int ng, double *o) {
    double acc_re = 0.0, acc_im = 0.0, pr[6];
    if (op == ORC_SLP || op == ORC_ADLP) {
        orc_pair(m, op, row, col, s_re, s_im, c, ng, pr);
        acc_re = pr[0];
        acc_im = pr[1];
    } else {
        /* P1 column: sum over the triangles of the vertex's support */
        for (int64_t p = m->v2t_ptr[col]; p < m->v2t_ptr[col + 1]; ++p) {
            orc_pair(m, op, row, m->v2t[p], s_re, s_im, c, ng, pr);
            int l = m->v2t_loc[p];
            acc_re += pr[2 * l];
            acc_im += pr[2 * l + 1];
        }
    }
    o[0] = acc_re;
    o[1] = acc_im;
}

void orc_entries(const orc_mesh *m, int op, const int32_t *rows, int64_t nr, const int32_t *cols,
                 int64_t nc, const double *s, int64_t nf, double c, int ng, double *out) {
#pragma omp parallel for collapse(2) schedule(dynamic, 4)
    for (int64_t f = 0; f < nf; ++f)
        for (int64_t r = 0; r < nr; ++r)
            for (int64_t q = 0; q < nc; ++q)
                orc_entry(m, op, rows[r], cols[q], s[2 * f], s[2 * f + 1], c, ng,
                          out + 2 * ((f * nr + r) * nc + q));
}

/* Magnitude sum of an entry: the same quadrature (7 x 7 rule or
 * Sauter-Schwab points, same weights and P1 hat weights) with every term
 * replaced by a bound of its modulus, |exp(-s r/c)| / (4 pi r) for the single
 * layer and |exp(-s r/c)(1 + s r/c)| / (4 pi r^2) for the double layer (the
 * factor |(x - y).n_y| bounded by |x - y|). */
static double entry_mag(const orc_mesh *m, int op, int64_t row, int64_t col, cplx sc, int ng) {
    if (op == ORC_SLP || op == ORC_ADLP) {
        cplx out[3] = {0, 0, 0};
        pair_any(m, op, 1, row, col, sc, ng, out);
        return creal(out[0]);
    }
    double acc = 0.0;
    for (int64_t p = m->v2t_ptr[col]; p < m->v2t_ptr[col + 1]; ++p) {
        cplx out[3] = {0, 0, 0};
        pair_any(m, op, 1, row, m->v2t[p], sc, ng, out);
        acc += creal(out[m->v2t_loc[p]]);
    }
    return acc;
}

void orc_entries_mag(const orc_mesh *m, int op, const int32_t *rows, int64_t nr, const int32_t *cols,
                     int64_t nc, const double *s, int64_t nf, double c, int ng, double *out) {
#pragma omp parallel for collapse(2) schedule(dynamic, 4)
    for (int64_t f = 0; f < nf; ++f)
        for (int64_t r = 0; r < nr; ++r)
            for (int64_t q = 0; q < nc; ++q)
                out[(f * nr + r) * nc + q] = entry_mag(m, op, rows[r], cols[q], (s[2 * f] + I * s[2 * f + 1]) / c, ng);
}
