// Host planner of the tdbem library: element adjacency, quadrature rules,
// the PCA cluster trees and the block cluster tree (Sec. 4, eq. admissible).
//
// The trees are built in IEEE FP64 using only +, -, *, / and sqrt in a fixed
// order (this file is compiled with -ffp-contract=off), so the result is
// reproducible bit for bit:
//   - DOF points: triangle centroids ((v0 + v1) + v2) / 3 (P0), vertices (P1);
//   - cluster box: axis-aligned box of the vertices of the DOF supports;
//   - split iff n > leaf: sort the DOFs by (projection of p - mean on the
//     principal axis, DOF index) and cut at floor(n/2); the principal axis is
//     the eigenvector of the largest eigenvalue of sum (p - mean)(p - mean)^T,
//     from ten cyclic Jacobi sweeps, signed so that its largest-magnitude
//     component is positive;
//   - block (tau, sigma): far iff dist > 0 and min(diam) <= eta dist (box
//     diagonal, box distance), else near iff either is a leaf, else the four
//     son pairs (0,0), (0,1), (1,0), (1,1) in this order.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.h"

void td_rule7(double bary[7][3], double w[7]) {
    // Radon's degree-5 rule: centroid and two orbits (a, a, 1-2a), (b, b, 1-2b),
    // a, b = (6 -/+ sqrt 15)/21, weights 9/40 and (155 -/+ sqrt 15)/1200.
    const double s15 = std::sqrt(15.0);
    const double a = (6.0 - s15) / 21.0, b = (6.0 + s15) / 21.0;
    const double wa = (155.0 - s15) / 1200.0, wb = (155.0 + s15) / 1200.0;
    const double pts[7][3] = {{1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0}, {a, a, 1.0 - 2.0 * a},
                              {a, 1.0 - 2.0 * a, a},             {1.0 - 2.0 * a, a, a},
                              {b, b, 1.0 - 2.0 * b},             {b, 1.0 - 2.0 * b, b},
                              {1.0 - 2.0 * b, b, b}};
    const double ww[7] = {9.0 / 40.0, wa, wa, wa, wb, wb, wb};
    for (int q = 0; q < 7; ++q) {
        for (int k = 0; k < 3; ++k) bary[q][k] = pts[q][k];
        w[q] = ww[q];
    }
}

// Gauss-Legendre nodes and weights on [0, 1]: roots of P_n by Newton's
// method from Chebyshev-like starting values; weight 2/((1-z^2) P_n'(z)^2)
// on [-1, 1], halved for [0, 1].
int td_gauss01(int n, double *x, double *w) {
    if (n < 1 || n > 32) return -1;
    const double pi = std::acos(-1.0);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(pi * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double pm = 1.0, p = z;
            for (int k = 2; k <= n; ++k) {
                double pn = ((2 * k - 1) * z * p - (k - 1) * pm) / k;
                pm = p;
                p = pn;
            }
            if (n == 1) pm = 1.0;
            dp = n * (z * p - pm) / (z * z - 1.0);
            double step = p / dp;
            z -= step;
            if (std::fabs(step) < 1e-16) {
                pm = 1.0;
                p = z;
                for (int k = 2; k <= n; ++k) {
                    double pn = ((2 * k - 1) * z * p - (k - 1) * pm) / k;
                    pm = p;
                    p = pn;
                }
                if (n == 1) pm = 1.0;
                dp = n * (z * p - pm) / (z * z - 1.0);
                break;
            }
        }
        x[i] = 0.5 * (1.0 - z);
        w[i] = 1.0 / ((1.0 - z * z) * dp * dp);
    }
    return 0;
}

void td_mesh_adjacency(tdbem_mesh *m) {
    const int64_t nv = m->nv, nt = m->nt;
    m->v2t_ptr.assign(nv + 1, 0);
    for (int64_t e = 0; e < 3 * nt; ++e) m->v2t_ptr[m->tris[e] + 1]++;
    for (int64_t v = 0; v < nv; ++v) m->v2t_ptr[v + 1] += m->v2t_ptr[v];
    m->v2t.assign(3 * nt, 0);
    m->v2t_loc.assign(3 * nt, 0);
    std::vector<int32_t> fill(nv, 0);
    for (int64_t e = 0; e < nt; ++e)
        for (int k = 0; k < 3; ++k) {
            int32_t v = m->tris[3 * e + k];
            int32_t p = m->v2t_ptr[v] + fill[v]++;
            m->v2t[p] = (int32_t)e;
            m->v2t_loc[p] = (int8_t)k;
        }
    // triangles sharing at least one vertex (the triangle itself included)
    m->tp_ptr.assign(nt + 1, 0);
    m->tp_tri.clear();
    std::vector<int32_t> tmp;
    for (int64_t e = 0; e < nt; ++e) {
        tmp.clear();
        for (int k = 0; k < 3; ++k) {
            int32_t v = m->tris[3 * e + k];
            for (int32_t p = m->v2t_ptr[v]; p < m->v2t_ptr[v + 1]; ++p) tmp.push_back(m->v2t[p]);
        }
        std::sort(tmp.begin(), tmp.end());
        tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
        m->tp_tri.insert(m->tp_tri.end(), tmp.begin(), tmp.end());
        m->tp_ptr[e + 1] = (int32_t)m->tp_tri.size();
    }
}

namespace {

struct Builder {
    const tdbem_mesh *m;
    int basis;
    std::vector<double> pt;            // [n][3]
    std::vector<int32_t> sup_ptr, sup; // support vertices
    HostTree *t;

    void points() {
        const int64_t nt = m->nt, nv = m->nv;
        const double *v = m->verts.data();
        const int32_t *tr = m->tris.data();
        if (basis == TDBEM_P0) {
            t->n = nt;
            pt.resize(3 * nt);
            sup_ptr.resize(nt + 1);
            sup.resize(3 * nt);
            for (int64_t e = 0; e < nt; ++e) {
                const double *a = v + 3 * tr[3 * e], *b = v + 3 * tr[3 * e + 1],
                             *c = v + 3 * tr[3 * e + 2];
                for (int k = 0; k < 3; ++k) pt[3 * e + k] = ((a[k] + b[k]) + c[k]) / 3.0;
                sup_ptr[e] = (int32_t)(3 * e);
                for (int k = 0; k < 3; ++k) sup[3 * e + k] = tr[3 * e + k];
            }
            sup_ptr[nt] = (int32_t)(3 * nt);
        } else {
            t->n = nv;
            pt.assign(v, v + 3 * nv);
            sup_ptr.assign(nv + 1, 0);
            for (int64_t p = 0; p < nv; ++p)
                sup_ptr[p + 1] = sup_ptr[p] + 3 * (m->v2t_ptr[p + 1] - m->v2t_ptr[p]);
            sup.resize(sup_ptr[nv]);
            for (int64_t p = 0; p < nv; ++p) {
                int32_t o = sup_ptr[p];
                for (int32_t q = m->v2t_ptr[p]; q < m->v2t_ptr[p + 1]; ++q)
                    for (int k = 0; k < 3; ++k) sup[o++] = tr[3 * m->v2t[q] + k];
            }
        }
    }

    int32_t node(int32_t b, int32_t e) {
        ClusterNode nd;
        nd.begin = b;
        nd.end = e;
        nd.son0 = nd.son1 = -1;
        for (int k = 0; k < 3; ++k) {
            nd.box[k] = INFINITY;
            nd.box[3 + k] = -INFINITY;
        }
        for (int32_t pos = b; pos < e; ++pos) {
            int32_t d = t->perm[pos];
            for (int32_t s = sup_ptr[d]; s < sup_ptr[d + 1]; ++s) {
                const double *x = m->verts.data() + 3 * sup[s];
                for (int k = 0; k < 3; ++k) {
                    nd.box[k] = std::min(nd.box[k], x[k]);
                    nd.box[3 + k] = std::max(nd.box[3 + k], x[k]);
                }
            }
        }
        t->nodes.push_back(nd);
        return (int32_t)t->nodes.size() - 1;
    }

    static void jacobi_axis(double a[3][3], double axis[3]) {
        double V[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
        const int P[3] = {0, 0, 1}, Q[3] = {1, 2, 2};
        for (int sweep = 0; sweep < 10; ++sweep)
            for (int r = 0; r < 3; ++r) {
                const int p = P[r], q = Q[r];
                if (a[p][q] == 0.0) continue;
                const double tau = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
                const double t = (tau >= 0.0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
                const double c = 1.0 / std::sqrt(1.0 + t * t);
                const double s = t * c;
                const double app = a[p][p], aqq = a[q][q], apq = a[p][q];
                for (int k = 0; k < 3; ++k) {
                    if (k == p || k == q) continue;
                    const double akp = a[k][p], akq = a[k][q];
                    a[k][p] = a[p][k] = c * akp - s * akq;
                    a[k][q] = a[q][k] = s * akp + c * akq;
                }
                a[p][p] = (c * c) * app - (2.0 * c * s) * apq + (s * s) * aqq;
                a[q][q] = (s * s) * app + (2.0 * c * s) * apq + (c * c) * aqq;
                a[p][q] = a[q][p] = 0.0;
                for (int k = 0; k < 3; ++k) {
                    const double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - s * vkq;
                    V[k][q] = s * vkp + c * vkq;
                }
            }
        int best = 0;
        for (int k = 1; k < 3; ++k)
            if (a[k][k] > a[best][best]) best = k;
        for (int k = 0; k < 3; ++k) axis[k] = V[k][best];
        int big = 0;
        for (int k = 1; k < 3; ++k)
            if (std::fabs(axis[k]) > std::fabs(axis[big])) big = k;
        if (axis[big] < 0.0)
            for (int k = 0; k < 3; ++k) axis[k] = -axis[k];
    }

    void split(int32_t id, int leaf) {
        const int32_t b = t->nodes[id].begin, e = t->nodes[id].end, n = e - b;
        if (n <= leaf) return;
        double mean[3] = {0.0, 0.0, 0.0};
        for (int32_t pos = b; pos < e; ++pos)
            for (int k = 0; k < 3; ++k) mean[k] += pt[3 * t->perm[pos] + k];
        for (int k = 0; k < 3; ++k) mean[k] /= (double)n;
        double C[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int32_t pos = b; pos < e; ++pos) {
            const double *p = &pt[3 * t->perm[pos]];
            const double d[3] = {p[0] - mean[0], p[1] - mean[1], p[2] - mean[2]};
            for (int x = 0; x < 3; ++x)
                for (int y = 0; y < 3; ++y) C[x][y] += d[x] * d[y];
        }
        double ax[3];
        jacobi_axis(C, ax);
        std::vector<std::pair<double, int32_t>> keys(n);
        for (int32_t pos = b; pos < e; ++pos) {
            const double *p = &pt[3 * t->perm[pos]];
            const double pr = (p[0] - mean[0]) * ax[0] + (p[1] - mean[1]) * ax[1] +
                              (p[2] - mean[2]) * ax[2];
            keys[pos - b] = {pr, t->perm[pos]};
        }
        std::sort(keys.begin(), keys.end());
        for (int32_t k = 0; k < n; ++k) t->perm[b + k] = keys[k].second;
        const int32_t mid = b + n / 2;
        const int32_t s0 = node(b, mid);
        const int32_t s1 = node(mid, e);
        t->nodes[id].son0 = s0;
        t->nodes[id].son1 = s1;
        split(s0, leaf);
        split(s1, leaf);
    }
};

double box_diam(const ClusterNode &a) {
    double s = 0.0;
    for (int k = 0; k < 3; ++k) {
        const double d = a.box[3 + k] - a.box[k];
        s += d * d;
    }
    return std::sqrt(s);
}

double box_dist(const ClusterNode &a, const ClusterNode &b) {
    double s = 0.0;
    for (int k = 0; k < 3; ++k) {
        double g = 0.0;
        if (b.box[k] - a.box[3 + k] > g) g = b.box[k] - a.box[3 + k];
        if (a.box[k] - b.box[3 + k] > g) g = a.box[k] - b.box[3 + k];
        s += g * g;
    }
    return std::sqrt(s);
}

void block_rec(const HostTree &R, const HostTree &Cc, int32_t ia, int32_t ib, double eta,
               std::vector<int32_t> &out) {
    const ClusterNode &a = R.nodes[ia], &b = Cc.nodes[ib];
    const double da = box_diam(a), db = box_diam(b), ds = box_dist(a, b);
    const double dmin = da < db ? da : db;
    int far = -1;
    if (ds > 0.0 && dmin <= eta * ds)
        far = 1;
    else if (a.son0 < 0 || b.son0 < 0)
        far = 0;
    if (far >= 0) {
        const int32_t blk[5] = {a.begin, a.end, b.begin, b.end, far};
        out.insert(out.end(), blk, blk + 5);
        return;
    }
    const int32_t sa[2] = {a.son0, a.son1}, sb[2] = {b.son0, b.son1};
    for (int x = 0; x < 2; ++x)
        for (int y = 0; y < 2; ++y) block_rec(R, Cc, sa[x], sb[y], eta, out);
}

}  // namespace

void td_plan_tree(const tdbem_mesh *m, int basis, int leaf, HostTree &t) {
    t = HostTree();
    t.basis = basis;
    Builder B{m, basis, {}, {}, {}, &t};
    B.points();
    t.perm.resize(t.n);
    for (int64_t k = 0; k < t.n; ++k) t.perm[k] = (int32_t)k;
    const int32_t root = B.node(0, (int32_t)t.n);
    B.split(root, leaf);
}

void td_plan_blocks(const HostTree &rows, const HostTree &cols, double eta,
                    std::vector<int32_t> &blocks) {
    blocks.clear();
    block_rec(rows, cols, 0, 0, eta, blocks);
}

// ---------------------------------------------------------------------------
// Compression partition for the persistent far phase: far blocks whose
// entry count exceeds twice the mean far work of one persistent CTA
// (total far entries / nctas) are replaced by the blocks of their clusters'
// sons (both sides where both have sons), recursively.  Sub-blocks of an
// admissible block are admissible (smaller boxes, larger distance), so the
// result is again an admissible partition; near blocks are kept.
namespace {
int node_of(const HostTree &t, int32_t b, int32_t e) {
    int id = 0;
    for (;;) {
        const ClusterNode &n = t.nodes[id];
        if (n.begin == b && n.end == e) return id;
        if (n.son0 < 0) return -1;
        id = (b < t.nodes[n.son0].end) ? n.son0 : n.son1;
    }
}

void split_far(const HostTree &R, const HostTree &C, int a, int b, double lim, std::vector<int32_t> &out) {
    const ClusterNode &x = R.nodes[a], &y = C.nodes[b];
    const double e = (double)(x.end - x.begin) * (double)(y.end - y.begin);
    const bool sx = x.son0 >= 0, sy = y.son0 >= 0;
    if (e <= lim || (!sx && !sy)) {
        const int32_t bl[5] = {x.begin, x.end, y.begin, y.end, 1};
        out.insert(out.end(), bl, bl + 5);
        return;
    }
    const int xs[2] = {sx ? x.son0 : a, sx ? x.son1 : -1};
    const int ys[2] = {sy ? y.son0 : b, sy ? y.son1 : -1};
    for (int p = 0; p < 2; ++p)
        for (int q = 0; q < 2; ++q)
            if (xs[p] >= 0 && ys[q] >= 0) split_far(R, C, xs[p], ys[q], lim, out);
}
}  // namespace

void td_balance_partition(const HostTree &R, const HostTree &C, const std::vector<int32_t> &blocks, int64_t nctas,
                          std::vector<int32_t> &out) {
    const size_t nb = blocks.size() / 5;
    double tot = 0.0;
    for (size_t b = 0; b < nb; ++b)
        if (blocks[5 * b + 4]) tot += (double)(blocks[5 * b + 1] - blocks[5 * b]) * (double)(blocks[5 * b + 3] - blocks[5 * b + 2]);
    const double lim = 2.0 * tot / (double)(nctas > 0 ? nctas : 1);
    out.clear();
    out.reserve(blocks.size());
    for (size_t b = 0; b < nb; ++b) {
        const int32_t *bl = &blocks[5 * b];
        const int a = bl[4] ? node_of(R, bl[0], bl[1]) : -1, c = bl[4] ? node_of(C, bl[2], bl[3]) : -1;
        if (a < 0 || c < 0)
            out.insert(out.end(), bl, bl + 5);
        else
            split_far(R, C, a, c, lim, out);
    }
}
