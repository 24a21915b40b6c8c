/*
 * Oracle (test infrastructure only): cluster tree and block cluster tree.
 *
 * Sec. 4 ("The face is an H-matrix"): the index set is split recursively into
 * two sons by principal component analysis, giving a balanced cluster tree;
 * a block of clusters (Cl_x, Cl_y) is admissible (far field, low rank) when
 *   min{diam(Cl_x), diam(Cl_y)} <= eta dist(Cl_x, Cl_y)      (eq. admissible)
 * and near field (dense) otherwise.
 *
 * Readings where the text is silent (the library's planner follows the same
 * steps so that both trees agree bit for bit; compile with -ffp-contract=off):
 *   - DOF points: triangle centroids ((v0 + v1) + v2) / 3 for P0, vertices
 *     for P1; a cluster's box is the axis-aligned box of the vertices of the
 *     supports of its DOFs; diam = box diagonal, dist = distance of the boxes;
 *   - a cluster of n DOFs is split iff n > leaf, at position floor(n/2) of
 *     the DOFs sorted by (projection on the principal axis, DOF index);
 *   - principal axis: eigenvector of the largest eigenvalue of the scatter
 *     matrix sum (p - mean)(p - mean)^T (sums in ascending cluster position),
 *     by 10 cyclic Jacobi sweeps, sign fixed so that its largest-magnitude
 *     component (lowest index on ties) is positive;
 *   - far iff dist > 0 and the criterion holds; near iff not far and either
 *     cluster is a leaf; otherwise recurse into the son pairs (0,0), (0,1),
 *     (1,0), (1,1); blocks are listed in that depth-first order.
 */
#include "orc.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t begin, end, son0, son1;
    double box[6]; /* lo xyz, hi xyz */
} node;

typedef struct {
    int64_t n;
    double *pt;      /* [n][3] DOF points */
    int64_t *sup_ptr; /* support vertices per DOF (CSR) */
    int32_t *sup;
    const double *verts;
    int32_t *perm;
    node *nodes;
    int64_t nnodes, cap;
} ctree;

struct orc_tree {
    ctree side[2];
    int32_t *blocks; /* [nb][5] */
    int64_t nb, capb;
};

/* read-only view of the mesh arrays (defined in orc_geom.c) */
void orc_mesh_view(const orc_mesh *m, int64_t *nv, int64_t *nt, const double **v,
                   const int32_t **t);

static void ctree_points(const orc_mesh *m, int basis, ctree *t) {
    int64_t nv, nt;
    const double *v;
    const int32_t *tr;
    orc_mesh_view(m, &nv, &nt, &v, &tr);
    t->verts = v;
    if (basis == ORC_P0) {
        t->n = nt;
        t->pt = malloc(sizeof(double) * 3 * nt);
        t->sup_ptr = malloc(sizeof(int64_t) * (nt + 1));
        t->sup = malloc(sizeof(int32_t) * 3 * nt);
        for (int64_t e = 0; e < nt; ++e) {
            const double *a = v + 3 * tr[3 * e], *b = v + 3 * tr[3 * e + 1],
                         *c = v + 3 * tr[3 * e + 2];
            for (int k = 0; k < 3; ++k) t->pt[3 * e + k] = ((a[k] + b[k]) + c[k]) / 3.0;
            t->sup_ptr[e] = 3 * e;
            for (int k = 0; k < 3; ++k) t->sup[3 * e + k] = tr[3 * e + k];
        }
        t->sup_ptr[nt] = 3 * nt;
    } else {
        t->n = nv;
        t->pt = malloc(sizeof(double) * 3 * nv);
        memcpy(t->pt, v, sizeof(double) * 3 * nv);
        /* support of the hat of vertex p: all vertices of triangles containing p */
        int64_t *cnt = calloc(nv + 1, sizeof(int64_t));
        for (int64_t e = 0; e < 3 * nt; ++e) cnt[tr[e] + 1] += 3;
        for (int64_t p = 0; p < nv; ++p) cnt[p + 1] += cnt[p];
        t->sup_ptr = cnt;
        t->sup = malloc(sizeof(int32_t) * cnt[nv]);
        int64_t *fill = calloc(nv, sizeof(int64_t));
        for (int64_t e = 0; e < nt; ++e)
            for (int k = 0; k < 3; ++k) {
                int32_t p = tr[3 * e + k];
                for (int q = 0; q < 3; ++q) t->sup[cnt[p] + fill[p]++] = tr[3 * e + q];
            }
        free(fill);
    }
}

/* cyclic Jacobi on a symmetric 3x3; returns the eigenvector of the largest
 * eigenvalue in axis[3] */
static void principal_axis(double a[3][3], double axis[3]) {
    double V[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    static const int PQ[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    for (int sweep = 0; sweep < 10; ++sweep)
        for (int r = 0; r < 3; ++r) {
            int p = PQ[r][0], q = PQ[r][1];
            if (a[p][q] == 0.0) continue;
            double tau = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
            double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            double c = 1.0 / sqrt(1.0 + t * t);
            double s = t * c;
            double app = a[p][p], aqq = a[q][q], apq = a[p][q];
            for (int k = 0; k < 3; ++k) {
                if (k == p || k == q) continue;
                double akp = a[k][p], akq = a[k][q];
                a[k][p] = a[p][k] = c * akp - s * akq;
                a[k][q] = a[q][k] = s * akp + c * akq;
            }
            a[p][p] = (c * c) * app - (2.0 * c * s) * apq + (s * s) * aqq;
            a[q][q] = (s * s) * app + (2.0 * c * s) * apq + (c * c) * aqq;
            a[p][q] = a[q][p] = 0.0;
            for (int k = 0; k < 3; ++k) {
                double vkp = V[k][p], vkq = V[k][q];
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
        if (fabs(axis[k]) > fabs(axis[big])) big = k;
    if (axis[big] < 0.0)
        for (int k = 0; k < 3; ++k) axis[k] = -axis[k];
}

typedef struct {
    double key;
    int32_t idx;
} keyed;

static int cmp_keyed(const void *x, const void *y) {
    const keyed *a = x, *b = y;
    if (a->key < b->key) return -1;
    if (a->key > b->key) return 1;
    return (a->idx > b->idx) - (a->idx < b->idx);
}

static int32_t new_node(ctree *t, int32_t b, int32_t e) {
    if (t->nnodes == t->cap) {
        t->cap = t->cap ? 2 * t->cap : 64;
        t->nodes = realloc(t->nodes, sizeof(node) * t->cap);
    }
    node *nd = &t->nodes[t->nnodes];
    nd->begin = b;
    nd->end = e;
    nd->son0 = nd->son1 = -1;
    for (int k = 0; k < 3; ++k) {
        nd->box[k] = INFINITY;
        nd->box[3 + k] = -INFINITY;
    }
    for (int32_t pos = b; pos < e; ++pos) {
        int32_t d = t->perm[pos];
        for (int64_t s = t->sup_ptr[d]; s < t->sup_ptr[d + 1]; ++s) {
            const double *x = t->verts + 3 * t->sup[s];
            for (int k = 0; k < 3; ++k) {
                if (x[k] < nd->box[k]) nd->box[k] = x[k];
                if (x[k] > nd->box[3 + k]) nd->box[3 + k] = x[k];
            }
        }
    }
    return (int32_t)(t->nnodes++);
}

static void split(ctree *t, int32_t id, int leaf) {
    int32_t b = t->nodes[id].begin, e = t->nodes[id].end, n = e - b;
    if (n <= leaf) return;
    double mean[3] = {0, 0, 0};
    for (int32_t pos = b; pos < e; ++pos)
        for (int k = 0; k < 3; ++k) mean[k] += t->pt[3 * t->perm[pos] + k];
    for (int k = 0; k < 3; ++k) mean[k] /= (double)n;
    double C[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int32_t pos = b; pos < e; ++pos) {
        const double *p = t->pt + 3 * t->perm[pos];
        double d[3] = {p[0] - mean[0], p[1] - mean[1], p[2] - mean[2]};
        for (int x = 0; x < 3; ++x)
            for (int y = 0; y < 3; ++y) C[x][y] += d[x] * d[y];
    }
    double axis[3];
    principal_axis(C, axis);
    keyed *ks = malloc(sizeof(keyed) * n);
    for (int32_t pos = b; pos < e; ++pos) {
        const double *p = t->pt + 3 * t->perm[pos];
        double pr = (p[0] - mean[0]) * axis[0] + (p[1] - mean[1]) * axis[1] +
                    (p[2] - mean[2]) * axis[2];
        ks[pos - b].key = pr;
        ks[pos - b].idx = t->perm[pos];
    }
    qsort(ks, n, sizeof(keyed), cmp_keyed);
    for (int32_t k = 0; k < n; ++k) t->perm[b + k] = ks[k].idx;
    free(ks);
    int32_t mid = b + n / 2;
    int32_t s0 = new_node(t, b, mid);
    int32_t s1 = new_node(t, mid, e);
    t->nodes[id].son0 = s0;
    t->nodes[id].son1 = s1;
    split(t, s0, leaf);
    split(t, s1, leaf);
}

static void ctree_build(const orc_mesh *m, int basis, int leaf, ctree *t) {
    memset(t, 0, sizeof *t);
    ctree_points(m, basis, t);
    t->perm = malloc(sizeof(int32_t) * t->n);
    for (int64_t k = 0; k < t->n; ++k) t->perm[k] = (int32_t)k;
    int32_t root = new_node(t, 0, (int32_t)t->n);
    split(t, root, leaf);
}

static double diam(const node *a) {
    double s = 0.0;
    for (int k = 0; k < 3; ++k) {
        double d = a->box[3 + k] - a->box[k];
        s += d * d;
    }
    return sqrt(s);
}

static double dist(const node *a, const node *b) {
    double s = 0.0;
    for (int k = 0; k < 3; ++k) {
        double g = 0.0;
        if (b->box[k] - a->box[3 + k] > g) g = b->box[k] - a->box[3 + k];
        if (a->box[k] - b->box[3 + k] > g) g = a->box[k] - b->box[3 + k];
        s += g * g;
    }
    return sqrt(s);
}

static void push_block(orc_tree *T, const node *a, const node *b, int far) {
    if (T->nb == T->capb) {
        T->capb = T->capb ? 2 * T->capb : 256;
        T->blocks = realloc(T->blocks, sizeof(int32_t) * 5 * T->capb);
    }
    int32_t *o = T->blocks + 5 * T->nb++;
    o[0] = a->begin;
    o[1] = a->end;
    o[2] = b->begin;
    o[3] = b->end;
    o[4] = far;
}

static void block_rec(orc_tree *T, int32_t ia, int32_t ib, double eta) {
    const node *a = &T->side[0].nodes[ia], *b = &T->side[1].nodes[ib];
    double da = diam(a), db = diam(b), ds = dist(a, b);
    double dmin = da < db ? da : db;
    if (ds > 0.0 && dmin <= eta * ds) {
        push_block(T, a, b, 1);
        return;
    }
    if (a->son0 < 0 || b->son0 < 0) {
        push_block(T, a, b, 0);
        return;
    }
    int32_t sa[2] = {a->son0, a->son1}, sb[2] = {b->son0, b->son1};
    for (int x = 0; x < 2; ++x)
        for (int y = 0; y < 2; ++y) block_rec(T, sa[x], sb[y], eta);
}

orc_tree *orc_tree_build(const orc_mesh *m, int row_basis, int col_basis, int leaf, double eta) {
    if (leaf < 1 || !(eta > 0.0)) return NULL;
    orc_tree *T = calloc(1, sizeof *T);
    ctree_build(m, row_basis, leaf, &T->side[0]);
    ctree_build(m, col_basis, leaf, &T->side[1]);
    block_rec(T, 0, 0, eta);
    return T;
}

void orc_tree_free(orc_tree *T) {
    if (!T) return;
    for (int s = 0; s < 2; ++s) {
        free(T->side[s].pt);
        free(T->side[s].sup_ptr);
        free(T->side[s].sup);
        free(T->side[s].perm);
        free(T->side[s].nodes);
    }
    free(T->blocks);
    free(T);
}

int64_t orc_tree_nblocks(const orc_tree *T) { return T->nb; }

void orc_tree_export(const orc_tree *T, int32_t *perm_rows, int32_t *perm_cols, int32_t *blocks) {
    if (perm_rows) memcpy(perm_rows, T->side[0].perm, sizeof(int32_t) * T->side[0].n);
    if (perm_cols) memcpy(perm_cols, T->side[1].perm, sizeof(int32_t) * T->side[1].n);
    if (blocks) memcpy(blocks, T->blocks, sizeof(int32_t) * 5 * T->nb);
}

int64_t orc_tree_nclusters(const orc_tree *T, int side) { return T->side[side].nnodes; }

void orc_tree_clusters(const orc_tree *T, int side, int32_t *nodes, double *bbox) {
    const ctree *t = &T->side[side];
    for (int64_t k = 0; k < t->nnodes; ++k) {
        nodes[4 * k] = t->nodes[k].begin;
        nodes[4 * k + 1] = t->nodes[k].end;
        nodes[4 * k + 2] = t->nodes[k].son0;
        nodes[4 * k + 3] = t->nodes[k].son1;
        memcpy(bbox + 6 * k, t->nodes[k].box, sizeof(double) * 6);
    }
}

/* internal: perm of a side and block list, used by the compressor */
const int32_t *orc_tree_perm(const orc_tree *T, int side) { return T->side[side].perm; }
const int32_t *orc_tree_blocks(const orc_tree *T) { return T->blocks; }
