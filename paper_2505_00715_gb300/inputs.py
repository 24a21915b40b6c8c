"""Seeded synthetic inputs shared by the library's tests, the bench and the oracle checks.

This module holds input generation only (meshes, random right-hand sides and
time-step sequences) and none of the method's arithmetic.  It imports neither
the CUDA binding nor the oracle.

Meshes are flat-triangle surfaces with counter-clockwise triangles seen from
outside (outward normals), vertices as float64 [nv, 3], triangles int32 [nt, 3].
"""
import math

import numpy as np

__all__ = ["icosahedron", "octahedron", "icosphere", "housing", "cube", "random_weights", "graded_steps"]


def octahedron(R=1.0):
    v = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], dtype=np.float64)
    t = np.array([[0, 2, 4], [2, 1, 4], [1, 3, 4], [3, 0, 4],
                  [2, 0, 5], [1, 2, 5], [3, 1, 5], [0, 3, 5]], dtype=np.int32)
    return R * v, t


def icosahedron(R=1.0):
    p = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array([[-1, p, 0], [1, p, 0], [-1, -p, 0], [1, -p, 0],
                  [0, -1, p], [0, 1, p], [0, -1, -p], [0, 1, -p],
                  [p, 0, -1], [p, 0, 1], [-p, 0, -1], [-p, 0, 1]], dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    t = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
                  [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
                  [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
                  [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int32)
    return R * v, _orient_outward(R * v, t)


def _orient_outward(v, t):
    """Flip triangles whose normal points towards the origin (star-shaped surfaces)."""
    a, b, c = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    n = np.cross(b - a, c - a)
    flip = np.einsum("ij,ij->i", n, (a + b + c) / 3.0) < 0
    t = t.copy()
    t[flip] = t[flip][:, [0, 2, 1]]
    return t


def icosphere(level, R=1.0):
    """Icosahedron subdivided 4-to-1 `level` times (midpoints cached by the
    sorted vertex pair) and projected to the sphere of radius R:
    20 * 4**level triangles, 10 * 4**level + 2 vertices."""
    v, t = icosahedron(1.0)
    verts = [tuple(x) for x in v]
    tris = [tuple(x) for x in t]
    for _ in range(level):
        cache = {}
        new = []

        def mid(i, j):
            key = (i, j) if i < j else (j, i)
            k = cache.get(key)
            if k is None:
                m = (np.asarray(verts[i]) + np.asarray(verts[j])) * 0.5
                m /= np.linalg.norm(m)
                verts.append(tuple(m))
                k = len(verts) - 1
                cache[key] = k
            return k

        for (a, b, c) in tris:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            new += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        tris = new
    V = np.array(verts, dtype=np.float64) * R
    T = np.array(tris, dtype=np.int32)
    return V, _orient_outward(V, T)


def _outline(radius, nfins, fin_h, fin_t, n_arc):
    """Closed polygon of a circle of `radius` with `nfins` radial fins of
    height fin_h and thickness fin_t (counter-clockwise, z = 0)."""
    pts = []
    half = math.asin(min(0.99, fin_t / (2.0 * radius)))
    for f in range(nfins):
        th0 = 2.0 * math.pi * f / nfins
        th1 = 2.0 * math.pi * (f + 1) / nfins
        # fin at th0: left flank, tip, right flank (counter-clockwise order)
        a0 = th0 + half
        # flank points at the fin root (angle th0 +/- half) and tip
        pts.append(((radius + fin_h) * math.cos(th0) + fin_t / 2 * math.sin(th0),
                    (radius + fin_h) * math.sin(th0) - fin_t / 2 * math.cos(th0)))
        pts.append(((radius + fin_h) * math.cos(th0) - fin_t / 2 * math.sin(th0),
                    (radius + fin_h) * math.sin(th0) + fin_t / 2 * math.cos(th0)))
        # arc from this fin's left root to the next fin's right root
        a1 = th1 - half
        for k in range(n_arc + 1):
            th = a0 + (a1 - a0) * k / n_arc
            pts.append((radius * math.cos(th), radius * math.sin(th)))
    return np.array(pts, dtype=np.float64)


def _zipper(outer, oang, inner, iang, emit):
    """Triangulate the annulus between two closed rings of vertex ids whose
    polar angles (`oang`, `iang`, increasing, unwrapped, first angles within
    one step of each other) go once around: advance on the side whose next
    angle comes first."""
    no, ni = len(outer), len(inner)
    i = j = 0
    while i < no or j < ni:
        to = oang[(i + 1) % no] + (2 * math.pi if i + 1 >= no else 0.0)
        tn = iang[(j + 1) % ni] + (2 * math.pi if j + 1 >= ni else 0.0)
        if j >= ni or (i < no and to <= tn):
            emit(outer[i % no], outer[(i + 1) % no], inner[j % ni])
            i += 1
        else:
            emit(outer[i % no], inner[(j + 1) % ni], inner[j % ni])
            j += 1


def _cap_counts(n_disk, nrings):
    """Points of the end-cap rings: ring 0 is the outline's circle part
    (n_disk points), ring r >= 1 a circle of relative size 1 - r/nrings with
    proportionally fewer points."""
    return [n_disk] + [max(6, int(round(n_disk * (1.0 - r / nrings)))) for r in range(1, nrings)]


def housing(n_target, radius=0.1, length=0.3, nfins=12, fin_h=0.015, fin_t=0.005, jitter=0.01, seed=0):
    """Synthetic electric-machine housing: a closed finned cylinder along z.

    The cross-section is a circle with `nfins` radial fins; it is extruded
    over `length` and closed by flat end caps.  In a cap, every fin's cross
    section is split into two triangles and the disk inside the fin roots is
    triangulated in rings of points on concentric circles, each ring with a
    number of points proportional to its radius, neighbouring rings joined
    by angle (no sliver triangles).  The resolution is chosen so that the
    triangle count is close to `n_target`.  Every vertex is moved by a
    seeded uniform random offset in a ball of radius `jitter` times the mean
    edge length (flat end caps and fins stay closed because only vertex
    positions move)."""
    best = None
    for n_arc in range(2, 400):
        out = _outline(radius, nfins, fin_h, fin_t, n_arc)
        P = len(out)
        perim = np.sum(np.linalg.norm(np.roll(out, -1, axis=0) - out, axis=1))
        h = perim / P
        nz = max(2, int(round(length / h)))
        nrings = max(1, int(round(radius / h)))
        cnt = _cap_counts(P - 2 * nfins, nrings)
        ntri = 2 * P * nz + 2 * (2 * nfins + sum(cnt[r] + cnt[r + 1] for r in range(nrings - 1)) + cnt[-1])
        if best is None or abs(ntri - n_target) < abs(best[0] - n_target):
            best = (ntri, n_arc, nz, nrings)
        if ntri > 1.3 * n_target:
            break
    _, n_arc, nz, nrings = best
    out = _outline(radius, nfins, fin_h, fin_t, n_arc)
    P = len(out)
    per_fin = n_arc + 3  # two tip points, then the arc to the next fin
    verts = []
    tris = []
    # side wall: layers k = 0..nz
    for k in range(nz + 1):
        z = -length / 2 + length * k / nz
        for p in range(P):
            verts.append((out[p, 0], out[p, 1], z))

    def vid(k, p):
        return k * P + (p % P)
    for k in range(nz):
        for p in range(P):
            a, b, c, d = vid(k, p), vid(k, p + 1), vid(k + 1, p + 1), vid(k + 1, p)
            tris.append((a, b, c))
            tris.append((a, c, d))
    disk = [p for p in range(P) if p % per_fin >= 2]       # outline points on the circle
    disk_ang = np.unwrap([math.atan2(out[p, 1], out[p, 0]) for p in disk])
    cnt = _cap_counts(len(disk), nrings)
    for cap, k in ((0, 0), (1, nz)):
        z = -length / 2 + length * k / nz

        def emit(a, b, c):
            # cap 1 (z = +L/2) keeps (a, b, c); cap 0 is seen from the other side
            tris.append((a, b, c) if cap == 1 else (a, c, b))
        # fin cross sections: (right root, tip 1, tip 2, left root)
        for f in range(nfins):
            t1, t2, rl = f * per_fin, f * per_fin + 1, f * per_fin + 2
            rr = (f * per_fin - 1) % P
            emit(vid(k, rr), vid(k, t1), vid(k, t2))
            emit(vid(k, rr), vid(k, t2), vid(k, rl))
        # disk rings
        ids = [[vid(k, p) for p in disk]]
        angs = [disk_ang]
        for r in range(1, nrings):
            rad = radius * (1.0 - r / nrings)
            n = cnt[r]
            th = disk_ang[0] + 2 * math.pi * np.arange(n) / n
            cur = []
            for t in th:
                verts.append((rad * math.cos(t), rad * math.sin(t), z))
                cur.append(len(verts) - 1)
            ids.append(cur)
            angs.append(th)
        verts.append((0.0, 0.0, z))
        centre = len(verts) - 1
        for r in range(nrings - 1):
            _zipper(ids[r], angs[r], ids[r + 1], angs[r + 1], emit)
        last = ids[-1]
        for i in range(len(last)):
            emit(last[i], last[(i + 1) % len(last)], centre)
    V = np.array(verts, dtype=np.float64)
    T = np.array(tris, dtype=np.int32)
    if jitter > 0:
        rng = np.random.default_rng(seed)
        e = np.concatenate([T[:, [0, 1]], T[:, [1, 2]], T[:, [2, 0]]])
        h = np.mean(np.linalg.norm(V[e[:, 0]] - V[e[:, 1]], axis=1))
        d = rng.normal(size=V.shape)
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        rad = jitter * h * rng.random(len(V)) ** (1.0 / 3.0)
        V = V + d * rad[:, None]
    return V, T


def cube(level, L=1.0):
    """Cube [-L/2, L/2]^3 (the paper's unit cube, Sec. 5): level 1 splits
    every face into 2 x 2 squares and every square into 4 triangles at its
    centre (96 triangles, 50 vertices, h = L/2); each further level splits
    every triangle into 4 at its edge midpoints (384 / 194, 1536 / 770, ...)."""
    verts, index = [], {}

    def vid(p):
        key = tuple(np.round(np.asarray(p) * 2 ** 20).astype(np.int64))
        if key not in index:
            index[key] = len(verts)
            verts.append(np.asarray(p, dtype=np.float64))
        return index[key]

    tris = []
    h = L / 2.0
    for axis in range(3):
        for sign in (-1.0, 1.0):
            u, w = [(axis + 1) % 3, (axis + 2) % 3]
            for a in range(2):
                for b in range(2):
                    def pt(x, y):
                        p = np.zeros(3)
                        p[axis] = sign * h
                        p[u] = -h + x * h
                        p[w] = -h + y * h
                        return p
                    c = vid(pt(a + 0.5, b + 0.5))
                    q = [vid(pt(a, b)), vid(pt(a + 1, b)), vid(pt(a + 1, b + 1)), vid(pt(a, b + 1))]
                    for k in range(4):
                        tris.append((q[k], q[(k + 1) % 4], c))
    V = np.array(verts)
    T = np.array(tris, dtype=np.int32)
    for _ in range(level - 1):
        cache, new = {}, []

        def mid(i, j):
            key = (i, j) if i < j else (j, i)
            if key not in cache:
                cache[key] = len(V_l)
                V_l.append(0.5 * (V_l[i] + V_l[j]))
            return cache[key]
        V_l = list(V)
        for a, b, c in T:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            new += [(a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca)]
        V, T = np.array(V_l), np.array(new, dtype=np.int32)
    # outward orientation: the normal points away from the cube's centre
    a, b, c = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    n = np.cross(b - a, c - a)
    flip = np.einsum("ij,ij->i", n, (a + b + c) / 3.0) < 0
    T[flip] = T[flip][:, [0, 2, 1]]
    return V, T


def random_weights(nf, n, nrhs, seed=1, dtype=np.complex128):
    """Seeded complex Gaussian weights W[nf, n, nrhs] (unit variance per component)."""
    rng = np.random.default_rng(seed)
    W = rng.standard_normal((nf, n, nrhs)) + 1j * rng.standard_normal((nf, n, nrhs))
    return W.astype(dtype)


def graded_steps(N, ratio, T):
    """N geometrically graded time steps dt_i = dt_1 ratio^(i-1) summing to T."""
    dt1 = T * (ratio - 1.0) / (ratio ** N - 1.0) if ratio != 1.0 else T / N
    return dt1 * ratio ** np.arange(N)
