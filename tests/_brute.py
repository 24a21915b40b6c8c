"""Independent brute-force integrators used to pin the oracle (test-side only).

They use numpy's Gauss-Legendre nodes (a library routine) on collapsed
(Duffy) squares of recursively subdivided triangles, and the closed-form
potential of a uniformly charged flat triangle, so that none of the oracle's
own rules or transforms is reused.
"""
import numpy as np


def subdivide(P, level):
    """Split triangle P (3x3) into 4**level congruent sub-triangles."""
    tris = [np.asarray(P, dtype=np.float64)]
    for _ in range(level):
        nxt = []
        for a, b, c in tris:
            ab, bc, ca = (a + b) / 2, (b + c) / 2, (c + a) / 2
            nxt += [np.array([a, ab, ca]), np.array([ab, b, bc]), np.array([ca, bc, c]),
                    np.array([ab, bc, ca])]
        tris = nxt
    return tris


def collapsed_rule(P, level, n):
    """Points [m,3], weights [m] and barycentric coordinates [m,3] of a
    composite collapsed Gauss rule (n x n per sub-triangle) on triangle P."""
    g, w = np.polynomial.legendre.leggauss(n)
    g = 0.5 * (g + 1.0)
    w = 0.5 * w
    U, Vv = np.meshgrid(g, g, indexing="ij")
    WU = np.outer(w, w)
    pts, wts = [], []
    for A, B, C in subdivide(P, level):
        area = 0.5 * np.linalg.norm(np.cross(B - A, C - A))
        x = A[None, None, :] + U[..., None] * (B - A) + (U * Vv)[..., None] * (C - B)
        pts.append(x.reshape(-1, 3))
        wts.append((2.0 * area * U * WU).reshape(-1))
    pts = np.concatenate(pts)
    wts = np.concatenate(wts)
    P = np.asarray(P, dtype=np.float64)
    # barycentric coordinates w.r.t. the parent triangle
    T = np.stack([P[1] - P[0], P[2] - P[0]], axis=1)
    sol = np.linalg.lstsq(T, (pts - P[0]).T, rcond=None)[0].T
    bary = np.stack([1.0 - sol[:, 0] - sol[:, 1], sol[:, 0], sol[:, 1]], axis=1)
    return pts, wts, bary


def triangle_potential(P, x):
    """int_T 1/|x - y| dy for flat triangle P (3x3, any orientation) at points
    x [m,3] (closed form for a uniformly charged triangle: in-plane edge
    logarithms minus the height times the subtended-angle terms)."""
    P = np.asarray(P, dtype=np.float64)
    n = np.cross(P[1] - P[0], P[2] - P[0])
    n /= np.linalg.norm(n)
    d = (x - P[0]) @ n
    rho = x - d[:, None] * n[None, :]
    ad = np.abs(d)
    out = np.zeros(len(x))
    for a, b in ((0, 1), (1, 2), (2, 0)):
        t = P[b] - P[a]
        t /= np.linalg.norm(t)
        m = np.cross(t, n)  # outward in-plane normal of the edge
        lp = (P[b] - rho) @ t
        lm = (P[a] - rho) @ t
        p0 = (P[a] - rho) @ m
        r02 = p0 * p0 + d * d
        rp = np.sqrt(r02 + lp * lp)
        rm = np.sqrt(r02 + lm * lm)
        with np.errstate(divide="ignore", invalid="ignore"):
            log_t = np.where(np.abs(p0) > 0, p0 * np.log((rp + lp) / (rm + lm)), 0.0)
            ang = np.arctan2(p0 * lp, r02 + ad * rp) - np.arctan2(p0 * lm, r02 + ad * rm)
        out += log_t - ad * ang
    return out


def slp_pair_brute(Pi, Pj, s, c=1.0, level_outer=4, n_outer=6, level_smooth=3, n_smooth=4):
    """int_Pi int_Pj exp(-s r/c)/(4 pi r) = [int Phi_j + int int (exp(-s r/c)-1)/r] / (4 pi)."""
    x, wx, _ = collapsed_rule(Pi, level_outer, n_outer)
    sing = np.sum(wx * triangle_potential(Pj, x))
    xs, ws, _ = collapsed_rule(Pi, level_smooth, n_smooth)
    ys, vs, _ = collapsed_rule(Pj, level_smooth, n_smooth)
    smooth = 0.0 + 0.0j
    sc = s / c
    for k in range(len(xs)):
        r = np.linalg.norm(ys - xs[k], axis=1)
        with np.errstate(divide="ignore", invalid="ignore"):
            g = np.where(r > 0, np.expm1(-sc * r) / np.where(r > 0, r, 1.0), -sc)
        smooth += ws[k] * np.sum(vs * g)
    return (sing + smooth) / (4.0 * np.pi)


def pair_brute_regular(Pi, Pj, s, kernel, nj=None, c=1.0, level=2, n=5):
    """Composite collapsed-Gauss double integral for well-separated pairs.
    kernel 'slp' -> scalar; 'dlp' -> 3 values (P1 weights of Pj's vertices)."""
    x, wx, _ = collapsed_rule(Pi, level, n)
    y, wy, by = collapsed_rule(Pj, level, n)
    sc = s / c
    out = np.zeros(3, dtype=np.complex128)
    for k in range(len(x)):
        d = y - x[k]
        r = np.linalg.norm(d, axis=1)
        if kernel == "slp":
            out[0] += wx[k] * np.sum(wy * np.exp(-sc * r) / (4 * np.pi * r))
        else:
            kv = np.exp(-sc * r) * (1 + sc * r) * (-(d @ nj)) / (4 * np.pi * r ** 3)
            out += wx[k] * (wy * kv) @ by
    return out
