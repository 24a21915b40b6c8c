"""Pins of the oracle's quadrature rules and Galerkin entries (CPU only).

Sec. 3 "Spatial discretisation": regular pairs by a Gauss rule (here the
7-point degree-5 triangle rule), weakly singular pairs by the Sauter-Schwab
(Erichsen-Sauter) transforms.  Every check compares with something other than
the oracle itself: exact monomial integrals, numpy's Gauss-Legendre, the
closed-form potential of a charged triangle, closed forms on the sphere, and
Green's identity for linear harmonic functions.
"""
import math

import numpy as np
import pytest

from paper_2505_00715_gb300.inputs import icosphere, octahedron
from _brute import collapsed_rule, pair_brute_regular, slp_pair_brute


def test_rule7_exact_degree5(orc):
    b, w = orc.rule7()
    assert abs(w.sum() - 1.0) < 1e-15
    P = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    x = b @ P
    for a in range(6):
        for c in range(6 - a):
            q = 0.5 * np.sum(w * x[:, 0] ** a * x[:, 1] ** c)
            exact = math.factorial(a) * math.factorial(c) / math.factorial(a + c + 2)
            assert abs(q - exact) < 1e-15, (a, c)
    # degree 6 is not integrated exactly (so the rule is exactly degree 5)
    q6 = 0.5 * np.sum(w * x[:, 0] ** 6)
    assert abs(q6 - math.factorial(6) / math.factorial(8)) > 1e-6


@pytest.mark.parametrize("n", [1, 2, 5, 8, 16])
def test_gauss_legendre_matches_numpy(orc, n):
    x, w = orc.gauss01(n)
    g, gw = np.polynomial.legendre.leggauss(n)
    assert np.allclose(np.sort(x), 0.5 * (g + 1.0), atol=1e-15, rtol=0)
    assert np.allclose(w[np.argsort(x)], 0.5 * gw, atol=1e-15, rtol=0)
    for k in range(2 * n):
        assert abs(np.sum(w * x ** k) - 1.0 / (k + 1)) < 1e-14


@pytest.fixture(scope="module")
def sphere1(orc):
    V, T = icosphere(1)
    return V, T, orc.Mesh(V, T)


def _touching(T, i):
    return [j for j in range(len(T)) if len(set(T[i]) & set(T[j])) > 0]


@pytest.mark.parametrize("s", [0.0, 3.0 + 2.0j])
def test_singular_slp_pairs_vs_charged_triangle(orc, sphere1, s):
    """Identical, common-edge and common-vertex SLP pairs vs an independent
    integral: closed-form inner potential of the 1/r part plus composite
    Gauss for the bounded remainder (exp(-sr)-1)/r."""
    V, T, m = sphere1
    seen = set()
    for j in _touching(T, 0):
        cls, val = m.pair(orc.SLP, 0, j, s, ng=16)
        if cls in seen:
            continue
        seen.add(cls)
        ls = 4 if (cls == 3 and s != 0) else 3
        ref = slp_pair_brute(V[T[0]], V[T[j]], s, level_outer=5, level_smooth=ls)
        tol = 2e-6 if cls != 3 else (1e-6 if s == 0 else 8e-6)
        assert abs(ref - val[0]) <= tol * abs(ref), (cls, abs(ref - val[0]) / abs(ref))
    assert seen == {1, 2, 3}


def test_singular_converges_in_ng(orc, sphere1):
    V, T, m = sphere1
    for j in _touching(T, 0):
        for op in (orc.SLP, orc.DLP):
            _, a = m.pair(op, 0, j, 4.0 + 3.0j, ng=14)
            _, b = m.pair(op, 0, j, 4.0 + 3.0j, ng=20)
            scale = np.max(np.abs(b)) + 1e-300
            assert np.max(np.abs(a - b)) <= 1e-10 * scale


def test_regular_pairs_vs_composite_gauss(orc, sphere1):
    V, T, m = sphere1
    c = V[T].mean(axis=1)
    far = int(np.argmax(np.linalg.norm(c - c[0], axis=1)))
    mid = int(np.argsort(np.linalg.norm(c - c[0], axis=1))[len(T) // 4])
    for j, tol in ((far, 1e-5), (mid, 2e-3)):
        for op, name in ((orc.SLP, "slp"), (orc.DLP, "dlp")):
            cls, val = m.pair(op, 0, j, 2.0 + 1.0j)
            assert cls == 0
            nrm = np.cross(V[T[j]][1] - V[T[j]][0], V[T[j]][2] - V[T[j]][0])
            nrm /= np.linalg.norm(nrm)
            ref = pair_brute_regular(V[T[0]], V[T[j]], 2.0 + 1.0j, name, nj=nrm, level=2, n=5)
            k = 1 if name == "slp" else 3
            err = np.max(np.abs(val[:k] - ref[:k])) / np.max(np.abs(ref[:k]))
            assert err < tol, (j, name, err)


def test_conjugate_symmetry(orc, sphere1):
    V, T, m = sphere1
    rows = np.arange(0, len(T), 7)
    a = m.entries(orc.SLP, rows, np.arange(len(T)), [2.0 + 5.0j, 2.0 - 5.0j])
    assert np.allclose(a[1], np.conj(a[0]), rtol=1e-14, atol=0)
    b = m.entries(orc.DLP, rows, np.arange(len(V)), [2.0 + 5.0j, 2.0 - 5.0j])
    assert np.allclose(b[1], np.conj(b[0]), rtol=1e-14, atol=1e-300)


def test_slp_symmetric(orc, sphere1):
    V, T, m = sphere1
    n = len(T)
    a = m.entries(orc.SLP, np.arange(n), np.arange(n), [1.5 + 2.0j], ng=6)[0]
    assert np.max(np.abs(a - a.T)) <= 1e-15 * np.max(np.abs(a))


@pytest.mark.parametrize("op", ["slp", "dlp", "adlp"])
def test_sphere_closed_form_order2(orc, op):
    """Row sums of the Galerkin matrices on icospheres converge at O(h^2) to
    (1 - e^{-2sR/c})/(2s/c)      (SLP applied to 1, per unit test area) and
    e^{-2sR/c}/2 - (1-e^{-2sR/c})/(2sR/c)  (DLP and its adjoint applied to 1:
    on a sphere (x - y).n_y = (y - x).n_x, so both kernels coincide there).
    The adjoint converges at O(h) only: its row sum weighs the facet normal
    n_x, which deviates by O(h) from the sphere's, while the double layer's
    row sum is a solid angle of the polyhedron (Gauss' law at s = 0) and
    keeps O(h^2)."""
    s, R = 2.0 + 1.0j, 1.0
    errs = []
    for lev in (2, 3, 4):
        V, T = icosphere(lev, R)
        m = orc.Mesh(V, T)
        n = len(T)
        rows = np.arange(0, n, max(1, n // 12))
        area = 0.5 * np.linalg.norm(np.cross(V[T[:, 1]] - V[T[:, 0]], V[T[:, 2]] - V[T[:, 0]]), axis=1)
        if op == "slp":
            A = m.entries(orc.SLP, rows, np.arange(n), [s], ng=6)[0]
            cf = (1 - np.exp(-2 * s * R)) / (2 * s)
        else:
            op_, ncol = (orc.DLP, len(V)) if op == "dlp" else (orc.ADLP, n)
            A = m.entries(op_, rows, np.arange(ncol), [s], ng=6)[0]
            cf = np.exp(-2 * s * R) / 2 - (1 - np.exp(-2 * s * R)) / (2 * s * R)
        errs.append(np.max(np.abs(A.sum(1) / area[rows] - cf)) / abs(cf))
    order = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    if op == "adlp":
        assert order[0] > 0.95 and order[1] > 0.95, (errs, order)
        assert errs[0] < 0.04, errs
        return
    assert order[0] > 1.7 and order[1] > 1.85, (errs, order)
    assert errs[0] < (0.005 if op == "slp" else 0.02)


def test_dlp_green_identity_linear(orc):
    """Green's representation for a linear (harmonic) g on a closed polyhedron at s = 0:
    sum_v K0[i,v] g(v) = -1/2 int_{tau_i} g + sum_j V0[i,j] (grad g . n_j).
    Exact for the Galerkin P0 x P1 / P0 x P0 matrices up to quadrature error."""
    for V, T in (octahedron(), icosphere(2)):
        m = orc.Mesh(V, T)
        n = len(T)
        rng = np.random.default_rng(5)
        a, b0 = rng.standard_normal(3), 0.3
        g = V @ a + b0
        nrm = np.cross(V[T[:, 1]] - V[T[:, 0]], V[T[:, 2]] - V[T[:, 0]])
        area = 0.5 * np.linalg.norm(nrm, axis=1)
        nrm /= 2 * area[:, None]
        rows = np.arange(n) if n < 50 else np.arange(0, n, 9)
        K = m.entries(orc.DLP, rows, np.arange(len(V)), [0.0], ng=8)[0]
        Vm = m.entries(orc.SLP, rows, np.arange(n), [0.0], ng=8)[0]
        gc = V[T].mean(axis=1) @ a + b0
        lhs = K @ g
        rhs = -0.5 * area[rows] * gc[rows] + Vm @ (nrm @ a)
        err = np.max(np.abs(lhs - rhs)) / np.max(np.abs(area[rows] * gc[rows]))
        assert err < (2e-4 if n < 50 else 2e-5), err


def test_octahedron_brute_force_dense(orc):
    """Whole SLP matrix of the octahedron at two frequencies: each entry vs the
    independent integrators (touching pairs) or composite Gauss (others)."""
    V, T = octahedron()
    m = orc.Mesh(V, T)
    n = len(T)
    for s in (0.5 + 0.0j, 1.0 + 2.0j):
        A = m.entries(orc.SLP, np.arange(n), np.arange(n), [s], ng=12)[0]
        for i in range(0, n, 3):
            for j in range(n):
                shared = len(set(T[i]) & set(T[j]))
                if shared:
                    ref = slp_pair_brute(V[T[i]], V[T[j]], s, level_outer=4,
                                         level_smooth=4 if shared == 3 else 3)
                    tol = 2e-5
                else:
                    ref = pair_brute_regular(V[T[i]], V[T[j]], s, "slp", level=2, n=5)[0]
                    tol = 2e-3  # the 7x7 rule itself on touching-distance pairs
                assert abs(A[i, j] - ref) <= tol * abs(ref), (i, j, shared)


# ---------------------------------------------------------------- magnitude sums
def test_magnitude_sums_equal_modulus_for_positive_terms(orc, sphere1):
    """Single layer at real s: every quadrature term is positive, so the
    magnitude sum equals |entry| (touching and regular pairs alike)."""
    V, T, m = sphere1
    rows = np.array([0, 3, 7], dtype=np.int32)
    cols = np.arange(len(T), dtype=np.int32)
    for s in (0.0, 2.5):
        a = m.entries(orc.SLP, rows, cols, [s], c=1.0, ng=6)
        g = m.entries_mag(orc.SLP, rows, cols, [s], c=1.0, ng=6)
        assert np.max(np.abs(g - np.abs(a)) / np.abs(a)) < 1e-13


@pytest.mark.parametrize("op", ["SLP", "DLP", "ADLP"])
def test_magnitude_sums_bound_the_entries(orc, sphere1, op):
    """Triangle inequality: the magnitude sum bounds |entry| at complex s,
    and for the double layer and its adjoint the bound is strict on curved
    neighbours; a flat panel with itself contributes nothing to K' (entry
    and magnitude sum both zero)."""
    V, T, m = sphere1
    rows = np.array([0, 5, 11], dtype=np.int32)
    cols = np.arange(len(V) if op == "DLP" else len(T), dtype=np.int32)
    s = [1.5 + 7.0j, 0.3 - 2.0j]
    a = m.entries(getattr(orc, op), rows, cols, s, c=1.0, ng=6)
    g = m.entries_mag(getattr(orc, op), rows, cols, s, c=1.0, ng=6)
    assert np.all(g >= np.abs(a) * (1 - 1e-12))
    if op == "ADLP":
        own = np.zeros(g.shape, dtype=bool)
        own[:, np.arange(len(rows)), rows] = True
        assert np.all(g[own] == 0) and np.all(a[own] == 0)
        g, a = g[~own], a[~own]
    assert np.all(g > 0)
    if op != "SLP":
        assert np.median(g / np.maximum(np.abs(a), 1e-300)) > 1.5


def test_dlp_magnitude_of_stacked_small_triangles(orc):
    """Two small parallel triangles a distance R apart, one above the other:
    |x - y| and |(x - y).n_y| agree to O((h/R)^2), so the double-layer entry
    summed over the trial hats and its magnitude sum both approach the
    far-field value |T0| |T1| |exp(-sR)(1 + sR)| / (4 pi R^2)."""
    h, R = 1e-2, 1.0
    P = np.array([[0.0, 0.0, 0.0], [h, 0.0, 0.0], [0.0, h, 0.0]])
    V = np.vstack([P, P + [0.0, 0.0, R]])
    T = np.array([[0, 1, 2], [3, 4, 5]], dtype=np.int32)  # both normals +z
    m = orc.Mesh(V, T)
    s = 3.0 + 4.0j
    ent = m.entries(orc.DLP, [0], [3, 4, 5], [s], c=1.0, ng=6)[0, 0].sum()
    mag = m.entries_mag(orc.DLP, [0], [3, 4, 5], [s], c=1.0, ng=6)[0, 0].sum()
    area = 0.5 * h * h
    far = area * area * abs(np.exp(-s * R) * (1 + s * R)) / (4 * np.pi * R * R)
    assert abs(abs(ent) - mag) <= 1e-3 * mag
    assert abs(mag - far) <= 1e-3 * far


def test_adjoint_double_layer_is_the_transposed_p0_double_layer(orc):
    """K' (eq. adlp, conormal derivative at x) with P0 x P0 is the transpose of
    the P0 x P0 double layer: swapping test and trial triangles turns
    (x - y).n_y into (y - x).n_x.  The oracle forms the two by different code
    paths (test normal vs trial normal, the P1 hat weights of the double layer
    summed to the P0 trial function, touching pairs parametrised from the other
    triangle), so a dropped sign, the wrong normal or a transposed operand
    fails here.  Checked on a jittered sphere (no symmetry) for regular,
    vertex, edge and identical pairs at a complex frequency."""
    V, T = icosphere(1)
    rng = np.random.default_rng(3)
    V = V * (1.0 + 0.08 * rng.standard_normal((len(V), 1)))
    m = orc.Mesh(V, T)
    s = 1.3 + 2.1j
    seen = set()
    for ti in range(len(T)):
        for tj in range(len(T)):
            cls, kp = m.pair(orc.ADLP, ti, tj, s, ng=12)
            cls2, kt = m.pair(orc.DLP, tj, ti, s, ng=12)
            assert cls == cls2
            seen.add(cls)
            ref = kt.sum()  # P1 hats of the trial triangle sum to its P0 function
            assert abs(kp[0] - ref) <= 1e-8 * max(abs(ref), 1e-3), (ti, tj, cls, kp[0], ref)
            if cls == 3:
                assert kp[0] == 0.0
    assert seen == {0, 1, 2, 3}
