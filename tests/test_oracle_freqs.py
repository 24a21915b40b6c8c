"""Pins of the oracle's frequency sets (BDF2 CQ and the gCQ contour of App. A)."""
import math

import numpy as np
import pytest


def test_bdf2_points_invert_generating_function(orc):
    """s_k = delta(zeta_k)/dt with delta(z) = (1-z) + (1-z)^2/2: the root of
    delta(z) = dt s near z = 1 is z = 2 - sqrt(1 + 2 dt s); it must lie on the
    circle |z| = lambda at angle 2 pi k / N."""
    N, dt = 16, 0.1
    lam = 1e-8 ** (1.0 / (2 * N))
    s = orc.freqs_bdf2(N, dt)
    z = 2.0 - np.sqrt(1.0 + 2.0 * dt * s)
    k = np.arange(N)
    assert np.allclose(np.abs(z), lam, rtol=1e-13)
    ang = np.angle(z * np.exp(-2j * np.pi * k / N))
    assert np.max(np.abs(ang)) < 1e-12
    # conjugate pairs, s_0 real, right half plane
    assert np.allclose(s[1:], np.conj(s[1:][::-1]), rtol=1e-13)
    assert abs(s[0].imag) < 1e-14 and np.all(s.real > 0)


def test_bdf2_cq_weights_of_integration(orc):
    """CQ weights of the integration operator K(s) = 1/s recovered from the
    points by the scaled trapezoidal rule equal the power-series coefficients
    of dt / delta(z) (computed here by series division), up to lambda^N."""
    N, dt = 32, 0.05
    lam = 1e-8 ** (1.0 / (2 * N))
    s = orc.freqs_bdf2(N, dt)
    n = np.arange(N)
    zeta = np.exp(2j * np.pi * np.arange(N) / N)
    w_cq = (lam ** (-n) / N) * np.array([np.sum((1.0 / s) * zeta ** (-j)) for j in n])
    # delta(z) = 3/2 - 2 z + z^2/2; dt/delta as a power series
    d = np.array([1.5, -2.0, 0.5])
    c = np.zeros(N)
    for j in range(N):
        acc = (dt if j == 0 else 0.0)
        for i in range(1, 3):
            if j - i >= 0:
                acc -= d[i] * c[j - i]
        c[j] = acc / d[0]
    # aliasing error of the scaled trapezoidal rule: ~ lambda^N = 1e-4
    assert np.max(np.abs(w_cq.real - c)) < 2.0 * lam ** N * np.max(np.abs(c))
    assert np.max(np.abs(w_cq.imag)) < 1e-9 * np.max(np.abs(c))


@pytest.mark.parametrize("m", [0.0, 1e-6, 0.1, 0.5, 0.9, 0.999999])
def test_ellipk_matches_scipy(orc, m):
    sp = pytest.importorskip("scipy.special")
    assert abs(orc.ellipk(m) - sp.ellipk(m)) <= 1e-14 * sp.ellipk(m)


@pytest.mark.parametrize("m", [1e-3, 0.3, 0.7, 0.99, 0.999999])
def test_ellipj_real_matches_scipy(orc, m):
    sp = pytest.importorskip("scipy.special")
    for u in (-3.1, -0.4, 0.0, 0.77, 2.5, 6.0):
        ours = orc.ellipj(u, m)
        ref = sp.ellipj(u, m)[:3]
        assert np.allclose(ours, ref, atol=2e-14, rtol=0), (u, m, ours, ref)


@pytest.mark.parametrize("m", [0.01, 0.5, 0.95])
def test_ellipj_complex_matches_mpmath(orc, m):
    mp = pytest.importorskip("mpmath")
    for z in (0.3 + 0.2j, -1.2 + 0.9j, 2.0 - 0.4j, 0.1 + 1.5j):
        sn, cn, dn = orc.ellipj_complex(z, m)
        for name, ours in (("sn", sn), ("cn", cn), ("dn", dn)):
            ref = complex(mp.ellipfun(name, mp.mpc(z.real, z.imag), m=m))
            assert abs(ours - ref) <= 1e-13 * max(1.0, abs(ref)), (name, z, m)
        assert abs(sn * sn + cn * cn - 1) < 1e-13 * max(1, abs(sn) ** 2)
        assert abs(dn * dn + m * sn * sn - 1) < 1e-13 * max(1, abs(sn) ** 2)


def _radau_eigs():
    A = np.array([[5 / 12, -1 / 12], [3 / 4, 1 / 4]])
    return np.linalg.eigvals(A)


@pytest.mark.parametrize("rk,ratio", [(1, 12.6), (1, 1.0), (0, 12.6)])
def test_gcq_contour_cauchy(orc, rk, ratio):
    """The quadrature sum w_l g(s_l) ~ (1/2 pi i) oint g ds (positive
    orientation) reproduces the Cauchy formula for g = 1/(s - z): winding
    number 1 for the implicit-Euler resolvent poles z = 1/dt of every step
    size in [dt_min, dt_max] and for the Radau IIA poles 1/(dt_max lambda(A)),
    0 for points outside.  The set is symmetric under conjugation and lies in
    the right half plane."""
    dt_min = 1e-3
    dt_max = dt_min * ratio
    NQ = 128
    s, w, info = orc.freqs_gcq(dt_min, dt_max, rk, NQ)
    assert np.all(s.real > 0)
    assert np.allclose(s, np.conj(s[::-1]), rtol=1e-12)
    inside = [1.0 / dt for dt in np.geomspace(dt_min, dt_max, 5)]
    if rk == 1 and ratio > 2:
        # (for dt close to dt_min the Radau poles (2 -/+ 1.41i)/dt lie outside
        # the circle of radius 1/dt_min; the formula of App. A is kept as printed)
        inside += list(1.0 / (dt_max * _radau_eigs()))
    for z in inside:
        val = np.sum(w / (s - z))
        assert abs(val - 1.0) < 1e-6, (z, val)
    for z in (-10.0 / dt_min, 1e3 / dt_min, 1e2 / dt_min * 1j):
        assert abs(np.sum(w / (s - z))) < 1e-6
    assert info["lifted"] == (rk == 0 and ratio == 1.0)


def test_gcq_contour_is_circle_through_0_and_2_over_dtmin(orc):
    """gamma maps Im sigma = K'/2 onto the circle |s - 1/dt_min| = 1/dt_min
    (sn(+-K + i K'/2) = +-1/sqrt(k) gives gamma = 2/dt_min and 0); q only
    changes how the points cluster towards 0."""
    for rk, ratio in ((1, 12.6), (0, 3.0)):
        dt_min = 2e-3
        s, w, info = orc.freqs_gcq(dt_min, ratio * dt_min, rk, 64)
        r = np.abs(s - 1.0 / dt_min)
        assert np.max(np.abs(r - 1.0 / dt_min)) < 1e-9 / dt_min
        # clustering: more points near 0 for larger q
        assert np.sum(s.real < 0.25 / dt_min) > np.sum(s.real > 1.75 / dt_min)


def test_gcq_degenerate_q_lifted(orc):
    s, w, info = orc.freqs_gcq(1e-3, 1e-3, 0, 32)
    assert info["lifted"] and info["q"] > 1.0 and np.all(np.isfinite(s))
