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


def _stability(z, rk):
    """R(z) = 1 + z b^T (I - z A)^{-1} 1 from the Butcher tableau."""
    if rk == 0:
        A, b = np.array([[1.0]]), np.array([1.0])
    else:
        A, b = np.array([[5 / 12, -1 / 12], [3 / 4, 1 / 4]]), np.array([3 / 4, 1 / 4])
    m = len(b)
    return np.array([1 + zz * b @ np.linalg.solve(np.eye(m) - zz * A, np.ones(m)) for zz in np.atleast_1d(z)])


@pytest.mark.parametrize("rk,ratio,nsteps", [(1, 12.6, 256), (1, 1.0, 10), (1, 12.6, 1), (0, 12.6, 256)])
def test_gcq_contour_cauchy(orc, rk, ratio, nsteps):
    """The quadrature sum w_l g(s_l) ~ (1/2 pi i) oint g ds (positive
    orientation) reproduces the Cauchy formula for g = 1/(s - z): winding
    number 1 at every resolvent pole of the steps, z = 1/dt (implicit Euler)
    and z = 1/(dt lambda_i(A)) (Radau IIA) for dt in [dt_min, dt_max]; 0 for
    points outside.  The set is symmetric under conjugation and lies in the
    right half plane."""
    dt_min = 1e-3
    dt_max = dt_min * ratio
    NQ = 256
    s, w, info = orc.freqs_gcq(dt_min, dt_max, rk, NQ, nsteps)
    assert np.all(s.real > 0)
    assert np.allclose(s, np.conj(s[::-1]), rtol=1e-12)
    inside = [1.0 / dt for dt in np.geomspace(dt_min, dt_max, 5)]
    if rk == 1:
        inside += [z for dt in np.geomspace(dt_min, dt_max, 5) for z in 1.0 / (dt * _radau_eigs())]
    for z in inside:
        val = np.sum(w / (s - z))
        assert abs(val - 1.0) < 1e-6, (z, val)
    R = info["rho"] / dt_min
    for z in (-10.0 / dt_min, 3 * R, 2 * R * 1j):
        assert abs(np.sum(w / (s - z))) < 1e-6
    assert info["lifted"] == (rk == 0 and ratio == 1.0)


@pytest.mark.parametrize("rk,nsteps", [(1, 1), (1, 10), (1, 64), (1, 512), (0, 512)])
def test_gcq_contour_radius(orc, rk, nsteps):
    """The circle |s - R| = R, R = rho / dt_min (gamma maps Im sigma = K'/2
    onto it: sn(+-K + i K'/2) = +-1/sqrt(k) gives gamma = 2R and 0; q only
    clusters the points towards 0).  rho = 1 for implicit Euler (|R(dt s)| = 1
    on the whole circle); for Radau IIA rho >= 1/min|lambda_i(A)| = sqrt(6)
    (the poles inside) and the Runge-Kutta stages grow by at most 1e4 over the
    nsteps steps along the contour, max |R(dt_min s_l)|^nsteps <= 1e4, with a
    radius 5 % smaller violating that bound unless rho = sqrt(6)."""
    dt_min = 2e-3
    s, w, info = orc.freqs_gcq(dt_min, 12.6 * dt_min, rk, 256, nsteps)
    rho = info["rho"]
    R = rho / dt_min
    assert np.max(np.abs(np.abs(s - R) - R)) < 1e-9 * R
    assert np.sum(s.real < 0.25 * R) > np.sum(s.real > 1.75 * R)
    if rk == 0:
        assert rho == 1.0
        assert np.allclose(np.abs(_stability(dt_min * s, 0)), 1.0, rtol=1e-9)
        return
    assert rho >= np.sqrt(6.0) - 1e-12
    th = 2 * np.pi * np.arange(1, 4096) / 4096
    grow = np.max(np.abs(_stability(rho * (1 + np.exp(1j * th)), 1)))
    assert nsteps * np.log(grow) <= np.log(1e4) + 1e-9
    assert nsteps * np.log(np.max(np.abs(_stability(dt_min * s, 1)))) <= np.log(1e4) + 1e-6
    if rho > np.sqrt(6.0) + 1e-9:
        smaller = np.max(np.abs(_stability(rho / 1.05 * (1 + np.exp(1j * th)), 1)))
        assert nsteps * np.log(smaller) > np.log(1e4)
    assert orc.gcq_radius(rk, nsteps) == rho


def test_gcq_printed_contour(orc):
    """rho = 1: the contour as printed in App. A, the circle through 0 and
    2/dt_min whatever the method."""
    for rk in (0, 1):
        dt_min = 2e-3
        s, w, info = orc.freqs_gcq(dt_min, 12.6 * dt_min, rk, 64, 256, rho=1.0)
        assert info["rho"] == 1.0
        assert np.max(np.abs(np.abs(s - 1.0 / dt_min) - 1.0 / dt_min)) < 1e-9 / dt_min


def test_gcq_degenerate_q_lifted(orc):
    s, w, info = orc.freqs_gcq(1e-3, 1e-3, 0, 32, 4)
    assert info["lifted"] and info["q"] > 1.0 and np.all(np.isfinite(s))
