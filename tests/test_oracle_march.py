"""Pins of the oracle's gCQ time marching (Sec. 3 eqs. gCQ_xn, gcq_formula;
App. A), on convolutions with closed-form results (CPU only).

- Damped integrator V(s) = 1/(s + a) (analytic inside the contour):
  (V * q)(t) = int_0^t exp(-a (t - tau)) q(tau) dtau, so V * q = t^3 gives
  q = 3 t^2 + a t^3; solved by the marching (implicit Euler and 2-stage
  Radau IIA), with constant and with geometrically graded steps.
- Retarded kernel V(s) = exp(-s R)/(4 pi R), the single-layer kernel of one
  point pair at distance R (c = 1): (V * q)(t) = q(t - R)/(4 pi R); the
  forward convolution of a smooth q is reproduced.
Convergence orders under step halving: the stage values of implicit Euler
converge linearly; those of Radau IIA at least quadratically (stage order 2).
"""
import numpy as np
import pytest

from oracle import march


def _contour(orc, dts, rk, N):
    s, w, _ = orc.freqs_gcq(float(np.min(dts)), float(np.max(dts)), rk, march.nq_points(N), len(dts))
    return s, w


def _integrator_error(orc, rk, N, graded):
    T = 2.0
    # graded: dt_max / dt_min = 4 at every N, so that doubling N refines the grading
    dts = march.graded_steps(N, 4.0 ** (1.0 / (N - 1)), T) if graded else np.full(N, T / N)
    s, w = _contour(orc, dts, rk, N)
    t = march.stage_times(dts, rk)
    a = 0.7
    f = (t ** 3)[:, None, :].astype(np.complex128)
    q = march.solve(lambda z: np.array([[1.0 / (z + a)]]), f, dts, rk, s, w)
    exact = 3.0 * t ** 2 + a * t ** 3
    return np.max(np.abs(q[:, 0, :] - exact)) / np.max(exact), np.max(np.abs(q.imag))


@pytest.mark.parametrize("rk,order", [(0, 0.8), (1, 1.8)])
@pytest.mark.parametrize("graded", [False, True])
def test_integrator_solve(orc, rk, order, graded):
    e1, im1 = _integrator_error(orc, rk, 10, graded)
    print("integrator rk %d graded %s" % (rk, graded))
    e2, im2 = _integrator_error(orc, rk, 20, graded)
    e3, _ = _integrator_error(orc, rk, 40, graded)
    assert e3 < e2 < e1 and e3 < (0.2 if rk == 0 else 2e-3), (e1, e2, e3)
    assert np.log2(e2 / e3) > order, (e1, e2, e3)
    assert im1 < 1e-9 and im2 < 1e-9  # the conjugate-symmetric contour gives real results


def _retarded_error(orc, rk, N):
    R, T = 0.5, 3.0
    dts = np.full(N, T / N)
    s, w = _contour(orc, dts, rk, N)
    t = march.stage_times(dts, rk)

    def qf(tt):
        return np.where(tt > 0, tt ** 4 * np.exp(-np.maximum(tt, 0.0)), 0.0)

    q = qf(t)[:, None, :].astype(np.complex128)
    out = march.convolve(lambda z: np.array([[np.exp(-z * R) / (4 * np.pi * R)]]), q, dts, rk, s, w)
    exact = qf(t - R) / (4 * np.pi * R)
    return np.max(np.abs(out[:, 0, :] - exact)) / np.max(np.abs(exact))


@pytest.mark.parametrize("rk,order", [(0, 0.8), (1, 1.8)])
def test_retarded_kernel_convolution(orc, rk, order):
    e = [_retarded_error(orc, rk, N) for N in (20, 40, 80)]
    print("retarded kernel rk %d errors %s" % (rk, e))
    assert e[2] < e[1] < e[0], e
    assert np.log2(e[1] / e[2]) > order, e


def test_matrix_argument_is_the_operator_of_the_step_resolvent(orc):
    """op((dt A)^{-1}) through the eigen-decomposition equals the Cauchy
    integral (1/2 pi i) oint op(s) (s I - (dt A)^{-1})^{-1} ds evaluated with
    the gCQ contour of that step (op entire: exp(-s))."""
    A, _, _ = march.radau_iia2()
    dt = 0.2
    s, w = _contour(orc, np.array([dt]), 1, 40)
    data = np.array([[1.0, -2.0]])
    op = lambda z: np.array([[np.exp(-z)]])
    direct = march.apply_matrix_arg(op, dt, A, data)
    B = np.linalg.inv(dt * A)
    cauchy = sum(wl * np.exp(-sl) * np.linalg.solve(sl * np.eye(2) - B, data[0]) for sl, wl in zip(s, w))
    assert np.allclose(direct[0], cauchy, rtol=1e-8, atol=1e-10)


def test_cube_dirichlet_oracle_converges(orc):
    """The oracle's dense marching of the direct Dirichlet problem on the unit
    cube (Sec. 5, eq. load; 2-stage Radau IIA) converges towards the exact
    Neumann datum: the L_max error of eq. error falls by more than half from
    level 1 (96 triangles, 10 steps) to level 2 (384, 20 steps)."""
    from _cube import CubeProblem, oracle_solution
    bary, w7 = orc.rule7()
    e = []
    for level in (1, 2):
        P = CubeProblem(level)
        e.append(P.lmax(oracle_solution(orc, P), bary, w7))
    print("cube Dirichlet L_max levels 1, 2: %s, eoc %.2f" % (e, np.log2(e[0] / e[1])))
    assert e[1] < 0.5 * e[0] and e[1] < 0.6, e
