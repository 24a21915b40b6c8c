"""Oracle of the gCQ time marching (Sec. 3 "Temporal discretisation", eqs.
gCQ_xn and gcq_formula; App. A).

TEST INFRASTRUCTURE ONLY: a plain numpy restatement, in the paper's order, of
the Runge-Kutta based generalised convolution quadrature, used to check the
CUDA library's marching.  Nothing in the library may import it.

Notation (Sec. 3): steps dt_1..dt_N, Runge-Kutta matrix A (m x m) with
b^T A^{-1} = (0, ..., 1); q_n collects the m stage values of step n (times
t_{n-1} + c_i dt_n); contour points s_l and weights w_l of App. A in the
positively oriented convention of the frequency sets (sum_l w_l g(s_l) ~
(1/2 pi i) oint g ds).

  x_{n-1}(s_l) = (I - dt_{n-1} s_l A)^{-1} ((b^T A^{-1} . x_{n-2}(s_l)) 1 + dt_{n-1} A q_{n-1})
  W_l          = omega_l (b^T A^{-1} . x_{n-1}(s_l)) (I - dt_n s_l A)^{-1} 1,  omega_l = -w_l
  (V * q)_n    = V((dt_n A)^{-1}) q_n + sum_l V(s_l) W_l

V((dt A)^{-1}) is the operator at the matrix argument: with (dt A)^{-1} =
P diag(mu) P^{-1}, its action on stage data is P diag(V(mu_k)) P^{-1} over
the stage index.  Operators are callables s -> dense matrix (or a scalar for
the pins of the scalar convolutions).
"""
import numpy as np


def radau_iia2():
    """2-stage Radau IIA: A, b, c."""
    A = np.array([[5.0 / 12.0, -1.0 / 12.0], [3.0 / 4.0, 1.0 / 4.0]])
    return A, np.array([3.0 / 4.0, 1.0 / 4.0]), np.array([1.0 / 3.0, 1.0])


def implicit_euler():
    return np.array([[1.0]]), np.array([1.0]), np.array([1.0])


def rk_tableau(rk):
    return radau_iia2() if rk == 1 else implicit_euler()


def graded_steps(N, ratio, T):
    """N steps growing geometrically by `ratio` and summing to T."""
    dt1 = T * (ratio - 1.0) / (ratio ** N - 1.0)
    return dt1 * ratio ** np.arange(N)


def stage_times(dts, rk):
    """[N][m] stage times t_{n-1} + c_i dt_n."""
    _, _, c = rk_tableau(rk)
    t0 = np.concatenate([[0.0], np.cumsum(dts)[:-1]])
    return t0[:, None] + np.asarray(dts)[:, None] * c[None, :]


class History:
    """The x(s_l) states of one data series (all contour points), and the
    weighted data W_l of the next step."""

    def __init__(self, s, w, A, shape):
        self.s, self.w, self.A = np.asarray(s), np.asarray(w), A
        self.m = A.shape[0]
        self.X = np.zeros((len(self.s),) + tuple(shape) + (self.m,), dtype=np.complex128)

    def advance(self, dt_prev, data_prev):
        """x_{n-1}(s_l) from x_{n-2}(s_l) and the stage data of step n-1
        (data_prev [..., m])."""
        I = np.eye(self.m)
        for l, sl in enumerate(self.s):
            R = np.linalg.inv(I - dt_prev * sl * self.A)
            xend = self.X[l][..., -1]  # b^T A^{-1} x = the last stage
            rhs = xend[..., None] * np.ones(self.m) + dt_prev * data_prev @ self.A.T
            self.X[l] = rhs @ R.T

    def weights(self, dt):
        """W_l [NQ, ..., m] of the step with size dt."""
        I = np.eye(self.m)
        W = np.zeros_like(self.X)
        for l, sl in enumerate(self.s):
            r1 = np.linalg.solve(I - dt * sl * self.A, np.ones(self.m))
            # omega_l of eq. gcq_formula = -w_l: the step's value is minus the
            # positively oriented contour integral of V(s) times the Runge-Kutta
            # stages (their poles lie inside the contour, the convolution's
            # Bromwich line to their left)
            W[l] = -self.w[l] * self.X[l][..., -1][..., None] * r1
        return W


def step_eigs(dt, A):
    """mu_k = 1/(dt lambda_k) and P with (dt A)^{-1} = P diag(mu) P^{-1}."""
    lam, P = np.linalg.eig(A)
    return 1.0 / (dt * lam), P


def apply_matrix_arg(op, dt, A, data):
    """op((dt A)^{-1}) applied to stage data [n, m] (op(mu) an [*, n] matrix)."""
    mu, P = step_eigs(dt, A)
    dt_ = data @ np.linalg.inv(P).T  # [:, k] = sum_j (P^-1)_{kj} data[:, j]
    out = np.stack([op(mu[k]) @ dt_[:, k] for k in range(len(mu))], axis=1)
    return out @ P.T


def solve_matrix_arg(op, dt, A, rhs):
    """Solves op((dt A)^{-1}) q = rhs for stage data q [n, m]."""
    mu, P = step_eigs(dt, A)
    rt = rhs @ np.linalg.inv(P).T
    qt = np.stack([np.linalg.solve(op(mu[k]), rt[:, k]) for k in range(len(mu))], axis=1)
    return qt @ P.T


def history_sum(op, s, W):
    """sum_l op(s_l) W_l for W [NQ, n, m]."""
    return sum(op(sl) @ W[l] for l, sl in enumerate(s))


def convolve(op, q, dts, rk, s, w):
    """Forward gCQ convolution (V * q)_n at the stage times for stage data
    q [N, n, m] (eq. gcq_formula with q given)."""
    A, _, _ = rk_tableau(rk)
    N, n, m = q.shape
    H = History(s, w, A, (n,))
    out = []
    for k in range(N):
        v = apply_matrix_arg(op, dts[k], A, q[k])
        if k >= 1:
            H.advance(dts[k - 1], q[k - 1])
            v = v + history_sum(op, s, H.weights(dts[k]))
        out.append(v)
    return np.stack(out)


def solve(opV, f, dts, rk, s, w):
    """Solves the convolution equation V * q = f (eq. gcq_formula with the
    right-hand side given) for stage data q [N, n, m]; f [N, n, m]."""
    A, _, _ = rk_tableau(rk)
    N, n, m = f.shape
    H = History(s, w, A, (n,))
    q = np.zeros((N, n, m), dtype=np.complex128)
    for k in range(N):
        rhs = f[k]
        if k >= 1:
            H.advance(dts[k - 1], q[k - 1])
            rhs = rhs - history_sum(opV, s, H.weights(dts[k]))
        q[k] = solve_matrix_arg(opV, dts[k], A, rhs)
    return q


def solve_dirichlet(opV, opK, mass_half, g, dts, rk, s, w):
    """The direct Dirichlet problem V * q = (1/2 M + K) * g (Sec. 2, Galerkin
    form with P0 test functions): g [N, nv, m] the Dirichlet data at the stage
    times, returns q [N, nt, m] (real).  opV(s) [nt, nt], opK(s) [nt, nv],
    mass_half [nt, nv] = 1/2 the P0 x P1 mass matrix."""
    f = np.einsum("ij,njm->nim", mass_half, g) + convolve(opK, g, dts, rk, s, w)
    return solve(opV, f, dts, rk, s, w).real


def nq_points(N):
    """N_Q = N (ln N)^2 contour points (App. A, m > 1 stages), rounded up to
    an even count (the points come in conjugate pairs)."""
    n = int(np.ceil(N * np.log(N) ** 2))
    return max(2, n + (n % 2))


# ---------------------------------------------------------------- analytic loads
def pulse(tau, c=1.0):
    """f(tau) = tau^2 exp(-c tau) H(tau) of the smooth-pulse load (Sec. 5,
    eq. load) and its derivative."""
    tau = np.asarray(tau, dtype=np.float64)
    pos = tau > 0
    f = np.where(pos, tau * tau * np.exp(-c * np.where(pos, tau, 0.0)), 0.0)
    fp = np.where(pos, (2.0 * tau - c * tau * tau) * np.exp(-c * np.where(pos, tau, 0.0)), 0.0)
    return f, fp


def pulse_field(y, t, x_src, c=1.0):
    """u(y, t) = f(t - r/c) / r, r = |x_src - y| (eq. load)."""
    r = np.linalg.norm(np.asarray(y) - np.asarray(x_src), axis=-1)
    f, _ = pulse(t - r / c, c)
    return f / r


def pulse_flux(y, n, t, x_src, c=1.0):
    """q = du/dn_y of the pulse field: -(f'(tau)/(c r) + f(tau)/r^2) (y - x_src).n / r."""
    d = np.asarray(y) - np.asarray(x_src)
    r = np.linalg.norm(d, axis=-1)
    f, fp = pulse(t - r / c, c)
    return -(fp / (c * r) + f / (r * r)) * np.sum(d * n, axis=-1) / r


class CachedOperator:
    """s -> dense operator matrix, computed once per frequency (conjugate
    frequencies by conjugation, A(conj s) = conj A(s))."""

    def __init__(self, fn):
        self.fn, self.cache = fn, {}

    def __call__(self, s):
        s = complex(s)
        key = (round(s.real, 12), round(abs(s.imag), 12))
        if key not in self.cache:
            self.cache[key] = (s, self.fn(complex(s.real, abs(s.imag))))
        _, M = self.cache[key]
        return M if s.imag >= 0 else np.conj(M)
