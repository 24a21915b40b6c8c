"""The unit-cube Dirichlet problem of Sec. 5 (eq. load) for the marching
tests: the cube [-0.5, 0.5]^3 (tests use its levels 1-3: 96 / 384 / 1536
triangles, dt = 0.3 / 2^(level-1), N = 10 * 2^(level-1) steps to T = 3 s,
c = 1), the smooth pulse u(y, t) = f(t - r)/r, f(tau) = tau^2 exp(-tau) H(tau),
r = |y - x|, emitted at x = (0.8, 0.2, 0.3) outside the cube, its Dirichlet
data g (P1 nodal values at the stage times) and the L2 error of a computed
Neumann datum q (P0) against du/dn at the step ends t_n (the last stage,
c_m = 1), integrated with the 7-point rule."""
import numpy as np

from oracle import march
from paper_2505_00715_gb300.inputs import cube

X_SRC = np.array([0.8, 0.2, 0.3])


class CubeProblem:
    def __init__(self, level, rk=1):
        self.level, self.rk = level, rk
        self.V, self.T = cube(level)
        self.N = 10 * 2 ** (level - 1)
        self.dt = 0.3 / 2 ** (level - 1)
        self.dts = np.full(self.N, self.dt)
        self.NQ = march.nq_points(self.N)
        self.ts = march.stage_times(self.dts, rk)
        self.m = self.ts.shape[1]
        a, b, c = (self.V[self.T[:, k]] for k in range(3))
        cr = np.cross(b - a, c - a)
        self.area = 0.5 * np.linalg.norm(cr, axis=1)
        self.nrm = cr / np.linalg.norm(cr, axis=1, keepdims=True)
        self.corners = (a, b, c)

    def g(self):
        """[N, nv, m] Dirichlet data at the stage times."""
        return np.stack([np.stack([march.pulse_field(self.V, self.ts[n, k], X_SRC) for k in range(self.m)], axis=1)
                         for n in range(self.N)])

    def mass_half(self):
        Mh = np.zeros((len(self.T), len(self.V)))
        for i, tri in enumerate(self.T):
            for v in tri:
                Mh[i, v] += 0.5 * self.area[i] / 3.0
        return Mh

    def lmax(self, q, bary, w7):
        """max over steps of the L2 error of q[n, :, last stage] at t_n."""
        a, b, c = self.corners
        errs = []
        for n in range(self.N):
            e2 = 0.0
            for k in range(7):
                y = bary[k, 0] * a + bary[k, 1] * b + bary[k, 2] * c
                qe = march.pulse_flux(y, self.nrm, self.ts[n, -1], X_SRC)
                e2 += np.sum(w7[k] * self.area * (q[n, :, -1] - qe) ** 2)
            errs.append(np.sqrt(e2))
        return max(errs)


def oracle_solution(orc, P):
    """The oracle's dense FP64 marching of the problem (Sauter-Schwab ng = 5)."""
    m = orc.Mesh(P.V, P.T)
    rows, cols = np.arange(len(P.T)), np.arange(len(P.V))
    opV = march.CachedOperator(lambda z: m.entries(orc.SLP, rows, rows, [z], c=1.0, ng=5)[0])
    opK = march.CachedOperator(lambda z: m.entries(orc.DLP, rows, cols, [z], c=1.0, ng=5)[0])
    s, w, _ = orc.freqs_gcq(P.dt, P.dt, P.rk, P.NQ, P.N)
    return march.solve_dirichlet(opV, opK, P.mass_half(), P.g(), P.dts, P.rk, s, w)
