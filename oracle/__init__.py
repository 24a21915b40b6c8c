"""Oracle: a plain, slow FP64 CPU restatement of the time-domain BEM tensor path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library in ``paper_2505_00715_gb300`` and never imports it.

The numerics live in C (``orc_*.c``); this module only marshals numpy arrays.
Complex arrays cross the boundary as complex128 numpy arrays.

Parity unpinned: nothing here — every routine is pinned by ``tests/test_oracle_*``
(closed forms, exact quadrature, brute force, library routines, invariants).
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

SLP, DLP, ADLP = 0, 1, 2
P0, P1 = 0, 1
EULER, RADAU2 = 0, 1

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        vp, i64, i32, d = C.c_void_p, C.c_int64, C.c_int, C.c_double
        sig = {
            "orc_mesh_new": (vp, [vp, i64, vp, i64]),
            "orc_mesh_free": (None, [vp]),
            "orc_mesh_ndof": (i64, [vp, i32]),
            "orc_rule7": (None, [vp, vp]),
            "orc_gauss01": (i32, [i32, vp, vp]),
            "orc_pair": (i32, [vp, i32, i64, i64, d, d, d, i32, vp]),
            "orc_pair_regular": (None, [vp, i32, i64, i64, d, d, d, vp]),
            "orc_entry": (None, [vp, i32, i64, i64, d, d, d, i32, vp]),
            "orc_entries": (None, [vp, i32, vp, i64, vp, i64, vp, i64, d, i32, vp]),
            "orc_entries_mag": (None, [vp, i32, vp, i64, vp, i64, vp, i64, d, i32, vp]),
            "orc_freqs_bdf2": (i32, [i32, d, d, vp]),
            "orc_ellipk": (d, [d]),
            "orc_ellipj": (None, [d, d, vp, vp, vp]),
            "orc_ellipj_complex": (None, [d, d, d, vp, vp, vp]),
            "orc_freqs_gcq": (i32, [d, d, i32, i32, d, i32, vp, vp, vp]),
            "orc_gcq_radius": (d, [i32, i32]),
            "orc_tree_build": (vp, [vp, i32, i32, i32, d]),
            "orc_tree_free": (None, [vp]),
            "orc_tree_nblocks": (i64, [vp]),
            "orc_tree_export": (None, [vp, vp, vp, vp]),
            "orc_tree_nclusters": (i64, [vp, i32]),
            "orc_tree_clusters": (None, [vp, i32, vp, vp]),
            "orc_aca_dense": (i32, [vp, i32, i32, d, i32, vp, vp]),
            "orc_aca3d_dense": (i32, [vp, i32, i32, i32, d, i32, vp, vp, vp]),
            "orc_aca3d_dense_acaface": (i32, [vp, i32, i32, i32, d, d, i32, vp, vp, vp, vp]),
            "orc_compress": (vp, [vp, i32, d, i32, vp, i32, vp, d, d, i32, i32, vp]),
            "orc_tensor_free": (None, [vp]),
            "orc_tensor_stats": (None, [vp, vp]),
            "orc_tensor_block_ranks": (None, [vp, vp, vp]),
            "orc_tensor_entry": (None, [vp, i64, i64, i32, vp]),
            "orc_tensor_apply": (None, [vp, vp, i32, vp]),
            "orc_dense_apply_rows": (None, [vp, i32, d, i32, vp, i32, vp, i64, vp, i32, vp, i32]),
            "orc_mlp_nparams": (i32, []),
            "orc_mlp_forward": (None, [vp, vp, i64, vp]),
            "orc_mlp_loss_grad": (d, [vp, vp, vp, i64, vp]),
            "orc_adam_step": (None, [vp, vp, vp, vp, i64, d, d, d, d, i32]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


class Mesh:
    """Flat triangle mesh (vertices FP64 [nv,3], triangles int32 [nt,3])."""

    def __init__(self, verts, tris):
        self.verts = np.ascontiguousarray(verts, dtype=np.float64)
        self.tris = np.ascontiguousarray(tris, dtype=np.int32)
        self.h = lib().orc_mesh_new(_p(self.verts), len(self.verts), _p(self.tris), len(self.tris))
        if not self.h:
            raise ValueError("invalid mesh (index out of range or degenerate triangle)")

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.orc_mesh_free(self.h)
            self.h = None

    def ndof(self, basis):
        return int(lib().orc_mesh_ndof(self.h, basis))

    def pair(self, op, ti, tj, s, c=1.0, ng=6):
        out = np.zeros(6)
        cls = lib().orc_pair(self.h, op, ti, tj, float(np.real(s)), float(np.imag(s)), c, ng, _p(out))
        return cls, out.view(np.complex128)

    def pair_regular(self, op, ti, tj, s, c=1.0):
        out = np.zeros(6)
        lib().orc_pair_regular(self.h, op, ti, tj, float(np.real(s)), float(np.imag(s)), c, _p(out))
        return out.view(np.complex128)

    def entry(self, op, row, col, s, c=1.0, ng=6):
        out = np.zeros(2)
        lib().orc_entry(self.h, op, row, col, float(np.real(s)), float(np.imag(s)), c, ng, _p(out))
        return complex(out[0], out[1])

    def entries(self, op, rows, cols, s, c=1.0, ng=6):
        rows = np.ascontiguousarray(rows, dtype=np.int32)
        cols = np.ascontiguousarray(cols, dtype=np.int32)
        s = _c128(np.atleast_1d(s))
        out = np.zeros((len(s), len(rows), len(cols)), dtype=np.complex128)
        lib().orc_entries(self.h, op, _p(rows), len(rows), _p(cols), len(cols), _p(s), len(s), c, ng,
                          _p(out))
        return out

    def entries_mag(self, op, rows, cols, s, c=1.0, ng=6):
        """Magnitude sums [nf, nr, nc] (real) of the entries: the same
        quadrature with every term replaced by a bound of its modulus."""
        rows = np.ascontiguousarray(rows, dtype=np.int32)
        cols = np.ascontiguousarray(cols, dtype=np.int32)
        s = _c128(np.atleast_1d(s))
        out = np.zeros((len(s), len(rows), len(cols)))
        lib().orc_entries_mag(self.h, op, _p(rows), len(rows), _p(cols), len(cols), _p(s), len(s), c, ng,
                              _p(out))
        return out

    def dense_apply_rows(self, op, s, rows, W, c=1.0, ng=6, nthreads=0):
        """y[r] = sum_f sum_j A(s_f)[rows[r], j] W[f, j, :]."""
        rows = np.ascontiguousarray(rows, dtype=np.int32)
        s = _c128(s)
        W = _c128(W)
        nrhs = W.shape[2]
        y = np.zeros((len(rows), nrhs), dtype=np.complex128)
        lib().orc_dense_apply_rows(self.h, op, c, ng, _p(s), len(s), _p(rows), len(rows), _p(W), nrhs,
                                   _p(y), nthreads)
        return y


def rule7():
    b = np.zeros((7, 3))
    w = np.zeros(7)
    lib().orc_rule7(_p(b), _p(w))
    return b, w


def gauss01(n):
    x = np.zeros(n)
    w = np.zeros(n)
    if lib().orc_gauss01(n, _p(x), _p(w)) != 0:
        raise ValueError("bad order")
    return x, w


def freqs_bdf2(N, dt, lam=0.0):
    s = np.zeros(N, dtype=np.complex128)
    if lib().orc_freqs_bdf2(N, dt, lam, _p(s)) != 0:
        raise ValueError("bad BDF2 parameters")
    return s


def ellipk(m):
    return lib().orc_ellipk(m)


def ellipj(u, m):
    sn, cn, dn = C.c_double(), C.c_double(), C.c_double()
    lib().orc_ellipj(u, m, C.byref(sn), C.byref(cn), C.byref(dn))
    return sn.value, cn.value, dn.value


def ellipj_complex(z, m):
    sn, cn, dn = np.zeros(2), np.zeros(2), np.zeros(2)
    lib().orc_ellipj_complex(float(np.real(z)), float(np.imag(z)), m, _p(sn), _p(cn), _p(dn))
    return complex(*sn), complex(*cn), complex(*dn)


def freqs_gcq(dt_min, dt_max, rk, NQ, nsteps, rho=0.0):
    """gCQ contour points and weights (App. A) for nsteps steps in
    [dt_min, dt_max]; rk 0 implicit Euler, 1 Radau IIA (2 stages).  rho > 0:
    the circle through 0 and 2 rho / dt_min (rho = 1: as printed); rho <= 0:
    the radius that the marching needs (orc_gcq_radius)."""
    s = np.zeros(NQ, dtype=np.complex128)
    w = np.zeros(NQ, dtype=np.complex128)
    info = np.zeros(5)
    rc = lib().orc_freqs_gcq(dt_min, dt_max, rk, nsteps, float(rho), NQ, _p(s), _p(w), _p(info))
    if rc < 0:
        raise ValueError("bad gCQ parameters")
    return s, w, dict(q=info[0], k=info[1], K=info[2], Kp=info[3], rho=info[4], lifted=bool(rc))


def gcq_radius(rk, nsteps):
    return float(lib().orc_gcq_radius(rk, nsteps))


class Tree:
    """PCA cluster trees (rows P0, cols P0/P1) and the block cluster tree."""

    def __init__(self, mesh, row_basis, col_basis, leaf, eta):
        self.mesh = mesh
        self.h = lib().orc_tree_build(mesh.h, row_basis, col_basis, leaf, eta)
        if not self.h:
            raise ValueError("bad tree parameters")
        nb = lib().orc_tree_nblocks(self.h)
        self.perm_rows = np.zeros(mesh.ndof(row_basis), dtype=np.int32)
        self.perm_cols = np.zeros(mesh.ndof(col_basis), dtype=np.int32)
        self.blocks = np.zeros((nb, 5), dtype=np.int32)
        lib().orc_tree_export(self.h, _p(self.perm_rows), _p(self.perm_cols), _p(self.blocks))

    def clusters(self, side):
        n = lib().orc_tree_nclusters(self.h, side)
        nodes = np.zeros((n, 4), dtype=np.int32)
        box = np.zeros((n, 6))
        lib().orc_tree_clusters(self.h, side, _p(nodes), _p(box))
        return nodes, box

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.orc_tree_free(self.h)
            self.h = None


def aca_dense(a, eps, kmax=None):
    a = _c128(a)
    nI, nJ = a.shape
    kmax = kmax or min(nI, nJ)
    U = np.zeros((nI, kmax), dtype=np.complex128)
    V = np.zeros((nJ, kmax), dtype=np.complex128)
    r = lib().orc_aca_dense(_p(a), nI, nJ, eps, kmax, _p(U), _p(V))
    return U[:, :r], V[:, :r]


def aca3d_dense(t, eps, eps_aca=None):
    """3D-ACA of an explicit tensor t[k, i, j]; dense faces if eps_aca is None."""
    t = _c128(t)
    nK, nI, nJ = t.shape
    rmax = nK + 1
    kp = np.zeros(rmax, dtype=np.int32)
    H = np.zeros((rmax, nI, nJ), dtype=np.complex128)
    f = np.zeros((rmax, nK), dtype=np.complex128)
    if eps_aca is None:
        r = lib().orc_aca3d_dense(_p(t), nI, nJ, nK, eps, rmax, _p(kp), _p(H), _p(f))
        fr = None
    else:
        fr = np.zeros(rmax, dtype=np.int32)
        r = lib().orc_aca3d_dense_acaface(_p(t), nI, nJ, nK, eps, eps_aca, rmax, _p(kp), _p(H), _p(f),
                                          _p(fr))
        fr = fr[:r]
    return kp[:r], H[:r], f[:r], fr


class Tensor:
    """Block-compressed operator tensor from the oracle's 3D-ACA."""

    def __init__(self, mesh, op, s, tree, eps, eps_aca, c=1.0, ng=6, nthreads=0, block_stride=1, block_mask=None):
        """block_stride / block_mask: compress only every block_stride-th
        block, or only the blocks where block_mask (bool [nblocks]) is set."""
        self.s = _c128(s)
        self.mesh, self.tree = mesh, tree
        mask = None if block_mask is None else np.ascontiguousarray(block_mask, dtype=np.uint8)
        self._mask = mask
        self.h = lib().orc_compress(mesh.h, op, c, ng, _p(self.s), len(self.s), tree.h, eps, eps_aca,
                                    nthreads, block_stride, None if mask is None else _p(mask))
        st = np.zeros(9)
        lib().orc_tensor_stats(self.h, _p(st))
        self.stats = dict(nblocks=int(st[0]), nfar=int(st[1]), sum_rank=int(st[2]), max_rank=int(st[3]),
                          stored=st[4], dense=st[5], evals=st[6], sum_face_rank=int(st[7]), block_seconds=st[8])
        self.nrows = mesh.ndof(P0)
        self.ncols = mesh.ndof(P1 if op == DLP else P0)

    def block_ranks(self):
        nb = self.stats["nblocks"]
        r = np.zeros(nb, dtype=np.int32)
        k = np.zeros(nb, dtype=np.int32)
        lib().orc_tensor_block_ranks(self.h, _p(r), _p(k))
        return r, k

    def entry(self, row, col, f):
        out = np.zeros(2)
        lib().orc_tensor_entry(self.h, row, col, f, _p(out))
        return complex(out[0], out[1])

    def apply(self, W):
        W = _c128(W)
        nrhs = W.shape[2]
        y = np.zeros((self.nrows, nrhs), dtype=np.complex128)
        lib().orc_tensor_apply(self.h, _p(W), nrhs, _p(y))
        return y

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.orc_tensor_free(self.h)
            self.h = None


def mlp_nparams():
    return lib().orc_mlp_nparams()


def mlp_forward(params, x):
    params = np.ascontiguousarray(params, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros((len(x), 16))
    lib().orc_mlp_forward(_p(params), _p(x), len(x), _p(out))
    return out


def mlp_loss_grad(params, x, labels, want_grad=True):
    params = np.ascontiguousarray(params, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    g = np.zeros_like(params) if want_grad else None
    loss = lib().orc_mlp_loss_grad(_p(params), _p(x), _p(labels), len(x), _p(g) if want_grad else None)
    return loss, g


def adam_step(params, grad, m, v, lr, t, b1=0.9, b2=0.999, eps=1e-8):
    lib().orc_adam_step(_p(params), _p(np.ascontiguousarray(grad)), _p(m), _p(v), len(params), lr, b1, b2,
                        eps, t)


def conj_partner_apply(apply_fn, W_unique, W_partner):
    """sum over the full frequency list when A(conj s) = conj(A(s)):
    y = apply(W_u) + conj(apply(conj(W_partner))) (W_partner zero where a
    unique frequency has no partner)."""
    return apply_fn(W_unique) + np.conj(apply_fn(np.conj(W_partner)))


__all__ = ["Mesh", "Tree", "Tensor", "rule7", "gauss01", "freqs_bdf2", "freqs_gcq", "ellipk", "ellipj",
           "ellipj_complex", "aca_dense", "aca3d_dense", "mlp_nparams", "mlp_forward", "mlp_loss_grad",
           "adam_step", "SLP", "DLP", "ADLP", "P0", "P1", "EULER", "RADAU2", "lib"]
os.environ.setdefault("OMP_WAIT_POLICY", "PASSIVE")
