"""tdbem: GB300 library for the 3D-ACA-compressed operator tensor of a
time-domain Galerkin BEM over convolution-quadrature frequencies, and its
multi-frequency apply.

Method: Schanz, Lakshmi Keshava, De Gersem, "Comparison of H-matrix- and
FMM-based 3D-ACA for a time-domain boundary element method" (arXiv 2505.00715).

This package is a thin layer over the C-ABI of libtdbem.so (include/tdbem.h);
PyTorch is used only for device buffers.  All numerical work runs in the CUDA
library; the calls raise if the library or a CUDA device is unavailable.
"""
import ctypes as C
import os

import numpy as np

from . import _lib
from ._lib import ADLP, DLP, EULER, FP64, MIXED, P0, P1, RADAU2, SLP, TdbemError

__all__ = ["Context", "Mesh", "Freqs", "Tree", "Tensor", "Model", "entries", "PATH_GENERIC", "PATH_NEAR",
           "PATH_FIBRE", "compress", "harvest", "rank_bin", "autotune",
           "SLP", "DLP", "ADLP", "P0", "P1", "FP64", "MIXED", "EULER", "RADAU2", "TdbemError", "March", "march_step_points",
           "lowrank_recompress"]
NPARAMS = 5648


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise TdbemError("tdbem needs a CUDA device; none is available")
    return torch


def _ptr(t):
    if not t.is_contiguous():
        raise TdbemError("tensor must be contiguous")
    return C.c_void_p(t.data_ptr())


def _np_ptr(a):
    return a.ctypes.data_as(C.c_void_p)


class Context:
    """One CUDA device and stream (the torch current stream by default)."""

    def __init__(self, device=0, stream=None):
        torch = _torch()
        self.L = _lib.load()
        self.device = device
        torch.cuda.set_device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        h = C.c_void_p()
        rc = self.L.tdbem_ctx_create(device, C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if rc != 0:
            raise TdbemError("tdbem_ctx_create failed with status %d" % rc)
        self.h = h

    def check(self, rc, what):
        _lib.check(rc, self.h, what)

    def sync(self):
        self.check(self.L.tdbem_ctx_sync(self.h), "tdbem_ctx_sync")

    def measure_peak(self, what):
        """Measured operations per second: "fma32", "sfu", "fma64" or "pair64"
        (FP64 single-layer point pairs)."""
        code = {"fma32": 0, "sfu": 1, "fma64": 2, "pair64": 3}[what]
        v = C.c_double()
        self.check(self.L.tdbem_measure_peak(self.h, code, C.byref(v)), "tdbem_measure_peak")
        return v.value

    def set_pool_scale(self, scale):
        """Scale of the far part of the first face-pool size in compress."""
        self.check(self.L.tdbem_ctx_set_pool_scale(self.h, float(scale)), "tdbem_ctx_set_pool_scale")

    def set_wait_limit(self, polls):
        """Poll limit of the tensor-core waits (0: default); see tdbem_ctx_set_wait_limit."""
        self.check(self.L.tdbem_ctx_set_wait_limit(self.h, int(polls)), "tdbem_ctx_set_wait_limit")

    def set_near_batch(self, nbytes):
        """Buffer size (bytes) of the batched near-field tensor in compress."""
        self.check(self.L.tdbem_ctx_set_near_batch(self.h, int(nbytes)), "tdbem_ctx_set_near_batch")

    def __del__(self):
        if getattr(self, "h", None) and _lib._lib is not None:
            _lib._lib.tdbem_ctx_destroy(self.h)
            self.h = None


class Mesh:
    def __init__(self, ctx, verts, tris):
        self.ctx = ctx
        self.verts = np.ascontiguousarray(verts, dtype=np.float64)
        self.tris = np.ascontiguousarray(tris, dtype=np.int32)
        h = C.c_void_p()
        ctx.check(ctx.L.tdbem_mesh_create(ctx.h, _np_ptr(self.verts), len(self.verts), _np_ptr(self.tris),
                                          len(self.tris), C.byref(h)), "tdbem_mesh_create")
        self.h = h

    def ndof(self, basis):
        return int(self.ctx.L.tdbem_mesh_ndof(self.h, basis))

    def __del__(self):
        if getattr(self, "h", None) and _lib._lib is not None:
            _lib._lib.tdbem_mesh_destroy(self.h)
            self.h = None


class Freqs:
    def __init__(self, ctx, h):
        self.ctx, self.h = ctx, h
        NQ, Nu = C.c_int32(), C.c_int32()
        ctx.check(ctx.L.tdbem_freqs_get(h, None, None, C.byref(NQ), C.byref(Nu), None), "tdbem_freqs_get")
        self.NQ, self.Nu = NQ.value, Nu.value
        s = np.zeros(2 * self.NQ)
        w = np.zeros(2 * self.NQ)
        u = np.zeros(self.NQ, dtype=np.int32)
        ctx.check(ctx.L.tdbem_freqs_get(h, _np_ptr(s), _np_ptr(w), None, None, _np_ptr(u)), "tdbem_freqs_get")
        self.s = s.view(np.complex128)
        self.w = w.view(np.complex128)
        self.unique_map = u
        # representative point of each unique frequency (u[k] = rep + 1 there)
        self.unique = np.array([k for k in range(self.NQ) if u[k] > 0], dtype=np.int32)

    @classmethod
    def bdf2(cls, ctx, N, dt, lam=0.0):
        h = C.c_void_p()
        ctx.check(ctx.L.tdbem_freqs_cq_bdf2(ctx.h, N, dt, lam, C.byref(h)), "tdbem_freqs_cq_bdf2")
        return cls(ctx, h)

    @classmethod
    def gcq(cls, ctx, dts, rk, NQ, rho=0.0):
        """gCQ contour of App. A for the time steps dts (host array) and the
        Runge-Kutta method rk (EULER or RADAU2), NQ contour points; the circle
        through 0 and 2 rho / dt_min (rho = 1: as printed; rho <= 0: the
        radius the time marching needs)."""
        h = C.c_void_p()
        d = np.ascontiguousarray(dts, dtype=np.float64)
        ctx.check(ctx.L.tdbem_freqs_gcq(ctx.h, _np_ptr(d), len(d), rk, NQ, float(rho), C.byref(h)), "tdbem_freqs_gcq")
        return cls(ctx, h)

    @classmethod
    def points(cls, ctx, s, w=None):
        """A set of explicit points (host complex array, Re s > 0), optional weights."""
        sv = np.ascontiguousarray(np.asarray(s, dtype=np.complex128)).view(np.float64)
        wv = None if w is None else np.ascontiguousarray(np.asarray(w, dtype=np.complex128)).view(np.float64)
        h = C.c_void_p()
        ctx.check(ctx.L.tdbem_freqs_points(ctx.h, _np_ptr(sv), None if wv is None else _np_ptr(wv), len(sv) // 2,
                                           C.byref(h)), "tdbem_freqs_points")
        return cls(ctx, h)

    def steps(self):
        """Time steps of a gCQ set (empty for BDF2)."""
        n = C.c_int32()
        self.ctx.check(self.ctx.L.tdbem_freqs_steps(self.h, None, C.byref(n)), "tdbem_freqs_steps")
        d = np.zeros(n.value)
        if n.value:
            self.ctx.check(self.ctx.L.tdbem_freqs_steps(self.h, _np_ptr(d), C.byref(n)), "tdbem_freqs_steps")
        return d

    def __del__(self):
        if getattr(self, "h", None) and _lib._lib is not None:
            _lib._lib.tdbem_freqs_destroy(self.h)
            self.h = None


class Tree:
    def __init__(self, mesh, row_basis, col_basis, leaf, eta):
        self.mesh = mesh
        ctx = mesh.ctx
        h = C.c_void_p()
        ctx.check(ctx.L.tdbem_tree_build(mesh.h, row_basis, col_basis, leaf, eta, C.byref(h)), "tdbem_tree_build")
        self.h = h
        nb = C.c_int64()
        ctx.check(ctx.L.tdbem_tree_export(h, None, None, C.byref(nb), None), "tdbem_tree_export")
        self.perm_rows = np.zeros(mesh.ndof(row_basis), dtype=np.int32)
        self.perm_cols = np.zeros(mesh.ndof(col_basis), dtype=np.int32)
        self.blocks = np.zeros((nb.value, 5), dtype=np.int32)
        ctx.check(ctx.L.tdbem_tree_export(h, _np_ptr(self.perm_rows), _np_ptr(self.perm_cols), None,
                                          _np_ptr(self.blocks)), "tdbem_tree_export")

    def __del__(self):
        if getattr(self, "h", None) and _lib._lib is not None:
            _lib._lib.tdbem_tree_destroy(self.h)
            self.h = None


def _op(op, prec, c, ng):
    return _lib.Op(op, prec, c, ng, 0)


def _cdtype(prec):
    torch = _torch()
    return torch.complex128 if prec == FP64 else torch.complex64


PATH_GENERIC, PATH_NEAR, PATH_FIBRE = 0, 1, 2


def entries(mesh, op, freqs, rows, cols, fidx, prec=MIXED, c=1.0, ng=5, path=PATH_GENERIC):
    """A[rows, cols](s_fidx) as a device tensor [nf, nr, nc] (complex64 MIXED, complex128 FP64).
    path selects the kernel: PATH_GENERIC (tdbem_entries), PATH_NEAR (the
    compression's touching-pair table and near-field tensor kernels on the
    block rows x cols) or PATH_FIBRE (the far-field engine's point-pair groups;
    regular rule on every pair)."""
    torch = _torch()
    ctx = mesh.ctx
    dev = torch.device("cuda", ctx.device)
    r = torch.as_tensor(np.asarray(rows, dtype=np.int32), device=dev)
    q = torch.as_tensor(np.asarray(cols, dtype=np.int32), device=dev)
    f = torch.as_tensor(np.asarray(fidx, dtype=np.int32), device=dev)
    out = torch.empty((len(f), len(r), len(q)), dtype=_cdtype(prec), device=dev)
    o = _op(op, prec, c, ng)
    if path == PATH_GENERIC:
        ctx.check(ctx.L.tdbem_entries(mesh.h, C.byref(o), freqs.h, _ptr(r), len(r), _ptr(q), len(q), _ptr(f), len(f),
                                      _ptr(out)), "tdbem_entries")
    else:
        ctx.check(ctx.L.tdbem_entries_path(mesh.h, C.byref(o), freqs.h, _ptr(r), len(r), _ptr(q), len(q), _ptr(f),
                                           len(f), int(path), _ptr(out)), "tdbem_entries_path")
    return out


class Tensor:
    """3D-ACA compressed operator tensor held in device memory."""

    def __init__(self, ctx, h, mesh=None, freqs=None, tree=None):
        self.ctx, self.h, self.mesh, self.freqs, self.tree = ctx, h, mesh, freqs, tree
        op, prec, nq, nu = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        nr, nc = C.c_int64(), C.c_int64()
        ctx.check(ctx.L.tdbem_tensor_info(h, C.byref(op), C.byref(prec), C.byref(nr), C.byref(nc), C.byref(nq),
                                          C.byref(nu)), "tdbem_tensor_info")
        self.op, self.prec = op.value, prec.value
        self.nrows, self.ncols, self.NQ, self.Nu = nr.value, nc.value, nq.value, nu.value

    @classmethod
    def load(cls, ctx, path, mesh=None, freqs=None, tree=None):
        """Read a tensor written by save() (the mesh, frequency set and tree
        are not stored; pass them to keep them attached)."""
        h = C.c_void_p()
        ctx.check(ctx.L.tdbem_tensor_load(ctx.h, os.fsencode(path), C.byref(h)), "tdbem_tensor_load")
        return cls(ctx, h, mesh, freqs, tree)

    def save(self, path):
        self.ctx.check(self.ctx.L.tdbem_tensor_save(self.h, os.fsencode(path)), "tdbem_tensor_save")

    def stats(self):
        st = _lib.Stats()
        self.ctx.check(self.ctx.L.tdbem_tensor_stats(self.h, C.byref(st)), "tdbem_tensor_stats")
        return st.as_dict()

    def partition(self):
        """The compression partition [nblocks][5] (row/column ranges in the
        tree's permuted order, far flag); it refines the tree's blocks."""
        nb = C.c_int64()
        self.ctx.check(self.ctx.L.tdbem_tensor_partition(self.h, C.byref(nb), None), "tdbem_tensor_partition")
        out = np.zeros((nb.value, 5), dtype=np.int32)
        self.ctx.check(self.ctx.L.tdbem_tensor_partition(self.h, C.byref(nb), _np_ptr(out)), "tdbem_tensor_partition")
        return out

    def blocks(self):
        nb = self.stats()["nblocks"]
        r = np.zeros(nb, dtype=np.int32)
        k = np.zeros(nb, dtype=np.int32)
        kp = np.zeros((nb, self.Nu + 1), dtype=np.int32)
        self.ctx.check(self.ctx.L.tdbem_tensor_blocks(self.h, _np_ptr(r), _np_ptr(k), _np_ptr(kp)),
                       "tdbem_tensor_blocks")
        return r, k, kp

    def entries(self, rows, cols, fidx):
        torch = _torch()
        dev = torch.device("cuda", self.ctx.device)
        r = torch.as_tensor(np.asarray(rows, dtype=np.int32), device=dev)
        q = torch.as_tensor(np.asarray(cols, dtype=np.int32), device=dev)
        f = torch.as_tensor(np.asarray(fidx, dtype=np.int32), device=dev)
        out = torch.empty(len(r), dtype=_cdtype(self.prec), device=dev)
        self.ctx.check(self.ctx.L.tdbem_tensor_entries(self.h, _ptr(r), _ptr(q), _ptr(f), len(r), _ptr(out)),
                       "tdbem_tensor_entries")
        return out

    def apply_weighted(self, W, y=None):
        """y = sum_l A(s_l) W[l]; W: device tensor [NQ, ncols, nrhs] of the tensor's complex dtype."""
        torch = _torch()
        nrhs = W.shape[2]
        if y is None:
            y = torch.empty((self.nrows, nrhs), dtype=W.dtype, device=W.device)
        self.ctx.check(self.ctx.L.tdbem_apply_weighted(self.h, _ptr(W), nrhs, _ptr(y)), "tdbem_apply_weighted")
        return y

    def apply_freq(self, fidx, x, y=None):
        torch = _torch()
        nrhs = x.shape[1]
        if y is None:
            y = torch.empty((self.nrows, nrhs), dtype=x.dtype, device=x.device)
        self.ctx.check(self.ctx.L.tdbem_apply_freq(self.h, fidx, _ptr(x), nrhs, _ptr(y)), "tdbem_apply_freq")
        return y

    def apply_weighted_host(self, W_host, y_host):
        """Host buffers (numpy or pinned torch CPU tensors); copies are part of the call."""
        wp = C.c_void_p(W_host.data_ptr()) if hasattr(W_host, "data_ptr") else _np_ptr(W_host)
        yp = C.c_void_p(y_host.data_ptr()) if hasattr(y_host, "data_ptr") else _np_ptr(y_host)
        nrhs = W_host.shape[2]
        self.ctx.check(self.ctx.L.tdbem_apply_weighted_host(self.h, wp, nrhs, yp), "tdbem_apply_weighted_host")
        return y_host

    def recompress(self, eps):
        """QR + SVD recompression of every far face to ||H - H'||_F <= eps ||H||_F."""
        self.ctx.check(self.ctx.L.tdbem_tensor_recompress(self.h, float(eps)), "tdbem_tensor_recompress")
        return self

    def solve(self, fidx, b, tol=1e-6, maxit=500, restart=30, x=None, check=True):
        """x with A(s_fidx) x = b by restarted GMRES; b: device [nrows, nrhs].
        Returns (x, iterations, relative residuals).  With check=False a
        solve that stops above tol returns its last iterate instead of raising."""
        torch = _torch()
        nrhs = b.shape[1]
        if x is None:
            x = torch.empty_like(b)
        it = C.c_int32()
        rr = np.zeros(nrhs)
        rc = self.ctx.L.tdbem_solve(self.h, fidx, _ptr(b), nrhs, _ptr(x), tol, maxit, restart, C.byref(it), _np_ptr(rr))
        if check or rc != _lib.ERR_NOT_CONVERGED:
            self.ctx.check(rc, "tdbem_solve")
        return x, it.value, rr

    def __del__(self):
        if getattr(self, "h", None) and _lib._lib is not None:
            _lib._lib.tdbem_tensor_destroy(self.h)
            self.h = None


def compress(mesh, op, freqs, tree, eps=1e-4, eps_aca=1e-6, prec=MIXED, c=1.0, ng=5, max_face_rank=64,
             use_graph=True, model=None, dense_faces=True, balance=True):
    """3D-ACA compression of the operator tensor on the tree's blocks.
    balance=False keeps the tree's partition; by default far blocks larger
    than twice the mean far work of one persistent CTA are compressed as the
    blocks of their clusters' sons (Tensor.partition())."""
    ctx = mesh.ctx
    o = _op(op, prec, c, ng)
    flags = (0 if use_graph else 1) | (0 if dense_faces else 2) | (0 if balance else 4)
    cfg = _lib.AcaCfg(eps, eps_aca, max_face_rank, flags, model.h if model is not None else None)
    h = C.c_void_p()
    ctx.check(ctx.L.tdbem_compress(ctx.h, mesh.h, C.byref(o), freqs.h, tree.h, C.byref(cfg), C.byref(h)),
              "tdbem_compress")
    return Tensor(ctx, h, mesh, freqs, tree)


def autotune(mesh, op, freqs, tree, eps=1e-4, eps_aca=1e-6, prec=MIXED, c=1.0, ng=5, max_face_rank=64, model=None):
    """Time the compression with candidate launch parameters and keep the fastest
    per phase in the context; returns (far threads per CTA, far CTAs per SM,
    touching-pair frequencies per pass, near-field frequencies per pass)."""
    ctx = mesh.ctx
    o = _op(op, prec, c, ng)
    cfg = _lib.AcaCfg(eps, eps_aca, max_face_rank, 0, model.h if model is not None else None)
    ch = (C.c_int32 * 4)()
    ctx.check(ctx.L.tdbem_autotune(ctx.h, mesh.h, C.byref(o), freqs.h, tree.h, C.byref(cfg), ch), "tdbem_autotune")
    return tuple(int(x) for x in ch)


def lowrank_recompress(ctx, U, V, eps):
    """Recompress one face U V^T (device tensors U [k, nI], V [k, nJ], complex64
    or complex128) to ||H - H'||_F <= eps ||H||_F; returns (U', V')."""
    torch = _torch()
    k, nI = U.shape
    nJ = V.shape[1]
    prec = FP64 if U.dtype == torch.complex128 else MIXED
    Uo, Vo = torch.empty_like(U), torch.empty_like(V)
    kn = C.c_int32()
    ctx.check(ctx.L.tdbem_lowrank_recompress(ctx.h, prec, nI, nJ, k, _ptr(U.contiguous()), _ptr(V.contiguous()),
                                             float(eps), _ptr(Uo), _ptr(Vo), C.byref(kn)), "tdbem_lowrank_recompress")
    return Uo[:kn.value], Vo[:kn.value]


def march_step_points(dts, rk):
    """The distinct step frequencies 1/(dt lambda_k(A)) of the steps (complex array)."""
    L = _lib.load()
    d = np.ascontiguousarray(dts, dtype=np.float64)
    n = C.c_int32()
    _lib.check(L.tdbem_march_step_points(_np_ptr(d), len(d), rk, None, C.byref(n)), None, "tdbem_march_step_points")
    out = np.zeros(2 * n.value)
    _lib.check(L.tdbem_march_step_points(_np_ptr(d), len(d), rk, _np_ptr(out), C.byref(n)), None,
               "tdbem_march_step_points")
    return out.view(np.complex128)


class March:
    """gCQ time marching of the direct Dirichlet problem V * q = (1/2 M + K) * g
    (include/tdbem.h): V, K compressed over a gCQ contour, Vstep, Kstep over
    the step frequencies."""

    def __init__(self, V, K, Vstep, Kstep, dts, rk, nrhs):
        self.ctx = V.ctx
        self.tensors = (V, K, Vstep, Kstep)
        d = np.ascontiguousarray(dts, dtype=np.float64)
        h = C.c_void_p()
        self.ctx.check(self.ctx.L.tdbem_march_create(V.h, K.h, Vstep.h, Kstep.h, _np_ptr(d), len(d), rk, nrhs,
                                                     C.byref(h)), "tdbem_march_create")
        self.h = h
        self.m = 2 if rk == RADAU2 else 1
        self.nrhs = nrhs

    def step(self, g, q=None, tol=1e-8, maxit=500):
        """g: device float64 [nv, m, nrhs]; returns q: device float64 [nt, m, nrhs] and the GMRES steps."""
        torch = _torch()
        if q is None:
            q = torch.empty((self.tensors[0].nrows, self.m, self.nrhs), dtype=torch.float64, device=g.device)
        it = C.c_int32()
        self.ctx.check(self.ctx.L.tdbem_march_step(self.h, _ptr(g), _ptr(q), tol, maxit, C.byref(it)),
                       "tdbem_march_step")
        return q, it.value

    def __del__(self):
        if getattr(self, "h", None) and _lib._lib is not None:
            _lib._lib.tdbem_march_destroy(self.h)
            self.h = None


def zgemm(ctx, A, B, D=None):
    """D = A @ B for complex64 device matrices on the tensor cores (split BF16)."""
    torch = _torch()
    M, K = A.shape
    K2, N = B.shape
    assert K2 == K and A.dtype == torch.complex64 and B.dtype == torch.complex64
    A = A.contiguous()
    B = B.contiguous()
    if D is None:
        D = torch.empty((M, N), dtype=torch.complex64, device=A.device)
    ctx.check(ctx.L.tdbem_zgemm(ctx.h, M, N, K, _ptr(A), K, _ptr(B), N, _ptr(D), N), "tdbem_zgemm")
    return D


def rank_bin(rank):
    return int(_lib.load().tdbem_rank_bin(int(rank)))


class Model:
    """Rank-predictor MLP (6 -> 64 -> 64 -> 16) held on the device."""

    def __init__(self, ctx, seed=2):
        self.ctx = ctx
        h = C.c_void_p()
        ctx.check(ctx.L.tdbem_model_create(ctx.h, seed, C.byref(h)), "tdbem_model_create")
        self.h = h

    def params(self):
        p = np.zeros(NPARAMS, dtype=np.float32)
        self.ctx.check(self.ctx.L.tdbem_model_get_params(self.h, _np_ptr(p)), "tdbem_model_get_params")
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        self.ctx.check(self.ctx.L.tdbem_model_set_params(self.h, _np_ptr(p)), "tdbem_model_set_params")

    def loss_grad(self, x, labels):
        torch = _torch()
        g = torch.empty(NPARAMS, dtype=torch.float32, device=x.device)
        loss = torch.empty(1, dtype=torch.float32, device=x.device)
        self.ctx.check(self.ctx.L.tdbem_model_loss_grad(self.h, _ptr(x), _ptr(labels), x.shape[0], _ptr(g), _ptr(loss)),
                       "tdbem_model_loss_grad")
        return loss, g

    def adam_step(self, grad, lr, t):
        self.ctx.check(self.ctx.L.tdbem_model_adam_step(self.h, _ptr(grad), lr, t), "tdbem_model_adam_step")

    def train(self, x, labels, epochs=10, batch=4096, lr=3e-3, seed=3):
        fl = C.c_double()
        self.ctx.check(self.ctx.L.tdbem_model_train(self.h, _ptr(x), _ptr(labels), x.shape[0], epochs, batch, lr, seed,
                                                    C.byref(fl)), "tdbem_model_train")
        return fl.value

    def save(self, path):
        self.ctx.check(self.ctx.L.tdbem_model_save(self.h, os.fsencode(path)), "tdbem_model_save")

    @classmethod
    def load(cls, ctx, path):
        m = cls.__new__(cls)
        m.ctx = ctx
        m.h = None
        h = C.c_void_p()
        ctx.check(ctx.L.tdbem_model_load(ctx.h, os.fsencode(path), C.byref(h)), "tdbem_model_load")
        m.h = h
        return m

    def predict(self, x, logits=False):
        torch = _torch()
        bins = torch.empty(x.shape[0], dtype=torch.int32, device=x.device)
        lg = torch.empty((x.shape[0], 16), dtype=torch.float32, device=x.device) if logits else None
        self.ctx.check(self.ctx.L.tdbem_model_predict(self.h, _ptr(x), x.shape[0], _ptr(bins),
                                                      _ptr(lg) if logits else None), "tdbem_model_predict")
        return (bins, lg) if logits else bins

    def __del__(self):
        if getattr(self, "h", None) and _lib._lib is not None:
            _lib._lib.tdbem_model_destroy(self.h)
            self.h = None


def harvest(mesh, op, freqs, tree, eps_aca=1e-6, prec=MIXED, c=1.0, ng=5, max_face_rank=64):
    """(features [n, 6] float32, face-ACA ranks [n] int32) device tensors for
    every (far block, unique frequency) of the tree."""
    torch = _torch()
    ctx = mesh.ctx
    o = _op(op, prec, c, ng)
    cfg = _lib.AcaCfg(1e-4, eps_aca, max_face_rank, 0, None)
    n = C.c_int64()
    ctx.check(ctx.L.tdbem_harvest(ctx.h, mesh.h, C.byref(o), freqs.h, tree.h, C.byref(cfg), None, None, 0, C.byref(n)),
              "tdbem_harvest")
    dev = torch.device("cuda", ctx.device)
    x = torch.empty((n.value, 6), dtype=torch.float32, device=dev)
    r = torch.empty(n.value, dtype=torch.int32, device=dev)
    ctx.check(ctx.L.tdbem_harvest(ctx.h, mesh.h, C.byref(o), freqs.h, tree.h, C.byref(cfg), _ptr(x), _ptr(r), n.value,
                                  C.byref(n)), "tdbem_harvest")
    return x, r
