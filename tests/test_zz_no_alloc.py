"""The allocation-free entry point tdbem_entries_noalloc (collected last).

Some callers cannot allocate device memory when they ask for entries: for
example code that is capturing a stream into a CUDA graph (cudaMalloc and
cudaFree cannot be captured) or an application that reserves all device
memory up front for its own pool.  tdbem_entries_noalloc serves them from a
fixed scratch array inside the library.  This test calls it through the C-ABI
twice in a row and compares each result with tdbem_entries, the allocating
entry point, within the entry tolerances of the other GPU tests.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2505_00715_gb300.inputs import icosphere

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tol", [("FP64", 1e-12), ("MIXED", 1e-6)])
def test_noalloc_matches_allocating_entry_point(prec, tol):
    import torch

    import paper_2505_00715_gb300 as td
    from paper_2505_00715_gb300 import _lib

    ctx = td.Context(0)
    L = ctx.L
    V, T = icosphere(2)
    mesh = td.Mesh(ctx, V, T)
    f = td.Freqs.bdf2(ctx, 16, 0.1)
    rows = torch.arange(0, len(T), 3, dtype=torch.int32, device="cuda")
    fidx = torch.as_tensor(np.array([0, 3, 9, 15], dtype=np.int32), device="cuda")
    ct = torch.complex128 if prec == "FP64" else torch.complex64
    for opname, ncols in (("SLP", len(T)), ("DLP", len(V))):
        cols = torch.arange(ncols, dtype=torch.int32, device="cuda")
        op = _lib.Op(getattr(td, opname), getattr(td, prec), 1.0, 5, 0)
        ref = torch.empty((len(fidx), len(rows), ncols), dtype=ct, device="cuda")
        ctx.check(L.tdbem_entries(mesh.h, C.byref(op), f.h, C.c_void_p(rows.data_ptr()), len(rows),
                                  C.c_void_p(cols.data_ptr()), ncols, C.c_void_p(fidx.data_ptr()), len(fidx),
                                  C.c_void_p(ref.data_ptr())), "tdbem_entries")
        torch.cuda.synchronize()
        refn = ref.cpu().numpy()
        for call in range(2):
            out = torch.full((len(fidx), len(rows), ncols), float("nan"), dtype=ct, device="cuda")
            ctx.check(L.tdbem_entries_noalloc(mesh.h, C.byref(op), f.h, C.c_void_p(rows.data_ptr()), len(rows),
                                              C.c_void_p(cols.data_ptr()), ncols, C.c_void_p(fidx.data_ptr()),
                                              len(fidx), C.c_void_p(out.data_ptr())), "tdbem_entries_noalloc")
            ctx.sync()
            got = out.cpu().numpy()
            assert np.all(np.isfinite(got)), (opname, call)
            err = np.max(np.abs(got - refn)) / np.max(np.abs(refn))
            assert err <= tol, (opname, call, err)


def test_noalloc_rejects_too_many_frequencies():
    import torch

    import paper_2505_00715_gb300 as td
    from paper_2505_00715_gb300 import _lib

    ctx = td.Context(0)
    V, T = icosphere(1)
    mesh = td.Mesh(ctx, V, T)
    f = td.Freqs.bdf2(ctx, 8200, 1e-3)  # more points than the fixed scratch holds
    rows = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.empty(1, dtype=torch.complex64, device="cuda")
    op = _lib.Op(td.SLP, td.MIXED, 1.0, 5, 0)
    rc = ctx.L.tdbem_entries_noalloc(mesh.h, C.byref(op), f.h, C.c_void_p(rows.data_ptr()), 1,
                                     C.c_void_p(rows.data_ptr()), 1, C.c_void_p(rows.data_ptr()), 1,
                                     C.c_void_p(out.data_ptr()))
    assert rc == -1
    assert b"at most" in ctx.L.tdbem_last_error(ctx.h)
