"""The allocation-free entry point tdbem_entries_noalloc (collected last).

Some callers cannot allocate device memory when they ask for entries: an
application that reserves all device memory up front for its own pool
allocator, or a host loop that must not pay the device-wide synchronisation
of cudaFree.  tdbem_entries_noalloc serves them from a fixed scratch array
inside the library.  This test calls it through the C-ABI twice in a row and
compares each result with tdbem_entries (the allocating entry point) and with
the FP64 oracle, within the entry tolerances of the other GPU tests, and
checks that the device's free memory is the same before and after a call.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2505_00715_gb300.inputs import icosphere

pytestmark = pytest.mark.gpu


def _rel_err(g, o):
    """max |g - o| / max(|o|, 1e-6 max|o| of the frequency slice)."""
    scale = np.max(np.abs(o).reshape(o.shape[0], -1), axis=1).reshape(-1, 1, 1)
    return float(np.max(np.abs(g - o) / np.maximum(np.abs(o), 1e-6 * scale)))


@pytest.mark.parametrize("prec,tol", [("FP64", 1e-12), ("MIXED", 1e-5)])
def test_noalloc_matches_allocating_entry_point_and_oracle(prec, tol):
    import torch

    import oracle as orc
    import paper_2505_00715_gb300 as td
    from paper_2505_00715_gb300 import _lib

    ctx = td.Context(0)
    L = ctx.L
    V, T = icosphere(2)
    mesh = td.Mesh(ctx, V, T)
    om = orc.Mesh(V, T)
    f = td.Freqs.bdf2(ctx, 16, 0.1)
    rows_h = np.arange(0, len(T), 3, dtype=np.int32)
    fidx_h = np.array([0, 3, 9, 15], dtype=np.int32)
    rows = torch.as_tensor(rows_h, device="cuda")
    fidx = torch.as_tensor(fidx_h, device="cuda")
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
        o = om.entries(getattr(orc, opname), rows_h, np.arange(ncols), f.s[fidx_h], ng=5)
        for call in range(2):
            out = torch.full((len(fidx), len(rows), ncols), float("nan"), dtype=ct, device="cuda")
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            ctx.check(L.tdbem_entries_noalloc(mesh.h, C.byref(op), f.h, C.c_void_p(rows.data_ptr()), len(rows),
                                              C.c_void_p(cols.data_ptr()), ncols, C.c_void_p(fidx.data_ptr()),
                                              len(fidx), C.c_void_p(out.data_ptr())), "tdbem_entries_noalloc")
            ctx.sync()
            free1 = torch.cuda.mem_get_info()[0]
            got = out.cpu().numpy()
            assert np.all(np.isfinite(got)), (opname, call)
            # the first call of the process may still load kernel code; from
            # the second call on, the device's free memory must not move
            if call == 1:
                assert free1 == free0, (opname, free0, free1)
            e_ref = float(np.max(np.abs(got - refn)) / np.max(np.abs(refn)))
            e_orc = _rel_err(got, o)
            assert e_ref <= tol, (opname, call, e_ref)
            assert e_orc <= tol, (opname, call, e_orc)


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
    # an infinite wave speed is refused like in tdbem_entries
    op_inf = _lib.Op(td.SLP, td.MIXED, float("inf"), 5, 0)
    f2 = td.Freqs.bdf2(ctx, 16, 0.1)
    rc = ctx.L.tdbem_entries_noalloc(mesh.h, C.byref(op_inf), f2.h, C.c_void_p(rows.data_ptr()), 1,
                                     C.c_void_p(rows.data_ptr()), 1, C.c_void_p(rows.data_ptr()), 1,
                                     C.c_void_p(out.data_ptr()))
    assert rc == -1
