"""Per-frequency GMRES solve on the compressed tensor, and tensor/model
persistence (run with -m gpu).

The solve is checked against a dense LU solve of the FP64 oracle matrix:
the residual of the GPU solution under the oracle matrix is bounded by the
GMRES tolerance plus the compression error, and the solution error by the
condition number times that bound.
"""
import numpy as np
import pytest

from paper_2505_00715_gb300.inputs import icosphere

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def td():
    import paper_2505_00715_gb300 as td
    return td


@pytest.fixture(scope="module")
def ctx(td):
    return td.Context(0)


@pytest.fixture(scope="module")
def sphere2(td, ctx, orc):
    V, T = icosphere(2)
    gm, om = td.Mesh(ctx, V, T), orc.Mesh(V, T)
    f = td.Freqs.bdf2(ctx, 16, 0.1)
    dense = om.entries(orc.SLP, np.arange(len(T)), np.arange(len(T)), f.s, ng=5)
    return V, T, gm, f, dense


@pytest.mark.parametrize("prec,eps,tol", [("FP64", 1e-8, 1e-10), ("MIXED", 1e-4, 1e-5)])
@pytest.mark.parametrize("fidx", [0, 5, 13])
def test_solve_matches_dense_oracle(td, ctx, sphere2, prec, eps, tol, fidx):
    import torch
    V, T, gm, f, dense = sphere2
    tree = td.Tree(gm, td.P0, td.P0, 16, 2.0)
    X = td.compress(gm, td.SLP, f, tree, eps=eps, eps_aca=eps * 1e-2, prec=getattr(td, prec))
    rng = np.random.default_rng(11 + fidx)
    b = rng.standard_normal((len(T), 3)) + 1j * rng.standard_normal((len(T), 3))
    ct = torch.complex128 if prec == "FP64" else torch.complex64
    x, it, rr = X.solve(fidx, torch.as_tensor(b, dtype=ct, device="cuda"), tol=tol, maxit=400, restart=40)
    x = x.cpu().numpy().astype(np.complex128)
    assert np.all(rr <= tol * 1.0000001) and 0 < it <= 400
    A = dense[fidx]
    res = np.linalg.norm(b - A @ x, axis=0) / np.linalg.norm(b, axis=0)
    bound = tol + 3 * eps * np.linalg.norm(A, 2) * np.linalg.norm(x, axis=0) / np.linalg.norm(b, axis=0)
    assert np.all(res <= 2 * bound), (res, bound)
    xr = np.linalg.solve(A, b)
    kappa = np.linalg.cond(A)
    err = np.linalg.norm(x - xr, axis=0) / np.linalg.norm(xr, axis=0)
    assert np.all(err <= kappa * 2 * bound), (err, kappa, bound)
    print("f%d %s: %d GMRES steps, residual vs oracle %s, error %s, cond %.1f"
          % (fidx, prec, it, res, err, kappa))


def test_solve_reports_non_convergence(td, ctx, sphere2):
    import torch
    V, T, gm, f, dense = sphere2
    tree = td.Tree(gm, td.P0, td.P0, 16, 2.0)
    X = td.compress(gm, td.SLP, f, tree, prec=td.FP64, eps=1e-8, eps_aca=1e-10)
    b = torch.ones((len(T), 1), dtype=torch.complex128, device="cuda")
    with pytest.raises(td.TdbemError):
        X.solve(3, b, tol=1e-14, maxit=2)
    x, it, rr = X.solve(3, b, tol=1e-14, maxit=2, check=False)
    assert it == 2 and rr[0] > 1e-14 and np.isfinite(x.cpu().numpy()).all()
    with pytest.raises(td.TdbemError):
        X.solve(16, b)          # frequency index out of range
    with pytest.raises(td.TdbemError):
        X.solve(0, b, tol=0.0)


def test_solve_rejects_rectangular_operator(td, ctx, sphere2):
    import torch
    V, T, gm, f, dense = sphere2
    tree = td.Tree(gm, td.P0, td.P1, 16, 2.0)
    X = td.compress(gm, td.DLP, f, tree, prec=td.MIXED)
    b = torch.ones((len(T), 1), dtype=torch.complex64, device="cuda")
    with pytest.raises(td.TdbemError):
        X.solve(0, b)


@pytest.mark.parametrize("prec", ["MIXED", "FP64"])
def test_tensor_save_load_roundtrip(td, ctx, sphere2, tmp_path, prec):
    import torch
    V, T, gm, f, dense = sphere2
    tree = td.Tree(gm, td.P0, td.P0, 16, 2.0)
    X = td.compress(gm, td.SLP, f, tree, prec=getattr(td, prec))
    path = str(tmp_path / "x.tdbem")
    X.save(path)
    Y = td.Tensor.load(ctx, path)
    assert (Y.op, Y.prec, Y.nrows, Y.ncols, Y.NQ, Y.Nu) == (X.op, X.prec, X.nrows, X.ncols, X.NQ, X.Nu)
    sx, sy = X.stats(), Y.stats()
    for k in ("nblocks", "nfar", "sum_rank", "sum_face_rank", "stored_complex"):
        assert sx[k] == sy[k]
    for a, b in zip(X.blocks(), Y.blocks()):
        assert np.array_equal(a, b)
    rng = np.random.default_rng(4)
    rows = rng.integers(0, len(T), 500)
    cols = rng.integers(0, len(T), 500)
    fid = rng.integers(0, 16, 500)
    assert torch.equal(X.entries(rows, cols, fid), Y.entries(rows, cols, fid))
    ct = torch.complex128 if prec == "FP64" else torch.complex64
    W = torch.as_tensor(rng.standard_normal((16, len(T), 2)), dtype=ct, device="cuda")
    # the apply sums block contributions with atomics: same values up to the
    # order of the additions
    ya, yb = X.apply_weighted(W), Y.apply_weighted(W)
    tol = 1e-12 if prec == "FP64" else 1e-5
    assert (torch.linalg.norm(ya - yb) <= tol * torch.linalg.norm(ya)).item()


def test_load_rejects_foreign_files(td, ctx, tmp_path):
    p = tmp_path / "junk.bin"
    p.write_bytes(b"not a tensor file at all" * 10)
    with pytest.raises(td.TdbemError):
        td.Tensor.load(ctx, str(p))
    with pytest.raises(td.TdbemError):
        td.Model.load(ctx, str(p))
    with pytest.raises(td.TdbemError):
        td.Tensor.load(ctx, str(tmp_path / "missing.bin"))


def test_model_save_load_roundtrip(td, ctx, tmp_path):
    import torch
    M = td.Model(ctx, seed=9)
    path = str(tmp_path / "m.bin")
    M.save(path)
    N = td.Model.load(ctx, path)
    assert np.array_equal(M.params(), N.params())
    x = torch.randn((100, 6), device="cuda")
    assert torch.equal(M.predict(x), N.predict(x))
