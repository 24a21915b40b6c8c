"""GPU parity of the CUDA library against the FP64 oracle (run with -m gpu).

Tolerances: tree and admissibility bit-exact; frequencies 1e-13 relative;
entries 1e-12 (FP64 form) and 1e-5 (mixed form), each relative to the entry
with a floor of 1e-6 times the largest entry of the same frequency slice
(FP32 underflows exp(-Re(s) r) for the largest Re(s) r); compressed-tensor
apply within 3 eps (relative Frobenius) of the dense FP64 apply.
"""
import numpy as np
import pytest

from paper_2505_00715_gb300.inputs import graded_steps, housing, icosphere, random_weights

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def td():
    import paper_2505_00715_gb300 as td
    return td


@pytest.fixture(scope="module")
def ctx(td):
    return td.Context(0)


def _entry_err(g, o):
    """max over entries of |g - o| / max(|o|, 1e-6 max|o| of the slice)."""
    g = np.asarray(g)
    o = np.asarray(o)
    scale = np.max(np.abs(o).reshape(o.shape[0], -1), axis=1).reshape((-1,) + (1,) * (o.ndim - 1))
    den = np.maximum(np.abs(o), 1e-6 * scale)
    return float(np.max(np.abs(g - o) / den))


# ---------------------------------------------------------------- tree
@pytest.mark.parametrize("mesh,cols,leaf,eta", [("sphere3", 0, 32, 2.0), ("sphere3", 1, 32, 2.0),
                                                 ("housing", 0, 64, 2.0), ("housing", 1, 64, 2.0),
                                                 ("sphere4", 0, 32, 2.0)])
def test_tree_bit_exact(td, ctx, orc, mesh, cols, leaf, eta):
    V, T = {"sphere3": lambda: icosphere(3), "sphere4": lambda: icosphere(4),
            "housing": lambda: housing(3000, seed=0)}[mesh]()
    g = td.Tree(td.Mesh(ctx, V, T), td.P0, cols, leaf, eta)
    o = orc.Tree(orc.Mesh(V, T), 0, cols, leaf, eta)
    assert np.array_equal(g.perm_rows, o.perm_rows)
    assert np.array_equal(g.perm_cols, o.perm_cols)
    assert np.array_equal(g.blocks, o.blocks)


# ---------------------------------------------------------------- frequencies
@pytest.mark.parametrize("N,dt", [(16, 0.1), (64, 0.05)])
def test_freqs_bdf2(td, ctx, orc, N, dt):
    f = td.Freqs.bdf2(ctx, N, dt)
    s = orc.freqs_bdf2(N, dt)
    assert np.max(np.abs(f.s - s)) <= 1e-13 * np.max(np.abs(s))
    assert f.Nu == N // 2 + 1
    for k in range(N):
        u = f.unique_map[k]
        rep = f.unique[abs(u) - 1]
        assert np.allclose(f.s[k], f.s[rep] if u > 0 else np.conj(f.s[rep]), rtol=1e-13)


@pytest.mark.parametrize("rk,NQ,rho", [(1, 256, 1.0), (1, 256, 0.0), (0, 64, 0.0), (1, 128, 2.5)])
def test_freqs_gcq(td, ctx, orc, rk, NQ, rho):
    dts = graded_steps(256, 1.01, 0.015)
    f = td.Freqs.gcq(ctx, dts, rk, NQ, rho=rho)
    s, w, _ = orc.freqs_gcq(dts.min(), dts.max(), rk, NQ, len(dts), rho=rho)
    assert np.array_equal(f.steps(), dts)
    assert np.max(np.abs(f.s - s)) <= 1e-12 * np.max(np.abs(s))
    assert np.max(np.abs(f.w - w)) <= 1e-12 * np.max(np.abs(w))
    assert f.Nu == NQ // 2


# ---------------------------------------------------------------- entries
@pytest.fixture(scope="module")
def sphere2(td, ctx, orc):
    V, T = icosphere(2)
    return V, T, td.Mesh(ctx, V, T), orc.Mesh(V, T)


@pytest.mark.parametrize("prec,tol", [("FP64", 1e-12), ("MIXED", 1e-5)])
@pytest.mark.parametrize("op", ["SLP", "DLP", "ADLP"])
def test_entries_vs_oracle(td, ctx, orc, sphere2, prec, tol, op):
    V, T, gm, om = sphere2
    f = td.Freqs.bdf2(ctx, 16, 0.1)
    fidx = f.unique
    rows = np.arange(len(T))
    cols = np.arange(len(V) if op == "DLP" else len(T))
    opc = getattr(td, op)
    g = td.entries(gm, opc, f, rows, cols, fidx, prec=getattr(td, prec), ng=5).cpu().numpy()
    o = om.entries(getattr(orc, op), rows, cols, f.s[fidx], ng=5)
    err = _entry_err(g, o)
    assert err <= tol, err


def test_entries_edge_cases(td, ctx, orc, sphere2):
    V, T, gm, om = sphere2
    f = td.Freqs.bdf2(ctx, 16, 0.1)
    out = td.entries(gm, td.SLP, f, [], [0, 1], [0])
    assert out.numel() == 0
    # a single touching pair at a conjugate frequency (k = 15 is conj of k = 1)
    g = td.entries(gm, td.SLP, f, [0], [0], [15], prec=td.FP64).cpu().numpy()[0, 0, 0]
    o = om.entries(orc.SLP, [0], [0], [f.s[15]], ng=5)[0, 0, 0]
    assert abs(g - o) <= 1e-12 * abs(o)
    with pytest.raises(td.TdbemError):
        td.entries(gm, td.SLP, f, [0], [0], [0], ng=0)


def test_mesh_errors(td, ctx):
    V, T = icosphere(1)
    bad = T.copy()
    bad[0, 0] = len(V)
    with pytest.raises(td.TdbemError):
        td.Mesh(ctx, V, bad)
    Vn = V.copy()
    Vn[3, 1] = np.nan
    with pytest.raises(td.TdbemError):
        td.Mesh(ctx, Vn, T)
    deg = T.copy()
    deg[1] = [deg[1, 0], deg[1, 0], deg[1, 2]]
    with pytest.raises(td.TdbemError):
        td.Mesh(ctx, V, deg)


# ---------------------------------------------------------------- compression + apply
def _dense_all(om, orc, op, f, nrows, ncols):
    return om.entries(getattr(orc, op), np.arange(nrows), np.arange(ncols), f.s, ng=5)


@pytest.mark.parametrize("dense_faces", [True, False])
@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
@pytest.mark.parametrize("op", ["SLP", "DLP", "ADLP"])
def test_compress_small_vs_dense(td, ctx, orc, sphere2, prec, op, dense_faces):
    """320-triangle sphere, leaf 16 (leaf 32 has no admissible block here),
    eta 2, BDF2 N = 16: rebuilt tensor and apply vs the dense oracle, with the
    far blocks' dense working faces and with the low-rank evaluation."""
    import torch
    V, T, gm, om = sphere2
    f = td.Freqs.bdf2(ctx, 16, 0.1)
    cols_b = td.P1 if op == "DLP" else td.P0
    tree = td.Tree(gm, td.P0, cols_b, 16, 2.0)
    eps = 1e-4
    X = td.compress(gm, getattr(td, op), f, tree, eps=eps, eps_aca=1e-6, prec=getattr(td, prec),
                    dense_faces=dense_faces)
    st = X.stats()
    assert st["nfar"] > 0 and st["nnear"] > 0
    nr, nc = len(T), (len(V) if op == "DLP" else len(T))
    dense = _dense_all(om, orc, op, f, nr, nc)  # all 16 frequencies
    rr, cc = np.meshgrid(np.arange(nr), np.arange(nc), indexing="ij")
    reb = np.stack([X.entries(rr.ravel(), cc.ravel(), np.full(rr.size, k)).cpu().numpy().reshape(nr, nc)
                    for k in range(16)])
    err_t = np.linalg.norm(reb - dense) / np.linalg.norm(dense)
    assert err_t < 3 * eps, err_t
    ct = torch.complex128 if prec == "FP64" else torch.complex64
    W = random_weights(16, nc, 4, seed=1)
    y = X.apply_weighted(torch.as_tensor(W, dtype=ct, device="cuda")).cpu().numpy()
    yd = np.einsum("fij,fjq->iq", dense, W)
    err_a = np.linalg.norm(y - yd) / np.linalg.norm(yd)
    assert err_a < 3 * eps, err_a
    x = W[5]
    y5 = X.apply_freq(13, torch.as_tensor(x, dtype=ct, device="cuda")).cpu().numpy()
    assert np.linalg.norm(y5 - dense[13] @ x) / np.linalg.norm(dense[13] @ x) < 3 * eps
    # host-buffer apply returns the same result
    yh = np.zeros_like(y)
    X.apply_weighted_host(W.astype(np.complex128 if prec == "FP64" else np.complex64), yh)
    assert np.linalg.norm(yh - y) <= 1e-5 * np.linalg.norm(y)


@pytest.mark.parametrize("op,prec", [("SLP", "MIXED"), ("SLP", "FP64"), ("DLP", "MIXED"), ("ADLP", "MIXED")])
def test_sphere5120_sampled_apply(td, ctx, orc, op, prec):
    """5120-triangle sphere, SLP (P0 x P0), DLP (P0 x P1) and K' (P0 x P0), BDF2 N = 64,
    dt = 0.05, leaf 32, eta 2, eps 1e-4: apply on sampled rows vs the dense
    FP64 oracle apply."""
    import torch
    V, T = icosphere(4)
    gm, om = td.Mesh(ctx, V, T), orc.Mesh(V, T)
    f = td.Freqs.bdf2(ctx, 64, 0.05)
    cols_b = td.P1 if op == "DLP" else td.P0
    ncols = len(V) if op == "DLP" else len(T)
    tree = td.Tree(gm, td.P0, cols_b, 32, 2.0)
    eps = 1e-4
    X = td.compress(gm, getattr(td, op), f, tree, eps=eps, eps_aca=1e-6, prec=getattr(td, prec))
    st = X.stats()
    print("sphere5120 %s %s stats: %s" % (op, prec, st))
    assert st["stored_complex"] < 0.5 * st["dense_complex"]
    nrhs = 2
    W = random_weights(64, ncols, nrhs, seed=1)
    ct = torch.complex128 if prec == "FP64" else torch.complex64
    y = X.apply_weighted(torch.as_tensor(W, dtype=ct, device="cuda")).cpu().numpy()
    rng = np.random.default_rng(7)
    rows = np.sort(rng.choice(len(T), 12, replace=False)).astype(np.int32)
    yd = om.dense_apply_rows(getattr(orc, op), f.s, rows, W, ng=5)
    err = np.linalg.norm(y[rows] - yd) / np.linalg.norm(yd)
    print("sphere5120 %s %s sampled apply error %.2e" % (op, prec, err))
    assert err < 3 * eps, err


def test_autotune_keeps_results(td, ctx, orc, sphere2):
    """The autotuner changes launch parameters only (far launch shape,
    frequencies per pass of the entry kernels); the compressed tensor applies
    identically (to FP32 rounding: the entry kernels' summation order is the
    same per frequency)."""
    import torch
    V, T, gm, om = sphere2
    f = td.Freqs.bdf2(ctx, 16, 0.1)
    tree = td.Tree(gm, td.P0, td.P0, 16, 2.0)
    X0 = td.compress(gm, td.SLP, f, tree, prec=td.MIXED)
    nt, cps, sfc, nfc = td.autotune(gm, td.SLP, f, tree, prec=td.MIXED)
    assert nt in (64, 128, 256) and cps >= 1 and sfc in (4, 8, 16) and nfc in (4, 8, 16)
    X1 = td.compress(gm, td.SLP, f, tree, prec=td.MIXED)
    W = torch.as_tensor(random_weights(16, len(T), 2, seed=3), dtype=torch.complex64, device="cuda")
    y0 = X0.apply_weighted(W).cpu().numpy()
    y1 = X1.apply_weighted(W).cpu().numpy()
    assert np.linalg.norm(y1 - y0) <= 1e-5 * np.linalg.norm(y0)


# ---------------------------------------------------------------- balanced partition
@pytest.mark.parametrize("op", ["SLP", "DLP"])
def test_balanced_partition_refines_tree(td, ctx, orc, op):
    """The compression partition refines the tree's partition (every block
    lies inside one tree block of the same kind, the blocks tile the matrix
    once), splits the largest far blocks, and both partitions compress to
    3 eps of the dense FP64 apply."""
    import torch
    V, T = icosphere(3)
    gm, om = td.Mesh(ctx, V, T), orc.Mesh(V, T)
    f = td.Freqs.bdf2(ctx, 64, 0.05)
    cols = td.P0 if op == "SLP" else td.P1
    tree = td.Tree(gm, td.P0, cols, 32, 2.0)
    eps = 1e-4
    Xb = td.compress(gm, getattr(td, op), f, tree, eps=eps, eps_aca=1e-6, prec=td.MIXED)
    Xt = td.compress(gm, getattr(td, op), f, tree, eps=eps, eps_aca=1e-6, prec=td.MIXED, balance=False)
    tb, pb, pt = np.asarray(tree.blocks), Xb.partition(), Xt.partition()
    assert np.array_equal(pt, tb)
    assert len(pb) > len(tb) and Xb.stats()["nblocks"] == len(pb)
    nr, nc = Xb.nrows, Xb.ncols
    label = np.full((nr, nc), -1, dtype=np.int64)
    for q, (i0, i1, j0, j1, far) in enumerate(tb):
        label[i0:i1, j0:j1] = q
    cover = np.zeros((nr, nc), dtype=np.int32)
    for i0, i1, j0, j1, far in pb:
        cover[i0:i1, j0:j1] += 1
        lab = np.unique(label[i0:i1, j0:j1])
        assert len(lab) == 1 and tb[lab[0], 4] == far
    assert np.all(cover == 1)
    e_t = (tb[:, 1] - tb[:, 0]) * (tb[:, 3] - tb[:, 2])
    e_b = (pb[:, 1] - pb[:, 0]) * (pb[:, 3] - pb[:, 2])
    assert e_b[pb[:, 4] == 1].max() < e_t[tb[:, 4] == 1].max()
    nrhs = 2
    W = random_weights(64, nc, nrhs, seed=5)
    Wt = torch.as_tensor(W, dtype=torch.complex64, device="cuda")
    rows = np.sort(np.random.default_rng(2).choice(nr, 24, replace=False)).astype(np.int32)
    orc_op = getattr(orc, op)
    yd = om.dense_apply_rows(orc_op, f.s, rows, W, ng=5)
    for X in (Xb, Xt):
        y = X.apply_weighted(Wt).cpu().numpy()
        err = np.linalg.norm(y[rows] - yd) / np.linalg.norm(yd)
        print("%s %s partition: %d blocks, sampled apply error %.2e" % (op, "balanced" if X is Xb else "tree",
                                                                       X.stats()["nblocks"], err))
        assert err < 3 * eps, err


def test_near_batches_give_the_same_tensor(td, ctx):
    """Forming and compressing the near-field tensor in several batches of
    near blocks (a small batch buffer) gives the same blocks and entries as
    one batch."""
    import torch
    V, T = icosphere(3)
    gm = td.Mesh(ctx, V, T)
    f = td.Freqs.bdf2(ctx, 64, 0.05)
    tree = td.Tree(gm, td.P0, td.P0, 32, 2.0)
    X1 = td.compress(gm, td.SLP, f, tree, prec=td.MIXED)
    ctx.set_near_batch(8 << 20)
    try:
        X2 = td.compress(gm, td.SLP, f, tree, prec=td.MIXED)
    finally:
        ctx.set_near_batch(16 << 30)
    with pytest.raises(td.TdbemError):
        ctx.set_near_batch(0)
    for a, b in zip(X1.blocks(), X2.blocks()):
        assert np.array_equal(a, b)
    s1, s2 = X1.stats(), X2.stats()
    assert s1["stored_complex"] == s2["stored_complex"] and s1["entries_regular"] == s2["entries_regular"]
    rng = np.random.default_rng(9)
    rows, cols, fid = rng.integers(0, len(T), 4000), rng.integers(0, len(T), 4000), rng.integers(0, 64, 4000)
    assert torch.equal(X1.entries(rows, cols, fid), X2.entries(rows, cols, fid))


def test_face_pool_growth_redoes_far_blocks(td, ctx):
    """A first face pool far too small: the pool grows (keeping the stored
    faces), the far blocks it stopped are redone, and the tensor equals the
    one compressed with a large enough pool."""
    import torch
    V, T = icosphere(3)
    gm = td.Mesh(ctx, V, T)
    f = td.Freqs.bdf2(ctx, 64, 0.05)
    tree = td.Tree(gm, td.P0, td.P0, 32, 2.0)
    X1 = td.compress(gm, td.SLP, f, tree, prec=td.MIXED)
    assert X1.stats()["pool_growths"] == 0
    ctx.set_pool_scale(1e-3)
    try:
        X2 = td.compress(gm, td.SLP, f, tree, prec=td.MIXED)
    finally:
        ctx.set_pool_scale(1.0)
    with pytest.raises(td.TdbemError):
        ctx.set_pool_scale(0.0)
    s1, s2 = X1.stats(), X2.stats()
    assert s2["pool_growths"] >= 1
    for a, b in zip(X1.blocks(), X2.blocks()):
        assert np.array_equal(a, b)
    assert s1["stored_complex"] == s2["stored_complex"]
    rng = np.random.default_rng(10)
    rows, cols, fid = rng.integers(0, len(T), 4000), rng.integers(0, len(T), 4000), rng.integers(0, 64, 4000)
    assert torch.equal(X1.entries(rows, cols, fid), X2.entries(rows, cols, fid))
