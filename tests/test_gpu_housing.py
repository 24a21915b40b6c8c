"""Finned machine housing with the gCQ contour (run with -m gpu).

The batched-uneven-blocks configuration: a finned housing of about 30k
flat triangles (radius 0.1 m, length 0.3 m, 12 fins, 1 % vertex jitter),
c = 343 m/s, gCQ with 256 graded steps (ratio 1.01, T = 0.015 s, 2-stage
Radau IIA, N_Q = 256, 128 unique points), leaf 64, eta 2, eps 1e-4; and a
smaller housing for the per-frequency GMRES solve of the time-marching
configuration.  References: the FP64 oracle's dense apply on sampled rows
(3 eps relative), and the oracle's dense matrix for the solve.
"""
import time

import numpy as np
import pytest

from paper_2505_00715_gb300.inputs import graded_steps, housing, random_weights

pytestmark = pytest.mark.gpu

C_AIR = 343.0


@pytest.fixture(scope="module")
def td():
    import paper_2505_00715_gb300 as td
    return td


@pytest.fixture(scope="module")
def ctx(td):
    return td.Context(0)


def test_housing_gcq_sampled_apply(td, ctx, orc):
    import torch
    V, T = housing(30000, seed=0)
    dts = graded_steps(256, 1.01, 0.015)
    gm = td.Mesh(ctx, V, T)
    f = td.Freqs.gcq(ctx, dts, td.RADAU2, 256, rho=1.0)
    assert f.NQ == 256 and f.Nu == 128
    tree = td.Tree(gm, td.P0, td.P0, 64, 2.0)
    eps = 1e-4
    t0 = time.time()
    X = td.compress(gm, td.SLP, f, tree, eps=eps, eps_aca=1e-6, prec=td.MIXED, c=C_AIR)
    ctx.sync()
    st = X.stats()
    print("housing %d triangles: compress %.2f s, far %.0f ms, near %.0f ms, singular %.0f ms, rate %.3f, sum rank %d"
          % (len(T), time.time() - t0, st["ms_far"], st["ms_near"], st["ms_singular"],
             st["stored_complex"] / st["dense_complex"], st["sum_rank"]))
    assert st["nfar"] > 0 and st["stored_complex"] < st["dense_complex"]
    nrhs = 2
    W = random_weights(256, len(T), nrhs, seed=1)
    y = X.apply_weighted(torch.as_tensor(W, dtype=torch.complex64, device="cuda")).cpu().numpy()
    ctx.sync()
    rng = np.random.default_rng(7)
    rows = np.sort(rng.choice(len(T), 16, replace=False)).astype(np.int32)
    om = orc.Mesh(V, T)
    yd = om.dense_apply_rows(orc.SLP, f.s, rows, W, c=C_AIR, ng=5)
    err = np.linalg.norm(y[rows] - yd) / np.linalg.norm(yd)
    print("sampled apply error %.2e" % err)
    assert err < 3 * eps, err


def test_housing_gmres_per_frequency(td, ctx, orc):
    """GMRES to 1e-6 at several gCQ points on a 2k-triangle housing (no
    preconditioner; restart 200), checked with the oracle's dense matrix."""
    import torch
    V, T = housing(2000, seed=0)
    dts = graded_steps(64, 1.01, 0.015)
    gm = td.Mesh(ctx, V, T)
    f = td.Freqs.gcq(ctx, dts, td.RADAU2, 64, rho=1.0)
    tree = td.Tree(gm, td.P0, td.P0, 64, 2.0)
    eps = 1e-6
    X = td.compress(gm, td.SLP, f, tree, eps=eps, eps_aca=1e-8, prec=td.FP64, c=C_AIR)
    om = orc.Mesh(V, T)
    rng = np.random.default_rng(3)
    b = rng.standard_normal((len(T), 4)) + 1j * rng.standard_normal((len(T), 4))
    for fidx in (0, 17, 40):
        x, it, rr = X.solve(fidx, torch.as_tensor(b, device="cuda"), tol=1e-6, maxit=1500, restart=200)
        x = x.cpu().numpy()
        A = om.entries(orc.SLP, np.arange(len(T)), np.arange(len(T)), f.s[fidx:fidx + 1], c=C_AIR, ng=5)[0]
        res = np.linalg.norm(b - A @ x, axis=0) / np.linalg.norm(b, axis=0)
        print("gCQ point %d (s = %.3g%+.3gi): %d GMRES steps, oracle residual %s"
              % (fidx, f.s[fidx].real, f.s[fidx].imag, it, res))
        assert np.all(rr <= 1e-6 * 1.0000001)
        assert np.all(res <= 1e-6 + 10 * eps), res


def test_housing80k_gcq512_apply_and_gmres(td, ctx, orc):
    """The operator of the time-marching configuration: an 80k-triangle
    housing, gCQ with 512 contour points (256 unique; 512 steps graded to the
    dt_max / dt_min of 256 steps of ratio 1.01), 32 right-hand sides (16
    right-hand sides x 2 Radau stages).  Sampled apply against the oracle's
    dense FP64 apply (8 rows: the oracle evaluates 512 x 77,760 entries per
    row) and one GMRES solve to 1e-6."""
    import torch
    V, T = housing(80000, seed=0)
    dts = graded_steps(512, 1.01 ** (255.0 / 511.0), 0.015)
    gm = td.Mesh(ctx, V, T)
    f = td.Freqs.gcq(ctx, dts, td.RADAU2, 512, rho=1.0)
    assert f.NQ == 512 and f.Nu == 256
    tree = td.Tree(gm, td.P0, td.P0, 64, 2.0)
    eps = 1e-4
    X = td.compress(gm, td.SLP, f, tree, eps=eps, eps_aca=1e-6, prec=td.MIXED, c=C_AIR)
    ctx.sync()
    st = X.stats()
    print("housing %d triangles, N_Q 512: compress %.2f s (far %.0f ms), rate %.4f, sum rank %d, max rank %d"
          % (len(T), st["ms_total"] / 1e3, st["ms_far"], st["stored_complex"] / st["dense_complex"],
             st["sum_rank"], st["max_rank"]))
    g = torch.Generator(device="cuda")
    g.manual_seed(1)
    W = torch.randn((512, len(T), 32), dtype=torch.complex64, device="cuda", generator=g)
    y = X.apply_weighted(W)
    ts = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        X.apply_weighted(W, y)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    print("apply with 32 right-hand sides: %.1f ms" % min(ts))
    del W, y
    W2 = random_weights(512, len(T), 1, seed=1)
    y2 = X.apply_weighted(torch.as_tensor(W2, dtype=torch.complex64, device="cuda")).cpu().numpy()
    rows = np.sort(np.random.default_rng(7).choice(len(T), 8, replace=False)).astype(np.int32)
    yd = orc.Mesh(V, T).dense_apply_rows(orc.SLP, f.s, rows, W2, c=C_AIR, ng=5)
    err = np.linalg.norm(y2[rows] - yd) / np.linalg.norm(yd)
    print("sampled apply error %.2e" % err)
    assert err < 3 * eps, err
    rng = np.random.default_rng(3)
    b = rng.standard_normal((len(T), 1)) + 1j * rng.standard_normal((len(T), 1))
    x, it, rr = X.solve(170, torch.as_tensor(b, dtype=torch.complex64, device="cuda"), tol=1e-6, maxit=2000,
                        restart=200)
    print("GMRES at gCQ point 170: %d steps, relative residual %.3e" % (it, rr[0]))
    assert rr[0] <= 1e-6 * 1.0000001
