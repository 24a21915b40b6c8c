"""GPU rank-predictor MLP against the FP64 oracle, and the predictor's effect
on the compression (run with -m gpu).

Tolerances: FP32 gradients 1e-5 relative to the largest gradient entry;
BF16-weight inference compared with the oracle evaluated on the same
BF16-rounded weights (FP32 accumulation), 1e-5; Adam 1e-6.
"""
import numpy as np
import pytest

from paper_2505_00715_gb300.inputs import icosphere, random_weights

pytestmark = pytest.mark.gpu

BIN_EDGES = np.array([1, 2, 3, 4, 6, 8, 10, 12, 16, 20, 24, 32, 40, 48, 64])


def bins_of(r):
    return np.searchsorted(BIN_EDGES, np.asarray(r), side="left").astype(np.int32)


@pytest.fixture(scope="module")
def td():
    import paper_2505_00715_gb300 as td
    return td


@pytest.fixture(scope="module")
def ctx(td):
    return td.Context(0)


def _data(seed, n):
    rng = np.random.default_rng(seed)
    P = (rng.standard_normal(5648) * 0.3).astype(np.float32)
    x = rng.standard_normal((n, 6)).astype(np.float32)
    lab = rng.integers(0, 16, n).astype(np.int32)
    return P, x, lab


def test_rank_bins(td):
    for r in (1, 2, 5, 6, 7, 16, 17, 64, 65, 500):
        assert td.rank_bin(r) == bins_of([r])[0]


def test_grad_matches_oracle(td, ctx, orc):
    import torch
    P, x, lab = _data(2, 300)
    M = td.Model(ctx)
    M.set_params(P)
    loss, g = M.loss_grad(torch.as_tensor(x, device="cuda"), torch.as_tensor(lab, device="cuda"))
    lo, go = orc.mlp_loss_grad(P.astype(np.float64), x.astype(np.float64), lab)
    assert abs(loss.item() - lo) <= 1e-5 * abs(lo)
    assert np.max(np.abs(g.cpu().numpy() - go)) <= 1e-5 * np.max(np.abs(go))


def test_bf16_inference_matches_oracle(td, ctx, orc):
    import torch
    P, x, _ = _data(3, 257)
    M = td.Model(ctx)
    M.set_params(P)
    bins, lg = M.predict(torch.as_tensor(x, device="cuda"), logits=True)
    Pb = torch.as_tensor(P).to(torch.bfloat16).to(torch.float64).numpy()
    ref = orc.mlp_forward(Pb, x.astype(np.float64))
    lg = lg.cpu().numpy()
    assert np.max(np.abs(lg - ref)) <= 1e-5 * np.max(np.abs(ref))
    top2 = np.sort(ref, axis=1)[:, -2:]
    clear = (top2[:, 1] - top2[:, 0]) > 1e-4 * np.max(np.abs(ref))
    assert np.array_equal(bins.cpu().numpy()[clear], np.argmax(ref, axis=1)[clear])


def test_adam_matches_oracle(td, ctx, orc):
    import torch
    P, _, _ = _data(4, 1)
    rng = np.random.default_rng(5)
    M = td.Model(ctx)
    M.set_params(P)
    p64 = P.astype(np.float64)
    m = np.zeros_like(p64)
    v = np.zeros_like(p64)
    for t in (1, 2, 3):
        g = (rng.standard_normal(5648) * 0.01).astype(np.float32)
        M.adam_step(torch.as_tensor(g, device="cuda"), 1e-3, t)
        orc.adam_step(p64, g.astype(np.float64), m, v, 1e-3, t)
    assert np.max(np.abs(M.params() - p64)) <= 1e-6


@pytest.fixture(scope="module")
def trained(td, ctx):
    """Harvest (far block, frequency, face rank) samples from the plain method
    on 320- and 1280-triangle spheres (SLP and DLP), train on the GPU."""
    import torch
    xs, ys = [], []
    for lev, leaf in ((2, 16), (3, 32)):
        V, T = icosphere(lev)
        m = td.Mesh(ctx, V, T)
        f = td.Freqs.bdf2(ctx, 64, 0.05)
        for op, cb in ((td.SLP, td.P0), (td.DLP, td.P1)):
            tr = td.Tree(m, td.P0, cb, leaf, 2.0)
            x, r = td.harvest(m, op, f, tr, eps_aca=1e-6)
            xs.append(x)
            ys.append(torch.as_tensor(bins_of(r.cpu().numpy()), device="cuda"))
    x = torch.cat(xs)
    y = torch.cat(ys)
    M = td.Model(ctx, seed=2)
    l0 = M.loss_grad(x, y)[0].item()
    loss = M.train(x, y, epochs=30, batch=2048, lr=3e-3, seed=3)
    return M, x, y, l0, loss


def test_training_learns_rank_bins(td, ctx, trained):
    M, x, y, l0, loss = trained
    assert loss < 0.6 * l0, (l0, loss)
    pred = M.predict(x).cpu().numpy()
    yy = y.cpu().numpy()
    acc = np.mean(pred == yy)
    major = np.max(np.bincount(yy, minlength=16)) / len(yy)
    within1 = np.mean(np.abs(pred - yy) <= 1)
    print("samples %d  loss %.3f -> %.3f  accuracy %.3f (majority %.3f, within one bin %.3f)"
          % (len(yy), l0, loss, acc, major, within1))
    assert acc > major + 0.05 and within1 > 0.8


def test_predictor_keeps_the_adaptive_result(td, ctx, orc, trained):
    """The prediction only orders blocks and defers the first ACA norm checks;
    the adaptive criterion still decides: same ranks, same apply."""
    import torch
    M = trained[0]
    V, T = icosphere(4)
    gm = td.Mesh(ctx, V, T)
    f = td.Freqs.bdf2(ctx, 64, 0.05)
    tree = td.Tree(gm, td.P0, td.P0, 32, 2.0)
    X0 = td.compress(gm, td.SLP, f, tree, prec=td.MIXED)
    X1 = td.compress(gm, td.SLP, f, tree, prec=td.MIXED, model=M)
    r0, k0, _ = X0.blocks()
    r1, k1, _ = X1.blocks()
    assert np.mean(r0 == r1) > 0.99
    assert abs(int(k0.sum()) - int(k1.sum())) <= 0.01 * k0.sum()
    W = random_weights(64, len(T), 2, seed=1)
    Wd = torch.as_tensor(W, dtype=torch.complex64, device="cuda")
    y0 = X0.apply_weighted(Wd).cpu().numpy()
    y1 = X1.apply_weighted(Wd).cpu().numpy()
    assert np.linalg.norm(y1 - y0) <= 1e-4 * np.linalg.norm(y0)
    s0, s1 = X0.stats(), X1.stats()
    print("far phase without / with predictor: %.1f / %.1f ms; first face pool %.3e / %.3e values (stored %.3e, "
          "pool growths %d)" % (s0["ms_far"], s1["ms_far"], s0["pool_first"], s1["pool_first"], s1["stored_complex"],
                                s1["pool_growths"]))


def test_predictor_gain_fewer_aca_tests(td, ctx, trained):
    """What the trained network gains over the method without it: on faces
    whose ACA norm comes from the factor Grams (above 1600 entries), the
    steps below the predicted face rank run without their synchronised
    stopping test and are tested in one batched round, so a compression
    takes fewer test rounds (block barriers); the ranks stay those of the
    adaptive criterion (previous test)."""
    M = trained[0]
    V, T = icosphere(4)
    gm = td.Mesh(ctx, V, T)
    f = td.Freqs.bdf2(ctx, 64, 0.05)
    tree = td.Tree(gm, td.P0, td.P0, 32, 2.0)
    s0 = td.compress(gm, td.SLP, f, tree, prec=td.MIXED).stats()
    s1 = td.compress(gm, td.SLP, f, tree, prec=td.MIXED, model=M).stats()
    print("ACA stopping-test rounds without / with predictor: %d / %d (%.2f); far %.1f / %.1f ms"
          % (s0["aca_tests"], s1["aca_tests"], s1["aca_tests"] / max(1, s0["aca_tests"]), s0["ms_far"], s1["ms_far"]))
    assert s0["aca_tests"] > 0
    assert s1["aca_tests"] < s0["aca_tests"]


def test_predictor_on_housing60k(td, ctx, orc):
    """The learned-predictor configuration: the network is trained on about
    2M (block, frequency, rank-bin) samples harvested from the sphere
    configurations (icospheres with 1280 / 5120 / 20480 triangles, single and
    double layer, two BDF2 frequency sets) and evaluated on the 60k-triangle
    finned housing with the 256-point gCQ contour (c = 343 m/s).  Its bin
    accuracy there is reported; what it gains is the size of the first face
    pool of the compression (presized from the predicted face ranks instead
    of a size-based bound), while the adaptive criterion keeps the result:
    the same ranks and an apply within 3 eps of the oracle's dense apply."""
    import sys
    import os
    import torch
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    from paper_2505_00715_gb300.inputs import graded_steps, housing
    x, y = bench.harvest_training_set(td, ctx, "cuda")
    assert len(y) > 1_500_000
    M = td.Model(ctx, seed=2)
    loss = M.train(x, y, epochs=8, batch=4096, lr=3e-3, seed=3)
    cfg = dict(bench.WORKLOADS["housing60k_slp_gcq256"])
    V, T = housing(60000, seed=0)
    gm = td.Mesh(ctx, V, T)
    f = td.Freqs.gcq(ctx, graded_steps(256, 1.01, 0.015), td.RADAU2, 256, rho=1.0)
    tree = td.Tree(gm, td.P0, td.P0, 64, 2.0)
    acc = bench.predictor_accuracy(td, M, gm, td.SLP, f, tree, cfg)
    kw = dict(eps=1e-4, eps_aca=1e-6, prec=td.MIXED, c=343.0, ng=5)
    X0 = td.compress(gm, td.SLP, f, tree, **kw)
    s0 = X0.stats()
    r0 = X0.blocks()[0]
    del X0
    X1 = td.compress(gm, td.SLP, f, tree, model=M, **kw)
    s1 = X1.stats()
    r1 = X1.blocks()[0]
    print("housing60k: %d training samples, loss %.3f; bin accuracy %.3f (within one bin %.3f, majority %.3f); "
          "first face pool without / with predictor %.3e / %.3e values (stored %.3e); time to tensor %.2f / %.2f s"
          % (len(y), loss, acc["bin_accuracy"], acc["within_one_bin"], acc["majority_bin_share"], s0["pool_first"],
             s1["pool_first"], s1["stored_complex"], s0["ms_total"] / 1e3, s1["ms_total"] / 1e3))
    assert s1["pool_first"] < s0["pool_first"]
    assert s1["pool_first"] >= s1["stored_complex"] or s1["pool_growths"] > 0
    assert np.mean(r0 == r1) > 0.99
    W = random_weights(256, len(T), 2, seed=1)
    yg = X1.apply_weighted(torch.as_tensor(W, dtype=torch.complex64, device="cuda")).cpu().numpy()
    rows = np.sort(np.random.default_rng(5).choice(len(T), 4, replace=False)).astype(np.int32)
    yd = orc.Mesh(V, T).dense_apply_rows(orc.SLP, f.s, rows, W, c=343.0, ng=5)
    err = np.linalg.norm(yg[rows] - yd) / np.linalg.norm(yd)
    print("housing60k sampled apply error with the predictor %.2e" % err)
    assert err < 3e-4
