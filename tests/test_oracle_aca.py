"""Pins of the oracle's ACA, 3D-ACA (Algorithm 1, eq. norm) and apply (eq. product).

Separable tensors of known rank are recovered exactly; on a BEM operator the
compressed tensor is compared with the dense oracle tensor, and the apply
with the dense apply.
"""
import numpy as np
import pytest

from paper_2505_00715_gb300.inputs import icosphere, random_weights


def _crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("k", [1, 3, 7])
def test_matrix_aca_recovers_rank(orc, k):
    rng = np.random.default_rng(k)
    A = _crandn(rng, 40, k) @ _crandn(rng, k, 33)
    U, V = orc.aca_dense(A, 1e-12)
    assert U.shape[1] <= k + 1
    assert np.linalg.norm(A - U @ V.T) <= 1e-12 * np.linalg.norm(A)


@pytest.mark.parametrize("r", [1, 2, 5, 8])
def test_aca3d_dense_faces_recovers_separable_rank(orc, r):
    """T = sum_q A_q (x) c_q with A_q random dense faces: Algorithm 1 with the
    criterion of eq. norm returns exactly r terms and reproduces T."""
    rng = np.random.default_rng(10 + r)
    nI, nJ, nK = 12, 9, 20
    A = _crandn(rng, r, nI, nJ)
    cvec = _crandn(rng, r, nK)
    T = np.einsum("qij,qk->kij", A, cvec)
    kp, H, f, _ = orc.aca3d_dense(T, 1e-6)
    assert len(kp) == r
    approx = np.einsum("dij,dk->kij", H, f)
    assert np.linalg.norm(T - approx) <= 1e-12 * np.linalg.norm(T)
    # the fibre is 1 at its own frequency (f_l[k_l] = 1 by construction)
    assert np.allclose(f[np.arange(r), kp], 1.0, atol=1e-12)


@pytest.mark.parametrize("r", [1, 3, 6])
def test_aca3d_aca_faces_recovers_separable_rank(orc, r):
    """Faces of rank <= 2r (sums of outer products): the far-field form with
    ACA faces is also exact."""
    rng = np.random.default_rng(20 + r)
    nI, nJ, nK = 30, 25, 16
    a, b = _crandn(rng, r, 2, nI), _crandn(rng, r, 2, nJ)
    faces = np.einsum("qti,qtj->qij", a, b)
    cvec = _crandn(rng, r, nK)
    T = np.einsum("qij,qk->kij", faces, cvec)
    kp, H, f, fr = orc.aca3d_dense(T, 1e-6, eps_aca=1e-13)
    assert len(kp) == r
    assert np.all(fr <= 2 * r + 1)
    approx = np.einsum("dij,dk->kij", H, f)
    assert np.linalg.norm(T - approx) <= 1e-11 * np.linalg.norm(T)


def test_aca3d_stops_on_eps(orc):
    """Exponentially decaying spectrum: the number of terms grows as eps shrinks
    and the error stays of order eps (the criterion is heuristic)."""
    rng = np.random.default_rng(3)
    nI, nJ, nK, R = 15, 15, 24, 12
    A = _crandn(rng, R, nI, nJ)
    cvec = _crandn(rng, R, nK) * (10.0 ** -np.arange(R))[:, None]
    T = np.einsum("qij,qk->kij", A, cvec)
    ranks = []
    for eps in (1e-2, 1e-5, 1e-8):
        kp, H, f, _ = orc.aca3d_dense(T, eps)
        err = np.linalg.norm(T - np.einsum("dij,dk->kij", H, f)) / np.linalg.norm(T)
        ranks.append(len(kp))
        assert err < 50 * eps
    assert ranks[0] < ranks[1] < ranks[2]


@pytest.fixture(scope="module")
def bem320(orc):
    V, T = icosphere(2)
    m = orc.Mesh(V, T)
    s = orc.freqs_bdf2(16, 0.1)[:9]
    return V, T, m, s


@pytest.mark.parametrize("op", ["slp", "dlp"])
def test_compress_bem_vs_dense(orc, bem320, op):
    """Algorithm 1 per block of the block cluster tree (leaf 16, eta 2; leaf 32
    leaves no admissible block at this size) on the 320-triangle sphere: rebuilt tensor within a few eps of the dense tensor
    (Frobenius), apply (eq. product) within 3 eps of the dense apply."""
    V, T, m, s = bem320
    opc = orc.SLP if op == "slp" else orc.DLP
    cols = 0 if op == "slp" else 1
    tr = orc.Tree(m, 0, cols, 16, 2.0)
    eps, eps_aca = 1e-4, 1e-6
    X = orc.Tensor(m, opc, s, tr, eps, eps_aca, ng=5)
    nr, nc = m.ndof(0), m.ndof(cols)
    dense = m.entries(opc, np.arange(nr), np.arange(nc), s, ng=5)
    rebuilt = np.zeros_like(dense)
    for f in range(len(s)):
        for i in range(0, nr, 4):
            for j in range(nc):
                rebuilt[f, i, j] = X.entry(i, j, f)
    sub = dense[:, ::4, :]
    err = np.linalg.norm(sub - rebuilt[:, ::4, :]) / np.linalg.norm(sub)
    assert err < 3 * eps, err
    W = random_weights(len(s), nc, 3, seed=1)
    y = X.apply(W)
    yd = np.einsum("fij,fjq->iq", dense, W)
    assert np.linalg.norm(y - yd) / np.linalg.norm(yd) < 3 * eps
    assert X.stats["nfar"] > 0 and X.stats["stored"] < X.stats["dense"]
    r, _ = X.block_ranks()
    assert r.max() <= len(s) and r.min() >= 1


def test_dense_apply_rows_matches_entries(orc, bem320):
    V, T, m, s = bem320
    rows = np.array([0, 17, 301], dtype=np.int32)
    W = random_weights(len(s), len(T), 2, seed=4)
    y = m.dense_apply_rows(orc.SLP, s, rows, W, ng=5)
    A = m.entries(orc.SLP, rows, np.arange(len(T)), s, ng=5)
    assert np.allclose(y, np.einsum("fij,fjq->iq", A, W), rtol=1e-13, atol=0)
