"""QR + SVD recompression of the ACA faces (Sec. 4, the H-matrix variant;
run with -m gpu).

One face: U V^T built from seeded random orthonormal factors with
prescribed singular values (geometric decay); the recompressed rank must be
the one the truncation rule sum_{i >= k'} s_i^2 <= eps^2 sum s_i^2 gives for
those values (+-1 in FP32 where a value sits at the threshold) and the
recompressed product must be within eps (relative Frobenius) of U V^T,
computed densely with numpy.  Whole tensor: the 5120-triangle sphere
recompressed at eps_aca stores fewer values and still applies within 3 eps
of the oracle's dense FP64 apply.
"""
import numpy as np
import pytest

from paper_2505_00715_gb300.inputs import icosphere, random_weights

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def td():
    import paper_2505_00715_gb300 as td
    return td


@pytest.fixture(scope="module")
def ctx(td):
    return td.Context(0)


def _orth(rng, n, k):
    A = rng.standard_normal((n, k)) + 1j * rng.standard_normal((n, k))
    return np.linalg.qr(A)[0]


@pytest.mark.parametrize("prec,nI,nJ,k,eps", [("MIXED", 300, 200, 40, 1e-5), ("FP64", 300, 200, 40, 1e-10),
                                              ("MIXED", 50, 90, 64, 1e-4), ("FP64", 30, 70, 45, 1e-8),
                                              ("MIXED", 20, 20, 1, 1e-4)])
def test_lowrank_recompress_matches_svd(td, ctx, prec, nI, nJ, k, eps):
    import torch
    rng = np.random.default_rng(11)
    r = min(k, nI, nJ)
    sig = np.concatenate([np.geomspace(1.0, 1e-12, r), np.zeros(k - r)])
    U = _orth(rng, nI, r) @ np.diag(sig[:r]) @ _orth(rng, k, r).T  # nI x k, rank r
    V = _orth(rng, nJ, k)  # nJ x k
    H = U @ V.T
    s = np.linalg.svd(H, compute_uv=False)
    tail = np.cumsum((s ** 2)[::-1])[::-1]  # tail[i] = sum_{j >= i} s_j^2
    k_ref = max(1, int(np.sum(tail > eps * eps * np.sum(s ** 2))))
    ct = torch.complex128 if prec == "FP64" else torch.complex64
    Ut = torch.as_tensor(np.ascontiguousarray(U.T), dtype=ct, device="cuda")
    Vt = torch.as_tensor(np.ascontiguousarray(V.T), dtype=ct, device="cuda")
    Uo, Vo = td.lowrank_recompress(ctx, Ut, Vt, eps)
    kn = Uo.shape[0]
    Hn = Uo.cpu().numpy().T.astype(np.complex128) @ Vo.cpu().numpy().astype(np.complex128)
    err = np.linalg.norm(Hn - H) / np.linalg.norm(H)
    print("%s %dx%d rank %d eps %g: rank %d (numpy %d), error %.2e" % (prec, nI, nJ, k, eps, kn, k_ref, err))
    assert abs(kn - k_ref) <= (0 if prec == "FP64" else 1)
    assert err <= 1.05 * eps + (3e-7 if prec == "MIXED" else 1e-13)


def test_tensor_recompress_sphere(td, ctx, orc):
    import torch
    V, T = icosphere(4)
    gm, om = td.Mesh(ctx, V, T), orc.Mesh(V, T)
    f = td.Freqs.bdf2(ctx, 64, 0.05)
    tree = td.Tree(gm, td.P0, td.P0, 32, 2.0)
    X = td.compress(gm, td.SLP, f, tree, eps=1e-4, eps_aca=1e-6, prec=td.MIXED)
    s0 = X.stats()
    W = torch.as_tensor(random_weights(64, len(T), 2, seed=1), dtype=torch.complex64, device="cuda")
    y0 = X.apply_weighted(W).cpu().numpy()
    X.recompress(1e-6)
    s1 = X.stats()
    y1 = X.apply_weighted(W).cpu().numpy()
    rows = np.sort(np.random.default_rng(7).choice(len(T), 12, replace=False)).astype(np.int32)
    yd = om.dense_apply_rows(orc.SLP, f.s, rows, W.cpu().numpy().astype(np.complex128), ng=5)
    err = np.linalg.norm(y1[rows] - yd) / np.linalg.norm(yd)
    print("recompression: stored %d -> %d complex values, face ranks %d -> %d; apply change %.2e; "
          "sampled apply error %.2e" % (s0["stored_complex"], s1["stored_complex"], s0["sum_face_rank"],
                                        s1["sum_face_rank"], np.linalg.norm(y1 - y0) / np.linalg.norm(y0), err))
    assert s1["stored_complex"] < s0["stored_complex"] and s1["sum_face_rank"] < s0["sum_face_rank"]
    assert np.linalg.norm(y1 - y0) <= 1e-4 * np.linalg.norm(y0)
    assert err < 3e-4
