"""Pins of the oracle's cluster tree and block cluster tree (Sec. 4, eq. admissible).

Checked independently of the oracle: a bijective permutation, balanced sons,
leaf sizes, the split along the principal axis computed here with
numpy.linalg.eigh, cluster boxes recomputed from the supports, an exact tiling
of the matrix by the blocks, and the admissibility condition for every block.
"""
import numpy as np
import pytest

from paper_2505_00715_gb300.inputs import housing, icosphere


def _supports(V, T, basis):
    if basis == 0:
        return [T[e] for e in range(len(T))], V[T].sum(axis=1) / 3.0
    sup = [[] for _ in range(len(V))]
    for t in T:
        for v in t:
            sup[v].extend(t)
    return [np.array(s) for s in sup], V.copy()


def _box(V, sups, idx):
    pts = V[np.concatenate([sups[i] for i in idx])]
    return pts.min(axis=0), pts.max(axis=0)


@pytest.mark.parametrize("mesh,cols,leaf,eta", [
    ("sphere3", 0, 32, 2.0), ("sphere3", 1, 32, 2.0), ("housing", 0, 64, 2.0), ("sphere3", 0, 20, 0.8)])
def test_tree_invariants(orc, mesh, cols, leaf, eta):
    V, T = icosphere(3) if mesh == "sphere3" else housing(3000, seed=0)
    m = orc.Mesh(V, T)
    tr = orc.Tree(m, 0, cols, leaf, eta)
    for side, basis, perm in ((0, 0, tr.perm_rows), (1, cols, tr.perm_cols)):
        n = m.ndof(basis)
        assert np.array_equal(np.sort(perm), np.arange(n))
        nodes, box = tr.clusters(side)
        sups, pts = _supports(V, T, basis)
        for k, (b, e, s0, s1) in enumerate(nodes):
            lo, hi = _box(V, sups, perm[b:e])
            assert np.array_equal(lo, box[k, :3]) and np.array_equal(hi, box[k, 3:])
            if s0 < 0:
                assert e - b <= leaf
                continue
            assert e - b > leaf
            nb, ne = nodes[s0][:2]
            assert nb == b and ne == b + (e - b) // 2 and nodes[s1][0] == ne and nodes[s1][1] == e
            # split along the principal axis (numpy eigh), projection order respected
            P = pts[perm[b:e]]
            d = P - P.mean(axis=0)
            w, U = np.linalg.eigh(d.T @ d)
            if w[-1] - w[-2] < 1e-6 * w[-1]:
                continue  # degenerate principal axis (e.g. a whole sphere): any axis in the eigenspace
            ax = U[:, -1]
            pr = d @ ax
            left, right = pr[: ne - b], pr[ne - b:]
            gap = np.sign(ax[np.argmax(np.abs(ax))])
            if gap < 0:
                left, right = -left, -right
            tol = 1e-9 * (np.max(np.abs(pr)) + 1e-300)
            assert np.max(left) <= np.min(right) + tol
    # blocks tile rows x cols exactly once and satisfy the admissibility rule
    nr, nc = m.ndof(0), m.ndof(cols)
    cover = np.zeros((nr, nc), dtype=np.int32)
    sr, _ = _supports(V, T, 0)
    sc, _ = _supports(V, T, cols)
    nfar = 0
    nodes_r, _ = tr.clusters(0)
    nodes_c, _ = tr.clusters(1)
    leaves_r = {(b, e) for b, e, s0, _ in nodes_r if s0 < 0}
    leaves_c = {(b, e) for b, e, s0, _ in nodes_c if s0 < 0}
    for i0, i1, j0, j1, far in tr.blocks:
        cover[i0:i1, j0:j1] += 1
        lo1, hi1 = _box(V, sr, tr.perm_rows[i0:i1])
        lo2, hi2 = _box(V, sc, tr.perm_cols[j0:j1])
        diam = min(np.linalg.norm(hi1 - lo1), np.linalg.norm(hi2 - lo2))
        gap = np.maximum(0, np.maximum(lo2 - hi1, lo1 - hi2))
        dist = np.linalg.norm(gap)
        if far:
            nfar += 1
            assert dist > 0 and diam <= eta * dist * (1 + 1e-12)
        else:
            assert not (dist > 0 and diam < eta * dist * (1 - 1e-12))
            assert (i0, i1) in leaves_r or (j0, j1) in leaves_c
    assert np.all(cover == 1)
    assert nfar > 0


def test_tree_deterministic(orc):
    V, T = icosphere(3)
    m = orc.Mesh(V, T)
    a = orc.Tree(m, 0, 0, 32, 2.0)
    b = orc.Tree(m, 0, 0, 32, 2.0)
    assert np.array_equal(a.perm_rows, b.perm_rows) and np.array_equal(a.blocks, b.blocks)
