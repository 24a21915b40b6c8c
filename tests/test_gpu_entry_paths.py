"""Entry-level parity of the kernels that tdbem_compress runs (run with -m gpu).

The compression forms its entries with three kernels that tdbem_entries does
not use: the touching-pair table (Sauter-Schwab, FP64 geometry; in the mixed
form with the smooth factor and the lane sums in FP32), the dense near-field
tensor kernel (regular pairs with the point geometry shared across
frequencies) and the far-field engine's 8-lane point-pair groups (row and
column fibres and frequency tubes of Algorithm 1).  tdbem_entries_path runs
each of them on its own; here each is compared entry by entry with the FP64
oracle at 1e-5 (mixed form) and 1e-12 (FP64 form), on the 320-triangle sphere
(BDF2 N = 16, c = 1) and on a 2640-triangle finned housing (c = 343 m/s, gCQ
of 2-stage Radau IIA over 256 graded steps), where the phases s r / c reach
tens of radians.

Relative error of an entry: |g - o| / max(M, 1e-6 * scale_k), M the oracle's
magnitude sum of the entry (the same quadrature with every term replaced by a
bound of its modulus; |(x - y).n_y| bounded by |x - y| for the double layer)
and scale_k the largest magnitude sum of a self-interaction entry of the
sampled rows at s_k.  For the single layer at real s, M = |o|.  An entry's
terms may cancel (oscillating phases; the double-layer factor (x - y).n_y on
nearly flat neighbourhoods), and floating-point evaluation in either
precision is accurate only relative to M; the floor covers FP32 underflow of
exp(-Re(s) r / c).
"""
import numpy as np
import pytest

from paper_2505_00715_gb300.inputs import graded_steps, housing, icosphere

pytestmark = pytest.mark.gpu

TOL = {"FP64": 1e-12, "MIXED": 1e-5}


@pytest.fixture(scope="module")
def td():
    import paper_2505_00715_gb300 as td
    return td


@pytest.fixture(scope="module")
def ctx(td):
    return td.Context(0)


class Case:
    pass


@pytest.fixture(scope="module")
def sphere(td, ctx, orc):
    k = Case()
    k.V, k.T = icosphere(2)
    k.gm, k.om = td.Mesh(ctx, k.V, k.T), orc.Mesh(k.V, k.T)
    k.f = td.Freqs.bdf2(ctx, 16, 0.1)
    k.fidx = np.concatenate([k.f.unique, [11, 15]]).astype(np.int32)  # two conjugate points as well
    k.c = 1.0
    k.leaf = 16
    return k


@pytest.fixture(scope="module")
def hous(td, ctx, orc):
    k = Case()
    k.V, k.T = housing(2000, seed=0)
    k.gm, k.om = td.Mesh(ctx, k.V, k.T), orc.Mesh(k.V, k.T)
    k.f = td.Freqs.gcq(ctx, graded_steps(256, 1.01, 0.015), td.RADAU2, 256, rho=1.0)
    u = k.f.unique
    # 32 of the 128 unique contour points, spread over the contour (the
    # largest |Im s| and Re s among them), and two conjugate points
    k.fidx = np.concatenate([u[::4], [u[-1] + 1, 255 - u[5]]]).astype(np.int32)
    k.c = 343.0
    k.leaf = 64
    return k


def _own_dof(k, op, rows):
    if op == "SLP":
        return np.asarray(rows, dtype=np.int32)
    if op == "DLP":
        return k.T[np.asarray(rows), 0].astype(np.int32)
    # K' of a flat panel with itself is zero: a neighbour across vertex 0 instead
    out = []
    for r in rows:
        v = k.T[r, 0]
        out.append(next(t for t in np.nonzero((k.T == v).any(axis=1))[0] if t != r))
    return np.asarray(out, dtype=np.int32)


def _scale(k, orc, op, rows, fidx):
    """Largest magnitude sum over the self-interaction entries of the rows
    (for K', whose self-interaction vanishes, over entries of a neighbour
    across the row's first vertex)."""
    own = _own_dof(k, op, rows)
    diag = np.stack([k.om.entries_mag(getattr(orc, op), [r], [q], k.f.s[fidx], c=k.c, ng=5)[:, 0, 0]
                     for r, q in zip(rows[:8], own[:8])], axis=1)
    return diag.max(axis=1)


def _rel_err(g, o, mag, scale):
    den = np.maximum(mag, 1e-6 * scale.reshape((-1,) + (1,) * (o.ndim - 1)))
    return np.abs(g - o) / den


def _oracle(k, orc, op, rows, cols, fidx):
    o = k.om.entries(getattr(orc, op), rows, cols, k.f.s[fidx], c=k.c, ng=5)
    mag = k.om.entries_mag(getattr(orc, op), rows, cols, k.f.s[fidx], c=k.c, ng=5)
    return o, mag, _scale(k, orc, op, rows, fidx)


def _near_strip(td, k, op):
    """A row leaf of the tree and every column of its near-field blocks."""
    cols_b = td.P1 if op == "DLP" else td.P0
    tree = td.Tree(k.gm, td.P0, cols_b, k.leaf, 2.0)
    b = tree.blocks
    near = b[b[:, 4] == 0]
    # the row range with the most near-field columns
    keys = {}
    for i0, i1, j0, j1, _ in near:
        keys.setdefault((i0, i1), []).append((j0, j1))
    (i0, i1), js = max(keys.items(), key=lambda kv: sum(j1 - j0 for j0, j1 in kv[1]))
    rows = tree.perm_rows[i0:i1]
    cols = np.concatenate([tree.perm_cols[j0:j1] for j0, j1 in sorted(js)])
    return rows.astype(np.int32), cols.astype(np.int32)


def _touch_mask(k, rows, cols, op):
    """True where test triangle rows[r] touches (shares a vertex with) the
    support of column cols[c]."""
    tv = [set(k.T[r]) for r in rows]
    if op != "DLP":
        cv = [set(k.T[c]) for c in cols]
    else:
        sup = {}
        for t, tri in enumerate(k.T):
            for v in tri:
                sup.setdefault(int(v), set()).update(int(x) for x in tri)
        cv = [sup[int(c)] for c in cols]
    return np.array([[bool(a & b) for b in cv] for a in tv])


@pytest.mark.parametrize("prec", ["MIXED", "FP64"])
@pytest.mark.parametrize("op", ["SLP", "DLP", "ADLP"])
@pytest.mark.parametrize("mesh", ["sphere", "housing"])
def test_near_path_vs_oracle(td, orc, sphere, hous, mesh, op, prec):
    """Touching-pair table + near-field tensor kernel on a near-field row
    strip (identical, edge, vertex and regular pairs), every listed
    frequency, against the oracle's entries (Sauter-Schwab ng = 5 and the
    7 x 7 rule)."""
    k = sphere if mesh == "sphere" else hous
    rows, cols = _near_strip(td, k, op)
    fidx = k.fidx if (mesh == "sphere" or op != "DLP") else k.fidx[::2]
    g = td.entries(k.gm, getattr(td, op), k.f, rows, cols, fidx, prec=getattr(td, prec), c=k.c, ng=5,
                   path=td.PATH_NEAR).cpu().numpy()
    o, mag, sc = _oracle(k, orc, op, rows, cols, fidx)
    err = _rel_err(g, o, mag, sc)
    touch = np.broadcast_to(_touch_mask(k, rows, cols, op), err.shape)
    e_t, e_r = float(err[touch].max()), float(err[~touch].max())
    print("near path %s %s %s: %d x %d x %d entries, max rel err touching %.2e, regular %.2e"
          % (mesh, op, prec, len(rows), len(cols), len(fidx), e_t, e_r))
    assert np.all(np.isfinite(g))
    assert max(e_t, e_r) <= TOL[prec], (e_t, e_r)


@pytest.mark.parametrize("prec", ["MIXED", "FP64"])
@pytest.mark.parametrize("op", ["SLP", "DLP", "ADLP"])
@pytest.mark.parametrize("mesh", ["sphere", "housing"])
def test_generic_path_vs_oracle(td, orc, sphere, hous, mesh, op, prec):
    """tdbem_entries on the same near-field strip (its touching pairs are
    integrated in FP64 in both forms)."""
    k = sphere if mesh == "sphere" else hous
    rows, cols = _near_strip(td, k, op)
    fidx = k.fidx[::2]
    g = td.entries(k.gm, getattr(td, op), k.f, rows, cols, fidx, prec=getattr(td, prec), c=k.c,
                   ng=5).cpu().numpy()
    o, mag, sc = _oracle(k, orc, op, rows, cols, fidx)
    err = float(_rel_err(g, o, mag, sc).max())
    print("generic path %s %s %s: max rel err %.2e" % (mesh, op, prec, err))
    assert err <= TOL[prec], err


@pytest.mark.parametrize("prec", ["MIXED", "FP64"])
@pytest.mark.parametrize("op", ["SLP", "DLP", "ADLP"])
@pytest.mark.parametrize("mesh", ["sphere", "housing"])
def test_fibre_path_vs_oracle(td, orc, sphere, hous, mesh, op, prec):
    """The far-field engine's point-pair groups on rows x columns of
    admissible blocks (the nearest and the farthest ones, where the phase
    s r / c is largest), every listed frequency: the entries of its row and
    column fibres and of its frequency tubes."""
    k = sphere if mesh == "sphere" else hous
    cols_b = td.P1 if op == "DLP" else td.P0
    tree = td.Tree(k.gm, td.P0, cols_b, k.leaf, 2.0)
    b = tree.blocks
    far = b[b[:, 4] == 1]
    assert len(far) > 0
    size = (far[:, 1] - far[:, 0]) * (far[:, 3] - far[:, 2])
    pick = far[np.unique(np.r_[np.argsort(size)[:3], np.argsort(size)[-3:]])]
    worst = 0.0
    for i0, i1, j0, j1, _ in pick:
        rows = tree.perm_rows[i0:min(i1, i0 + 6)].astype(np.int32)
        cols = tree.perm_cols[j0:j1][:96].astype(np.int32)
        assert not _touch_mask(k, rows, cols, op).any()
        g = td.entries(k.gm, getattr(td, op), k.f, rows, cols, k.fidx, prec=getattr(td, prec), c=k.c, ng=5,
                       path=td.PATH_FIBRE).cpu().numpy()
        o, mag, sc = _oracle(k, orc, op, rows, cols, k.fidx)
        worst = max(worst, float(_rel_err(g, o, mag, sc).max()))
    print("fibre path %s %s %s: max rel err %.2e over %d far blocks" % (mesh, op, prec, worst, len(pick)))
    assert worst <= TOL[prec], worst


def test_path_argument_errors(td, sphere):
    k = sphere
    with pytest.raises(td.TdbemError):
        td.entries(k.gm, td.SLP, k.f, [0], [len(k.T)], [0], path=td.PATH_NEAR)  # column out of range
    with pytest.raises(td.TdbemError):
        td.entries(k.gm, td.SLP, k.f, [0], [0], [16], path=td.PATH_FIBRE)  # frequency out of range
    with pytest.raises(td.TdbemError):
        td.entries(k.gm, td.SLP, k.f, [0], [0], [0], path=7)
    assert td.entries(k.gm, td.SLP, k.f, [], [0], [0], path=td.PATH_NEAR).numel() == 0
