"""Pins of the oracle's rank-predictor MLP (forward, loss, gradient, Adam)."""
import numpy as np
import pytest


def _init(orc, seed=2):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(orc.mlp_nparams()) * 0.3


def _data(n, seed=0):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, 6))
    lab = rng.integers(0, 16, size=n).astype(np.int32)
    return x, lab


def test_forward_matches_library_gelu(orc):
    """Forward pass against numpy matmuls with GELU from scipy's erf."""
    sp = pytest.importorskip("scipy.special")
    P = _init(orc)
    x, _ = _data(7)
    o = 0
    W1 = P[o:o + 384].reshape(64, 6); o += 384
    b1 = P[o:o + 64]; o += 64
    W2 = P[o:o + 4096].reshape(64, 64); o += 4096
    b2 = P[o:o + 64]; o += 64
    W3 = P[o:o + 1024].reshape(16, 64); o += 1024
    b3 = P[o:o + 16]
    g = lambda z: 0.5 * z * (1 + sp.erf(z / np.sqrt(2)))
    ref = g(g(x @ W1.T + b1) @ W2.T + b2) @ W3.T + b3
    assert np.allclose(orc.mlp_forward(P, x), ref, rtol=1e-13, atol=1e-13)


def test_gradient_central_differences(orc):
    P = _init(orc)
    x, lab = _data(9)
    loss, g = orc.mlp_loss_grad(P, x, lab)
    rng = np.random.default_rng(1)
    idx = rng.choice(len(P), 60, replace=False)
    h = 1e-6
    for k in idx:
        Pp, Pm = P.copy(), P.copy()
        Pp[k] += h
        Pm[k] -= h
        fd = (orc.mlp_loss_grad(Pp, x, lab, False)[0] - orc.mlp_loss_grad(Pm, x, lab, False)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(fd)) + 1e-9, (k, fd, g[k])
    # loss is the mean softmax cross-entropy (scipy logsumexp)
    sp = pytest.importorskip("scipy.special")
    lg = orc.mlp_forward(P, x)
    ref = np.mean(sp.logsumexp(lg, axis=1) - lg[np.arange(len(x)), lab])
    assert abs(loss - ref) < 1e-12


def test_adam_first_step_is_lr_sign(orc):
    """With zero moments the first Adam step moves every parameter by lr*sign(g)
    (bias correction makes m_hat = g and v_hat = g^2)."""
    P = _init(orc)
    x, lab = _data(16)
    _, g = orc.mlp_loss_grad(P, x, lab)
    m, v = np.zeros_like(P), np.zeros_like(P)
    P1 = P.copy()
    orc.adam_step(P1, g, m, v, 1e-3, 1, eps=1e-30)
    nz = np.abs(g) > 1e-20
    assert np.allclose((P - P1)[nz], 1e-3 * np.sign(g[nz]), rtol=1e-12)


def test_training_reduces_loss(orc):
    P = _init(orc)
    x, lab = _data(64)
    lab = (x[:, 0] > 0).astype(np.int32) * 3 + (x[:, 1] > 0).astype(np.int32)
    m, v = np.zeros_like(P), np.zeros_like(P)
    l0 = orc.mlp_loss_grad(P, x, lab, False)[0]
    for t in range(1, 201):
        _, g = orc.mlp_loss_grad(P, x, lab)
        orc.adam_step(P, g, m, v, 1e-2, t)
    assert orc.mlp_loss_grad(P, x, lab, False)[0] < 0.2 * l0
