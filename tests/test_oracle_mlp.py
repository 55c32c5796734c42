"""Pins of the oracle's learned-warm-start MLP (forward, gradient, AdamW)."""
import math

import numpy as np
import pytest


def _init(rng, dims, scale=0.3):
    Nk, H1, H2, K = dims
    parts = [rng.normal(0, scale / math.sqrt(Nk), (H1, Nk)), rng.normal(0, 0.1, H1),
             rng.normal(0, scale / math.sqrt(H1), (H2, H1)), rng.normal(0, 0.1, H2),
             rng.normal(0, scale / math.sqrt(H2), (K, H2)), rng.normal(0, 0.1, K)]
    return np.concatenate([p.ravel() for p in parts])


def test_activation_closed_forms(orc):
    assert orc.gelu(0.0) == 0.0
    assert abs(orc.gelu(1.0) - 0.8413447460685429) < 1e-15          # 1 * Phi(1)
    assert abs(orc.gelu(-1.0) - (-0.15865525393145707)) < 1e-15     # -1 * Phi(-1)
    assert abs(orc.gelu(8.0) - 8.0) < 1e-12
    assert abs(orc.softplus(0.0) - math.log(2.0)) < 1e-16
    assert orc.softplus(30.0) == 30.0                               # threshold branch
    assert abs(orc.softplus(-30.0) - math.exp(-30.0)) < 1e-25


def test_zero_weights_give_softplus_of_bias(orc):
    dims = (7, 5, 4, 3)
    prm = np.zeros(orc.mlp_nparams(*dims))
    prm[-3:] = [0.0, 1.0, -2.0]
    Y = orc.mlp_forward(prm, np.random.default_rng(0).uniform(size=(4, 7)), dims)
    np.testing.assert_allclose(Y, np.tile([math.log(2), math.log1p(math.e), math.log1p(math.exp(-2))], (4, 1)),
                               rtol=1e-15)


def test_forward_matches_layerwise_numpy(orc):
    # the packed layout and layer order, checked against an independent numpy evaluation
    from scipy.special import erf

    rng = np.random.default_rng(1)
    dims = (9, 6, 5, 2)
    prm = _init(rng, dims)
    X = rng.uniform(size=(3, 9))
    Nk, H1, H2, K = dims
    o = 0
    W1 = prm[o:o + H1 * Nk].reshape(H1, Nk); o += H1 * Nk
    b1 = prm[o:o + H1]; o += H1
    W2 = prm[o:o + H2 * H1].reshape(H2, H1); o += H2 * H1
    b2 = prm[o:o + H2]; o += H2
    W3 = prm[o:o + K * H2].reshape(K, H2); o += K * H2
    b3 = prm[o:o + K]
    g = lambda z: 0.5 * z * (1 + erf(z / math.sqrt(2)))
    ref = np.log1p(np.exp(g(g(X @ W1.T + b1) @ W2.T + b2) @ W3.T + b3))
    np.testing.assert_allclose(orc.mlp_forward(prm, X, dims), ref, rtol=1e-13)


def test_gradient_matches_central_differences(orc):
    rng = np.random.default_rng(2)
    dims = (11, 8, 6, 3)
    prm = _init(rng, dims, scale=1.0)
    X = rng.uniform(size=(5, 11))
    T = rng.uniform(0.1, 1.0, size=(5, 3))
    loss, G = orc.mlp_grad(prm, X, T, dims)
    _, loss2 = orc.mlp_forward(prm, X, dims, T)
    assert abs(loss - loss2) < 1e-15
    idx = rng.choice(prm.size, 40, replace=False)
    for i in idx:
        h = 1e-6
        p1, p2 = prm.copy(), prm.copy()
        p1[i] += h
        p2[i] -= h
        fd = (orc.mlp_forward(p1, X, dims, T)[1] - orc.mlp_forward(p2, X, dims, T)[1]) / (2 * h)
        assert abs(fd - G[i]) <= 1e-7 * max(1e-3, abs(G[i])) + 1e-10, (i, fd, G[i])


def test_adamw_first_step_and_decay(orc):
    # t = 1: bias-corrected m/sqrt(v) = g/|g|, so the step is lr*sign(g) (eps aside) plus lr*wd*w
    w = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 0.0])
    m, v = np.zeros(3), np.zeros(3)
    orc.adamw(w, g, m, v, 1, lr=0.01, eps=0.0 + 1e-12, wd=0.1)
    np.testing.assert_allclose(w, [1.0 - 0.01 - 0.001, -2.0 + 0.01 + 0.002, 0.5 - 0.0005], rtol=1e-9)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_training_reduces_loss(orc):
    # a few AdamW steps on a learnable map (targets from a teacher network)
    rng = np.random.default_rng(3)
    dims = (6, 8, 6, 2)
    teacher = _init(rng, dims, scale=1.5)
    X = rng.uniform(size=(64, 6))
    T = orc.mlp_forward(teacher, X, dims)
    prm = _init(rng, dims)
    m, v = np.zeros_like(prm), np.zeros_like(prm)
    l0, _ = orc.mlp_grad(prm, X, T, dims)
    for t in range(1, 201):
        loss, G = orc.mlp_grad(prm, X, T, dims)
        orc.adamw(prm, G, m, v, t, lr=3e-3, wd=0.0)
    assert loss < 0.2 * l0


def test_softplus_follows_its_definition_up_to_the_threshold(orc):
    # log(1 + e^z) itself (via e^-z, exact to rounding) for z up to 20, z beyond it
    for z in (5.0, 10.5, 15.0, 19.9):
        ref = z + math.log1p(math.exp(-z))
        assert abs(orc.softplus(z) - ref) <= 2e-16 * ref
    assert orc.softplus(20.5) == 20.5
