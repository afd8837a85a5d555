"""Pins of the selector-network oracle (oracle/mlp.py) that do not come from
the oracle itself: central differences of its loss, closed forms of a network
whose output equals its last bias, and ReLU gating of the hidden layers."""

import numpy as np
import pytest

from oracle import mlp


def _random(seed, n=7):
    rng = np.random.default_rng(seed)
    params = rng.normal(0, 0.3, size=mlp.P)
    X = rng.normal(0, 1, size=(n, mlp.IN))
    C = rng.uniform(0, 2, size=(n, mlp.OUT))
    C[np.arange(n), rng.integers(0, mlp.OUT, size=n)] = 0.0
    return params, X, C


def test_parameter_count():
    assert mlp.P == 64 * 12 + 64 + 64 * 64 + 64 + 15 * 64 + 15 == 5967


@pytest.mark.parametrize("seed,tau", [(0, 0.0), (1, 0.0), (2, 0.0), (3, 0.05), (4, 0.5)])
def test_gradient_matches_central_differences(seed, tau):
    params, X, C = _random(seed)
    _, g = mlp.loss_and_grad(params, X, C, tau)
    rng = np.random.default_rng(100 + seed)
    idx = rng.choice(mlp.P, size=300, replace=False)
    h = 1e-6
    for q in idx:
        e = np.zeros(mlp.P)
        e[q] = h
        num = (mlp.loss(params + e, X, C, tau) - mlp.loss(params - e, X, C, tau)) / (2 * h)
        assert num == pytest.approx(g[q], rel=1e-5, abs=1e-9)


def test_cross_entropy_of_uniform_logits_is_log_classes():
    """Equal logits give p = 1/15 whatever the target, so -sum q log p = ln 15."""
    _, X, C = _random(7)
    assert mlp.loss(np.zeros(mlp.P), X, C, 0.05) == pytest.approx(np.log(15.0), rel=1e-12)


def test_cross_entropy_sharp_target_is_negative_log_likelihood():
    """With one class 1+ cheaper than every other and tau = 1e-3, the soft
    target is one-hot up to exp(-1000): the loss is -log p of that class."""
    params, X, C = _random(8)
    best = np.argmin(C, axis=1)
    C = C + 1.0
    C[np.arange(len(C)), best] = 0.0
    z, _ = mlp.forward(params, X)
    zs = z - z.max(axis=1, keepdims=True)
    nll = -(zs[np.arange(len(z)), best] - np.log(np.exp(zs).sum(axis=1)))
    assert mlp.loss(params, X, C, 1e-3) == pytest.approx(nll.mean(), rel=1e-12)


def test_cross_entropy_splits_ties_evenly():
    """Two zero-cost classes and the rest far more expensive: the target puts
    one half on each tie, so the loss of a network that does the same is ln 2."""
    d = {name: np.zeros(shape) for name, shape in mlp.SHAPES}
    d["b3"] = np.full(mlp.OUT, -1e3)
    d["b3"][[2, 9]] = 0.0
    C = np.full((3, mlp.OUT), 50.0)
    C[:, [2, 9]] = 0.0
    X = np.random.default_rng(9).normal(size=(3, mlp.IN))
    assert mlp.loss(mlp.pack(d), X, C, 0.1) == pytest.approx(np.log(2.0), rel=1e-9)


def test_constant_logits_closed_form():
    """All weights zero: every sample's logits are b3, p = softmax(b3); the loss
    is mean_i p . C_i and dL/db3 = mean_i p * (C_i - p . C_i)."""
    rng = np.random.default_rng(4)
    d = {name: np.zeros(shape) for name, shape in mlp.SHAPES}
    d["b3"] = rng.normal(size=mlp.OUT)
    params = mlp.pack(d)
    X = rng.normal(size=(5, mlp.IN))
    C = rng.uniform(0, 3, size=(5, mlp.OUT))
    p = np.exp(d["b3"]) / np.exp(d["b3"]).sum()
    L, g = mlp.loss_and_grad(params, X, C)
    assert L == pytest.approx(np.mean(C @ p), rel=1e-12)
    gb3 = g[-mlp.OUT:]
    expect = np.mean([p * (c - p @ c) for c in C], axis=0)
    np.testing.assert_allclose(gb3, expect, rtol=1e-10, atol=1e-14)
    # zero weights: no gradient flows below the last layer's weights
    assert np.all(g[: mlp.P - mlp.OUT - mlp.OUT * 64] == 0.0)


def test_uniform_choice_loss_is_mean_cost():
    params = np.zeros(mlp.P)
    _, X, C = _random(5)
    assert mlp.loss(params, X, C) == pytest.approx(C.mean(), rel=1e-12)


def test_relu_blocks_negative_hidden_units():
    params, X, C = _random(6)
    w = mlp.unpack(params.copy())
    w["b1"][:] = -1e6  # every first-layer unit off
    params = mlp.pack(w)
    _, g = mlp.loss_and_grad(params, X, C)
    d = mlp.unpack(g)
    assert np.all(d["W1"] == 0) and np.all(d["b1"] == 0) and np.all(d["W2"] == 0)


def test_adam_first_step_moves_by_lr_against_the_gradient_sign():
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    p, m, v = mlp.adam(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, 0.01)
    np.testing.assert_allclose(p[:3], -0.01 * np.sign(g[:3]), rtol=1e-4)
    assert p[3] == 0.0
