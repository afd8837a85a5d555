"""CPU oracle for the selector network (test infrastructure only).

Plain numpy in fp64: the 12 -> 64 -> 64 -> 15 multilayer perceptron with ReLU
hidden layers and a softmax output, its two training losses over the relative
slowdowns C_ic of plan class c on sample i -- the expected regret of the
softmax choice, mean_i sum_c p_ic C_ic (tau = 0), and the cross-entropy
toward the soft target q_i = softmax(-C_i / tau), mean_i -sum_c q_ic log p_ic
(tau > 0) -- the gradient by backpropagation, and one Adam step. Parameter packing matches the library's: W1[64][12], b1[64],
W2[64][64], b2[64], W3[15][64], b3[15], each row-major (out x in).

Pinned by tests/test_oracle_mlp_pins.py: central differences of the loss,
closed forms of a network whose output is its last bias, and ReLU gating.
"""

from __future__ import annotations

import numpy as np

IN, HID, OUT = 12, 64, 15
SHAPES = [("W1", (HID, IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)), ("W3", (OUT, HID)),
          ("b3", (OUT,))]
P = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(params):
    params = np.asarray(params, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = params[o:o + n].reshape(shape)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def forward(params, X):
    """Logits z[n][15] and the hidden activations."""
    w = unpack(params)
    X = np.asarray(X, dtype=np.float64)
    a1 = X @ w["W1"].T + w["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ w["W2"].T + w["b2"]
    h2 = np.maximum(a2, 0.0)
    z = h2 @ w["W3"].T + w["b3"]
    return z, (X, a1, h1, a2, h2)


def softmax(z):
    e = np.exp(z - z.max(axis=1, keepdims=True))
    return e / e.sum(axis=1, keepdims=True)


def log_softmax(z):
    s = z - z.max(axis=1, keepdims=True)
    return s - np.log(np.exp(s).sum(axis=1, keepdims=True))


def loss(params, X, C, tau=0.0):
    z, _ = forward(params, X)
    C = np.asarray(C, dtype=np.float64)
    if tau > 0:
        q = softmax(-C / tau)
        return float(np.mean(-np.sum(q * log_softmax(z), axis=1)))
    return float(np.mean(np.sum(softmax(z) * C, axis=1)))


def loss_and_grad(params, X, C, tau=0.0):
    """The mean loss (expected regret for tau = 0, soft-target cross-entropy
    for tau > 0) and its gradient (packed like params)."""
    w = unpack(params)
    C = np.asarray(C, dtype=np.float64)
    n = C.shape[0]
    z, (X, a1, h1, a2, h2) = forward(params, X)
    p = softmax(z)
    if tau > 0:
        q = softmax(-C / tau)
        per = -np.sum(q * log_softmax(z), axis=1)
        dz = (p - q) / n                     # d/dz of -q . log softmax(z)
    else:
        per = np.sum(p * C, axis=1)
        dz = p * (C - per[:, None]) / n      # d/dz of p . c for a softmax p
    g = {"W3": dz.T @ h2, "b3": dz.sum(0)}
    dh2 = dz @ w["W3"]
    da2 = dh2 * (a2 > 0)
    g["W2"] = da2.T @ h1
    g["b2"] = da2.sum(0)
    dh1 = da2 @ w["W2"]
    da1 = dh1 * (a1 > 0)
    g["W1"] = da1.T @ X
    g["b1"] = da1.sum(0)
    return float(per.mean()), pack(g)


def adam(params, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015); returns new (params, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v
