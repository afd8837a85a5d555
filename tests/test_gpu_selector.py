"""The selector network's kernels vs the fp64 oracle (oracle/mlp.py), and the
learned selector inside EIGER_AUTO: it changes only which plan runs, never the
join result."""

import numpy as np
import pytest
import torch

from oracle import mlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eiger():
    from paper_2607_04489_gb300 import eiger

    eiger.load()
    return eiger


def _problem(seed, n):
    rng = np.random.default_rng(seed)
    params = rng.normal(0, 0.25, size=mlp.P).astype(np.float32)
    X = rng.normal(0, 1, size=(n, mlp.IN)).astype(np.float32)
    C = rng.uniform(0, 3, size=(n, mlp.OUT)).astype(np.float32)
    C[np.arange(n), rng.integers(0, mlp.OUT, size=n)] = 0
    return params, X, C


def test_param_count(eiger):
    assert eiger.mlp_param_count() == mlp.P


@pytest.mark.parametrize("n", [1, 5, 300, 2500])
def test_forward_matches_oracle(eiger, n):
    params, X, _ = _problem(n, n)
    z = eiger.mlp_forward(torch.from_numpy(params).cuda(), torch.from_numpy(X).cuda()).cpu().numpy()
    zo, _ = mlp.forward(params.astype(np.float64), X.astype(np.float64))
    np.testing.assert_allclose(z, zo, rtol=1e-4, atol=1e-4 * np.abs(zo).max())


@pytest.mark.parametrize("n,tau", [(3, 0.0), (257, 0.0), (2500, 0.0), (3, 0.05), (257, 0.05), (2500, 0.5)])
def test_gradient_matches_oracle(eiger, n, tau):
    params, X, C = _problem(100 + n, n)
    L, g = eiger.mlp_grad(torch.from_numpy(params).cuda(), torch.from_numpy(X).cuda(),
                          torch.from_numpy(C).cuda(), tau)
    Lo, go = mlp.loss_and_grad(params.astype(np.float64), X.astype(np.float64), C.astype(np.float64), tau)
    g = g.cpu().numpy()
    assert float(L) == pytest.approx(Lo, rel=1e-5)
    # relative error of the whole gradient vector, and per component
    assert np.linalg.norm(g - go) <= 1e-4 * np.linalg.norm(go)
    big = np.abs(go) > 1e-3 * np.abs(go).max()
    np.testing.assert_allclose(g[big], go[big], rtol=1e-3)


def test_adam_matches_oracle(eiger):
    rng = np.random.default_rng(3)
    p = rng.normal(size=mlp.P).astype(np.float32)
    g = rng.normal(size=mlp.P).astype(np.float32)
    m = rng.normal(size=mlp.P).astype(np.float32) * 0.1
    v = np.abs(rng.normal(size=mlp.P)).astype(np.float32) * 0.1
    tp, tg, tm, tv = (torch.from_numpy(a.copy()).cuda() for a in (p, g, m, v))
    eiger.mlp_adam(tp, tg, tm, tv, 7, 1e-3)
    po, mo, vo = mlp.adam(p.astype(np.float64), g.astype(np.float64), m.astype(np.float64),
                          v.astype(np.float64), 7, 1e-3)
    np.testing.assert_allclose(tp.cpu().numpy(), po, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(tm.cpu().numpy(), mo, rtol=1e-5, atol=1e-7)


def test_training_with_library_kernels_lowers_the_loss(eiger):
    from paper_2607_04489_gb300 import selector

    rng = np.random.default_rng(9)
    X = rng.normal(size=(400, mlp.IN)).astype(np.float32)
    best = (X[:, 0] > 0).astype(int) * 6  # a learnable rule: class 0 or 6
    T = np.full((400, mlp.OUT), 3.0)
    T[np.arange(400), best] = 1.0
    model = selector.train(X, T, steps=600, lr=5e-3, n_train=300)
    hist = model["loss_history"]
    assert hist[-1][1] < 0.3 * hist[0][1]
    ev = selector.evaluate(model, X, T, T[:, 0], n_train=300)
    assert ev["learned"]["mean"] < 0.2


def test_learned_selector_drives_auto_without_changing_results(eiger, oracle_mod):
    from paper_2607_04489_gb300 import selector, workloads

    rng = np.random.default_rng(5)
    params = (rng.normal(0, 0.5, size=mlp.P)).astype(np.float32)
    model = {"params": params.tolist(), "mean": [0.0] * 12, "scale": [1.0] * 12}
    cases = [workloads.variant_sweep(1 << 16, 4, keys="dense", seed=1),
             workloads.variant_sweep(1 << 15, 2, keys="random", theta=1.0, seed=2),
             workloads.small_static(nb=1 << 14, np_=1 << 16)]
    try:
        selector.use(model)
        for w in cases:
            bk, pk = w.build_keys.cuda(), w.probe_keys.cuda()
            r = eiger.join(bk, pk, variant="auto")
            assert r.plan.selector == 1
            # the class the oracle network picks from the library's own features
            dt = eiger.I32 if bk.dtype == torch.int32 else eiger.I64
            f = eiger.features(eiger.stats(bk), eiger.stats(pk[: 1 << 20]), bk.numel(), pk.numel(), dt)
            z, _ = mlp.forward(params.astype(np.float64), f[None, :].astype(np.float64))
            want = eiger.class_plan(int(np.argmax(z)))
            assert (r.plan.variant, r.plan.bits1, r.plan.bits2) == (want.variant, want.bits1, want.bits2)
            eb, ep, n = oracle_mod.join(w.build_keys.numpy(), w.probe_keys.numpy())
            assert r.count == n
            b = r.build_idx.cpu().numpy().astype(np.int64)
            p = r.probe_idx.cpu().numpy().astype(np.int64)
            o = np.lexsort((b, p))
            np.testing.assert_array_equal(b[o], eb.astype(np.int64))
            np.testing.assert_array_equal(p[o], ep.astype(np.int64))
    finally:
        eiger.selector_set(None)
    r = eiger.join(cases[0].build_keys.cuda(), cases[0].probe_keys.cuda(), variant="auto")
    assert r.plan.selector == 0
