"""The seeded input generators against the recipes they state (CPU only).

Both the oracle and the CUDA path read these inputs, so the properties the
parity tests and the closed forms rely on are checked here directly: unique
build keys, probe keys drawn from the build keys, the dense span that makes
narrowing apply, the star schema's absent-key fraction and filter, the
batched joins' sizes, and determinism under a seed.
"""

import numpy as np
import pytest
import torch

from paper_2607_04489_gb300 import workloads


def test_small_static_recipe():
    w = workloads.small_static(nb=1 << 12, np_=1 << 14)
    bk = w.build_keys.numpy()
    assert w.build_keys.dtype == torch.int32 and np.array_equal(np.sort(bk), np.arange(1 << 12))
    assert np.array_equal(w.build_pay.numpy(), (np.arange(1 << 12) ^ 0x5A5A5A5A).astype(np.int32))
    pk = w.probe_keys.numpy()
    assert pk.min() >= 0 and pk.max() < (1 << 12) and np.array_equal(w.probe_pay.numpy(), np.arange(1 << 14))


@pytest.mark.parametrize("keys", ["dense", "random"])
@pytest.mark.parametrize("theta", [0.0, 1.0])
def test_variant_sweep_recipe(keys, theta):
    nb, ratio = 1 << 14, 4
    w = workloads.variant_sweep(nb, ratio, keys=keys, theta=theta, seed=3)
    bk, pk = w.build_keys.numpy(), w.probe_keys.numpy()
    assert w.build_keys.dtype == torch.int64 and w.np == ratio * nb
    assert np.unique(bk).size == nb  # unique build keys
    assert np.isin(pk, bk).all()  # every probe row matches exactly once
    span = int(bk.max()) - int(bk.min())
    if keys == "dense":
        assert span == nb - 1 and abs(int(bk.min())) <= 1 << 40  # narrows to 32 bits
    else:
        assert span > 1 << 32  # spread over 64 bits: no narrowing
    counts = np.unique(pk, return_counts=True)[1]
    if theta == 0.0:
        assert counts.max() < 20  # uniform: about 4 per key
    else:
        assert counts.max() > 0.05 * pk.size  # Zipf 1: the hottest key takes a large share


def test_variant_sweep_is_deterministic_per_seed():
    a = workloads.variant_sweep(1 << 12, 2, seed=5)
    b = workloads.variant_sweep(1 << 12, 2, seed=5)
    c = workloads.variant_sweep(1 << 12, 2, seed=6)
    for x, y in ((a.build_keys, b.build_keys), (a.probe_keys, b.probe_keys), (a.probe_pay, b.probe_pay)):
        assert torch.equal(x, y)
    assert not torch.equal(a.build_keys, c.build_keys)


@pytest.mark.parametrize("sel", [1.0, 0.1])
@pytest.mark.parametrize("theta", [0.0, 1.0])
def test_star_schema_recipe(sel, theta):
    n_dim, n_fact = 20_000, 100_000
    w = workloads.star_schema(n_dim=n_dim, n_fact=n_fact, theta=theta, selectivity=sel, seed=2)
    dk, fk = w.build_keys.numpy(), w.probe_keys.numpy()
    assert w.build_keys.dtype == torch.int32 and w.probe_keys.dtype == torch.int32
    assert np.array_equal(np.sort(dk), np.arange(1, n_dim + 1))  # dense keys 1..n_dim
    assert w.build_pay.dtype == torch.int64 and w.probe_pay.dtype == torch.int64
    assert 0 <= int(w.build_pay.min()) and int(w.build_pay.max()) < 10**9
    assert 0 <= int(w.probe_pay.min()) and int(w.probe_pay.max()) < 10**7
    assert abs(fk.size / n_fact - sel) < 0.01  # the filter keeps its fraction of the fact rows
    absent = fk > n_dim
    assert abs(absent.mean() - 0.10) < 0.01 and (fk[absent] <= 2 * n_dim + 1).all()
    assert (fk >= 1).all()


def test_batched_small_recipe():
    b = workloads.batched_small(k=24, log2_lo=6, log2_hi=12, seed=4)
    assert len(b.builds) == len(b.probes) == len(b.thetas) == 24
    for bk, pk, th in zip(b.builds, b.probes, b.thetas):
        assert bk.dtype == torch.int32 and 64 <= bk.numel() <= 4096
        assert pk.numel() == 4 * bk.numel() and 0.0 <= th <= 1.0
        k = bk.numpy()
        assert np.unique(k).size == k.size and np.isin(pk.numpy(), k).all()
    assert b.tuples == sum(5 * x.numel() for x in b.builds)
