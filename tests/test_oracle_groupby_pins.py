"""Pins of the group-by oracle (oracle_groupby) against facts that do not come
from it: a Python dict brute force on small inputs, closed forms of keys
i mod g over values i, and the invariants that the counts add up to the rows
and the group sums to the column sum (modulo 2^64)."""

import numpy as np
import pytest

M64 = 1 << 64


def _wrap(x):
    x %= M64
    return x - M64 if x >= 1 << 63 else x


def _brute(keys, aggs):
    groups = {}
    for i, k in enumerate(keys.tolist()):
        acc = groups.setdefault(k, [None] * len(aggs))
        for a, (op, vals) in enumerate(aggs):
            v = None if vals is None else int(vals[i])
            if op == "sum":
                acc[a] = _wrap((acc[a] or 0) + v)
            elif op == "count":
                acc[a] = (acc[a] or 0) + 1
            elif op == "min":
                acc[a] = v if acc[a] is None else min(acc[a], v)
            else:
                acc[a] = v if acc[a] is None else max(acc[a], v)
    ks = sorted(groups)
    return ks, [[groups[k][a] for k in ks] for a in range(len(aggs))]


@pytest.mark.parametrize("kdt,vdt,seed", [(np.int32, np.int32, 0), (np.int64, np.int64, 1),
                                          (np.int32, np.int64, 2), (np.int64, np.int32, 3)])
def test_groupby_matches_dict_brute_force(oracle_mod, kdt, vdt, seed):
    rng = np.random.default_rng(seed)
    info_k, info_v = np.iinfo(kdt), np.iinfo(vdt)
    keys = rng.integers(-30, 30, size=3000).astype(kdt)
    keys[:3] = [info_k.min, info_k.max, 0]
    v1 = rng.integers(info_v.min, info_v.max, size=3000, dtype=np.int64).astype(vdt)
    v1[:4] = [info_v.min, info_v.max, info_v.max, -1]   # sums that wrap
    v2 = rng.integers(-1000, 1000, size=3000).astype(vdt)
    aggs = [("sum", v1), ("count", None), ("min", v2), ("max", v1)]
    ks, cols = oracle_mod.groupby(keys, aggs)
    bk, bcols = _brute(keys, aggs)
    assert ks.tolist() == bk
    for got, want in zip(cols, bcols):
        assert got.tolist() == want


@pytest.mark.parametrize("n,g", [(1000, 7), (4096, 4096), (10_000, 1), (12_345, 1000)])
def test_groupby_closed_form_of_modular_keys(oracle_mod, n, g):
    i = np.arange(n, dtype=np.int64)
    ks, (s, c, mn, mx) = oracle_mod.groupby(i % g, [("sum", i), ("count", None), ("min", i), ("max", i)])
    k = np.arange(min(g, n))
    cnt = (n - 1 - k) // g + 1
    assert ks.tolist() == k.tolist()
    assert c.tolist() == cnt.tolist()
    assert s.tolist() == (cnt * k + g * cnt * (cnt - 1) // 2).tolist()
    assert mn.tolist() == k.tolist()
    assert mx.tolist() == (k + (cnt - 1) * g).tolist()


def test_groupby_counts_and_sums_add_up(oracle_mod):
    rng = np.random.default_rng(9)
    keys = rng.integers(-2**63, 2**63 - 1, size=50_000, dtype=np.int64) >> rng.integers(40, 63)
    vals = rng.integers(-2**63, 2**63 - 1, size=keys.size, dtype=np.int64)
    ks, (s, c) = oracle_mod.groupby(keys, [("sum", vals), ("count", None)])
    assert ks.tolist() == np.unique(keys).tolist()
    assert int(c.sum()) == keys.size
    total = _wrap(sum(int(v) for v in vals.tolist()))
    assert _wrap(sum(int(x) for x in s.tolist())) == total


def test_groupby_empty_input(oracle_mod):
    ks, (s,) = oracle_mod.groupby(np.empty(0, np.int32), [("sum", np.empty(0, np.int32))])
    assert ks.size == 0 and s.size == 0
