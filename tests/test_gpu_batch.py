"""Batched joins (eiger_join_batched) vs the oracle, join by join.

Every join of a batch is compared with the oracle's canonical pairs; the
cases cover empty joins, single rows, duplicate-heavy keys, int32 and int64
keys, small joins whose tables live in shared memory (with the path on and
off), per-join output capacities smaller than the result, CUDA-graph capture
and replay, and the status word for an undersized workspace. The full
4096-join workload is checked by counts (unique build keys, every probe key
drawn from them: |J_j| = np_j) and by exact parity on sampled joins.
"""

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eiger():
    from paper_2607_04489_gb300 import eiger

    eiger.load()
    return eiger


def _canon(b, p):
    b = b.cpu().numpy().astype(np.int64) & 0xFFFFFFFF
    p = p.cpu().numpy().astype(np.int64) & 0xFFFFFFFF
    o = np.lexsort((b, p))
    return b[o], p[o]


def _check_join(oracle_mod, bj, j, bk, pk, cap=None):
    n, gb, gp = bj.result(j)
    eb, ep, en = oracle_mod.join(bk.cpu().numpy(), pk.cpu().numpy())
    assert n == en, j
    if cap is None or en <= cap:
        b, p = _canon(gb, gp)
        np.testing.assert_array_equal(b, eb.astype(np.int64))
        np.testing.assert_array_equal(p, ep.astype(np.int64))


def _mixed_batch(dtype, seed, k=60):
    rng = np.random.default_rng(seed)
    builds, probes = [], []
    for j in range(k):
        kind = j % 6
        nb = int(rng.choice([0, 1, 7, 500, 4097, 20_000, 70_000]))
        np_ = int(rng.choice([0, 1, 3, 1000, 33_333, 100_000]))
        if kind == 0:    # unique keys, probes drawn from them
            bk = rng.permutation(max(nb, 1))[:nb] * 3 - 100
            pk = bk[rng.integers(0, max(nb, 1), size=np_)] if nb else rng.integers(0, 9, size=np_)
        elif kind == 1:  # duplicates
            bk = rng.integers(0, 40, size=nb)
            pk = rng.integers(0, 50, size=np_)
        elif kind == 2:  # disjoint ranges
            bk = rng.integers(0, 1000, size=nb)
            pk = rng.integers(5000, 6000, size=np_)
        else:            # wide keys
            lo, hi = (-2**31, 2**31 - 1) if dtype == np.int32 else (-2**62, 2**62)
            bk = rng.integers(lo, hi, size=nb)
            pk = np.concatenate([bk[rng.integers(0, max(nb, 1), size=np_ // 2)] if nb else np.zeros(0, np.int64),
                                 rng.integers(lo, hi, size=np_ - (np_ // 2 if nb else 0))])
        builds.append(torch.from_numpy(np.asarray(bk, dtype=dtype)).cuda())
        probes.append(torch.from_numpy(np.asarray(pk, dtype=dtype)).cuda())
    return builds, probes


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
@pytest.mark.parametrize("threads,chunk", [(128, 4096), (256, 16384), (512, 65536)])
def test_batched_matches_oracle_per_join(eiger, oracle_mod, dtype, threads, chunk):
    builds, probes = _mixed_batch(dtype, seed=threads + chunk)
    caps = []
    for b, p in zip(builds, probes):
        caps.append(oracle_mod.join_count(b.cpu().numpy(), p.cpu().numpy()))
    bj = eiger.BatchedJoin(builds, probes, capacities=caps,
                           knobs=eiger.BatchKnobs(threads, chunk, 0.5))
    bj.run()
    torch.cuda.synchronize()
    assert int(bj.status) == 0
    for j in range(len(builds)):
        _check_join(oracle_mod, bj, j, builds[j], probes[j])


def _small_batch(dtype, smax, seed, k=48):
    """Joins around the shared-memory limit of build rows: unique keys with
    probes drawn from them, duplicate-heavy keys, a handful of all-equal build
    rows, and random full-width keys; probe sides of one row to a few chunks."""
    rng = np.random.default_rng(seed)
    lo, hi = (-2**31, 2**31 - 1) if dtype == np.int32 else (-2**62, 2**62)
    builds, probes = [], []
    for j in range(k):
        nb = int(rng.choice([1, 2, 63, 64, 65, 1000, smax - 1, smax, smax + 1]))
        np_ = int(rng.choice([1, 100, 4095, 4096, 4097, 9000]))
        kind = j % 4
        if kind == 0:
            bk = rng.permutation(10 * nb)[:nb] * 7 - 5000
            pk = np.concatenate([bk[rng.integers(0, nb, size=np_ - np_ // 4)], rng.integers(lo, hi, size=np_ // 4)])
        elif kind == 1:
            bk = rng.integers(0, max(1, nb // 8), size=nb)
            pk = rng.integers(0, max(1, nb // 6), size=np_)
        elif kind == 2:
            nb = min(nb, 9)
            bk = np.full(nb, 7)
            pk = np.where(rng.random(np_) < 0.5, 7, rng.integers(8, 100, size=np_))
        else:
            bk = rng.integers(lo, hi, size=nb)
            pk = np.concatenate([bk[rng.integers(0, nb, size=np_ // 2)], rng.integers(lo, hi, size=np_ - np_ // 2)])
        builds.append(torch.from_numpy(np.asarray(bk, dtype=dtype)).cuda())
        probes.append(torch.from_numpy(np.asarray(pk, dtype=dtype)).cuda())
    return builds, probes


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
@pytest.mark.parametrize("small,load", [("max", 0.35), ("max", 0.7), ("none", 0.5)])
def test_batched_small_joins_shared_memory_tables(eiger, oracle_mod, dtype, small, load):
    """Small joins (at most small_rows build rows) run one CTA per 4096-row
    probe chunk with the table in shared memory (at the largest size the
    table is capped, so a 0.35 load factor runs at 0.5); the same joins with
    the path off take global tables. Both agree with the oracle join by join."""
    smax = eiger.BATCH_SMALL_MAX_I32 if dtype == np.int32 else eiger.BATCH_SMALL_MAX_I64
    builds, probes = _small_batch(dtype, smax, seed=31 + int(load * 100))
    caps = [oracle_mod.join_count(b.cpu().numpy(), p.cpu().numpy()) for b, p in zip(builds, probes)]
    knobs = eiger.BatchKnobs(256, 4096, load, smax if small == "max" else 0)
    bj = eiger.BatchedJoin(builds, probes, capacities=caps, knobs=knobs)
    bj.run()
    torch.cuda.synchronize()
    assert int(bj.status) == 0
    for j in range(len(builds)):
        _check_join(oracle_mod, bj, j, builds[j], probes[j])


def test_batched_small_joins_graph_replay(eiger, oracle_mod):
    """A batch of only small joins (64 to 2048 build rows), captured and
    replayed: every replay redoes each join from its own tables."""
    from paper_2607_04489_gb300 import workloads

    w = workloads.batched_small(k=256, log2_lo=6, log2_hi=11, seed=12, device="cuda")
    bj = eiger.BatchedJoin(w.builds, w.probes, knobs=eiger.BatchKnobs(512, 4096, 0.5, eiger.BATCH_SMALL_MAX_I32))
    g = bj.capture()
    for _ in range(2):
        bj.counts.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        assert int(bj.status) == 0
        assert bj.counts.cpu().tolist() == [p.numel() for p in w.probes]
    for j in range(0, 256, 17):
        _check_join(oracle_mod, bj, j, w.builds[j], w.probes[j])


def test_batched_capacity_caps_each_join(eiger, oracle_mod):
    builds, probes = _mixed_batch(np.int32, seed=5, k=24)
    full = [oracle_mod.join_count(b.cpu().numpy(), p.cpu().numpy()) for b, p in zip(builds, probes)]
    caps = [max(0, f // 2) for f in full]
    bj = eiger.BatchedJoin(builds, probes, capacities=caps)
    bj.out_bidx.fill_(-5)
    bj.out_pidx.fill_(-5)
    bj.run()
    torch.cuda.synchronize()
    assert int(bj.status) == 0
    for j in range(len(builds)):
        n, gb, gp = bj.result(j)
        assert n == full[j] and gb.numel() == caps[j]
        # rows written within capacity are genuine matches
        bk, pk = builds[j].cpu().numpy(), probes[j].cpu().numpy()
        b = gb.cpu().numpy().astype(np.int64)
        p = gp.cpu().numpy().astype(np.int64)
        assert np.all(bk[b] == pk[p])


def test_batched_graph_replay_matches_eager(eiger, oracle_mod):
    from paper_2607_04489_gb300 import workloads

    w = workloads.batched_small(k=64, log2_lo=8, log2_hi=15, seed=11, device="cuda")
    bj = eiger.BatchedJoin(w.builds, w.probes)
    g = bj.capture()
    for _ in range(2):
        bj.counts.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        assert int(bj.status) == 0
        for j in range(0, 64, 7):
            _check_join(oracle_mod, bj, j, w.builds[j], w.probes[j])
        assert bj.counts.cpu().tolist() == [p.numel() for p in w.probes]


def test_batched_undersized_workspace_reports_status(eiger):
    b = [torch.arange(5000, dtype=torch.int32, device="cuda")] * 3
    bj = eiger.BatchedJoin(b, b)
    bj.workspace = bj.workspace[: bj.workspace.numel() // 4]
    bj.run()
    torch.cuda.synchronize()
    assert int(bj.status) == eiger.ERR_WORKSPACE
    bj2 = eiger.BatchedJoin(b, b)  # the library stays usable
    bj2.run()
    torch.cuda.synchronize()
    assert int(bj2.status) == 0 and bj2.counts.cpu().tolist() == [5000] * 3


def test_batched_full_workload_4096_joins(eiger, oracle_mod):
    """4096 joins, build sizes 2^U(10,20), probe 4x build, per-join skew."""
    from paper_2607_04489_gb300 import workloads

    free, _ = torch.cuda.mem_get_info()
    if free < (64 << 30):
        pytest.skip("needs 64 GB of free device memory")
    w = workloads.batched_small(seed=0, device="cuda")
    bj = eiger.BatchedJoin(w.builds, w.probes)
    bj.run()
    torch.cuda.synchronize()
    assert int(bj.status) == 0
    assert bj.counts.cpu().tolist() == [p.numel() for p in w.probes]
    rng = np.random.default_rng(1)
    for j in rng.choice(4096, size=12, replace=False):
        _check_join(oracle_mod, bj, int(j), w.builds[j], w.probes[j])
