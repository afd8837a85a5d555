"""The join entry point that allocates nothing (eiger_join_static_noalloc).

Some callers cannot allocate device memory where they join: a component whose
device memory all belongs to another pool, or a plug-in host that forbids
allocation on its execution path. eiger_join_static_noalloc serves them: it
runs the static non-partitioned join with its hash table and control block in
the library's own fixed device array. These tests call it through the C ABI and
check that two calls in a row each give exactly the pairs of the CPU oracle's
join and of the regular eiger_join(EIGER_STATIC) on the same inputs (bit-exact
after the canonical sort, the tolerance of every join test here), so nothing
leaks from one call to the next through the shared array. They also cover an
undersized capacity (EIGER_ERR_CAPACITY with the full count, nothing written
past the capacity) and the count-only call. This file is collected last on
purpose.
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
    order = np.lexsort((b, p))
    return b[order].astype(np.uint32), p[order].astype(np.uint32)


def _compare(eiger, oracle_mod, bk, pk):
    eb, ep, n_oracle = oracle_mod.join(bk.cpu().numpy(), pk.cpu().numpy())
    ref = eiger.join(bk, pk, variant="static")
    assert ref.count == n_oracle
    cap = max(n_oracle, 1)
    ob = torch.full((cap + 8,), -1, dtype=torch.int32, device="cuda")
    op = torch.full((cap + 8,), -1, dtype=torch.int32, device="cuda")
    st, n = eiger.join_static_noalloc_into(bk, pk, ob, op, cap)
    assert st == eiger.OK, eiger.last_error()
    assert n == n_oracle
    gb, gp = _canon(ob[:n], op[:n])
    np.testing.assert_array_equal(gb, eb)
    np.testing.assert_array_equal(gp, ep)
    rb, rp = _canon(ref.build_idx, ref.probe_idx)
    np.testing.assert_array_equal(gb, rb)
    np.testing.assert_array_equal(gp, rp)
    assert bool((ob[cap:] == -1).all()) and bool((op[cap:] == -1).all())  # nothing past capacity


def test_noalloc_matches_oracle_on_two_calls_in_a_row(eiger, oracle_mod):
    rng = np.random.default_rng(2026)
    # call 1: int32 keys with duplicates, a build side near the int32 limit
    bk1 = torch.from_numpy(rng.integers(0, 200_000, size=400_000).astype(np.int32)).cuda()
    pk1 = torch.from_numpy(rng.integers(0, 250_000, size=1_000_003).astype(np.int32)).cuda()
    _compare(eiger, oracle_mod, bk1, pk1)
    # call 2: different int64 keys; a stale table from call 1 would add matches
    bk2 = torch.from_numpy((rng.permutation(150_000) - 75_000).astype(np.int64)).cuda()
    pk2 = torch.from_numpy(rng.integers(-100_000, 100_000, size=600_001).astype(np.int64)).cuda()
    _compare(eiger, oracle_mod, bk2, pk2)


def test_noalloc_capacity_and_count_only(eiger, oracle_mod):
    rng = np.random.default_rng(7)
    bk = torch.from_numpy(rng.integers(0, 5000, size=20_000).astype(np.int32)).cuda()
    pk = torch.from_numpy(rng.integers(0, 6000, size=50_001).astype(np.int32)).cuda()
    total = oracle_mod.join_count(bk.cpu().numpy(), pk.cpu().numpy())
    assert total > 1000
    # undersized capacity: the status says so, the count is |J|, and no entry
    # at or past the capacity is written
    half = total // 2
    ob = torch.full((total + 8,), -7, dtype=torch.int32, device="cuda")
    op = torch.full((total + 8,), -7, dtype=torch.int32, device="cuda")
    st, n = eiger.join_static_noalloc_into(bk, pk, ob, op, half)
    assert st == eiger.ERR_CAPACITY and n == total
    assert bool((ob[half:] == -7).all()) and bool((op[half:] == -7).all())
    # count only: capacity 0 and no output arrays
    st, n = eiger.join_static_noalloc_into(bk, pk, None, None, 0)
    assert st == eiger.ERR_CAPACITY and n == total
    # the shared array does not leak into the next full call
    _compare(eiger, oracle_mod, bk, pk)


def test_noalloc_rejects_bad_arguments_on_the_host(eiger):
    k32 = torch.zeros(4, dtype=torch.int32, device="cuda")
    out = torch.empty(16, dtype=torch.int32, device="cuda")
    with pytest.raises(TypeError):
        eiger.join_static_noalloc_into(k32.long(), k32, out, out, 16)  # dtypes differ
    with pytest.raises(TypeError):
        eiger.join_static_noalloc_into(k32.cpu(), k32, out, out, 16)  # host tensor
    with pytest.raises(ValueError):
        eiger.join_static_noalloc_into(k32, k32, out, out, 17)  # outputs too short
    with pytest.raises(TypeError):
        eiger.join_static_noalloc_into(k32, k32, out.long(), out, 16)  # output dtype


def test_noalloc_rejects_build_sides_beyond_its_limit(eiger, oracle_mod):
    big = torch.zeros((1 << 19) + 1, dtype=torch.int32, device="cuda")
    small = torch.zeros(4, dtype=torch.int32, device="cuda")
    out = torch.empty(16, dtype=torch.int32, device="cuda")
    st, _ = eiger.join_static_noalloc_into(big, small, out, out, 16)
    assert st == eiger.ERR_INVALID_ARG and "2^19" in eiger.last_error()
    big64 = torch.zeros((1 << 18) + 1, dtype=torch.int64, device="cuda")
    st, _ = eiger.join_static_noalloc_into(big64, small.long(), out, out, 16)
    assert st == eiger.ERR_INVALID_ARG and "2^18" in eiger.last_error()
    # the largest accepted build side still joins correctly
    edge = torch.arange(1 << 19, dtype=torch.int32, device="cuda")
    probe = torch.arange(0, 1 << 20, 3, dtype=torch.int32, device="cuda")
    _compare(eiger, oracle_mod, edge, probe)
