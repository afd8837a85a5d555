"""The join entry point that allocates nothing (eiger_join_static_noalloc).

Some callers cannot allocate device memory where they join: a component whose
device memory all belongs to another pool, or a plug-in host that forbids
allocation on its execution path. eiger_join_static_noalloc serves them: it
runs the static non-partitioned join with its hash table and control block in
the library's own fixed device array. These tests call it through the C ABI and
check that two calls in a row each give exactly the pairs the regular
eiger_join(EIGER_STATIC) gives on the same inputs (bit-exact after sorting, the
tolerance of every join test here), so nothing leaks from one call to the next
through the shared array. This file is collected last on purpose.
"""

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _canon(b, p):
    b = b.cpu().numpy().astype(np.int64) & 0xFFFFFFFF
    p = p.cpu().numpy().astype(np.int64) & 0xFFFFFFFF
    order = np.lexsort((b, p))
    return b[order], p[order]


def _compare(eiger, bk, pk):
    ref = eiger.join(bk, pk, variant="static")
    cap = max(ref.count, 1)
    ob = torch.full((cap + 8,), -1, dtype=torch.int32, device="cuda")
    op = torch.full((cap + 8,), -1, dtype=torch.int32, device="cuda")
    st, n = eiger.join_static_noalloc_into(bk, pk, ob, op, cap)
    assert st == eiger.OK, eiger.last_error()
    assert n == ref.count
    gb, gp = _canon(ob[:n], op[:n])
    rb, rp = _canon(ref.build_idx, ref.probe_idx)
    np.testing.assert_array_equal(gb, rb)
    np.testing.assert_array_equal(gp, rp)
    assert bool((ob[cap:] == -1).all())  # nothing written past capacity


def test_noalloc_matches_static_join_on_two_calls_in_a_row():
    from paper_2607_04489_gb300 import eiger

    eiger.load()
    rng = np.random.default_rng(2026)
    # call 1: int32 keys with duplicates, a build side near the int32 limit
    bk1 = torch.from_numpy(rng.integers(0, 200_000, size=400_000).astype(np.int32)).cuda()
    pk1 = torch.from_numpy(rng.integers(0, 250_000, size=1_000_003).astype(np.int32)).cuda()
    _compare(eiger, bk1, pk1)
    # call 2: different int64 keys; a stale table from call 1 would add matches
    bk2 = torch.from_numpy((rng.permutation(150_000) - 75_000).astype(np.int64)).cuda()
    pk2 = torch.from_numpy(rng.integers(-100_000, 100_000, size=600_001).astype(np.int64)).cuda()
    _compare(eiger, bk2, pk2)


def test_noalloc_rejects_build_sides_beyond_its_limit():
    from paper_2607_04489_gb300 import eiger

    eiger.load()
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
    _compare(eiger, edge, probe)
