"""The partitioned join's index-pair output through per-warp output runs.

Each warp of the join reserves runs of consecutive output positions and
fills them in order; afterwards the pairs stored at or above the match count
move into the holes left below it, and positions at or above the caller's
capacity go to workspace overflow, never to the caller's arrays. These cases
drive that path at its edges and compare every pair with the oracle after the
canonical sort: capacity exactly the count (overflow used), capacity with
spare room (scratch written below capacity, nothing past it), capacity below
the count (count reported, nothing past capacity), no matches at all, a
single match, duplicate-heavy keys (many matches per lane across run
boundaries), and repeated calls on one workspace.
"""

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

I32, I64 = np.int32, np.int64


@pytest.fixture(scope="module")
def eiger():
    from paper_2607_04489_gb300 import eiger

    eiger.load()
    return eiger


def _canon(b, p):
    b = np.asarray(b).astype(np.int64) & 0xFFFFFFFF
    p = np.asarray(p).astype(np.int64) & 0xFFFFFFFF
    order = np.lexsort((b, p))
    return b[order].astype(np.uint32), p[order].astype(np.uint32)


PLANS = [("phj1", 6, 0), ("phj2", 4, 5)]


def _call(eiger, bk, pk, plan, cap, guard=64, ws=None):
    dbk, dpk = torch.from_numpy(bk).cuda(), torch.from_numpy(pk).cuda()
    knobs = eiger.Plan(plan[0], plan[1], plan[2], 1)
    if ws is None:
        ws = torch.empty(eiger.join_workspace(bk.size, pk.size, eiger.I64 if bk.dtype == I64 else eiger.I32,
                                              plan[0], knobs), dtype=torch.uint8, device="cuda")
    ob = torch.full((cap + guard,), -7, dtype=torch.int32, device="cuda")
    op = torch.full((cap + guard,), -7, dtype=torch.int32, device="cuda")
    st, cnt, used = eiger.join_into(dbk, dpk, variant=plan[0], knobs=knobs, out_bidx=ob, out_pidx=op,
                                    capacity=cap, workspace=ws)
    torch.cuda.synchronize()
    assert (used.variant, used.bits1) == (plan[0], plan[1])
    # nothing is ever written past the capacity
    assert bool((ob[cap:] == -7).all()) and bool((op[cap:] == -7).all())
    return st, cnt, ob, op


def _unique(rng, nb, np_):
    bk = (rng.permutation(nb) + 1000).astype(I64)
    return bk, bk[rng.integers(0, nb, size=np_)]


@pytest.mark.parametrize("plan", PLANS)
@pytest.mark.parametrize("slack", [0, 1, 777, 1 << 20])
def test_capacity_at_and_above_count(eiger, oracle_mod, plan, slack):
    """Unique build keys, 300K probe rows over many warps' runs: with the
    capacity exactly the count the last runs land in the overflow area; with
    spare room they land in the caller's array below the capacity."""
    rng = np.random.default_rng(41 + slack)
    bk, pk = _unique(rng, 60_000, 300_001)
    eb, ep, n = oracle_mod.join(bk, pk)
    st, cnt, ob, op = _call(eiger, bk, pk, plan, n + slack)
    assert st == eiger.OK and cnt == n
    gb, gp = _canon(ob[:n].cpu().numpy(), op[:n].cpu().numpy())
    np.testing.assert_array_equal(gp, ep)
    np.testing.assert_array_equal(gb, eb)


@pytest.mark.parametrize("plan", PLANS)
@pytest.mark.parametrize("frac", [0.0, 0.5, 0.999])
def test_capacity_below_count(eiger, oracle_mod, plan, frac):
    rng = np.random.default_rng(7)
    bk, pk = _unique(rng, 30_000, 100_000)
    n = oracle_mod.join_count(bk, pk)
    cap = int(n * frac)
    st, cnt, _, _ = _call(eiger, bk, pk, plan, cap)
    assert st == eiger.ERR_CAPACITY and cnt == n


@pytest.mark.parametrize("plan", PLANS)
def test_no_match_and_single_match(eiger, oracle_mod, plan):
    bk = np.arange(0, 50_000, dtype=I64) * 2
    pk = np.arange(0, 70_000, dtype=I64) * 2 + 1  # odd: never in the build side
    st, cnt, _, _ = _call(eiger, bk, pk, plan, 16)
    assert st == eiger.OK and cnt == 0
    pk[12_345] = 400  # build row 200
    st, cnt, ob, op = _call(eiger, bk, pk, plan, 1)
    assert st == eiger.OK and cnt == 1
    assert (int(ob[0]), int(op[0])) == (200, 12_345)


@pytest.mark.parametrize("plan", PLANS)
def test_duplicate_keys_cross_run_boundaries(eiger, oracle_mod, plan):
    """Build keys repeat (about 40 rows per key), so one probe row matches
    tens of build rows and a warp fills several runs in one probe step."""
    rng = np.random.default_rng(19)
    bk = rng.integers(0, 1500, size=60_000).astype(I32)
    pk = rng.integers(-10, 1600, size=20_000).astype(I32)
    eb, ep, n = oracle_mod.join(bk, pk)
    st, cnt, ob, op = _call(eiger, bk, pk, plan, n)
    assert st == eiger.OK and cnt == n
    gb, gp = _canon(ob[:n].cpu().numpy(), op[:n].cpu().numpy())
    np.testing.assert_array_equal(gp, ep)
    np.testing.assert_array_equal(gb, eb)


def test_repeated_calls_share_a_workspace(eiger, oracle_mod):
    """The warp records and overflow of one call do not leak into the next:
    a large join, then a small one, then the large one again, on one
    workspace."""
    rng = np.random.default_rng(23)
    big = _unique(rng, 100_000, 400_000)
    small = _unique(rng, 3_000, 5_000)
    plan = ("phj2", 5, 5)
    knobs = eiger.Plan(plan[0], plan[1], plan[2], 1)
    ws = torch.empty(eiger.join_workspace(big[0].size, big[1].size, eiger.I64, plan[0], knobs),
                     dtype=torch.uint8, device="cuda")
    for bk, pk in (big, small, big):
        eb, ep, n = oracle_mod.join(bk, pk)
        st, cnt, ob, op = _call(eiger, bk, pk, plan, n, ws=ws)
        assert st == eiger.OK and cnt == n
        gb, gp = _canon(ob[:n].cpu().numpy(), op[:n].cpu().numpy())
        np.testing.assert_array_equal(gp, ep)
        np.testing.assert_array_equal(gb, eb)
