"""GPU joins vs the CPU oracle, every variant, through the C ABI.

Every case compares the full multiset of (build_idx, probe_idx) pairs after
canonical sorting by (probe, build): bit-exact, no tolerance. Sizes span
several partitioning tiles (4096 rows) with ragged tails; the edge cases cover
empty sides, single rows, all-equal keys (the stage spill path and build
partitions larger than one shared-memory table), int32/int64 extremes, key
spans of exactly 2^32 - 1 (narrowable) and 2^32 (not), and probe keys outside
the build range.
"""

import zlib

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


def _narrowable(bk):
    if bk.size == 0:
        return False
    if bk.dtype == np.int32:
        return True
    return int(bk.max()) - int(bk.min()) <= 0xFFFFFFFF


def _knobs(eiger, variant, bk, **kw):
    if variant in ("auto", "static", "nphj") and not kw:
        return None
    return eiger.Plan(variant, narrow=1 if _narrowable(bk) else 0, **kw)


def _run(eiger, oracle_mod, bk, pk, variant, knobs=None, capacity=None):
    eb, ep, n = oracle_mod.join(bk, pk)
    r = eiger.join(torch.from_numpy(bk).cuda(), torch.from_numpy(pk).cuda(), variant=variant,
                   knobs=knobs, capacity=capacity)
    assert r.count == n, (variant, knobs, r.count, n)
    gb, gp = _canon(r.build_idx.cpu().numpy(), r.probe_idx.cpu().numpy())
    np.testing.assert_array_equal(gp, ep)
    np.testing.assert_array_equal(gb, eb)
    return r


# ------------------------------------------------------------------ inputs

def _unique_perm_i32(rng, nb=5000, np_=70_001):
    return rng.permutation(nb).astype(I32), rng.integers(0, nb, size=np_).astype(I32)


def _dense_i64_zipf(rng, nb=20_000, np_=80_003):
    base = int(rng.integers(-2**40, 2**40))
    bk = (rng.permutation(nb) + base).astype(I64)
    w = 1.0 / np.arange(1, nb + 1) ** 1.5
    rank = rng.choice(nb, size=np_, p=w / w.sum())
    return bk, bk[rng.permutation(nb)[rank]]


def _wide_random_i64(rng, nb=9000, np_=30_000):
    bk = np.unique(rng.integers(-2**63, 2**63 - 1, size=nb, dtype=np.int64))
    rng.shuffle(bk)
    hit = bk[rng.integers(0, bk.size, size=np_ // 2)]
    miss = rng.integers(-2**63, 2**63 - 1, size=np_ - np_ // 2, dtype=np.int64)
    pk = np.concatenate([hit, miss])
    rng.shuffle(pk)
    return bk, pk


def _dup_heavy_i64(rng, nb=3000, np_=5000):
    return rng.integers(-20, 30, size=nb).astype(I64), rng.integers(-25, 35, size=np_).astype(I64)


def _extremes_i64(rng, nb=4500, np_=9000):
    ext = np.array([-2**63, 2**63 - 1, 0, -1, 1, 2**32, -2**32], np.int64)
    bk = np.concatenate([ext, rng.integers(-2**63, 2**63 - 1, size=nb, dtype=np.int64)])
    pk = np.concatenate([ext, ext, bk[rng.integers(0, bk.size, size=np_)]])
    return bk, pk


def _extremes_i32(rng, nb=4500, np_=9000):
    ext = np.array([-2**31, 2**31 - 1, 0, -1, 1], np.int32)
    bk = np.concatenate([ext, rng.integers(-2**31, 2**31 - 1, size=nb).astype(I32)])
    pk = np.concatenate([ext, bk[rng.integers(0, bk.size, size=np_)]])
    return bk, pk


def _span_2_32_minus_1(rng, nb=6000, np_=12_000):
    lo = -2**31 - 7
    hi = lo + 0xFFFFFFFF
    bk = np.concatenate([[lo, hi], rng.integers(lo, hi, size=nb - 2)]).astype(I64)
    pk = np.concatenate([[lo - 1, hi + 1, lo, hi], bk[rng.integers(0, nb, size=np_)]]).astype(I64)
    return bk, pk


def _span_2_32(rng, nb=6000, np_=12_000):
    lo = 12345
    hi = lo + 0x100000000
    bk = np.concatenate([[lo, hi], rng.integers(lo, hi, size=nb - 2)]).astype(I64)
    # keys equal modulo 2^32 but different: must not match
    pk = np.concatenate([[lo + 0x100000000 - 1, hi - 0x100000000, lo, hi],
                         bk[rng.integers(0, nb, size=np_)]]).astype(I64)
    return bk, pk


CASES = {
    "unique_perm_i32": _unique_perm_i32,
    "dense_i64_zipf": _dense_i64_zipf,
    "wide_random_i64": _wide_random_i64,
    "dup_heavy_i64": _dup_heavy_i64,
    "extremes_i64": _extremes_i64,
    "extremes_i32": _extremes_i32,
    "span_2_32_minus_1": _span_2_32_minus_1,
    "span_2_32": _span_2_32,
}

PLANS = [
    ("static", {}),
    ("auto", {}),
    ("nphj", {}),
    ("nphj", {"load_factor": 0.85}),
    ("phj1", {"bits1": 1}),
    ("phj1", {"bits1": 6}),
    ("phj1", {"bits1": 12}),
    ("phj2", {"bits1": 2, "bits2": 3}),
    ("phj2", {"bits1": 7, "bits2": 5}),
    ("phj2", {"bits1": 12, "bits2": 8}),
    ("smj", {}),
    ("smj", {"bits1": 3}),
]


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("variant,kw", PLANS, ids=[f"{v}-{'-'.join(map(str, k.values()))}" for v, k in PLANS])
def test_join_parity(eiger, oracle_mod, case, variant, kw):
    rng = np.random.default_rng(zlib.crc32(case.encode()))
    bk, pk = CASES[case](rng)
    _run(eiger, oracle_mod, bk, pk, variant, _knobs(eiger, variant, bk, **kw))


@pytest.mark.parametrize("variant", ["static", "auto", "nphj", "phj1", "phj2", "smj"])
@pytest.mark.parametrize("nb,np_", [(0, 0), (0, 10), (10, 0), (1, 1), (1, 5000), (4097, 8193),
                                    (4096, 4096)])
def test_join_small_and_empty(eiger, oracle_mod, variant, nb, np_):
    rng = np.random.default_rng(nb * 7 + np_)
    bk = rng.integers(0, 100, size=nb).astype(I64)
    pk = rng.integers(0, 120, size=np_).astype(I64)
    kw = {"bits1": 4} if variant == "phj1" else {"bits1": 3, "bits2": 3} if variant == "phj2" else {}
    _run(eiger, oracle_mod, bk, pk, variant, _knobs(eiger, variant, bk, **kw))


@pytest.mark.parametrize("variant,kw", [("nphj", {}), ("phj1", {"bits1": 3}),
                                        ("phj2", {"bits1": 2, "bits2": 2}), ("static", {}), ("smj", {})])
def test_join_single_key_many_duplicates(eiger, oracle_mod, variant, kw):
    """10,000 equal build keys: one build partition spans three shared-memory
    tables, and every probe row yields 10,000 matches (stage spill path; for
    the sort-merge join a build window of three staged segments and the
    load-balanced expansion)."""
    bk = np.full(10_000, 77, I64)
    pk = np.array([77, 5, 77, 77, 78] * 3, I64)
    _run(eiger, oracle_mod, bk, pk, variant, _knobs(eiger, variant, bk, **kw))


def test_join_probe_outside_build_range(eiger, oracle_mod):
    bk = np.arange(1000, 2000, dtype=I64)
    pk = np.concatenate([np.arange(0, 1000), np.arange(2000, 3000)]).astype(I64)
    for v in ("auto", "phj2", "static", "smj"):
        r = _run(eiger, oracle_mod, bk, pk, v, _knobs(eiger, v, bk, bits1=3, bits2=3) if v == "phj2" else None)
        assert r.count == 0


def test_plan_reports_statistics_and_choice(eiger):
    bk = torch.arange(-500, 1500, dtype=torch.int64, device="cuda")
    pk = torch.arange(0, 4000, dtype=torch.int64, device="cuda")
    r = eiger.join(bk, pk, variant="auto")
    assert r.plan.variant == "nphj" and r.plan.narrow == 1 and r.plan.selector == 0
    assert (r.plan.key_min, r.plan.key_max) == (-500, 1499)
    r = eiger.join(bk, pk, variant="phj2", knobs=eiger.Plan("phj2", 4, 5, 1))
    assert (r.plan.variant, r.plan.bits1, r.plan.bits2, r.plan.selector) == ("phj2", 4, 5, 2)
    r = eiger.join(bk, pk, variant="static")
    assert r.plan.variant == "static" and r.plan.narrow == 0 and r.plan.selector == 3
    assert r.count == 1500


def test_small_static_join_full_size(eiger, oracle_mod):
    """The plain static join of 1M unique int32 build keys with 4M probes, and
    the adaptive join of the same input."""
    from paper_2607_04489_gb300 import workloads

    w = workloads.small_static(device="cpu")
    bk, pk = w.build_keys.numpy(), w.probe_keys.numpy()
    for v in ("static", "auto"):
        r = _run(eiger, oracle_mod, bk, pk, v)
        assert r.count == 1 << 22
    inv = np.empty(bk.size, np.int64)
    inv[bk] = np.arange(bk.size)
    gb, gp = _canon(r.build_idx.cpu().numpy(), r.probe_idx.cpu().numpy())
    np.testing.assert_array_equal(gb, inv[pk].astype(np.uint32))  # closed form


def test_payload_materialisation(eiger, oracle_mod):
    rng = np.random.default_rng(21)
    bk, pk = _dup_heavy_i64(rng, 2000, 3000)
    bp = rng.integers(-2**62, 2**62, size=bk.size).astype(np.int64)
    pp = rng.integers(-2**62, 2**62, size=pk.size).astype(np.int64)
    for v, kn in (("nphj", None), ("phj2", eiger.Plan("phj2", 3, 2, 1)), ("static", None), ("smj", None)):
        r = eiger.join(torch.from_numpy(bk).cuda(), torch.from_numpy(pk).cuda(),
                       build_pay=torch.from_numpy(bp).cuda(), probe_pay=torch.from_numpy(pp).cuda(),
                       variant=v, knobs=kn, payloads=True)
        b = r.build_idx.cpu().numpy().astype(np.int64)
        p = r.probe_idx.cpu().numpy().astype(np.int64)
        np.testing.assert_array_equal(r.build_pay.cpu().numpy(), bp[b])
        np.testing.assert_array_equal(r.probe_pay.cpu().numpy(), pp[p])
        assert r.count == oracle_mod.join_count(bk, pk)


@pytest.mark.parametrize("mat", ["auto", "gfur"])
@pytest.mark.parametrize("variant,kn", [("auto", None), ("nphj", None), ("static", None),
                                        ("phj1", ("phj1", 5, 0, 1)), ("phj2", ("phj2", 4, 4, 1)),
                                        ("smj", None), ("smj", ("smj", 5, 0, 1))])
def test_join_sum_parity(eiger, oracle_mod, variant, kn, mat):
    rng = np.random.default_rng(31)
    n_dim, n_fact = 30_000, 200_000
    dk = (rng.permutation(n_dim) + 1).astype(np.int32)
    dp = rng.integers(0, 10**9, size=n_dim).astype(np.int64)
    fk = rng.integers(1, n_dim + 1, size=n_fact).astype(np.int32)
    fk[rng.random(n_fact) < 0.1] = n_dim + 1 + rng.integers(0, n_dim, size=1)[0]
    fp = rng.integers(0, 10**7, size=n_fact).astype(np.int64)
    s, c = oracle_mod.join_sum(dk, dp, fk, fp)
    knobs = eiger.Plan(*kn) if kn else None
    gs, gc, plan = eiger.join_sum(torch.from_numpy(dk).cuda(), torch.from_numpy(dp).cuda(),
                                  torch.from_numpy(fk).cuda(), torch.from_numpy(fp).cuda(),
                                  variant=variant, knobs=knobs, materialize=mat)
    assert (gs, gc) == (s, c)
    if mat == "gfur" or plan.variant not in ("phj1", "phj2", "smj"):
        assert plan.materialize == "gfur"


@pytest.mark.parametrize("variant,kn", [("phj2", ("phj2", 4, 4, 1)), ("phj1", ("phj1", 6, 0, 1))])
def test_join_sum_auto_materialisation_follows_the_match_estimate(eiger, oracle_mod, variant, kn):
    """AUTO carries the payloads when that moves fewer bytes than gathering
    them (many matches per build row) and gathers them otherwise: 200K
    distinct build keys with 20K probe rows gathers, with 800K probe rows
    carries. Both sums stay exact."""
    rng = np.random.default_rng(33)
    nb = 200_000
    bk = (rng.permutation(nb) * 3 + 11).astype(np.int32)
    bp = rng.integers(-2**40, 2**40, size=nb).astype(np.int64)
    for npr, want in ((20_000, "gfur"), (800_000, "gftr")):
        pk = bk[rng.integers(0, nb, size=npr)]
        pp = rng.integers(-2**40, 2**40, size=npr).astype(np.int64)
        s, c = oracle_mod.join_sum(bk, bp, pk, pp)
        gs, gc, plan = eiger.join_sum(torch.from_numpy(bk).cuda(), torch.from_numpy(bp).cuda(),
                                      torch.from_numpy(pk).cuda(), torch.from_numpy(pp).cuda(),
                                      variant=variant, knobs=eiger.Plan(*kn))
        assert (gs, gc) == (s, c)
        assert plan.materialize == want, (npr, plan)


@pytest.mark.parametrize("pay", [np.int32, np.int64])
@pytest.mark.parametrize("mat", ["gftr", "gfur"])
@pytest.mark.parametrize("kn", [("phj1", 1, 0, 0), ("phj2", 1, 1, 1), ("phj2", 3, 3, 0), ("smj", 6, 0, 1)])
def test_join_sum_duplicates_carried_and_gathered(eiger, oracle_mod, kn, mat, pay):
    """Duplicate-heavy int64 keys (2000 build rows per key, so the general
    probe path runs and 1-bit partitions hold several build chunks), 4- and
    8-byte payloads spanning the full range so the sum wraps: carrying the
    payloads (GFTR) and gathering them by tuple ID (GFUR) give the oracle's
    sum and count."""
    rng = np.random.default_rng(32)
    bk = rng.integers(0, 10, size=20_000).astype(I64) * 1_000_003 - 7
    pk = rng.integers(-2, 12, size=30_000).astype(I64) * 1_000_003 - 7
    info = np.iinfo(pay)
    bp = rng.integers(info.min, info.max, size=bk.size, dtype=np.int64).astype(pay)
    pp = rng.integers(info.min, info.max, size=pk.size, dtype=np.int64).astype(pay)
    s, c = oracle_mod.join_sum(bk, bp, pk, pp)
    gs, gc, plan = eiger.join_sum(torch.from_numpy(bk).cuda(), torch.from_numpy(bp).cuda(),
                                  torch.from_numpy(pk).cuda(), torch.from_numpy(pp).cuda(),
                                  variant=kn[0], knobs=eiger.Plan(*kn), materialize=mat)
    assert (gs, gc) == (s, c)
    assert plan.materialize == mat


def test_join_sum_gftr_rejected_without_partitioning(eiger):
    k = torch.arange(100, dtype=torch.int32, device="cuda")
    with pytest.raises(eiger.EigerError, match="GFTR"):
        eiger.join_sum(k, k.long(), k, k.long(), variant="nphj", materialize="gftr")


def test_capacity_errors_and_retry(eiger, oracle_mod):
    rng = np.random.default_rng(5)
    bk, pk = _dup_heavy_i64(rng, 500, 800)
    n = oracle_mod.join_count(bk, pk)
    dbk, dpk = torch.from_numpy(bk).cuda(), torch.from_numpy(pk).cuda()
    ws = torch.empty(eiger.join_workspace(bk.size, pk.size, eiger.I64), dtype=torch.uint8, device="cuda")
    cap = n // 3
    guard = 16
    ob = torch.full((cap + guard,), -7, dtype=torch.int32, device="cuda")
    op = torch.full((cap + guard,), -7, dtype=torch.int32, device="cuda")
    st, cnt, _ = eiger.join_into(dbk, dpk, out_bidx=ob, out_pidx=op, capacity=cap, workspace=ws)
    assert st == eiger.ERR_CAPACITY and cnt == n
    assert bool((ob[cap:] == -7).all()) and bool((op[cap:] == -7).all())  # nothing past capacity
    st, cnt, _ = eiger.join_into(dbk, dpk, capacity=0, workspace=ws)  # count-only query
    assert st == eiger.ERR_CAPACITY and cnt == n
    r = eiger.join(dbk, dpk, capacity=1)  # retries with the exact size
    assert r.count == n and r.build_idx.numel() == n


def test_workspace_too_small_and_bad_knobs_leave_library_usable(eiger, oracle_mod):
    bk = torch.arange(0, 3000, dtype=torch.int64, device="cuda")
    pk = torch.arange(0, 9000, dtype=torch.int64, device="cuda") % 3000
    tiny = torch.empty(1024, dtype=torch.uint8, device="cuda")
    st, _, _ = eiger.join_into(bk, pk, capacity=0, workspace=tiny)
    assert st == eiger.ERR_WORKSPACE
    wide = torch.tensor([0, 2**40], dtype=torch.int64, device="cuda")
    with pytest.raises(eiger.EigerError) as ei:
        eiger.join(wide, wide, variant="phj1", knobs=eiger.Plan("phj1", 3, 0, 1))
    assert ei.value.status == eiger.ERR_INVALID_ARG
    with pytest.raises(eiger.EigerError):
        eiger.join(bk, pk, variant="phj2", knobs=eiger.Plan("phj2", 13, 1, 1))
    with pytest.raises(eiger.EigerError):
        eiger.join(bk, pk, variant="nphj", knobs=eiger.Plan("nphj", load_factor=0.95, narrow=1))
    r = eiger.join(bk, pk)
    assert r.count == 9000


def test_table_full_is_reported_not_faulted(eiger, monkeypatch):
    """Host-injected undersized table: bounded probe loops set the device error
    flag, the call returns EIGER_ERR_TABLE_FULL, and the next call works."""
    bk = torch.arange(0, 500, dtype=torch.int64, device="cuda")
    monkeypatch.setenv("EIGER_FAULT", "table_full")
    with pytest.raises(eiger.EigerError) as ei:
        eiger.join(bk, bk, variant="nphj")
    assert ei.value.status == eiger.ERR_TABLE_FULL
    monkeypatch.delenv("EIGER_FAULT")
    assert eiger.join(bk, bk, variant="nphj").count == 500


def test_host_buffers_end_to_end(eiger, oracle_mod):
    rng = np.random.default_rng(8)
    bk, pk = _unique_perm_i32(rng, 3000, 9000)
    r = eiger.join(torch.from_numpy(bk).pin_memory(), torch.from_numpy(pk).pin_memory(), to_host=True)
    assert not r.build_idx.is_cuda
    eb, ep, n = oracle_mod.join(bk, pk)
    gb, gp = _canon(r.build_idx.numpy(), r.probe_idx.numpy())
    assert r.count == n
    np.testing.assert_array_equal(gb, eb)
    np.testing.assert_array_equal(gp, ep)


@pytest.mark.parametrize("keys", ["dense", "random"])
def test_variant_sweep_parity_moderate(eiger, oracle_mod, keys):
    """The benchmark's workload generator at 2^18 x 4, every variant."""
    from paper_2607_04489_gb300 import workloads

    w = workloads.variant_sweep(1 << 18, 4, keys=keys, theta=1.0, seed=3, device="cpu")
    bk, pk = w.build_keys.numpy(), w.probe_keys.numpy()
    for v, kw in (("auto", {}), ("static", {}), ("phj1", {"bits1": 7}), ("phj2", {"bits1": 4, "bits2": 3})):
        _run(eiger, oracle_mod, bk, pk, v, _knobs(eiger, v, bk, **kw))


def test_headline_join_full_size(eiger):
    """The benchmark's call at full size: AUTO on 2^26 dense int64 build keys and
    2^28 uniform probes. Build keys are unique and every probe key is drawn
    from them, so the result is exactly one pair per probe row whose keys are
    equal; checked for every pair on the device."""
    from paper_2607_04489_gb300 import workloads

    free, _ = torch.cuda.mem_get_info()
    if free < (24 << 30):
        pytest.skip("needs 24 GB of free device memory")
    w = workloads.variant_sweep(1 << 26, 4, keys="dense", theta=0.0, seed=0, device="cuda")
    r = eiger.join(w.build_keys, w.probe_keys, variant="auto")
    assert r.plan.variant in ("phj1", "phj2") and r.plan.narrow == 1
    assert r.count == w.np
    p = r.probe_idx.long()
    b = r.build_idx.long()
    assert int(torch.bincount(p, minlength=w.np).max()) == 1
    assert bool((w.build_keys[b] == w.probe_keys[p]).all())
