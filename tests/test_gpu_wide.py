"""Wide joins (several payload columns per side) and the sort-merge join vs the
CPU oracle, through the C ABI.

Every case materialises the tuple IDs together with the columns, sorts the
matches canonically by (probe, build) and compares every column bit for bit
with the oracle's wide join. Both materialisation strategies (gather by tuple
ID from the caller's columns, GFUR; gather by position from the partitioned or
sorted copies, GFTR) must give the same result for every variant that allows
them.
"""

import zlib

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eiger():
    from paper_2607_04489_gb300 import eiger

    eiger.load()
    return eiger


def _narrowable(bk):
    return bk.size > 0 and (bk.dtype == np.int32 or int(bk.max()) - int(bk.min()) <= 0xFFFFFFFF)


def _columns(rng, n, kinds):
    out = []
    for k in kinds:
        if k == 4:
            out.append(rng.integers(-2**31, 2**31, size=n).astype(np.int32))
        else:
            out.append(rng.integers(-2**63, 2**63 - 1, size=n, dtype=np.int64))
    return out


def _check(eiger, oracle_mod, bk, pk, bcols, pcols, variant, mat, knobs=None, indices=True):
    eb, ep, ebc, epc = oracle_mod.join_wide(bk, pk, bcols, pcols)
    r = eiger.join_wide(torch.from_numpy(bk).cuda(), torch.from_numpy(pk).cuda(),
                        [torch.from_numpy(c).cuda() for c in bcols], [torch.from_numpy(c).cuda() for c in pcols],
                        variant=variant, materialize=mat, knobs=knobs, indices=indices)
    assert r.count == eb.size
    if indices:
        b = r.build_idx.cpu().numpy().astype(np.int64) & 0xFFFFFFFF
        p = r.probe_idx.cpu().numpy().astype(np.int64) & 0xFFFFFFFF
        o = np.lexsort((b, p))
        np.testing.assert_array_equal(b[o], eb.astype(np.int64))
        np.testing.assert_array_equal(p[o], ep.astype(np.int64))
        for got, want in zip(r.build_cols, ebc):
            np.testing.assert_array_equal(got.cpu().numpy()[o], want)
        for got, want in zip(r.probe_cols, epc):
            np.testing.assert_array_equal(got.cpu().numpy()[o], want)
    return r


def _dense_zipf(rng, dtype, nb=20_000, np_=70_001):
    base = 0 if dtype == np.int32 else int(rng.integers(-2**40, 2**40))
    bk = (rng.permutation(nb) + base).astype(dtype)
    w = 1.0 / np.arange(1, nb + 1) ** 1.2
    rank = rng.choice(nb, size=np_, p=w / w.sum())
    pk = bk[rng.permutation(nb)[rank]]
    return bk, pk


def _dups(rng, dtype, nb=6000, np_=9001):
    return rng.integers(-40, 40, size=nb).astype(dtype), rng.integers(-50, 50, size=np_).astype(dtype)


def _spread_i64(rng, nb=9000, np_=30_000):
    bk = np.unique(rng.integers(-2**63, 2**63 - 1, size=nb, dtype=np.int64))
    rng.shuffle(bk)
    pk = np.concatenate([bk[rng.integers(0, bk.size, size=np_ // 2)],
                         rng.integers(-2**63, 2**63 - 1, size=np_ - np_ // 2, dtype=np.int64)])
    rng.shuffle(pk)
    return bk, pk


INPUTS = {
    "dense_zipf_i32": lambda rng: _dense_zipf(rng, np.int32),
    "dense_zipf_i64": lambda rng: _dense_zipf(rng, np.int64),
    "dups_i32": lambda rng: _dups(rng, np.int32),
    "dups_i64": lambda rng: _dups(rng, np.int64),
    "spread_i64": _spread_i64,
}

PLANS = [
    ("nphj", "gfur", None),
    ("static", "gfur", None),
    ("phj1", "gfur", (6, 0)),
    ("phj1", "gftr", (6, 0)),
    ("phj2", "gfur", (4, 5)),
    ("phj2", "gftr", (4, 5)),
    ("smj", "gfur", None),
    ("smj", "gftr", None),
    ("smj", "gftr", (4, 0)),
    ("auto", "auto", None),
]


@pytest.mark.parametrize("case", sorted(INPUTS))
@pytest.mark.parametrize("variant,mat,bits", PLANS, ids=[f"{v}-{m}-{b}" for v, m, b in PLANS])
def test_wide_join_parity(eiger, oracle_mod, case, variant, mat, bits):
    rng = np.random.default_rng(zlib.crc32(case.encode()))
    bk, pk = INPUTS[case](rng)
    bcols = _columns(rng, bk.size, (8, 4, 8))
    pcols = _columns(rng, pk.size, (4, 8, 4, 8))
    knobs = None
    if bits is not None:
        knobs = eiger.Plan(variant, bits[0], bits[1], 1 if _narrowable(bk) else 0)
    r = _check(eiger, oracle_mod, bk, pk, bcols, pcols, variant, mat, knobs)
    if variant in ("phj1", "phj2", "smj"):
        assert r.plan.materialize == mat
    if variant == "auto" and r.plan.variant not in ("phj1", "phj2", "smj"):
        assert r.plan.materialize == "gfur"


@pytest.mark.parametrize("variant,mat", [("phj2", "gftr"), ("smj", "gftr"), ("nphj", "gfur")])
def test_wide_join_columns_without_indices(eiger, oracle_mod, variant, mat):
    """Columns only: a probe column holding the row number and a build column
    holding the row number identify each match, the others must follow."""
    rng = np.random.default_rng(11)
    bk, pk = _dups(rng, np.int64, 3000, 5000)
    bcols = [np.arange(bk.size, dtype=np.int32)] + _columns(rng, bk.size, (8,))
    pcols = [np.arange(pk.size, dtype=np.int64)] + _columns(rng, pk.size, (4,))
    knobs = eiger.Plan("phj2", 3, 3, 1) if variant == "phj2" else None
    eb, ep, ebc, epc = oracle_mod.join_wide(bk, pk, bcols, pcols)
    r = eiger.join_wide(torch.from_numpy(bk).cuda(), torch.from_numpy(pk).cuda(),
                        [torch.from_numpy(c).cuda() for c in bcols], [torch.from_numpy(c).cuda() for c in pcols],
                        variant=variant, materialize=mat, knobs=knobs, indices=False)
    assert r.build_idx is None and r.count == eb.size
    b = r.build_cols[0].cpu().numpy().astype(np.int64)
    p = r.probe_cols[0].cpu().numpy()
    o = np.lexsort((b, p))
    np.testing.assert_array_equal(b[o], eb.astype(np.int64))
    np.testing.assert_array_equal(p[o], ep.astype(np.int64))
    np.testing.assert_array_equal(r.build_cols[1].cpu().numpy()[o], ebc[1])
    np.testing.assert_array_equal(r.probe_cols[1].cpu().numpy()[o], epc[1])


def test_gftr_needs_a_transformed_plan(eiger):
    bk = torch.arange(100, dtype=torch.int64, device="cuda")
    col = torch.arange(100, dtype=torch.int64, device="cuda")
    with pytest.raises(eiger.EigerError) as e:
        eiger.join_wide(bk, bk, [col], [col], variant="nphj", materialize="gftr")
    assert e.value.status == eiger.ERR_INVALID_ARG


def test_wide_join_one_side_columns_and_capacity(eiger, oracle_mod):
    """Columns on the probe side only; a first call with too small a capacity
    reports |J| and writes nothing past it."""
    rng = np.random.default_rng(12)
    bk, pk = _dups(rng, np.int32, 800, 1200)
    pcols = _columns(rng, pk.size, (8, 4))
    n = oracle_mod.join_count(bk, pk)
    dbk, dpk = torch.from_numpy(bk).cuda(), torch.from_numpy(pk).cuda()
    dpc = [torch.from_numpy(c).cuda() for c in pcols]
    for variant, mat in (("phj1", "gftr"), ("smj", "gftr"), ("smj", "gfur")):
        knobs = eiger.Plan("phj1", 4, 0, 1) if variant == "phj1" else None
        ws = torch.empty(eiger.join_wide_workspace(bk.size, pk.size, eiger.I32, [], dpc, variant, mat, knobs),
                         dtype=torch.uint8, device="cuda")
        cap = n // 2
        outs = [torch.full((cap + 8,), -3, dtype=c.dtype, device="cuda") for c in dpc]
        st, cnt, _ = eiger.join_wide_into(dbk, dpk, [], dpc, [], outs, variant=variant, materialize=mat,
                                          knobs=knobs, capacity=cap, workspace=ws)
        assert st == eiger.ERR_CAPACITY and cnt == n
        assert all(bool((o[cap:] == -3).all()) for o in outs)
        _check(eiger, oracle_mod, bk, pk, [], pcols, variant, mat, knobs)


@pytest.mark.parametrize("dtype,span", [(np.int32, 1 << 12), (np.int32, 1 << 31), (np.int64, 1 << 40),
                                        (np.int64, 1 << 62)])
def test_smj_sort_passes_follow_the_key_span(eiger, oracle_mod, dtype, span):
    """The sort orders only the build span's significant bits: ceil(bits / 8)
    passes with the bits spread evenly; the result is exact either way."""
    rng = np.random.default_rng(span % 1000 + 3)
    lo = -(span // 2)
    bk = np.concatenate([[lo, lo + span - 1], rng.integers(lo, lo + span, size=7000)]).astype(dtype)
    pk = bk[rng.integers(0, bk.size, size=20_000)]
    bits = int(span - 1).bit_length()
    r = _check(eiger, oracle_mod, bk, pk, [], [], "smj", "gfur")
    passes = (bits + 7) // 8
    assert (r.plan.variant, r.plan.bits2, r.plan.bits1) == ("smj", passes, (bits + passes - 1) // passes)


def test_smj_headline_shape_moderate(eiger, oracle_mod):
    """2^20 unique dense int64 build keys, 2^22 uniform probes: every probe
    row matches exactly its build row (closed form), through the sort-merge
    join, with one payload column per side carried through the sort."""
    from paper_2607_04489_gb300 import workloads

    w = workloads.variant_sweep(1 << 20, 4, keys="dense", seed=3)
    bk, pk = w.build_keys.numpy(), w.probe_keys.numpy()
    r = eiger.join_wide(w.build_keys.cuda(), w.probe_keys.cuda(), [w.build_pay.cuda()], [w.probe_pay.cuda()],
                        variant="smj", materialize="gftr")
    assert r.count == pk.size
    b = r.build_idx.cpu().numpy().astype(np.int64)
    p = r.probe_idx.cpu().numpy().astype(np.int64)
    assert np.array_equal(np.sort(p), np.arange(pk.size))
    np.testing.assert_array_equal(bk[b], pk[p])  # every pair joins equal keys
    np.testing.assert_array_equal(r.build_cols[0].cpu().numpy(), w.build_pay.numpy()[b])
    np.testing.assert_array_equal(r.probe_cols[0].cpu().numpy(), w.probe_pay.numpy()[p])
