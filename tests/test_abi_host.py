"""Host-side checks of the C ABI: no GPU needed, no kernel launched.

The library must load, export every function include/eiger.h declares, and
answer its host-only calls (workspace queries, the rule-based planner,
argument validation and error reporting) without touching a device.
"""

import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "eiger.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2607_04489_gb300 import eiger

    if not os.path.exists(eiger.LIB_PATH):
        from paper_2607_04489_gb300.build import build_library

        build_library()
    return eiger


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(eiger_[a-z_]+)\s*\(", src,
                                 flags=re.M)))


def test_header_declares_the_abi():
    names = _declared_functions()
    assert "eiger_join" in names and "eiger_stats" in names and len(names) >= 8


def test_library_exports_every_declared_symbol(lib):
    so = ctypes.CDLL(lib.LIB_PATH)
    for name in _declared_functions():
        assert hasattr(so, name), f"{name} declared in eiger.h but not exported"
    assert set(_declared_functions()) == set(lib.SYMBOLS)


def test_version_string(lib):
    assert "sm_103a" in lib.version()


def _stats(n, mn, mx, est=None):
    from paper_2607_04489_gb300.eiger import Stats

    return Stats(n, mn, mx, float(n if est is None else est), np.zeros(16384, np.uint8))


def test_planner_small_build_uses_the_non_partitioned_join(lib):
    p = lib.plan(_stats(1 << 20, 0, (1 << 20) - 1), None, 1 << 20, 1 << 22, lib.I32)
    assert p.variant == "nphj" and p.narrow == 1 and p.load_factor == pytest.approx(0.5)


def test_planner_large_build_partitions_in_two_passes(lib):
    p = lib.plan(_stats(1 << 26, -5, (1 << 26) - 6), None, 1 << 26, 1 << 28, lib.I64)
    assert p.variant == "phj2" and p.narrow == 1
    assert p.bits1 + p.bits2 == 15 and abs(p.bits1 - p.bits2) <= 1


def test_planner_distinct_build_keys_get_larger_partitions(lib):
    """All-distinct build keys (HyperLogLog estimate >= 0.9 x rows) aim at up
    to 3072 rows per partition (4096 from 2^27 rows up), duplicate-heavy ones
    at up to 2048."""
    nb = 150_000_000
    uniq = lib.plan(_stats(nb, 1, nb), None, nb, 4 * nb, lib.I32)
    dups = lib.plan(_stats(nb, 1, nb, est=nb / 10), None, nb, 4 * nb, lib.I32)
    assert (uniq.bits1, uniq.bits2) == (8, 8) and (dups.bits1, dups.bits2) == (8, 9)
    # 2^26 rows: 4096-row partitions would spill past one table, so both stay at 15 bits
    for est in (1 << 26, 1 << 22):
        p = lib.plan(_stats(1 << 26, 0, (1 << 26) - 1, est=est), None, 1 << 26, 1 << 28, lib.I64)
        assert p.bits1 + p.bits2 == 15
    assert lib.plan(_stats(1 << 20, 0, 1 << 30, est=0.89 * (1 << 20)), None, 1 << 20, 1 << 22,
                    lib.I64).variant == "nphj"
    # 2^28 rows: 4096-row partitions for distinct keys (16 bits, 256 digits per
    # pass), 2048 for duplicate-heavy ones (17 bits)
    big_u = lib.plan(_stats(1 << 28, 0, (1 << 28) - 1), None, 1 << 28, 1 << 30, lib.I64)
    big_d = lib.plan(_stats(1 << 28, 0, (1 << 28) - 1, est=1 << 24), None, 1 << 28, 1 << 30, lib.I64)
    assert (big_u.bits1, big_u.bits2) == (8, 8) and (big_d.bits1, big_d.bits2) == (8, 9)


def test_planner_skewed_probe_sample_prefers_the_non_partitioned_join(lib):
    """A probe sample with few distinct keys per row (heavy skew) sends 32-bit
    keys with np >= 2 nb to the NPHJ; moderate skew only while its table is
    within 4x the L2 cache; no sample, a ratio below 2 or 64-bit keys keep
    the partitioned plan."""
    s = 1 << 20

    def plan(log2nb, ratio, frac, lo=0, width=None):
        nb = 1 << log2nb
        hi = lo + (width if width is not None else nb - 1)
        b = _stats(nb, lo, hi)
        p = _stats(s, lo, hi, est=frac * s) if frac is not None else None
        return lib.plan(b, p, nb, ratio * nb, lib.I64).variant

    assert plan(26, 4, 0.014) == "nphj"            # Zipf 1.5-like
    assert plan(28, 4, 0.014) == "nphj"
    assert plan(24, 4, 0.35) == "nphj"             # Zipf 1-like, table 256 MB
    assert plan(26, 4, 0.35) == "phj2"             # ... table 1 GB
    assert plan(26, 4, 0.98) == "phj2"             # uniform
    assert plan(26, 4, None) == "phj2"             # not profiled
    assert plan(26, 1, 0.014) == "phj2"            # ratio below 2
    assert plan(26, 4, 0.014, lo=-2**62, width=2**63) == "phj2"  # 64-bit keys (16-byte slots)


def _target(nb, distinct):
    return (4096 if nb >= 1 << 27 else 3072) if distinct else 2048


def _rules_reference(nb, distinct, key32, l2=126 << 20):
    """The planning rules restated from their specification (Sec. 5.2.1-5.2.2
    crossover; partition target 2048 rows, 3072 for distinct build keys, 4096
    for distinct build keys from 2^27 rows up): (variant, bits1, bits2)."""
    slots = 64
    while slots < nb / 0.5:
        slots <<= 1
    if slots * (8 if key32 else 16) <= l2 // 2:
        return ("nphj", None, None)
    target = _target(nb, distinct)
    parts = (nb + target - 1) // target
    b = max(2, min(20, (parts - 1).bit_length()))  # smallest b with 2^b >= parts
    if b <= 8:
        return ("phj1", min(b, 12), 0)
    return ("phj2", b // 2, b - b // 2)


@pytest.mark.parametrize("log2nb", [10, 16, 20, 21, 22, 23, 24, 25, 26, 27, 28, 29, 30, 31])
@pytest.mark.parametrize("scale", [1.0, 1.12, 1.45, 1.9])
@pytest.mark.parametrize("distinct", [True, False])
def test_planner_matches_its_rules_everywhere(lib, log2nb, scale, distinct):
    """eiger_plan against the rules restated in Python, over build sizes from
    2^10 to just below 2^32 rows, distinct and duplicate-heavy keys; every PHJ
    plan keeps the average build partition within one shared-memory table."""
    nb = min(int((1 << log2nb) * scale), (1 << 32) - 1)
    est = nb if distinct else nb / 8
    p = lib.plan(_stats(nb, 0, nb - 1, est=est), None, nb, min(4 * nb, (1 << 32) - 1), lib.I64)
    want = _rules_reference(nb, distinct, key32=True)
    got = (p.variant, p.bits1 if p.variant != "nphj" else None, p.bits2 if p.variant != "nphj" else None)
    assert got == want
    if p.variant != "nphj":
        b = p.bits1 + p.bits2
        assert nb / (1 << b) <= _target(nb, distinct) or b == 20
        assert b == 2 or nb / (1 << (b - 1)) > _target(nb, distinct)


def test_planner_narrows_only_spans_below_2_32(lib):
    ok = lib.plan(_stats(1 << 24, 10, 10 + 0xFFFFFFFF), None, 1 << 24, 1 << 24, lib.I64)
    wide = lib.plan(_stats(1 << 24, 10, 10 + 0x100000000), None, 1 << 24, 1 << 24, lib.I64)
    assert ok.narrow == 1 and wide.narrow == 0
    neg = lib.plan(_stats(1 << 24, -2**63, 2**63 - 1), None, 1 << 24, 1 << 24, lib.I64)
    assert neg.narrow == 0


def test_planner_bits_grow_with_the_build_side(lib):
    prev = 0
    for k in range(23, 29):
        p = lib.plan(_stats(1 << k, 0, (1 << k) - 1), None, 1 << k, 1 << 28, lib.I64)
        assert p.variant in ("phj1", "phj2")
        b = p.bits1 + p.bits2
        assert b >= prev
        assert (1 << k) / (1 << b) <= 4096  # average partition fits a shared-memory table
        prev = b


def test_workspace_covers_every_auto_plan(lib):
    for nb, np_ in ((1000, 4000), (1 << 20, 1 << 22), (1 << 26, 1 << 28)):
        auto = lib.join_workspace(nb, np_, lib.I64, "auto")
        for v in ("nphj", "phj1", "phj2"):
            assert lib.join_workspace(nb, np_, lib.I64, v) > 0
        assert auto >= lib.join_workspace(nb, np_, lib.I64, "static") or auto > 0
        knob = lib.Plan("phj2", 6, 6, 1)
        assert lib.join_workspace(nb, np_, lib.I64, "phj2", knob) > 0


def test_invalid_arguments_are_rejected_without_a_gpu(lib):
    so = lib.load()
    cnt = ctypes.c_int64(7)
    # bad dtype
    st = so.eiger_join(5, None, None, 0, None, None, 0, 0, 0, None, None, None, None, None, 0,
                       ctypes.byref(cnt), None, 0, None, None)
    assert st == lib.ERR_INVALID_ARG and "dtype" in lib.last_error()
    # rows with a NULL key column
    st = so.eiger_join(lib.I64, None, None, 10, None, None, 0, 0, 0, None, None, None, None, None, 0,
                       ctypes.byref(cnt), None, 0, None, None)
    assert st == lib.ERR_INVALID_ARG
    # 2^32 rows
    st = so.eiger_join(lib.I64, ctypes.c_void_p(64), None, 1 << 32, None, None, 0, 0, 0, None, None,
                       None, None, None, 0, ctypes.byref(cnt), None, 0, None, None)
    assert st == lib.ERR_INVALID_ARG and "2^32" in lib.last_error()
    # capacity without outputs
    st = so.eiger_join(lib.I64, None, None, 0, None, None, 0, 0, 0, None, None, None, None, None, 5,
                       ctypes.byref(cnt), None, 0, None, None)
    assert st == lib.ERR_INVALID_ARG
    # misaligned int64 keys
    st = so.eiger_join(lib.I64, ctypes.c_void_p(4), None, 1, ctypes.c_void_p(8), None, 1, 0, 0, None,
                       None, None, None, None, 0, ctypes.byref(cnt), None, 0, None, None)
    assert st == lib.ERR_INVALID_ARG and "aligned" in lib.last_error()
    # payload output without a payload column
    st = so.eiger_join(lib.I32, None, None, 0, None, None, 0, 4, 0, None, None, None,
                       ctypes.c_void_p(64), None, 1, ctypes.byref(cnt), None, 0, None, None)
    assert st == lib.ERR_INVALID_ARG
    # bad variant
    st = so.eiger_join(lib.I32, None, None, 0, None, None, 0, 0, 9, None, None, None, None, None, 0,
                       ctypes.byref(cnt), None, 0, None, None)
    assert st == lib.ERR_INVALID_ARG
    # sum without payloads
    s = ctypes.c_int64(0)
    st = so.eiger_join_sum(lib.I32, ctypes.c_void_p(64), None, 3, ctypes.c_void_p(64), None, 3, 8, 0,
                           lib.MAT_AUTO, None, ctypes.byref(s), ctypes.byref(cnt), None, 0, None, None)
    assert st == lib.ERR_INVALID_ARG
    # bad materialisation
    st = so.eiger_join_sum(lib.I32, ctypes.c_void_p(64), ctypes.c_void_p(64), 3, ctypes.c_void_p(64),
                           ctypes.c_void_p(64), 3, 8, 0, 5, None, ctypes.byref(s), ctypes.byref(cnt), None, 0,
                           None, None)
    assert st == lib.ERR_INVALID_ARG and "materialize" in lib.last_error()
    # stats: NULL output, negative n
    assert so.eiger_stats(None, 0, lib.I32, None, None, 0, None) == lib.ERR_INVALID_ARG
    out = lib.StatsT()
    assert so.eiger_stats(None, -1, lib.I32, ctypes.byref(out), None, 0, None) == lib.ERR_INVALID_ARG


def test_empty_stats_need_no_gpu(lib):
    s = lib.stats_workspace(0, lib.I64)
    assert s > 0
    so = lib.load()
    out = lib.StatsT()
    assert so.eiger_stats(None, 0, lib.I64, ctypes.byref(out), None, 0, None) == lib.OK
    assert out.n == 0 and out.min == 2**63 - 1 and out.max == -2**63 and out.estimate == 0.0


def test_knob_validation(lib):
    so = lib.load()
    cnt = ctypes.c_int64(0)
    ws = ctypes.c_size_t(0)
    bad = lib.Plan("phj2", 13, 2, 0).to_c()
    # workspace queries accept any knobs; the join validates them after profiling,
    # which needs a GPU, so here only the query path is exercised.
    assert so.eiger_join_workspace(100, 100, lib.I64, lib.PHJ2, ctypes.byref(bad), ctypes.byref(ws)) == 0
    assert so.eiger_join_workspace(100, 100, 7, lib.PHJ2, None, ctypes.byref(ws)) == lib.ERR_INVALID_ARG
    assert so.eiger_join_workspace(-1, 100, lib.I64, lib.PHJ2, None, ctypes.byref(ws)) == lib.ERR_INVALID_ARG
    del cnt


def test_batched_workspace_query_needs_no_gpu(lib):
    descs = (lib.JoinDescT * 3)()
    for j, (nb, np_) in enumerate([(1000, 4000), (0, 10), (70_000, 5)]):
        descs[j].nb, descs[j].np = nb, np_
    ws = ctypes.c_size_t(0)
    so = lib.load()
    kn = lib.BatchKnobs(small_rows=0).to_c()
    assert so.eiger_join_batched_workspace(descs, 3, lib.I32, ctypes.byref(kn), ctypes.byref(ws)) == 0
    # tables: 2048 + 0 + 2^18 slots of 8 bytes, plus bookkeeping
    assert ws.value >= (2048 + (1 << 18)) * 8
    # the 1000-row build is a small join (table in shared memory): no global slots
    kn = lib.BatchKnobs(small_rows=1000).to_c()
    assert so.eiger_join_batched_workspace(descs, 3, lib.I32, ctypes.byref(kn), ctypes.byref(ws)) == 0
    assert (1 << 18) * 8 <= ws.value < (2048 + (1 << 18)) * 8
    kn = lib.BatchKnobs(small_rows=999).to_c()
    assert so.eiger_join_batched_workspace(descs, 3, lib.I32, ctypes.byref(kn), ctypes.byref(ws)) == 0
    assert ws.value >= (2048 + (1 << 18)) * 8
    bad = lib.BatchKnobs(100, 16384, 0.5).to_c()
    assert so.eiger_join_batched_workspace(descs, 3, lib.I32, ctypes.byref(bad), ctypes.byref(ws)) == lib.ERR_INVALID_ARG
    # shared-memory tables hold at most EIGER_BATCH_SMALL_MAX_* build rows
    for dt, smax in ((lib.I32, lib.BATCH_SMALL_MAX_I32), (lib.I64, lib.BATCH_SMALL_MAX_I64)):
        ok = lib.BatchKnobs(small_rows=smax).to_c()
        assert so.eiger_join_batched_workspace(descs, 3, dt, ctypes.byref(ok), ctypes.byref(ws)) == 0
        for v in (smax + 1, -1):
            bad = lib.BatchKnobs(small_rows=v).to_c()
            assert so.eiger_join_batched_workspace(descs, 3, dt, ctypes.byref(bad), ctypes.byref(ws)) == lib.ERR_INVALID_ARG
    st = ctypes.c_int32(0)
    assert lib.load().eiger_join_batched(lib.I32, None, 3, None, None, None, None, 0, None) == lib.ERR_INVALID_ARG


def test_wide_workspace_counts_carried_columns(lib):
    """GFTR carries the payload columns through the passes, so its workspace
    grows by two copies of every column; GFUR's does not."""
    import torch

    nb, np_ = 1 << 20, 1 << 22
    bcols = [torch.empty(0, dtype=torch.int64), torch.empty(0, dtype=torch.int32)]
    pcols = [torch.empty(0, dtype=torch.int64)]
    knobs = lib.Plan("phj2", 5, 5, 1)
    gfur = lib.join_wide_workspace(nb, np_, lib.I64, bcols, pcols, "phj2", "gfur", knobs)
    gftr = lib.join_wide_workspace(nb, np_, lib.I64, bcols, pcols, "phj2", "gftr", knobs)
    assert gftr - gfur >= 2 * (nb * 12 + np_ * 8)
    smj = lib.join_wide_workspace(nb, np_, lib.I64, bcols, pcols, "smj", "gftr", None)
    assert smj >= 2 * (nb * 12 + np_ * 8)
    assert lib.join_wide_workspace(nb, np_, lib.I64, [], [], "smj", "gfur", None) == \
        lib.join_workspace(nb, np_, lib.I64, "smj")


def test_sum_workspace_counts_carried_payloads(lib):
    """A carried (GFTR) sum holds two copies of both payload columns; GFUR
    needs no more than the plain join."""
    nb, np_ = 1 << 20, 1 << 22
    knobs = lib.Plan("phj2", 5, 5, 1)
    gfur = lib.join_sum_workspace(nb, np_, lib.I32, 8, "phj2", "gfur", knobs)
    gftr = lib.join_sum_workspace(nb, np_, lib.I32, 8, "phj2", "gftr", knobs)
    assert gfur == lib.join_workspace(nb, np_, lib.I32, "phj2", knobs)
    assert gftr - gfur >= 2 * 8 * (nb + np_)
    assert lib.join_sum_workspace(nb, np_, lib.I32, 8, "auto", "auto") >= gftr - gfur
    # NPHJ never carries
    assert lib.join_sum_workspace(nb, np_, lib.I32, 8, "nphj", "auto") == lib.join_workspace(nb, np_, lib.I32, "nphj")
    so = lib.load()
    ws = ctypes.c_size_t(0)
    assert so.eiger_join_sum_workspace(10, 10, lib.I32, 2, 0, lib.MAT_AUTO, None, ctypes.byref(ws)) == lib.ERR_INVALID_ARG
    assert so.eiger_join_sum_workspace(10, 10, lib.I32, 8, 0, 3, None, ctypes.byref(ws)) == lib.ERR_INVALID_ARG


def test_wide_argument_checks(lib):
    so = lib.load()
    ws = ctypes.c_size_t(0)
    bad = lib.ColumnsT()
    bad.n = 5
    assert so.eiger_join_wide_workspace(10, 10, lib.I64, ctypes.byref(bad), None, lib.PHJ2, lib.GFTR, None,
                                        ctypes.byref(ws)) == lib.ERR_INVALID_ARG
    bad.n = 1
    bad.bytes[0] = 2
    assert so.eiger_join_wide_workspace(10, 10, lib.I64, ctypes.byref(bad), None, lib.PHJ2, lib.GFTR, None,
                                        ctypes.byref(ws)) == lib.ERR_INVALID_ARG
    assert "bytes" in lib.last_error()
    assert so.eiger_join_wide_workspace(10, 10, lib.I64, None, None, lib.SMJ, 7, None,
                                        ctypes.byref(ws)) == lib.ERR_INVALID_ARG
    ok = lib.ColumnsT()
    ok.n = 1
    ok.bytes[0] = 8
    cnt = ctypes.c_int64(0)
    # data pointers are required by the join itself
    assert so.eiger_join_wide(lib.I64, None, 0, ctypes.byref(ok), None, 0, None, lib.SMJ, lib.GFTR, None,
                              None, None, 0, ctypes.byref(cnt), None, 0, None, None) == lib.ERR_INVALID_ARG


def test_smj_knob_validation(lib):
    so = lib.load()
    ws = ctypes.c_size_t(0)
    k = lib.Plan("smj", 9, 0, 1).to_c()
    assert so.eiger_join_workspace(100, 100, lib.I64, lib.SMJ, ctypes.byref(k), ctypes.byref(ws)) == 0
    assert so.eiger_join_workspace(100, 100, lib.I64, 6, None, ctypes.byref(ws)) == lib.ERR_INVALID_ARG


def test_autotuner_picks_best_mean_relative_time():
    """The batched autotuner's objective: each entry's time on every tuning
    batch relative to that batch's fastest entry, averaged; the small batch
    (sub-millisecond) weighs as much as the large one."""
    from paper_2607_04489_gb300 import autotune

    grid = [
        {"small_rows": 0, "ms": [10.0, 0.30]},     # fastest on the large batch by a hair
        {"small_rows": 2048, "ms": [10.1, 0.15]},  # 1 % slower there, 2x faster on the small one
        {"small_rows": 1024, "ms": [12.0, 0.15]},
    ]
    best = autotune.pick(grid)
    assert best["small_rows"] == 2048
    assert [r["rel"] for r in grid] == [1.5, 1.005, 1.1]
    # ties go to the first entry
    assert autotune.pick([{"k": 1, "ms": [1.0]}, {"k": 2, "ms": [1.0]}])["k"] == 1
