"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test checks one oracle function against something the paper or the
mathematics fixes: brute force on tiny inputs, the cardinality identity
|J| = sum_k cnt_R(k) * cnt_S(k), closed forms of permutation workloads, the
published SplitMix64 sequence, HyperLogLog invariants and its 1.04/sqrt(m)
standard error. A plausible slip in the oracle (a dropped match, a swapped
side, a rank off by one, a wrong register split) fails at least one of them.
"""

import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
M64 = (1 << 64) - 1


def _nested_loop(bk, pk):
    """All (b, p) with bk[b] == pk[p], sorted by (p, b): plain brute force."""
    if bk.size == 0 or pk.size == 0:
        return np.empty(0, np.uint32), np.empty(0, np.uint32)
    eq = bk.astype(np.int64)[:, None] == pk.astype(np.int64)[None, :]
    b, p = np.nonzero(eq)
    order = np.lexsort((b, p))
    return b[order].astype(np.uint32), p[order].astype(np.uint32)


def _edge_keys(rng, n, dtype, span):
    info = np.iinfo(dtype)
    base = rng.integers(-span, span, size=n, dtype=np.int64)
    v = base.astype(dtype) if dtype == np.int32 else base
    if n >= 4:
        v[0] = info.min
        v[1] = info.max
        v[2] = 0
        v[3] = -1
    return v


# --------------------------------------------------------------------- hash

def test_h64_published_splitmix64_sequence(oracle_mod):
    gamma = 0x9E3779B97F4A7C15
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64_state0.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 5
    for k, out in rows:
        assert oracle_mod.h64((int(k) * gamma) & M64) == int(out, 16)


def test_h64_bijective_on_sample(oracle_mod):
    rng = np.random.default_rng(7)
    x = np.unique(rng.integers(0, 2**63, size=1 << 16, dtype=np.int64).astype(np.uint64))
    y = {oracle_mod.h64(int(v)) for v in x}
    assert len(y) == x.size
    assert oracle_mod.h64(0) == 0  # xor-shift/multiply steps fix zero


# --------------------------------------------------------------------- join

@pytest.mark.parametrize("dtype", [np.int32, np.int64])
def test_join_matches_nested_loop(oracle_mod, dtype):
    rng = np.random.default_rng(11 if dtype == np.int32 else 12)
    for trial in range(60):
        nb = int(rng.integers(0, 200))
        np_ = int(rng.integers(0, 300))
        span = int(rng.choice([3, 40, 1000, 2**31 - 1]))
        bk = _edge_keys(rng, nb, dtype, span)
        pk = _edge_keys(rng, np_, dtype, span)
        if np_ and nb:  # make some probe keys copy build keys
            sel = rng.integers(0, nb, size=np_ // 2)
            pk[: sel.size] = bk[sel]
        b, p, n = oracle_mod.join(bk, pk)
        eb, ep = _nested_loop(bk, pk)
        assert n == eb.size
        np.testing.assert_array_equal(b, eb)
        np.testing.assert_array_equal(p, ep)


@pytest.mark.parametrize("threads", [1, 2, 3, 8])
def test_threaded_join_equals_one_thread_and_nested_loop(oracle_mod, threads):
    """The -t N mode splits only the probe loop: its canonical output is the
    one-thread join's, element for element, and the brute force's."""
    rng = np.random.default_rng(31 + threads)
    for trial in range(12):
        nb = int(rng.integers(0, 400))
        np_ = int(rng.integers(0, 700))
        bk = rng.integers(-20, 20, size=nb).astype(np.int64)
        pk = rng.integers(-25, 25, size=np_).astype(np.int64)
        b1, p1, n1 = oracle_mod.join(bk, pk)
        bt, pt, nt = oracle_mod.join_mt(bk, pk, threads)
        eb, ep = _nested_loop(bk, pk)
        assert n1 == nt == eb.size
        np.testing.assert_array_equal(bt, b1)
        np.testing.assert_array_equal(pt, p1)
        np.testing.assert_array_equal(bt, eb)
        np.testing.assert_array_equal(pt, ep)


def _py_h64(z):
    """SplitMix64's output function in plain Python integers (the published
    definition; the oracle's h64 is pinned to its sequence above)."""
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


@pytest.mark.parametrize("threads", [1, 4])
def test_join_fingerprint_matches_brute_force_pairs(oracle_mod, threads):
    """The streamed fingerprint equals the sum / xor over the nested-loop
    pairs, with each pair read as build_idx * 2^32 + probe_idx; a swapped
    side or a dropped pair changes it."""
    rng = np.random.default_rng(41)
    bk = rng.integers(0, 30, size=150).astype(np.int32)
    pk = rng.integers(0, 40, size=260).astype(np.int32)
    eb, ep = _nested_loop(bk, pk)
    s = x = 0
    for b, p in zip(eb.tolist(), ep.tolist()):
        w = (b << 32) | p
        s = (s + _py_h64(w)) & M64
        x ^= _py_h64((w + 0x9E3779B97F4A7C15) & M64)
    n, fs, fx = oracle_mod.join_fingerprint(bk, pk, threads)
    assert (n, fs, fx) == (eb.size, s, x)
    swapped = 0
    for b, p in zip(eb.tolist(), ep.tolist()):
        swapped = (swapped + _py_h64((p << 32) | b)) & M64
    assert swapped != fs
    assert oracle_mod.join_fingerprint(bk, pk[:-1], threads)[1:] != (fs, fx) or \
        int((bk == pk[-1]).sum()) == 0
    assert oracle_mod.join_fingerprint(bk[:0], pk, threads) == (0, 0, 0)


def test_join_int64_extremes_and_wide_span(oracle_mod):
    # keys that agree in the low 32 bits but differ above must not match
    bk = np.array([2**32, 0, -2**63, 2**63 - 1, 5, 5], np.int64)
    pk = np.array([0, 2**32, 2**32 + 2**33, -2**63, 2**63 - 1, 5, 2**32 + 5], np.int64)
    b, p, n = oracle_mod.join(bk, pk)
    eb, ep = _nested_loop(bk, pk)
    assert n == 6
    np.testing.assert_array_equal(b, eb)
    np.testing.assert_array_equal(p, ep)


def test_join_cardinality_identity(oracle_mod):
    rng = np.random.default_rng(3)
    for distinct in (5, 300, 20000):
        bk = rng.integers(0, distinct, size=8000).astype(np.int64)
        pk = rng.integers(0, distinct, size=30000).astype(np.int64)
        ub, cb = np.unique(bk, return_counts=True)
        up, cp = np.unique(pk, return_counts=True)
        _, ib, ip = np.intersect1d(ub, up, return_indices=True)
        expect = int(np.sum(cb[ib].astype(np.int64) * cp[ip].astype(np.int64)))
        assert oracle_mod.join_count(bk, pk) == expect
        b, p, n = oracle_mod.join(bk, pk, cap=min(expect, 1000))
        assert n == expect and b.size == min(expect, 1000)
        assert np.all(bk[b] == pk[p])


def test_join_permutation_closed_form(oracle_mod):
    nb, np_ = 1 << 14, 1 << 16
    rng = np.random.default_rng(0)
    perm = rng.permutation(nb).astype(np.int32)
    pk = rng.integers(0, nb, size=np_).astype(np.int32)
    inv = np.empty(nb, np.int64)
    inv[perm] = np.arange(nb)
    b, p, n = oracle_mod.join(perm, pk)
    assert n == np_
    np.testing.assert_array_equal(p, np.arange(np_, dtype=np.uint32))
    np.testing.assert_array_equal(b, inv[pk].astype(np.uint32))


def test_join_sum_direct_addressing(oracle_mod):
    rng = np.random.default_rng(5)
    n_dim, n_fact = 5000, 40000
    dk = (rng.permutation(n_dim) + 1).astype(np.int32)
    dp = rng.integers(0, 10**9, size=n_dim).astype(np.int64)
    fk = rng.integers(1, 2 * n_dim + 1, size=n_fact).astype(np.int32)  # about half absent
    fp = rng.integers(0, 10**7, size=n_fact).astype(np.int64)
    row_of_key = np.full(2 * n_dim + 2, -1, np.int64)
    row_of_key[dk] = np.arange(n_dim)
    r = row_of_key[fk]
    hit = r >= 0
    expect = (int(dp[r[hit]].sum()) + int(fp[hit].sum())) % (1 << 64)
    if expect >= 1 << 63:
        expect -= 1 << 64
    s, c = oracle_mod.join_sum(dk, dp, fk, fp)
    assert c == int(hit.sum())
    assert s == expect


def test_join_sum_wraps_modulo_2_64(oracle_mod):
    bk = np.array([1, 2], np.int64)
    bp = np.array([2**62, -7], np.int64)
    pk = np.array([1, 1, 1, 1, 2], np.int64)
    pp = np.array([2**62, 2**62, 0, 3, 9], np.int64)
    # four matches of key 1: 4 * bp[0] + (2^62 + 2^62 + 0 + 3); one of key 2: -7 + 9
    expect = (4 * 2**62 + 2 * 2**62 + 3 + (-7 + 9)) % (1 << 64)
    expect = expect - (1 << 64) if expect >= 1 << 63 else expect
    s, c = oracle_mod.join_sum(bk, bp, pk, pp)
    assert c == 5 and s == expect


def test_join_empty_sides(oracle_mod):
    e = np.empty(0, np.int64)
    k = np.arange(10, dtype=np.int64)
    for bk, pk in ((e, k), (k, e), (e, e)):
        b, p, n = oracle_mod.join(bk, pk)
        assert n == 0 and b.size == 0


# --------------------------------------------------------------------- stats

@pytest.mark.parametrize("dtype", [np.int32, np.int64])
def test_minmax_matches_numpy(oracle_mod, dtype):
    rng = np.random.default_rng(1)
    for n in (1, 2, 17, 1000):
        k = _edge_keys(rng, n, dtype, 2**31 - 1)
        mn, mx, _ = oracle_mod.stats(k)
        assert mn == int(k.min()) and mx == int(k.max())


def test_stats_empty(oracle_mod):
    mn, mx, regs = oracle_mod.stats(np.empty(0, np.int64))
    assert mn == 2**63 - 1 and mx == -2**63
    assert not regs.any()
    assert oracle_mod.hll_estimate(regs) == 0.0


def test_hll_registers_see_the_set_not_the_multiset(oracle_mod):
    rng = np.random.default_rng(2)
    k = rng.integers(-10**6, 10**6, size=50000).astype(np.int64)
    u = np.unique(k)
    _, _, r1 = oracle_mod.stats(k)
    _, _, r2 = oracle_mod.stats(u)
    _, _, r3 = oracle_mod.stats(rng.permutation(np.repeat(u, 3)))
    np.testing.assert_array_equal(r1, r2)
    np.testing.assert_array_equal(r1, r3)


def test_hll_union_is_registerwise_max(oracle_mod):
    rng = np.random.default_rng(4)
    a = rng.integers(0, 2**62, size=70000).astype(np.int64)
    b = rng.integers(0, 2**62, size=30000).astype(np.int64)
    _, _, ra = oracle_mod.stats(a)
    _, _, rb = oracle_mod.stats(b)
    _, _, rab = oracle_mod.stats(np.concatenate([a, b]))
    np.testing.assert_array_equal(rab, np.maximum(ra, rb))


def test_hll_int32_and_int64_hash_alike(oracle_mod):
    rng = np.random.default_rng(9)
    k32 = rng.integers(-2**31, 2**31, size=40000).astype(np.int32)
    _, _, r32 = oracle_mod.stats(k32)
    _, _, r64 = oracle_mod.stats(k32.astype(np.int64))
    np.testing.assert_array_equal(r32, r64)


def test_hll_single_key_sets_one_register(oracle_mod):
    for key in (0, 1, -1, 2**40 + 3):
        _, _, regs = oracle_mod.stats(np.array([key], np.int64))
        nz = np.nonzero(regs)[0]
        assert nz.size == 1 and 1 <= regs[nz[0]] <= 51
        # the register index is the top 14 bits of the hash
        assert nz[0] == oracle_mod.h64(key & M64) >> 50


def test_hll_estimate_constant_registers_closed_form(oracle_mod):
    # With every register equal to r the raw estimator alpha m^2 / sum 2^-reg
    # reduces to alpha * m * 2^r; r = 0 instead takes linear counting m ln 1 = 0.
    m = oracle_mod.HLL_M
    alpha = 0.7213 / (1 + 1.079 / m)
    for r in (1, 3, 10, 20, 51):
        e = oracle_mod.hll_estimate(np.full(m, r, np.uint8))
        assert e == pytest.approx(alpha * m * 2.0**r, rel=1e-12)
    assert oracle_mod.hll_estimate(np.zeros(m, np.uint8)) == 0.0


def test_hll_estimate_linear_counting_closed_form(oracle_mod):
    m = oracle_mod.HLL_M
    for v in (1, 100, 8000, m - 1):
        regs = np.zeros(m, np.uint8)
        regs[v:] = 1  # v zero registers, the rest 1 -> raw estimate <= 2.5 m
        assert oracle_mod.hll_estimate(regs) == pytest.approx(m * math.log(m / v), rel=1e-12)


def test_hll_standard_error(oracle_mod):
    """RMS relative error within 1.2 x 1.04/sqrt(m), no run beyond 4 sigma."""
    m = oracle_mod.HLL_M
    sigma = 1.04 / math.sqrt(m)
    rng = np.random.default_rng(2024)
    errs = []
    plan = [(10**5, 40), (10**6, 40), (10**7, 20)]
    for n, reps in plan:
        for _ in range(reps):
            k = rng.integers(-2**63, 2**63 - 1, size=n, dtype=np.int64)
            true = oracle_mod.exact_ndv(k)
            _, _, regs = oracle_mod.stats(k)
            errs.append(oracle_mod.hll_estimate(regs) / true - 1.0)
    errs = np.array(errs)
    assert math.sqrt(np.mean(errs**2)) <= 1.2 * sigma
    assert np.max(np.abs(errs)) <= 4 * sigma


def test_hll_linear_counting_small_cardinalities(oracle_mod):
    """Below ~2.5 m the estimate is linear counting; its standard error is
    sqrt(m (e^t - t - 1)) / n with t = n / m (Whang et al. 1990)."""
    m = oracle_mod.HLL_M
    rng = np.random.default_rng(77)
    for n in (10, 100, 1000, 5000):
        t = n / m
        sd = math.sqrt(m * (math.exp(t) - t - 1)) / n
        for _ in range(10):
            k = np.unique(rng.integers(0, 2**62, size=n, dtype=np.int64))
            _, _, regs = oracle_mod.stats(k)
            e = oracle_mod.hll_estimate(regs)
            assert abs(e / k.size - 1) <= max(5 * sd, 1e-9)


def test_exact_ndv_matches_set(oracle_mod):
    rng = np.random.default_rng(8)
    for dtype in (np.int32, np.int64):
        k = rng.integers(-50, 50, size=3000).astype(dtype)
        assert oracle_mod.exact_ndv(k) == len(set(k.tolist()))
    assert oracle_mod.exact_ndv(np.empty(0, np.int64)) == 0


def test_wide_join_matches_nested_loop_with_columns(oracle_mod):
    """Every (i, j) with equal keys, found by a nested loop, carries row i of
    each build column and row j of each probe column."""
    rng = np.random.default_rng(77)
    bk = rng.integers(-5, 6, size=40).astype(np.int64)
    pk = rng.integers(-7, 8, size=60).astype(np.int64)
    bc = [rng.integers(-2**62, 2**62, size=40), rng.integers(-2**31, 2**31, size=40).astype(np.int32)]
    pc = [rng.integers(0, 1000, size=60).astype(np.int32)]
    want = sorted((j, i, tuple(int(c[i]) for c in bc), tuple(int(c[j]) for c in pc))
                  for j in range(60) for i in range(40) if bk[i] == pk[j])
    b, p, obc, opc = oracle_mod.join_wide(bk, pk, bc, pc)
    got = [(int(p[k]), int(b[k]), tuple(int(c[k]) for c in obc), tuple(int(c[k]) for c in opc))
           for k in range(len(b))]
    assert got == want


def test_torch_pair_fingerprint_matches_oracle(oracle_mod):
    """The torch fingerprint that the full-size GPU tests compute from the
    GPU's pairs is the oracle's join_fingerprint (on the CPU, from the
    oracle's own canonical pairs, duplicates and both dtypes)."""
    import torch

    from fingerprint import pair_fingerprint

    rng = np.random.default_rng(43)
    for dtype in (np.int32, np.int64):
        bk = rng.integers(-50, 50, size=3000).astype(dtype)
        pk = rng.integers(-60, 60, size=7001).astype(dtype)
        b, p, n = oracle_mod.join(bk, pk)
        got = pair_fingerprint(torch.from_numpy(b.astype(np.int64)), torch.from_numpy(p.astype(np.int64)),
                               chunk=4096)
        assert got == oracle_mod.join_fingerprint(bk, pk, 3)
        order = rng.permutation(n)  # order-independent
        assert pair_fingerprint(torch.from_numpy(b[order].astype(np.int64)),
                                torch.from_numpy(p[order].astype(np.int64))) == got
