"""The largest joins of the variant sweep, in the launch configuration the
benchmark times, checked on the device; and a full-size join with duplicate
build keys checked against the oracle through order-independent fingerprints.

Variant-sweep joins have unique build keys and every probe key drawn from
them, so the exact result is one pair per probe row whose keys are equal:
the checks below (count = np, every probe row exactly once, every pair's
keys equal) pin every pair without a host sort. 2^28 build rows at ratio 4
(2^30 probe rows) is the largest sweep size whose tuple IDs fit 32 bits at
that ratio. Inputs: dense keys (narrowed to 32-bit offsets), random 64-bit
keys (not narrowable: the 64-bit partitioned path), and Zipf 1.5 probes
(one key takes ~38 % of the probe rows: multi-chunk probe partitions).
"""

import os

import numpy as np
import pytest
import torch

from fingerprint import pair_fingerprint

pytestmark = pytest.mark.gpu

GB = 1 << 30


@pytest.fixture(scope="module")
def eiger():
    from paper_2607_04489_gb300 import eiger

    eiger.load()
    return eiger


def _need(gb):
    free, _ = torch.cuda.mem_get_info()
    if free < gb * GB:
        pytest.skip(f"needs {gb} GB of free device memory")


def _check_unique_build_result(w, r):
    """Every probe row appears exactly once and every pair joins equal keys."""
    assert r.count == w.np
    p = r.probe_idx.long() & 0xFFFFFFFF
    b = r.build_idx.long() & 0xFFFFFFFF
    cnt = torch.bincount(p, minlength=w.np)
    assert int(cnt.min()) == 1 and int(cnt.max()) == 1
    del cnt
    assert bool((w.build_keys[b] == w.probe_keys[p]).all())


@pytest.mark.parametrize("keys,theta,variant", [("dense", 0.0, "phj2"), ("random", 0.0, "phj2"),
                                                 ("dense", 1.5, "nphj")])
def test_largest_sweep_join(eiger, keys, theta, variant):
    """AUTO at nb = 2^28, np = 2^30 (the benchmark's default call for dense
    uniform keys); with Zipf 1.5 probes the probe sample sends it to the
    non-partitioned join."""
    from paper_2607_04489_gb300 import workloads

    _need(110)
    w = workloads.variant_sweep(1 << 28, 4, keys=keys, theta=theta, seed=0, device="cuda", payload_bytes=8)
    w.build_pay = w.probe_pay = None
    torch.cuda.empty_cache()
    r = eiger.join(w.build_keys, w.probe_keys, variant="auto")
    assert r.plan.variant == variant
    assert r.plan.narrow == (1 if keys == "dense" else 0)
    _check_unique_build_result(w, r)


def test_largest_sweep_join_skewed_partitioned(eiger):
    """The partitioned join forced on the Zipf 1.5 probes at 2^28 x 2^30: one
    key takes ~38 % of the probe rows, so its partition's probe side is cut
    into thousands of chunks over one build table."""
    from paper_2607_04489_gb300 import workloads

    _need(110)
    w = workloads.variant_sweep(1 << 28, 4, keys="dense", theta=1.5, seed=0, device="cuda", payload_bytes=8)
    w.build_pay = w.probe_pay = None
    torch.cuda.empty_cache()
    r = eiger.join(w.build_keys, w.probe_keys, variant="phj2", knobs=eiger.Plan("phj2", 8, 8, 1))
    assert (r.plan.variant, r.plan.bits1, r.plan.bits2) == ("phj2", 8, 8)
    _check_unique_build_result(w, r)


def test_largest_sweep_join_static(eiger):
    """The static hash join on the benchmark's inputs (16-byte slots, 2^29 of them)."""
    from paper_2607_04489_gb300 import workloads

    _need(110)
    w = workloads.variant_sweep(1 << 28, 4, keys="dense", theta=0.0, seed=0, device="cuda", payload_bytes=8)
    w.build_pay = w.probe_pay = None
    torch.cuda.empty_cache()
    r = eiger.join(w.build_keys, w.probe_keys, variant="static")
    _check_unique_build_result(w, r)


def test_random_keys_forced_twelve_plus_eight_bits(eiger):
    """Two passes of 12 + 8 bits (2^20 partitions of ~64 build rows) on
    non-narrowable 64-bit keys at 2^26 x 2^28 with Zipf 1.0 probes."""
    from paper_2607_04489_gb300 import workloads

    _need(40)
    w = workloads.variant_sweep(1 << 26, 4, keys="random", theta=1.0, seed=2, device="cuda", payload_bytes=8)
    w.build_pay = w.probe_pay = None
    r = eiger.join(w.build_keys, w.probe_keys, variant="phj2", knobs=eiger.Plan("phj2", 12, 8, 0))
    assert (r.plan.bits1, r.plan.bits2, r.plan.narrow) == (12, 8, 0)
    _check_unique_build_result(w, r)


@pytest.mark.parametrize("key_bytes,variant", [(8, "auto"), (8, "nphj"), (4, "auto")])
def test_duplicate_build_keys_fingerprint(eiger, oracle_mod, key_bytes, variant):
    """2^25 build rows over 2^21 distinct keys (16 rows per key on average),
    2^25 Zipf(1.0) probe rows: about 2^29 pairs, too many to sort on the host.
    The GPU's pairs and the oracle's multimap join agree in count and in both
    64-bit fingerprints of the pair multiset."""
    from paper_2607_04489_gb300 import selector

    _need(24)
    spec = selector.JoinSpec(seed=77, nb=1 << 25, np=1 << 25, key_bytes=key_bytes,
                             span_log2=40.0 if key_bytes == 8 else 32.0, distinct_frac=1.0 / 16, theta=1.0)
    bk, pk = selector.make_join(spec, device="cuda")
    cnt = oracle_mod.join_count(bk.cpu().numpy(), pk.cpu().numpy())
    assert cnt < (1 << 31)
    r = eiger.join(bk, pk, variant=variant, capacity=cnt)
    assert r.count == cnt
    got = pair_fingerprint(r.build_idx[:cnt], r.probe_idx[:cnt])
    del r
    torch.cuda.empty_cache()
    threads = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    want = oracle_mod.join_fingerprint(bk.cpu().numpy(), pk.cpu().numpy(), threads)
    assert got == want
