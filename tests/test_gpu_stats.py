"""GPU column statistics vs the CPU oracle: min/max and HyperLogLog registers
bit-exact, the estimate bit-exact given the registers."""

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

I64_MIN, I64_MAX = -2**63, 2**63 - 1


@pytest.fixture(scope="module")
def eiger():
    from paper_2607_04489_gb300 import eiger

    eiger.load()
    return eiger


def _check(eiger, oracle_mod, keys_np, device_keys=None):
    t = torch.from_numpy(keys_np).cuda() if device_keys is None else device_keys
    st = eiger.stats(t)
    mn, mx, regs = oracle_mod.stats(keys_np)
    assert st.n == keys_np.size
    assert st.min == mn and st.max == mx
    np.testing.assert_array_equal(st.hll, regs)
    assert st.estimate == oracle_mod.hll_estimate(regs)
    return st


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 17, 1000, 4096 * 3 + 7, 100_003, (1 << 22) + 5])
def test_stats_parity_sizes(eiger, oracle_mod, dtype, n):
    rng = np.random.default_rng(n)
    info = np.iinfo(dtype)
    k = rng.integers(info.min, info.max, size=n, dtype=np.int64, endpoint=True).astype(dtype)
    _check(eiger, oracle_mod, k)


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
def test_stats_parity_unaligned_start(eiger, oracle_mod, dtype):
    rng = np.random.default_rng(3)
    base = torch.from_numpy(rng.integers(-1000, 1000, size=70_001).astype(dtype)).cuda()
    for off in (1, 2, 3):
        view = base[off:]
        _check(eiger, oracle_mod, base.cpu().numpy()[off:], device_keys=view)


def test_stats_extremes_and_duplicates(eiger, oracle_mod):
    k = np.array([I64_MIN, I64_MAX, 0, -1, 1] * 1000, np.int64)
    st = _check(eiger, oracle_mod, k)
    assert st.min == I64_MIN and st.max == I64_MAX
    _check(eiger, oracle_mod, np.full(123_457, 42, np.int64))
    _check(eiger, oracle_mod, np.full(99, np.iinfo(np.int32).min, np.int32))


def test_stats_empty(eiger):
    st = eiger.stats(torch.empty(0, dtype=torch.int64, device="cuda"))
    assert st.n == 0 and st.min == I64_MAX and st.max == I64_MIN and st.estimate == 0.0
    assert not st.hll.any()


def test_stats_small_static_probe_side(eiger, oracle_mod):
    """eiger_stats on the 4M int32 probe keys of the small static join."""
    from paper_2607_04489_gb300 import workloads

    w = workloads.small_static(device="cpu")
    st = _check(eiger, oracle_mod, w.probe_keys.numpy())
    # about 2^20 (1 - e^-4) distinct values; the sketch is within a few sigma
    assert abs(st.estimate / oracle_mod.exact_ndv(w.probe_keys.numpy()) - 1) < 0.04


def test_stats_full_size_build_column(eiger, oracle_mod):
    """Statistics of the 2^26-row int64 build column the benchmark profiles."""
    from paper_2607_04489_gb300 import workloads

    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    keys = torch.randperm(1 << 26, generator=g, device="cuda") + 123456789
    _check(eiger, oracle_mod, keys.cpu().numpy(), device_keys=keys)
    del workloads
