"""Order-independent fingerprint of a join's pair multiset, computed with torch
on whatever device holds the pairs (test helper, not a test module).

With w = build_idx * 2^32 + probe_idx per pair, the summary is (|J|,
sum of h64(w) mod 2^64, xor of h64(w + 0x9E3779B97F4A7C15)), h64 being
SplitMix64's output function: the same definition as the oracle's
join_fingerprint, so a GPU result too large to sort on the host is compared
with the oracle through these three numbers. torch's int64 arithmetic wraps
modulo 2^64, and the logical right shifts are written as arithmetic shifts
masked to the shifted width.
"""

import torch

M64 = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15


def _s64(c: int) -> int:
    """An unsigned 64-bit constant as the int64 with the same bits."""
    return c - (1 << 64) if c >= (1 << 63) else c


_C1 = _s64(0xBF58476D1CE4E5B9)
_C2 = _s64(0x94D049BB133111EB)
_G = _s64(_GAMMA)


def _shr(z: torch.Tensor, s: int) -> torch.Tensor:
    return (z >> s) & ((1 << (64 - s)) - 1)


def h64(z: torch.Tensor) -> torch.Tensor:
    z = (z ^ _shr(z, 30)) * _C1
    z = (z ^ _shr(z, 27)) * _C2
    return z ^ _shr(z, 31)


def _xor_reduce(x: torch.Tensor) -> int:
    while x.numel() > 1:
        if x.numel() & 1:
            x = torch.cat([x, x.new_zeros(1)])
        h = x.numel() // 2
        x = x[:h] ^ x[h:]
    return int(x[0]) & M64 if x.numel() else 0


def pair_fingerprint(build_idx: torch.Tensor, probe_idx: torch.Tensor, chunk: int = 1 << 26):
    """(count, fp_sum, fp_xor) of the pairs (build_idx[k], probe_idx[k]);
    index tensors of any integer dtype holding values in [0, 2^32)."""
    n = int(build_idx.numel())
    s, x = 0, 0
    for a in range(0, n, chunk):
        b = build_idx[a:a + chunk].to(torch.int64) & 0xFFFFFFFF
        p = probe_idx[a:a + chunk].to(torch.int64) & 0xFFFFFFFF
        w = (b << 32) | p
        del b, p
        s = (s + (int(h64(w).sum(dtype=torch.int64)) & M64)) & M64
        x ^= _xor_reduce(h64(w + _G))
    return n, s, x
