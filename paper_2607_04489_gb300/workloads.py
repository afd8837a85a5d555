"""Seeded synthetic join inputs shaped like the paper's join workloads.

This module only draws inputs. It holds none of the join, hash or sketch
arithmetic, so both the CUDA path and the CPU oracle can be fed from it. Every
generator takes a seed and a torch device; on a given device and torch build
the same seed gives the same tensors. Small parity cases are drawn on the CPU
and copied to the GPU; full-size benchmark inputs are drawn on the GPU.

Workload shapes (Sec. 5.2 of the paper: |R| the smaller build side, |S| the
probe side, narrow joins of one key and one payload column per side; the
star-schema foreign-key join takes the shape of the TPC-H joins of Sec. 5.7,
whose data is not used):

- ``small_static``: unique int32 build keys (a permutation of 0..nb-1), int32
  payloads, probe keys uniform over the build keys, so every probe row matches
  exactly once.
- ``variant_sweep``: unique int64 build keys, either dense (a seeded base plus a
  permutation of 0..nb-1: span < 2^32, so the keys narrow to uint32) or spread
  over the whole 64-bit range; probe keys drawn from the build keys uniformly or
  Zipf(theta) over a seeded rank order; 8-byte payloads.
- ``batched_small``: k independent int32 joins; build sizes 2^U(lo, hi)
  (log-uniform), unique keys a seeded affine bijection of 0..nb-1 on 32 bits,
  probe = ratio x build rows drawn from the build keys with a per-join
  power-law skew theta_j ~ U(0, theta_max) (continuous inverse-CDF
  approximation of Zipf) over a seeded row permutation.
- ``star_schema``: dimension keys a permutation of 1..n_dim (int32) with int64
  cents payloads in [0, 1e9); fact foreign keys uniform or Zipf over 1..n_dim,
  a seeded fraction replaced by keys absent from the dimension, int64 payloads
  in [0, 1e7), then filtered by a seeded Bernoulli mask and compacted.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import torch

_CHUNK = 1 << 24


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=torch.device(device))
    g.manual_seed(int(seed) & 0x7FFFFFFFFFFFFFFF)
    return g


def _sub(seed: int, k: int) -> int:
    """Independent stream number ``k`` of a workload seed."""
    return int(seed) * 1000003 + k


def permutation(n: int, seed: int, device="cpu") -> torch.Tensor:
    """A uniformly random permutation of 0..n-1 (int64)."""
    return torch.randperm(n, generator=_gen(seed, device), device=device, dtype=torch.int64)


def uniform_ints(n: int, lo: int, hi: int, seed: int, device="cpu") -> torch.Tensor:
    """n integers uniform in [lo, hi) (int64)."""
    return torch.randint(lo, hi, (n,), generator=_gen(seed, device), device=device,
                         dtype=torch.int64)


def bernoulli_mask(n: int, p: float, seed: int, device="cpu") -> torch.Tensor:
    g = _gen(seed, device)
    out = torch.empty(n, dtype=torch.bool, device=device)
    for s in range(0, n, _CHUNK):
        e = min(n, s + _CHUNK)
        out[s:e] = torch.rand(e - s, generator=g, device=device, dtype=torch.float64) < p
    return out


def zipf_ranks(n_items: int, theta: float, count: int, seed: int, device="cpu") -> torch.Tensor:
    """``count`` 0-based ranks with P(rank = k) proportional to (k + 1)^-theta.

    theta = 0 is the uniform distribution. Sampled by inverting the cumulative
    distribution (fp64 prefix sums, binary search), chunked to bound memory.
    """
    if count == 0:
        return torch.empty(0, dtype=torch.int64, device=device)
    g = _gen(seed, device)
    if theta == 0.0:
        return torch.randint(0, n_items, (count,), generator=g, device=device, dtype=torch.int64)
    w = torch.arange(1, n_items + 1, dtype=torch.float64, device=device).pow_(-float(theta))
    cdf = torch.cumsum(w, 0)
    del w
    cdf /= cdf[-1].clone()
    out = torch.empty(count, dtype=torch.int64, device=device)
    for s in range(0, count, _CHUNK):
        e = min(count, s + _CHUNK)
        u = torch.rand(e - s, generator=g, device=device, dtype=torch.float64)
        out[s:e] = torch.searchsorted(cdf, u, right=True).clamp_(max=n_items - 1)
    return out


@dataclass
class JoinInput:
    """One join's columns. ``probe_keys`` etc. may live on any device."""

    build_keys: torch.Tensor
    build_pay: torch.Tensor | None
    probe_keys: torch.Tensor
    probe_pay: torch.Tensor | None
    desc: str

    @property
    def nb(self) -> int:
        return int(self.build_keys.numel())

    @property
    def np(self) -> int:
        return int(self.probe_keys.numel())

    def to(self, device) -> "JoinInput":
        mv = lambda t: None if t is None else t.to(device)
        return JoinInput(mv(self.build_keys), mv(self.build_pay), mv(self.probe_keys),
                         mv(self.probe_pay), self.desc)


def small_static(nb: int = 1 << 20, np_: int = 1 << 22, device="cpu") -> JoinInput:
    """Unique int32 build keys (permutation, seed 0), int32 payloads
    ``i ^ 0x5A5A5A5A``; probe keys uniform over 0..nb-1 (seed 1), payload = row."""
    bk = permutation(nb, 0, device).to(torch.int32)
    bp = (torch.arange(nb, device=device, dtype=torch.int64) ^ 0x5A5A5A5A).to(torch.int32)
    pk = uniform_ints(np_, 0, nb, 1, device).to(torch.int32)
    pp = torch.arange(np_, device=device, dtype=torch.int32)
    return JoinInput(bk, bp, pk, pp, f"small_static nb={nb} np={np_} int32")


def variant_sweep(nb: int, ratio: int, keys: str = "dense", theta: float = 0.0, seed: int = 0,
                  device="cpu", payload_bytes: int = 8) -> JoinInput:
    """Unique int64 build keys and probe keys drawn from them (see module doc)."""
    if keys not in ("dense", "random"):
        raise ValueError("keys must be 'dense' or 'random'")
    np_ = nb * ratio
    p = permutation(nb, _sub(seed, 0), device)
    if keys == "dense":
        base = int(uniform_ints(1, -(1 << 40), 1 << 40, _sub(seed, 1), "cpu")[0])
        bk = p + base
    else:
        bits = max(1, math.ceil(math.log2(max(nb, 2))))
        lim = 1 << (63 - bits)
        hi = uniform_ints(nb, -lim, lim, _sub(seed, 1), device)
        bk = hi * (1 << bits) + p
        del hi
    del p
    rowperm = permutation(nb, _sub(seed, 2), device)
    rank = zipf_ranks(nb, theta, np_, _sub(seed, 3), device)
    pk = bk[rowperm[rank]]
    del rank, rowperm
    pdt = torch.int64 if payload_bytes == 8 else torch.int32
    big = (1 << 62) if payload_bytes == 8 else (1 << 30)
    bp = uniform_ints(nb, -big, big, _sub(seed, 4), device).to(pdt)
    pp = uniform_ints(np_, -big, big, _sub(seed, 5), device).to(pdt)
    return JoinInput(bk, bp, pk, pp,
                     f"variant_sweep nb={nb} np={np_} keys={keys} theta={theta} int64")


def star_schema(n_dim: int = 150_000_000, n_fact: int = 600_000_000, theta: float = 0.0,
                absent: float = 0.10, selectivity: float = 1.0, seed: int = 0,
                device="cpu") -> JoinInput:
    """Dimension (build) and filtered fact (probe) sides of a foreign-key join."""
    dk = (permutation(n_dim, _sub(seed, 0), device) + 1).to(torch.int32)
    dp = uniform_ints(n_dim, 0, 1_000_000_000, _sub(seed, 1), device)
    fk = zipf_ranks(n_dim, theta, n_fact, _sub(seed, 2), device) + 1
    miss = bernoulli_mask(n_fact, absent, _sub(seed, 3), device)
    r = uniform_ints(n_fact, 0, n_dim, _sub(seed, 4), device)
    fk = torch.where(miss, n_dim + 1 + r, fk)
    del miss, r
    fp = uniform_ints(n_fact, 0, 10_000_000, _sub(seed, 5), device)
    if selectivity < 1.0:
        keep = bernoulli_mask(n_fact, selectivity, _sub(seed, 6), device)
        fk = fk[keep]
        fp = fp[keep]
        del keep
    return JoinInput(dk, dp, fk.to(torch.int32), fp,
                     f"star_schema dim={n_dim} fact={n_fact} theta={theta} sel={selectivity}")


@dataclass
class BatchInput:
    builds: list
    probes: list
    thetas: list

    @property
    def tuples(self) -> int:
        return sum(int(b.numel()) for b in self.builds) + sum(int(p.numel()) for p in self.probes)


def power_law_ranks(n: int, theta: float, count: int, g: torch.Generator, device) -> torch.Tensor:
    """0-based ranks with density proportional to (x + 1)^-theta on [0, n),
    by inverting the continuous power-law CDF (an approximation of Zipf)."""
    u = torch.rand(count, generator=g, device=device, dtype=torch.float64)
    if theta == 0.0:
        r = torch.floor(u * n)
    else:
        e = 1.0 - theta
        r = torch.floor((1.0 + u * ((n + 1.0) ** e - 1.0)) ** (1.0 / e)) - 1.0
    return r.clamp_(0, n - 1).to(torch.int64)


def batched_small(k: int = 4096, log2_lo: float = 10.0, log2_hi: float = 20.0, ratio: int = 4,
                  theta_max: float = 1.0, seed: int = 0, device="cpu") -> BatchInput:
    """k independent int32 joins of uneven sizes (see module doc)."""
    g = _gen(_sub(seed, 0), device)
    gc = _gen(_sub(seed, 1), "cpu")
    u = torch.rand(k, generator=gc, dtype=torch.float64)
    sizes = torch.floor(torch.pow(2.0, log2_lo + (log2_hi - log2_lo) * u)).to(torch.int64).tolist()
    thetas = (torch.rand(k, generator=gc, dtype=torch.float64) * theta_max).tolist()
    mults = (torch.randint(0, 1 << 31, (k,), generator=gc, dtype=torch.int64) * 2 + 1).tolist()
    adds = torch.randint(0, 1 << 32, (k,), generator=gc, dtype=torch.int64).tolist()
    builds, probes = [], []
    for j in range(k):
        nb = max(1, int(sizes[j]))
        i = torch.arange(nb, device=device, dtype=torch.int64)
        key = (i * mults[j] + adds[j]) & 0xFFFFFFFF
        key = torch.where(key >= (1 << 31), key - (1 << 32), key).to(torch.int32)
        rowperm = torch.randperm(nb, generator=g, device=device)
        rank = power_law_ranks(nb, thetas[j], ratio * nb, g, device)
        builds.append(key)
        probes.append(key[rowperm[rank]])
    return BatchInput(builds, probes, thetas)
