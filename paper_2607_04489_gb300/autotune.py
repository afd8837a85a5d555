"""Autotuner of the batched join's launch shape.

Times eiger_join_batched, replayed from a CUDA graph, for every combination of
block threads x rows per work item x table load factor on seeded tuning
batches (seeds 10000 and up, disjoint from benchmark and test seeds), and
stores the fastest combination with the GPU model it was tuned on in
``tuned_batch.json`` beside this file. ``BatchedJoin`` picks it up when no
knobs are given.

Usage (on the GPU): ``python -m paper_2607_04489_gb300.autotune [out.json]``.
"""

from __future__ import annotations

import itertools
import json
import os
import sys
import time

import torch

from . import eiger, workloads

BLOCKS = (128, 256, 512)
CHUNKS = (4096, 16384, 65536)
LOADS = (0.35, 0.5, 0.7)


def time_knobs(batch: workloads.BatchInput, knobs: eiger.BatchKnobs, reps: int = 3) -> float:
    """Median ms of `reps` graph replays of the whole batch."""
    bj = eiger.BatchedJoin(batch.builds, batch.probes, knobs=knobs)
    g = bj.capture()
    g.replay()
    torch.cuda.synchronize()
    if int(bj.status) != 0:
        raise RuntimeError(f"batched join failed with status {int(bj.status)}")
    times = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(reps):
        e0.record()
        g.replay()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    del g, bj
    return sorted(times)[len(times) // 2]


def tune(joins: int = 1024, seeds=(10000, 10001), out: str | None = None) -> dict:
    batches = [workloads.batched_small(k=joins, seed=s, device="cuda") for s in seeds]
    grid = []
    for bt, ch, lf in itertools.product(BLOCKS, CHUNKS, LOADS):
        kn = eiger.BatchKnobs(bt, ch, lf)
        ms = sum(time_knobs(b, kn) for b in batches)
        grid.append({"block_threads": bt, "chunk_rows": ch, "load_factor": lf, "ms": round(ms, 3)})
        torch.cuda.empty_cache()
    best = min(grid, key=lambda r: r["ms"])
    result = {
        "version": 1,
        "device": torch.cuda.get_device_name(),
        "tuned_on": f"batched_small k={joins} seeds={list(seeds)} (sum of median replay ms)",
        "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()),
        "knobs": {k: best[k] for k in ("block_threads", "chunk_rows", "load_factor")},
        "grid": grid,
    }
    path = out or os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned_batch.json")
    with open(path, "w") as f:
        json.dump(result, f, indent=1)
    return result


if __name__ == "__main__":
    r = tune(out=sys.argv[1] if len(sys.argv) > 1 else None)
    print(json.dumps(r["knobs"]))
