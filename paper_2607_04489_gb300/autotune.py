"""Autotuner of the batched join's launch shape.

Times eiger_join_batched, replayed from a CUDA graph, for every combination of
block threads x rows per work item x table load factor x the build size up to
which a join's table lives in shared memory (0: never) on seeded tuning
batches (seeds 10000 and up, disjoint from benchmark and test seeds): one of
joins of 2^10 to 2^20 build rows and one of small joins, and stores the best
combination with the GPU model it was tuned on in
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
SMALLS = (0, 1024, 2048)  # int32 joins: at most EIGER_BATCH_SMALL_MAX_I32


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


def pick(grid: list) -> dict:
    """Sets each entry's objective "rel", the mean over the batches of its time
    ("ms", one per batch) relative to that batch's fastest entry, and returns
    the entry with the smallest objective (the first one on ties)."""
    nb = len(grid[0]["ms"])
    best_ms = [min(r["ms"][i] for r in grid) for i in range(nb)]
    for r in grid:
        r["rel"] = round(sum(x / b for x, b in zip(r["ms"], best_ms)) / nb, 4)
    return min(grid, key=lambda r: r["rel"])


def tune(joins: int = 1024, seeds=(10000, 10001), out: str | None = None) -> dict:
    """Times every knob combination on two kinds of seeded batches: `joins`
    joins of 2^U(10,20) build rows, and 4 * `joins` small joins of 2^U(6,11)
    build rows (where the shared-memory tables matter). The objective is the
    mean over the batches of each batch's time relative to its fastest
    combination, so the small batch weighs as much as the large one."""
    batches = [workloads.batched_small(k=joins, seed=seeds[0], device="cuda"),
               workloads.batched_small(k=4 * joins, log2_lo=6.0, log2_hi=11.0, seed=seeds[1], device="cuda")]
    grid = []
    for bt, ch, lf, sm in itertools.product(BLOCKS, CHUNKS, LOADS, SMALLS):
        kn = eiger.BatchKnobs(bt, ch, lf, sm)
        ms = [time_knobs(b, kn) for b in batches]
        grid.append({"block_threads": bt, "chunk_rows": ch, "load_factor": lf, "small_rows": sm,
                     "ms": [round(x, 4) for x in ms]})
        torch.cuda.empty_cache()
    best = pick(grid)
    result = {
        "version": 3,
        "device": torch.cuda.get_device_name(),
        "tuned_on": f"batched_small k={joins} 2^U(10,20) seed {seeds[0]} and k={4 * joins} 2^U(6,11) "
                    f"seed {seeds[1]} (median replay ms; objective: mean time relative to each batch's best)",
        "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()),
        "knobs": {k: best[k] for k in ("block_threads", "chunk_rows", "load_factor", "small_rows")},
        "grid": grid,
    }
    path = out or os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned_batch.json")
    with open(path, "w") as f:
        json.dump(result, f, indent=1)
    return result


if __name__ == "__main__":
    r = tune(out=sys.argv[1] if len(sys.argv) > 1 else None)
    print(json.dumps(r["knobs"]))
