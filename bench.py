"""Benchmark of the adaptive equi-join on GB300.

One step = one eiger_join(AUTO) call on resident device inputs: build-side
statistics (min/max + HyperLogLog++), plan, radix partitioning of both sides,
the shared-memory join, and the match count readback. The default workload is
the largest variant-sweep join that fits the 32-bit tuple IDs at ratio 4:
nb = 2^28 unique dense int64 build keys (span < 2^32, so keys narrow to
uint32) and np = 2^30 probe keys drawn uniformly from them; output = the 2^30
(build_idx, probe_idx) pairs. Inputs (10.7 GB) exceed the L2 cache, so no
flush is needed between steps.

The headline `value` is timed with nothing but the calls between two CUDA
events. A second pass of the same steps then records per-launch CUDA events
(eiger_profile) for the stage breakdown and the roofline of the dominant
kernel. Also measured, on the same inputs: the static hash join (no
statistics, no narrowing, no partitioning: the single fixed method) and the
end-to-end call from pinned host buffers (keys copied in, pairs copied out,
every step).

Multi-GPU: replicas only (each rank joins its own seeded copy; no collective
on the data path); value = all ranks' tuples / the slowest rank's time.

``--impl reference`` times the CPU oracle (the unordered_multimap join plus
canonical sort, probe loop split over the host's cores) on a bounded sample
of the same workload.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "join tuples/s and HBM GB/s vs peak: adaptive vs static hash join"
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["eiger", "reference"], default="eiger")
    ap.add_argument("--log2-nb", type=int, default=28)
    ap.add_argument("--ratio", type=int, default=4)
    ap.add_argument("--keys", choices=["dense", "random"], default="dense")
    ap.add_argument("--theta", type=float, default=0.0)
    ap.add_argument("--variant", default="auto")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--copy-streams", type=int, default=1,
                    help="end to end: each host<->device copy is split over this many streams per direction")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-static", action="store_true")
    ap.add_argument("--selectivity", type=float, default=1.0, help="star workload: fact rows kept")
    ap.add_argument("--grid-sizes", default="20,22,24,26,28", help="grid workload: log2 build sizes")
    ap.add_argument("--grid-reps", type=int, default=3, help="grid workload: timed runs per plan")
    ap.add_argument("--workload", choices=["sweep", "batched", "wide", "groupby", "star", "grid", "small"],
                    default="sweep",
                    help="sweep: the headline join; batched: 4096 small joins in one launch; "
                         "wide: four columns per relation, the payloads materialised; "
                         "groupby: 2^28 rows, two aggregations, 2^--groups-log2 groups; "
                         "star: the 150M x 600M foreign-key join with the exact payload sum; "
                         "grid: the variant-sweep grid, every plan timed at every point (one JSON line each); "
                         "small: the 1M x 4M int32 static-join workload with the probe statistics")
    ap.add_argument("--groups-log2", type=int, default=20, help="groupby workload: log2 of the group count")
    ap.add_argument("--log2-rows", type=int, default=28, help="groupby workload: log2 of the rows")
    ap.add_argument("--key-bytes", type=int, choices=[4, 8], default=4, help="wide workload key/payload width")
    ap.add_argument("--batch-joins", type=int, default=4096)
    ap.add_argument("--batch-log2", default="10,20",
                    help="batched workload: build rows 2^U(lo,hi), given as lo,hi")
    ap.add_argument("--profile-steps", type=int, default=3,
                    help="steps of the separate per-launch profiling pass (stages, roofline)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value: float, world: int, device=None) -> float:
    """Largest value over ranks (the slowest rank's time); identity for 1 rank."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


# Source files that define each timed kernel (its own translation unit and the
# headers it includes); recorded ncu counters stay valid while these hash the same.
KERNEL_SOURCES = {
    "phj_join": ("phj.cu", "chunks.cuh", "emit.cuh", "common.cuh", "kernels.cuh"),
    "part_scatter": ("partition.cu", "common.cuh", "kernels.cuh"),
    "part_hist": ("partition.cu", "common.cuh", "kernels.cuh"),
}


def kernel_sources_digest(kernel: str) -> str | None:
    """Digest of the CUDA sources that define `kernel` (a stage name such as
    "phj_join" or "part_scatter.p1.probe"), to tell whether recorded ncu
    counters still describe the kernel that runs; None for an unlisted one."""
    import hashlib

    files = KERNEL_SOURCES.get(kernel.split(".")[0])
    if not files:
        return None
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2607_04489_gb300", "csrc")
    for name in files:
        h.update(name.encode())
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, workload: str | None):
    """DRAM bytes per launch of `kernel` in `workload` from
    profiles/dram_traffic.txt (lines: workload kernel bytes sources-digest),
    or None when there is no such entry or the kernel's sources changed since
    the counters were taken."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    try:
        with open(path) as f:
            rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    except OSError:
        return None
    for r in rows:
        if len(r) == 4 and (r[0], r[1]) == (workload, kernel) and r[3] == kernel_sources_digest(kernel):
            return float(r[2])
    return None


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": FALLBACK_HBM_GBS}, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.rows = []
        self.proc = None
        self.target = None
        try:
            import torch

            uuid = str(torch.cuda.get_device_properties(device_index).uuid)
            self.target = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
        except Exception:
            self.target = None

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "200"]
        if self.target:
            cmd += ["-i", self.target]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except OSError:
            self.proc = None
            return self
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = self.rows
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        num = lambda x: float(x) if x.replace(".", "", 1).isdigit() else float("nan")
        sm = [num(r[1]) for r in rows]
        mx = [num(r[2]) for r in rows]
        loaded = [s for s, r in zip(sm, rows) if num(r[3]) > 200] or sm
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i - 5] for r in rows for i in range(5, 9)
                          if r[i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(mx), "samples": len(rows),
                "power_w_max": max(num(r[3]) for r in rows), "reasons": reasons}


def sweep_traffic_key(args):
    """Which recorded ncu traffic applies to this run of the sweep workload:
    only the default sizes, keys and skew were captured."""
    if (args.ratio, args.keys, args.theta) != (4, "dense", 0.0):
        return None
    key = {"auto": "sweep", "smj": "smj"}.get(args.variant)
    return None if key is None else f"{key}{args.log2_nb}"


def workload_desc(args):
    nb = 1 << args.log2_nb
    return (f"variant_sweep join: nb=2^{args.log2_nb} unique {args.keys} int64 build keys, "
            f"np={args.ratio}*nb probe keys drawn from them (zipf theta={args.theta}), "
            f"output (build_idx, probe_idx) pairs"), nb, nb * args.ratio


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def _oracle_leg(bk, pk, threads, min_seconds, max_runs=64):
    import oracle

    runs, t0 = 0, time.perf_counter()
    while True:
        if threads == 1:
            oracle.join(bk, pk)
        else:
            oracle.join_mt(bk, pk, threads)
        runs += 1
        el = time.perf_counter() - t0
        if el >= min_seconds or runs >= max_runs:
            break
    return runs * (bk.size + pk.size) / el, runs, el


def cpu_oracle_sample(args, min_seconds=10.0):
    """The oracle, as it stands, on a bounded sample of the workload: once on
    all host cores (the probe loop split, -t N) and once on one thread."""
    from paper_2607_04489_gb300 import workloads

    log2 = min(args.log2_nb, 20)
    w = workloads.variant_sweep(1 << log2, args.ratio, keys=args.keys, theta=args.theta, seed=0,
                                device="cpu", payload_bytes=8)
    bk, pk = w.build_keys.numpy(), w.probe_keys.numpy()
    cores = host_cores()
    tn, rn, en = _oracle_leg(bk, pk, cores, min_seconds)
    t1, r1, e1 = _oracle_leg(bk, pk, 1, min_seconds)
    sample = f"nb=2^{log2}, np={args.ratio}*2^{log2}, same key/probe distribution"
    return {"value": tn, "unit": "tuples/s", "cores": cores, "kind": "oracle",
            "sample": f"{sample}; {rn} run(s) of the full join with canonical pair sort in {en:.1f} s, "
                      f"probe loop split over {cores} threads (multimap build and sort on one)",
            "one_thread": {"value": t1, "unit": "tuples/s", "cores": 1,
                           "sample": f"{sample}; {r1} run(s) in {e1:.1f} s"}}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2607_04489_gb300 import workloads

    desc, nb, np_ = workload_desc(args)
    log2 = min(args.log2_nb, 20)
    w = workloads.variant_sweep(1 << log2, args.ratio, keys=args.keys, theta=args.theta, seed=0,
                                device="cpu", payload_bytes=8)
    bk, pk = w.build_keys.numpy(), w.probe_keys.numpy()
    cores = host_cores()
    import oracle

    for _ in range(args.warmup):
        oracle.join_mt(bk, pk, cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.join_mt(bk, pk, cores)
    el = time.perf_counter() - t0
    tput = args.steps * (bk.size + pk.size) / el
    sample = (f"nb=2^{log2}, np={args.ratio}*2^{log2} per step (bounded sample of the workload), "
              f"probe loop split over {cores} threads")
    line = {"impl": "reference", "metric": METRIC, "value": tput, "unit": "tuples/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": desc, "nb": nb, "np": np_},
            "cpu_baseline": {"value": tput, "unit": "tuples/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": tput, "unit": "tuples/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_eiger(args):
    import torch

    from paper_2607_04489_gb300 import eiger, workloads

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    eiger.load()
    desc, nb, np_ = workload_desc(args)
    w = workloads.variant_sweep(nb, args.ratio, keys=args.keys, theta=args.theta, seed=rank,
                                device=dev, payload_bytes=8)
    w.build_pay = w.probe_pay = None
    torch.cuda.empty_cache()
    # Everything below runs on one created (non-blocking) stream rather than
    # the legacy default stream, whose implicit synchronisation would tie the
    # joins to the end-to-end copies' streams.
    torch.cuda.synchronize(dev)
    torch.cuda.set_stream(torch.cuda.Stream(dev))
    bk, pk = w.build_keys, w.probe_keys
    out_b = torch.empty(np_, dtype=torch.int32, device=dev)
    out_p = torch.empty(np_, dtype=torch.int32, device=dev)
    ws = torch.empty(eiger.join_workspace(nb, np_, eiger.I64, args.variant), dtype=torch.uint8,
                     device=dev)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def step(variant, workspace):
        st, cnt, plan = eiger.join_into(bk, pk, variant=variant, out_bidx=out_b, out_pidx=out_p,
                                        capacity=np_, workspace=workspace, stream=stream)
        if st != eiger.OK or cnt != np_:
            raise RuntimeError(f"join failed: status {st}, count {cnt}: {eiger.last_error()}")
        return plan

    def timed(variant, workspace, steps):
        barrier(world)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(steps):
            plan = step(variant, workspace)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier(world)
        return max_over_ranks(e0.elapsed_time(e1) / steps, world, dev), plan

    # ---- adaptive join: warm-up, then the timed region (nothing but the calls)
    for _ in range(args.warmup):
        plan = step(args.variant, ws)
    sampler = ClockSampler(local).start()
    ms_step, plan = timed(args.variant, ws, args.steps)
    clocks = sampler.stop()
    tuples = world * (nb + np_)
    value = tuples / (ms_step * 1e-3)

    # ---- the same steps again with per-launch CUDA events (stage breakdown)
    stages = {}
    launches = 0
    eiger.profile(True)
    barrier(world)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(args.profile_steps):
        step(args.variant, ws)
        for name, ms, nl, by in eiger.profile_read():
            s_ = stages.setdefault(name, [0.0, 0.0, 0])
            s_[0] += ms
            s_[1] += by
            s_[2] += 1
            launches += nl
    e1.record(stream)
    torch.cuda.synchronize(dev)
    eiger.profile(False)
    ms_prof = e0.elapsed_time(e1) / max(1, args.profile_steps)
    launches_per_step = launches // max(1, args.profile_steps)

    # ---- the static hash join on the same inputs
    static = None
    if not args.no_static:
        del ws
        torch.cuda.empty_cache()
        ws_s = torch.empty(eiger.join_workspace(nb, np_, eiger.I64, "static"), dtype=torch.uint8,
                           device=dev)
        for _ in range(args.warmup):
            step("static", ws_s)
        sms, _ = timed("static", ws_s, args.steps)
        static = {"value": tuples / (sms * 1e-3), "unit": "tuples/s", "ms_per_step": sms,
                  "speedup_of_adaptive": sms / ms_step}
        del ws_s
        torch.cuda.empty_cache()
        ws = torch.empty(eiger.join_workspace(nb, np_, eiger.I64, args.variant), dtype=torch.uint8,
                         device=dev)

    # ---- end to end from pinned host buffers. Every step copies its own keys
    # in and its pairs out (torch copies on two extra streams around the
    # device-pointer C-ABI call, eiger_join); consecutive steps are pipelined
    # with double-buffered device arrays, as a caller streaming batches would
    # run them: step i+1's upload and step i-1's download overlap step i's
    # join. The downloads of all steps land in one pinned host pair (copies on
    # one stream run in order).
    e2e = None
    if not args.no_e2e:
        hb = torch.empty(nb, dtype=bk.dtype, pin_memory=True)
        hp = torch.empty(np_, dtype=pk.dtype, pin_memory=True)
        hb.copy_(bk)
        hp.copy_(pk)
        hob = torch.empty(np_, dtype=torch.int32, pin_memory=True)
        hop = torch.empty(np_, dtype=torch.int32, pin_memory=True)
        dbk = [bk, torch.empty_like(bk)]
        dpk = [pk, torch.empty_like(pk)]
        dob = [out_b, torch.empty_like(out_b)]
        dop = [out_p, torch.empty_like(out_p)]
        # each direction's copies are split into --copy-streams chunks on as
        # many streams, so several copy engines run at once
        cs = max(1, args.copy_streams)
        h2ds = [torch.cuda.Stream(dev) for _ in range(cs)]
        d2hs = [torch.cuda.Stream(dev) for _ in range(cs)]
        h2d, d2h = h2ds[0], d2hs[0]
        up_done = [[torch.cuda.Event() for _ in range(cs)] for _ in range(2)]
        join_done = [torch.cuda.Event() for _ in range(2)]
        down_done = [[torch.cuda.Event() for _ in range(cs)] for _ in range(2)]

        def split_copy(streams, done, pairs, after):
            for q, s_ in enumerate(streams):
                s_.wait_event(after)
                with torch.cuda.stream(s_):
                    for dst, src in pairs:
                        dst.chunk(cs)[q].copy_(src.chunk(cs)[q], non_blocking=True)
                done[q].record(s_)

        def upload(slot):
            # after the join that last read this slot
            split_copy(h2ds, up_done[slot], [(dbk[slot], hb), (dpk[slot], hp)], join_done[slot])

        def run_steps(n):
            for q in range(2):
                join_done[q].record(stream)
                for ev in down_done[q]:
                    ev.record(stream)
            upload(0)
            for i in range(n):
                slot = i & 1
                if i + 1 < n:
                    upload(slot ^ 1)
                for ev in up_done[slot]:
                    stream.wait_event(ev)
                for ev in down_done[slot]:
                    stream.wait_event(ev)  # its output arrays were copied out
                st, cnt, _ = eiger.join_into(dbk[slot], dpk[slot], variant=args.variant, out_bidx=dob[slot],
                                             out_pidx=dop[slot], capacity=np_, workspace=ws, stream=stream)
                if st != eiger.OK or cnt != np_:
                    raise RuntimeError(f"join failed: {eiger.last_error()}")
                join_done[slot].record(stream)
                split_copy(d2hs, down_done[slot], [(hob, dob[slot]), (hop, dop[slot])], join_done[slot])

        run_steps(max(2, args.warmup))
        torch.cuda.synchronize(dev)
        barrier(world)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(h2d)
        for s_ in h2ds[1:] + d2hs + [stream]:
            s_.wait_stream(h2d)  # nothing of the timed steps starts before t0
        run_steps(args.steps)
        for q in range(2):
            for ev in down_done[q]:
                d2h.wait_event(ev)
            d2h.wait_event(join_done[q])
        t1.record(d2h)
        torch.cuda.synchronize(dev)
        barrier(world)
        ems = max_over_ranks(t0.elapsed_time(t1) / args.steps, world, dev)
        e2e = {"value": tuples / (ems * 1e-3), "unit": "tuples/s", "ms_per_step": ems,
               "h2d_bytes_per_step": int(bk.numel() * 8 + pk.numel() * 8),
               "d2h_bytes_per_step": int(2 * 4 * np_),
               "through": "torch copies from/to pinned host memory around the device-pointer C-ABI call "
                          "eiger_join (the ABI takes device pointers)",
               "copy_streams_per_direction": cs,
               "pipelining": "upload of step i+1 and download of step i-1 overlap the join of step i"}
        del dbk[1], dpk[1], dob[1], dop[1], hb, hp, hob, hop

    # ---- roofline of the dominant stage (from the profiling pass)
    peaks, peak_src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS))
    stage_rows = stage_table(stages, max(1, args.profile_steps))
    dom = stage_rows[0] if stage_rows else {"stage": None, "gbs": 0.0, "bytes": 0.0}
    compulsory = nb * 8 + np_ * 8 + np_ * 8  # keys in, pairs out
    line = {
        "metric": METRIC, "value": value, "unit": "tuples/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        "config": {"workload": desc, "nb": nb, "np": np_, "keys": args.keys, "theta": args.theta,
                   "variant": args.variant,
                   "l2": f"inputs ({(nb + np_) * 8 / 1e9:.1f} GB) larger than L2; no flush",
                   "parallelism": f"replicas x{world}"},
        "hbm_gbs_compulsory": compulsory / (ms_step * 1e-3) / 1e9,
        "plan": {"variant": plan.variant, "bits1": plan.bits1, "bits2": plan.bits2,
                 "narrow": plan.narrow, "load_factor": plan.load_factor},
        "roofline": {"bound": "hbm", "kernel": dom["stage"], "achieved": dom["gbs"], "peak": hbm,
                     "peak_source": peak_src, "unit": "GB/s", "frac": dom["gbs"] / hbm,
                     "traffic": recorded_traffic(dom["stage"], sweep_traffic_key(args)),
                     "algorithmic_bytes": dom["bytes"],
                     "timing": f"CUDA events around each launch on its stream, {args.profile_steps} "
                               "profiled steps after the timed region"},
        "stages": stage_rows,
        "profiled_ms_per_step": ms_prof,
        "gpu_launches": launches_per_step * args.steps,
        "static": static,
        "e2e": e2e,
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_oracle_sample(args)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def run_batched(args):
    """Independent int32 joins (default 4096, build 2^U(10,20) rows, probe 4x,
    per-join skew): one eiger_join_batched call replayed from a CUDA graph,
    against the same joins with every table in global memory (small joins'
    shared-memory tables off) and as sequential static eiger_join calls."""
    import torch

    from paper_2607_04489_gb300 import eiger, workloads

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    eiger.load()
    lo, hi = (float(x) for x in args.batch_log2.split(","))
    w = workloads.batched_small(k=args.batch_joins, log2_lo=lo, log2_hi=hi, seed=rank, device=dev)
    tuples = w.tuples
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def time_batch(knobs, steps, sample_clocks=False):
        bj = eiger.BatchedJoin(w.builds, w.probes, knobs=knobs)
        graph = bj.capture()
        for _ in range(args.warmup):
            graph.replay()
        sampler = ClockSampler(local).start() if sample_clocks else None
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(steps):
            graph.replay()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        clocks = sampler.stop() if sampler else None
        if int(bj.status) != 0 or bj.counts[: bj.k].cpu().tolist() != [p.numel() for p in w.probes]:
            raise RuntimeError(f"batched join failed: status {int(bj.status)}")
        return bj, e0.elapsed_time(e1) / steps, clocks

    bj, ms, clocks = time_batch(None, args.steps, sample_clocks=True)
    # the same batch with every join's table in global memory
    knobs_global = eiger.BatchKnobs(**{**vars(bj.knobs), "small_rows": 0})
    _, gms, _ = time_batch(knobs_global, max(1, min(args.steps, 3)))
    global_only = {"value": tuples / (gms * 1e-3), "unit": "tuples/s", "ms_per_step": gms,
                   "knobs": vars(knobs_global), "speedup_of_batched": gms / ms}
    # the same joins as sequential static calls, each synchronising for its count
    seq_steps = 0 if args.no_static else max(1, min(args.steps, 2))
    sequential = None
    if seq_steps:
        ws = torch.empty(max(eiger.join_workspace(b.numel(), p.numel(), eiger.I32, "static")
                             for b, p in zip(w.builds, w.probes)), dtype=torch.uint8, device=dev)
        def seq():
            for j, (b, p) in enumerate(zip(w.builds, w.probes)):
                a = int(bj.off[j])
                st, n, _ = eiger.join_into(b, p, variant="static", out_bidx=bj.out_bidx[a:],
                                           out_pidx=bj.out_pidx[a:], capacity=bj.capacities[j],
                                           workspace=ws, stream=stream)
                if st != eiger.OK:
                    raise RuntimeError(eiger.last_error())
        seq()
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(seq_steps):
            seq()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        sms = e0.elapsed_time(e1) / seq_steps
        sequential = {"value": tuples / (sms * 1e-3), "unit": "tuples/s", "ms_per_step": sms,
                      "speedup_of_batched": sms / ms}
    lo_s, hi_s = (f"{x:g}" for x in (lo, hi))
    line = {"metric": METRIC, "value": tuples / (ms * 1e-3), "unit": "tuples/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": f"batched: {args.batch_joins} int32 joins, build 2^U({lo_s},{hi_s}) rows, "
                                   "probe 4x build, per-join power-law skew U(0,1); one graph replay",
                       "joins": args.batch_joins, "tuples": tuples,
                       "knobs": vars(bj.knobs) if hasattr(bj.knobs, "__dict__") else str(bj.knobs)},
            "global_tables_only": global_only,
            "sequential_static": sequential,
            "roofline": batch_roofline(w, ms),
            # setup, the persistent join kernel, the small joins' kernel, status
            "gpu_launches": (4 if bj.knobs.small_rows > 0 else 3) * args.steps, "clocks": clocks}
    if rank == 0:
        print(json.dumps(line))
    return 0


def batch_roofline(w, ms):
    """Compulsory bytes of one replay of the batch (every 4-byte build and
    probe key read once, one 8-byte pair written per match; every probe row of
    this workload matches once) over the whole replay's time, which also holds
    the setup and status launches and the small joins' kernel: a lower bound
    on batch_join's own bandwidth."""
    peaks, src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS))
    nb = sum(int(b.numel()) for b in w.builds)
    np_ = sum(int(p.numel()) for p in w.probes)
    by = 4.0 * (nb + np_) + 8.0 * np_
    gbs = by / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": "batch_join", "achieved": gbs, "peak": hbm, "peak_source": src,
            "unit": "GB/s", "frac": gbs / hbm, "traffic": None, "algorithmic_bytes": by,
            "timing": "CUDA events around whole graph replays (batch_join, batch_small when small "
                      "joins run in shared memory, and the setup and status launches)"}


def profile_pass(step, steps):
    """Per-launch CUDA-event stage times of `steps` more calls of `step`,
    after the timed region (which runs without the events): name ->
    [ms, bytes, entries] summed over the steps, and the launches."""
    from paper_2607_04489_gb300 import eiger

    stages, launches = {}, 0
    eiger.profile(True)
    try:
        for _ in range(steps):
            step()
            for name, ms, nl, by in eiger.profile_read():
                st_ = stages.setdefault(name, [0.0, 0.0, 0])
                st_[0] += ms
                st_[1] += by
                st_[2] += 1
                launches += nl
    finally:
        eiger.profile(False)
    return stages, launches


def stage_table(stages, steps):
    """Per-step device time and algorithmic bytes of each named stage (a name
    that occurs several times in a step, like the statistics of the build side
    and of a probe sample, adds up), sorted by time."""
    rows = []
    for name, (ms_tot, by_tot, cnt) in stages.items():
        ms_avg, by_avg = ms_tot / steps, by_tot / steps
        rows.append({"stage": name, "ms": round(ms_avg, 4), "bytes": by_avg,
                     "gbs": by_avg / (ms_avg * 1e-3) / 1e9 if ms_avg > 0 else None})
    rows.sort(key=lambda r: -r["ms"])
    return rows


def run_small(args):
    """The small static-join workload: 2^20 unique int32 build keys (a
    permutation), 2^22 uniform probe keys over them (every probe row matches
    once), and eiger_stats on the probe keys. AUTO and the static join are
    timed per call; the CPU oracle runs the same full join (canonical pair
    sort included) on all host cores and on one."""
    import torch

    from paper_2607_04489_gb300 import eiger, workloads

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    eiger.load()
    wc = workloads.small_static(1 << 20, 1 << 22, device="cpu")
    bk, pk = wc.build_keys.to(dev), wc.probe_keys.to(dev)
    nb, np_ = bk.numel(), pk.numel()
    ob = torch.empty(np_, dtype=torch.int32, device=dev)
    op = torch.empty_like(ob)
    torch.cuda.synchronize(dev)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / args.steps

    arms = {}
    for variant in ("auto", "static"):
        ws = torch.empty(eiger.join_workspace(nb, np_, eiger.I32, variant), dtype=torch.uint8, device=dev)
        holder = {}

        def call():
            st, cnt, plan = eiger.join_into(bk, pk, variant=variant, out_bidx=ob, out_pidx=op, capacity=np_,
                                            workspace=ws, stream=stream)
            if st != eiger.OK or cnt != np_:
                raise RuntimeError(f"join failed: {eiger.last_error()}")
            holder["plan"] = plan

        ms = timed(call)
        arms[variant] = {"ms_per_step": ms, "value": (nb + np_) / (ms * 1e-3), "unit": "tuples/s",
                         "plan": f"{holder['plan'].variant} {holder['plan'].bits1}+{holder['plan'].bits2}"}
    sws = torch.empty(eiger.stats_workspace(np_, eiger.I32), dtype=torch.uint8, device=dev)
    sms = timed(lambda: eiger.stats(pk, workspace=sws, stream=stream))
    import oracle

    b, p = wc.build_keys.numpy(), wc.probe_keys.numpy()
    cores = host_cores()
    tn, rn, en = _oracle_leg(b, p, cores, 3.0, max_runs=8)
    t1, r1, e1_ = _oracle_leg(b, p, 1, 3.0, max_runs=8)
    ms = arms["auto"]["ms_per_step"]
    line = {"metric": METRIC, "value": arms["auto"]["value"], "unit": "tuples/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "small static join: 2^20 unique int32 build keys (permutation), 2^22 "
                                   "uniform probe keys over them; eiger_stats on the probe keys",
                       "l2": "inputs (20 MB) fit L2: the 60 % HBM target does not apply"},
            "arms": arms, "static_speedup_of_auto": arms["static"]["ms_per_step"] / ms,
            "probe_stats_ms": sms,
            "cpu_baseline": {"value": tn, "unit": "tuples/s", "cores": cores, "kind": "oracle",
                             "sample": f"the whole workload; {rn} run(s) with canonical pair sort in {en:.1f} s",
                             "one_thread": {"value": t1, "unit": "tuples/s", "cores": 1,
                                            "sample": f"the whole workload; {r1} run(s) in {e1_:.1f} s"}}}
    print(json.dumps(line))
    return 0


def grid_plans(nb: int, auto_plan):
    """Forced plans timed at one variant-sweep point besides AUTO and STATIC:
    the non-partitioned join, one pass of 6, 8, 10 and 12 radix bits, and two
    passes of the AUTO plan's total bits and one bit fewer or more (split as
    the rules split them). Plans whose average build partition would exceed
    four shared-memory tables (each further table re-streams the probe
    partition) are listed with a reason instead of being timed."""
    from paper_2607_04489_gb300 import eiger

    limit = 4 * 4096
    out = [("nphj", eiger.Plan("nphj", narrow=auto_plan.narrow))]
    for b in (6, 8, 10, 12):
        out.append((f"phj1-{b}", eiger.Plan("phj1", b, 0, auto_plan.narrow) if nb >> b <= limit else None))
    tot = auto_plan.bits1 + auto_plan.bits2 if auto_plan.variant == "phj2" else \
        auto_plan.bits1 if auto_plan.variant == "phj1" else max(2, (nb // 2048).bit_length())
    for t in (tot - 1, tot, tot + 1):
        if 2 <= t <= 24:
            b1 = t // 2
            plan = eiger.Plan("phj2", b1, t - b1, auto_plan.narrow)
            out.append((f"phj2-{b1}+{t - b1}", plan if nb >> t <= limit else None))
    return out


def run_grid(args):
    """The variant-sweep grid: build sizes 2^k (--grid-sizes), probe ratio 1,
    4 and 16, dense (narrowable) and random 64-bit keys, probe skew theta 0,
    0.5, 1 and 1.5. At every point AUTO (statistics and plan included), the
    static join and the forced plans of grid_plans are each timed
    --grid-reps times after one warm-up call (the minimum is reported, as the
    paper reports minima); AUTO's regret is its time over the fastest plan's.
    Points whose probe side needs 32-bit tuple IDs beyond 2^32 - 1 rows are
    skipped. One JSON line per point."""
    import torch

    from paper_2607_04489_gb300 import eiger, workloads

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    eiger.load()
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for log2 in [int(x) for x in args.grid_sizes.split(",")]:
        for ratio in (1, 4, 16):
            nb = 1 << log2
            np_ = nb * ratio
            if np_ >= (1 << 32):
                continue
            for keys in ("dense", "random"):
                for theta in (0.0, 0.5, 1.0, 1.5):
                    w = workloads.variant_sweep(nb, ratio, keys=keys, theta=theta, seed=0, device=dev,
                                                payload_bytes=8)
                    w.build_pay = w.probe_pay = None
                    torch.cuda.empty_cache()
                    bk, pk = w.build_keys, w.probe_keys
                    ob = torch.empty(np_, dtype=torch.int32, device=dev)
                    op = torch.empty(np_, dtype=torch.int32, device=dev)

                    def timed(variant, knobs):
                        ws = torch.empty(eiger.join_workspace(nb, np_, eiger.I64, variant, knobs),
                                         dtype=torch.uint8, device=dev)
                        best, plan = float("inf"), None
                        for rep in range(args.grid_reps + 1):
                            e0.record(stream)
                            st, cnt, plan = eiger.join_into(bk, pk, variant=variant, knobs=knobs, out_bidx=ob,
                                                            out_pidx=op, capacity=np_, workspace=ws,
                                                            stream=stream)
                            e1.record(stream)
                            torch.cuda.synchronize(dev)
                            if st != eiger.OK or cnt != np_:
                                raise RuntimeError(f"{variant} {knobs}: status {st}, count {cnt}: "
                                                   f"{eiger.last_error()}")
                            if rep:
                                best = min(best, e0.elapsed_time(e1))
                        del ws
                        return best, plan

                    auto_ms, auto_plan = timed("auto", None)
                    static_ms, _ = timed("static", None)
                    times = {"auto": auto_ms, "static": static_ms}
                    skipped = []
                    for name, knobs in grid_plans(nb, auto_plan):
                        if knobs is None:
                            skipped.append(name)
                            continue
                        times[name], _ = timed(knobs.variant, knobs)
                    forced = {k: v for k, v in times.items() if k not in ("auto",)}
                    best_name = min(forced, key=forced.get)
                    print(json.dumps({
                        "nb": nb, "np": np_, "keys": keys, "theta": theta,
                        "auto_plan": f"{auto_plan.variant} {auto_plan.bits1}+{auto_plan.bits2} "
                                     f"narrow={auto_plan.narrow}",
                        "ms": {k: round(v, 4) for k, v in times.items()},
                        "best": best_name, "auto_regret": round(auto_ms / forced[best_name] - 1.0, 4),
                        "auto_vs_static": round(static_ms / auto_ms, 3),
                        "auto_tuples_per_s": (nb + np_) / (auto_ms * 1e-3),
                        "skipped": skipped}), flush=True)
                    del w, bk, pk, ob, op
                    torch.cuda.empty_cache()
    return 0


def run_wide(args):
    """The wide join (Sec. 5.2: four columns per relation, the three non-key
    columns of both sides materialised for every match): nb unique dense keys,
    np = ratio * nb probe keys drawn from them, `--key-bytes` wide keys and
    payloads. Arms: AUTO (its plan, payloads carried through the partitioning
    passes, GFTR), the same plan gathering by tuple ID (GFUR), the sort-merge
    join with both strategies, and the non-partitioned and static joins
    (GFUR only)."""
    import torch

    from paper_2607_04489_gb300 import eiger, workloads

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    eiger.load()
    nb = 1 << args.log2_nb
    np_ = nb * args.ratio
    kt = torch.int32 if args.key_bytes == 4 else torch.int64
    w = workloads.variant_sweep(nb, args.ratio, keys="dense", theta=args.theta, seed=rank, device=dev)
    base = int(w.build_keys.min())
    bk = (w.build_keys - base).to(kt) if kt == torch.int32 else w.build_keys
    pk = (w.probe_keys - base).to(kt) if kt == torch.int32 else w.probe_keys
    del w
    big = 1 << (30 if args.key_bytes == 4 else 62)
    bcols = [workloads.uniform_ints(nb, -big, big, 100 + c, dev).to(kt) for c in range(3)]
    pcols = [workloads.uniform_ints(np_, -big, big, 200 + c, dev).to(kt) for c in range(3)]
    bout = [torch.empty(np_, dtype=kt, device=dev) for _ in range(3)]
    pout = [torch.empty(np_, dtype=kt, device=dev) for _ in range(3)]
    torch.cuda.empty_cache()
    stream = torch.cuda.current_stream(dev)
    dt = eiger.I32 if kt == torch.int32 else eiger.I64
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def arm(variant, mat, knobs=None, profile=False):
        ws = torch.empty(eiger.join_wide_workspace(nb, np_, dt, bcols, pcols, variant, mat, knobs),
                         dtype=torch.uint8, device=dev)

        def step():
            st, cnt, plan = eiger.join_wide_into(bk, pk, bcols, pcols, bout, pout, variant=variant,
                                                 materialize=mat, knobs=knobs, capacity=np_, workspace=ws,
                                                 stream=stream)
            if st != eiger.OK or cnt != np_:
                raise RuntimeError(f"wide join failed: status {st}, count {cnt}: {eiger.last_error()}")
            return plan

        for _ in range(args.warmup):
            plan = step()
        barrier(world)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(args.steps):
            plan = step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier(world)
        ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)
        stages, launches = profile_pass(step, args.steps) if profile else ({}, 0)
        del ws
        torch.cuda.empty_cache()
        return ms, plan, stages, launches

    tuples = world * (nb + np_)
    sampler = ClockSampler(local).start()
    ms, plan, stages, launches = arm("auto", "auto", profile=True)
    clocks = sampler.stop()
    same = eiger.Plan(plan.variant, plan.bits1, plan.bits2, plan.narrow, plan.load_factor)
    arms = {}
    for name, variant, mat, knobs in (("auto_plan_gfur", plan.variant, "gfur", same),
                                      ("smj_gftr", "smj", "gftr", None), ("smj_gfur", "smj", "gfur", None),
                                      ("nphj_gfur", "nphj", "gfur", None), ("static_gfur", "static", "gfur", None)):
        if variant == "static":
            knobs = None
        ams, aplan, _, _ = arm(variant, mat, knobs)
        arms[name] = {"ms_per_step": ams, "value": tuples / (ams * 1e-3), "unit": "tuples/s",
                      "plan": f"{aplan.variant}/{aplan.bits1}/{aplan.bits2}/{aplan.materialize}"}
    peaks, peak_src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS))
    rows = stage_table(stages, args.steps)
    dom = rows[0]
    line = {"metric": METRIC, "value": tuples / (ms * 1e-3), "unit": "tuples/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32" if kt == torch.int32 else "int64",
            "data": "synthetic",
            "config": {"workload": f"wide join: nb=2^{args.log2_nb} unique dense keys, np={args.ratio}*nb "
                                   f"drawn from them (zipf theta={args.theta}), {args.key_bytes}-byte keys and "
                                   "3 payload columns per side, all 6 payloads materialised per match",
                       "nb": nb, "np": np_, "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2; no flush"},
            "plan": {"variant": plan.variant, "bits1": plan.bits1, "bits2": plan.bits2,
                     "materialize": plan.materialize},
            "roofline": {"bound": "hbm", "kernel": dom["stage"], "achieved": dom["gbs"], "peak": hbm,
                         "peak_source": peak_src, "unit": "GB/s", "frac": dom["gbs"] / hbm,
                         "traffic": recorded_traffic(dom["stage"], "wide" if (args.log2_nb, args.ratio,
                                                     args.key_bytes) == (26, 4, 4) else None),
                         "algorithmic_bytes": dom["bytes"]},
            "stages": rows, "arms": arms, "gpu_launches": launches, "clocks": clocks}
    if rank == 0:
        print(json.dumps(line))
    return 0


def run_groupby(args):
    """Group-by microbenchmark (Sec. 5.4: 2^28 rows, two aggregations, 4-byte
    keys and payloads, g groups): keys are g distinct values drawn uniformly,
    aggregates SUM(v1) and MAX(v2). Arms: AUTO (statistics pick the algorithm
    and size the table; its time includes the statistics), HASH and
    PARTITION forced."""
    import torch

    from paper_2607_04489_gb300 import eiger, workloads

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    eiger.load()
    n = 1 << args.log2_rows
    g = 1 << args.groups_log2
    vals = (workloads.permutation(g, 300 + rank, dev) * 3).to(torch.int32)
    keys = vals[workloads.uniform_ints(n, 0, g, 301 + rank, dev)]
    del vals
    v1 = workloads.uniform_ints(n, -(1 << 30), 1 << 30, 302 + rank, dev).to(torch.int32)
    v2 = workloads.uniform_ints(n, -(1 << 30), 1 << 30, 303 + rank, dev).to(torch.int32)
    aggs = [("sum", v1), ("max", v2)]
    cap = min(n, 2 * g + 1024)
    out_k = torch.empty(cap, dtype=torch.int32, device=dev)
    outs = [torch.empty(cap, dtype=torch.int64, device=dev) for _ in aggs]
    torch.cuda.empty_cache()
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def arm(variant, profile=False):
        ws = torch.empty(eiger.groupby_workspace(n, eiger.I32, aggs, variant), dtype=torch.uint8, device=dev)

        def step():
            st, cnt, plan = eiger.groupby_into(keys, aggs, out_k, outs, variant=variant, capacity=cap,
                                               workspace=ws, stream=stream)
            if st != eiger.OK:
                raise RuntimeError(f"group-by failed: status {st}: {eiger.last_error()}")
            return plan, cnt

        for _ in range(args.warmup):
            plan, cnt = step()
        barrier(world)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(args.steps):
            plan, cnt = step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier(world)
        ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)
        stages, launches = profile_pass(step, args.steps) if profile else ({}, 0)
        del ws
        torch.cuda.empty_cache()
        return ms, plan, cnt, stages, launches

    tuples = world * n
    sampler = ClockSampler(local).start()
    ms, plan, groups, stages, launches = arm("auto", profile=True)
    clocks = sampler.stop()
    arms = {}
    for v in ("hash", "partition"):
        ams, aplan, acnt, _, _ = arm(v)
        if acnt != groups:
            raise RuntimeError(f"{v}: {acnt} groups, auto found {groups}")
        arms[v] = {"ms_per_step": ams, "value": tuples / (ams * 1e-3), "unit": "rows/s",
                   "plan": f"{aplan.variant}/{aplan.bits1}/{aplan.bits2}/{aplan.table_slots}"}
    peaks, peak_src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS))
    rows = stage_table(stages, args.steps)
    dom = rows[0]
    line = {"metric": "group-by rows/s: HLL-guided choice vs hash and partition", "value": tuples / (ms * 1e-3),
            "unit": "rows/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": f"group-by: 2^{args.log2_rows} int32 rows over 2^{args.groups_log2} uniform "
                                   "groups, SUM and MAX of two int32 columns",
                       "rows": n, "groups": groups, "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2; no flush"},
            "plan": {"variant": plan.variant, "bits1": plan.bits1, "bits2": plan.bits2,
                     "table_slots": plan.table_slots, "estimate": plan.estimate},
            "roofline": {"bound": "hbm", "kernel": dom["stage"], "achieved": dom["gbs"], "peak": hbm,
                         "peak_source": peak_src, "unit": "GB/s", "frac": dom["gbs"] / hbm,
                         "traffic": recorded_traffic(dom["stage"], f"groupby{args.groups_log2}"
                                                     if args.log2_rows == 28 else None),
                         "algorithmic_bytes": dom["bytes"]},
            "stages": rows, "arms": arms, "gpu_launches": launches, "clocks": clocks}
    if rank == 0:
        print(json.dumps(line))
    return 0


def run_star(args):
    """The star-schema-shaped foreign-key join: 150M dimension rows (dense
    int32 keys, int64 payloads), 600M fact rows (uniform or Zipf(--theta)
    foreign keys, 10 % absent), filtered to --selectivity; one step is
    eiger_join_sum (the exact sum of matched dimension + fact payloads), AUTO
    (payloads carried through the partitioning) against the same plan with
    the payloads gathered by tuple ID and against the static join."""
    import torch

    from paper_2607_04489_gb300 import eiger, workloads

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    eiger.load()
    w = workloads.star_schema(theta=args.theta, selectivity=args.selectivity, seed=rank, device=dev)
    torch.cuda.empty_cache()
    nd, nf = w.nb, w.np
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    pay_bytes = w.build_pay.element_size()

    def arm(variant, profile=False, mat="auto"):
        ws = torch.empty(eiger.join_sum_workspace(nd, nf, eiger.I32, pay_bytes, variant, mat),
                         dtype=torch.uint8, device=dev)
        res = None
        for _ in range(args.warmup):
            res = eiger.join_sum(w.build_keys, w.build_pay, w.probe_keys, w.probe_pay, variant=variant,
                                 materialize=mat, workspace=ws, stream=stream)
        def step():
            return eiger.join_sum(w.build_keys, w.build_pay, w.probe_keys, w.probe_pay, variant=variant,
                                  materialize=mat, workspace=ws, stream=stream)

        barrier(world)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(args.steps):
            res = step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier(world)
        ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)
        stages, launches = profile_pass(step, args.steps) if profile else ({}, 0)
        del ws
        torch.cuda.empty_cache()
        return ms, res, stages, launches

    tuples = world * (nd + nf)
    sampler = ClockSampler(local).start()
    ms, (total, matches, plan), stages, launches = arm("auto", profile=True)
    clocks = sampler.stop()
    sms, (stotal, smatches, _), _, _ = arm("static")
    if (stotal, smatches) != (total, matches):
        raise RuntimeError("static and adaptive sums differ")
    gms, (gtotal, gmatches, _), _, _ = arm("auto", mat="gfur")
    if (gtotal, gmatches) != (total, matches):
        raise RuntimeError("gathered and carried sums differ")
    peaks, peak_src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS))
    rows = stage_table(stages, args.steps)
    dom = rows[0]
    line = {"metric": METRIC, "value": tuples / (ms * 1e-3), "unit": "tuples/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": f"star-schema foreign-key join: 150M dimension rows, 600M fact rows "
                                   f"(zipf theta={args.theta}, 10% absent) filtered to {args.selectivity}, "
                                   "exact sum of matched payloads",
                       "dim_rows": nd, "fact_rows": nf, "matches": matches,
                       "parallelism": f"replicas x{world}", "l2": "inputs larger than L2; no flush"},
            "plan": {"variant": plan.variant, "bits1": plan.bits1, "bits2": plan.bits2,
                     "materialize": plan.materialize},
            "static": {"ms_per_step": sms, "value": tuples / (sms * 1e-3), "unit": "tuples/s",
                       "speedup_of_adaptive": sms / ms},
            "arms": {"auto_plan_gfur": {"ms_per_step": gms, "value": tuples / (gms * 1e-3), "unit": "tuples/s"}},
            "roofline": {"bound": "hbm", "kernel": dom["stage"], "achieved": dom["gbs"], "peak": hbm,
                         "peak_source": peak_src, "unit": "GB/s", "frac": dom["gbs"] / hbm,
                         "traffic": recorded_traffic(dom["stage"], f"star{args.theta:g}"
                                                     if args.selectivity == 1.0 else None),
                         "algorithmic_bytes": dom["bytes"]},
            "stages": rows, "gpu_launches": launches, "clocks": clocks}
    if rank == 0:
        print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "wide":
        return run_wide(args)
    if args.workload == "groupby":
        return run_groupby(args)
    if args.workload == "star":
        return run_star(args)
    if args.workload == "grid":
        return run_grid(args)
    if args.workload == "small":
        return run_small(args)
    return run_eiger(args)


if __name__ == "__main__":
    sys.exit(main())
