"""Learned variant selector: timing sweep, training, evaluation, persistence.

The paper chooses join algorithms and knobs at run time from cheap statistics
(Sec. 1, Table 1, Sec. 4). Here that choice is learned: every seeded synthetic
join is timed under each of the 15 plan classes (eiger_class_plan), and a
small network (the library's FP32 kernels, eiger_mlp_*) is trained on the 12
runtime features (eiger_features) toward the classes near the fastest (a
soft-target cross-entropy over the measured slowdowns). The exhaustive
choice (fastest measured class) is the yardstick; the rule-based selector
(eiger_plan) is the fallback and the comparison.

Pipeline (all steps on the GPU, each writes plain text under selector_data/):
  sweep(...)  -> timings.csv (one row per join; resumable, append-only)
  train(...)  -> model.json (parameters, feature normalisation, split, scores)
  evaluate()  -> regret on the held-out joins, learned vs rules.
``load_model`` + ``use`` install the trained network into EIGER_AUTO.
"""

from __future__ import annotations

import json
import math
import os
import random
import time
from dataclasses import dataclass

import numpy as np
import torch

from . import eiger, workloads

HERE = os.path.dirname(os.path.abspath(__file__))
DATA_DIR = os.path.join(HERE, "selector_data")
TIMINGS = os.path.join(DATA_DIR, "timings.csv")
MODEL = os.path.join(DATA_DIR, "model.json")
CLASSES = eiger.MLP_OUT
COST_CAP = 4.0             # relative slowdown assigned to unmeasured (dominated) classes
PROBE_SAMPLE = 1 << 20     # probe rows profiled for the features
MAX_MATCHES = 1 << 30      # joins with larger outputs are redrawn
BUILD_CAP = 4608           # rows per shared-memory table of the partitioned join

COLUMNS = (["seed", "dtype", "nb", "np", "matches"] + [f"f{i}" for i in range(eiger.MLP_IN)] +
           [f"t{c}" for c in range(CLASSES)] + ["t_rules", "rules_class"])


@dataclass
class JoinSpec:
    seed: int
    nb: int
    np: int
    key_bytes: int
    span_log2: float
    distinct_frac: float
    theta: float
    unique: bool = False  # build keys are distinct (each of the ndv = nb values once)


def draw_spec(seed: int, log2_lo: float = 10.0, log2_hi: float = 24.0, large_hi: float = 27.0,
              p_large: float = 0.1, p_unique: float = 0.25) -> JoinSpec:
    """Build 2^U(lo, hi) rows (one join in ten: 2^U(hi, large_hi)), probe
    ratio U(1, 16), key width 4 or 8 bytes, key span 2^U(16, 63) clamped to
    the width, probe skew theta U(0, 1.5). One join in four has unique build
    keys (span at least twice the rows); the others draw their build rows from
    a distinct fraction U(0.01, 1) of nb values, with repetition."""
    r = np.random.default_rng(seed)
    large = r.uniform() < p_large
    nb = int(2 ** (r.uniform(log2_hi, large_hi) if large else r.uniform(log2_lo, log2_hi)))
    np_ = min(int(nb * r.uniform(1, 16)), (1 << 32) - 1)
    kb = int(r.choice([4, 8]))
    span_log2 = min(float(r.uniform(16, 63)), 32.0 if kb == 4 else 63.0)
    unique = bool(r.uniform() < p_unique)
    frac = float(r.uniform(0.01, 1.0))
    theta = float(r.uniform(0.0, 1.5))
    if unique:
        frac = 1.0
        span_log2 = min(max(span_log2, math.log2(max(nb, 2)) + 1.0), 32.0 if kb == 4 else 63.0)
    return JoinSpec(seed, max(nb, 1), max(np_, 1), kb, span_log2, frac, theta, unique)


def make_join(spec: JoinSpec, device="cuda"):
    """Build and probe key columns of a spec (see draw_spec)."""
    g = torch.Generator(device=device)
    g.manual_seed(spec.seed * 7919 + 1)
    dt = torch.int32 if spec.key_bytes == 4 else torch.int64
    kmin, kmax = (-(1 << 31), (1 << 31) - 1) if spec.key_bytes == 4 else (-(1 << 63), (1 << 63) - 1)
    span = min(int(2 ** spec.span_log2), kmax - kmin)
    ndv = max(1, min(int(round(spec.distinct_frac * spec.nb)), span))
    lo = kmin + random.Random(spec.seed).randrange(0, max(1, kmax - kmin - span))
    if span <= 8 * ndv + 1024:
        vals = torch.randperm(span, generator=g, device=device)[:ndv] + lo
    else:
        vals = torch.empty(0, dtype=torch.int64, device=device)
        while vals.numel() < ndv:
            want = int((ndv - vals.numel()) * 1.05) + 16
            hi = min(lo + span, kmax)
            draw = torch.randint(lo, hi, (want,), generator=g, device=device, dtype=torch.int64)
            vals = torch.unique(torch.cat([vals, draw]))
        vals = vals[torch.randperm(vals.numel(), generator=g, device=device)[:ndv]]
    if spec.unique and ndv == spec.nb:
        bk = vals.to(dt)  # every value once, in random order
    else:
        bk = vals[torch.randint(0, ndv, (spec.nb,), generator=g, device=device)].to(dt)
    rank = workloads.zipf_ranks(ndv, spec.theta, spec.np, spec.seed * 7919 + 2, device)
    order = torch.randperm(ndv, generator=g, device=device)
    pk = vals[order[rank]].to(dt)
    return bk, pk


def dominated(cls: int, nb: int) -> bool:
    """Partitioned classes whose average build partition exceeds four shared-
    memory tables re-stream every probe partition at least four times and
    cannot be the fastest; they are not timed."""
    p = eiger.class_plan(cls)
    if p.variant == "nphj":
        return False
    bits = p.bits1 + p.bits2
    return nb / float(1 << bits) > 4 * BUILD_CAP


def class_of(plan: eiger.Plan) -> int:
    if plan.variant == "nphj":
        return 0
    if plan.variant == "phj1" and 8 <= plan.bits1 <= 12:
        return plan.bits1 - 7
    if plan.variant == "phj2" and 10 <= plan.bits1 + plan.bits2 <= 18:
        return plan.bits1 + plan.bits2 - 4
    return -1


def _time(fn, reps: int) -> float:
    fn()
    torch.cuda.synchronize()
    ts = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(reps):
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return sorted(ts)[len(ts) // 2]


def measure(spec: JoinSpec, reps: int = 3):
    """(features, per-class median ms with inf for dominated, rules ms, rules
    class, matches) for one join, or None when its output is too large."""
    bk, pk = make_join(spec)
    dt = eiger.I32 if bk.dtype == torch.int32 else eiger.I64
    bst = eiger.stats(bk)
    pst = eiger.stats(pk[:PROBE_SAMPLE])
    feats = eiger.features(bst, pst, bk.numel(), pk.numel(), dt)
    ws = torch.empty(eiger.join_workspace(bk.numel(), pk.numel(), dt, "auto"), dtype=torch.uint8, device="cuda")
    st, m, _ = eiger.join_into(bk, pk, capacity=0, workspace=ws)
    if m > MAX_MATCHES:
        return None
    ob = torch.empty(max(m, 1), dtype=torch.int32, device="cuda")
    op = torch.empty_like(ob)
    narrow = 1 if (dt == eiger.I32 or bst.max - bst.min <= 0xFFFFFFFF) else 0
    times = []
    for cls in range(CLASSES):
        if dominated(cls, bk.numel()):
            times.append(math.inf)
            continue
        p = eiger.class_plan(cls)
        p.narrow = narrow
        run = lambda: _ok(eiger.join_into(bk, pk, variant=p.variant, knobs=p, out_bidx=ob, out_pidx=op,
                                          capacity=m, workspace=ws), m)
        times.append(_time(run, reps))
    eiger.selector_set(None)
    plan_holder = {}

    def auto():
        st2, n2, plan = eiger.join_into(bk, pk, out_bidx=ob, out_pidx=op, capacity=m, workspace=ws)
        _ok((st2, n2, plan), m)
        plan_holder["p"] = plan

    t_rules = _time(auto, reps)
    return feats, times, t_rules, class_of(plan_holder["p"]), m


def _ok(res, m):
    st, n, _ = res
    if st != eiger.OK or n != m:
        raise RuntimeError(f"join failed: status {st}, {n} != {m}: {eiger.last_error()}")


def sweep(n_joins: int = 3000, start_seed: int = 0, out: str = TIMINGS, log2_hi: float = 24.0,
          time_budget_s: float | None = None) -> int:
    """Times joins with seeds start_seed.. (skipping rows already in `out`);
    appends one CSV row per join. Returns the number of rows written now."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    done = set()
    if os.path.exists(out):
        with open(out) as f:
            for line in f:
                if line and line[0].isdigit():
                    done.add(int(line.split(",", 1)[0]))
    new = 0
    t0 = time.time()
    fresh = not os.path.exists(out) or os.path.getsize(out) == 0
    with open(out, "a") as f:
        if fresh:
            f.write(",".join(COLUMNS) + "\n")
        for seed in range(start_seed, start_seed + n_joins):
            if seed in done:
                continue
            if time_budget_s is not None and time.time() - t0 > time_budget_s:
                break
            attempt, res = 0, None
            while res is None:
                spec = draw_spec(seed + 1_000_000 * attempt, log2_hi=log2_hi)
                res = measure(spec)
                attempt += 1
            feats, times, t_rules, rules_cls, m = res
            row = [seed, spec.key_bytes, spec.nb, spec.np, m] + [f"{v:.6g}" for v in feats]
            row += ["inf" if math.isinf(t) else f"{t:.5g}" for t in times] + [f"{t_rules:.5g}", rules_cls]
            f.write(",".join(str(v) for v in row) + "\n")
            f.flush()
            new += 1
            torch.cuda.empty_cache()
    return new


def load_timings(path: str = TIMINGS):
    rows = []
    with open(path) as f:
        header = f.readline().strip().split(",")
        for line in f:
            if line.strip():
                rows.append(line.strip().split(","))
    col = {h: i for i, h in enumerate(header)}
    seeds = np.array([int(r[col["seed"]]) for r in rows])
    order = np.argsort(seeds, kind="stable")
    rows = [rows[i] for i in order]
    X = np.array([[float(r[col[f"f{i}"]]) for i in range(eiger.MLP_IN)] for r in rows], np.float32)
    T = np.array([[float(r[col[f"t{c}"]]) for c in range(CLASSES)] for r in rows], np.float64)
    t_rules = np.array([float(r[col["t_rules"]]) for r in rows])
    meta = {"seed": seeds[order], "nb": np.array([int(r[col["nb"]]) for r in rows]),
            "np": np.array([int(r[col["np"]]) for r in rows])}
    return X, T, t_rules, meta


def cost_matrix(T: np.ndarray) -> np.ndarray:
    """Relative slowdown of each class against the fastest measured one,
    capped (and unmeasured classes set) at COST_CAP."""
    best = np.min(T, axis=1, keepdims=True)
    R = T / best - 1.0
    R[~np.isfinite(R)] = COST_CAP
    return np.minimum(R, COST_CAP).astype(np.float32)


def split(n: int, n_train: int = 2500):
    """Joins in seed order: the first n_train train, the rest are held out."""
    return np.arange(min(n_train, n)), np.arange(min(n_train, n), n)


def init_params(seed: int = 0) -> np.ndarray:
    """He-uniform weights, zero biases, packed like the library's parameters."""
    r = np.random.default_rng(seed)
    parts = []
    for fan_out, fan_in in ((64, 12), (64, 64), (15, 64)):
        lim = math.sqrt(6.0 / fan_in)
        parts += [r.uniform(-lim, lim, size=fan_out * fan_in), np.zeros(fan_out)]
    return np.concatenate(parts).astype(np.float32)


TAU = 0.05  # temperature of the soft target softmax(-slowdown / TAU)


def train(X: np.ndarray, T: np.ndarray, steps: int = 4000, lr: float = 2e-3, seed: int = 0,
          n_train: int = 2500, tau: float = TAU):
    """Full-batch Adam on the training joins with the library's gradient and
    optimiser kernels. The loss is the cross-entropy toward the soft target
    softmax(-slowdown / tau): every class within a few tau of the fastest
    shares the target, so near-ties cost little, and unlike the expected
    regret (tau = 0) the loss does not flatten once a class dominates the
    softmax. Returns the model dict (see save_model)."""
    tr, _ = split(len(X), n_train)
    mean = X[tr].mean(axis=0)
    scale = np.maximum(X[tr].std(axis=0), 1e-3)
    dev = torch.device("cuda")
    x = torch.from_numpy(((X[tr] - mean) / scale).astype(np.float32)).to(dev)
    c = torch.from_numpy(cost_matrix(T[tr])).to(dev)
    p = torch.from_numpy(init_params(seed)).to(dev)
    m, v = torch.zeros_like(p), torch.zeros_like(p)
    ws = None
    hist = []
    for step in range(1, steps + 1):
        L, g = eiger.mlp_grad(p, x, c, tau, workspace=ws)
        eiger.mlp_adam(p, g, m, v, step, lr)
        if step % 200 == 0 or step == 1:
            hist.append((step, float(L)))
    return {"params": p.cpu().numpy().tolist(), "mean": mean.tolist(), "scale": scale.tolist(),
            "n_train": int(len(tr)), "steps": steps, "lr": lr, "seed": seed, "tau": tau, "loss_history": hist}


def predict(model: dict, X: np.ndarray) -> np.ndarray:
    """Class chosen by the network (library forward kernel) for each row of X."""
    dev = torch.device("cuda")
    p = torch.tensor(model["params"], dtype=torch.float32, device=dev)
    mean, scale = np.array(model["mean"], np.float32), np.array(model["scale"], np.float32)
    x = torch.from_numpy(((X - mean) / scale).astype(np.float32)).to(dev)
    return eiger.mlp_forward(p, x).argmax(dim=1).cpu().numpy()


def regret(T: np.ndarray, chosen_ms: np.ndarray) -> dict:
    best = np.min(T, axis=1)
    r = chosen_ms / best - 1.0
    return {"mean": float(np.mean(r)), "p90": float(np.percentile(r, 90)),
            "total_time": float(chosen_ms.sum() / best.sum() - 1.0), "n": int(len(r))}


def chosen_times(T: np.ndarray, cls: np.ndarray) -> np.ndarray:
    """Measured time of each chosen class; an unmeasured (dominated) class is
    charged COST_CAP + 1 times the best."""
    t = T[np.arange(len(cls)), cls]
    best = np.min(T, axis=1)
    return np.where(np.isfinite(t), t, (COST_CAP + 2.0) * best)


def evaluate(model: dict, X, T, t_rules, n_train: int = 2500) -> dict:
    _, te = split(len(X), n_train)
    cls = predict(model, X[te])
    return {"learned": regret(T[te], chosen_times(T[te], cls)),
            "rules": regret(T[te], t_rules[te]),
            "exhaustive_class_histogram": np.bincount(np.argmin(T[te], axis=1), minlength=CLASSES).tolist(),
            "learned_class_histogram": np.bincount(cls, minlength=CLASSES).tolist()}


def save_model(model: dict, path: str = MODEL) -> None:
    os.makedirs(os.path.dirname(path), exist_ok=True)
    with open(path, "w") as f:
        json.dump(model, f)


def load_model(path: str = MODEL) -> dict:
    with open(path) as f:
        return json.load(f)


def use(model: dict | None = None) -> None:
    """Install the network into EIGER_AUTO (None: the stored model)."""
    model = model or load_model()
    p = torch.tensor(model["params"], dtype=torch.float32, device="cuda")
    eiger.selector_set(p, model["mean"], model["scale"])


def main(argv=None):
    import argparse

    ap = argparse.ArgumentParser(description="learned selector pipeline")
    ap.add_argument("step", choices=["sweep", "train", "all"])
    ap.add_argument("--joins", type=int, default=3000)
    ap.add_argument("--budget", type=float, default=None, help="seconds for the sweep")
    ap.add_argument("--timings", default=TIMINGS)
    ap.add_argument("--model", default=MODEL)
    a = ap.parse_args(argv)
    if a.step in ("sweep", "all"):
        n = sweep(a.joins, out=a.timings, time_budget_s=a.budget)
        print(f"timed {n} joins")
    if a.step in ("train", "all"):
        X, T, t_rules, _ = load_timings(a.timings)
        model = train(X, T)
        model["evaluation"] = evaluate(model, X, T, t_rules)
        save_model(model, a.model)
        print(json.dumps(model["evaluation"]))


if __name__ == "__main__":
    main()
