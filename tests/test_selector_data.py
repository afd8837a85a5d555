"""The stored learned selector against its stored timings, on the CPU.

`selector_data/timings.csv` holds every plan class's measured time for 3000
seeded joins (GB300) and `selector_data/model.json` the network trained on
the first 2500 with the library's kernels. Here the fp64 oracle network
(oracle/mlp.py) replays the stored model on the 500 held-out joins: its
choices must cost less than 10 % over the exhaustive choice on average and
beat the rule-based selector, whose own choice and time are in the timings.
"""

import csv
import json
import os

import numpy as np
import pytest

from oracle import mlp

DATA = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2607_04489_gb300",
                    "selector_data")


@pytest.fixture(scope="module")
def data():
    with open(os.path.join(DATA, "timings.csv")) as f:
        rows = sorted(csv.DictReader(f), key=lambda r: int(r["seed"]))
    X = np.array([[float(r[f"f{i}"]) for i in range(mlp.IN)] for r in rows])
    T = np.array([[float(r[f"t{c}"]) for c in range(mlp.OUT)] for r in rows])
    rules = np.array([float(r["t_rules"]) for r in rows])
    with open(os.path.join(DATA, "model.json")) as f:
        model = json.load(f)
    return X, T, rules, model


def test_timings_cover_every_class_and_seed(data):
    X, T, rules, model = data
    assert X.shape == (3000, mlp.IN) and T.shape == (3000, mlp.OUT)
    assert np.all(np.isfinite(T[:, 0]))  # the non-partitioned class is timed for every join
    best = np.argmin(T, axis=1)
    assert len(set(best.tolist())) >= 10  # the fastest class varies across the joins
    assert model["n_train"] == 2500 and len(model["params"]) == mlp.P


def test_stored_model_beats_the_rules_on_held_out_joins(data):
    X, T, rules, model = data
    te = np.arange(model["n_train"], len(X))
    mean, scale = np.array(model["mean"]), np.array(model["scale"])
    z, _ = mlp.forward(np.array(model["params"]), (X[te] - mean) / scale)
    choice = np.argmax(z, axis=1)
    best = np.min(T[te], axis=1)
    chosen = T[te, choice]
    chosen = np.where(np.isfinite(chosen), chosen, 6.0 * best)  # an untimed class counts as very slow
    learned = float(np.mean(chosen / best - 1.0))
    rule = float(np.mean(rules[te] / best - 1.0))
    assert learned < 0.10, learned
    assert learned < 0.5 * rule, (learned, rule)
    ev = model.get("evaluation", {}).get("learned", {})
    if "mean" in ev:  # the GPU evaluation stored with the model agrees with the fp64 replay
        assert ev["mean"] == pytest.approx(learned, abs=0.01)
