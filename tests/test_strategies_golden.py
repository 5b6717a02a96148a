"""The search strategies of Sec. 3 replayed over a real landscape: the
brute-force timing table of the full space (5,576 valid configurations) that
one GB300 recorded for the 4096x4096 / 17x17 workload
(tests/golden/gb300_full_f17_times.txt, written by make_table_golden.py from
``bench.py --table-out``).  The exhaustive optimum comes from the oracle's
ranking of the same table; brute force must return it, and random sampling
(10 % of the space) and simulated annealing (same budget; 1 and 16 walkers)
must land within 5 % of it as a median over 20 seeds."""
import math
import os

import numpy as np
import pytest

from oracle import analysis, space as ospace

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "gb300_full_f17_times.txt")


def load_times():
    n_raw = len(ospace.enumerate_space("full", 17, 17, valid_only=False))
    t = np.full(n_raw, np.nan)
    with open(GOLDEN) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            i, v = line.split()
            t[int(i)] = float(v)
    return t


def optimum(times):
    rows = [dict(index=i, status=0, t=float(v)) for i, v in enumerate(times) if math.isfinite(v)]
    best = analysis.rank(rows)[0]
    return best["index"], best["t"]


def test_golden_table_covers_the_valid_space():
    t = load_times()
    valid = {i for i, _ in ospace.enumerate_space("full", 17, 17)}
    assert {i for i in range(len(t)) if math.isfinite(t[i])} == valid
    assert len(valid) == 5576 and np.nanmin(t) > 0


def test_brute_force_replay_returns_the_oracle_optimum(ctlib):
    t = load_times()
    i_opt, t_opt = optimum(t)
    p = ctlib.make_problem(4096, 4096, 17, 17)
    tab = ctlib.tune_replay(p, "full", "brute", t)
    best = tab.rows[tab.info["best_row"]]
    assert best["index"] == i_opt and best["t_med_ms"] == t_opt and len(tab.rows) == 5576


@pytest.mark.parametrize("strategy,chains", [("random", 1), ("anneal", 1), ("anneal", 16)])
def test_strategy_within_five_percent_on_the_recorded_table(ctlib, strategy, chains):
    t = load_times()
    _, t_opt = optimum(t)
    p = ctlib.make_problem(4096, 4096, 17, 17)
    budget = math.ceil(0.10 * 5576)
    ratios = []
    for seed in range(20):
        tab = ctlib.tune_replay(p, "full", strategy, t, seed=seed, anneal_chains=chains)
        assert len(tab.rows) <= budget
        ratios.append(tab.rows[tab.info["best_row"]]["t_med_ms"] / t_opt)
    print(strategy, chains, "median", float(np.median(ratios)), "max", max(ratios))
    assert float(np.median(ratios)) <= 1.05, ratios
    assert min(ratios) >= 1.0
