"""Ranking and the paper's tuning metrics over a timing table — TEST INFRASTRUCTURE.

A timing table is a list of rows; each row is a dict with at least
``index`` (canonical index), ``status`` (0 = measured) and ``t`` (median
time, smaller is better).  Performance P = flops / t.

Definitions followed (Sec. 4, "Evaluation metrics"):
  * tuning impact = performance of the global optimum / median performance of
    the configurations in the space (Sec. 4; Table 4 caption: "maximum over
    the median").  With an even count the median is the mean of the two middle
    values (the ordinary definition).
  * proportion of centrality C_p (Eq. 1) on the fitness flow graph.
  * performance portability PP (Eq. 2) as the harmonic mean of the
    application efficiencies e_i (Eq. 3).
Plain Python; sorting and numpy's percentile are the only library steps.
"""
from __future__ import annotations

import math

import numpy as np


def valid_rows(rows):
    return [r for r in rows if r["status"] == 0 and math.isfinite(r["t"]) and r["t"] > 0]


def rank(rows):
    """Valid rows sorted by (time ascending, canonical index ascending)."""
    return sorted(valid_rows(rows), key=lambda r: (r["t"], r["index"]))


def median(values):
    v = sorted(values)
    n = len(v)
    if n == 0:
        return float("nan")
    if n % 2:
        return float(v[n // 2])
    return 0.5 * (v[n // 2 - 1] + v[n // 2])


def stats(rows, flops, default_index=None):
    """The per-run summary: optimum, median, impact, tuned/default,
    tuned/median, fraction within 10 %, violin quantiles."""
    ok = rank(rows)
    if not ok:
        return None
    perf = [flops / r["t"] for r in ok]
    best = ok[0]
    p_max = flops / best["t"]
    p_med = median(perf)
    t_med = median([r["t"] for r in ok])
    res = {
        "best_index": best["index"],
        "t_best": best["t"],
        "p_max": p_max,
        "p_median": p_med,
        "impact": p_max / p_med,
        "tuned_vs_median_time": t_med / best["t"],
        "frac_within_10pct": sum(1 for r in ok if r["t"] <= 1.10 * best["t"]) / len(ok),
        "n_valid": len(ok),
        "quantiles": {q: float(np.percentile(perf, q)) for q in (0, 10, 25, 50, 75, 90, 100)},
    }
    if default_index is not None:
        d = [r for r in ok if r["index"] == default_index]
        res["tuned_vs_default"] = d[0]["t"] / best["t"] if d else float("nan")
    return res


# ---------------------------------------------------------------- Eq. 1 ------
def fitness_flow_graph(points, fitness, neighbours):
    """Directed edges x -> y between neighbouring points where y has the
    strictly better (smaller) fitness.  ``points`` is a list of hashable keys,
    ``fitness`` a dict key -> value, ``neighbours(key)`` the candidate keys
    (keys not in ``fitness`` are skipped)."""
    edges = {p: [] for p in points}
    for p in points:
        for q in neighbours(p):
            if q in fitness and fitness[q] < fitness[p]:
                edges[p].append(q)
    return edges


def pagerank(edges, damping=0.85, tol=1e-13, max_iter=100000):
    """Standard PageRank by power iteration; a node without out-edges spreads
    its mass uniformly over all nodes."""
    nodes = list(edges)
    n = len(nodes)
    pos = {p: k for k, p in enumerate(nodes)}
    r = np.full(n, 1.0 / n)
    for _ in range(max_iter):
        nxt = np.full(n, (1.0 - damping) / n)
        sink = 0.0
        for p in nodes:
            out = edges[p]
            rp = r[pos[p]]
            if out:
                share = damping * rp / len(out)
                for q in out:
                    nxt[pos[q]] += share
            else:
                sink += rp
        nxt += damping * sink / n
        if np.abs(nxt - r).sum() < tol:
            r = nxt
            break
        r = nxt
    return {p: float(r[pos[p]]) for p in nodes}


def proportion_of_centrality(edges, fitness, p, centrality=None):
    """C_p (Eq. 1): PageRank mass of the local minima whose fitness is within
    (1+p) of the optimum, over the mass of all local minima.  Local minima are
    the sinks of the fitness flow graph.  The bound is taken inclusively so
    that p = 0 selects the global optimum itself."""
    c = centrality if centrality is not None else pagerank(edges)
    minima = [x for x, out in edges.items() if not out]
    f_opt = min(fitness[x] for x in edges)
    num = sum(c[x] for x in minima if fitness[x] <= (1.0 + p) * f_opt)
    den = sum(c[x] for x in minima)
    return num / den


# ------------------------------------------------------------ Eqs. 2-3 -------
def application_efficiency(perf_by_device):
    """Eq. 3: e_i(x) = P_i(x) / max_x P_i(x).  ``perf_by_device`` maps device ->
    {config: performance}; returns device -> {config: efficiency}."""
    out = {}
    for dev, perf in perf_by_device.items():
        best = max(perf.values())
        out[dev] = {x: v / best for x, v in perf.items()}
    return out


def performance_portability(eff_by_device, x):
    """Eq. 2: |H| / sum_i 1/e_i(x); zero if x fails (or is missing) anywhere."""
    inv = 0.0
    for eff in eff_by_device.values():
        e = eff.get(x, 0.0)
        if e <= 0.0:
            return 0.0
        inv += 1.0 / e
    return len(eff_by_device) / inv
