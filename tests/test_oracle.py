"""CPU tests that pin the oracle (correlation, spaces, ranking and the paper's
metrics) to facts outside itself."""
import math
import os

import numpy as np
import pytest

import oracle
import synthetic
from oracle import analysis, space
from tests import oracle_pins

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("pin", oracle_pins.ALL_PINS, ids=lambda p: p.__name__)
def test_corr2d_pins(pin):
    pin(oracle.corr2d_f64)


def test_points_match_full():
    img, f = synthetic.make_problem(5, 37, 29, 5, 7)
    full, S = oracle.corr2d_f64(img, f, 37, 29)
    xs, ys = synthetic.sample_points(5, 37, 29, 50)
    o, s = oracle.corr2d_points(img, f, xs, ys)
    assert np.array_equal(o, full[ys, xs]) and np.array_equal(s, S[ys, xs])


def test_bf16_widening_matches_f32():
    """bf16 bit patterns widened exactly give the same result as the float32
    oracle on the same (bf16-representable) values."""
    import torch
    img, f = synthetic.make_problem(9, 21, 13, 3, 5)
    ib = torch.from_numpy(img).to(torch.bfloat16)
    fb = torch.from_numpy(f).to(torch.bfloat16)
    o_b, S_b = oracle.corr2d_bf16_f64(ib.view(torch.int16).numpy().view(np.uint16),
                                      fb.view(torch.int16).numpy().view(np.uint16), 21, 13)
    o_f, S_f = oracle.corr2d_f64(ib.float().numpy(), fb.float().numpy(), 21, 13)
    assert np.array_equal(o_b, o_f) and np.array_equal(S_b, S_f)


def test_empty_and_threads():
    img, f = synthetic.make_problem(1, 0, 4, 3, 3)
    o, S = oracle.corr2d_f64(img, f, 0, 4)
    assert o.shape == (4, 0)
    img, f = synthetic.make_problem(2, 40, 30, 5, 5)
    a, _ = oracle.corr2d_f64(img, f, 40, 30, nthreads=1)
    b, _ = oracle.corr2d_f64(img, f, 40, 30, nthreads=0)
    assert np.array_equal(a, b)


# ------------------------------------------------------------ generator -----
def test_generator_grid_and_determinism():
    v = synthetic.uniform_pm1(1, 0, 100000)
    assert v.dtype == np.float32 and v.min() >= -1.0 and v.max() < 1.0
    k = (v.astype(np.float64) + 1.0) * 2 ** 23
    assert np.array_equal(k, np.round(k))            # on the 2^-23 grid
    assert np.array_equal(v, synthetic.uniform_pm1(1, 0, 100000))
    assert np.array_equal(v[500:600], synthetic.uniform_pm1(1, 500, 100))
    assert abs(float(v.mean())) < 0.01 and abs(float(v.var()) - 1 / 3) < 0.01


def test_splitmix64_published_values():
    # First outputs of SplitMix64 seeded with 0 / 1234567 (the values printed
    # with Vigna's reference C implementation of the generator).
    z = synthetic.splitmix64(0, 0, 3)
    assert [int(x) for x in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    z = synthetic.splitmix64(1234567, 0, 5)
    assert [int(x) for x in z] == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                                   4593380528125082431, 16408922859458223821]


# ------------------------------------------------------------- spaces -------
def test_space_counts():
    assert len(space.enumerate_space("small", 5, 5)) == 256
    assert len(space.enumerate_space("small", 5, 5, valid_only=False)) == 256
    raw = space.enumerate_space("full", 17, 17, valid_only=False)
    assert len(raw) == 5 * 5 * 8 * 8 * 2 * 2
    by_threads = [c for _, c in raw if c["block_x"] * c["block_y"] <= 1024]
    assert len(by_threads) == 22 * 64 * 4 == 5632
    valid = space.enumerate_space("full", 17, 17)
    # the halo tile of smem configurations must fit 227 KB: count the excluded
    # ones by direct arithmetic on the tile size
    over = sum(1 for c in by_threads if c["smem"] and
               (c["block_y"] * c["tile_y"] + 16) * (c["block_x"] * c["tile_x"] + 16) * 4 > 232448)
    assert over == 56 and len(valid) == 5632 - 56


def test_space_canonical_and_neighbours():
    ents = space.enumerate_space("full", 17, 17, valid_only=False)
    for idx, cfg in ents[::97]:
        assert space.canonical_index("full", cfg) == idx
    cfg = {"block_x": 16, "block_y": 16, "tile_x": 8, "tile_y": 1, "smem": 0, "unroll": 1}
    nb = space.neighbours("full", cfg)
    assert len(nb) == 6   # bx up, by down (16 is last), tx down (8 is last), ty up, smem, unroll
    for c in nb:
        assert sum(c[k] != cfg[k] for k in cfg) == 1


# ----------------------------------------------------------- analysis -------
def _golden_table4():
    rows = []
    with open(os.path.join(GOLDEN, "table4_tuning_impact.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            k, d, med, mx, imp = line.split()
            rows.append((k, d, float(med), float(mx), float(imp)))
    return rows


def test_impact_reproduces_table4():
    """impact = maximum / median reproduces the printed impacts within the
    rounding of the printed medians and maxima (interval arithmetic)."""
    rows = _golden_table4()
    assert len(rows) == 16
    for k, d, med, mx, imp in rows:
        lo = (mx - 0.5) / (med + 0.5)
        hi = (mx + 0.5) / (med - 0.5)
        assert lo - 0.05 <= imp <= hi + 0.05, (k, d, lo, imp, hi)
        # the reversed ratio or a mean-based one would not fit
        assert not (lo - 0.05 <= med / mx <= hi + 0.05)


def test_stats_hand_table():
    flops = 100.0
    rows = [dict(index=i, status=0, t=t) for i, t in enumerate([4.0, 2.0, 2.0, 8.0, 1.0, 1.05])]
    rows.append(dict(index=6, status=-4, t=float("nan")))       # failed launch
    rows.append(dict(index=7, status=0, t=0.5 / 0.0 if False else float("inf")))
    r = analysis.rank(rows)
    assert [x["index"] for x in r] == [4, 5, 1, 2, 0, 3]          # tie 1,2 by index
    st = analysis.stats(rows, flops, default_index=0)
    perf = sorted(flops / t for t in [4.0, 2.0, 2.0, 8.0, 1.0, 1.05])
    assert st["p_max"] == 100.0
    assert st["p_median"] == 0.5 * (perf[2] + perf[3])           # even count
    assert st["impact"] == st["p_max"] / st["p_median"]
    assert st["tuned_vs_default"] == 4.0
    assert st["frac_within_10pct"] == 2 / 6
    assert st["tuned_vs_median_time"] == 2.0
    assert st["n_valid"] == 6


def test_pagerank_closed_form_and_library():
    # two nodes a -> b (b is a sink); solved by hand:
    # r_a = (1-d)/2 + d r_b/2 and r_a + r_b = 1  =>  r_a = ((1-d)/2 + d/2) / (1 + d/2)
    d = 0.85
    pr = analysis.pagerank({"a": ["b"], "b": []}, damping=d)
    ra = ((1 - d) / 2 + d / 2) / (1 + d / 2)
    assert abs(pr["a"] - ra) < 1e-12 and abs(pr["b"] - (1 - ra)) < 1e-12
    nx = pytest.importorskip("networkx")
    edges = {0: [1, 2], 1: [3], 2: [3, 1], 3: [], 4: [3], 5: [4, 0]}
    ours = analysis.pagerank(edges)
    g = nx.DiGraph()
    g.add_nodes_from(edges)
    for u, vs in edges.items():
        for v in vs:
            g.add_edge(u, v)
    ref = nx.pagerank(g, alpha=0.85, tol=1e-14, max_iter=10000)
    for k in edges:
        assert abs(ours[k] - ref[k]) < 1e-9


def test_proportion_of_centrality_chain():
    """A 1D chain with fitness [3, 1, 2, 0.5, 4]: local minima are positions 1
    (f=1) and 3 (f=0.5); C_0 is the optimum's share, C_p for p >= 1 is 1."""
    fit = {0: 3.0, 1: 1.0, 2: 2.0, 3: 0.5, 4: 4.0}
    nb = lambda p: [q for q in (p - 1, p + 1) if q in fit]
    edges = analysis.fitness_flow_graph(list(fit), fit, nb)
    assert edges == {0: [1], 1: [], 2: [1, 3], 3: [], 4: [3]}
    c = analysis.pagerank(edges)
    c0 = analysis.proportion_of_centrality(edges, fit, 0.0, c)
    assert abs(c0 - c[3] / (c[1] + c[3])) < 1e-15
    assert analysis.proportion_of_centrality(edges, fit, 0.99, c) == c0
    assert analysis.proportion_of_centrality(edges, fit, 1.0, c) == 1.0
    assert 0.0 < c0 < 1.0


def test_performance_portability():
    perf = {"gpuA": {"x": 10.0, "y": 5.0, "z": 0.0}, "gpuB": {"x": 2.0, "y": 4.0, "z": 1.0}}
    eff = analysis.application_efficiency(perf)
    assert eff["gpuA"] == {"x": 1.0, "y": 0.5, "z": 0.0} and eff["gpuB"]["y"] == 1.0
    scipy_stats = pytest.importorskip("scipy.stats")
    assert math.isclose(analysis.performance_portability(eff, "x"), scipy_stats.hmean([1.0, 0.5]))
    assert math.isclose(analysis.performance_portability(eff, "y"), scipy_stats.hmean([0.5, 1.0]))
    assert analysis.performance_portability(eff, "z") == 0.0   # fails on one device
    single = analysis.application_efficiency({"g": {"a": 3.0, "b": 6.0}})
    assert analysis.performance_portability(single, "b") == 1.0
