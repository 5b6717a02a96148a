"""CPU-only tests of the C-ABI library: it loads, exports every declared
symbol, validates arguments, enumerates spaces exactly as the oracle defines
them, compiles variants with NVRTC (no GPU needed) and runs the search
strategies over given timing landscapes (replay mode)."""
import math
import os
import re

import numpy as np
import pytest
import torch

from oracle import analysis, space as ospace

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NO_GPU = not torch.cuda.is_available()


def header_symbols():
    text = open(os.path.join(ROOT, "include", "convtune.h")).read()
    return sorted(set(re.findall(r"CT_API\s+[\w\s\*]+?\b(ct_\w+)\s*\(", text)))


def test_library_exports_every_declared_symbol(ctlib):
    syms = header_symbols()
    assert len(syms) >= 20
    lib = ctlib.lib()
    for s in syms:
        assert hasattr(lib, s), s
    assert set(syms) == set(ctlib.EXPORTED)
    assert "sm_103a" in ctlib.version()


@pytest.mark.skipif(not NO_GPU, reason="checks the no-device path")
def test_no_device_paths(ctlib):
    with pytest.raises(ctlib.CTError) as e:
        ctlib.device_query()
    assert e.value.status == -8
    p = ctlib.make_problem(64, 64, 5, 5)
    with pytest.raises(ctlib.CTError) as e:
        ctlib.tune(p, "small", "brute")
    assert e.value.status == -8


def _raw_status(ctlib, p, c):
    import ctypes
    return ctlib.lib().ct_check_config(ctypes.byref(p), ctypes.byref(c), 232448)


def test_argument_validation(ctlib):
    ok = ctlib.make_problem(64, 32, 5, 3)
    assert _raw_status(ctlib, ok, ctlib.config()) == 0
    bad = [
        (ctlib.Problem(64, 32, 0, 3, 68, 64, 0, 0), ctlib.config(), -1),      # filter width 0
        (ctlib.Problem(64, 32, 33, 3, 100, 64, 0, 0), ctlib.config(), -1),    # filter too wide
        (ctlib.Problem(64, 32, 5, 3, 66, 64, 0, 0), ctlib.config(), -1),      # pitch not 16-byte
        (ctlib.Problem(64, 32, 5, 3, 64, 64, 0, 0), ctlib.config(), -1),      # pitch < in_w
        (ctlib.Problem(64, 32, 5, 3, 68, 62, 0, 0), ctlib.config(), -1),      # out pitch < out_w
        (ctlib.Problem(64, 32, 5, 3, 68, 64, 7, 0), ctlib.config(), -1),      # bad dtype
        (ctlib.Problem(64, 32, 5, 3, 68, 64, 1, 0), ctlib.config(), -1),      # bf16 pitch 68*2 not /16
        (ok, ctlib.config(64, 32), -2),                                        # 2048 threads
        (ok, ctlib.config(tile_x=17), -2),
        (ok, ctlib.config(use_smem=2), -2),
        (ok, ctlib.config(block_x=2, use_smem=1), -2),                         # smem tile unaligned
        (ctlib.make_problem(4096, 4096, 17, 17), ctlib.config(256, 2, 8, 8, 1, 1), -2),  # smem > limit
    ]
    for p, c, want in bad:
        st = _raw_status(ctlib, p, c)
        assert st == want, (p.out_w, p.filter_w, p.in_pitch, c, st)
        assert ctlib.lib().ct_last_error().decode()
    assert _raw_status(ctlib, ctlib.Problem(64, 32, 5, 3, 72, 64, 1, 0), ctlib.config()) == 0


@pytest.mark.parametrize("name,fw,fh", [("small", 5, 5), ("full", 17, 17), ("full", 3, 3), ("full", 31, 9)])
def test_space_enumeration_matches_oracle(ctlib, name, fw, fh):
    p = ctlib.make_problem(256, 256, fw, fh)
    sp = ctlib.Space(name)
    ours = sp.enumerate(p, 232448)
    ref = ospace.enumerate_space(name, fw, fh, smem_limit=232448)
    assert len(ours) == len(ref)
    for (i1, c1), (i2, c2) in zip(ours, ref):
        assert i1 == i2
        d = c1.as_dict()
        d["smem"] = d.pop("use_smem")
        assert d.pop("persist") == 0 and d.pop("taps") == 0 and d.pop("fma2") == 0 and d.pop("shfl") == 0
        assert d == c2
    raw, valid = sp.count(p, 232448)
    assert raw == len(ospace.enumerate_space(name, fw, fh, valid_only=False)) and valid == len(ref)


def test_space_counts_named_workloads(ctlib):
    assert ctlib.Space("small").count(ctlib.make_problem(256, 256, 5, 5), 232448) == (256, 256)
    assert ctlib.Space("full").count(ctlib.make_problem(4096, 4096, 17, 17), 232448) == (6400, 5576)
    raw, valid = ctlib.Space("paper").count(ctlib.make_problem(4096, 4096, 17, 17), 232448)
    assert raw == 16 * 5 * 4 * 4 * 2 * 2


def test_partial_unroll_factors(ctlib):
    """unroll takes 0 (rolled), 1 (full) and the partial factors 2 and 4."""
    p = ctlib.make_problem(128, 128, 5, 5)
    sp = ctlib.Space('{"block_x": [32], "block_y": [8], "unroll": [0, 1, 2, 4]}')
    assert [c.unroll for _, c in sp.enumerate(p, 232448)] == [0, 1, 2, 4]
    for u in (0, 1, 2, 4):
        ctlib.check_config(p, ctlib.config(32, 8, 1, 1, 0, u))
    for u in (3, 8, -1):
        with pytest.raises(ctlib.CTError) as e:
            ctlib.check_config(p, ctlib.config(32, 8, 1, 1, 0, u))
        assert e.value.status == -2
    info = ctlib.compile_variant(p, ctlib.config(32, 8, 2, 2, 1, 4))
    assert info["regs"] > 0


def test_space_from_json(ctlib):
    sp = ctlib.Space('{"block_x": [32, 64], "tile_y": [1, 2, 4], "unroll": [0, 1]}')
    p = ctlib.make_problem(128, 128, 3, 3)
    ents = sp.enumerate(p, 232448)
    assert len(ents) == 12
    assert all(c.block_y == 8 and c.tile_x == 1 and c.use_smem == 0 for _, c in ents)
    with pytest.raises(ctlib.CTError):
        ctlib.Space('{"block_q": [1]}')
    with pytest.raises(ctlib.CTError):
        ctlib.Space("nonexistent")


def test_nvrtc_compiles_variants_without_gpu(ctlib):
    """NVRTC builds sm_103a cubins on a machine with no GPU.  A variant's
    dynamic shared memory is its halo tile; variants whose halo box (width
    rounded to 16 bytes) is at most 256 x 256 elements load it with one tensor
    copy and ask for 128 bytes more, to place it on a 128-byte boundary."""
    p = ctlib.make_problem(4096, 4096, 17, 17)
    for c, tensor_copy in [(ctlib.default_config(), False), (ctlib.config(32, 4, 4, 8, 1, 1), True),
                           (ctlib.config(16, 8, 3, 5, 1, 0), True), (ctlib.config(64, 2, 2, 2, 0, 1), False),
                           (ctlib.config(128, 2, 2, 4, 1, 1), False), (ctlib.config(16, 16, 4, 2, 1, 1), True)]:
        info = ctlib.compile_variant(p, c)
        assert info["cubin_bytes"] > 1000 and info["regs"] > 0, (c, info)
        assert info["smem_bytes"] == ospace.smem_bytes(
            {"block_x": c.block_x, "block_y": c.block_y, "tile_x": c.tile_x, "tile_y": c.tile_y,
             "smem": c.use_smem}, 17, 17) + (128 if tensor_copy else 0), c
    pb = ctlib.make_problem(1024, 1024, 9, 9, dtype=ctlib.CT_BF16)
    assert ctlib.compile_variant(pb, ctlib.config(32, 4, 4, 4, 1, 1))["regs"] > 0


def test_compile_failure_is_reported(ctlib, monkeypatch):
    monkeypatch.setenv("CONVTUNE_NVRTC_EXTRA", "-DCT_INJECT_COMPILE_ERROR=1")
    p = ctlib.make_problem(100, 100, 7, 3)
    with pytest.raises(ctlib.CTError) as e:
        ctlib.compile_variant(p, ctlib.config(48, 2, 1, 3, 0, 0))
    assert e.value.status == -3 and "CT_INJECT_COMPILE_ERROR" in str(e.value)
    monkeypatch.delenv("CONVTUNE_NVRTC_EXTRA")
    assert ctlib.compile_variant(p, ctlib.config(48, 2, 1, 3, 0, 0))["regs"] > 0


def test_disk_cache(ctlib, tmp_path):
    ctlib.set_cache_dir(str(tmp_path))
    try:
        p = ctlib.make_problem(300, 200, 11, 7)
        c = ctlib.config(16, 4, 2, 3, 1, 1)
        ctlib.clear_cache()
        a = ctlib.compile_variant(p, c)
        assert any(f.endswith(".cubin") for f in os.listdir(tmp_path))
        ctlib.clear_cache()
        b = ctlib.compile_variant(p, c)
        assert b["from_cache"] == 1 and b["cubin_bytes"] == a["cubin_bytes"] and b["regs"] == a["regs"]
    finally:
        ctlib.set_cache_dir(None)
        ctlib.clear_cache()


# ---------------------------------------------------- strategies (replay) ---
def landscape(name, fw, fh, seed, fail_every=0):
    """A synthetic timing landscape over the canonical indices of a space:
    multiplicative per-parameter effects, an interaction that punishes large
    register tiles with large blocks, and seeded noise; optional failures."""
    from synthetic import uniform_pm1
    ents = ospace.enumerate_space(name, fw, fh, valid_only=False)
    noise = uniform_pm1(seed, 0, len(ents)).astype(np.float64)
    t = np.full(len(ents), np.nan)
    valid = {i for i, _ in ospace.enumerate_space(name, fw, fh)}
    for (i, c), nz in zip(ents, noise):
        if i not in valid:
            continue
        threads = c["block_x"] * c["block_y"]
        tile = c["tile_x"] * c["tile_y"]
        v = 1.0
        v *= 1.0 + 0.3 * abs(math.log2(threads / 128))
        v *= 1.0 + 0.5 / tile + 0.02 * max(0, tile - 24) ** 1.2
        v *= 0.9 if c["smem"] else 1.0
        v *= 0.8 if c["unroll"] and tile <= 32 else 1.15
        v *= 1.0 + 0.04 * nz
        t[i] = v
        if fail_every and i % fail_every == 0:
            t[i] = np.nan
    return t


def oracle_rows(table):
    return [dict(index=r["index"], status=r["status"], t=r["t_med_ms"]) for r in table.rows]


def test_brute_force_equals_oracle_ranking(ctlib):
    p = ctlib.make_problem(256, 256, 5, 5)
    times = landscape("small", 5, 5, 11, fail_every=37)
    tab = ctlib.tune_replay(p, "small", "brute", times)
    assert len(tab.rows) == 256 and [r["eval_order"] for r in tab.rows] == list(range(256))
    assert [r["index"] for r in tab.rows] == list(range(256))
    ranked = analysis.rank(oracle_rows(tab))
    assert tab.best.as_tuple() == tab.rows[ranked[0]["index"]]["cfg"].as_tuple()
    assert ranked[0]["index"] == int(np.nanargmin(times))
    failed = [r for r in tab.rows if r["status"] != 0]
    assert len(failed) == len([i for i in range(256) if i % 37 == 0])
    assert tab.info["n_valid_space"] == 256 and tab.info["best_row"] == ranked[0]["index"]


def test_ties_break_to_lower_index(ctlib):
    p = ctlib.make_problem(256, 256, 5, 5)
    times = np.full(256, 2.0)
    times[[200, 17, 90]] = 1.0
    tab = ctlib.tune_replay(p, "small", "brute", times)
    assert tab.rows[tab.info["best_row"]]["index"] == 17


def test_random_sampling(ctlib):
    p = ctlib.make_problem(4096, 4096, 17, 17)
    times = landscape("full", 17, 17, 5)
    n_valid = int(np.sum(np.isfinite(times)))
    a = ctlib.tune_replay(p, "full", "random", times, seed=7)
    b = ctlib.tune_replay(p, "full", "random", times, seed=7)
    c = ctlib.tune_replay(p, "full", "random", times, seed=8)
    idx = [r["index"] for r in a.rows]
    assert len(idx) == math.ceil(0.10 * n_valid) == len(set(idx))
    assert all(np.isfinite(times[i]) for i in idx)
    assert idx == [r["index"] for r in b.rows] and idx != [r["index"] for r in c.rows]
    best = min(a.rows, key=lambda r: (r["t_med_ms"], r["index"]))
    assert a.best.as_tuple() == best["cfg"].as_tuple()


def test_annealing_within_five_percent(ctlib):
    """Median over 20 seeds of t_found / t_opt on the 17x17 full space."""
    p = ctlib.make_problem(4096, 4096, 17, 17)
    times = landscape("full", 17, 17, 3)
    t_opt = np.nanmin(times)
    n_valid = int(np.sum(np.isfinite(times)))
    ratios = []
    for seed in range(20):
        tab = ctlib.tune_replay(p, "full", "anneal", times, seed=seed)
        assert len(tab.rows) <= math.ceil(0.1 * n_valid)
        assert len({r["index"] for r in tab.rows}) == len(tab.rows)       # memoised
        ratios.append(tab.rows[tab.info["best_row"]]["t_med_ms"] / t_opt)
    assert float(np.median(ratios)) <= 1.05, ratios


@pytest.mark.parametrize("chains", [1, 4, 16])
def test_annealing_replay_is_deterministic(ctlib, chains):
    """Without compiles every walker's candidate is ready at once, so the
    walkers take turns in order: one seed gives one evaluation sequence, with
    any number of walkers, and the walkers share the budget."""
    p = ctlib.make_problem(4096, 4096, 17, 17)
    times = landscape("full", 17, 17, 5)
    runs = [ctlib.tune_replay(p, "full", "anneal", times, seed=7, max_evals=200, anneal_chains=chains)
            for _ in range(2)]
    seqs = [[r["index"] for r in sorted(t.rows, key=lambda r: r["eval_order"])] for t in runs]
    assert seqs[0] == seqs[1] and len(seqs[0]) == 200
    other = ctlib.tune_replay(p, "full", "anneal", times, seed=8, max_evals=200, anneal_chains=chains)
    assert [r["index"] for r in sorted(other.rows, key=lambda r: r["eval_order"])] != seqs[0]


@pytest.mark.parametrize("chains", [1, 16])
def test_annealing_restart_moves_every_walker_to_the_best(ctlib, tmp_path, chains):
    """Sec. 3's annealing restarts from the best point found so far.  After
    each restart every walker's next step starts from that point (a candidate
    a walker proposed from its old point is dropped, not measured), so the
    step's candidate is the best point's neighbour or a jump; steps never come
    from an earlier restart epoch; and every non-jump candidate is a neighbour
    of the point it was proposed from."""
    import json
    p = ctlib.make_problem(4096, 4096, 17, 17)
    times = landscape("full", 17, 17, 9)
    trace = tmp_path / "trace.jsonl"
    ctlib.tune_replay(p, "full", "anneal", times, seed=3, anneal_chains=chains, trace_path=str(trace))
    ev = [json.loads(line) for line in open(trace)]
    restarts = [k for k, e in enumerate(ev) if e["ev"] == "restart"]
    assert len(restarts) >= 2, "the landscape must force restarts"
    cfg_of = dict(ospace.enumerate_space("full", 17, 17, valid_only=False))
    for k in restarts:
        # the restart point is the fastest point measured before it
        measured = [e for e in ev[:k] if e["ev"] in ("start", "step") and e["f"] > 0]
        f_min = min(e["f"] for e in measured)
        assert ev[k]["f"] == f_min and times[ev[k]["best"]] == f_min
        nxt = next((j for j in restarts if j > k), len(ev))
        for w in range(chains):
            first = next((e for e in ev[k + 1:nxt] if e["ev"] == "step" and e["walker"] == w), None)
            if first is None:
                continue
            assert first["epoch"] == ev[k]["epoch"] and first["from"] == ev[k]["best"], (k, w, first)
            if not first["jump"]:
                assert cfg_of[first["cand"]] in ospace.neighbours("full", cfg_of[ev[k]["best"]])
    epochs = [e["epoch"] for e in ev if e["ev"] == "step"]
    assert epochs == sorted(epochs)
    for e in ev:
        if e["ev"] == "step" and not e["jump"]:
            assert cfg_of[e["cand"]] in ospace.neighbours("full", cfg_of[e["from"]])


def test_annealing_with_failures_and_budget(ctlib):
    p = ctlib.make_problem(256, 256, 5, 5)
    times = landscape("small", 5, 5, 4, fail_every=5)
    tab = ctlib.tune_replay(p, "small", "anneal", times, seed=1, max_evals=60)
    assert len(tab.rows) == 60
    assert any(r["status"] != 0 for r in tab.rows)
    assert tab.rows[tab.info["best_row"]]["status"] == 0


def test_resume_uses_recorded_rows(ctlib, tmp_path):
    p = ctlib.make_problem(256, 256, 5, 5)
    times = landscape("small", 5, 5, 9)
    path = str(tmp_path / "table.jsonl")
    first = ctlib.tune_replay(p, "small", "brute", times, resume_path=path)
    lines = open(path).read().splitlines()
    assert len(lines) == 256
    # a second run over a different landscape takes every row from the file
    second = ctlib.tune_replay(p, "small", "brute", times * 3.0 + 1.0, resume_path=path)
    assert [r["t_med_ms"] for r in second.rows] == [r["t_med_ms"] for r in first.rows]
    assert len(open(path).read().splitlines()) == 256      # nothing re-measured
    # another problem ignores those rows
    p2 = ctlib.make_problem(128, 256, 5, 5)
    third = ctlib.tune_replay(p2, "small", "brute", times * 2.0, resume_path=path)
    assert third.rows[0]["t_med_ms"] == pytest.approx(times[0] * 2.0)


def test_batch_validation_without_gpu(ctlib):
    import ctypes
    items = (ctlib.BatchItem * 1)()
    items[0] = ctlib.BatchItem(16, 16, 16, 64, 64, 5, 5, 66, 64)      # pitch 66 is not 16-byte aligned
    h = ctlib.vp()
    st = ctlib.lib().ct_batch_create(items, 1, None, ctypes.byref(h))
    assert st == -1 and b"item 0" in ctlib.lib().ct_last_error()
    assert ctlib.lib().ct_batch_create(items, 0, None, ctypes.byref(h)) == -1
    good = (ctlib.BatchItem * 1)()
    good[0] = ctlib.BatchItem(16, 16, 16, 64, 64, 5, 5, 68, 64)
    for field, bad in (("min_blocks_per_sm", 9), ("min_blocks_per_sm", -1), ("threads", 100)):
        o = ctlib.BatchOpts()
        setattr(o, field, bad)
        assert ctlib.lib().ct_batch_create(good, 1, ctypes.byref(o), ctypes.byref(h)) == -1, field
    if NO_GPU:
        items[0] = ctlib.BatchItem(16, 16, 16, 64, 64, 5, 5, 68, 64)
        assert ctlib.lib().ct_batch_create(items, 1, None, ctypes.byref(h)) == -8


@pytest.mark.skipif(not NO_GPU, reason="checks the no-device path")
def test_server_without_gpu(ctlib):
    with pytest.raises(ctlib.CTError) as e:
        ctlib.Server(1 << 20, tune=False)
    assert e.value.status == -8
    import ctypes
    h = ctlib.vp()
    assert ctlib.lib().ct_server_create(None, ctypes.byref(h)) == -1
    assert ctlib.lib().ct_server_run(None, None, None) == -1


def _oracle_analysis(table, space_name, flops, p_values):
    rows = oracle_rows(table)
    st = analysis.stats(rows, flops)
    ok = {r["index"]: r["t"] for r in analysis.valid_rows(rows)}
    cfg_of = {r["index"]: {"block_x": r["block_x"], "block_y": r["block_y"], "tile_x": r["tile_x"],
                           "tile_y": r["tile_y"], "smem": r["use_smem"], "unroll": r["unroll"]} for r in table.rows}
    nb = lambda i: [ospace.canonical_index(space_name, c) for c in ospace.neighbours(space_name, cfg_of[i])]
    edges = analysis.fitness_flow_graph(list(ok), ok, nb)
    c = analysis.pagerank(edges)
    cps = {p: analysis.proportion_of_centrality(edges, ok, p, c) for p in p_values}
    return st, edges, cps


@pytest.mark.parametrize("strategy", ["brute", "random"])
def test_table_analysis_matches_oracle(ctlib, strategy):
    p = ctlib.make_problem(4096, 4096, 17, 17)
    times = landscape("full", 17, 17, 21, fail_every=53)
    tab = ctlib.tune_replay(p, "full", strategy, times, seed=4)
    a = tab.analysis
    flops = 2.0 * 4096 * 4096 * 289
    # oracle performance = flops / t_ms; / 1e6 turns flops per ms into GFLOP/s
    st, edges, cps = _oracle_analysis(tab, "full", flops / 1e6, ctlib.P_VALUES)
    assert a["n_valid"] == st["n_valid"]
    assert a["best_index"] == st["best_index"]
    for k, ko in (("p_max", "p_max"), ("p_median", "p_median"), ("impact", "impact"),
                  ("tuned_vs_median", "tuned_vs_median_time"), ("frac_within_10pct", "frac_within_10pct")):
        assert a[k] == pytest.approx(st[ko], rel=1e-12), k
    for q, v in st["quantiles"].items():
        assert a["quantiles"][q] == pytest.approx(v, rel=1e-12)
    assert a["n_minima"] == sum(1 for out in edges.values() if not out)
    for pv in ctlib.P_VALUES:
        assert a["cp"][pv] == pytest.approx(cps[pv], abs=1e-9), pv
    assert a["cp"][0.0] <= a["cp"][0.05] <= a["cp"][0.15] <= 1.0
