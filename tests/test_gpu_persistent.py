"""The persistent grid (ct_config.persist = 1), the tuner's timing of both
grid forms, the re-measurement of the fastest configurations and the clock
recorded beside each timing.

A persistent launch runs as many blocks as the GPU holds at once, each taking
every G-th tile; it must give the same bits as one block per tile for every
staging form, keep its stores inside the output, and give up a wait for its
input copy within the bounded time like the tile-per-block launch does."""
import math
import time

import numpy as np
import pytest
import torch

import oracle
import synthetic
from tests.gpu_util import SENTINEL, assert_parity, run_config, upload_image

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cfg", [(16, 1, 1, 1, 0, 0), (16, 16, 4, 2, 1, 1), (32, 4, 4, 8, 1, 0),
                                 (128, 2, 2, 4, 1, 1), (64, 2, 3, 5, 0, 1), (256, 4, 8, 1, 1, 0)],
                         ids=lambda c: "_".join(map(str, c)))
def test_persistent_grid_same_bits(ctlib, cuda_device, cfg):
    """More tiles than the GPU holds at once (so persistent blocks loop),
    ragged sides, NaN in the padding columns: the persistent launch matches
    the oracle and one-block-per-tile bit for bit, with intact guard bands."""
    ow, oh, fw, fh = 1501, 1203, 11, 7
    img, f = synthetic.make_problem(31, ow, oh, fw, fh, pad_value=np.nan)
    ref, S = oracle.corr2d_f64(img, f, ow, oh)
    d_img = upload_image(img, cuda_device)
    a, ok_a = run_config(ctlib, d_img, f, ctlib.config(*cfg, persist=0), ow, oh, in_w=ow + fw - 1)
    b, ok_b = run_config(ctlib, d_img, f, ctlib.config(*cfg, persist=1), ow, oh, in_w=ow + fw - 1)
    assert ok_a and ok_b
    assert_parity(b, ref, S, f"persistent {cfg}")
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    ctlib.device_check()


def test_persistent_grid_bf16(ctlib, cuda_device):
    ow, oh, fs = 1024, 1024, 9
    img, f = synthetic.make_problem(4, ow, oh, fs, fs, pitch_align=8)
    ib = torch.from_numpy(img).to(torch.bfloat16)
    fb = torch.from_numpy(f).to(torch.bfloat16)
    ref, S = oracle.corr2d_bf16_f64(ib.view(torch.int16).numpy().view(np.uint16),
                                    fb.view(torch.int16).numpy().view(np.uint16), ow, oh)
    d_img = ib.to(cuda_device)
    for cfg in [(16, 8, 1, 2, 1, 0), (32, 2, 2, 2, 0, 1)]:
        a, ok_a = run_config(ctlib, d_img, fb, ctlib.config(*cfg), ow, oh, in_w=ow + fs - 1)
        b, ok_b = run_config(ctlib, d_img, fb, ctlib.config(*cfg, persist=1), ow, oh, in_w=ow + fs - 1)
        assert ok_a and ok_b
        assert_parity(b, ref, S, f"bf16 persistent {cfg}")
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_persistent_wait_timeout_is_reported(ctlib, cuda_device, monkeypatch):
    """A tensor-staged variant built to expect 16 bytes more than its copy
    delivers, launched persistent over 4,096 tiles: every block gives up at
    its first tile after the bounded wait, the whole launch ends within
    seconds, nothing is stored, the error is reported and the next launch is
    correct."""
    ow = oh = 2048
    img, f = synthetic.make_problem(6, ow, oh, 5, 5)
    d_img = upload_image(img, cuda_device)
    c = ctlib.config(32, 4, 4, 2, 1, 1, persist=1)   # tile 128 x 8: 16 x 256 tiles, halo box 132 x 12
    ctlib.device_check()
    ctlib.clear_cache()
    monkeypatch.setenv("CONVTUNE_NVRTC_EXTRA", "-DCT_TEST_EXTRA_TX=16")
    try:
        t0 = time.time()
        out, ok = run_config(ctlib, d_img, f, c, ow, oh, in_w=ow + 4)
        assert time.time() - t0 < 30.0
    finally:
        monkeypatch.delenv("CONVTUNE_NVRTC_EXTRA")
        ctlib.clear_cache()
    assert ok
    assert np.all(out.view(np.uint32) == np.array(SENTINEL).view(np.uint32))
    with pytest.raises(ctlib.CTError) as e:
        ctlib.device_check()
    assert e.value.status == -7
    ctlib.device_check()
    xs, ys = synthetic.sample_points(6, ow, oh, 2000)
    ref, S = oracle.corr2d_points(img, f, xs, ys)
    out, ok = run_config(ctlib, d_img, f, c, ow, oh, in_w=ow + 4)
    assert ok and np.all(np.abs(out[ys, xs] - ref) <= 1e-5 * S)
    ctlib.device_check()


def test_tuner_times_both_grids_and_remeasures(ctlib, cuda_device):
    """grid_modes = 1: every row whose problem has more tiles than the GPU
    holds at once carries both medians, t_med_ms is the smaller and
    cfg.persist names it; each row has the SM clock it ran at; the
    re-measurement covers the k fastest rows and best_row is the fastest of
    them by the re-measured median."""
    p = ctlib.make_problem(4096, 4096, 17, 17)     # every kernel long enough for single-launch timing
    tab = ctlib.tune(p, "full", "random", seed=5, max_evals=24, repeats=5, grid_modes=1, remeasure_top=4,
                     remeasure_repeats=9, flush_l2=True, remeasure_forms=3)
    ok = [r for r in tab.rows if r["status"] == 0]
    assert ok
    both = [r for r in ok if math.isfinite(r["t_persist_ms"])]
    assert both, "no row timed the persistent grid"
    for r in ok:
        assert math.isfinite(r["t_tiles_ms"])
        if math.isfinite(r["t_persist_ms"]):
            assert r["t_med_ms"] == min(r["t_tiles_ms"], r["t_persist_ms"])
            assert r["persist"] == (1 if r["t_persist_ms"] < r["t_tiles_ms"] else 0)
        else:
            assert r["persist"] == 0 and r["t_med_ms"] == r["t_tiles_ms"]
        assert r["sm_mhz"] > 0
    assert tab.info["sm_mhz_median"] > 0
    re = [r for r in tab.rows if math.isfinite(r["t_remeasured_ms"])]
    assert tab.info["remeasured"] == len(re) == 4
    fastest = sorted(ok, key=lambda r: (r["t_med_ms"], r["index"]))[:4]
    assert {r["index"] for r in re} == {r["index"] for r in fastest}
    best = tab.rows[tab.info["best_row"]]
    assert best["t_remeasured_ms"] == min(r["t_remeasured_ms"] for r in re)
    assert tab.best.as_tuple() == best["cfg"].as_tuple()
    for r in tab.rows:                       # the re-measurement may move an unrolled row to another form
        assert r["taps"] == 0 or (r["unroll"] == 1 and math.isfinite(r["t_remeasured_ms"]))
        assert r["fma2"] == 0 or (r["unroll"] == 1 and r["tile_y"] >= 2 and r["taps"] == 0
                                  and math.isfinite(r["t_remeasured_ms"]))
    # the returned configuration, in whatever form won, reproduces the oracle
    img, f = synthetic.make_problem(1, 4096, 4096, 17, 17)
    xs, ys = synthetic.sample_points(1, 4096, 4096, 2000)
    ref, S = oracle.corr2d_points(img, f, xs, ys)
    d_img = upload_image(img, cuda_device)
    out, good = run_config(ctlib, d_img, f, tab.best, 4096, 4096)
    assert good and np.all(np.abs(out[ys, xs] - ref) <= 1e-5 * S)


def test_tuner_with_compiled_taps(ctlib, cuda_device):
    """taps_imm = 1: the unrolled configurations are measured with the
    problem's taps compiled in (taps = 1 in their rows), the others with the
    parameter-block taps, and the returned configuration reproduces the
    oracle on the tuned problem."""
    ow = oh = 1024
    img, f = synthetic.make_problem(9, ow, oh, 17, 17)
    d_img = upload_image(img, cuda_device)
    p = ctlib.problem_for(d_img, f)
    tab = ctlib.tune(p, "full", "random", image=d_img, filt=f, seed=11, max_evals=16, repeats=3, taps_imm=1,
                     grid_modes=1, remeasure_top=3, remeasure_repeats=5)
    ok = [r for r in tab.rows if r["status"] == 0]
    assert ok and any(r["unroll"] for r in ok)
    for r in ok:
        assert r["taps"] == r["unroll"]
    xs, ys = synthetic.sample_points(9, ow, oh, 3000)
    ref, S = oracle.corr2d_points(img, f, xs, ys)
    out, good = run_config(ctlib, d_img, f, tab.best, ow, oh)
    assert good and np.all(np.abs(out[ys, xs] - ref) <= 1e-5 * S)


def test_remeasure_stands_down_for_graph_timed_optima(ctlib, cuda_device):
    """A problem whose fastest kernels are timed as graphs of back-to-back
    launches (here 256x256 / 5x5, a few microseconds each) keeps those
    figures: nothing is re-measured by single launches, and the optimum is
    the sweep's."""
    p = ctlib.make_problem(256, 256, 5, 5)
    tab = ctlib.tune(p, "small", "brute", seed=0, remeasure_top=8, remeasure_forms=3)
    assert tab.info["remeasured"] == 0
    assert all(not math.isfinite(r["t_remeasured_ms"]) for r in tab.rows)
    ok = [r for r in tab.rows if r["status"] == 0]
    best = min(ok, key=lambda r: (r["t_med_ms"], r["index"]))
    assert tab.rows[tab.info["best_row"]]["index"] == best["index"]
