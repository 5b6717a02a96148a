"""GPU parity of the correlation variants against the FP64 oracle, through
the C-ABI.  Bar: |gpu - oracle| <= 1e-5 * sum|in*f| per pixel (FP32);
bit-exact where the arithmetic is exact (integer inputs, impulse filters).
Every launch also checks sentinel guard bands around the output."""
import concurrent.futures as cf
import time

import numpy as np
import pytest
import torch

import oracle
import synthetic
from oracle import space as ospace
from tests.gpu_util import SENTINEL, assert_parity, run_config, upload_image

pytestmark = pytest.mark.gpu


def _cfg(ct, d):
    return ct.config(d["block_x"], d["block_y"], d["tile_x"], d["tile_y"], d["smem"], d["unroll"])


def _precompile(ct, problem, cfgs):
    with cf.ThreadPoolExecutor(16) as ex:
        list(ex.map(lambda c: ct.compile_variant(problem, c), cfgs))


# a spread of the full space: block shapes, tiles (incl. odd), smem and unroll
SPREAD = [
    (32, 8, 1, 1, 0, 0), (16, 1, 1, 1, 0, 0), (32, 4, 4, 8, 1, 1), (64, 2, 3, 5, 1, 0), (128, 8, 8, 1, 0, 1),
    (16, 16, 2, 2, 1, 1), (256, 4, 1, 2, 1, 1), (16, 4, 8, 8, 1, 1), (32, 1, 2, 4, 0, 1), (64, 16, 1, 1, 1, 0),
    (16, 2, 7, 3, 0, 1), (32, 2, 6, 6, 1, 1), (128, 1, 5, 7, 0, 0), (16, 8, 4, 4, 0, 1),
]


def test_device_is_gb300(ctlib, cuda_device):
    d = ctlib.device_query()
    assert (d.cc_major, d.cc_minor) == (10, 3), d.name
    assert d.sm_count >= 100 and d.smem_optin_bytes >= 200 * 1024


def test_small_space_every_config(ctlib, cuda_device):
    """The 256-config small space on output 256x256 / filter 5x5 / seed 0:
    every configuration matches the oracle and all are bit-identical."""
    ow = oh = 256
    img, f = synthetic.make_problem(0, ow, oh, 5, 5)
    ref, S = oracle.corr2d_f64(img, f, ow, oh)
    d_img = upload_image(img, cuda_device)
    p = ctlib.problem_for(d_img, f, in_w=ow + 4)
    ents = ospace.enumerate_space("small", 5, 5)
    assert len(ents) == 256
    cfgs = [_cfg(ctlib, c) for _, c in ents]
    _precompile(ctlib, p, cfgs)
    first = None
    for c in cfgs:
        out, ok = run_config(ctlib, d_img, f, c, ow, oh, in_w=ow + 4)
        assert ok, f"guard band overwritten by {c}"
        assert_parity(out, ref, S, repr(c))
        if first is None:
            first = out
        else:
            assert np.array_equal(out.view(np.uint32), first.view(np.uint32)), f"{c} differs bitwise"


@pytest.mark.parametrize("shape", [(333, 157, 17, 17), (64, 64, 3, 3), (97, 211, 9, 5)])
def test_integer_inputs_bit_exact(ctlib, cuda_device, shape):
    ow, oh, fw, fh = shape
    img, f = synthetic.make_problem(77, ow, oh, fw, fh, kind="int")
    ref, _ = oracle.corr2d_f64(img, f, ow, oh)
    d_img = upload_image(img, cuda_device)
    p = ctlib.problem_for(d_img, f, in_w=ow + fw - 1)
    cfgs = [ctlib.config(*c) for c in SPREAD]
    cfgs = [c for c in cfgs if ospace.is_valid(dict(zip(ospace.PARAMS, c.as_tuple())), fw, fh)]
    _precompile(ctlib, p, cfgs)
    for c in cfgs:
        out, ok = run_config(ctlib, d_img, f, c, ow, oh, in_w=ow + fw - 1)
        assert ok
        assert np.array_equal(out.astype(np.float64), ref), repr(c)


def test_impulse_filters_shift_exactly(ctlib, cuda_device):
    ow, oh, fw, fh = 130, 70, 7, 5
    img, _ = synthetic.make_problem(5, ow, oh, fw, fh, pad_value=np.nan)
    d_img = upload_image(img, cuda_device)
    for a, b in [(0, 0), (4, 6), (2, 3), (0, 6), (4, 0)]:
        f = np.zeros((fh, fw), np.float32)
        f[a, b] = 1.0
        for c in [ctlib.config(32, 8, 1, 1, 0, 0), ctlib.config(16, 4, 4, 4, 1, 1), ctlib.config(64, 2, 3, 2, 1, 0)]:
            out, ok = run_config(ctlib, d_img, f, c, ow, oh, in_w=ow + fw - 1)
            assert ok and np.array_equal(out, img[a:a + oh, b:b + ow]), (a, b, c)


EDGE_SHAPES = [(1, 1, 1, 1), (1, 1, 17, 17), (257, 131, 3, 7), (131, 257, 7, 3), (5, 300, 1, 1),
               (1000, 3, 31, 2), (33, 33, 32, 32), (17, 1, 2, 9), (4, 4, 4, 4), (2049, 19, 17, 17)]


@pytest.mark.parametrize("shape", EDGE_SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_edge_shapes(ctlib, cuda_device, shape):
    """Ragged sizes (not multiples of any tile), Fw != Fh, 1x1 filters,
    1x1 outputs, the largest filter; NaN in the input padding columns."""
    ow, oh, fw, fh = shape
    img, f = synthetic.make_problem(1000 + ow + oh, ow, oh, fw, fh, pad_value=np.nan)
    ref, S = oracle.corr2d_f64(img, f, ow, oh)
    d_img = upload_image(img, cuda_device)
    p = ctlib.problem_for(d_img, f, in_w=ow + fw - 1)
    cfgs = [ctlib.config(*c) for c in SPREAD]
    if fw * fh > 300:   # keep compile time of the widest filters modest
        cfgs = [c for c in cfgs if c.tile_x * c.tile_y <= 16]
    cfgs = [c for c in cfgs if ospace.is_valid(dict(zip(ospace.PARAMS, c.as_tuple())), fw, fh)]
    _precompile(ctlib, p, cfgs)
    for c in cfgs:
        out, ok = run_config(ctlib, d_img, f, c, ow, oh, in_w=ow + fw - 1)
        assert ok, f"guard band overwritten by {c}"
        assert_parity(out, ref, S, f"{shape} {c}")


def test_empty_output_is_a_noop(ctlib, cuda_device):
    img, f = synthetic.make_problem(3, 0, 10, 3, 3)
    d_img = upload_image(img, cuda_device)
    out = torch.full((10, 4), 7.0, device=cuda_device)
    r = ctlib.conv2d(d_img, f, ctlib.config(), in_w=2, out=out)
    torch.cuda.synchronize()
    assert r.shape == (10, 0) and bool((out == 7.0).all())


def test_invalid_config_enqueues_nothing(ctlib, cuda_device):
    img, f = synthetic.make_problem(3, 64, 64, 5, 5)
    d_img = upload_image(img, cuda_device)
    out = torch.full((64, 64), 7.0, device=cuda_device)
    for bad, status in [(ctlib.config(64, 32), -2), (ctlib.config(tile_x=0), -2)]:
        with pytest.raises(ctlib.CTError) as e:
            ctlib.conv2d(d_img, f, bad, in_w=68, out=out)
        assert e.value.status == status
    with pytest.raises(ctlib.CTError) as e:     # misaligned image base
        ctlib.conv2d(d_img.view(-1)[1:].as_strided((60, 72), (72, 1)), f, ctlib.config(), in_w=64, out=out)
    assert e.value.status == -1
    torch.cuda.synchronize()
    assert bool((out == 7.0).all())


def test_full_size_sampled(ctlib, cuda_device):
    """Output 4096x4096, filter 17x17, seed 1, at the launch shapes the
    benchmark uses: 4096 sampled pixels plus the corners against the oracle
    evaluated pixel by pixel, and all configurations bit-identical."""
    ow = oh = 4096
    img, f = synthetic.make_problem(1, ow, oh, 17, 17)
    d_img = upload_image(img, cuda_device)
    xs, ys = synthetic.sample_points(1, ow, oh, 4096)
    ref, S = oracle.corr2d_points(img, f, xs, ys)
    p = ctlib.problem_for(d_img, f)
    cfgs = [ctlib.config(*c) for c in SPREAD if ospace.is_valid(dict(zip(ospace.PARAMS, c)), 17, 17)]
    _precompile(ctlib, p, cfgs)
    first = None
    for c in cfgs:
        out, ok = run_config(ctlib, d_img, f, c, ow, oh)
        assert ok
        got = out[ys, xs].astype(np.float64)
        bad = ~(np.abs(got - ref) <= 1e-5 * S)
        assert not bad.any(), (c, int(bad.sum()))
        if first is None:
            first = out
        else:
            assert np.array_equal(out.view(np.uint32), first.view(np.uint32)), repr(c)


def test_bf16_storage(ctlib, cuda_device):
    """BF16 image and filter widened exactly to FP32: parity against the
    oracle run on the same BF16 values; error against the FP32-input oracle
    reported (bounded by the BF16 rounding of the inputs)."""
    ow = oh = 1024
    img, f = synthetic.make_problem(4, ow, oh, 9, 9, pitch_align=8)
    ib = torch.from_numpy(img).to(torch.bfloat16)
    fb = torch.from_numpy(f).to(torch.bfloat16)
    ref, S = oracle.corr2d_bf16_f64(ib.view(torch.int16).numpy().view(np.uint16),
                                    fb.view(torch.int16).numpy().view(np.uint16), ow, oh)
    d_img = ib.to(cuda_device)
    cfgs = [ctlib.config(32, 8, 1, 1, 0, 0), ctlib.config(32, 4, 4, 8, 1, 1), ctlib.config(16, 8, 3, 2, 1, 0),
            ctlib.config(64, 2, 2, 4, 0, 1)]
    ref32, S32 = oracle.corr2d_f64(img, f, ow, oh)
    for c in cfgs:
        out, ok = run_config(ctlib, d_img, fb, c, ow, oh, in_w=ow + 8)
        assert ok
        assert_parity(out, ref, S, f"bf16 {c}")
        # against the FP32-input oracle: within the bf16 input rounding (2 * 2^-8 relative per product)
        assert np.all(np.abs(out - ref32) <= 2 ** -7 * S32 + 1e-5 * S)


def test_stream_and_host_entry_point(ctlib, cuda_device):
    ow, oh, fw, fh = 500, 300, 11, 5
    img, f = synthetic.make_problem(8, ow, oh, fw, fh)
    ref, S = oracle.corr2d_f64(img, f, ow, oh)
    d_img = upload_image(img, cuda_device)
    s = torch.cuda.Stream()
    c = ctlib.config(32, 4, 2, 4, 1, 1)
    out, ok = run_config(ctlib, d_img, f, c, ow, oh, in_w=ow + fw - 1, stream=s)
    assert ok
    assert_parity(out, ref, S, "side stream")
    p = ctlib.problem_for(d_img, f, in_w=ow + fw - 1)
    h_img = torch.from_numpy(img).pin_memory()
    h_out = torch.empty((oh, p.out_pitch), dtype=torch.float32).pin_memory()
    ws_img = torch.empty_like(d_img)
    ws_out = torch.empty((oh, p.out_pitch), dtype=torch.float32, device=cuda_device)
    ctlib.conv2d_host(p, c, h_img, np.ascontiguousarray(f), h_out, ws_img, ws_out, stream=s)
    assert np.array_equal(h_out.numpy()[:, :ow], out)


def test_tune_small_brute_matches_oracle_ranking(ctlib, cuda_device):
    """ct_tune brute force over the 256-config small space: every row
    measured, and the returned optimum is the oracle's ranking of the same
    timing table."""
    from oracle import analysis
    p = ctlib.make_problem(256, 256, 5, 5)
    tab = ctlib.tune(p, "small", "brute", seed=0)
    assert len(tab.rows) == 256 and all(r["status"] == 0 and r["n"] == 7 for r in tab.rows)
    ranked = analysis.rank([dict(index=r["index"], status=r["status"], t=r["t_med_ms"]) for r in tab.rows])
    assert tab.best.as_tuple() == tab.rows[ranked[0]["index"]]["cfg"].as_tuple()
    st = analysis.stats([dict(index=r["index"], status=r["status"], t=r["t_med_ms"]) for r in tab.rows],
                        2.0 * 256 * 256 * 25)
    assert st["impact"] >= 1.0 and 0.0 < st["frac_within_10pct"] <= 1.0


@pytest.mark.parametrize("strategy", ["random", "anneal"])
def test_tune_strategies_on_gpu(ctlib, cuda_device, strategy):
    p = ctlib.make_problem(1024, 1024, 17, 17)
    tab = ctlib.tune(p, "full", strategy, seed=3, max_evals=24, repeats=3)
    assert len(tab.rows) == 24 and len({r["index"] for r in tab.rows}) == 24
    ok = [r for r in tab.rows if r["status"] == 0]
    assert ok
    best = min(ok, key=lambda r: (r["t_med_ms"], r["index"]))
    assert tab.best.as_tuple() == best["cfg"].as_tuple()
    info = tab.info
    assert info["wall_ms"] >= info["bench_ms"] > 0 and info["compile_cpu_ms"] >= 0


def test_host_entry_point_bands(ctlib, cuda_device):
    """The banded host pipeline (8 bands here) gives the device path's bits."""
    ow, oh, fw, fh = 1000, 2048 + 37, 9, 13
    img, f = synthetic.make_problem(12, ow, oh, fw, fh)
    d_img = upload_image(img, cuda_device)
    c = ctlib.config(32, 8, 4, 5, 1, 0)
    out, ok = run_config(ctlib, d_img, f, c, ow, oh, in_w=ow + fw - 1)
    assert ok
    p = ctlib.problem_for(d_img, f, in_w=ow + fw - 1)
    h_img = torch.from_numpy(img).pin_memory()
    h_out = torch.full((oh, p.out_pitch), float("nan"), dtype=torch.float32).pin_memory()
    ws_img = torch.zeros_like(d_img)
    ws_out = torch.zeros((oh, p.out_pitch), dtype=torch.float32, device=cuda_device)
    for _ in range(2):
        ctlib.conv2d_host(p, c, h_img, np.ascontiguousarray(f), h_out, ws_img, ws_out)
        assert np.array_equal(h_out.numpy()[:, :ow].view(np.uint32), out.view(np.uint32))


def test_host_entry_point_pitched(ctlib, cuda_device):
    """Host rows with a wider pitch than the device rows (2D copies)."""
    big, f = synthetic.make_problem(13, 1500, 1200, 7, 5)   # host image with a wide pitch
    ow, oh = 701, 999
    img = np.ascontiguousarray(big[:oh + 4, :ow + 6])
    ref, S = oracle.corr2d_f64(img, f, ow, oh)
    c = ctlib.config(16, 16, 4, 2, 1, 1)
    p = ctlib.make_problem(ow, oh, 7, 5)
    h_big = torch.from_numpy(big).pin_memory()
    h_out = torch.full((oh, 1000), float("nan"), dtype=torch.float32).pin_memory()
    ws_img = torch.zeros((oh + 4, p.in_pitch), dtype=torch.float32, device=cuda_device)
    ws_out = torch.zeros((oh, p.out_pitch), dtype=torch.float32, device=cuda_device)
    ctlib.conv2d_host_pitched(p, c, h_big.data_ptr(), big.shape[1], np.ascontiguousarray(f), h_out.data_ptr(), 1000,
                              ws_img.data_ptr(), ws_out.data_ptr())
    got = h_out.numpy()
    assert_parity(got[:, :ow], ref, S, "pitched host path")
    assert np.isnan(got[:, ow:]).all()


@pytest.mark.parametrize("shape", [(1024, 1024, 9), (4096, 4096, 17)])
def test_bf16_error_against_fp32_inputs(ctlib, cuda_device, shape):
    """BF16 storage error against the FP64 oracle on the ORIGINAL FP32 inputs
    (seed 4), reported per configuration; every configuration gives the same
    bits, so the error is the same for all of them."""
    ow, oh, fs = shape
    img, f = synthetic.make_problem(4, ow, oh, fs, fs, pitch_align=8)
    if ow <= 1024:
        ref, S = oracle.corr2d_f64(img, f, ow, oh)
        sel = (slice(None), slice(None))
    else:
        xs, ys = synthetic.sample_points(4, ow, oh, 20000)
        ref, S = oracle.corr2d_points(img, f, xs, ys)
        sel = (ys, xs)
    d_img = torch.from_numpy(img).to(torch.bfloat16).to(cuda_device)
    fb = torch.from_numpy(f).to(torch.bfloat16)
    first = None
    for c in [ctlib.config(16, 16, 4, 2, 1, 1), ctlib.config(32, 8, 4, 4, 1, 0), ctlib.config(64, 4, 2, 3, 0, 1)]:
        out = ctlib.conv2d(d_img, fb, c, in_w=ow + fs - 1)
        torch.cuda.synchronize()
        got = out.cpu().numpy()[sel].astype(np.float64)
        err = np.abs(got - ref)
        rep = {"shape": f"{ow}x{oh}/f{fs}", "config": c.as_tuple(), "max_abs_err": float(err.max()),
               "rms_err": float(np.sqrt(np.mean(err ** 2))), "max_err_over_S": float((err / S).max()),
               "rms_ref": float(np.sqrt(np.mean(ref ** 2)))}
        print("BF16_ERROR", rep)
        assert np.all(err <= 2.0 ** -7 * S + 1e-5 * S)
        if first is None:
            first = got
        else:
            assert np.array_equal(got, first)


def test_host_entry_point_async_overlapping_calls(ctlib, cuda_device):
    """Two asynchronous host-buffer calls in flight at once (distinct buffers)
    give the same bits as the synchronous path."""
    ow, oh, fw, fh = 1500, 1300, 9, 9
    probs = [synthetic.make_problem(21 + k, ow, oh, fw, fh) for k in range(2)]
    p = ctlib.make_problem(ow, oh, fw, fh)
    c = ctlib.config(16, 16, 4, 2, 1, 1)
    h_imgs = [torch.from_numpy(img).pin_memory() for img, _ in probs]
    h_outs = [torch.full((oh, p.out_pitch), float("nan")).pin_memory() for _ in range(2)]
    ws_i = [torch.empty((oh + fh - 1, p.in_pitch), device=cuda_device) for _ in range(2)]
    ws_o = [torch.empty((oh, p.out_pitch), device=cuda_device) for _ in range(2)]
    ev = [torch.cuda.Event(), torch.cuda.Event()]
    for k in range(2):
        ctlib.conv2d_host_async(p, c, h_imgs[k].data_ptr(), p.in_pitch, np.ascontiguousarray(probs[k][1]),
                                h_outs[k].data_ptr(), p.out_pitch, ws_i[k].data_ptr(), ws_o[k].data_ptr(), ev[k])
    for k in range(2):
        ev[k].synchronize()
        d = upload_image(probs[k][0], cuda_device)
        ref, ok = run_config(ctlib, d, probs[k][1], c, ow, oh, in_w=ow + fw - 1)
        assert np.array_equal(h_outs[k].numpy()[:, :ow].view(np.uint32), ref.view(np.uint32))


def test_tensor_copy_variants_leave_the_error_word_clear(ctlib, cuda_device):
    """Variants staged by a tensor copy (halo box <= 256 x 256) and by
    per-thread copies agree bit for bit on an image whose row padding holds
    NaN (the tensor copy reads zeros past the row, the per-thread copy the
    padding; neither reaches a stored output), and no wait gives up."""
    ow, oh, fs = 700, 333, 17
    img, f = synthetic.make_problem(11, ow, oh, fs, fs, pitch_align=8, pad_value=np.nan)
    d_img = upload_image(img, cuda_device)
    ref, S = oracle.corr2d_f64(img, f, ow, oh)
    ctlib.device_check()
    outs = []
    for c in [ctlib.config(16, 16, 4, 2, 1, 1), ctlib.config(32, 4, 4, 8, 1, 0), ctlib.config(128, 2, 2, 4, 1, 1),
              ctlib.config(32, 8, 1, 1, 0, 0)]:
        out, ok = run_config(ctlib, d_img, f, c, ow, oh, in_w=ow + fs - 1)
        assert ok
        assert_parity(out, ref, S, repr(c))
        outs.append(out)
    for o in outs[1:]:
        assert np.array_equal(o.view(np.uint32), outs[0].view(np.uint32))
    ctlib.device_check()


def test_tensor_copy_wait_timeout_is_reported(ctlib, cuda_device, monkeypatch):
    """A tensor-staged variant compiled to expect 16 bytes more than its copy
    delivers cannot complete its wait: every block gives up after the bounded
    wait and stores nothing, ct_device_check reports CT_ERR_TIMEOUT, and the
    context stays usable."""
    ow = oh = 128
    img, f = synthetic.make_problem(5, ow, oh, 5, 5)
    d_img = upload_image(img, cuda_device)
    c = ctlib.config(32, 4, 4, 2, 1, 1)          # halo box 132 x 12: staged by a tensor copy
    ctlib.device_check()
    ctlib.clear_cache()                           # in-memory variants are keyed by configuration only
    monkeypatch.setenv("CONVTUNE_NVRTC_EXTRA", "-DCT_TEST_EXTRA_TX=16")
    try:
        t0 = time.time()
        out, ok = run_config(ctlib, d_img, f, c, ow, oh, in_w=ow + 4)
        assert time.time() - t0 < 30.0
    finally:
        monkeypatch.delenv("CONVTUNE_NVRTC_EXTRA")
        ctlib.clear_cache()
    assert ok
    assert np.all(out.view(np.uint32) == np.array(SENTINEL).view(np.uint32))   # nothing stored
    with pytest.raises(ctlib.CTError) as e:
        ctlib.device_check()
    assert e.value.status == -7
    ctlib.device_check()                          # cleared
    ref, S = oracle.corr2d_f64(img, f, ow, oh)
    out, ok = run_config(ctlib, d_img, f, c, ow, oh, in_w=ow + 4)
    assert ok
    assert_parity(out, ref, S, "after a timed-out launch")
    ctlib.device_check()
