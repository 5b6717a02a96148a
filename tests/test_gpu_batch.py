"""GPU tests of the batched persistent path (many uneven correlations in one
launch): every problem matches the FP64 oracle within 1e-5 * sum|in*f| and is
bit-identical to the single-problem kernel; guard bands stay intact; the
graph can be replayed; bucket tuning reports a valid PP score; the plan's
error word stays clear, and a wait that cannot complete gives up and is
reported."""
import time

import numpy as np
import pytest
import torch

import oracle
import synthetic
from tests.gpu_util import SENTINEL, assert_parity

pytestmark = pytest.mark.gpu


def _alloc_out(ow, oh, device, extra_rows=2, extra_cols=8):
    pitch = synthetic.round_up(max(ow, 1), 4) + extra_cols
    buf = torch.empty((oh + extra_rows, pitch), dtype=torch.float32, device=device)
    buf.view(torch.int32).fill_(int(np.array(SENTINEL).view(np.int32)))
    return buf


def _guards_ok(buf, ow, oh):
    bits = buf.cpu().numpy().view(np.uint32)
    sent = np.array(SENTINEL).view(np.uint32)
    return bool(np.all(bits[:oh, ow:] == sent) and np.all(bits[oh:, :] == sent))


def _make(shapes, seed, device, dtype=torch.float32):
    probs = []
    for k, (ow, oh, fw, fh) in enumerate(shapes):
        img, f = synthetic.make_problem(seed * 1000 + k, ow, oh, fw, fh, pitch_align=8, pad_value=np.nan)
        d_img = torch.from_numpy(img)
        if dtype == torch.bfloat16:
            d_img = d_img.to(torch.bfloat16)
            f = torch.from_numpy(f).to(torch.bfloat16)
        probs.append((img, f, d_img.to(device), _alloc_out(ow, oh, device), ow, oh, fw, fh))
    return probs


SHAPES = [(700, 650, 17, 17), (513, 300, 11, 11), (128, 128, 3, 3), (1, 1, 5, 5), (37, 401, 7, 7),
          (999, 17, 3, 7), (256, 256, 5, 5), (600, 600, 17, 17), (96, 33, 1, 1), (300, 1, 9, 2),
          (64, 64, 17, 17), (1024, 200, 7, 7)]


@pytest.mark.parametrize("tune,forms,order", [(True, "both", "timed"), (False, "both", "buckets"),
                                              (True, "paired", "interleaved"), (False, "paired", "interleaved")])
def test_batch_matches_oracle_and_single_kernel(ctlib, cuda_device, tune, forms, order):
    """forms = "paired": every bucket tile that allows it runs paired
    multiply-adds over output-row pairs (filters of 1, 2 and more rows, odd
    and even widths), with the same bits as the scalar single-problem kernel.
    order: the persistent launch's work list bucket by bucket, interleaved,
    or whichever timed faster."""
    probs = _make(SHAPES, 3, cuda_device)
    b = ctlib.Batch([(d, f, out, ow + fw - 1) for (_, f, d, out, ow, oh, fw, fh) in probs], tune=tune,
                    max_tune_items=4, solo_wave_pct=-1, bucket_forms=forms,
                    work_order=order)   # every problem in the persistent launch
    info = b.info()
    assert info["work_interleaved"] == {"buckets": 0, "interleaved": 1}.get(order, info["work_interleaved"])
    if forms == "paired":
        paired = [bk for bk in b.buckets() if bk["config"]["fma2"]]
        assert len(paired) >= len(b.buckets()) - 1, b.buckets()
        assert any(bk["filter"][1] == 1 for bk in paired) and any(bk["filter"] == (17, 17) for bk in paired)
        for bk in paired:
            assert bk["config"]["unroll"] == 1 and bk["config"]["tile_y"] % 2 == 0
    assert info["n_items"] == len(SHAPES) and info["n_work"] > 0 and info["grid"] > 0
    for rep in range(2):       # the graph is replayable
        b.run()
        torch.cuda.synchronize()
        b.check()
        for (img, f, d, out, ow, oh, fw, fh) in probs:
            assert _guards_ok(out, ow, oh), (ow, oh, fw, fh)
            got = out[:oh, :ow].cpu().numpy()
            ref, S = oracle.corr2d_f64(img, f, ow, oh)
            assert_parity(got, ref, S, f"batch {ow}x{oh} f{fw}x{fh}")
            single = ctlib.conv2d(d, f, ctlib.config(32, 4, 4, 2, 1, 0), in_w=ow + fw - 1)
            torch.cuda.synchronize()
            assert np.array_equal(got.view(np.uint32), single.cpu().numpy().view(np.uint32))
            out[:oh, :ow].fill_(float("nan"))
    for bk in b.buckets():
        c = bk["config"]
        assert c["block_x"] * c["block_y"] == 256 and c["tile_x"] >= 1 and c["tile_y"] >= 1
        if tune:
            assert 0.0 < bk["pp"] <= 1.0 + 1e-12
    # every item is in a bucket of its own filter size
    for i, (_, _, _, _, ow, oh, fw, fh) in enumerate(probs):
        assert b.buckets()[b.item_bucket(i)]["filter"] == (fw, fh)


@pytest.mark.parametrize("forms", ["both", "paired"])
def test_batch_bf16(ctlib, cuda_device, forms):
    shapes = [(300, 200, 9, 9), (1024, 64, 17, 17), (50, 77, 3, 5)]
    probs = _make(shapes, 4, cuda_device, dtype=torch.bfloat16)
    b = ctlib.Batch([(d, f, out, ow + fw - 1) for (_, f, d, out, ow, oh, fw, fh) in probs], tune=False,
                    solo_wave_pct=-1, bucket_forms=forms)
    if forms == "paired":
        assert all(bk["config"]["fma2"] for bk in b.buckets())
    b.run()
    torch.cuda.synchronize()
    b.check()
    for (img, f, d, out, ow, oh, fw, fh) in probs:
        ib = torch.from_numpy(img).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
        fb = f.view(torch.int16).numpy().view(np.uint16)
        ref, S = oracle.corr2d_bf16_f64(ib, fb, ow, oh)
        assert_parity(out[:oh, :ow].cpu().numpy(), ref, S, "batch bf16")
        assert _guards_ok(out, ow, oh)


def test_batch_workload_sampled(ctlib, cuda_device):
    """The 64-problem uneven workload (sides log-uniform in [128, 4096],
    filters {3,5,7,11,17}, seed 2) in one launch, checked on sampled pixels."""
    shapes = synthetic.uneven_batch(2, 64, 128, 4096, (3, 5, 7, 11, 17))
    probs = []
    for k, (side, fs) in enumerate(shapes):
        img, f = synthetic.make_problem(2000 + k, side, side, fs, fs)
        probs.append((img, f, torch.from_numpy(img).to(cuda_device),
                      torch.empty((side, synthetic.round_up(side, 4)), device=cuda_device), side, fs))
    b = ctlib.Batch([(d, f, out, side + fs - 1) for (_, f, d, out, side, fs) in probs], tune=True,
                    max_tune_items=3, solo_evals=16)
    assert b.info()["n_solo"] >= 1        # the largest problems run as their own launches
    b.run()
    torch.cuda.synchronize()
    b.check()
    for k, (img, f, d, out, side, fs) in enumerate(probs):
        xs, ys = synthetic.sample_points(k, side, side, 64)
        ref, S = oracle.corr2d_points(img, f, xs, ys)
        got = out.cpu().numpy()[ys, xs].astype(np.float64)
        assert np.all(np.abs(got - ref) <= 1e-5 * S), (k, side, fs)


def test_tile_grid_limit(ctlib, cuda_device):
    """In the persistent launch, a problem wider than 65535 tiles of any
    candidate tile is refused at plan time (CT_ERR_UNSUPPORTED), tuned or
    not; no kernel runs.  (By default such a problem fills the GPU and runs
    as its own single-problem launch instead, which has no such limit.)"""
    ow = 1 << 24
    img = torch.zeros((1, ow), device=cuda_device)
    out = torch.empty((1, ow), device=cuda_device)
    f = np.ones((1, 1), np.float32)
    for tune in (True, False):
        with pytest.raises(ctlib.CTError) as e:
            ctlib.Batch([(img, f, out, ow)], tune=tune, solo_wave_pct=-1)
        assert e.value.status == -8


def test_wait_timeout_is_reported(ctlib, cuda_device, monkeypatch):
    """With the kernel built to expect 16 bytes per item more than its copies
    deliver, no wait can complete: every block gives up after its bounded
    wait, the error word reports CT_ERR_TIMEOUT, and the context stays usable
    for a normal batch afterwards."""
    probs = _make([(64, 64, 3, 3)], 9, cuda_device)
    items = [(d, f, out, ow + fw - 1) for (_, f, d, out, ow, oh, fw, fh) in probs]
    monkeypatch.setenv("CONVTUNE_NVRTC_EXTRA", "-DCT_TEST_EXTRA_TX=16")
    bad = ctlib.Batch(items, tune=False, solo_wave_pct=-1)
    monkeypatch.delenv("CONVTUNE_NVRTC_EXTRA")
    t0 = time.time()
    bad.run()
    torch.cuda.synchronize()
    assert time.time() - t0 < 30.0
    with pytest.raises(ctlib.CTError) as e:
        bad.check()
    assert e.value.status == -7
    del bad
    good = ctlib.Batch(items, tune=False, solo_wave_pct=-1)
    good.run()
    torch.cuda.synchronize()
    good.check()
    img, f, d, out, ow, oh, fw, fh = probs[0]
    ref, S = oracle.corr2d_f64(img, f, ow, oh)
    assert_parity(out[:oh, :ow].cpu().numpy(), ref, S, "batch after a timed-out run")


@pytest.mark.parametrize("layout", ["timed", "after", "beside"])
def test_solo_problems_in_the_graph(ctlib, cuda_device, layout):
    """A problem that fills the GPU on its own (here: one wave) runs as its
    own tuned single-problem launch in the plan's graph, the others in the
    persistent launch (after the solo launch, beside it, or whichever timed
    faster); all outputs are bit-identical to the single-problem kernel and
    match the oracle (sampled for the big one).  4500^2 outputs exceed one
    wave under every configuration of the space (at most 65,536 outputs per
    block, at most 2,048 threads per SM)."""
    shapes = [(4500, 4500, 17, 17), (300, 200, 17, 17), (513, 300, 11, 11), (64, 64, 3, 3)]
    probs = _make(shapes, 12, cuda_device)
    b = ctlib.Batch([(d, f, out, ow + fw - 1) for (_, f, d, out, ow, oh, fw, fh) in probs], tune=True,
                    max_tune_items=3, solo_wave_pct=100, solo_evals=12, persistent_layout=layout)
    info = b.info()
    assert info["n_solo"] == 1 and b.item_bucket(0) == -1
    assert info["persistent_beside"] == {"after": 0, "beside": 1}.get(layout, info["persistent_beside"])
    assert all(b.item_bucket(i) >= 0 for i in range(1, len(shapes)))
    for rep in range(2):
        b.run()
        torch.cuda.synchronize()
        b.check()
        for k, (img, f, d, out, ow, oh, fw, fh) in enumerate(probs):
            assert _guards_ok(out, ow, oh), (ow, oh, fw, fh)
            got = out[:oh, :ow].cpu().numpy()
            single = ctlib.conv2d(d, f, ctlib.config(32, 4, 4, 2, 1, 0), in_w=ow + fw - 1)
            torch.cuda.synchronize()
            assert np.array_equal(got.view(np.uint32), single.cpu().numpy().view(np.uint32)), k
            if k == 0:
                xs, ys = synthetic.sample_points(7, ow, oh, 2000)
                ref, S = oracle.corr2d_points(img, f, xs, ys)
                assert np.all(np.abs(got[ys, xs].astype(np.float64) - ref) <= 1e-5 * S)
            else:
                ref, S = oracle.corr2d_f64(img, f, ow, oh)
                assert_parity(got, ref, S, f"batch {ow}x{oh} f{fw}x{fh}")
            out[:oh, :ow].fill_(float("nan"))


def test_every_problem_solo(ctlib, cuda_device):
    """With every problem big enough to go solo the graph holds no
    persistent launch; results still match the single-problem kernel."""
    shapes = [(4500, 4500, 5, 5), (4600, 4500, 5, 5)]
    probs = _make(shapes, 13, cuda_device)
    b = ctlib.Batch([(d, f, out, ow + fw - 1) for (_, f, d, out, ow, oh, fw, fh) in probs], tune=False,
                    solo_wave_pct=100, solo_evals=8)
    info = b.info()
    assert info["n_solo"] == 2 and info["n_buckets"] == 0 and info["n_work"] == 0
    b.run()
    torch.cuda.synchronize()
    b.check()
    for (img, f, d, out, ow, oh, fw, fh) in probs:
        got = out[:oh, :ow].cpu().numpy()
        single = ctlib.conv2d(d, f, ctlib.config(16, 16, 4, 2, 1, 1), in_w=ow + fw - 1)
        torch.cuda.synchronize()
        assert np.array_equal(got.view(np.uint32), single.cpu().numpy().view(np.uint32))
        assert _guards_ok(out, ow, oh)


def test_bf16_plan_with_a_solo_problem(ctlib, cuda_device):
    """BF16 storage through a plan that holds a solo launch (4500^2, one wave)
    and a persistent launch (a small problem): bit-identical to the
    single-problem kernel, and within 1e-5 * S of the oracle on the
    BF16-rounded values (widened exactly to FP32; sampled for the big one)."""
    shapes = [(4500, 4500, 5, 5), (300, 200, 9, 9)]
    probs = _make(shapes, 14, cuda_device, dtype=torch.bfloat16)
    b = ctlib.Batch([(d, f, out, ow + fw - 1) for (_, f, d, out, ow, oh, fw, fh) in probs], tune=False,
                    solo_wave_pct=100, solo_evals=8)
    assert b.info()["n_solo"] == 1 and b.item_bucket(0) == -1 and b.item_bucket(1) >= 0
    b.run()
    torch.cuda.synchronize()
    b.check()
    for k, (img, f, d, out, ow, oh, fw, fh) in enumerate(probs):
        assert _guards_ok(out, ow, oh)
        got = out[:oh, :ow].cpu().numpy()
        single = ctlib.conv2d(d, f, ctlib.config(32, 4, 4, 2, 1, 0), in_w=ow + fw - 1)
        torch.cuda.synchronize()
        assert np.array_equal(got.view(np.uint32), single.cpu().numpy().view(np.uint32)), k
        img_b = torch.from_numpy(img).to(torch.bfloat16).float().numpy()
        f_b = f.float().numpy()
        if k == 0:
            xs, ys = synthetic.sample_points(9, ow, oh, 2000)
            ref, S = oracle.corr2d_points(img_b, f_b, xs, ys)
            assert np.all(np.abs(got[ys, xs].astype(np.float64) - ref) <= 1e-5 * S)
        else:
            ref, S = oracle.corr2d_f64(img_b, f_b, ow, oh)
            assert_parity(got, ref, S, "bf16 persistent part")
