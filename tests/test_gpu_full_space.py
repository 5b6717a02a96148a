"""Every configuration of the full tuning space against the FP64 oracle.

The tuner compiles and times every point of the space (Sec. 3; Table 1's
parameters plus the unroll switch), so every point must compute the same
correlation.  The problems are ragged (no side a multiple of any tile), the
image's padding columns and the rows below it hold NaN (a read outside the
valid input shows up as NaN in an output), and the output sits inside NaN
sentinel guard bands (a store outside it is caught).  Per pixel
|gpu - oracle| <= 1e-5 * sum|in*f|, and all configurations of one problem are
bit-identical (each adds the taps of an output in (i, j) order with one FMA
each).  Compiles go through the library's on-disk cubin cache in the
benchmark's default location, so a benchmark run after these tests finds the
17x17 variants already built."""
import concurrent.futures as cf
import os
import tempfile

import numpy as np
import pytest
import torch

import oracle
import synthetic
from oracle import space as ospace
from tests.gpu_util import assert_parity, run_config

pytestmark = pytest.mark.gpu

NAN_ROWS = 8


def _cfg(ct, d):
    return ct.config(d["block_x"], d["block_y"], d["tile_x"], d["tile_y"], d["smem"], d["unroll"])


def _image_with_nan_rows(img, device, bf16):
    """The image on the device followed by NAN_ROWS rows of NaN; returns the
    (in_h, pitch) view, whose allocation continues with the NaN rows."""
    full = np.full((img.shape[0] + NAN_ROWS, img.shape[1]), np.nan, dtype=np.float32)
    full[:img.shape[0]] = img
    t = torch.from_numpy(full)
    if bf16:
        t = t.to(torch.bfloat16)
    return t.to(device)[:img.shape[0]]


def _sweep(ct, device, ow, oh, fw, fh, seed, every, bf16=False, taps=0, fma2=0, shfl=0):
    img, f = synthetic.make_problem(seed, ow, oh, fw, fh, pad_value=np.nan, extra_pitch=8 if bf16 else 4,
                                    pitch_align=8 if bf16 else 4)
    if bf16:
        img_bits = torch.from_numpy(img).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
        f_t = torch.from_numpy(np.ascontiguousarray(f)).to(torch.bfloat16)
        f_bits = f_t.view(torch.int16).numpy().view(np.uint16)
        ref, S = oracle.corr2d_bf16_f64(img_bits, f_bits, ow, oh)
        filt = f_t
    else:
        ref, S = oracle.corr2d_f64(img, f, ow, oh)
        filt = f
    d_img = _image_with_nan_rows(img, device, bf16)
    in_w = ow + fw - 1
    p = ct.problem_for(d_img, filt, in_w=in_w)
    ents = ospace.enumerate_space("full", fw, fh)
    if taps:                                      # compiled-in taps apply to the unrolled variants
        ents = [e for e in ents if e[1]["unroll"]]
    if fma2:                                      # paired multiply-adds: unrolled, two output rows or more
        ents = [e for e in ents if e[1]["unroll"] and e[1]["tile_y"] >= 2]
    if shfl:                                      # shuffled windows: staged halo, whole warps, 4-wide tiles
        ents = [e for e in ents if e[1]["smem"] and e[1]["block_x"] % 32 == 0 and e[1]["tile_x"] % 4 == 0]
    ents = ents[::every]
    cfgs = [_cfg(ct, c) for _, c in ents]
    for c in cfgs:
        c.taps = taps
        c.fma2 = fma2
        c.shfl = shfl
    lib_cfgs = {c.space_tuple() for _, c in ct.Space("full").enumerate(p)}
    assert {c.space_tuple() for c in cfgs} <= lib_cfgs

    cache = os.path.join(tempfile.gettempdir(), f"convtune-cache-{os.getuid()}")
    ct.set_cache_dir(cache)
    try:
        first = None
        chunk = 256
        pre = lambda c: ct.compile_variant(p, c, filt)
        with cf.ThreadPoolExecutor(os.cpu_count() or 8) as ex:
            nxt = ex.map(pre, cfgs[:chunk])
            for k in range(0, len(cfgs), chunk):
                list(nxt)                                  # this chunk is compiled
                if k + chunk < len(cfgs):                  # the next one compiles while this one runs
                    nxt = ex.map(pre, cfgs[k + chunk:k + 2 * chunk])
                for c in cfgs[k:k + chunk]:
                    out, ok = run_config(ct, d_img, filt, c, ow, oh, in_w=in_w)
                    assert ok, f"guard band overwritten by {c}"
                    assert_parity(out, ref, S, f"{ow}x{oh}/{fw}x{fh} {c}")
                    if first is None:
                        first = out
                    else:
                        assert np.array_equal(out.view(np.uint32), first.view(np.uint32)), f"{c} differs bitwise"
                ct.clear_cache()                           # unload this chunk's modules
        ct.device_check()
    finally:
        ct.set_cache_dir(None)
    return len(cfgs), first


def test_full_space_every_config_17x17(ctlib, cuda_device):
    """All 5,576 valid points of the full space for a 17x17 filter (the
    filter of the 4096x4096 workload) on a 333x157 output."""
    n, _ = _sweep(ctlib, cuda_device, 333, 157, 17, 17, seed=21, every=1)
    assert n == 5576


def test_full_space_eighth_5x7(ctlib, cuda_device):
    """Every 8th valid point (canonical order) for a 5-wide, 7-high filter on
    a 301x163 output."""
    n, _ = _sweep(ctlib, cuda_device, 301, 163, 5, 7, seed=22, every=8)
    assert n == len(ospace.enumerate_space("full", 5, 7)[::8])


def test_full_space_bf16_sixteenth_9x9(ctlib, cuda_device):
    """BF16 storage: every 16th valid point for the 9x9 filter of the BF16
    workloads on a 259x131 output, against the oracle on the BF16 values."""
    n, _ = _sweep(ctlib, cuda_device, 259, 131, 9, 9, seed=23, every=16, bf16=True)
    assert n == len(ospace.enumerate_space("full", 9, 9)[::16])


@pytest.mark.parametrize("bf16", [False, True], ids=["f32", "bf16"])
def test_compiled_taps_same_bits(ctlib, cuda_device, bf16):
    """Taps compiled into the variant (ct_config.taps = 1): every 24th unrolled
    point of the full space for a 17x17 filter (every 48th for BF16) matches
    the oracle, and its bits equal those of the parameter-block form."""
    every = 48 if bf16 else 24
    n1, with_imm = _sweep(ctlib, cuda_device, 333, 157, 17, 17, seed=24, every=every, bf16=bf16, taps=1)
    n0, with_param = _sweep(ctlib, cuda_device, 333, 157, 17, 17, seed=24, every=10 ** 6, bf16=bf16, taps=0)
    assert n1 > 100 // (2 if bf16 else 1) and n0 == 1
    assert np.array_equal(with_imm.view(np.uint32), with_param.view(np.uint32))


def test_compiled_taps_follow_the_filter(ctlib, cuda_device):
    """Two filters of one size through the same compiled-taps configuration, one
    after the other and back: each call runs its own filter's variant; a
    filter with a non-finite tap falls back to the parameter-block form."""
    ow, oh, fs = 200, 120, 9
    img, f1 = synthetic.make_problem(41, ow, oh, fs, fs)
    _, f2 = synthetic.make_problem(42, ow, oh, fs, fs)
    d_img = torch.from_numpy(img).to(cuda_device)
    c_imm = ctlib.config(16, 8, 4, 2, 1, 1, taps=1)
    c_par = ctlib.config(16, 8, 4, 2, 1, 1, taps=0)
    for f in (f1, f2, f1):
        ref, S = oracle.corr2d_f64(img, f, ow, oh)
        a, ok_a = run_config(ctlib, d_img, f, c_imm, ow, oh, in_w=ow + fs - 1)
        b, ok_b = run_config(ctlib, d_img, f, c_par, ow, oh, in_w=ow + fs - 1)
        assert ok_a and ok_b
        assert_parity(a, ref, S, "compiled taps")
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    f3 = f1.copy()
    f3[4, 4] = np.inf
    a, ok_a = run_config(ctlib, d_img, f3, c_imm, ow, oh, in_w=ow + fs - 1)
    b, ok_b = run_config(ctlib, d_img, f3, c_par, ow, oh, in_w=ow + fs - 1)
    assert ok_a and ok_b and np.array_equal(a.view(np.uint32), b.view(np.uint32))


@pytest.mark.parametrize("case", ["f32_17x17", "f32_5x7", "bf16_9x9"])
def test_paired_fma_same_bits(ctlib, cuda_device, case):
    """Paired multiply-adds (ct_config.fma2 = 1, output rows 2k and 2k+1 share
    each input row through one f32x2 FMA per column and tap): a spread of the
    unrolled points with two or more output rows per thread (every 16th for
    17x17, every 4th for 5x7, every 24th for BF16 9x9) matches the oracle, and
    its bits equal those of the scalar form."""
    ow, oh, fw, fh, bf16, every = {"f32_17x17": (333, 157, 17, 17, False, 16), "f32_5x7": (301, 163, 5, 7, False, 4),
                                   "bf16_9x9": (259, 131, 9, 9, True, 24)}[case]
    n2, paired = _sweep(ctlib, cuda_device, ow, oh, fw, fh, seed=25, every=every, bf16=bf16, fma2=1)
    n0, scalar = _sweep(ctlib, cuda_device, ow, oh, fw, fh, seed=25, every=10 ** 6, bf16=bf16)
    assert n2 >= 40 and n0 == 1
    assert np.array_equal(paired.view(np.uint32), scalar.view(np.uint32))


@pytest.mark.parametrize("case", ["f32_17x17", "f32_5x7", "bf16_9x9"])
def test_shuffled_window_same_bits(ctlib, cuda_device, case):
    """Windows assembled by warp shuffles (ct_config.shfl = 1): a spread of the
    staged points with whole warps per thread row and 4-wide register tiles
    (every 4th for 17x17 and 5x7, every 6th for BF16 9x9; unrolled and rolled,
    tensor-copy and per-thread staging) matches the oracle, bit for bit the
    same as the shared-memory windows."""
    ow, oh, fw, fh, bf16, every = {"f32_17x17": (333, 157, 17, 17, False, 4), "f32_5x7": (301, 163, 5, 7, False, 4),
                                   "bf16_9x9": (259, 131, 9, 9, True, 6)}[case]
    n1, shuffled = _sweep(ctlib, cuda_device, ow, oh, fw, fh, seed=26, every=every, bf16=bf16, shfl=1)
    n0, plain = _sweep(ctlib, cuda_device, ow, oh, fw, fh, seed=26, every=10 ** 6, bf16=bf16)
    assert n1 >= 30 and n0 == 1
    assert np.array_equal(shuffled.view(np.uint32), plain.view(np.uint32))


@pytest.mark.parametrize("fw,fh", [(17, 17), (5, 7)])
def test_partial_unroll_same_bits(ctlib, cuda_device, fw, fh):
    """Partial unroll factors 2 and 4 of the filter-row loop (Sec. 3) over a
    spread of block shapes, tiles and both staging forms: every variant matches
    the oracle and gives the bits of the rolled and fully unrolled forms."""
    ow, oh = 301, 163
    img, f = synthetic.make_problem(27, ow, oh, fw, fh, pad_value=np.nan, extra_pitch=4)
    ref, S = oracle.corr2d_f64(img, f, ow, oh)
    d_img = _image_with_nan_rows(img, cuda_device, False)
    p = ctlib.problem_for(d_img, f, in_w=ow + fw - 1)
    sp = ctlib.Space('{"block_x": [16, 32], "block_y": [4, 8], "tile_x": [1, 2, 4], "tile_y": [1, 3], '
                     '"use_smem": [0, 1], "unroll": [0, 1, 2, 4]}')
    cfgs = [c for _, c in sp.enumerate(p)]
    assert len(cfgs) == 2 * 2 * 3 * 2 * 2 * 4
    with cf.ThreadPoolExecutor(os.cpu_count() or 8) as ex:
        list(ex.map(lambda c: ctlib.compile_variant(p, c), cfgs))
    first = None
    for c in cfgs:
        out, ok = run_config(ctlib, d_img, f, c, ow, oh, in_w=ow + fw - 1)
        assert ok, f"guard band overwritten by {c}"
        assert_parity(out, ref, S, repr(c))
        if first is None:
            first = out
        else:
            assert np.array_equal(out.view(np.uint32), first.view(np.uint32)), f"{c} differs bitwise"
    ctlib.clear_cache()
