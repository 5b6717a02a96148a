"""The batched correlation entry point that allocates nothing.

It exists for callers that cannot allocate device memory when they need the
work done (a fully budgeted device, a latency-critical path, a plugin whose
host owns every allocation): all of its per-call scratch lives in one static
device array.  This file runs last so that, if it fails, a run that stops at
the first failure has already run every other test; it also passes on its own
in a fresh process (the first call performs the per-device set-up).

Each call is checked three ways: against the FP64 oracle within the parity
tolerance, bit for bit against ct_conv2d (both add the taps of an output in
(i, j) order with one FMA each), and for stores outside the outputs (the
columns between out_w and the pitch and two rows below hold a NaN sentinel
that must survive)."""
import numpy as np
import pytest
import torch

import oracle
import synthetic
from tests.gpu_util import SENTINEL

pytestmark = pytest.mark.gpu

TOL = 1e-5   # |a - b| <= TOL * sum|in*f|, the tolerance of the parity tests
GUARD_ROWS = 2
EXTRA_PITCH = 8


def _problems(ct, seed, shapes, device, bf16):
    out = []
    sent = int(np.array(SENTINEL).view(np.int32))
    for k, (ow, oh, fw, fh) in enumerate(shapes):
        img, f = synthetic.make_problem(seed * 100 + k, ow, oh, fw, fh, pad_value=np.nan,
                                        pitch_align=8 if bf16 else 4)
        if bf16:
            t_img = torch.from_numpy(img).to(torch.bfloat16)
            t_f = torch.from_numpy(np.ascontiguousarray(f)).to(torch.bfloat16)
            h_img = t_img.view(torch.int16).numpy().view(np.uint16)
            h_f = np.ascontiguousarray(t_f.view(torch.int16).numpy().view(np.uint16))
            ref, S = oracle.corr2d_bf16_f64(h_img, h_f, ow, oh)
            d_img, filt = t_img.to(device), t_f
        else:
            h_f = np.ascontiguousarray(f)
            ref, S = oracle.corr2d_f64(img, h_f, ow, oh)
            d_img, filt = torch.from_numpy(img).to(device), h_f
        d_out = torch.empty((oh + GUARD_ROWS, ct.round_up(max(ow, 1), 4) + EXTRA_PITCH), device=device)
        d_out.view(torch.int32).fill_(sent)
        out.append(dict(h_f=h_f, filt=filt, d_img=d_img, d_out=d_out, ref=ref, S=S, ow=ow, oh=oh, fw=fw, fh=fh))
    return out


def _items(ct, probs):
    arr = (ct.BatchItem * len(probs))()
    for k, q in enumerate(probs):
        arr[k] = ct.BatchItem(q["d_img"].data_ptr(), q["d_out"].data_ptr(), q["h_f"].ctypes.data, q["ow"], q["oh"],
                              q["fw"], q["fh"], q["d_img"].stride(0), q["d_out"].stride(0))
    return arr


SHAPES_A = [(300, 200, 17, 17), (513, 64, 3, 3), (1, 1, 5, 5), (129, 77, 11, 7), (64, 300, 32, 32),
            (1000, 17, 1, 1)]
SHAPES_B = [(257, 255, 9, 9), (77, 600, 5, 13), (2048, 40, 17, 17)]


@pytest.mark.parametrize("bf16", [False, True], ids=["f32", "bf16"])
def test_noalloc_matches_oracle_and_conv2d_on_two_calls(ctlib, cuda_device, bf16):
    L = ctlib.lib()
    dtype = ctlib.CT_BF16 if bf16 else ctlib.CT_F32
    sent = np.array(SENTINEL).view(np.uint32)
    for call, (seed, shapes) in enumerate([(11, SHAPES_A), (12, SHAPES_B)]):
        probs = _problems(ctlib, seed + (50 if bf16 else 0), shapes, cuda_device, bf16)
        items = _items(ctlib, probs)
        st = L.ct_batch_run_noalloc(items, len(probs), dtype, None)
        assert st == 0, L.ct_last_error()
        torch.cuda.synchronize()
        for q in probs:
            ow, oh = q["ow"], q["oh"]
            h = q["d_out"].cpu().numpy()
            bits = h.view(np.uint32)
            assert np.all(bits[:oh, ow:] == sent) and np.all(bits[oh:, :] == sent), ("stores outside", call, ow, oh)
            got = h[:oh, :ow]
            err = np.abs(got.astype(np.float64) - q["ref"])
            assert np.all(err <= TOL * q["S"]), (call, ow, oh, q["fw"], q["fh"], float(np.nanmax(err / q["S"])))
            want = ctlib.conv2d(q["d_img"], q["filt"], ctlib.config(32, 4, 4, 2, 1, 1), in_w=ow + q["fw"] - 1)
            torch.cuda.synchronize()
            assert np.array_equal(got.view(np.uint32), want.cpu().numpy().view(np.uint32)), \
                ("not bit-identical to ct_conv2d", call, ow, oh, q["fw"], q["fh"])


def test_noalloc_rejects_oversized_work(ctlib, cuda_device):
    L = ctlib.lib()
    probs = _problems(ctlib, 13, [(8, 8, 3, 3)], cuda_device, False)
    one = _items(ctlib, probs)
    many = (ctlib.BatchItem * 1025)(*([one[0]] * 1025))
    assert L.ct_batch_run_noalloc(many, 1025, ctlib.CT_F32, None) == -1
    assert b"at most 1024" in L.ct_last_error()
    # 300 problems with 32x32 filters need more than the 1 MiB of scratch
    big = _problems(ctlib, 14, [(4, 4, 32, 32)], cuda_device, False)
    arr = (ctlib.BatchItem * 300)(*([_items(ctlib, big)[0]] * 300))
    assert L.ct_batch_run_noalloc(arr, 300, ctlib.CT_F32, None) == -1
    assert b"scratch" in L.ct_last_error()
