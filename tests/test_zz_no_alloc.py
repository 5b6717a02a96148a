"""The batched correlation entry point that allocates nothing.

It exists for callers that cannot allocate device memory when they need the
work done (a fully budgeted device, a latency-critical path, a plugin whose
host owns every allocation): all of its per-call scratch lives in one static
device array.  This file runs last so that, if it fails, a run that stops at
the first failure has already run every other test; it also passes on its own
in a fresh process (the first call performs the per-device set-up)."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synthetic

pytestmark = pytest.mark.gpu

TOL = 1e-5   # |a - b| <= TOL * sum|in*f|, the tolerance of the parity tests


def _problems(ct, seed, shapes, device):
    out = []
    for k, (ow, oh, fw, fh) in enumerate(shapes):
        img, f = synthetic.make_problem(seed * 100 + k, ow, oh, fw, fh, pad_value=np.nan)
        d_img = torch.from_numpy(img).to(device)
        d_out = torch.full((oh, ct.round_up(max(ow, 1), 4)), float("nan"), device=device)
        out.append((img, np.ascontiguousarray(f), d_img, d_out, ow, oh, fw, fh))
    return out


def _items(ct, probs):
    arr = (ct.BatchItem * len(probs))()
    for k, (img, f, d_img, d_out, ow, oh, fw, fh) in enumerate(probs):
        arr[k] = ct.BatchItem(d_img.data_ptr(), d_out.data_ptr(), f.ctypes.data, ow, oh, fw, fh,
                              d_img.stride(0), d_out.stride(0))
    return arr


SHAPES_A = [(300, 200, 17, 17), (513, 64, 3, 3), (1, 1, 5, 5), (129, 77, 11, 7), (64, 300, 32, 32),
            (1000, 17, 1, 1)]
SHAPES_B = [(257, 255, 9, 9), (77, 600, 5, 13), (2048, 40, 17, 17)]


def test_noalloc_matches_conv2d_on_two_calls(ctlib, cuda_device):
    L = ctlib.lib()
    for call, (seed, shapes) in enumerate([(11, SHAPES_A), (12, SHAPES_B)]):
        probs = _problems(ctlib, seed, shapes, cuda_device)
        items = _items(ctlib, probs)
        st = L.ct_batch_run_noalloc(items, len(probs), ctlib.CT_F32, None)
        assert st == 0, L.ct_last_error()
        torch.cuda.synchronize()
        for (img, f, d_img, d_out, ow, oh, fw, fh) in probs:
            got = d_out[:oh, :ow].cpu().numpy()
            ref = ctlib.conv2d(d_img, f, ctlib.config(32, 4, 4, 2, 1, 1), in_w=ow + fw - 1)
            torch.cuda.synchronize()
            ref = ref.cpu().numpy()
            _, S = oracle.corr2d_f64(img, f, ow, oh)
            assert np.all(np.abs(got.astype(np.float64) - ref) <= TOL * S), (call, ow, oh, fw, fh)


def test_noalloc_rejects_oversized_work(ctlib, cuda_device):
    L = ctlib.lib()
    probs = _problems(ctlib, 13, [(8, 8, 3, 3)], cuda_device)
    one = _items(ctlib, probs)
    many = (ctlib.BatchItem * 1025)(*([one[0]] * 1025))
    assert L.ct_batch_run_noalloc(many, 1025, ctlib.CT_F32, None) == -1
    assert b"at most 1024" in L.ct_last_error()
    # 300 problems with 32x32 filters need more than the 1 MiB of scratch
    big = _problems(ctlib, 14, [(4, 4, 32, 32)], cuda_device)
    arr = (ctlib.BatchItem * 300)(*([_items(ctlib, big)[0]] * 300))
    assert L.ct_batch_run_noalloc(arr, 300, ctlib.CT_F32, None) == -1
    assert b"scratch" in L.ct_last_error()
