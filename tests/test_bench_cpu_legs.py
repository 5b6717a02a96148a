"""The host-side checks bench.py attaches to its JSON line, on CPU: the
per-pixel parity record, and the oracle legs of the batched workload and the
BF16 cases fed with results that are right (float32 roundings of the oracle)
or wrong in one pixel."""
import numpy as np
import pytest

import bench
import oracle
import synthetic


def test_parity_record_bound_and_zero_weight_pixels():
    ref = np.array([[1.0, 2.0, 0.0]])
    S = np.array([[10.0, 10.0, 0.0]])
    ok = bench.parity_record(np.array([[1.00005, 2.0, 0.0]], np.float32), ref, S, "t")
    assert ok["ok"] and ok["n"] == 3 and ok["max_err_over_S"] <= 1e-5
    bad = bench.parity_record(np.array([[1.0002, 2.0, 0.0]], np.float32), ref, S, "t")
    assert not bad["ok"] and bad["max_err_over_S"] > 1e-5
    # S = 0 (all-zero window): only an exact zero passes
    zero = bench.parity_record(np.array([[1.0, 2.0, 1e-30]], np.float32), ref, S, "t")
    assert not zero["ok"] and zero["max_err_over_S"] == np.inf


def _batch_results(wrong=None):
    res = []
    for k, (side, fs) in enumerate([(40, 5), (23, 3), (17, 7)]):
        img, f = synthetic.make_problem(500 + k, side, side, fs, fs)
        ref, _ = oracle.corr2d_f64(img, f, side, side)
        got = ref.astype(np.float32)
        if wrong == k:
            got[3, 4] += np.float32(1e-3)
        res.append((img, f, got, side, fs))
    return res


def test_batch_leg_checks_every_pixel():
    rec = bench.cpu_baseline_batch(_batch_results(), 5.0)
    assert rec["parity"]["ok"] and rec["parity"]["problems"] == 3
    assert rec["parity"]["n"] == 40 * 40 + 23 * 23 + 17 * 17
    assert rec["kind"] == "oracle" and rec["value"] > 0
    assert not bench.cpu_baseline_batch(_batch_results(wrong=2), 5.0)["parity"]["ok"]


def test_bf16_leg_errors():
    import torch
    ow, oh, fs = 48, 31, 5
    img32, f32 = synthetic.make_problem(77, ow, oh, fs, fs, pitch_align=8)
    img_t = torch.from_numpy(img32).to(torch.bfloat16)
    f_t = torch.from_numpy(np.ascontiguousarray(f32)).to(torch.bfloat16)
    ib = img_t.view(torch.int16).numpy().view(np.uint16)
    fb = np.ascontiguousarray(f_t.view(torch.int16).numpy().view(np.uint16))
    refb, _ = oracle.corr2d_bf16_f64(ib, fb, ow, oh)
    ref32, S32 = oracle.corr2d_f64(img32, f32, ow, oh)
    good = refb.astype(np.float32)
    bad = good.copy()
    bad[0, 0] += np.float32(0.5)
    rec = bench.cpu_baseline_bf16((img32, np.ascontiguousarray(f32), ib, fb, ow, oh,
                                   {"tuned": good, "default": bad}))
    assert rec["tuned"]["parity_vs_bf16_oracle"]["ok"]
    assert not rec["default"]["parity_vs_bf16_oracle"]["ok"]
    # BF16 rounding of inputs costs far more than FP32 summation, far less than the values
    e = rec["tuned"]["max_err_over_S_vs_fp32_inputs"]
    assert 1e-5 < e < 2e-2
    want = np.sqrt(np.mean((refb - ref32) ** 2)) / np.sqrt(np.mean(ref32 ** 2))
    assert rec["tuned"]["rms_err_rel_vs_fp32_inputs"] == pytest.approx(want, rel=1e-3)
