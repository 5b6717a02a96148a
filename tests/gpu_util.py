"""Helpers for GPU parity tests: upload seeded inputs, run one configuration
through the C-ABI with sentinel guard bands around the output, compare with
the oracle under the per-pixel bound |gpu - ref| <= 1e-5 * sum|in*f|."""
from __future__ import annotations

import numpy as np
import torch

TOL = 1e-5          # per-pixel tolerance relative to S = sum |in * f|
SENTINEL = np.array([0x7FC0DEAD], dtype=np.uint32).view(np.float32)[0]   # a NaN with a payload


def upload_image(img: np.ndarray, device, dtype=torch.float32):
    t = torch.from_numpy(np.ascontiguousarray(img))
    if dtype == torch.bfloat16:
        t = t.to(torch.bfloat16)
    return t.to(device)


def run_config(ct, d_img, filt, cfg, out_w, out_h, *, in_w=None, guard_rows=2, extra_pitch=8, stream=None):
    """Runs cfg into an output buffer with padding columns and extra rows all
    holding SENTINEL; returns (result (out_h, out_w) float32 numpy, guards_ok)."""
    pitch = ct.round_up(max(out_w, 1), 4) + extra_pitch
    buf = torch.full((out_h + guard_rows, pitch), float("nan"), dtype=torch.float32, device=d_img.device)
    buf.view(torch.int32).fill_(int(np.array(SENTINEL).view(np.int32)))
    ct.conv2d(d_img, filt, cfg, in_w=in_w, out=buf, stream=stream)
    torch.cuda.synchronize()
    h = buf.cpu().numpy()
    bits = h.view(np.uint32)
    sent = np.array(SENTINEL).view(np.uint32)
    guards_ok = bool(np.all(bits[:out_h, out_w:] == sent) and np.all(bits[out_h:, :] == sent))
    return h[:out_h, :out_w].copy(), guards_ok


def assert_parity(gpu: np.ndarray, ref: np.ndarray, S: np.ndarray, what=""):
    assert gpu.shape == ref.shape, (gpu.shape, ref.shape)
    err = np.abs(gpu.astype(np.float64) - ref)
    bound = TOL * S
    bad = ~(err <= bound)
    if bad.any():
        y, x = np.argwhere(bad)[0]
        raise AssertionError(f"{what}: {int(bad.sum())} pixels outside 1e-5*S; first at (y={y}, x={x}): "
                             f"gpu={gpu[y, x]!r} ref={ref[y, x]!r} S={S[y, x]!r}")
