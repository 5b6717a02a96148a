"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds no arithmetic of the correlation method itself: it only turns
a seed into image/filter values.  Both the CUDA path and the CPU oracle consume
the arrays it returns, so neither side has to trust the other's generator.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), used in its counter form: the i-th draw
(i = 0, 1, ...) of stream ``seed`` is ``mix(seed + (i + 1) * GAMMA)``.

Value mapping (uniform on [-1, 1)): ``v = (u >> 40) * 2**-23 - 1``.  The top 24
bits of each draw give a multiple of 2**-23 in [-1, 1), which a float32 holds
exactly, so a float64 computation on these values starts from exactly the same
numbers the GPU sees.

Draw order for one problem: the image row-major (in_h rows of in_w values,
padding columns excluded), then the filter row-major (fh rows of fw values).
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Draws ``start .. start+count-1`` of the SplitMix64 stream ``seed`` (uint64)."""
    with np.errstate(over="ignore"):
        idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_pm1(seed: int, start: int, count: int) -> np.ndarray:
    """float32 values on the 2**-23 grid in [-1, 1)."""
    u = splitmix64(seed, start, count)
    k = (u >> np.uint64(40)).astype(np.int64)
    return (k.astype(np.float64) * 2.0 ** -23 - 1.0).astype(np.float32)


def small_ints(seed: int, start: int, count: int, lo: int = -8, hi: int = 8) -> np.ndarray:
    """Integer-valued float32 in [lo, hi] (for exact-arithmetic cases)."""
    u = splitmix64(seed, start, count)
    span = np.uint64(hi - lo + 1)
    return ((u >> np.uint64(32)) % span).astype(np.int64).astype(np.float32) + np.float32(lo)


def round_up(v: int, m: int) -> int:
    return (v + m - 1) // m * m


def make_problem(seed: int, out_w: int, out_h: int, fw: int, fh: int, *,
                 kind: str = "uniform", pitch_align: int = 4, pad_value: float = 0.0,
                 extra_pitch: int = 0):
    """Builds one single-channel problem.

    Returns ``(image, filt)``: ``image`` is float32 of shape (in_h, in_pitch)
    with ``in_h = out_h + fh - 1``, ``in_w = out_w + fw - 1`` valid columns and
    ``in_pitch = round_up(in_w, pitch_align) + extra_pitch`` (padding columns
    hold ``pad_value``); ``filt`` is float32 of shape (fh, fw).
    """
    in_w, in_h = out_w + fw - 1, out_h + fh - 1
    pitch = round_up(max(in_w, 1), pitch_align) + extra_pitch
    gen = {"uniform": uniform_pm1, "int": small_ints}[kind]
    vals = gen(seed, 0, in_w * in_h)
    img = np.full((in_h, pitch), pad_value, dtype=np.float32)
    img[:, :in_w] = vals.reshape(in_h, in_w)
    filt = gen(seed, in_w * in_h, fw * fh).reshape(fh, fw)
    return img, filt


def sample_points(seed: int, out_w: int, out_h: int, n: int):
    """n output coordinates (x, y) for sampled checks at full size, always
    including the four corners; drawn from stream ``seed`` at a far offset."""
    u = splitmix64(seed, 1 << 40, 2 * n)
    xs = (u[0::2] % np.uint64(out_w)).astype(np.int64)
    ys = (u[1::2] % np.uint64(out_h)).astype(np.int64)
    corners_x = np.array([0, out_w - 1, 0, out_w - 1], dtype=np.int64)
    corners_y = np.array([0, 0, out_h - 1, out_h - 1], dtype=np.int64)
    return np.concatenate([corners_x, xs]), np.concatenate([corners_y, ys])


def uneven_batch(seed: int, count: int, side_lo: int, side_hi: int, filters):
    """Shapes of a batch of uneven problems: square output sides log-uniform in
    [side_lo, side_hi] and filter sizes drawn uniformly from ``filters``.
    Returns a list of (side, f) pairs."""
    u = splitmix64(seed, 1 << 41, 2 * count)
    a = (u[0::2] >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    sides = np.rint(np.exp(np.log(side_lo) + a * (np.log(side_hi) - np.log(side_lo)))).astype(np.int64)
    fi = (u[1::2] % np.uint64(len(filters))).astype(np.int64)
    return [(int(s), int(filters[k])) for s, k in zip(sides, fi)]
