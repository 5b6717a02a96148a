"""Pins for the correlation oracle: checks against facts fixed by the
mathematics, not by the oracle itself.  Each pin takes ``corr(image, filt,
out_w, out_h) -> (out, S)`` so the same pins can be run against deliberately
broken copies of the oracle (see test_oracle_mutations.py)."""
from __future__ import annotations

from fractions import Fraction

import numpy as np

import synthetic


def _exact_fraction(image, filt, out_w, out_h):
    fh, fw = filt.shape
    out = [[Fraction(0)] * out_w for _ in range(out_h)]
    for y in range(out_h):
        for x in range(out_w):
            s = Fraction(0)
            for i in range(fh):
                for j in range(fw):
                    s += Fraction(float(image[y + i, x + j])) * Fraction(float(filt[i, j]))
            out[y][x] = s
    return out


def pin_bruteforce_fraction(corr):
    """Tiny inputs against exact rational arithmetic (pure Python loops)."""
    for k, (ow, oh, fw, fh) in enumerate([(1, 1, 1, 1), (5, 3, 3, 2), (4, 6, 2, 5), (8, 8, 3, 3), (3, 7, 5, 1)]):
        img, f = synthetic.make_problem(100 + k, ow, oh, fw, fh)
        out, S = corr(img, f, ow, oh)
        ex = _exact_fraction(img, f, ow, oh)
        for y in range(oh):
            for x in range(ow):
                err = abs(Fraction(out[y, x]) - ex[y][x])
                bound = Fraction(fw * fh + 1) * Fraction(2.0 ** -52) * Fraction(S[y, x])
                assert err <= bound, (ow, oh, fw, fh, y, x)
                # S is sum |in*f| (exact up to fp64 rounding)
                exS = sum(abs(Fraction(float(img[y + i, x + j])) * Fraction(float(f[i, j])))
                          for i in range(fh) for j in range(fw))
                assert abs(Fraction(S[y, x]) - exS) <= Fraction(fw * fh + 1) * Fraction(2.0 ** -52) * exS


def pin_exact_integers(corr):
    """Integer-valued inputs: every partial sum is an integer below 2**53, so
    the FP64 result must equal the integer sum exactly."""
    ow, oh, fw, fh = 9, 7, 4, 3
    img, f = synthetic.make_problem(7, ow, oh, fw, fh, kind="int")
    out, _ = corr(img, f, ow, oh)
    I = img.astype(np.int64)
    F = f.astype(np.int64)
    for y in range(oh):
        for x in range(ow):
            s = 0
            for i in range(fh):
                for j in range(fw):
                    s += int(I[y + i, x + j]) * int(F[i, j])
            assert out[y, x] == s


def pin_impulse(corr):
    """A filter that is 1 at (a, b) and 0 elsewhere selects in[y+a][x+b]:
    this fixes both offsets, the absence of a flip and the operand order."""
    ow, oh, fw, fh = 6, 5, 4, 3
    img, _ = synthetic.make_problem(3, ow, oh, fw, fh)
    for a in range(fh):
        for b in range(fw):
            f = np.zeros((fh, fw), np.float32)
            f[a, b] = 1.0
            out, _ = corr(img, f, ow, oh)
            assert np.array_equal(out, img[a:a + oh, b:b + ow].astype(np.float64)), (a, b)


def pin_linearity(corr):
    """Linear in the image and in the filter.  Integer-valued inputs make every
    step exact, so the identity must hold exactly; uniform inputs hold it up to
    the float32 rounding of the combined input (2**-24 relative per element)."""
    ow, oh, fw, fh = 11, 9, 5, 3
    x1, f1 = synthetic.make_problem(21, ow, oh, fw, fh, kind="int")
    x2, f2 = synthetic.make_problem(22, ow, oh, fw, fh, kind="int")
    a, b = np.float32(3.0), np.float32(-2.0)
    o1, _ = corr(x1, f1, ow, oh)
    o2, _ = corr(x2, f1, ow, oh)
    o12, _ = corr(a * x1 + b * x2, f1, ow, oh)
    assert np.array_equal(o12, 3.0 * o1 - 2.0 * o2)
    g1, _ = corr(x1, f1, ow, oh)
    g2, _ = corr(x1, f2, ow, oh)
    g12, _ = corr(x1, a * f1 + b * f2, ow, oh)
    assert np.array_equal(g12, 3.0 * g1 - 2.0 * g2)
    u1, h1 = synthetic.make_problem(23, ow, oh, fw, fh)
    u2, _ = synthetic.make_problem(24, ow, oh, fw, fh)
    c, d = np.float32(0.75), np.float32(-1.5)
    p1, S1 = corr(u1, h1, ow, oh)
    p2, S2 = corr(u2, h1, ow, oh)
    p12, _ = corr(c * u1 + d * u2, h1, ow, oh)
    assert np.all(np.abs(p12 - (0.75 * p1 - 1.5 * p2)) <= 2.0 ** -22 * (0.75 * S1 + 1.5 * S2))


def pin_shift(corr):
    """Shifting the image by (dy, dx) shifts the output by the same amount."""
    ow, oh, fw, fh = 10, 8, 3, 4
    big, f = synthetic.make_problem(31, ow + 3, oh + 2, fw, fh)
    full, _ = corr(big, f, ow + 3, oh + 2)
    for dy, dx in [(0, 0), (1, 2), (2, 3), (0, 1)]:
        sub = np.ascontiguousarray(big[dy:, dx:])
        o, _ = corr(sub, f, ow, oh)
        assert np.array_equal(o, full[dy:dy + oh, dx:dx + ow]), (dy, dx)


def pin_separable(corr):
    """f = u v^T: the 2D result equals a 1D correlation along x with v followed
    by one along y with u (numpy.correlate as the 1D routine).  u and v are
    small multiples of 1/8, so their outer product is exact in float32."""
    ow, oh, fw, fh = 12, 10, 5, 3
    img, _ = synthetic.make_problem(41, ow, oh, fw, fh)
    u = synthetic.small_ints(42, 0, fh).astype(np.float64) / 8.0
    v = synthetic.small_ints(43, 0, fw).astype(np.float64) / 8.0
    f = np.outer(u, v).astype(np.float32)
    assert np.array_equal(f.astype(np.float64), np.outer(u, v))
    out, S = corr(img, f, ow, oh)
    X = img[:oh + fh - 1, :ow + fw - 1].astype(np.float64)
    rows = np.stack([np.correlate(X[r], v, mode="valid") for r in range(X.shape[0])])
    ref = np.stack([np.correlate(rows[:, c], u, mode="valid") for c in range(rows.shape[1])], axis=1)
    assert np.all(np.abs(out - ref) <= 1e-12 * (S + 1.0))


def pin_torch_conv2d(corr):
    """torch.nn.functional.conv2d on CPU in float64 is a valid cross-correlation."""
    import torch
    ow, oh, fw, fh = 23, 17, 7, 5
    img, f = synthetic.make_problem(51, ow, oh, fw, fh)
    out, S = corr(img, f, ow, oh)
    X = torch.from_numpy(img[:oh + fh - 1, :ow + fw - 1].astype(np.float64))[None, None]
    W = torch.from_numpy(f.astype(np.float64))[None, None]
    ref = torch.nn.functional.conv2d(X, W)[0, 0].numpy()
    assert np.all(np.abs(out - ref) <= 1e-13 * S + 1e-300)


def pin_asymmetric(corr):
    """A non-symmetric filter on a ramp image: in[y][x] = 64 y + x gives
    out = sum f[i][j] (64 (y+i) + x + j), a closed form that a transposed,
    flipped or mis-offset filter breaks."""
    ow, oh, fw, fh = 7, 6, 3, 2
    H, W = oh + fh - 1, ow + fw - 1
    img = np.zeros((H, 12), np.float32)
    for y in range(H):
        for x in range(W):
            img[y, x] = 64 * y + x
    f = np.array([[1, 2, 3], [5, 7, 11]], np.float32)
    out, _ = corr(img, f, ow, oh)
    for y in range(oh):
        for x in range(ow):
            want = sum(float(f[i, j]) * (64 * (y + i) + x + j) for i in range(fh) for j in range(fw))
            assert out[y, x] == want


ALL_PINS = [pin_bruteforce_fraction, pin_exact_integers, pin_impulse, pin_linearity,
            pin_shift, pin_separable, pin_torch_conv2d, pin_asymmetric]
