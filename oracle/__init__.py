"""CPU oracle — TEST INFRASTRUCTURE, not part of the product.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA library
(``paper_2407_11488_gb300``) and never imports it.

Contents:
  * ``corr2d_f64`` / ``corr2d_points`` / ``corr2d_bf16_f64`` — the plain FP64
    definition of single-channel valid cross-correlation (C, OpenMP over rows;
    see ``corr2d_f64.c`` for the definition and its citation).
  * ``oracle.space``    — the tuning search spaces written out by definition.
  * ``oracle.analysis`` — ranking and the paper's metrics over a timing table
    (tuning impact, Sec. 4; proportion of centrality, Eq. 1; performance
    portability, Eqs. 2-3).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "corr2d_f64.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compiles the C oracle with gcc (OpenMP if available).  Plain -O2, no
    target-specific flags, so the same source builds on x86_64 and aarch64."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, i32, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
            lib.oracle_corr2d_f64.argtypes = [vp, i64, i32, i32, vp, i32, i32, vp, vp, i32]
            lib.oracle_corr2d_f64_points.argtypes = [vp, i64, vp, i32, i32, vp, vp, i64, vp, vp]
            lib.oracle_corr2d_bf16_f64.argtypes = [vp, i64, i32, i32, vp, i32, i32, vp, vp, i32]
            lib.oracle_max_threads.restype = i32
            _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def corr2d_f64(image: np.ndarray, filt: np.ndarray, out_w: int, out_h: int, nthreads: int = 0):
    """Valid cross-correlation in FP64.  ``image`` is float32 (in_h, in_pitch)
    with at least out_w+fw-1 valid columns; returns (out, S), both float64
    (out_h, out_w), with S = sum |in*f| per output."""
    image = np.ascontiguousarray(image, dtype=np.float32)
    filt = np.ascontiguousarray(filt, dtype=np.float32)
    fh, fw = filt.shape
    assert image.shape[0] >= out_h + fh - 1 and image.shape[1] >= out_w + fw - 1
    out = np.empty((out_h, out_w), dtype=np.float64)
    S = np.empty((out_h, out_w), dtype=np.float64)
    if out_w > 0 and out_h > 0:
        _load().oracle_corr2d_f64(_ptr(image), image.shape[1], out_w, out_h, _ptr(filt), fw, fh,
                                  _ptr(out), _ptr(S), nthreads)
    return out, S


def corr2d_points(image: np.ndarray, filt: np.ndarray, xs, ys):
    """The same definition at the points (xs[k], ys[k]) only; returns (out, S)."""
    image = np.ascontiguousarray(image, dtype=np.float32)
    filt = np.ascontiguousarray(filt, dtype=np.float32)
    xs = np.ascontiguousarray(xs, dtype=np.int64)
    ys = np.ascontiguousarray(ys, dtype=np.int64)
    fh, fw = filt.shape
    out = np.empty(len(xs), dtype=np.float64)
    S = np.empty(len(xs), dtype=np.float64)
    _load().oracle_corr2d_f64_points(_ptr(image), image.shape[1], _ptr(filt), fw, fh,
                                     _ptr(xs), _ptr(ys), len(xs), _ptr(out), _ptr(S))
    return out, S


def corr2d_bf16_f64(image_bits: np.ndarray, filt_bits: np.ndarray, out_w: int, out_h: int,
                    nthreads: int = 0):
    """Valid cross-correlation of BF16-stored inputs (raw uint16 bit patterns),
    widened exactly and summed in FP64.  Returns (out, S)."""
    image_bits = np.ascontiguousarray(image_bits, dtype=np.uint16)
    filt_bits = np.ascontiguousarray(filt_bits, dtype=np.uint16)
    fh, fw = filt_bits.shape
    out = np.empty((out_h, out_w), dtype=np.float64)
    S = np.empty((out_h, out_w), dtype=np.float64)
    if out_w > 0 and out_h > 0:
        _load().oracle_corr2d_bf16_f64(_ptr(image_bits), image_bits.shape[1], out_w, out_h,
                                       _ptr(filt_bits), fw, fh, _ptr(out), _ptr(S), nthreads)
    return out, S
