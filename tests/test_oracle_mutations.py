"""Mistakes planted in a copy of the CPU oracle must each fail at least one pin.

Each mutation rewrites one expression of the oracle's C source (on the CPU,
in a temporary directory), builds it with gcc and runs every pin from
oracle_pins against it.  A mutation that no pin catches would mean the pins
do not constrain that part of the definition."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from tests import oracle_pins

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "corr2d_f64.c")
FULL_BODY = "double p = (double)row[j] * (double)f[i * fw + j];"

MUTATIONS = {
    "flip_x": (FULL_BODY, "double p = (double)row[j] * (double)f[i * fw + (fw - 1 - j)];"),
    "transpose": (FULL_BODY, "double p = (double)row[j] * (double)f[j * fh + i];"),
    "flip_y": (FULL_BODY, "double p = (double)row[j] * (double)f[(fh - 1 - i) * fw + j];"),
    "drop_last_column": ("for (int j = 0; j < fw; ++j) {\n                    double p = (double)row[j] * (double)f[i * fw + j];",
                         "for (int j = 0; j < fw - 1; ++j) {\n                    double p = (double)row[j] * (double)f[i * fw + j];"),
    "no_row_step": ("const float* row = in + (int64_t)(y + i) * in_pitch + x;",
                    "const float* row = in + (int64_t)y * in_pitch + x + i;"),
    "sign_first_tap": ("                    s += p;\n                    a += fabs(p);\n                }\n            }\n            out[(int64_t)y * out_w + x] = s;\n            if (S) S[(int64_t)y * out_w + x] = a;\n        }\n    }\n    (void)nthreads;\n}\n\n/* The same",
                       "                    s += (i == 0 && j == 0) ? -p : p;\n                    a += fabs(p);\n                }\n            }\n            out[(int64_t)y * out_w + x] = s;\n            if (S) S[(int64_t)y * out_w + x] = a;\n        }\n    }\n    (void)nthreads;\n}\n\n/* The same"),
    "signed_S": ("                    a += fabs(p);\n                }\n            }\n            out[(int64_t)y * out_w + x] = s;\n            if (S) S[(int64_t)y * out_w + x] = a;\n        }\n    }\n    (void)nthreads;\n}\n\n/* The same",
                 "                    a += p;\n                }\n            }\n            out[(int64_t)y * out_w + x] = s;\n            if (S) S[(int64_t)y * out_w + x] = a;\n        }\n    }\n    (void)nthreads;\n}\n\n/* The same"),
    "float_accumulator": ("            double s = 0.0, a = 0.0;\n            for (int i = 0; i < fh; ++i) {\n                const float* row = in + (int64_t)(y + i) * in_pitch + x;",
                          "            float s = 0.0f; double a = 0.0;\n            for (int i = 0; i < fh; ++i) {\n                const float* row = in + (int64_t)(y + i) * in_pitch + x;"),
}


def _build_mutant(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, name
    mutated = src.replace(old, new, 1)
    assert mutated != src
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(mutated)
    subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", str(c), "-o", str(so), "-lm"],
                   check=True, capture_output=True)
    lib = ctypes.CDLL(str(so))
    i64, i32, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
    lib.oracle_corr2d_f64.argtypes = [vp, i64, i32, i32, vp, i32, i32, vp, vp, i32]

    def corr(image, filt, out_w, out_h):
        image = np.ascontiguousarray(image, dtype=np.float32)
        filt = np.ascontiguousarray(filt, dtype=np.float32)
        fh, fw = filt.shape
        out = np.empty((out_h, out_w), np.float64)
        S = np.empty((out_h, out_w), np.float64)
        p = lambda a: a.ctypes.data_as(vp)
        lib.oracle_corr2d_f64(p(image), image.shape[1], out_w, out_h, p(filt), fw, fh, p(out), p(S), 1)
        return out, S
    return corr


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(tmp_path, name):
    old, new = MUTATIONS[name]
    corr = _build_mutant(tmp_path, name, old, new)
    caught = []
    for pin in oracle_pins.ALL_PINS:
        try:
            pin(corr)
        except AssertionError:
            caught.append(pin.__name__)
    assert caught, f"mutation {name} passed every pin"
