"""The Python binding's ctypes mirrors have the layout of the C structs in
include/convtune.h: for every mirrored struct, a small C program compiled
against the header prints its size and each field's offset, and they must
equal the ctypes Structure's.  A field added on one side only (or out of
order) fails here, on the CPU, before any call passes a misread struct."""
import ctypes
import os
import shutil
import subprocess
import tempfile

import pytest

import paper_2407_11488_gb300 as ct

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MIRRORS = {
    "ct_problem": ct.Problem,
    "ct_config": ct.Config,
    "ct_variant_info": ct.VariantInfo,
    "ct_device_info": ct.DeviceInfo,
    "ct_tune_opts": ct.TuneOpts,
    "ct_row": ct.Row,
    "ct_table_info": ct.TableInfo,
    "ct_analysis": ct.Analysis,
    "ct_batch_item": ct.BatchItem,
    "ct_bucket_config": ct.BucketConfig,
    "ct_batch_opts": ct.BatchOpts,
    "ct_batch_info": ct.BatchInfo,
    "ct_server_opts": ct.ServerOpts,
    "ct_request": ct.Request,
    "ct_server_stats": ct.ServerStats,
    "ct_server_run_opts": ct.ServerRunOpts,
}


def _c_layouts():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "convtune.h"', "int main(void) {"]
    for cname, py in MIRRORS.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'    printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["    return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        with open(src, "w") as fh:
            fh.write("\n".join(lines) + "\n")
        subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    res = {}
    for line in out.splitlines():
        cname, what, v = line.split()
        res[(cname, what)] = int(v)
    return res


def test_ctypes_mirrors_match_the_header():
    c = _c_layouts()
    for cname, py in MIRRORS.items():
        assert ctypes.sizeof(py) == c[(cname, "size")], cname
        for fname, _ in py._fields_:
            assert getattr(py, fname).offset == c[(cname, fname)], (cname, fname)
