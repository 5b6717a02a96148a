"""In-tree build of libconvtune.so (host runtime + AOT helper kernels for sm_103a).

The correlation variants themselves are compiled at run time by NVRTC from
csrc/corr2d.cuh, which is embedded into the library as a string.

    python -m paper_2407_11488_gb300.build      # or build() from Python
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(BUILD, "libconvtune.so")

CPP = ["common.cpp", "variant.cpp", "tune.cpp", "capi.cpp", "batch.cpp", "serve.cpp", "analyze.cpp",
       "clocks.cpp"]
CU = ["aux_kernels.cu", "noalloc.cu"]
HEADERS = ["ct_internal.hpp", "batch_internal.hpp", "corr2d.cuh", "batch.cuh"]
GENCODE = "-gencode=arch=compute_103a,code=sm_103a"


def cuda_home() -> str:
    env = os.environ.get("CUDA_HOME") or os.environ.get("CUDA_PATH")
    if env and os.path.isdir(env):
        return env
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    return "/usr/local/cuda"


def _sources():
    srcs = [os.path.join(CSRC, f) for f in CPP + CU + HEADERS if os.path.exists(os.path.join(CSRC, f))]
    return srcs + [os.path.join(INCLUDE, "convtune.h"), os.path.abspath(__file__)]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources())


def _embed(src: str, dst: str, delim: str = "CTSRC") -> None:
    text = open(src).read()
    assert f"){delim}\"" not in text
    body = f'R"{delim}({text}){delim}"\n'
    if not os.path.exists(dst) or open(dst).read() != body:
        with open(dst, "w") as fh:
            fh.write(body)


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r


def build(force: bool = False, verbose: bool = False) -> str:
    """Builds libconvtune.so in-tree; returns its path.  Fails loudly."""
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    _embed(os.path.join(CSRC, "corr2d.cuh"), os.path.join(BUILD, "corr2d_src.inc"))
    if os.path.exists(os.path.join(CSRC, "batch.cuh")):
        _embed(os.path.join(CSRC, "batch.cuh"), os.path.join(BUILD, "batch_src.inc"), "CTBAT")
    home = cuda_home()
    inc = ["-I" + INCLUDE, "-I" + CSRC, "-I" + BUILD, "-I" + os.path.join(home, "include")]
    jobs = []
    for f in CPP:
        src = os.path.join(CSRC, f)
        if not os.path.exists(src):
            continue
        obj = os.path.join(BUILD, f + ".o")
        jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-fvisibility=hidden", "-Wall", "-Wno-unused-function",
                     *inc, "-c", src, "-o", obj])
    for f in CU:
        src = os.path.join(CSRC, f)
        obj = os.path.join(BUILD, f + ".o")
        jobs.append([os.path.join(home, "bin", "nvcc"), GENCODE, "-lineinfo", "-O3", "-std=c++17",
                     "-Xcompiler", "-fPIC,-fvisibility=hidden", *inc, "-c", src, "-o", obj])
    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        for r in ex.map(_run, jobs):
            if verbose:
                sys.stdout.write(r.stdout + r.stderr)
    objs = [j[-1] for j in jobs]
    tmp = LIB + f".tmp{os.getpid()}"
    lib64 = os.path.join(home, "lib64")
    if not os.path.isdir(lib64):
        lib64 = os.path.join(home, "lib")
    _run([os.path.join(home, "bin", "nvcc"), GENCODE, "-shared", "-o", tmp, *objs,
          "-cudart", "shared", "-L" + lib64, "-lnvrtc", "-lpthread", "-ldl", "-lrt",
          "-Xlinker", "--exclude-libs,ALL", "-Xlinker", "-rpath," + lib64])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
