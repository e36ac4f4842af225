"""Builds the CUDA library ``liblbm_gb300.so`` in-tree for sm_103a (GB300).

Five translation units compile in parallel and link into one shared library
with the C ABI of ``include/lbm.h``:

* ``lbm_fp32.cu``: FP32 kernels (fast path, FMA contraction allowed);
* ``lbm_fp64.cu``: FP64 kernels with ``-fmad=false`` (debug path, rounds like
  the FP64 CPU oracle);
* ``lbm_fp16.cu``: 16-bit (FP16, BF16) population storage, FP32 arithmetic;
* ``lbm_api.cu``: the C ABI, host code built with ``-ffp-contract=off``;
* ``lbm_noalloc.cu``: the allocation-free front-height entry point.

Run ``python -m paper_2303_02210_gb300.build`` or call ``build()``.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "liblbm_gb300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
UNITS = {
    "lbm_fp32": [],
    "lbm_fp64": ["-fmad=false"],
    "lbm_fp16": [],
    "lbm_api": [],
    "lbm_noalloc": [],
}


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _sources():
    out = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    out.append(os.path.join(os.path.dirname(HERE), "include", "lbm.h"))
    return out


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
                     "-I", os.path.join(os.path.dirname(HERE), "include")]
    procs = []
    objs = []
    for unit, extra in UNITS.items():
        obj = os.path.join(BUILD, unit + ".o")
        cmd = [nvcc] + common + extra + ["-c", os.path.join(CSRC, unit + ".cu"), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((cmd, out.decode(errors="replace")))
        elif verbose and out:
            print(out.decode(errors="replace"))
    if failed:
        msg = "\n".join(" ".join(c) + "\n" + o for c, o in failed)
        raise RuntimeError("nvcc failed:\n" + msg)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
