"""Builds the in-tree CUDA library ``_qft_gb300.so`` for sm_103a (GB300).

Each translation unit under ``csrc/`` is compiled by nvcc in parallel
(``-gencode arch=compute_103a,code=sm_103a``) and linked into one shared
library next to this file.  The library exports the C ABI declared in
``include/qft_gb300.h``; nothing here needs a GPU.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD_DIR = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "_qft_gb300.so")
SOURCES = ["qft_api.cu", "qft_k_c2c_f32.cu", "qft_k_c2c_f16.cu", "qft_k_c2c_bf16.cu", "qft_k_real.cu", "qft_filter.cu",
           "qft_k_node.cu", "qft_k_ragged.cu", "qft_filter_bwd.cu", "qft_k_r2r.cu",
           "qft_static.cu", "qft_k_fixed.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -fmad=false: the transform never needs a fused multiply-add, and ptxas must not
# contract the packed f32x2 multiplies and adds (that would change the rounding).
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-fmad=false", "-Xcompiler", "-fPIC", "-Xptxas", "-v"]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA 13 toolkit is required to build the library")
    return exe


def _deps():
    return (glob.glob(os.path.join(CSRC, "*")) + [os.path.join(ROOT, "include", "qft_gb300.h"),
                                                   os.path.abspath(__file__)])


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _deps())


def _compile(src: str, defines=(), tag: str = "") -> tuple[str, str]:
    obj = os.path.join(BUILD_DIR, os.path.splitext(src)[0] + tag + ".o")
    cmd = [nvcc(), *ARCH, *FLAGS, *[f"-D{d}" for d in defines], "-c", os.path.join(CSRC, src), "-o", obj]
    p = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{p.stdout}")
    return obj, p.stdout


def build(force: bool = False, verbose: bool = False, defines=(), out: str | None = None) -> str:
    """Compile and link the library if any source changed; returns its path.
    `defines`/`out` build a variant (e.g. for a diagnostic) at another path."""
    target = out or LIB
    if not force and not defines and out is None and up_to_date():
        return LIB
    os.makedirs(BUILD_DIR, exist_ok=True)
    tag = "_" + "_".join(d.lower() for d in defines) if defines else ""
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(lambda s: _compile(s, defines, tag), SOURCES))
    with open(os.path.join(BUILD_DIR, "ptxas.log"), "w") as f:
        for (_, log) in results:
            f.write(log)
    tmp = target + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *[o for o, _ in results], "-lcudart"]
    p = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"link failed:\n{p.stdout}")
    os.replace(tmp, target)
    if verbose:
        for (_, log) in results:
            sys.stdout.write(log)
    return target


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
