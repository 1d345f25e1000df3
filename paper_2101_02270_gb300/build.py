"""Build the in-tree shared library ``libnrpf.so`` (CUDA for sm_103a + host C++).

Each translation unit is compiled in parallel by nvcc, then linked with the
static CUDA runtime.  Usage: ``python paper_2101_02270_gb300/build.py`` (run as a script: importing the
package itself needs the built library).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libnrpf.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["api.cu", "kernels.cu", "dense_im.cu", "mlp.cu", "multi.cu", "noalloc.cu", "peak.cu", "flows.cu", "plan.cpp",
           "ordering.cpp", "retry.cpp",
           "cpu_batch.cpp"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _compile(src: str, nvcc: str, extra: list[str]) -> str:
    obj = os.path.join(BUILD, os.path.basename(src) + ".o")
    # host code at -O3: the batched host solver relies on the compiler's
    # vectoriser for its loops over instance lanes (no target-specific flags)
    host_opt = "-O3" if src.endswith(".cpp") else "-O2"
    cmd = [nvcc, "-c", os.path.join(CSRC, src), "-o", obj, "-O3", "-std=c++17", "-lineinfo",
           "-Xcompiler", "-fPIC", "-Xcompiler", host_opt, *ARCH, *extra]
    subprocess.run(cmd, check=True)
    return obj


def build(verbose: bool = False, extra: list[str] | None = None) -> str:
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    extra = list(extra or [])
    if verbose:
        extra += ["-Xptxas", "-v"]
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, nvcc, extra), SOURCES))
    tmp = LIB + ".tmp"
    subprocess.run([nvcc, "-shared", "-o", tmp, *objs, *ARCH, "-cudart", "static"], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
