"""Build the CUDA library (libbem_gb300.so) in-tree for sm_103a.

Each translation unit under csrc/ is compiled by nvcc in parallel, then linked into one shared
library with the CUDA runtime linked statically (no dependency on a particular libcudart on the
loader path).  Run: python -m paper_1511_04355_gb300.build
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libbem_gb300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
          "-Xcompiler", "-Wall", "-Wno-deprecated-gpu-targets"]


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found (CUDA toolkit required to build the library)")
    return exe


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC)
                  if f.endswith(".cu") or f.endswith(".cpp"))


# Per-file host flags: the H-matrix cluster tree compares coordinates and distances, and must
# round every product and sum separately on every host architecture (no fused multiply-add).
FILE_FLAGS = {"hmatrix_tree.cpp": ["-Xcompiler", "-ffp-contract=off"]}


def _compile(src, obj, extra):
    cmd = [nvcc(), *ARCH, *CFLAGS, *FILE_FLAGS.get(os.path.basename(src), []), *extra, "-c", src, "-o", obj]
    p = subprocess.run(cmd, capture_output=True, text=True)
    return src, p.returncode, p.stdout + p.stderr


def build(verbose: bool = False, extra=()) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    objs = []
    jobs = []
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        for src in sources():
            obj = os.path.join(OUT_DIR, os.path.basename(src) + ".o")
            objs.append(obj)
            jobs.append(ex.submit(_compile, src, obj, list(extra)))
        for j in jobs:
            src, rc, log = j.result()
            if rc != 0:
                raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{log}")
            if verbose and log.strip():
                print(log)
    tmp = LIB + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"link failed:\n{p.stdout}{p.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
