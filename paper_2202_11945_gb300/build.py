"""Build the in-tree CUDA library ``libfewha.so`` for sm_103a.

Three translation units (the CUDA C-ABI with its kernels, the batched kernels, and the
host set-up code)
are compiled in parallel with nvcc and linked into one shared library next to
this file.  Run as ``python -m paper_2202_11945_gb300.build`` or via
``__graft_entry__.build()``.
"""

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfewha.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O3"]
SOURCES = ["fewha_api.cu", "fewha_batch.cu", "fewha_setup.cpp"]


def nvcc():
    exe = shutil.which("nvcc")
    if exe is None and os.path.exists("/usr/local/cuda/bin/nvcc"):
        exe = "/usr/local/cuda/bin/nvcc"
    if exe is None:
        raise RuntimeError("nvcc not found: the FEWHA CUDA library cannot be built")
    return exe


def _compile(src, extra):
    out = os.path.join(OBJ, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc()] + ARCH + COMMON + extra + ["-c", os.path.join(CSRC, src), "-o", out]
    if src.endswith(".cpp"):
        cmd = [nvcc()] + COMMON + extra + ["-x", "c++", "-c", os.path.join(CSRC, src), "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed on %s:\n%s\n%s" % (src, r.stdout, r.stderr))
    return out, r.stderr


def build(verbose=False, extra=(), nvtx=False):
    """Compile and link the library; nvtx=True adds NVTX ranges around the entry points."""
    os.makedirs(OBJ, exist_ok=True)
    extra = list(extra) + (["-DFEWHA_NVTX"] if nvtx else [])
    if verbose:
        extra = extra + ["-Xptxas", "-v"]
    with ThreadPoolExecutor(len(SOURCES)) as ex:
        results = list(ex.map(lambda s: _compile(s, extra), SOURCES))
    objs = [o for o, _ in results]
    tmp = LIB + ".tmp"
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"] + (["-ldl"] if nvtx else [])
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, nvtx="--nvtx" in sys.argv))
