"""Build libcmcs.so in-tree for sm_103a with nvcc (no cmake, no torch extension machinery).

Each translation unit is compiled in parallel to an object file, then linked into
``paper_2310_00420_gb300/_build/libcmcs.so``.  Objects are rebuilt when their source or any
header is newer.  Run ``python -m paper_2310_00420_gb300.build`` or call ``build()``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libcmcs.so")
SOURCES = ["cmcs_api.cu", "kernels_op.cu", "kernels_cg.cu", "kernels_estep.cu", "kernels_tc.cu",
           "kernels_ozaki.cu", "noalloc.cu", "adjoint.cu", "kernels_dft.cu", "kernels_dft_large.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _headers_mtime() -> float:
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    paths.append(os.path.join(ROOT, "include", "cmcs.h"))
    return max(os.path.getmtime(p) for p in paths)


def _compile(nvcc: str, src: str, extra) -> str:
    obj = os.path.join(OUT, src.replace(".cu", ".o"))
    s = os.path.join(CSRC, src)
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(s), _headers_mtime()):
        return obj
    cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", s, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if r.stderr.strip():
        sys.stderr.write(r.stderr)
    return obj


def build(verbose_ptxas: bool = False, force: bool = False) -> str:
    """Compile and link libcmcs.so; returns its path."""
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    if force:
        for f in os.listdir(OUT):
            os.remove(os.path.join(OUT, f))
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(nvcc, s, extra), SOURCES))
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        cmd = [nvcc, *ARCH, "-shared", "-o", LIB, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    return LIB


if __name__ == "__main__":
    print(build(verbose_ptxas="-v" in sys.argv, force="-f" in sys.argv))
