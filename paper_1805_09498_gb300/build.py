"""Build libffca.so in-tree for sm_103a with nvcc (no cmake, parallel TUs).

    python -m paper_1805_09498_gb300.build [--force] [--verbose]

The kernel instantiations are split over one translation unit per (method,
precision, I) so that they compile in parallel.
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
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libffca.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]

I_VALUES = (1, 2, 3, 4, 8)


def _nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libffca.so")
    return exe


def _units():
    """(source, object, extra flags) for every translation unit."""
    units = [("ffca_api.cu", "ffca_api.o", []), ("ffca_fca_api.cu", "ffca_fca_api.o", []),
             ("ffca_stft.cu", "ffca_stft.o", []), ("ffca_probe.cu", "ffca_probe.o", []),
             ("ffca_mask.cu", "ffca_mask.o", [])]
    for part in (0, 1, 2, 3, 4):  # FastFCA-AS, conventional FCA, adjoint, normal EM, Newton
        for prec in (0, 1):
            for i in I_VALUES:
                units.append(("ffca_inst.cu", f"ffca_inst_k{part}_p{prec}_i{i}.o",
                              [f"-DFFCA_PART={part}", f"-DFFCA_PREC={prec}", f"-DFFCA_I={i}"]))
    return units


def _sources():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "ffca.h")]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources())


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile every translation unit and link libffca.so; returns its path."""
    if not force and not _stale():
        return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    extra = ["-Xptxas", "-v"] if ptxas_info else []

    def compile_one(u):
        src, obj, defs = u
        cmd = [nvcc, *ARCH, *FLAGS, *extra, *defs, "-c", os.path.join(CSRC, src),
               "-o", os.path.join(BUILD, obj)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {obj}:\n{r.stderr}")
        return obj, r.stderr

    jobs = min(len(_units()), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(jobs) as ex:
        results = list(ex.map(compile_one, _units()))
    if verbose or ptxas_info:
        for obj, err in results:
            if err.strip():
                print(f"== {obj}\n{err}", file=sys.stderr)
    tmp = LIB + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp] + [os.path.join(BUILD, o) for _, o, _ in _units()]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="--verbose" in sys.argv,
          ptxas_info="--ptxas" in sys.argv)
    print(LIB)
