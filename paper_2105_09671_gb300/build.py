"""Build the CUDA library ``_build/libac.so`` for sm_103a with nvcc.

Each ``csrc/*.cu`` translation unit compiles in parallel to an object file;
the objects link into one shared library (CUDA runtime linked statically).
The library is rebuilt only when a source or header is newer than it.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libac.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# Kernels use C++20 (templated lambdas for the unrolled streaming loops).
# ac_batch.cu, ac_net.cu and ac_slab.cu are host-only C++ that needs nothing newer than
# C++17, and nvcc 13.0's front end aborts on them in C++20 mode (an internal
# assertion when destroying std::vector elements of the C-linkage descriptor
# types), so they are compiled as C++17.
STD_OVERRIDE = {"ac_batch.cu": "-std=c++17", "ac_net.cu": "-std=c++17", "ac_slab.cu": "-std=c++17"}
# Sources compiled several times with different defines, one object each
# (the 3D stencil per tile shape: its kernel instantiations then compile in
# parallel processes).
_S3_TILES = 3
VARIANTS = {f"k_stream3d_{t}.cu": [f"-DAC_S3_TILE={i}" for i in range(_S3_TILES)]
            for t in ("f64", "f32", "f16")}
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++20", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-O2", "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libac.so")


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps() -> list[str]:
    return (sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
            + glob.glob(os.path.join(INCLUDE, "*.h")))


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in _deps())


def _units() -> list[tuple[str, str, list[str]]]:
    """(source, object, extra defines) of every compilation."""
    out = []
    for src in sources():
        base = os.path.basename(src)[:-3]
        defs = VARIANTS.get(os.path.basename(src))
        if defs is None:
            out.append((src, os.path.join(OUT_DIR, base + ".o"), []))
        else:
            for i, d in enumerate(defs):
                out.append((src, os.path.join(OUT_DIR, f"{base}_v{i}.o"), [d]))
    return out


def _compile(nvcc: str, unit: tuple[str, str, list[str]], verbose_ptxas: bool) -> str:
    src, obj, defs = unit
    flags = [STD_OVERRIDE.get(os.path.basename(src), f) if f.startswith("-std=") else f
             for f in NVCC_FLAGS]
    cmd = [nvcc, *ARCH, *flags, *defs, "-c", src, "-o", obj]
    if verbose_ptxas:
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stderr}")
    if verbose_ptxas:
        sys.stderr.write(r.stderr)
    return obj


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    """Compile every CUDA source and link libac.so; returns its path."""
    if not force and not verbose_ptxas and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    units = _units()
    # longest compilations first (the stencil kernels), so they start at once
    units.sort(key=lambda u: ("stream" not in u[0] and "batch" not in u[0] and "net" not in u[0], u[1]))
    with cf.ThreadPoolExecutor(max_workers=min(len(units), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda u: _compile(nvcc, u, verbose_ptxas), units))
    tmp = LIB + f".tmp{os.getpid()}"
    r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
