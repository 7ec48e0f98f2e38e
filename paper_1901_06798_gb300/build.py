"""Build the CUDA library in-tree for sm_103a (GB300).

``python -m paper_1901_06798_gb300.build`` compiles ``csrc/`` into
``_build/libtsunami.so``.  Translation units compile in parallel:

* ``step_f64.cu``, ``step_unsplit_f64.cu`` and ``amr_kernels.cu`` with
  ``--fmad=false`` so the FP64
  kernels round every product and sum separately, exactly like the FP64
  reference arithmetic;
* ``step_f32p.cu`` and ``step_unsplit_f32p.cu`` with contraction and CUDA's fast FP32 divide/sqrt allowed
  (the FP32 perturbation form, held to 1e-4 m of surface elevation);
* the host runtime (``tsu_api.cpp``, ``cluster.cpp``) with the host compiler, without
  contraction (its geometry tables round like the oracle's).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libtsunami.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


UNITS = [
    ("step_f64.cu", ["--fmad=false"]),
    ("step_f32p.cu", ["--fmad=true", "--use_fast_math"]),
    ("step_unsplit_f64.cu", ["--fmad=false"]),
    ("step_unsplit_f32p.cu", ["--fmad=true", "--use_fast_math"]),
    ("amr_kernels.cu", ["--fmad=false"]),
    ("tsu_api.cpp", []),
    ("cluster.cpp", []),
    ("noalloc.cu", []),
    ("cnn.cu", []),
    ("cnn_api.cpp", []),
]


def _sources():
    out = []
    for d in (CSRC, os.path.join(HERE, "..", "include")):
        for f in os.listdir(d):
            out.append(os.path.join(d, f))
    return out


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    if not force and os.path.exists(LIB):
        mt = os.path.getmtime(LIB)
        if all(os.path.getmtime(s) <= mt for s in _sources()):
            return LIB
    nvcc = _nvcc()

    def compile_one(unit):
        src, extra = unit
        obj = os.path.join(OUT, src.rsplit(".", 1)[0] + ".o")
        if src.endswith(".cu"):
            cmd = [nvcc, *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", *extra,
                   "-c", os.path.join(CSRC, src), "-o", obj]
        else:
            cmd = [nvcc, "-x", "c++", "-O2", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off", "-c",
                   os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"compiling {src} failed:\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stdout.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(compile_one, UNITS))
    tmp = LIB + ".tmp"
    r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart", "-lpthread"], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"linking failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
