"""In-tree build of the native parts: the CUDA library (sm_103a) and the input generator.

``build_cuda()`` compiles every ``csrc/*.cu`` translation unit in parallel with
``nvcc -gencode arch=compute_103a,code=sm_103a -lineinfo -O3`` and links ``libglu.so`` next to
this file (cudart linked statically, so the library needs only the driver at run time).
``build_synth()`` compiles ``inputs/synth.c`` into ``inputs/libglu_synth.so`` with gcc/OpenMP.
Outputs are git-ignored; object files go to ``_build/``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB_PATH = os.path.join(HERE, "libglu.so")
SYNTH_SRC = os.path.join(HERE, "inputs", "synth.c")
SYNTH_LIB = os.path.join(HERE, "inputs", "libglu_synth.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def _stale(out: str, inputs) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(i) > t for i in inputs)


def build_synth(force: bool = False) -> str:
    if force or _stale(SYNTH_LIB, [SYNTH_SRC]):
        _run(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-Wall",
              "-o", SYNTH_LIB, SYNTH_SRC, "-lm"])
    return SYNTH_LIB


def build_cuda(force: bool = False, verbose_ptxas: bool = False, extra_flags=None) -> str:
    nvcc = _nvcc()
    os.makedirs(OBJ, exist_ok=True)
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    headers = sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
                     + glob.glob(os.path.join(INCLUDE, "*.h")))
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
                    "-I", CSRC, "--expt-relaxed-constexpr", "-Xcompiler", "-ffp-contract=off"]
    if verbose_ptxas:
        flags += ["-Xptxas", "-v"]
    if extra_flags:
        flags += list(extra_flags)
    jobs = []
    objs = []
    for src in sources:
        obj = os.path.join(OBJ, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        if force or verbose_ptxas or _stale(obj, [src] + headers):
            jobs.append([nvcc] + flags + ["-c", src, "-o", obj])
    logs = []
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            logs = list(ex.map(_run, jobs))
    if force or jobs or _stale(LIB_PATH, objs):
        _run([nvcc] + ARCH + ["-shared", "-cudart", "static", "-o", LIB_PATH] + objs)
    if verbose_ptxas:
        return "\n".join(logs)
    return LIB_PATH


def build_all(force: bool = False) -> None:
    build_synth(force=force)
    build_cuda(force=force)


if __name__ == "__main__":
    import sys
    if "--ptxas" in sys.argv:
        print(build_cuda(verbose_ptxas=True))
    else:
        build_all(force="--force" in sys.argv)
        print(LIB_PATH)
