"""Build liblbm.so (CUDA, sm_103a) in-tree: paper_2009_04604_gb300/_build/liblbm.so.

Each translation unit compiles in its own nvcc process, in parallel; the objects
are linked with ``nvcc -shared`` (static CUDA runtime). No cmake. The fused step
kernel, step_inst.cu, is compiled once per (lattice, storage type), since its
instantiations dominate the build time.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liblbm.so")
# the bounds-checked build (LBM_DEBUG): every population index of the kernels is
# checked, and the first one out of range is reported by lbm_synchronize
DEBUG_BUILD = os.path.join(HERE, "_build_debug")
DEBUG_LIB = os.path.join(DEBUG_BUILD, "liblbm.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# Multiply-add fusion happens in the front end only (explicit fma.rn in the PTX):
# ptxas would otherwise fuse the remaining multiply/add pairs depending on each
# kernel's register budget, and the same per-node code would round differently
# in different kernels (a batched simulation against the same one stepped alone,
# one launch variant against another).
COMMON = ARCH + ["-O3", "-lineinfo", "-std=c++20", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
                 "-Xptxas", "--fmad=false", "-I", INCLUDE]
# per-file extra flags: the geometry kernels round like the plain FP64 definitions
EXTRA = {"geometry.cu": ["-fmad=false"]}
# step_inst.cu: one object per (lattice, storage type)
STEP_INSTANCES = [(lat, sto) for lat in ("D2Q9", "D3Q19", "D3Q27") for sto in ("double", "float", "__half", "__nv_bfloat16")]


def _nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbm")
    return cand


def _sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))


def _deps():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "lbm.h")]


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compile liblbm.so (debug: the bounds-checked build in _build_debug/)."""
    out_dir, lib = (DEBUG_BUILD, DEBUG_LIB) if debug else (BUILD, LIB)
    extra = ["-DLBM_DEBUG"] if debug else []
    if not force and up_to_date(lib):
        return lib
    os.makedirs(out_dir, exist_ok=True)
    nvcc = _nvcc()
    srcs = _sources()

    jobs = []
    for src in srcs:
        if src == "step_inst.cu":
            for lat, sto in STEP_INSTANCES:
                jobs.append((src, [f"-DLBM_STEP_LATTICE={lat}", f"-DLBM_STEP_STORE={sto}"],
                             f"step_{lat}_{sto.strip('_')}.o"))
        else:
            jobs.append((src, EXTRA.get(src, []), src.replace(".cu", ".o")))
    # the slowest units first, so that they overlap with the rest
    jobs.sort(key=lambda j: j[0] != "step_inst.cu")

    def compile_one(job):
        src, flags, name = job
        obj = os.path.join(out_dir, name)
        cmd = [nvcc] + COMMON + extra + flags + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src} {' '.join(flags)}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(os.cpu_count() or 8, len(jobs))) as ex:
        objs = list(ex.map(compile_one, jobs))
    tmp = lib + f".tmp{os.getpid()}"
    r = subprocess.run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, debug="--debug" in sys.argv))
