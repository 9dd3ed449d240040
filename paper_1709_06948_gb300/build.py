"""Build the library's CUDA C-ABI shared object in-tree (no torch extension machinery).

Every translation unit under csrc/ is compiled by nvcc for sm_103a only, in parallel,
then linked into _build/libmialign.so.  Host code is compiled with -ffp-contract=off.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libmialign.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
              "-Xcompiler", "-fno-fast-math", f"-I{INCLUDE}", f"-I{CSRC}", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    exe = shutil.which("nvcc")
    if exe:
        return exe
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found")


# eval.cu is compiled once per kernel shape (threads per CTA, points per thread per tile,
# resident CTAs per SM); see EvalKernels in csrc/align_internal.h.
EVAL_SHAPES = [("1024x1", 1024, 1, 1), ("1024x2", 1024, 2, 1), ("512x1", 512, 1, 2)]


def _units():
    """(source, object name, extra flags) for every translation unit."""
    units = []
    for f in sorted(os.listdir(CSRC)):
        if not f.endswith(".cu"):
            continue
        src = os.path.join(CSRC, f)
        if f == "eval.cu":
            for name, threads, ppt, ctas in EVAL_SHAPES:
                units.append((src, f"eval_{name}.o", [f"-DMI_EVAL_THREADS={threads}", f"-DMI_EVAL_PPT={ppt}",
                                                      f"-DMI_EVAL_CTAS_PER_SM={ctas}",
                                                      f"-DMI_EVAL_SHAPE_FN=eval_shape_{name}"]))
        else:
            units.append((src, f + ".o", []))
    return units


def _sources():
    return sorted({u[0] for u in _units()})


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    return max(os.path.getmtime(f) for f in files + [__file__])


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps():
        return LIB
    exe = nvcc()
    objs = []

    def compile_one(unit):
        src, obj_name, defs = unit
        obj = os.path.join(OUT_DIR, obj_name)
        cmd = [exe, *NVCC_FLAGS, *defs, *extra_flags, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        objs = list(ex.map(compile_one, _units()))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [exe, "-shared", *ARCH, "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose=True, extra_flags=sys.argv[1:]))
