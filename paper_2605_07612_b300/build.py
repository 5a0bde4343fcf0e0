"""Builds the CUDA library libamr_b300.so in-tree (paper_2605_07612_b300/_build).

nvcc compiles every translation unit for sm_103a only (B300); the host C++
parts go through nvcc as well so the library links as one shared object.
Run `python -m paper_2605_07612_b300.build` or call `build()`.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libamr_b300.so")
UNITS = ["amr_api.cu", "forest.cpp", "pattern.cpp", "noalloc.cu", "mlp.cu", "inst_ghost.cu", "inst_stage_f32_2d.cu",
         "inst_stage_f32_3d.cu", "inst_stage_f64_2d.cu", "inst_stage_f64_3d.cu", "inst_stage_pair.cu", "inst_stage_pair2d.cu",
         "inst_stage_pair_hll.cu", "inst_stage_pair2d_hll.cu",
         "inst_stage_f32_2d_gen.cu", "inst_stage_f32_3d_gen.cu", "inst_stage_f64_2d_gen.cu", "inst_stage_f64_3d_gen.cu",
         "inst_weno.cu", "inst_stage_adv.cu"]
HEADERS = ["common.cuh", "ghost.cuh", "stage.cuh", "stage_pair.cuh", "misc.cuh", "mlp.cuh", "mlp_tc.cuh", "forest.hpp", "pattern.hpp",
           "api_internal.cuh", "launch_kernels.cuh", "stage_weno.cuh", "stage_pair2d.cuh", "stage_adv.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


def _flags(unit: str):
    f = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC,-O3", "-lineinfo", "--expt-relaxed-constexpr"]
    if unit.endswith(".cu"):
        f += ARCH + ["-Xptxas", "-v"] if os.environ.get("AMR_PTXAS_VERBOSE") else ARCH
    else:
        f += ["-x", "cu"] + ARCH
    return f


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    include = os.path.join(os.path.dirname(HERE), "include")
    hdrs = [os.path.join(SRC, h) for h in HEADERS] + [os.path.join(include, "amr.h")]
    objs = []
    jobs = []
    for u in UNITS:
        src = os.path.join(SRC, u)
        obj = os.path.join(OUT_DIR, u + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + hdrs):
            cmd = [NVCC] + _flags(u) + ["-I", SRC, "-I", include, "-c", src, "-o", obj]
            jobs.append(cmd)
    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)
    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        list(ex.map(run, jobs))
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + ".%d.tmp" % os.getpid()
        cmd = [NVCC, "-shared"] + ARCH + ["-o", tmp] + objs + ["-lcudart"]
        run(cmd)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
