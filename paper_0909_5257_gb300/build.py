"""Build libmea.so (CUDA path + generator) in-tree for sm_103a with nvcc.

Each translation unit is compiled in parallel with
``nvcc -gencode arch=compute_103a,code=sm_103a -O3 -lineinfo`` and linked into
``paper_0909_5257_gb300/libmea.so``.  The library is rebuilt when a source is
newer than it.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libmea.so")
BUILD_DIR = os.path.join(ROOT, "_build")
SOURCES = ["generator.cpp", "helshare.cpp", "amp_kernel.cu", "amp_hs_kernel.cu", "ps_kernel.cu", "api.cu", "colour_gemm.cu", "jamp_gemm.cu", "batch.cu",
           "server.cu", "peak.cu"]
HEADERS = ["generator.h", "helshare.h", "kernels.h", "colour_gemm.h", "jamp_gemm.h", "tc_common.cuh", "process.h", "heget.cuh", "amp_common.cuh", "gen_kernel.cuh", "codegen.cpp",
           "../phasespace/phasespace.h", "../../include/mea.h"]
# Processes whose straight-line kernels are emitted at build time (live state
# small enough for registers); every other process runs on the interpreter.
GENERATED = ["21,21,21,21", "2,-2,21,21", "2,2,2,2", "21,21,21,21,21", "2,-2,21,21,21", "2,2,2,2,21"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    for f in SOURCES + HEADERS:
        if os.path.getmtime(os.path.join(CSRC, f)) > t:
            return True
    return os.path.getmtime(__file__) > t


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD_DIR, exist_ok=True)
    cc = nvcc()
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fopenmp,-O3",
                     "-I", os.path.join(ROOT, "include")]

    def compile_one(src):
        obj = os.path.join(BUILD_DIR, src + ".o")
        cmd = [cc] + common + ["-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cpp"):
            cmd = [cc] + common + ["-x", "cu", "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    # 1. emit the straight-line per-process kernels with the generator
    tool = os.path.join(BUILD_DIR, "mea_codegen")
    r = subprocess.run(["g++", "-O2", "-std=c++17", "-fopenmp", "-o", tool, os.path.join(CSRC, "codegen.cpp"),
                        os.path.join(CSRC, "generator.cpp")], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"codegen tool build failed:\n{r.stderr}")
    gen_dir = os.path.join(BUILD_DIR, "generated")
    os.makedirs(gen_dir, exist_ok=True)
    for f in os.listdir(gen_dir):
        os.remove(os.path.join(gen_dir, f))
    r = subprocess.run([tool, gen_dir] + GENERATED, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"codegen failed:\n{r.stderr}")
    gen_sources = sorted(os.listdir(gen_dir))

    def compile_generated(name):
        # one translation unit (one device module) per kernel variant, plus the table
        obj = os.path.join(BUILD_DIR, name + ".o")
        cmd = [cc] + common + ["-I", CSRC, "-c", os.path.join(gen_dir, name), "-o", obj]
        rr = subprocess.run(cmd, capture_output=True, text=True)
        if rr.returncode != 0:
            raise RuntimeError(f"nvcc failed on {name}:\n{rr.stdout}\n{rr.stderr}")
        return obj

    # 2. compile everything in parallel
    jobs = [(compile_one, s) for s in SOURCES] + [(compile_generated, g) for g in gen_sources]
    with cf.ThreadPoolExecutor(max_workers=max(4, min(len(jobs), os.cpu_count() or 4))) as ex:
        objs = list(ex.map(lambda j: j[0](j[1]), jobs))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-Xcompiler", "-fopenmp", "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
