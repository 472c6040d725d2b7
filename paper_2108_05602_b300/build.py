"""Build libvolks.so in-tree with nvcc for sm_103a (B300).

Each CUDA source is compiled to an object in parallel, then linked into
one shared library.  The benchmark's measurement helper (the FP32 FMA
probe) is linked into a library of its own, libvolks_bench.so, which only
the benchmark loads.

    python -m paper_2108_05602_b300.build [--verbose-ptxas]
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libvolks.so")
OBJ = os.path.join(HERE, "_build")
SOURCES = ["volks_kernels.cu", "volks_mma.cu", "volks_api.cu", "volks_plan.cu", "volks_server.cu",
           "volks_noalloc.cu", "volks_calib.cu", "volks_loc.cpp",
           "volks_search_mixed0.cu", "volks_search_mixed4.cu", "volks_refit.cu",
           "volks_search_slide0.cu", "volks_search_slide4.cu"]
BENCH_SOURCES = ["bench_probe.cu"]
BENCH_LIB = os.path.join(HERE, "libvolks_bench.so")
HEADERS = ["fft_regs.cuh", "twiddle_ce.h", "search_common.cuh", "search_kernel.cuh", "tcgen05.cuh", "volks_internal.h",
           "volks_job.h", "volks_result.h", os.path.join("..", "..", "include", "volks.h"),
           os.path.join("..", "..", "include", "volks_check.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found")
    return p


def needs_build() -> bool:
    if not (os.path.exists(LIB) and os.path.exists(BENCH_LIB)):
        return True
    t = min(os.path.getmtime(LIB), os.path.getmtime(BENCH_LIB))
    deps = [os.path.join(CSRC, s) for s in SOURCES + BENCH_SOURCES + HEADERS] + [__file__]
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src: str, verbose_ptxas: bool) -> tuple[str, str]:
    obj = os.path.join(OBJ, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc_path(), "-std=c++17", "-O3", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC",
           "--expt-relaxed-constexpr", "-I", os.path.join(HERE, "..", "include"), "-c",
           os.path.join(CSRC, src), "-o", obj]
    if verbose_ptxas:
        cmd += ["-Xptxas", "-v"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n" + res.stdout + res.stderr)
    return obj, res.stdout + res.stderr


def build(verbose_ptxas: bool = False, force: bool = False) -> str:
    if not force and not needs_build():
        return LIB
    os.makedirs(OBJ, exist_ok=True)
    with ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 1)) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose_ptxas), SOURCES + BENCH_SOURCES))
    if verbose_ptxas:
        for _, log in results:
            sys.stderr.write(log)
    objs = {os.path.basename(o): o for o, _ in results}
    for lib, srcs in ((LIB, SOURCES), (BENCH_LIB, BENCH_SOURCES)):
        cmd = [nvcc_path(), *ARCH, "-shared", "-o", lib + ".tmp"] + \
              [objs[os.path.splitext(s)[0] + ".o"] for s in srcs]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("nvcc link failed:\n" + res.stdout + res.stderr)
        os.replace(lib + ".tmp", lib)
    return LIB


if __name__ == "__main__":
    build(verbose_ptxas="--verbose-ptxas" in sys.argv, force=True)
    print(LIB)
