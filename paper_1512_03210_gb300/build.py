"""Build the CUDA library libfse.so in-tree (sm_103a) with nvcc, one process per source file."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libfse.so")
# arithmetic-throughput probes used by the benchmark's roofline (not the solver)
PEAKS_SRC = "fse_peaks.cu"
PEAKS_LIB = os.path.join(OUT, "libfse_peaks.so")
INCLUDE = os.path.join(ROOT, "include")

SOURCES = ["fse_api.cu", "fse_precompute.cu", "fse_observables.cu", "fse_adjoint.cu",
           "fse_col_f32.cu", "fse_col_f64.cu", "fse_x_f32.cu", "fse_x_f64.cu", "fse_noalloc.cu",
           "fse_batch.cu", "fse_ground.cu"]
HEADERS = ["fse_fft.cuh", "fse_fft_x2.cuh", "fse_xpass_x2.cuh", "fse_passes.cuh", "fse_launch.cuh", "fse_internal.h"]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _stale(obj: str, deps: list) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, force: bool = False) -> str:
    """Compile every .cu in parallel and link libfse.so; returns its path."""
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INCLUDE, "fse.h")]
    procs, objs = [], []
    for src in SOURCES:
        path = os.path.join(CSRC, src)
        if not os.path.exists(path):
            continue
        obj = os.path.join(OUT, src.replace(".cu", ".o"))
        objs.append(obj)
        if force or _stale(obj, [path] + hdrs):
            cmd = [nvcc, *ARCH, *FLAGS, "-c", path, "-o", obj]
            if verbose:
                print(" ".join(cmd), flush=True)
            procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    peaks_src = os.path.join(CSRC, PEAKS_SRC)
    if force or _stale(PEAKS_LIB, [peaks_src]):
        cmd = [nvcc, *ARCH, *FLAGS, "-shared", "-cudart", "shared", peaks_src, "-o", PEAKS_LIB]
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((PEAKS_SRC, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((src, out.decode(errors="replace")))
        elif verbose and out:
            print(out.decode(errors="replace"))
    if failed:
        msg = "\n".join(f"--- {s}\n{o}" for s, o in failed)
        raise RuntimeError(f"nvcc failed:\n{msg}")
    if force or any(src != PEAKS_SRC for src, _ in procs) or not os.path.exists(LIB):
        cuda_lib = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "lib64")
        cmd = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", LIB, *objs,
               "-Xlinker", f"-rpath,{cuda_lib}"]
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.run(cmd, check=True)
    return LIB


if __name__ == "__main__":
    build(verbose="-v" in sys.argv, force="-f" in sys.argv)
    print(LIB)
