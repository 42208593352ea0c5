"""Build the swedg CUDA library in-tree (sm_103a) with nvcc.

Each translation unit is compiled in parallel; the objects are linked into
paper_1804_02221_gb300/_lib/libswedg.so. Rebuilds only when a source is newer
than the library.
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libswedg.so")
SOURCES = ["capi.cu", "basis.cpp", "k_volume.cu", "k_volume_64.cu", "k_volume_256.cu", "k_volume_std.cu",
           "k_face.cu", "k_av.cu", "k_adjoint.cu", "noalloc.cu", "ensemble.cu"]
HEADERS = ["swe_internal.h", "kcommon.cuh", "k_volume.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the swedg CUDA library cannot be built")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS]
    deps.append(os.path.join(ROOT, "include", "swedg.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    tmpdir = os.path.join(OUT_DIR, f"obj{os.getpid()}")
    os.makedirs(tmpdir, exist_ok=True)
    cc = nvcc()
    common = ["-O3", "-std=c++17", "-lineinfo", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
              "-I", os.path.join(ROOT, "include")] + ARCH
    if verbose or os.environ.get("SWE_PTXAS_VERBOSE"):
        common += ["-Xptxas", "-v"]

    def compile_one(src):
        obj = os.path.join(tmpdir, os.path.splitext(src)[0] + ".o")
        cmd = [cc] + common + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        return obj, r.stderr

    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose or os.environ.get("SWE_PTXAS_VERBOSE"):
        for _, err in results:
            sys.stderr.write(err)
    tmp_lib = LIB + f".tmp{os.getpid()}"
    cmd = [cc, "-shared", "-o", tmp_lib] + [o for o, _ in results] + ARCH + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp_lib, LIB)
    shutil.rmtree(tmpdir, ignore_errors=True)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
