"""Build the CUDA library ``_build/libkss.so`` for sm_103a with nvcc.

Eight translation units (the kernels for FP32, FP64 and FP16-deviation storage, and
the host runtimes of single lattices, batches, the adjoint, regridding and the
allocation-free entry point) compile in parallel and link into one shared library with the C ABI of ``include/kss.h``.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libkss.so")
SOURCES = ["launch_f32.cu", "launch_f64.cu", "launch_f16.cu", "kss_runtime.cu", "kss_batch.cu",
           "kss_adjoint.cu", "kss_regrid.cu", "kss_noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    cand = [os.environ.get("NVCC", ""), shutil.which("nvcc") or "", "/usr/local/cuda/bin/nvcc"]
    for c in cand:
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def cuda_lib_dir() -> str:
    root = os.path.dirname(os.path.dirname(os.path.realpath(nvcc())))
    for d in ("lib64", "lib", "targets/sbsa-linux/lib", "targets/x86_64-linux/lib"):
        p = os.path.join(root, d)
        if os.path.exists(os.path.join(p, "libcudart.so")):
            return p
    return os.path.join(root, "lib64")


def source_hash() -> str:
    """sha256 (first 16 hex digits) of the CUDA sources and the build flags from the
    environment: the autotuner's cache entries carry it, so an entry measured on other
    kernels is not reused."""
    h = hashlib.sha256()
    for name in sorted(os.listdir(CSRC)):
        path = os.path.join(CSRC, name)
        if os.path.isfile(path):
            h.update(name.encode() + b"\0")
            with open(path, "rb") as fh:
                h.update(fh.read())
    h.update(os.environ.get("KSS_NVCC_EXTRA", "").encode())
    return h.hexdigest()[:16]


def flags(extra=()) -> list[str]:
    # KSS_NVCC_EXTRA: additional nvcc flags (tuning macros such as -DKSS_STEP_MIN_BLOCKS=3)
    env = os.environ.get("KSS_NVCC_EXTRA", "").split()
    return ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2",
                   "-I", os.path.join(ROOT, "include"), f"-DKSS_SOURCE_HASH=\"{source_hash()}\"",
                   *env, *extra]


def build(verbose: bool = False, ptxas_info: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    extra = ["-Xptxas", "-v"] if ptxas_info else []

    def compile_one(src: str) -> str:
        obj = os.path.join(OUT_DIR, src.replace(".cu", ".o"))
        cmd = [nvcc(), *flags(extra), "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if ptxas_info:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    libdir = cuda_lib_dir()
    tmp = LIB + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
           "-L", libdir, f"-Xlinker=-rpath,{libdir}"]
    if verbose:
        print(" ".join(cmd), flush=True)
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True)
