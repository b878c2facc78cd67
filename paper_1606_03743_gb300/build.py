"""Build libbem.so (the CUDA library behind include/bem.h) in-tree for sm_103a.

Every translation unit under csrc/ is compiled in parallel with nvcc and the
objects are linked into _build/libbem.so.  Rebuilds only when a source or
header is newer than the library.

The checked build (checked=True, into _build_checked/) compiles with
-DBEM_CHECKED=1: the kernels compare the global indices they write and the
near-pair records they read against the buffers' capacities, skip an access
that would fall outside, and the call that launched them returns an error
naming what was skipped.  It is a debugging build: the same results, slower.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libbem.so")
OUT_DIR_CHECKED = os.path.join(HERE, "_build_checked")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# The far-field kernel's FP32 values (squared distances >= ~1e-6, charges,
# sums) are nowhere near the FP32 denormal range, so it flushes denormals:
# rsqrtf then maps to the bare MUFU reciprocal square root.
PER_FILE_FLAGS = {"k_far.cu": ["-ftz=true"], "peaks.cu": ["-ftz=true"]}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libbem.so")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _inputs():
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(ROOT, "include", "*.h")) + [__file__]


def lib_path(checked: bool = False) -> str:
    return os.path.join(OUT_DIR_CHECKED if checked else OUT_DIR, "libbem.so")


def _stale(checked: bool = False) -> bool:
    lib = lib_path(checked)
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in _inputs())


def build(force: bool = False, verbose: bool = False, extra_flags=None, checked: bool = False) -> str:
    lib = lib_path(checked)
    if not force and not _stale(checked):
        return lib
    out_dir = os.path.dirname(lib)
    os.makedirs(out_dir, exist_ok=True)
    cc = nvcc()
    flags = ["-std=c++17", "-O3", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
             "-diag-suppress", "1444", "-Xcompiler", "-Wno-deprecated-declarations"]
    if checked:
        flags.append("-DBEM_CHECKED=1")
    if extra_flags:
        flags += list(extra_flags)
    objs = []

    def compile_one(src):
        obj = os.path.join(out_dir, os.path.basename(src)[:-3] + ".o")
        cmd = [cc, *flags, *PER_FILE_FLAGS.get(os.path.basename(src), []), "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = lib + f".{os.getpid()}.tmp"
    r = subprocess.run([cc, "-shared", *ARCH, "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, checked="--checked" in sys.argv))
