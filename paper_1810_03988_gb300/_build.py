"""In-tree build of libstitch.so for sm_103a (nvcc, one -gencode, translation units in parallel)."""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libstitch.so")
# the debug build: guard bands around every rig allocation and index checks in the fused kernels
DEBUG_LIB = os.path.join(BUILD, "libstitch_debug.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
              "--expt-relaxed-constexpr", f"-I{INCLUDE}", f"-I{CSRC}"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libstitch")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(INCLUDE, "stitch.h"), __file__]


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every csrc/*.cu for sm_103a and link libstitch.so (release) and libstitch_debug.so
    (STITCH_DEBUG) in _build/, all translation units of both in parallel."""
    todo = [(lib, flags) for lib, flags in ((LIB, []), (DEBUG_LIB, ["-DSTITCH_DEBUG"]))
            if force or not up_to_date(lib)]
    if not todo:
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    exe = nvcc()
    srcs = _sources()

    def compile_one(job):
        src, lib, flags = job
        sub = "debug" if flags else "release"
        os.makedirs(os.path.join(BUILD, sub), exist_ok=True)
        obj = os.path.join(BUILD, sub, os.path.basename(src)[:-3] + ".o")
        cmd = [exe, *ARCH, *NVCC_FLAGS, *flags, "-c", src, "-o", obj]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)} ({sub}):\n{res.stderr}")
        if verbose and res.stderr:
            print(res.stderr)
        return lib, obj

    jobs = [(src, lib, flags) for lib, flags in todo for src in srcs]
    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        done = list(ex.map(compile_one, jobs))
    for lib, _ in todo:
        objs = [o for l, o in done if l == lib]
        tmp = f"{lib}.{os.getpid()}.tmp"
        cmd = [exe, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-ldl", "-lpthread"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"link of {os.path.basename(lib)} failed:\n{res.stderr}")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
