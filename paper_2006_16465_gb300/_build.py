"""Build libhj.so (the C-ABI library) in-tree with nvcc for sm_103a.

Every .cu under csrc/ is one translation unit; they compile in parallel and
link into paper_2006_16465_gb300/libhj.so with the CUDA runtime linked
statically, so the library needs nothing but the driver at run time.

build(debug=True) makes libhj_debug.so instead (objects in _build_debug/):
the same sources compiled with -DHJ_DEBUG, whose kernels check their indices
and whose device allocations carry guard bands (hj_debug_check).  The
binding loads it when the environment variable HJ_LIBRARY is "debug".
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
BUILD = PKG / "_build"
LIB = PKG / "libhj.so"
BUILD_DEBUG = PKG / "_build_debug"
LIB_DEBUG = PKG / "libhj_debug.so"
HEADERS = [ROOT / "include" / "hj.h"] + sorted(CSRC.glob("*.cuh"))

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-fvisibility=hidden",
                  "-I", str(ROOT / "include")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and Path(cand).exists():
            return cand
    raise RuntimeError("nvcc not found")


def _stale(target: Path, deps) -> bool:
    if not target.exists():
        return True
    t = target.stat().st_mtime
    return any(Path(d).stat().st_mtime > t for d in deps)


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> Path:
    srcs = sorted(CSRC.glob("*.cu"))
    bdir, lib = (BUILD_DEBUG, LIB_DEBUG) if debug else (BUILD, LIB)
    flags = NVFLAGS + (["-DHJ_DEBUG"] if debug else [])
    bdir.mkdir(exist_ok=True)
    cc = nvcc()
    jobs = []
    for s in srcs:
        o = bdir / (s.stem + ".o")
        if force or _stale(o, [s] + HEADERS):
            jobs.append((s, o))

    def compile_one(so):
        s, o = so
        cmd = [cc] + flags + ["-c", str(s), "-o", str(o)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {s.name}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            print(r.stdout + r.stderr)
        return o

    if jobs:
        with ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            list(ex.map(compile_one, jobs))
    objs = [bdir / (s.stem + ".o") for s in srcs]
    if force or jobs or _stale(lib, objs):
        tmp = str(lib) + ".tmp"
        cmd = [cc] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + [str(o) for o in objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose=False))
