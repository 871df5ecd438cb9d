"""Build libmxm.so in-tree with nvcc for sm_103a (GB300).

Each ``csrc/*.cu`` file is compiled to an object in parallel, then linked
into ``paper_1211_1581_gb300/_build/libmxm.so`` against the shared CUDA
runtime.  Rebuilds only when a source or header is newer than the library.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libmxm.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    cand = [os.environ.get("NVCC", ""), shutil.which("nvcc") or "",
            "/usr/local/cuda/bin/nvcc"]
    for c in cand:
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: libmxm.so cannot be built")


def _cuda_lib_dir(nvcc: str) -> str:
    root = os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    for sub in ("lib64", "lib", "targets/sbsa-linux/lib", "targets/x86_64-linux/lib"):
        d = os.path.join(root, sub)
        if os.path.exists(os.path.join(d, "libcudart.so")):
            return d
    return os.path.join(root, "lib64")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _inputs():
    return (sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
            + glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)])


# The bounds-checked build (-DMXM_DEBUG_BOUNDS): the kernels check their tile
# coordinates, copy sources and tensor-memory columns and record a violation
# as MXM_ERR_INVALID_ARG in the device status word (never a trap).
LIB_DEBUG = os.path.join(BUILD, "libmxm_debug.so")
FLAVORS = {LIB: [], LIB_DEBUG: ["-DMXM_DEBUG_BOUNDS"]}


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _inputs())


def build(force: bool = False, verbose: bool = False, extra_flags=None, debug: bool = True) -> str:
    """Compile every CUDA source and link libmxm.so (and, with debug, the
    bounds-checked libmxm_debug.so, compiled in the same pool of parallel
    nvcc processes); returns the path of libmxm.so."""
    libs = [LIB] + ([LIB_DEBUG] if debug else [])
    todo = [lib for lib in libs if force or not up_to_date(lib)]
    if not todo:
        return LIB
    nvcc = _nvcc()
    srcs = sources()
    jobs = []
    for lib in todo:
        odir = os.path.join(BUILD, "debug") if lib == LIB_DEBUG else BUILD
        os.makedirs(odir, exist_ok=True)
        flags = (NVCC_FLAGS + ARCH + ["-I", CSRC, "-I", INCLUDE] + FLAVORS[lib] +
                 list(extra_flags or []))
        for src in srcs:
            jobs.append((lib, src, os.path.join(odir, os.path.basename(src)[:-3] + ".o"), flags))

    def compile_one(job):
        lib, src, obj, flags = job
        cmd = [nvcc, "-c", src, "-o", obj] + flags
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return lib, obj

    # the slowest translation units first, so that they start at once
    jobs.sort(key=lambda j: -os.path.getsize(j[1]))
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        done = list(ex.map(compile_one, jobs))
    libdir = _cuda_lib_dir(nvcc)
    for lib in todo:
        objs = [o for (l, o) in done if l == lib]
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc, "-shared", "-o", tmp] + objs + ARCH + [
            "-cudart", "shared", "-L", libdir, "-Xlinker", "-rpath," + libdir]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link of {os.path.basename(lib)} failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":  # pragma: no cover
    import sys
    print(build(force="--force" in sys.argv, verbose=True,
                extra_flags=["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else None))
