"""Build libbf (the CUDA library behind include/bf.h) in-tree with nvcc.

Each .cu file under csrc/ is compiled for sm_103a in parallel, then linked
into ``_build/libbf.so`` against the shared CUDA runtime.  Nothing is
installed outside the package directory.
"""
from __future__ import annotations

import glob
import hashlib
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libbf.so")
CHECKED_LIB = os.path.join(BUILD, "checked", "libbf_checked.so")  # BF_DEVICE_CHECKS: kernels check their indices
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps_hash(src: str, extra_flags=()) -> str:
    h = hashlib.sha1()
    for p in [src] + sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))):
        with open(p, "rb") as f:
            h.update(f.read())
    h.update(" ".join(ARCH + NVCC_FLAGS + list(extra_flags)).encode())
    return h.hexdigest()[:16]


def build(verbose: bool = False, jobs: int | None = None, extra_flags=(), lib_path: str = LIB) -> str:
    """Compile every csrc/*.cu for sm_103a and link the library at `lib_path`
    (libbf.so by default; objects go beside it); returns its path."""
    bdir = os.path.dirname(lib_path)
    os.makedirs(bdir, exist_ok=True)
    nvcc = _nvcc()
    srcs = _sources()
    objs = []

    def compile_one(src):
        base = os.path.splitext(os.path.basename(src))[0]
        obj = os.path.join(bdir, f"{base}.{_deps_hash(src, extra_flags)}.o")
        if not os.path.exists(obj):
            tmp = obj + f".tmp{os.getpid()}"
            cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra_flags, "-c", src, "-o", tmp]
            if verbose:
                print(" ".join(cmd), flush=True)
            subprocess.run(cmd, check=True)
            os.replace(tmp, obj)
        return obj

    with ThreadPoolExecutor(max_workers=jobs or min(8, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, srcs))
    stamp = hashlib.sha1("".join(objs).encode()).hexdigest()[:16]
    stamp_file = lib_path + ".stamp"
    if not (os.path.exists(lib_path) and os.path.exists(stamp_file) and open(stamp_file).read() == stamp):
        tmp = lib_path + f".tmp{os.getpid()}"
        cmd = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs]
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.run(cmd, check=True)
        os.replace(tmp, lib_path)
        with open(stamp_file, "w") as f:
            f.write(stamp)
    # drop stale objects
    keep = set(objs)
    for o in glob.glob(os.path.join(bdir, "*.o")):
        if o not in keep:
            try:
                os.remove(o)
            except OSError:
                pass
    return lib_path


def build_checked(verbose: bool = False) -> str:
    """The checked build: every kernel index check compiled in (BF_DEVICE_CHECKS);
    a failed check records BF_ERR_BOUNDS in the status word and skips the access."""
    return build(verbose=verbose, extra_flags=("-DBF_DEVICE_CHECKS",), lib_path=CHECKED_LIB)


if __name__ == "__main__":
    print(build(verbose=True))
