"""Compile libtraknn.so in-tree for sm_103a (nvcc, one -gencode, units in parallel).

build(bounds_check=True) compiles the debug variant libtraknn_bounds.so (its own
object folder): every guarded device-side index is checked against its buffer, and
a bad one is reported as TRAKNN_ERR_BOUNDS by traknn_sync_status instead of being
used."""
from __future__ import annotations

import concurrent.futures
import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(HERE, "libtraknn.so")
BOUNDS_LIB_PATH = os.path.join(HERE, "libtraknn_bounds.so")
ROOT = os.path.dirname(HERE)

NVCC = os.environ.get("NVCC", "nvcc")
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(
        os.path.join(CSRC, "*.cuh")) + [os.path.join(ROOT, "include", "traknn.h"), __file__]


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=None,
          bounds_check: bool = False) -> str:
    """Build (if stale) and return the path of libtraknn.so (or, with bounds_check,
    of the debug variant libtraknn_bounds.so)."""
    deps = _deps()
    lib_path = BOUNDS_LIB_PATH if bounds_check else LIB_PATH
    build_dir = BUILD_DIR + ("_bounds" if bounds_check else "")
    if not force and not _stale(lib_path, deps):
        return lib_path
    os.makedirs(build_dir, exist_ok=True)
    flags = NVCC_FLAGS + list(extra_flags or []) + (["-DTRAKNN_BOUNDS_CHECK"] if bounds_check
                                                     else [])
    headers = [d for d in deps if not d.endswith(".cu")]

    def compile_one(src):
        obj = os.path.join(build_dir, os.path.basename(src) + ".o")
        if force or _stale(obj, [src] + headers):
            cmd = [NVCC] + flags + ["-c", src, "-o", obj]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
            if verbose and (r.stdout or r.stderr):
                print(r.stdout, r.stderr)
        return obj

    with concurrent.futures.ThreadPoolExecutor(max_workers=8) as ex:
        objs = list(ex.map(compile_one, _sources()))
    tmp = lib_path + f".tmp{os.getpid()}"
    cmd = [NVCC, "-shared", "-o", tmp] + objs + ["-cudart=static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(verbose=True))
