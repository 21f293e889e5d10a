"""Build libfastcod.so in-tree: one nvcc per translation unit (in parallel),
then a shared-library link.  sm_103a only.  build(checked=True) builds the
bounds-checked variant (FASTCOD_CHECKED=1: every computed index of the
path's gathers, scatters and list writes is tested, a failure reported as an
error) as libfastcod_checked.so beside it."""
from __future__ import annotations

import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(CSRC, "_build")
OBJ_CHECKED = os.path.join(CSRC, "_build_checked")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libfastcod.so")
LIB_CHECKED = os.path.join(LIBDIR, "libfastcod_checked.so")
INCLUDE = os.path.join(ROOT, "include")

SOURCES = ["fastcod_capi.cu", "batch.cu", "server.cu", "noalloc.cu", "aux_capi.cu", "k_volume.cu", "k_prefilter.cu",
           "k_walk.cu", "k_aux.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler",
                     "-fvisibility=hidden", f"-I{INCLUDE}"]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _deps():
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    return hdrs + [os.path.join(INCLUDE, "fastcod.h")]


def build(force: bool = False, ptxas_verbose: bool = False, checked: bool = False) -> str:
    obj_dir, lib = (OBJ_CHECKED, LIB_CHECKED) if checked else (OBJ, LIB)
    flags = NVCC_FLAGS + (["-DFASTCOD_CHECKED=1"] if checked else [])
    os.makedirs(obj_dir, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    dep_time = max(os.path.getmtime(d) for d in _deps())
    nvcc = _nvcc()

    def obj_of(src):
        return os.path.join(obj_dir, src.replace(".cu", ".o"))

    def compile_one(src):
        s = os.path.join(CSRC, src)
        o = obj_of(src)
        if not force and os.path.exists(o) and os.path.getmtime(o) >= max(os.path.getmtime(s), dep_time):
            return ""
        cmd = [nvcc] + flags + (["-Xptxas", "-v"] if ptxas_verbose else []) + ["-c", s, "-o", o]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        return r.stderr

    with ThreadPoolExecutor(len(SOURCES)) as ex:
        logs = list(ex.map(compile_one, SOURCES))
    objs = [obj_of(s) for s in SOURCES]
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < max(os.path.getmtime(o) for o in objs):
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.check_call([nvcc] + ARCH + ["-shared", "-o", tmp] + objs)
        os.replace(tmp, lib)
    if ptxas_verbose:
        print("".join(logs))
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, ptxas_verbose="-v" in sys.argv, checked="--checked" in sys.argv))
