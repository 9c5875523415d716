"""Build libsdme.so in-tree: nvcc for the sm_103a translation units, g++ for
the host basis builder, compiled in parallel and linked with static cudart.

    python -m paper_2104_13466_gb300.build [--force]
"""
import concurrent.futures
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libsdme.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE]
GXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-I" + INCLUDE]

CU_SOURCES = ["api.cu", "noalloc.cu", "batch.cu", "batch_persist.cu"] + ["elem_p%d.cu" % p for p in range(1, 9)]
CPP_SOURCES = ["basis1d.cpp"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _headers_mtime():
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    paths.append(os.path.join(INCLUDE, "sdme.h"))
    return max(os.path.getmtime(p) for p in paths)


def _compile(src, force, hdr_mtime):
    obj = os.path.join(BUILD, src + ".o")
    path = os.path.join(CSRC, src)
    if not force and os.path.exists(obj):
        if os.path.getmtime(obj) >= max(os.path.getmtime(path), hdr_mtime):
            return obj, None
    if src.endswith(".cu"):
        cmd = [_nvcc()] + NVCC_FLAGS + ["-c", path, "-o", obj]
    else:
        cmd = ["g++"] + GXX_FLAGS + ["-c", path, "-o", obj]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        return obj, "%s\n%s\n%s" % (" ".join(cmd), res.stdout, res.stderr)
    return obj, None


def build(force=False, jobs=None, verbose=True):
    """Compile and link libsdme.so; returns its path.  Raises on failure."""
    os.makedirs(BUILD, exist_ok=True)
    hdr = _headers_mtime()
    srcs = CU_SOURCES + CPP_SOURCES
    jobs = jobs or min(len(srcs), max(2, os.cpu_count() or 2))
    with concurrent.futures.ThreadPoolExecutor(jobs) as ex:
        results = list(ex.map(lambda s: _compile(s, force, hdr), srcs))
    errors = [e for _, e in results if e]
    if errors:
        raise RuntimeError("libsdme build failed:\n" + "\n".join(errors))
    objs = [o for o, _ in results]
    newest = max(os.path.getmtime(o) for o in objs)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < newest:
        cmd = [_nvcc()] + ARCH + ["-shared", "-o", LIB] + objs + ["-cudart", "static"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("libsdme link failed:\n%s\n%s\n%s" % (" ".join(cmd), res.stdout, res.stderr))
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv)
