"""Builds the CUDA library libstdg.so in-tree (paper_1802_04516_gb300/_lib/).

nvcc compiles every translation unit of csrc/ for sm_103a in parallel, then links a
shared library against the shared CUDA runtime.  No CMake.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT, "libstdg.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"), "-I", SRC]


def nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def sources():
    return sorted(f for f in os.listdir(SRC) if f.endswith((".cu", ".cpp")))


def _compile(src, verbose):
    obj = os.path.join(OUT, src + ".o")
    cmd = [nvcc(), *ARCH, *FLAGS, "-c", os.path.join(SRC, src), "-o", obj]
    if src.endswith(".cpp"):
        cmd = [nvcc(), *FLAGS, "-x", "c++", "-c", os.path.join(SRC, src), "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
    return obj, r.stderr


def build(verbose=False, force=False):
    os.makedirs(OUT, exist_ok=True)
    srcs = sources()
    newest = max(os.path.getmtime(os.path.join(SRC, f)) for f in os.listdir(SRC))
    newest = max(newest, os.path.getmtime(os.path.join(ROOT, "include", "stdg.h")), os.path.getmtime(__file__))
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose), srcs))
    for _, log in results:
        if verbose and log:
            sys.stderr.write(log)
    cmd = [nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", LIB + ".tmp", *[o for o, _ in results]]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    t = __import__("time").time()
    print(build(verbose="-v" in sys.argv, force=True), "%.1fs" % (__import__("time").time() - t))
