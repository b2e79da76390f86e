"""Build libtdq.so (the CUDA library) in-tree for sm_103a.

Each translation unit under csrc/ is compiled by nvcc in parallel, then linked
into one shared library next to this file.  No PyTorch headers or libraries
are involved: the library's interface is the plain C ABI of include/tdq.h.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libtdq.so")
BUILD_DIR = os.path.join(PKG, "_build")
# The debug variant: every index computation of the search kernels checked
# against its bounds (-DTDQ_DEBUG; a failed check is reported, never a
# trap).  Built on request, for the tests.
LIB_DEBUG = os.path.join(PKG, "libtdq_debug.so")
BUILD_DIR_DEBUG = os.path.join(PKG, "_build_debug")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtdq")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _stale(target, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=(), debug: bool = False) -> str:
    """Build libtdq.so (debug=True: libtdq_debug.so, the bounds-checked
    variant) if it is missing or older than its sources; returns its path."""
    lib_path = LIB_DEBUG if debug else LIB
    build_dir = BUILD_DIR_DEBUG if debug else BUILD_DIR
    srcs = sources()
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(INCLUDE, "tdq.h"))
    if not force and not _stale(lib_path, srcs + headers + [__file__]):
        return lib_path
    os.makedirs(build_dir, exist_ok=True)
    cc = nvcc()
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-pthread", "-I",
                     INCLUDE, "-I", CSRC, "--expt-relaxed-constexpr"] + list(extra_flags)
    if debug:
        common.append("-DTDQ_DEBUG")
    if verbose:
        common += ["-Xptxas", "-v"]

    def compile_one(src):
        obj = os.path.join(build_dir, os.path.basename(src) + ".o")
        cmd = [cc, "-c", src, "-o", obj] + common
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        outs = list(ex.map(compile_one, srcs))
    if verbose:
        for _, err in outs:
            sys.stderr.write(err)
    tmp = lib_path + ".tmp%d" % os.getpid()
    cmd = [cc, "-shared", "-o", tmp] + [o for o, _ in outs] + ARCH + ["-lcudart", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug="--debug" in sys.argv))
