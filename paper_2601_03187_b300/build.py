"""Build libtang.so (the C-ABI library) in-tree with nvcc for sm_103a.

Objects go to _build/ at the repository root; the shared library is written next to this file.
Usage: python -m paper_2601_03187_b300.build [--force] [--checked]
--checked builds libtang_checked.so (objects in _build/checked/) with TANG_CHECKED: every table
index the search code forms is tested before the access (see tang_checked_build in tang.h).
"""
import concurrent.futures as cf
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libtang.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")
SOURCES = ["api.cu", "tss_host.cpp", "search.cu", "mlp_simt.cu", "trainer.cu", "tc_model.cu", "mlp_tc256.cu",
           "serve.cpp", "noalloc.cu", "tune.cu", "update.cpp", "hybrid.cpp",
           "selftest.cu"]
HEADERS = ["internal.h", "search_dev.cuh", "tc_ptx.cuh", "tc_common.cuh"]


LIB_CHECKED = os.path.join(PKG, "libtang_checked.so")


def _flags(checked=False):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O3", "-I", INCLUDE, "-I", CSRC] + (
        ["-DTANG_CHECKED"] if checked else [])


def _deps_mtime():
    files = [os.path.join(INCLUDE, "tang.h")] + [os.path.join(CSRC, h) for h in HEADERS]
    return max(os.path.getmtime(f) for f in files if os.path.exists(f))


def _compile(src, force, verbose, checked=False):
    s = os.path.join(CSRC, src)
    o = os.path.join(BUILD, "checked" if checked else "", src + ".o")
    if not force and os.path.exists(o) and os.path.getmtime(o) >= max(os.path.getmtime(s), _deps_mtime()):
        return o, ""
    cmd = [NVCC] + _flags(checked) + (["-Xptxas", "-v"] if verbose else []) + ["-c", s, "-o", o]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
    return o, r.stderr


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    os.makedirs(os.path.join(BUILD, "checked") if checked else BUILD, exist_ok=True)
    lib = LIB_CHECKED if checked else LIB
    with cf.ThreadPoolExecutor(max_workers=min(8, len(SOURCES))) as ex:
        results = list(ex.map(lambda s: _compile(s, force, verbose, checked), SOURCES))
    objs = [o for o, _ in results]
    if verbose:
        for (o, log), s in zip(results, SOURCES):
            if log:
                print("== %s\n%s" % (s, log))
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < max(os.path.getmtime(o) for o in objs):
        tmp = lib + ".tmp%d" % os.getpid()
        cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs + ["-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
