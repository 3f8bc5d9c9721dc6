"""Build libabp.so (sm_103a) in-tree with nvcc.

Each translation unit of ``csrc/`` is compiled in parallel for
``-gencode arch=compute_103a,code=sm_103a`` and linked into
``paper_1104_2499_gb300/_build/libabp.so``; the library exports only the C ABI of
``include/abp.h``.
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
OUT = os.path.join(PKG, "_build")
LIB = os.path.join(OUT, "libabp.so")
SOURCES = ["abp_api.cu", "abp_kernels.cu", "abp_adjoint.cu", "abp_noalloc.cu"]
HEADERS = ["abp_device.cuh", "abp_internal.cuh", "abp_ctx.cuh"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libabp.so")


def _flags():
    # host code: no contraction into fused multiply-adds, so the moments formed on the host
    # (abp_combine_moments) round as the device's explicitly rounded ones
    return [ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fvisibility=hidden,-ffp-contract=off",
            "-I", INCLUDE, "-I", CSRC, "--expt-relaxed-constexpr"]


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(INCLUDE, "abp.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra: list | None = None, out_dir: str | None = None) -> str:
    """Compile the library; ``out_dir`` (default ``_build/``) receives the objects and
    ``libabp.so``.  The checked build is ``extra=["-DABP_DEBUG_CHECKS=1"]`` into its own
    directory (``python -m paper_1104_2499_gb300.build --checked``)."""
    out = out_dir or OUT
    lib = os.path.join(out, "libabp.so")
    if not force and not _stale(lib):
        return lib
    os.makedirs(out, exist_ok=True)
    cc = nvcc()
    flags = _flags() + list(extra or [])

    def compile_one(src):
        obj = os.path.join(out, src.replace(".cu", ".o"))
        cmd = [cc] + flags + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + ".tmp.%d" % os.getpid()
    cmd = [cc, ARCH, "-shared", "-o", tmp] + objs + ["-lcudart_static", "-lrt", "-ldl", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, lib)
    return lib


CHECKED_OUT = os.path.join(PKG, "_build_checked")

if __name__ == "__main__":
    force = "--force" in sys.argv
    extra = ["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else []
    if "--checked" in sys.argv:
        print(build(force=force, verbose=True, extra=extra + ["-DABP_DEBUG_CHECKS=1"], out_dir=CHECKED_OUT))
    else:
        print(build(force=force, verbose=True, extra=extra or None))
