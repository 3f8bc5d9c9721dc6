"""Host-only checks of the C-ABI library: it builds for sm_103a, loads without a GPU and
exports every entry point that include/abp.h declares (no compute calls)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "abp.h")


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(abp_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1104_2499_gb300 import build as B

    try:
        B.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    return B.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("abp_create", "abp_set_params", "abp_integrate", "abp_reduce", "abp_backward",
                     "abp_destroy", "abp_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    for n in declared_functions():
        assert n in exported, n
    # only the C ABI is exported from our own code (no C++ mangled kernels or helpers)
    ours = {s for s in exported if s.startswith("_ZN3abp")}
    assert not ours, sorted(ours)[:5]


def test_library_is_built_for_sm103a(libpath):
    from paper_1104_2499_gb300 import build as B

    assert "compute_103a" in B.ARCH and "sm_103a" in B.ARCH
    assert os.path.getsize(libpath) > 0


def test_version_and_null_handling(libpath):
    lib = ctypes.CDLL(libpath)
    lib.abp_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.abp_version()
    lib.abp_last_error.restype = ctypes.c_char_p
    lib.abp_last_error.argtypes = [ctypes.c_void_p]
    assert lib.abp_last_error(None)
    lib.abp_destroy.argtypes = [ctypes.c_void_p]
    lib.abp_destroy(None)  # allowed, no CUDA call
    lib.abp_create.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.abp_create(None, None, None) == 1  # ABP_EINVAL before any CUDA call


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1104_2499_gb300 import abp as A

    monkeypatch.setattr(A, "LIB_PATH", str(tmp_path / "missing" / "libabp.so"))
    monkeypatch.setattr(A, "_lib", None)
    with pytest.raises(RuntimeError, match="libabp.so not found"):
        A.lib()


def test_product_path_does_not_use_the_oracle():
    pkg = os.path.join(ROOT, "paper_1104_2499_gb300")
    pat = re.compile(r"^\s*(from\s+oracle|import\s+oracle|#include\s+.*oracle)|abp_oracle|or_run_set", re.M)
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not pat.search(txt), f
