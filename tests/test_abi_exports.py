"""The C-ABI library builds for sm_103a and exports every function that
include/*.h declares.  No compute call is made (no GPU is needed)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(fp_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2205_09900_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_api():
    names = declared_functions()
    for required in ("fp_ensemble_create", "fp_trace_batch", "fp_frame_potential", "fp_ensemble_destroy",
                     "fp_last_error", "fp_export_gates", "fp_reduce_moments"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    import paper_2205_09900_gb300 as fp
    assert sorted(fp.EXPORTED) == declared_functions()


def test_last_error_without_gpu(lib):
    lib.fp_last_error.restype = ctypes.c_char_p
    assert isinstance(lib.fp_last_error(), bytes)


def test_gemm_argument_checks_without_gpu(lib):
    # shape and alignment checks run before any CUDA call
    f = lib.fp_gemm_bf16
    vp, i32 = ctypes.c_void_p, ctypes.c_int32
    f.argtypes = [i32, i32, i32, vp, i32, vp, i32, vp, i32, vp, vp, vp, vp, vp]
    f.restype = ctypes.c_int
    lib.fp_last_error.restype = ctypes.c_char_p
    fake = vp(1 << 20)   # never dereferenced: every call below fails its checks
    assert f(4, 24, 64, fake, 64, fake, 64, None, 0, None, fake, None, None, None) == -1   # N % 16
    assert b"N % 16" in lib.fp_last_error()
    assert f(4, 16, 60, fake, 64, fake, 64, None, 0, None, fake, None, None, None) == -1   # K % 8
    assert f(4, 16, 64, fake, 64, fake, 64, None, 2, None, fake, None, None, None) == -1   # mode 2 needs Z
    assert f(4, 16, 64, vp((1 << 20) + 8), 64, fake, 64, None, 0, None, fake, None, None, None) == -1  # alignment
    assert f(4, 16, 64, fake, 64, fake, 64, None, 0, None, None, None, None, None) == -1   # no output
