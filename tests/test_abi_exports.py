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


def test_derived_outputs_match_the_oracle_without_gpu(lib):
    # epsilon_max and the design-layer fit are host code behind the C ABI
    import math

    import numpy as np

    import oracle as O
    import paper_2205_09900_gb300 as fp
    for F, k, n in [(3.0, 2, 2), (2.25, 2, 50), (1.5, 2, 50), (6.2, 3, 20), (30.0, 4, 12)]:
        a, b = fp.epsilon_max_log10(F, k, n), O.log10_epsilon_max(F, k, n)
        assert (math.isnan(a) and math.isnan(b)) or abs(a - b) <= 1e-12 * abs(b)
    rng = np.random.default_rng(4)
    for k in (1, 2, 3):
        for _ in range(20):
            depths = np.arange(2, 14)
            F = math.factorial(k) * (1 + np.exp(rng.normal(1.0, 1.0) - depths / rng.uniform(1, 4)
                                                + rng.normal(0, 0.3, size=len(depths))))
            got = fp.design_layers(depths, F, k, 50)
            ref = O.design_layers(depths, F, k, 50)
            for g, r in zip(got, ref):
                assert (math.isnan(g) and math.isnan(r)) or abs(g - r) <= 1e-9 * abs(r), (got, ref)
