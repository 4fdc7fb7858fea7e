"""The library called from C through include/fp.h alone (tests/cpp/c_driver.c,
compiled and linked against libfp_gb300.so here, no ctypes): the host-side
calls on CPU, and one FP64 trace batch on the GPU against the oracle."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2205_09900_gb300")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_2205_09900_gb300 import build
    build.build()
    out = str(tmp_path_factory.mktemp("cdrv") / "c_driver")
    subprocess.check_call([cc, "-O1", "-std=c99", "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "cpp", "c_driver.c"), "-L", PKG, "-lfp_gb300",
                           f"-Wl,-rpath,{PKG}", "-lm", "-o", out])
    return out


def test_c_driver_host_calls(driver):
    r = subprocess.run([driver], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and "host ok" in r.stdout, r.stdout + r.stderr


@pytest.mark.gpu
def test_c_driver_traces_match_oracle(driver):
    r = subprocess.run([driver, "trace"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    lines = r.stdout.strip().splitlines()
    got = np.array([complex(float(a), float(b)) for a, b in (l.split() for l in lines[:16])])
    ref = O.trace_batch(O.desc(O.PARALLEL, 8, 4, seed=1), 0, 16, "dense")
    assert np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1.0)) <= 1e-10
    f = lines[16].split()
    assert f[0] == "F" and abs(float(f[1]) - 1.0) < 0.2     # F^(1) = 1 (1-design), 4096 pairs
