"""Host check of the spiral program of the paper's hardware-efficient ansatz:
tests/cpp/spiral_plan_check.cpp, compiled against the library's planner,
applies the spiral maps in FP64 and compares with dense Tr(U^dagger V), and
emulates the register-window kernel's addressing (swizzled slots, lane bits,
the 2- and 4-CTA splits) against the map-by-map sweep.  CPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2205_09900_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    cuda_inc = "/usr/local/cuda/include"
    out = str(tmp_path_factory.mktemp("spiral") / "spiral_plan_check")
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I", CSRC, "-I", cuda_inc,
                           os.path.join(ROOT, "tests", "cpp", "spiral_plan_check.cpp"), os.path.join(CSRC, "planner.cpp"),
                           "-o", out])
    return out


@pytest.mark.parametrize("n,L", [(3, 2), (4, 2), (4, 3), (5, 3), (6, 2), (7, 3), (8, 4), (9, 3), (7, 5), (6, 6),
                                 (9, 5)])
def test_spiral_program_matches_dense_trace(checker, n, L):
    r = subprocess.run([checker, str(n), str(L)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr


@pytest.mark.parametrize("n,L", [(50, 6), (50, 7), (50, 8), (51, 8)])
def test_spiral_windows_full_size(checker, n, L):
    # the benchmark's sizes: 2^11..2^15 amplitudes, every window layout the GPU runs
    r = subprocess.run([checker, str(n), str(L), "nodense"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "split 1" in r.stdout and "split 2" in r.stdout
