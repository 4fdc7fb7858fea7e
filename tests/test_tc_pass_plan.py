"""Host check of the tensor-core tile pass of the brickwork sweep:
tests/cpp/tc_pass_check.cpp, compiled against the library's brick planner,
emulates the kernel's data movement in FP64 (window-0 gather tables, dense
window matrices in the MMA's B layout, the MMA read through the hardware's
view of the swizzled K-major operands, the XOR-table scatter into the next
window's operand or the boundary) and compares it with the gate-by-gate
sweep of the same windows.  Every operand address is bounds-checked and every
window layout checked to be a bijection.  The "tcm" mode emulates the
tensor-memory operand form instead: every window's input through the
shared-memory exchange buffer, with every exchange checked to be a bijection
and every half-warp's 16 stores and loads to hit 16 distinct bank pairs.  CPU."""
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
    out = str(tmp_path_factory.mktemp("tc") / "tc_pass_check")
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                           "-I", "/usr/local/cuda/include", os.path.join(ROOT, "tests", "cpp", "tc_pass_check.cpp"),
                           os.path.join(CSRC, "brick_plan.cpp"), "-o", out])
    return out


@pytest.mark.parametrize("mode", ["smem", "tcm"])
@pytest.mark.parametrize("n,l", [(20, 8), (50, 8), (50, 9), (51, 9), (50, 10)])
def test_tc_pass_emulation_matches_gate_sweep(checker, n, l, mode):
    r = subprocess.run([checker, str(n), str(l), mode], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
