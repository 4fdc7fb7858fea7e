"""Monte Carlo contraction of qudit brickwork circuits (local dimension q = 3,
Haar U(9) gates) on the GPU: traces against the oracle's q-ary dense and
elimination contractions, Tr(U^dagger U) = q^n, one gate's k!, and F^(2) at
n = 50 against the exact qutrit value of the Weingarten transfer matrix."""
import math

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_09900_gb300 import build
    build.build()
    import paper_2205_09900_gb300 as fpm
    fpm.load()
    return fpm


def rel(a, b):
    return np.abs(a - b) / np.maximum(np.abs(b), 1.0)


@pytest.mark.parametrize("n,l,method", [(2, 2, "dense"), (3, 2, "dense"), (4, 3, "dense"), (5, 4, "dense"),
                                        (6, 3, "dense"), (7, 2, "ve"), (50, 2, "ve"), (50, 3, "ve"), (51, 4, "ve")])
def test_qudit_traces_match_oracle(fp, n, l, method):
    ens = fp.Ensemble(fp.PARALLEL, n, l, l, seed=41, q=3)
    N = 6 if n >= 50 else 10
    t64, _, _ = ens.trace_batch(0, N, fp.PREC_FP64)
    t32, _, _ = ens.trace_batch(0, N, fp.PREC_FP32_RAW)
    ref = np.array([O.trace_qudit(3, n, l, 41, p, method) for p in range(N)])
    assert rel(t64, ref).max() <= 1e-10, rel(t64, ref)
    assert np.abs(t32 - ref).max() <= 1e-4


def test_qudit_mixed_depths_and_global_state(fp):
    # depths 2..6 in one call (l = 6: 3^10 amplitudes per side, kept in global memory)
    ens = fp.Ensemble(fp.PARALLEL, 6, 2, 6, seed=43, q=3)
    t, _, g = ens.trace_batch(0, 40, fp.PREC_FP64)
    d = O.desc(O.PARALLEL, 6, 2, 6, seed=43)
    ls = [O.pair_depth(d, p) for p in range(40)]
    assert sorted(set(ls)) == [2, 3, 4, 5, 6] and np.array_equal(g, np.array(ls) - 2)
    ref = np.array([O.trace_qudit(3, 6, l, 43, p, "dense") for p, l in enumerate(ls)])
    assert rel(t, ref).max() <= 1e-10


def test_qudit_self_pair_is_dimension(fp):
    for l in (4, 6):
        ens = fp.Ensemble(fp.PARALLEL, 50, l, l, seed=44, q=3, flags=fp.FLAG_SELF_PAIR)
        t, _, _ = ens.trace_batch(0, 4, fp.PREC_FP64)
        assert np.all(np.abs(t / 3.0 ** 50 - 1) < 1e-10)


def test_qudit_single_gate_is_haar(fp):
    # n = 2: one Haar U(9) gate per circuit pair at any depth: F^(k) = k! for k <= 9
    ens = fp.Ensemble(fp.PARALLEL, 2, 2, 2, seed=45, q=3)
    F, se, st = ens.frame_potential(0, 400_000, 3, 0.0, fp.PREC_FP64)
    for k in (1, 2, 3):
        assert abs(F[0, k - 1] - math.factorial(k)) < 5 * se[0, k - 1], (k, F[0, k - 1], se[0, k - 1])


@pytest.mark.parametrize("l,pairs", [(4, 200_000), (5, 100_000), (6, 30_000)])
def test_qudit_frame_potential_matches_exact(fp, l, pairs):
    ens = fp.Ensemble(fp.PARALLEL, 50, l, l, seed=46, q=3)
    F, se, st = ens.frame_potential(0, pairs, 2, 0.0, fp.PREC_FP32)
    exact = fp.exact_brickwork_fk(50, l, 2, q=3)
    assert abs(F[0, 1] - exact) < 5 * se[0, 1], (l, F[0, 1], se[0, 1], exact)
    assert abs(F[0, 0] - 1.0) < 5 * se[0, 0]


def test_qudit_descriptor_checks(fp):
    with pytest.raises(fp.FpError):
        fp.Ensemble(fp.HEA, 10, 2, 2, q=3)            # qudits: brickwork only
    with pytest.raises(fp.FpError):
        fp.Ensemble(fp.PARALLEL, 10, 2, 2, q=5)
    with pytest.raises(fp.FpError):
        fp.Ensemble(fp.PARALLEL, 10, 1, 3, q=3)           # depth 1: not a dual-circuit sweep
    ens = fp.Ensemble(fp.PARALLEL, 50, 10, 10, q=3)   # 3^18 amplitudes: beyond the state limit
    with pytest.raises(fp.FpError) as e:
        ens.trace_batch(0, 2, fp.PREC_FP32)
    assert e.value.status == -5
