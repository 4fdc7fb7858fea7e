"""GPU transfer-matrix sweep for the exact ensemble F^(k) of brickwork circuits
(fp_exact_brickwork_fk; the statistical-mechanics model behind the paper's
Eq. theory_eq, Sec. "Frame potential") against the oracle's explicit
transfer matrix, and at sizes the oracle cannot reach against properties
that hold at any size.  Both sides are FP64: relative agreement 1e-11.
"""
import math

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

TOL = 1e-11


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


@pytest.mark.parametrize("n,l", [(2, 2), (2, 5), (3, 2), (3, 4), (4, 2), (4, 3), (5, 2), (6, 5), (8, 4),
                                 (17, 3), (50, 2), (50, 4), (50, 6)])
def test_exact_f2_matches_oracle(fp, n, l):
    got = fp.exact_brickwork_fk(n, l, 2)
    ref = O.weingarten_fk_brickwork(n, l, 2)
    assert abs(got - ref) <= TOL * abs(ref), (got, ref)


@pytest.mark.parametrize("n,l", [(2, 2), (2, 4), (3, 3), (4, 2), (4, 3), (5, 2), (12, 3), (50, 2)])
def test_exact_f3_matches_oracle(fp, n, l):
    got = fp.exact_brickwork_fk(n, l, 3)
    ref = O.weingarten_fk_brickwork(n, l, 3)
    assert abs(got - ref) <= TOL * abs(ref), (got, ref)


@pytest.mark.parametrize("q,n,l,k", [(3, 2, 3, 2), (3, 4, 2, 2), (3, 6, 3, 2), (3, 8, 4, 2), (4, 7, 3, 2),
                                     (3, 50, 4, 2), (3, 4, 2, 3), (3, 5, 3, 3), (4, 12, 3, 3)])
def test_exact_fk_qudits_match_oracle(fp, q, n, l, k):
    got = fp.exact_brickwork_fk(n, l, k, q=q)
    ref = O.weingarten_fk_brickwork(n, l, k, q)
    assert abs(got - ref) <= TOL * abs(ref), (got, ref)


def test_exact_fk_full_size_properties(fp):
    # n = 50 at every depth the benchmark draws: above the Haar value k!, below the
    # paper's F^(2) bound 2 (1 + (4/5)^{2(l-1)})^{n_g - 1} (Eq. theory_eq, q = 2), and
    # decreasing in l; F^(3) above 3! and decreasing, up to l = 6 (6^10 states)
    n, ng = 50, 25
    f2 = [fp.exact_brickwork_fk(n, l, 2) for l in range(2, 11)]
    for l, f in zip(range(2, 11), f2):
        assert 2.0 < f < 2 * (1 + 0.8 ** (2 * (l - 1))) ** (ng - 1)
    assert all(a > b for a, b in zip(f2, f2[1:]))
    f3 = [fp.exact_brickwork_fk(n, l, 3) for l in range(2, 7)]
    assert all(f > 6.0 for f in f3)
    assert all(a > b for a, b in zip(f3, f3[1:]))
    # n = 2 is one Haar U(4) gate at any depth: F^(3) = 3! at the largest k = 3 state
    assert abs(fp.exact_brickwork_fk(2, 7, 3) - 6.0) < 1e-11 * 6


def test_exact_f2_matches_gpu_monte_carlo_at_depth_10(fp):
    # the deepest benchmark depth, where the oracle's explicit transfer matrix is
    # out of reach: the Monte Carlo estimate of the contraction path agrees within 5 sigma
    exact = fp.exact_brickwork_fk(50, 10, 2)
    ens = fp.Ensemble(fp.PARALLEL, 50, 10, seed=2024)
    F, se, _ = ens.frame_potential(0, 60000, 2, 0.0, fp.PREC_FP32)
    ens.close()
    assert abs(F[0, 1] - exact) < 5 * se[0, 1], (F[0, 1], se[0, 1], exact)


def test_exact_fk_argument_checks(fp):
    for n, l, k in [(50, 1, 2), (50, 13, 2), (50, 8, 3), (50, 4, 4), (1, 4, 2)]:
        with pytest.raises(fp.FpError):
            fp.exact_brickwork_fk(n, l, k)
    with pytest.raises(fp.FpError):
        fp.exact_brickwork_fk(8, 3, 2, q=1)
