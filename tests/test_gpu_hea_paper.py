"""GPU parity for the paper's hardware-efficient ansatz (Fig. 2c; Sec.
"Hardware-efficient ansatze as approximate k-designs"): RY(pi/4) wall, random
Pauli rotations, CNOT (or CZ) walls on the even and then the odd bonds.

The CUDA path lays every CNOT out as H(target) CZ H(target); the oracle
contracts the plain CNOT matrix.  Tolerances as in test_gpu_parity.py:
FP64 |dTr| <= 1e-10 max(|Tr|, 1), FP32 |dTr| <= 1e-4.
"""
import math

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 1e-4


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


def make(fp, cz, n, L, L_max=None, seed=1, self_pair=False):
    Lmax = L if L_max is None else L_max
    od = O.desc(O.HEA_CZ if cz else O.HEA_CNOT, n, L, Lmax, seed=seed, self_pair=self_pair)
    flags = (fp.FLAG_HEA_CZ if cz else 0) | (fp.FLAG_SELF_PAIR if self_pair else 0)
    return fp.Ensemble(fp.HEA_PAULI, n, L, Lmax, seed=seed, flags=flags), od


def rel_err(a, b):
    return np.abs(a - b) / np.maximum(np.abs(b), 1.0)


@pytest.mark.parametrize("cz", [False, True])
def test_paper_hea_gates_match_oracle(fp, cz):
    n, L = 6, 3
    ens, od = make(fp, cz, n, L, seed=42)
    H = np.array([[1, 1], [1, -1]]) / math.sqrt(2)
    for pair in range(3):
        for which in (0, 1):
            g = ens.export_gates(pair, which)
            o = O.circuit(od, pair, which)
            i = 0
            for k2, q2, m2 in o:
                if k2 == O.OP_GATE2:
                    # CNOT as H(target) CZ H(target), with the same bond
                    (ka, qa, ma), (kb, qb, mb), (kc, qc, mc) = g[i:i + 3]
                    assert (ka, qa, kb, qb, kc, qc) == (1, q2 + 1, 2, q2, 1, q2 + 1)
                    prod = np.kron(np.eye(2), mc) @ np.diag(mb) @ np.kron(np.eye(2), ma)
                    assert np.abs(prod - np.asarray(m2)).max() < 1e-15
                    assert np.abs(ma - H).max() < 1e-15
                    i += 3
                else:
                    k1, q1, m1 = g[i]
                    assert (k1, q1) == (k2, q2)
                    assert np.abs(np.asarray(m1) - np.asarray(m2)).max() < 1e-13
                    i += 1
            assert i == len(g)


@pytest.mark.parametrize("cz,n,L,L_max,npairs,method", [
    (False, 2, 1, 3, 9, "dense"), (False, 3, 2, 2, 6, "dense"), (False, 7, 3, 3, 6, "dense"),
    (False, 8, 1, 4, 16, "dense"), (True, 8, 1, 4, 16, "dense"),
    (False, 50, 1, 1, 4, "ve"), (False, 50, 2, 2, 6, "ve"), (False, 50, 3, 3, 3, "ve"),
    (False, 51, 2, 2, 4, "ve"), (True, 50, 4, 4, 3, "ve"),
])
def test_paper_hea_fp64_matches_oracle(fp, cz, n, L, L_max, npairs, method):
    ens, od = make(fp, cz, n, L, L_max, seed=5 + n)
    tr, kap, grp = ens.trace_batch(0, npairs, fp.PREC_FP64)
    ref = O.trace_batch(od, 0, npairs, method, threads=8)
    assert rel_err(tr, ref).max() <= TOL64, (tr, ref)
    assert np.array_equal(grp, np.array([O.pair_depth(od, p) - L for p in range(npairs)]))


def test_paper_hea_fp32_matches_oracle_and_fp64(fp):
    ens, od = make(fp, False, 50, 2, 3, seed=19)
    N = 8
    tr32, _, _ = ens.trace_batch(0, N, fp.PREC_FP32)
    assert np.abs(tr32 - O.trace_batch(od, 0, N, "ve", threads=8)).max() <= TOL32
    # deeper layers (boundaries up to 2^17 amplitudes): FP32 against the GPU FP64 path
    ens, _ = make(fp, False, 50, 4, 8, seed=21)
    N = 64
    t64, _, _ = ens.trace_batch(0, N, fp.PREC_FP64)
    t32, _, _ = ens.trace_batch(0, N, fp.PREC_FP32)
    assert np.abs(t32 - t64).max() <= TOL32


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-5)])
def test_paper_hea_self_pair_full_size(fp, prec, tol):
    # Tr(U^dagger U) = 2^n at n = 50 for the deepest layers the bench runs
    ens, _ = make(fp, False, 50, 7, 8, seed=3, self_pair=True)
    tr, _, _ = ens.trace_batch(0, 6, prec)
    assert np.abs(tr / 2.0 ** 50 - 1).max() <= tol


def test_paper_hea_one_layer_frame_potential(fp):
    # L = 1 closed form (each qubit independent): E|t|^{2k} = binom(2k,k)/3 +
    # (2/3) binom(2k,k)^2/4^k, so F^(1) = (4/3)^n and F^(2) = (7/2)^n
    n = 4
    ens, _ = make(fp, False, n, 1, seed=77)
    F, se, st = ens.frame_potential(0, 200000, 2, 0.0, fp.PREC_FP64)
    for k in (1, 2):
        c = math.comb(2 * k, k)
        exact = (c / 3 + 2 / 3 * c * c / 4 ** k) ** n
        assert abs(F[0, k - 1] - exact) < 5 * se[0, k - 1], (k, F[0, k - 1], exact, se[0, k - 1])


def test_paper_hea_flag_checks(fp):
    with pytest.raises(fp.FpError):
        fp.Ensemble(fp.HEA, 8, 2, flags=fp.FLAG_HEA_CZ)
    with pytest.raises(fp.FpError):
        fp.Ensemble(fp.HEA_PAULI, 8, 2, flags=fp.FLAG_DIAGONAL_GATES)


@pytest.mark.parametrize("n,L_min,L_max", [(3, 2, 3), (4, 2, 4), (9, 2, 5), (50, 2, 8), (51, 3, 6)])
def test_paper_hea_spiral_matches_generic_sweep(fp, n, L_min, L_max):
    # the spiral sweep (default for CNOT walls) against the generic sweep on the same
    # pairs: FP64 to 1e-10 of max(|Tr|, 1), FP32 to 1e-4 absolute
    a = fp.Ensemble(fp.HEA_PAULI, n, L_min, L_max, seed=31 + n)
    b = fp.Ensemble(fp.HEA_PAULI, n, L_min, L_max, seed=31 + n, flags=fp.FLAG_GENERIC_ONLY)
    N = 40
    ta, _, ga = a.trace_batch(0, N, fp.PREC_FP64)
    tb, _, gb = b.trace_batch(0, N, fp.PREC_FP64)
    assert np.array_equal(ga, gb)
    assert rel_err(ta, tb).max() <= TOL64, (ta, tb)
    t32, _, _ = a.trace_batch(0, N, fp.PREC_FP32_RAW)
    assert np.abs(t32 - tb).max() <= TOL32


@pytest.mark.parametrize("n,L", [(12, 5), (50, 6), (50, 7), (50, 8), (51, 8)])
def test_spiral_window_kernels_match_map_by_map(fp, n, L, monkeypatch):
    # register windows of 4 and 5 bits (one CTA, or a 2-CTA cluster at 2^15
    # amplitudes) against one map per pass on the same pairs; FP_SPIRAL_WIN is
    # read when an ensemble plans a depth.  FP64 to 1e-10 of max(|Tr|, 1), FP32
    # to 1e-4 absolute
    N = 24
    out = {}
    for win in ("0", "4", "5"):
        monkeypatch.setenv("FP_SPIRAL_WIN", win)
        e = fp.Ensemble(fp.HEA_PAULI, n, L, seed=77 + L)
        t64, k64, _ = e.trace_batch(0, N, fp.PREC_FP64)
        t32, _, _ = e.trace_batch(0, N, fp.PREC_FP32_RAW)
        e.close()
        out[win] = (t64, t32, k64)
    t64, t32, k64 = out["0"]
    for win in ("4", "5"):
        assert rel_err(out[win][0], t64).max() <= TOL64, win
        assert np.abs(out[win][1] - t64).max() <= TOL32, win
        assert np.all(np.isfinite(out[win][2]))


def test_spiral_batch_beyond_grid_limit(fp):
    # more pairs of one depth than one launch's grid.y holds: the sub-batches of the
    # spiral path give every pair the same trace as a small batch at the same index
    e = fp.Ensemble(fp.HEA_PAULI, 4, 3, seed=12)
    big, _, _ = e.trace_batch(0, 70000, fp.PREC_FP32_RAW)
    for first in (0, 65530, 69990):
        small, _, _ = e.trace_batch(first, 10, fp.PREC_FP32_RAW)
        assert np.array_equal(big[first:first + 10], small)
    assert np.all(np.abs(big) <= 16 + 1e-3)
    e.close()
