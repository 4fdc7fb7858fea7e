"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Inputs are the same (seed, pair) on both sides; each side draws its own
random numbers from the Philox keying stated in include/fp.h and
oracle/fp_oracle.h.  Tolerances:
  FP64 path:  |dTr| <= 1e-10 * max(|Tr|, 1)
  FP32 path:  |dTr| <= 1e-4  (traces are plain Tr(U^dagger V), E|Tr|^2 = 1 for
              a 1-design), F^(k) within 1e-3 relative of the FP64 path.
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


KIND = {"parallel": (O.PARALLEL, 0), "hea": (O.HEA, 2), "local": (O.LOCAL, 1)}


def make(fp, kind, n, depth=1, depth_max=None, T=None, seed=1, flags=0):
    ok, fk = KIND[kind]
    dmax = depth if depth_max is None else depth_max
    if T is not None:
        Tmin, Tmax, Tstep = T
        od = O.desc(ok, n, 1, 1, T_min=Tmin, T_max=Tmax, T_step=Tstep, seed=seed,
                    self_pair=bool(flags & fp.FLAG_SELF_PAIR))
        ens = fp.Ensemble(fk, n, 1, 1, Tmin, Tmax, Tstep, seed=seed, flags=flags)
    else:
        od = O.desc(ok, n, depth, dmax, seed=seed, self_pair=bool(flags & fp.FLAG_SELF_PAIR))
        ens = fp.Ensemble(fk, n, depth, dmax, seed=seed, flags=flags)
    return ens, od


def rel_err(a, b):
    return np.abs(a - b) / np.maximum(np.abs(b), 1.0)


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind,n,depth,T", [("parallel", 8, 4, None), ("parallel", 7, 3, None),
                                            ("hea", 6, 3, None), ("local", 9, 1, (5, 25, 5))])
def test_sampler_matches_oracle(fp, kind, n, depth, T):
    ens, od = make(fp, kind, n, depth, T=T, seed=42)
    for pair in range(4):
        for which in (0, 1):
            g = ens.export_gates(pair, which)
            o = O.circuit(od, pair, which)
            assert len(g) == len(o)
            for (k1, q1, m1), (k2, q2, m2) in zip(g, o):
                assert (k1, q1) == (k2, q2)          # integer structure: bit-exact
                assert np.abs(np.asarray(m1) - np.asarray(m2)).max() < 1e-13


def test_pair_depth_draws_match_oracle(fp):
    ens, od = make(fp, "parallel", 50, 2, 10, seed=99)
    g = ens.pair_groups(0, 500)
    assert all(g[p] + 2 == O.pair_depth(od, p) for p in range(500))
    ens, od = make(fp, "local", 20, T=(20, 200, 20), seed=5)
    g = ens.pair_groups(1000, 300)
    assert all(20 + 20 * g[i] == O.pair_depth(od, 1000 + i) for i in range(300))


# ---------------------------------------------------------------------------
def test_fp64_brickwork_n8_l4_dense(fp):
    # the n=8, l=4 brickwork workload: every pair against the dense 256x256 oracle
    ens, od = make(fp, "parallel", 8, 4, seed=1)
    N = 512
    tr, kap, grp = ens.trace_batch(0, N, fp.PREC_FP64)
    ref = O.trace_batch(od, 0, N, "dense", threads=8)
    assert rel_err(tr, ref).max() <= TOL64
    assert np.all(kap >= 1.0 - 1e-12)


@pytest.mark.parametrize("kind,n,depth,T,npairs", [
    ("parallel", 2, 3, None, 8), ("parallel", 3, 2, None, 8), ("parallel", 8, 1, None, 8),
    ("parallel", 9, 3, None, 8), ("parallel", 50, 1, None, 4), ("parallel", 50, 2, None, 6),
    ("parallel", 50, 5, None, 4), ("parallel", 51, 4, None, 4), ("parallel", 50, 7, None, 2),
    ("hea", 2, 1, None, 8), ("hea", 7, 3, None, 6), ("hea", 50, 1, None, 4), ("hea", 50, 4, None, 4),
    ("hea", 50, 6, None, 2),
    ("local", 6, 1, (1, 12, 1), 12), ("local", 20, 1, (20, 60, 20), 6),
])
def test_fp64_trace_matches_oracle(fp, kind, n, depth, T, npairs):
    ens, od = make(fp, kind, n, depth, T=T, seed=7 + n)
    tr, kap, grp = ens.trace_batch(0, npairs, fp.PREC_FP64)
    ref = O.trace_batch(od, 0, npairs, "auto", threads=8)
    assert rel_err(tr, ref).max() <= TOL64, (tr, ref)


def test_fp64_mixed_depth_batch(fp):
    # pairs of depths 2..7 in one batch, ragged plan sizes in one launch
    ens, od = make(fp, "parallel", 50, 2, 7, seed=3)
    N = 24
    tr, kap, grp = ens.trace_batch(5, N, fp.PREC_FP64)
    ref = O.trace_batch(od, 5, N, "ve", threads=8)
    assert rel_err(tr, ref).max() <= TOL64
    assert sorted(set(grp.tolist())) == sorted(set((np.array([O.pair_depth(od, 5 + i) for i in range(N)]) - 2).tolist()))


# ---------------------------------------------------------------------------
# Full-size properties: hold at any depth, so they cover the largest boundaries.
@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-5)])
def test_self_pair_full_size(fp, prec, tol):
    ens, _ = make(fp, "parallel", 50, 9, 10, seed=11, flags=1)   # FLAG_SELF_PAIR
    tr, kap, grp = ens.trace_batch(0, 4, prec)
    assert np.all(np.abs(tr - 2.0 ** 50) <= tol * 2.0 ** 50), tr


def _diag_phases(seed, pair, which, g):
    x = O.philox4x64([0, g, pair, which], [seed, 0])
    return np.exp(2j * np.pi * np.array([(v >> 11) * 2.0 ** -53 for v in x]))


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-4)])
def test_diagonal_gates_full_size(fp, prec, tol):
    # diagonal gates: Tr(U^dagger V) is a classical 1D transfer-matrix product
    n, seed = 50, 17
    ens, od = make(fp, "parallel", n, 10, seed=seed, flags=2)    # FLAG_DIAGONAL_GATES
    tr, kap, grp = ens.trace_batch(0, 3, prec)
    for p in range(3):
        l = 10
        phase = {b: np.ones(4, dtype=complex) for b in range(n - 1)}
        g = 0
        for t in range(1, l + 1):
            for b in range((t - 1) % 2, n - 1, 2):
                phase[b] *= np.conj(_diag_phases(seed, p, 0, g)) * _diag_phases(seed, p, 1, g)
                g += 1
        v = np.ones(2, dtype=complex)
        for b in range(n - 1):
            v = v @ phase[b].reshape(2, 2)
        ref = v.sum()
        assert abs(tr[p] - ref) <= tol * max(1.0, abs(ref)), (p, tr[p], ref)


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind,n,depth,dmax,npairs", [("parallel", 50, 2, 8, 16), ("hea", 50, 2, 6, 12),
                                                      ("parallel", 8, 4, 4, 256)])
def test_fp32_path_matches_oracle(fp, kind, n, depth, dmax, npairs):
    ens, od = make(fp, kind, n, depth, dmax, seed=21)
    tr32, kap, _ = ens.trace_batch(0, npairs, fp.PREC_FP32)
    ref = O.trace_batch(od, 0, npairs, "auto", threads=8)
    err = np.abs(tr32 - ref)
    assert err.max() <= TOL32, (err.max(), kap[np.argmax(err)])


def test_error_estimate_bounds_fp32_error(fp):
    # the per-result error estimate is an upper bound of the actual FP32 error
    # (FP64 path as the reference) at every depth of the benchmark ensemble
    ens, _ = make(fp, "parallel", 50, 2, 10, seed=19)
    N = 3000
    t64, _, g, e64 = ens.trace_batch(0, N, fp.PREC_FP64, with_err=True)
    t32, _, _, e32 = ens.trace_batch(0, N, fp.PREC_FP32_RAW, with_err=True)
    actual = np.abs(t32 - t64)
    assert np.all(actual <= e32), (actual / e32).max()
    assert np.all(e64 < 1e-9)


def test_fp32_policy_recontracts_flagged_pairs(fp):
    # a tolerance below the FP32 error estimates forces every pair onto the FP64 path
    ens = fp.Ensemble(0, 20, 2, 6, seed=29, fp32_tol=1e-12)
    t32, _, _, e = ens.trace_batch(0, 64, fp.PREC_FP32, with_err=True)
    ref, _, _ = ens.trace_batch(0, 64, fp.PREC_FP64)
    assert rel_err(t32, ref).max() <= TOL64
    assert np.all(e < 1e-9)


def test_fp32_frame_potential_within_1e3_of_fp64(fp):
    ens, _ = make(fp, "parallel", 20, 2, 6, seed=23)
    N = 4000
    t64, _, g = ens.trace_batch(0, N, fp.PREC_FP64)
    t32, kap, _ = ens.trace_batch(0, N, fp.PREC_FP32)
    for k in (1, 2, 3, 4):
        f64 = np.mean(np.abs(t64) ** (2 * k))
        f32 = np.mean(np.abs(t32) ** (2 * k))
        assert abs(f32 - f64) <= 1e-3 * f64


# ---------------------------------------------------------------------------
def test_reduce_moments_matches_oracle(fp):
    import torch
    ens, _ = make(fp, "parallel", 8, 1, 3, seed=2)
    rng = np.random.default_rng(5)
    N, kmax = 30001, 4
    trc = rng.normal(size=N) + 1j * rng.normal(size=N)
    grp = rng.integers(0, 3, size=N).astype(np.int32)
    tr_d = torch.tensor(np.stack([trc.real, trc.imag], 1).reshape(-1), device="cuda", dtype=torch.float64)
    g_d = torch.tensor(grp, device="cuda")
    out = np.zeros(3 * (2 * kmax + 1))
    ens.reduce_moments(tr_d, g_d, N, kmax, out)
    out = out.reshape(3, 2 * kmax + 1)
    for gi in range(3):
        sel = trc[grp == gi]
        assert out[gi, 0] == len(sel)
        F, se = O.moments(sel, kmax)
        for k in range(1, kmax + 1):
            S, Q = out[gi, k], out[gi, kmax + k]
            n = len(sel)
            assert abs(S / n - F[k - 1]) <= 1e-12 * F[k - 1]
            se_gpu = math.sqrt((Q - S * S / n) / (n - 1) / n)
            assert abs(se_gpu - se[k - 1]) <= 1e-8 * se[k - 1]


def test_frame_potential_matches_weingarten(fp):
    ens, _ = make(fp, "parallel", 4, 2, seed=31)
    F, se, st = ens.frame_potential(0, 200000, 2, 0.0, fp.PREC_FP64)
    exact = O.weingarten_f2_brickwork(4, 2)
    assert abs(F[0, 0] - 1.0) < 5 * se[0, 0]
    assert abs(F[0, 1] - exact) < 5 * se[0, 1], (F, se, exact)
    assert st.pairs == 200000


@pytest.mark.parametrize("l", [5, 6])
def test_frame_potential_n50_matches_weingarten(fp, l):
    # full-size end-to-end check: the Monte Carlo F^(2) of the benchmark ensemble
    # (n = 50) against the exact ensemble value from the Weingarten transfer matrix
    ens = fp.Ensemble(0, 50, l, l, seed=123 + l)
    F, se, st = ens.frame_potential(0, 400000, 2, 0.0, fp.PREC_FP32)
    exact = O.weingarten_f2_brickwork(50, l)
    assert abs(F[0, 0] - 1.0) < 5 * se[0, 0]
    assert abs(F[0, 1] - exact) < 5 * se[0, 1], (F[0, 1], exact, se[0, 1])


def test_control_variate_is_unbiased(fp):
    # HEA n = 50, L = 4: the control-variate F^(2) and the plain estimate on its
    # correction pairs agree with an independent plain estimate on other pairs
    ens = fp.Ensemble(2, 50, 4, 4, seed=77)
    r = ens.cv_frame_potential(0, 20000, 20000, 400000, epochs=6)
    F, se, st = ens.frame_potential(10_000_000, 400000, 2, 0.0, fp.PREC_FP32)
    ref, ref_se = F[0, 1], se[0, 1]
    assert r.var_f > 0 and r.var_f_minus_g > 0 and r.stderr_ > 0
    assert abs(r.F2 - ref) < 5 * math.sqrt(r.stderr_ ** 2 + ref_se ** 2), (r.F2, r.stderr_, ref, ref_se)
    assert abs(r.F2_plain - ref) < 5 * math.sqrt(r.stderr_plain ** 2 + ref_se ** 2)
    assert math.isfinite(r.train_loss)


def test_control_variate_estimate_matches_oracle(fp):
    # The estimator arithmetic of fp_cv_frame_potential against the oracle's plain
    # two-pass FP64 sums on the same exported per-pair g and f; f against |Tr|^4 of
    # the FP64 path on the same correction pairs.
    import torch
    ens = fp.Ensemble(2, 50, 5, 5, seed=78)
    NT, NC, MS = 4096, 3000, 70000            # surrogate range spans two 2^16 chunks
    gc = np.zeros(NC)
    fc = torch.empty(NC, dtype=torch.float64, device="cuda")   # one device, two host outputs
    gs = np.zeros(MS)
    r = ens.cv_frame_potential(0, NT, NC, MS, epochs=2, g_correct=gc, f_correct=fc, g_surrogate=gs)
    f = fc.cpu().numpy()
    o = O.cv_estimate(gc, f, gs)
    for a, b in ((r.F2, o["F"]), (r.stderr_, o["stderr"]), (r.F2_plain, o["F_plain"]),
                 (r.stderr_plain, o["stderr_plain"]), (r.var_f, o["var_f"]), (r.var_f_minus_g, o["var_f_minus_g"]),
                 (r.var_g, o["var_g"])):
        assert abs(a - b) <= 1e-9 * abs(b), (a, b)
    t64, _, _ = ens.trace_batch(NT, NC, fp.PREC_FP64)
    assert np.max(np.abs(f - np.abs(t64) ** 4) / np.maximum(np.abs(t64) ** 4, 1.0)) < 1e-3
    assert np.all(np.isfinite(gs)) and np.all(np.isfinite(gc))


def test_frame_potential_single_haar_gate(fp):
    ens, _ = make(fp, "parallel", 2, 1, seed=37)
    F, se, st = ens.frame_potential(0, 300000, 4, 0.0, fp.PREC_FP64)
    for k in range(1, 5):
        assert abs(F[0, k - 1] - math.factorial(k)) < 5 * se[0, k - 1]


def test_frame_potential_stops_at_target(fp):
    ens, _ = make(fp, "parallel", 6, 3, seed=41)
    F, se, st = ens.frame_potential(0, 10 ** 7, 2, 0.02, fp.PREC_FP64)
    assert st.reached_target == 1
    assert se[0, 1] / F[0, 1] <= 0.02
    assert st.pairs < 10 ** 7


# ---------------------------------------------------------------------------
def test_errors_and_edges(fp):
    with pytest.raises(fp.FpError) as e:
        fp.Ensemble(0, 1, 2)
    assert e.value.status == -1
    ens, _ = make(fp, "parallel", 50, 14, seed=1)   # 26-bit boundary
    with pytest.raises(fp.FpError) as e:
        ens.trace_batch(0, 1, fp.PREC_FP64)
    assert e.value.status == -5
    ens, od = make(fp, "parallel", 8, 3, seed=1)
    tr, kap, g = ens.trace_batch(0, 0, fp.PREC_FP64)
    assert len(tr) == 0
    tr1, _, _ = ens.trace_batch(10, 1, fp.PREC_FP64)      # single pair, offset start
    assert rel_err(tr1, O.trace_batch(od, 10, 1, "dense")).max() <= TOL64


def test_device_output_pointers(fp):
    import torch
    ens, od = make(fp, "parallel", 8, 4, seed=1)
    N = 64
    tr = torch.zeros(2 * N, dtype=torch.float64, device="cuda")
    kap = torch.zeros(N, dtype=torch.float64, device="cuda")
    grp = torch.zeros(N, dtype=torch.int32, device="cuda")
    ens.trace_batch(0, N, fp.PREC_FP64, tr, kap, grp)
    t = tr.cpu().numpy()
    ref = O.trace_batch(od, 0, N, "dense", threads=8)
    assert rel_err(t[0::2] + 1j * t[1::2], ref).max() <= TOL64


# ---------------------------------------------------------------------------
# Brickwork fast path (dual-circuit sweep) against the generic path and the oracle.
@pytest.mark.parametrize("prec,tol", [(0, TOL64), (1, TOL32)])
def test_brick_path_matches_generic_and_oracle(fp, prec, tol):
    n, seed, N = 50, 13, 24
    ens, od = make(fp, "parallel", n, 2, 8, seed=seed)
    gen = fp.Ensemble(0, n, 2, 8, seed=seed, flags=fp.FLAG_GENERIC_ONLY)
    tb, kb, _ = ens.trace_batch(0, N, prec)
    tg, kg, _ = gen.trace_batch(0, N, prec)
    ref = O.trace_batch(od, 0, N, "ve", threads=8)
    if prec == 0:
        assert rel_err(tb, ref).max() <= TOL64
        assert rel_err(tg, ref).max() <= TOL64
    else:
        assert np.abs(tb - ref).max() <= TOL32
        assert np.abs(tg - ref).max() <= TOL32


@pytest.mark.parametrize("prec,tol", [(0, TOL64), (1, TOL32)])
def test_hea_brick_path_matches_generic_and_oracle(fp, prec, tol):
    # HEA on the dual-circuit kernels (rotations as diagonal maps, CZ ladders as
    # Hadamards on segment bits) against the generic planner path and the oracle
    n, seed, N = 50, 17, 16
    ens, od = make(fp, "hea", n, 2, 8, seed=seed)
    gen = fp.Ensemble(2, n, 2, 8, seed=seed, flags=fp.FLAG_GENERIC_ONLY)
    tb, _, _ = ens.trace_batch(0, N, prec)
    tg, _, _ = gen.trace_batch(0, N, prec)
    ref = O.trace_batch(od, 0, N, "ve", threads=8)
    if prec == 0:
        assert rel_err(tb, ref).max() <= TOL64
        assert rel_err(tg, ref).max() <= TOL64
    else:
        assert np.abs(tb - ref).max() <= TOL32
        assert np.abs(tg - ref).max() <= TOL32


@pytest.mark.parametrize("n,L", [(2, 2), (3, 3), (5, 4), (8, 2), (51, 5)])
def test_hea_small_and_odd_chains(fp, n, L):
    ens, od = make(fp, "hea", n, L, seed=n * 7 + L)
    tr, _, _ = ens.trace_batch(0, 12, fp.PREC_FP64)
    ref = O.trace_batch(od, 0, 12, "auto", threads=8)
    assert rel_err(tr, ref).max() <= TOL64


def test_hea_self_pair_full_size(fp):
    ens, _ = make(fp, "hea", 50, 8, seed=3, flags=1)
    for prec, tol in ((0, 1e-10), (1, 1e-5)):
        tr, _, _ = ens.trace_batch(0, 4, prec)
        assert np.all(np.abs(tr - 2.0 ** 50) <= tol * 2.0 ** 50), tr


@pytest.mark.parametrize("n,l", [(2, 2), (3, 2), (4, 5), (5, 3), (9, 6), (50, 6), (51, 7)])
def test_brick_small_and_odd_chains(fp, n, l):
    ens, od = make(fp, "parallel", n, l, seed=n * 10 + l)
    tr, _, _ = ens.trace_batch(0, 16, fp.PREC_FP64)
    ref = O.trace_batch(od, 0, 16, "auto", threads=8)
    assert rel_err(tr, ref).max() <= TOL64


@pytest.mark.parametrize("l,prec", [(8, 2), (10, 2), (6, 0)])
def test_graph_replay_matches_direct_launches(fp, l, prec, tmp_path, monkeypatch):
    # the same sub-batch shape three times: the first runs directly and is
    # captured, the next two replay the CUDA graph; results are bit-identical
    # to an ensemble that never uses graphs.  Both ensembles share one autotune
    # cache, so they run the same kernel variant (the tuner's timing-based pick
    # could otherwise differ, and with it the FP32 rounding).
    monkeypatch.setenv("FP_AUTOTUNE_CACHE", str(tmp_path / "tune.txt"))
    a = fp.Ensemble(0, 30, l, l, seed=5)
    b = fp.Ensemble(0, 30, l, l, seed=5, flags=fp.FLAG_NO_GRAPHS)
    for first in (0, 1000, 2000):
        ta, ka, _, ea = a.trace_batch(first, 96, prec, with_err=True)
        tb, kb, _, eb = b.trace_batch(first, 96, prec, with_err=True)
        assert np.array_equal(ta, tb) and np.array_equal(ka, kb) and np.array_equal(ea, eb)
    assert a.kernel_stats().graph_replays >= 2
    assert b.kernel_stats().graph_replays == 0


@pytest.mark.parametrize("variant", ["14 4 512 0", "14 5 256 0", "13 4 512 0", "13 4 256 0", "13 5 256 0",
                                     "13 4 512 1", "13 5 256 1", "12 4 256 0", "12 5 128 0",
                                     "12 5 256 3", "12 5 256 4"])
def test_every_tile_variant_matches_fp64(fp, variant, tmp_path, monkeypatch):
    # Each tiled variant the autotuner can pick (tile bits, window bits, threads,
    # pass kind: FMA, persistent double-buffered FMA, tensor cores with the tile's
    # operand in shared or in tensor memory), forced through the tuner's cache
    # file, at the two deepest benchmark depths (and at l = 7, where a 12-bit tile
    # is the whole ring, for the FMA passes); ragged batch (not a multiple of the grid).
    import torch
    cache = tmp_path / "tune.txt"
    name = torch.cuda.get_device_name(0)
    depths = (7, 9, 10) if variant.startswith("12 ") and variant.endswith(" 0") else (9, 10)
    cache.write_text("".join(f"{name} n=30 l={l} fp32|{variant}\n" for l in depths))
    monkeypatch.setenv("FP_AUTOTUNE_CACHE", str(cache))
    for l in depths:
        ens = fp.Ensemble(0, 30, l, l, seed=40 + l)
        t32, _, _ = ens.trace_batch(0, 77, fp.PREC_FP32_RAW)
        t64, _, _ = ens.trace_batch(0, 77, fp.PREC_FP64)
        assert np.abs(t32 - t64).max() <= TOL32, (variant, l)
        ens.close()


def test_bench_workload_sampled_parity(fp):
    # The benchmark's own ensemble (n = 50, l uniform in 2..10, seed 4) in the
    # benchmark's launch shape (one large batch split by depth), FP32 policy
    # path and FP64 path; sampled pairs of every depth against the oracle.
    import torch
    P = 20000
    ens, od = make(fp, "parallel", 50, 2, 10, seed=4)
    tr_d = torch.empty(2 * P, dtype=torch.float64, device="cuda")
    ka_d = torch.empty(P, dtype=torch.float64, device="cuda")
    gr_d = torch.empty(P, dtype=torch.int32, device="cuda")
    ens.trace_batch(0, P, fp.PREC_FP32, tr_d, ka_d, gr_d)
    t = tr_d.cpu().numpy()
    tr32 = t[0::2] + 1j * t[1::2]
    grp = gr_d.cpu().numpy()
    picks = []
    for g in range(9):               # depth 2 + g
        idx = np.nonzero(grp == g)[0]
        picks += list(idx[: (3 if g <= 6 else 1)])
    ref = {}
    import concurrent.futures as cf
    with cf.ThreadPoolExecutor(max_workers=16) as ex:
        for p, r in zip(picks, ex.map(lambda p: O.trace_batch(od, int(p), 1, "ve")[0], picks)):
            ref[p] = r
    tr64, _, _ = ens.trace_batch(0, 0, fp.PREC_FP64)   # no-op call keeps the ensemble warm
    for p in picks:
        assert abs(tr32[p] - ref[p]) <= TOL32, (p, grp[p] + 2, tr32[p], ref[p])
        t64, _, _ = ens.trace_batch(int(p), 1, fp.PREC_FP64)
        assert abs(t64[0] - ref[p]) <= TOL64 * max(1.0, abs(ref[p])), (p, grp[p] + 2, t64[0], ref[p])


def test_skip_infeasible_pairs(fp):
    # local circuits n = 20 with T in {20, 200}: T = 200 boundaries exceed 2^24 amplitudes.
    # Without the flag the call fails; with it those pairs come back NaN / group -1 and
    # the feasible ones still match the oracle.
    ens, od = make(fp, "local", 20, T=(20, 200, 180), seed=21)
    with pytest.raises(fp.FpError) as e:
        ens.trace_batch(0, 16, fp.PREC_FP64)
    assert e.value.status == -5
    ens2 = fp.Ensemble(1, 20, 1, 1, 20, 200, 180, seed=21, flags=fp.FLAG_SKIP_INFEASIBLE)
    tr, kap, grp = ens2.trace_batch(0, 16, fp.PREC_FP64)
    T = np.array([O.pair_depth(od, p) for p in range(16)])
    assert set(T.tolist()) == {20, 200}
    big = T == 200
    assert np.all(grp[big] == -1) and np.all(grp[~big] == 0)
    assert np.all(np.isnan(tr[big])) and np.all(np.isnan(kap[big]))
    idx = np.flatnonzero(~big)
    ref = np.array([O.trace_batch(od, int(p), 1, "ve")[0] for p in idx])
    assert rel_err(tr[idx], ref).max() <= TOL64
    F, se, st = ens2.frame_potential(0, 64, 2, 0.0, fp.PREC_FP32)
    assert st.infeasible + st.pairs == 64 and st.infeasible > 0
    assert np.isfinite(F[0, 0]) and np.isnan(F[1, 0])
    # brickwork depth 14 (26-bit boundary) under the flag: every pair skipped
    ens3 = fp.Ensemble(0, 50, 14, 14, seed=1, flags=fp.FLAG_SKIP_INFEASIBLE)
    tr3, _, grp3 = ens3.trace_batch(0, 4, fp.PREC_FP32)
    assert np.all(np.isnan(tr3)) and np.all(grp3 == -1)


@pytest.mark.parametrize("cluster", ["1", "4", "8", "16"])
def test_generic_sweep_cluster_sizes(fp, cluster, monkeypatch):
    # the generic sweep with every cluster size (CTAs sharing one pair's ops),
    # local circuits n = 20, T = 40..80, FP64 against the oracle and FP32 within 1e-4
    monkeypatch.setenv("FP_SWEEP_CLUSTER", cluster)
    ens, od = make(fp, "local", 20, T=(40, 80, 20), seed=31)
    N = 10
    tr, kap, grp = ens.trace_batch(0, N, fp.PREC_FP64)
    ref = O.trace_batch(od, 0, N, "ve", threads=8)
    assert rel_err(tr, ref).max() <= TOL64
    tr32, _, _ = ens.trace_batch(0, N, fp.PREC_FP32_RAW)
    assert np.abs(tr32 - ref).max() <= TOL32


def test_bootstrap_matches_oracle(fp):
    # traces of a mixed-depth brickwork batch; the GPU bootstrap against the
    # oracle's draw-by-draw resampling on the same traces (same Philox draws)
    import torch
    ens, od = make(fp, "parallel", 12, 2, 5, seed=17)
    N, K, B = 3000, 3, 64
    tr, kap, grp = ens.trace_batch(0, N, fp.PREC_FP64)
    t = np.ascontiguousarray(np.stack([tr.real, tr.imag], axis=1).reshape(-1))
    grp[::97] = -1                                   # ignored entries
    ref = O.bootstrap(tr, grp, 4, K, B, seed=23)
    got = ens.bootstrap(t, grp, N, K, B, seed=23)   # host inputs
    assert np.allclose(got, ref, rtol=1e-12, atol=0, equal_nan=True)
    td, gd = torch.from_numpy(t).cuda(), torch.from_numpy(grp).cuda()
    out = torch.empty(4 * K * B, dtype=torch.float64, device="cuda")
    ens.bootstrap(td, gd, N, K, B, seed=23, out=out)   # device inputs and output
    assert np.allclose(out.cpu().numpy().reshape(4, K, B), ref, rtol=1e-12, atol=0, equal_nan=True)
    # deterministic
    assert np.array_equal(ens.bootstrap(t, grp, N, K, B, seed=23), got, equal_nan=True)


# ---------------------------------------------------------------------------
# Local circuits at T = 100 (the deepest T of the local workload): the pairs
# whose boundaries reach 2^18-2^24 amplitudes and run on 4- and 16-CTA
# clusters, against the oracle's variable elimination in min-degree order
# (a fraction of a second per pair; the qubit-order elimination needs
# factors of 2^25-2^34 entries here), computed once for all cluster sizes.
_T100 = {}


def _t100_reference():
    if not _T100:
        od = O.desc(O.LOCAL, 20, 1, 1, T_min=100, T_max=100, T_step=20, seed=37)
        picks = list(range(8))
        _T100["picks"] = picks
        _T100["ref"] = np.array([O.trace_batch(od, p, 1, "ve_greedy")[0] for p in picks])
    return _T100["picks"], _T100["ref"]


@pytest.mark.parametrize("cluster", ["default", "4", "8", "16"])
def test_local_T100_matches_oracle(fp, cluster, monkeypatch):
    if cluster != "default":
        monkeypatch.setenv("FP_SWEEP_CLUSTER", cluster)
    picks, ref = _t100_reference()
    ens = fp.Ensemble(fp.LOCAL, 20, 1, 1, 100, 100, 20, seed=37)
    N = len(picks)
    tr, kap, grp = ens.trace_batch(0, N, fp.PREC_FP64)
    assert rel_err(tr, ref).max() <= TOL64, rel_err(tr, ref)
    tr32, _, _ = ens.trace_batch(0, N, fp.PREC_FP32_RAW)
    assert np.abs(tr32 - ref).max() <= TOL32
    tr32p, _, _ = ens.trace_batch(0, N, fp.PREC_FP32)        # with the FP64 recontraction policy
    assert np.abs(tr32p - ref).max() <= TOL32
    ens.close()


def test_fp32_frame_potential_within_1e3_of_fp64_bench_ensemble(fp):
    # The benchmark's ensemble (n = 50, l uniform in 2..10, seed 4): F^(k), k = 1..4,
    # of the FP32 policy path within 1e-3 relative of the FP64 path on the same
    # 20,000 pairs, per depth group.
    import torch
    P = 20000
    ens = fp.Ensemble(fp.PARALLEL, 50, 2, 10, seed=4)
    out = {}
    for prec in (fp.PREC_FP64, fp.PREC_FP32):
        tr_d = torch.empty(2 * P, dtype=torch.float64, device="cuda")
        gr_d = torch.empty(P, dtype=torch.int32, device="cuda")
        ens.trace_batch(1_000_000, P, prec, tr_d, None, gr_d)
        t = tr_d.cpu().numpy()
        out[prec] = (t[0::2] + 1j * t[1::2], gr_d.cpu().numpy())
    t64, g64 = out[fp.PREC_FP64]
    t32, g32 = out[fp.PREC_FP32]
    assert np.array_equal(g64, g32)
    for g in range(9):
        sel = g64 == g
        assert sel.sum() > 1500
        for k in (1, 2, 3, 4):
            f64 = np.mean(np.abs(t64[sel]) ** (2 * k))
            f32 = np.mean(np.abs(t32[sel]) ** (2 * k))
            assert abs(f32 - f64) <= 1e-3 * f64, (g + 2, k, f32, f64)
    ens.close()
