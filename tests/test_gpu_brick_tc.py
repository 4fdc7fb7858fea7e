"""The tensor-core tile pass of the brickwork sweep (kernels_brick_tc.cu):
window matrices on tcgen05 (TF32 x 3, FP32 accumulation in tensor memory),
forced through the autotuner's cache file, against the FP64 path and the
oracle at the deep depths l = 8, 9, 10 where it runs."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu
TC1 = "12 5 256 3"    # the tile's operand in shared memory, one tile per CTA, two CTAs per SM
TCM = "12 5 256 4"    # the tile's operand in tensor memory, persistent over the tiles
_ORACLE = {}


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


def _force(tmp_path, monkeypatch, n, depths, variant=TCM):
    import torch
    cache = tmp_path / "tune.txt"
    name = torch.cuda.get_device_name(0)
    cache.write_text("".join(f"{name} n={n} l={l} fp32|{variant}\n" for l in depths))
    monkeypatch.setenv("FP_AUTOTUNE_CACHE", str(cache))


@pytest.mark.parametrize("n,variant", [(30, TC1), (31, TC1), (30, TCM), (31, TCM)])
def test_tc_pass_matches_fp64(fp, n, variant, tmp_path, monkeypatch):
    # ragged batches (not a multiple of anything), even and odd chains; the
    # per-pair error estimate bounds the actual difference
    _force(tmp_path, monkeypatch, n, (8, 9, 10), variant)
    for l in (8, 9, 10):
        ens = fp.Ensemble(fp.PARALLEL, n, l, l, seed=60 + l)
        t32, _, _, e32 = ens.trace_batch(0, 77, fp.PREC_FP32_RAW, with_err=True)
        t64, _, _ = ens.trace_batch(0, 77, fp.PREC_FP64)
        d = np.abs(t32 - t64)
        assert d.max() <= 1e-4, (l, d.max())
        assert np.all(d <= e32), (l, (d / e32).max())
        ens.close()


PICKS = {8: 3, 9: 5, 10: 7}   # one pair of each deep depth of the benchmark ensemble


def _oracle_refs():
    # computed once per session (about a minute of CPU at l = 10)
    import concurrent.futures as cf
    if not _ORACLE:
        with cf.ThreadPoolExecutor(max_workers=3) as ex:
            futs = {l: ex.submit(lambda l=l: O.trace_batch(O.desc(O.PARALLEL, 50, l, seed=80 + l), PICKS[l], 1,
                                                           "ve")[0]) for l in PICKS}
            for l, f in futs.items():
                _ORACLE[l] = f.result()
    return _ORACLE


@pytest.mark.parametrize("variant", [TC1, TCM])
def test_tc_pass_matches_oracle_n50(fp, variant, tmp_path, monkeypatch):
    # one pair of each deep depth of the benchmark ensemble against the oracle
    _force(tmp_path, monkeypatch, 50, (8, 9, 10), variant)
    refs = _oracle_refs()
    for l, p in PICKS.items():
        ens = fp.Ensemble(fp.PARALLEL, 50, l, l, seed=80 + l)
        t32, _, _ = ens.trace_batch(p, 1, fp.PREC_FP32)
        assert abs(t32[0] - refs[l]) <= 1e-4, (l, t32[0], refs[l])
        ens.close()


@pytest.mark.parametrize("variant", [TC1, TCM])
def test_tc_pass_full_size_self_pair(fp, variant, tmp_path, monkeypatch):
    # V = U: Tr(U^dagger U) = 2^50 exactly, through the tensor-core passes at l = 10
    _force(tmp_path, monkeypatch, 50, (10,), variant)
    ens = fp.Ensemble(fp.PARALLEL, 50, 10, 10, seed=3, flags=fp.FLAG_SELF_PAIR)
    t, _, _ = ens.trace_batch(0, 8, fp.PREC_FP32_RAW)
    assert np.all(np.abs(t / 2.0 ** 50 - 1) < 1e-4), t
    ens.close()


def test_tc_pass_frame_potential_within_1e3(fp, tmp_path, monkeypatch):
    # F^(k), k = 1..4, of the FP32 policy (tensor-core passes) within 1e-3 of FP64
    _force(tmp_path, monkeypatch, 50, (8, 9, 10))
    for l in (8, 9, 10):
        ens = fp.Ensemble(fp.PARALLEL, 50, l, l, seed=90 + l)
        N = 1500
        t64, _, _ = ens.trace_batch(0, N, fp.PREC_FP64)
        t32, _, _ = ens.trace_batch(0, N, fp.PREC_FP32)
        for k in (1, 2, 3, 4):
            f64 = np.mean(np.abs(t64) ** (2 * k))
            f32 = np.mean(np.abs(t32) ** (2 * k))
            assert abs(f32 - f64) <= 1e-3 * f64, (l, k)
        ens.close()


@pytest.mark.parametrize("variant", [TC1, TCM, "13 5 256 0"])
def test_brick_variant_reports_the_forced_choice(fp, variant, tmp_path, monkeypatch):
    # fp_brick_variant: FP_ERR_ARG before the depth has run, then the variant the
    # tuner's cache file fixed, shared by FP32 and FP32 without recontraction
    _force(tmp_path, monkeypatch, 50, (10,), variant)
    ens = fp.Ensemble(fp.PARALLEL, 50, 10, 10, seed=5)
    with pytest.raises(fp.FpError):
        ens.brick_variant(10, fp.PREC_FP32)
    ens.trace_batch(0, 4, fp.PREC_FP32_RAW)
    want = tuple(int(x) for x in variant.split())
    assert ens.brick_variant(10, fp.PREC_FP32) == want
    assert ens.brick_variant(10, fp.PREC_FP32_RAW) == want
    with pytest.raises(fp.FpError):
        ens.brick_variant(10, fp.PREC_FP64)
    with pytest.raises(fp.FpError):
        ens.brick_variant(9, fp.PREC_FP32)
    ens.close()


def test_tune_cache_entries_are_per_kind(fp, tmp_path, monkeypatch):
    # 12-bit tiles through the 5 lowest bits, 128 threads: a brickwork choice at l = 7, 8;
    # the HEA's l = 7 plan of that shape has passes of 300 gates (over the limit of 255).
    # A brickwork entry does not apply to the HEA, and an HEA entry it cannot run is
    # retuned instead of failing the call.
    import torch
    name = torch.cuda.get_device_name(0)
    cache = tmp_path / "tune.txt"
    cache.write_text(f"{name} n=50 l=7 fp32|12 5 128 0\n{name} n=50 l=8 fp32|12 5 128 0\n"
                     f"{name} n=50 l=7 fp32 hea|12 5 128 0\n")
    monkeypatch.setenv("FP_AUTOTUNE_CACHE", str(cache))
    ens = fp.Ensemble(fp.HEA, 50, 7, 8, seed=4)
    t, _, _ = ens.trace_batch(0, 16, fp.PREC_FP32)
    assert np.all(np.isfinite(t))
    lines = cache.read_text().splitlines()
    assert sum(" n=50 l=7 fp32 hea|" in x for x in lines) == 2, lines   # the unusable entry, then the tuned one
    assert any(" n=50 l=8 fp32 hea|" in x for x in lines), lines
    assert ens.brick_variant(7, fp.PREC_FP32) != (12, 5, 128, 0)
    ens.close()
    brick = fp.Ensemble(fp.PARALLEL, 50, 7, 8, seed=4)
    brick.trace_batch(0, 8, fp.PREC_FP32)
    assert brick.brick_variant(7, fp.PREC_FP32) == (12, 5, 128, 0)
    assert brick.brick_variant(8, fp.PREC_FP32) == (12, 5, 128, 0)
    brick.close()


def test_tf32x3_precision_takes_the_tensor_cores(fp, tmp_path, monkeypatch):
    # FP_PREC_TF32X3: the autotuner restricted to the tensor-core passes at l >= 8,
    # the FMA passes below; the FP32 policy's results (within 1e-4 of FP64 and of
    # the oracle); an unknown precision is refused
    monkeypatch.setenv("FP_AUTOTUNE_CACHE", str(tmp_path / "tune.txt"))
    ens = fp.Ensemble(fp.PARALLEL, 50, 7, 10, seed=13)
    t, _, g = ens.trace_batch(0, 40, fp.PREC_TF32X3)
    t64, _, _ = ens.trace_batch(0, 40, fp.PREC_FP64)
    assert np.abs(t - t64).max() <= 1e-4
    for l in sorted(set(int(x) + 7 for x in g)):
        kind = ens.brick_variant(l, fp.PREC_TF32X3)[3]
        assert kind in ((3, 4) if l >= 8 else (0, 1)), (l, kind)
    with pytest.raises(fp.FpError):
        ens.trace_batch(0, 1, 4)
    ens.close()
    refs = _oracle_refs()
    for l, p in PICKS.items():
        e = fp.Ensemble(fp.PARALLEL, 50, l, l, seed=80 + l)
        t, _, _ = e.trace_batch(p, 1, fp.PREC_TF32X3)
        assert abs(t[0] - refs[l]) <= 1e-4, (l, t[0], refs[l])
        e.close()
