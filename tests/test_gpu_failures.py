"""Failure paths, in forms that fault and hang no GPU:
  * a bounded device wait that runs out (the time limit set far below the
    time a normal launch needs) is reported as FP_ERR_TIMEOUT, the kernel
    drains what it issued and frees its tensor memory, and the next launch
    with the default limit is correct;
  * host-side fault injection: a device allocation that fails returns
    FP_ERR_OOM and leaves the ensemble usable;
  * a cancelled Monte Carlo run returns FP_ERR_CANCELLED between batches;
  * checkpoint and resume: a run split into single batches, cancelled once and
    resumed on a second ensemble object, gives the same F and standard errors
    bit for bit as one uninterrupted run (the paper adds samples to stored ones
    until its error bars are small enough: Supplementary Methods,
    "Determination of sample sizes")."""
import numpy as np
import pytest

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


def test_gemm_wait_limit_runs_out(fp):
    import torch
    torch.manual_seed(0)
    M, N, K = 512, 256, 4096
    A = (torch.randn(M, K, device="cuda") / 8).to(torch.bfloat16)
    Bt = (torch.randn(N, K, device="cuda") / 8).to(torch.bfloat16)
    C = torch.empty(M, N, dtype=torch.float32, device="cuda")
    try:
        fp.set_wait_limit_ns(1)                      # 1 ns: the first wait on a TMA load runs out
        with pytest.raises(fp.FpError) as e:
            fp.gemm_bf16(A, Bt, C=C)
        assert e.value.status == -4
    finally:
        fp.set_wait_limit_ns(0)
    fp.gemm_bf16(A, Bt, C=C)                         # the context and the kernel are fine afterwards
    ref = A.double() @ Bt.double().T
    assert torch.max(torch.abs(C.double() - ref)).item() < 1e-3 * torch.max(torch.abs(ref)).item()


def test_allocation_failure_leaves_ensemble_usable(fp):
    ens = fp.Ensemble(fp.PARALLEL, 20, 2, 6, seed=9)
    fp.inject_alloc_failures(1)
    try:
        with pytest.raises(fp.FpError) as e:
            ens.trace_batch(0, 300, fp.PREC_FP64)
        assert e.value.status == -3
    finally:
        fp.inject_alloc_failures(0)
    got, _, _ = ens.trace_batch(0, 300, fp.PREC_FP64)
    ref, _, _ = fp.Ensemble(fp.PARALLEL, 20, 2, 6, seed=9).trace_batch(0, 300, fp.PREC_FP64)
    assert np.array_equal(got, ref)


def test_cancel_between_batches(fp):
    ens = fp.Ensemble(fp.PARALLEL, 20, 2, 5, seed=10)
    ens.cancel()
    with pytest.raises(fp.FpError) as e:
        ens.frame_potential(0, 50_000, 2, 0.0, fp.PREC_FP32)
    assert e.value.status == -6
    F, se, st = ens.frame_potential(0, 50_000, 2, 0.0, fp.PREC_FP32)   # consumed: runs normally
    assert st.pairs == 50_000 and np.all(np.isfinite(F))


def test_checkpoint_resume_is_bit_identical(fp):
    P, K, target = 60_000, 3, 1e-9       # the target is never met: batches 4096, 8192, ... up to P
    a = fp.Ensemble(fp.PARALLEL, 30, 2, 8, seed=12)
    Fa, sea, sta = a.frame_potential(500, P, K, target, fp.PREC_FP32)
    b = fp.Ensemble(fp.PARALLEL, 30, 2, 8, seed=12)
    ck = b.checkpoint(500, K)
    calls = 0
    while ck.pairs_done < P:
        if calls == 2:
            b.cancel()
            with pytest.raises(fp.FpError) as e:
                b.frame_potential_resume(ck, P, K, target, fp.PREC_FP32, max_batches=1)
            assert e.value.status == -6
            b = fp.Ensemble(fp.PARALLEL, 30, 2, 8, seed=12)    # resumed elsewhere
        Fb, seb, stb = b.frame_potential_resume(ck, P, K, target, fp.PREC_FP32, max_batches=1)
        calls += 1
    assert calls >= 4
    assert np.array_equal(Fa, Fb) and np.array_equal(sea, seb)
    assert stb.pairs == sta.pairs == P and ck.next_pair == 500 + P
