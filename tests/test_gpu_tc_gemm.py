"""The control-variate MLP's dense layer (fp_gemm_bf16, tcgen05 BF16 GEMM with
fused epilogues) against its plain definition: a float64 CPU matmul of the same
BF16-rounded operands, then the epilogue written out elementwise.

Tolerance: BF16 x BF16 products are exact in FP32, so the only error is the
FP32 accumulation of K terms (and the FP32 epilogue), bounded by
K * 2^-23 * sum_k |a_ik b_jk| plus the GELU evaluation error."""
import math

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_09900_gb300 import build
    build.build()
    import paper_2205_09900_gb300 as fpm
    fpm.load()
    return fpm, torch


def gelu64(x, torch):
    return 0.5 * x * (1.0 + torch.erf(x / math.sqrt(2.0)))


def gelu_grad64(z, torch):
    return 0.5 * (1.0 + torch.erf(z / math.sqrt(2.0))) + z * torch.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def run_case(fp, torch, M, N, K, mode, seed, lda=None):
    g = torch.Generator().manual_seed(seed)
    lda = K if lda is None else lda
    A_full = torch.randn(M, lda, generator=g).to(torch.bfloat16)
    A = A_full[:, :K]
    Bt = (torch.randn(N, K, generator=g) / math.sqrt(K)).to(torch.bfloat16)
    bias = torch.randn(N, generator=g, dtype=torch.float32)
    Zin = torch.randn(M, N, generator=g, dtype=torch.float32) if mode == 2 else None
    dev = "cuda"
    A_d = A_full.to(dev)[:, :K]
    Bt_d, bias_d = Bt.to(dev), bias.to(dev)
    Z_d = Zin.to(dev) if mode == 2 else torch.full((M, N), float("nan"), device=dev)
    C = torch.full((M, N), float("nan"), device=dev)
    Cb = torch.zeros((M, N), dtype=torch.bfloat16, device=dev)
    Ct = torch.zeros((N, M), dtype=torch.bfloat16, device=dev)
    fp.gemm_bf16(A_d, Bt_d, bias_d, mode, Z_d, C, Cb, Ct)
    torch.cuda.synchronize()
    a64, b64 = A.double(), Bt.double()
    pre = a64 @ b64.T + bias.double()
    bound = K * 2.0 ** -23 * (a64.abs() @ b64.abs().T) + 1e-6
    if mode == 0:
        ref, tol = pre, bound
    elif mode == 1:
        ref, tol = gelu64(pre, torch), 1.2 * bound + 1e-6 * (1 + pre.abs())
        Zc = Z_d.cpu().double()
        assert torch.all((Zc - pre).abs() <= bound)
    else:
        gz = gelu_grad64(Zin.double(), torch)
        ref, tol = pre * gz, bound * gz.abs() + 1e-5 * pre.abs() * (1 + gz.abs())
    Cc = C.cpu().double()
    err = (Cc - ref).abs()
    assert torch.all(err <= tol), (M, N, K, mode, float((err / tol).max()))
    # BF16 outputs: round-to-nearest of the FP32 result; the transposed copy is the same values
    assert torch.equal(Cb.cpu(), C.cpu().to(torch.bfloat16))
    assert torch.equal(Ct.cpu().T, Cb.cpu())


@pytest.mark.parametrize("M,N,K", [(1, 16, 8), (128, 256, 64), (300, 48, 200), (257, 512, 1000),
                                   (1000, 272, 64), (5, 16, 8), (512, 256, 1200), (1200, 256, 512)])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_gemm_bf16_matches_definition(env, M, N, K, mode):
    fp, torch = env
    run_case(fp, torch, M, N, K, mode, seed=M * 7 + N * 3 + K + mode)


def test_gemm_bf16_strided_a(env):
    fp, torch = env
    run_case(fp, torch, 200, 64, 96, 1, seed=5, lda=136)


def test_gemm_bf16_empty_and_errors(env):
    fp, torch = env
    A = torch.zeros((0, 64), dtype=torch.bfloat16, device="cuda")
    Bt = torch.zeros((16, 64), dtype=torch.bfloat16, device="cuda")
    C = torch.zeros((0, 16), device="cuda")
    fp.gemm_bf16(A, Bt, C=C)                       # M = 0: nothing to do
    A = torch.zeros((4, 64), dtype=torch.bfloat16, device="cuda")
    Bt = torch.zeros((24, 64), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(fp.FpError) as e:
        fp.gemm_bf16(A, Bt, C=torch.zeros((4, 24), device="cuda"))   # N % 16 != 0
    assert e.value.status == -1
    with pytest.raises(fp.FpError) as e:
        fp.gemm_bf16(A, torch.zeros((16, 64), dtype=torch.bfloat16, device="cuda"), mode=2,
                     C=torch.zeros((4, 16), device="cuda"))          # mode 2 without Z
    assert e.value.status == -1


def test_gemm_bf16_full_size_sampled(env):
    # the surrogate-inference shape of the first layer at L = 6 (65536 pairs per
    # chunk, 4nL = 1200 inputs, 256 hidden units), BF16 output only as in the
    # inference pass; 64 sampled rows against the float64 definition
    fp, torch = env
    M, N, K = 65536, 256, 1200
    g = torch.Generator(device="cuda").manual_seed(11)
    A = (torch.rand(M, K, device="cuda", generator=g) * 2 - 1).to(torch.bfloat16)
    Bt = (torch.randn(N, K, device="cuda", generator=g) / math.sqrt(K)).to(torch.bfloat16)
    bias = torch.randn(N, device="cuda", generator=g)
    Cb = torch.zeros(M, N, dtype=torch.bfloat16, device="cuda")
    fp.gemm_bf16(A, Bt, bias, 1, None, None, Cb)
    rows = torch.randint(0, M, (64,), generator=torch.Generator().manual_seed(3))
    rows[0], rows[1] = 0, M - 1
    a64, b64 = A[rows].cpu().double(), Bt.cpu().double()
    pre = a64 @ b64.T + bias.cpu().double()
    ref = gelu64(pre, torch)
    tol = 1.2 * (K * 2.0 ** -23 * (a64.abs() @ b64.abs().T) + 1e-6) + 2.0 ** -8 * ref.abs() + 1e-6
    err = (Cb[rows].cpu().double() - ref).abs()
    assert torch.all(err <= tol), float((err / tol).max())
