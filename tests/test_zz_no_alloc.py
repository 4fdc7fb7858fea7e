"""The allocation-free entry point (fp_trace_brick_static) against fp_trace_batch.

fp_trace_brick_static serves callers that cannot allocate device memory when
they need traces (inside a framework whose memory pool owns the device memory,
in loops that must not block in an allocator): it keeps every intermediate
buffer in one fixed scratch array of the library.  This file
runs last so that a failure here cannot hide any other test; it passes alone in
a fresh process too, because the first call on a device does the set-up.
"""
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


@pytest.mark.parametrize("n,l,prec,calls", [
    (50, 6, 2, [(0, 300), (7000, 257)]),      # FP32 (no recontraction), two calls in a row
    (20, 7, 0, [(11, 200), (5000, 150)]),     # FP64, left boundaries in the static scratch
    (21, 5, 0, [(3, 100), (900, 64)]),        # odd n: the right chain end starts on the other parity
])
def test_static_scratch_matches_trace_batch(fp, n, l, prec, calls):
    import torch
    seed = 31
    ens = fp.Ensemble(fp.PARALLEL, n, l, l, seed=seed)
    stream = torch.cuda.current_stream()
    # one call of this shape first: the first call on a device looks up the
    # scratch address, and CUDA loads the kernels' modules on first use
    warm = torch.empty(2, dtype=torch.float64, device="cuda")
    fp.trace_brick_static(n, l, seed, 0, 1, prec, warm, None, stream.cuda_stream)
    stream.synchronize()
    for first, count in calls:
        tr = torch.full((2 * count,), float("nan"), dtype=torch.float64, device="cuda")
        ka = torch.full((count,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        alloc0 = torch.cuda.memory_allocated()
        fp.trace_brick_static(n, l, seed, first, count, prec, tr, ka, stream.cuda_stream)
        stream.synchronize()
        # nothing was allocated on the device by the call (outputs were made above)
        assert torch.cuda.mem_get_info()[0] == free0
        assert torch.cuda.memory_allocated() == alloc0
        t = tr.cpu().numpy()
        got = t[0::2] + 1j * t[1::2]
        ref, ref_k, _ = ens.trace_batch(first, count, prec)
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1.0)) <= 1e-10
        assert np.max(np.abs(ka.cpu().numpy() - ref_k) / ref_k) <= 1e-10


def test_static_scratch_rejects_oversize_and_bad_args(fp):
    import torch
    tr = torch.zeros(2 * 100000, dtype=torch.float64, device="cuda")
    with pytest.raises(fp.FpError) as e:
        fp.trace_brick_static(50, 6, 1, 0, 100000, 2, tr)
    assert e.value.status == -1 and "at most" in str(e.value)
    with pytest.raises(fp.FpError) as e:
        fp.trace_brick_static(50, 9, 1, 0, 10, 2, tr)           # 16-bit boundary: not this path
    assert e.value.status == -1
    host = np.zeros(20)
    with pytest.raises(fp.FpError) as e:
        fp.trace_brick_static(50, 6, 1, 0, 10, 2, host)        # host output: rejected
    assert e.value.status == -1


def test_static_scratch_rejects_other_device(fp):
    """Outputs or a stream that belong to another GPU are refused before any launch."""
    import torch
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two devices")
    with torch.cuda.device(1):
        tr1 = torch.zeros(20, dtype=torch.float64, device="cuda:1")
        s1 = torch.cuda.Stream(device=1)
    tr0 = torch.zeros(20, dtype=torch.float64, device="cuda:0")
    with torch.cuda.device(0):
        with pytest.raises(fp.FpError) as e:
            fp.trace_brick_static(50, 6, 1, 0, 10, 2, tr1)
        assert e.value.status == -1 and "current device" in str(e.value)
        with pytest.raises(fp.FpError) as e:
            fp.trace_brick_static(50, 6, 1, 0, 10, 2, tr0, None, s1.cuda_stream)
        assert e.value.status == -1 and "device" in str(e.value)
