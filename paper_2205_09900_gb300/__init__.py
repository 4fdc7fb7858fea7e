"""Python binding of the GB300 frame-potential library (``libfp_gb300.so``).

Argument marshalling only: every step of the hot path (sampling, merging,
boundary sweeps, the FP64 meet and the moment reduction) runs in the CUDA
kernels behind the C ABI declared in ``include/fp.h``.  There is no CPU
fallback: importing the binding without the built library raises.

PyTorch supplies device memory and streams; tensors are passed by
``data_ptr()``.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfp_gb300.so")

PARALLEL, LOCAL, HEA, HEA_PAULI = 0, 1, 2, 3
PREC_FP64, PREC_FP32, PREC_FP32_RAW, PREC_TF32X3 = 0, 1, 2, 3
FLAG_SELF_PAIR, FLAG_DIAGONAL_GATES, FLAG_GENERIC_ONLY, FLAG_TIMING, FLAG_NO_GRAPHS = 1, 2, 4, 8, 16
FLAG_SKIP_INFEASIBLE, FLAG_HEA_CZ = 32, 64
K_SAMPLE, K_MERGE, K_TABLES, K_SWEEP, K_BRICK, K_MOMENTS, K_BOOTSTRAP, K_SPIRAL, K_CLASSES = 0, 1, 2, 3, 4, 5, 6, 7, 8
K_NAMES = {0: "sample", 1: "merge", 2: "tables", 3: "sweep_generic", 4: "sweep_brick", 5: "moments",
           6: "bootstrap", 7: "sweep_spiral"}
MAX_STATE_BITS = 24
STATUS = {0: "FP_OK", -1: "FP_ERR_ARG", -2: "FP_ERR_CUDA", -3: "FP_ERR_OOM", -4: "FP_ERR_TIMEOUT",
          -5: "FP_ERR_INFEASIBLE", -6: "FP_ERR_CANCELLED"}

EXPORTED = ["fp_ensemble_create", "fp_ensemble_destroy", "fp_groups", "fp_pair_groups", "fp_export_gates",
            "fp_trace_batch", "fp_reduce_moments", "fp_frame_potential", "fp_kernel_stats_get", "fp_brick_variant",
            "fp_trace_brick_static", "fp_cv_frame_potential", "fp_gemm_bf16", "fp_bootstrap", "fp_epsilon_max",
            "fp_design_layers", "fp_exact_brickwork_fk", "fp_exact_brickwork_fkq", "fp_measure_peak",
            "fp_frame_potential_resume", "fp_cancel", "fp_inject_alloc_failures", "fp_set_wait_limit_ns",
            "fp_last_error"]


class FpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Desc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("n", ctypes.c_int32), ("depth_min", ctypes.c_int32),
                ("depth_max", ctypes.c_int32), ("T_min", ctypes.c_int32), ("T_max", ctypes.c_int32),
                ("T_step", ctypes.c_int32), ("flags", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("kappa_max", ctypes.c_double), ("fp32_tol", ctypes.c_double), ("workspace_bytes", ctypes.c_uint64),
                ("q", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class RunStats(ctypes.Structure):
    _fields_ = [("pairs", ctypes.c_uint64), ("fp64_recontracted", ctypes.c_uint64),
                ("gpu_seconds", ctypes.c_double), ("max_kappa", ctypes.c_double),
                ("n_groups", ctypes.c_int32), ("reached_target", ctypes.c_int32), ("infeasible", ctypes.c_uint64)]


class Checkpoint(ctypes.Structure):
    _fields_ = [("next_pair", ctypes.c_uint64), ("next_batch", ctypes.c_uint64), ("pairs_done", ctypes.c_uint64),
                ("k_max", ctypes.c_int32), ("n_groups", ctypes.c_int32), ("sums", ctypes.c_void_p),
                ("stats", RunStats)]


class KernelStats(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 8), ("launches", ctypes.c_uint64 * 8), ("work", ctypes.c_double * 8),
                ("pairs", ctypes.c_uint64), ("graph_replays", ctypes.c_uint64), ("mma_flops", ctypes.c_double)]


class CvConfig(ctypes.Structure):
    _fields_ = [("hidden", ctypes.c_int32), ("epochs", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("lr", ctypes.c_double), ("first", ctypes.c_uint64),
                ("n_train", ctypes.c_uint64), ("n_correct", ctypes.c_uint64), ("m_surrogate", ctypes.c_uint64),
                ("g_correct", ctypes.c_void_p), ("f_correct", ctypes.c_void_p), ("g_surrogate", ctypes.c_void_p)]


class CvResult(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("F2", "stderr_", "F2_plain", "stderr_plain", "var_f", "var_f_minus_g",
                                               "var_g", "target_scale", "train_loss", "gpu_seconds_exact",
                                               "gpu_seconds_train", "gpu_seconds_surrogate")]


class GateRec(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("q", ctypes.c_int32), ("m", ctypes.c_double * 32)]


_lib = None


def load(path: str = LIB_PATH):
    """Load the shared library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2205_09900_gb300.build.build()")
    L = ctypes.CDLL(path)
    P, vp = ctypes.POINTER, ctypes.c_void_p
    L.fp_ensemble_create.argtypes = [P(Desc), vp, P(vp)]
    L.fp_ensemble_destroy.argtypes = [vp]
    L.fp_ensemble_destroy.restype = None
    L.fp_groups.argtypes = [vp, P(ctypes.c_int32), vp]
    L.fp_pair_groups.argtypes = [vp, ctypes.c_uint64, ctypes.c_uint64, vp]
    L.fp_export_gates.argtypes = [vp, ctypes.c_uint64, ctypes.c_int32, vp, P(ctypes.c_size_t)]
    L.fp_trace_batch.argtypes = [vp, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int32, vp, vp, vp, vp]
    L.fp_reduce_moments.argtypes = [vp, vp, vp, ctypes.c_uint64, ctypes.c_int32, vp]
    L.fp_frame_potential.argtypes = [vp, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int32, ctypes.c_double,
                                     ctypes.c_int32, vp, vp, P(RunStats)]
    L.fp_kernel_stats_get.argtypes = [vp, P(KernelStats), ctypes.c_int32]
    L.fp_brick_variant.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, P(ctypes.c_int32)]
    L.fp_trace_brick_static.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint64,
                                        ctypes.c_uint64, ctypes.c_int32, vp, vp, vp]
    L.fp_cv_frame_potential.argtypes = [vp, P(CvConfig), P(CvResult)]
    i32 = ctypes.c_int32
    L.fp_gemm_bf16.argtypes = [i32, i32, i32, vp, i32, vp, i32, vp, i32, vp, vp, vp, vp, vp]
    f64, u64 = ctypes.c_double, ctypes.c_uint64
    L.fp_bootstrap.argtypes = [vp, vp, vp, u64, i32, i32, u64, vp]
    L.fp_epsilon_max.argtypes = [f64, i32, i32, i32, P(f64)]
    L.fp_design_layers.argtypes = [i32, vp, vp, i32, i32, i32, f64, f64, P(f64), P(f64), P(f64)]
    L.fp_exact_brickwork_fk.argtypes = [i32, i32, i32, vp, P(f64)]
    L.fp_exact_brickwork_fkq.argtypes = [i32, i32, i32, i32, vp, P(f64)]
    L.fp_measure_peak.argtypes = [i32, i32, vp, vp]
    L.fp_frame_potential_resume.argtypes = [vp, P(Checkpoint), u64, u64, i32, f64, i32, vp, vp]
    L.fp_cancel.argtypes = [vp]
    L.fp_inject_alloc_failures.argtypes = [i32]
    L.fp_set_wait_limit_ns.argtypes = [u64]
    L.fp_last_error.restype = ctypes.c_char_p
    for name in EXPORTED:
        if name not in ("fp_ensemble_destroy", "fp_last_error"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(status):
    if status != 0:
        raise FpError(status, load().fp_last_error().decode())


def _ptr(x):
    """Address of a torch tensor, a numpy array, or None."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    return ctypes.c_void_p(x.ctypes.data)


def trace_brick_static(n, l, seed, first, count, prec, tr, kappa=None, stream=None):
    """Brickwork traces through the allocation-free entry point.  `tr` (2*count
    float64) and `kappa` (count float64, optional) must be CUDA tensors; the
    launches are ordered on `stream` (a cudaStream_t handle, None = default) and
    the call does not wait for them."""
    st = None if stream is None else ctypes.c_void_p(stream)
    _check(load().fp_trace_brick_static(n, l, seed, first, count, prec, _ptr(tr), _ptr(kappa), st))
    return tr, kappa


def gemm_bf16(A, Bt, bias=None, mode=0, Z=None, C=None, C_bf16=None, Ct_bf16=None, stream=None):
    """The control-variate MLP's dense layer on the tensor cores (fp_gemm_bf16):
    C = A . Bt^T + bias, then mode 0 (as is), 1 (GELU; pre-activation to Z) or
    2 (times GELU'(Z)).  A [M x K] and Bt [N x K] are bfloat16 CUDA tensors
    (row-major, leading dimensions from their strides); bias [N], Z [M x N], C
    [M x N] float32, C_bf16 [M x N] and Ct_bf16 [N x M] bfloat16 CUDA tensors
    (contiguous) owned by the caller.  Waits for the result."""
    M, K = A.shape
    N = Bt.shape[0]
    st = None if stream is None else ctypes.c_void_p(stream)
    _check(load().fp_gemm_bf16(M, N, K, _ptr(A), A.stride(0), _ptr(Bt), Bt.stride(0), _ptr(bias), mode, _ptr(Z),
                               _ptr(C), _ptr(C_bf16), _ptr(Ct_bf16), st))


def exact_brickwork_fk(n, l, k, stream=None, q=2):
    """Exact ensemble F^(k) (k = 2, 3) of depth-l brickwork circuits on n qubits (or
    qudits of local dimension q), by the Weingarten transfer-matrix sweep on the GPU
    (fp_exact_brickwork_fk / fp_exact_brickwork_fkq)."""
    out = ctypes.c_double()
    st = None if stream is None else ctypes.c_void_p(stream)
    if q == 2:
        _check(load().fp_exact_brickwork_fk(n, l, k, st, ctypes.byref(out)))
    else:
        _check(load().fp_exact_brickwork_fkq(n, l, k, q, st, ctypes.byref(out)))
    return out.value


PEAK_FFMA, PEAK_FFMA2, PEAK_DFMA, PEAK_TC_TF32, PEAK_TC_BF16 = 0, 1, 2, 3, 4


def measure_peak(which, iters=0, stream=None):
    """Measured peak of one arithmetic pipe (fp_measure_peak): dict with tflops, ms,
    sm_mhz (clock during the run), flops_per_clk_sm and sms."""
    import numpy as np
    out = np.zeros(5)
    st = None if stream is None else ctypes.c_void_p(stream)
    _check(load().fp_measure_peak(which, iters, st, _ptr(out)))
    return {"tflops": float(out[0]), "ms": float(out[1]), "sm_mhz": float(out[2]),
            "flops_per_clk_sm": float(out[3]), "sms": int(out[4])}


def inject_alloc_failures(count):
    """The next `count` device allocations of ensemble workspaces fail (fp_inject_alloc_failures)."""
    _check(load().fp_inject_alloc_failures(count))


def set_wait_limit_ns(ns):
    """Time limit of every bounded device wait (fp_set_wait_limit_ns; 0: default 1 s)."""
    _check(load().fp_set_wait_limit_ns(ns))


def epsilon_max_log10(F, k, n, q=2):
    """log10 of epsilon_max = q^{nk} sqrt(F - k!) (fp_epsilon_max); NaN when F <= k!."""
    out = ctypes.c_double()
    _check(load().fp_epsilon_max(float(F), k, n, q, ctypes.byref(out)))
    return out.value


def design_layers(depths, F, k, n, q=2, eps=0.1, dev_max=5.0):
    """(l_eps, A, C) of the exponential fit of F - k! over depths (fp_design_layers)."""
    import numpy as np
    d = np.ascontiguousarray(depths, dtype=np.float64)
    f = np.ascontiguousarray(F, dtype=np.float64)
    le, A, C = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load().fp_design_layers(len(d), _ptr(d), _ptr(f), k, n, q, eps, dev_max, ctypes.byref(le),
                                   ctypes.byref(A), ctypes.byref(C)))
    return le.value, A.value, C.value


class Ensemble:
    """One ensemble of circuit pairs (``fp_ensemble``)."""

    def __init__(self, kind, n, depth_min=1, depth_max=None, T_min=0, T_max=0, T_step=1, seed=1,
                 flags=0, kappa_max=0.0, fp32_tol=0.0, workspace_bytes=0, stream=None, q=2):
        L = load()
        self.desc = Desc(kind, n, depth_min, depth_min if depth_max is None else depth_max, T_min, T_max,
                         T_step, flags, seed, kappa_max, fp32_tol, workspace_bytes, q, 0)
        h = ctypes.c_void_p()
        st = None if stream is None else ctypes.c_void_p(stream)
        _check(L.fp_ensemble_create(ctypes.byref(self.desc), st, ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().fp_ensemble_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def groups(self):
        import numpy as np
        ng = ctypes.c_int32()
        _check(load().fp_groups(self._h, ctypes.byref(ng), None))
        vals = np.zeros(ng.value, dtype=np.int32)
        _check(load().fp_groups(self._h, ctypes.byref(ng), _ptr(vals)))
        return vals

    def pair_groups(self, first, count):
        import numpy as np
        g = np.zeros(count, dtype=np.int32)
        _check(load().fp_pair_groups(self._h, first, count, _ptr(g)))
        return g

    def export_gates(self, pair, which):
        """Sampled gates of U (which=0) or V (which=1): list of (kind, qubit, matrix)."""
        import numpy as np
        nb = ctypes.c_size_t(0)
        _check(load().fp_export_gates(self._h, pair, which, None, ctypes.byref(nb)))
        cnt = nb.value // ctypes.sizeof(GateRec)
        buf = (GateRec * max(1, cnt))()
        _check(load().fp_export_gates(self._h, pair, which, ctypes.cast(buf, ctypes.c_void_p), ctypes.byref(nb)))
        out = []
        for i in range(cnt):
            m = np.array(buf[i].m[:])
            z = m[0::2] + 1j * m[1::2]
            if buf[i].kind == 0:
                mat = z.reshape(4, 4)
            elif buf[i].kind == 1:
                mat = z[:4].reshape(2, 2)
            else:
                mat = z[:4].copy()
            out.append((buf[i].kind, buf[i].q, mat))
        return out

    def trace_batch(self, first, count, prec=PREC_FP64, tr=None, kappa=None, group=None, err=None,
                    with_err=False):
        """Contract pairs first..first+count-1 into caller buffers (torch tensors or numpy
        arrays, host or device).  Allocates numpy host arrays for omitted ones and
        returns (tr complex, kappa, group), or (tr, kappa, group, err) with with_err."""
        import numpy as np
        own = tr is None
        if own:
            tr = np.zeros(2 * count, dtype=np.float64)
            kappa = np.zeros(count, dtype=np.float64) if kappa is None else kappa
            group = np.zeros(count, dtype=np.int32) if group is None else group
            if with_err and err is None:
                err = np.zeros(count, dtype=np.float64)
        _check(load().fp_trace_batch(self._h, first, count, prec, _ptr(tr), _ptr(kappa), _ptr(err), _ptr(group)))
        out = (tr[0::2] + 1j * tr[1::2], kappa, group) if own else (tr, kappa, group)
        return out + (err,) if with_err else out

    def bootstrap(self, tr, group, count, k_max, n_resamples=300, seed=1, out=None):
        """Bootstrap distribution of F^(k) per group (fp_bootstrap): tr [2*count] float64 and
        group [count] int32 (host or device); returns (or fills) [n_groups, k_max, n_resamples]."""
        import numpy as np
        ng = len(self.groups())
        own = out is None
        if own:
            out = np.zeros(ng * k_max * n_resamples, dtype=np.float64)
        _check(load().fp_bootstrap(self._h, _ptr(tr), _ptr(group), count, k_max, n_resamples, seed, _ptr(out)))
        return out.reshape(ng, k_max, n_resamples) if own else out

    def reduce_moments(self, tr_dev, group_dev, count, k_max, out):
        _check(load().fp_reduce_moments(self._h, _ptr(tr_dev), _ptr(group_dev), count, k_max, _ptr(out)))
        return out

    def brick_variant(self, depth, prec=PREC_FP32):
        """(tile bits, window bits, threads, pass kind) of the brickwork sweep the
        autotuner chose for `depth` at `prec` (see fp_brick_variant)."""
        out = (ctypes.c_int32 * 4)()
        _check(load().fp_brick_variant(self._h, int(depth), int(prec), out))
        return tuple(int(x) for x in out)

    def kernel_stats(self, reset=False):
        st = KernelStats()
        _check(load().fp_kernel_stats_get(self._h, ctypes.byref(st), int(bool(reset))))
        return st

    def cv_frame_potential(self, first, n_train, n_correct, m_surrogate, hidden=256, epochs=20, batch=512, lr=1e-3,
                           g_correct=None, f_correct=None, g_surrogate=None):
        """Control-variate F^(2) of a single-depth HEA ensemble (see fp_cv_frame_potential);
        g_correct, f_correct [n_correct] and g_surrogate [m_surrogate] float64 arrays (host or
        device, optional) receive the per-pair values behind the estimate."""
        p = lambda x: None if x is None else _ptr(x).value
        cfg = CvConfig(hidden, epochs, batch, 0, lr, first, n_train, n_correct, m_surrogate, p(g_correct),
                       p(f_correct), p(g_surrogate))
        res = CvResult()
        _check(load().fp_cv_frame_potential(self._h, ctypes.byref(cfg), ctypes.byref(res)))
        return res

    def checkpoint(self, first, k_max):
        """A fresh run state for frame_potential_resume (keeps its sums array alive)."""
        import numpy as np
        ck = Checkpoint()
        ck.next_pair = first
        ck._sums = np.zeros(2 * len(self.groups()) * (2 * k_max + 1))
        ck.sums = ck._sums.ctypes.data
        return ck

    def frame_potential_resume(self, ck, max_pairs, k_max, target_rel_stderr=0.0, prec=PREC_FP64, max_batches=0):
        """Continue the run in `ck` (fp_frame_potential_resume); returns (F, stderr, stats)."""
        import numpy as np
        ng = len(self.groups())
        F = np.zeros(ng * k_max)
        se = np.zeros(ng * k_max)
        _check(load().fp_frame_potential_resume(self._h, ctypes.byref(ck), max_pairs, max_batches, k_max,
                                                target_rel_stderr, prec, _ptr(F), _ptr(se)))
        return F.reshape(ng, k_max), se.reshape(ng, k_max), ck.stats

    def cancel(self):
        """Stop a running (or the next) Monte Carlo run before its next batch (fp_cancel)."""
        _check(load().fp_cancel(self._h))

    def frame_potential(self, first, max_pairs, k_max, target_rel_stderr=0.0, prec=PREC_FP64):
        import numpy as np
        ng = len(self.groups())
        F = np.zeros(ng * k_max)
        se = np.zeros(ng * k_max)
        st = RunStats()
        _check(load().fp_frame_potential(self._h, first, max_pairs, k_max, target_rel_stderr, prec, _ptr(F),
                                         _ptr(se), ctypes.byref(st)))
        return F.reshape(ng, k_max), se.reshape(ng, k_max), st
