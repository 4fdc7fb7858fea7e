"""Plain FP64 CPU oracle for the frame-potential estimator (arXiv:2205.09900).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the
benchmark's CPU-baseline leg are the only callers.  The product library never
imports this module, and this module never imports the product library.

The C source (``fp_oracle.c``) is compiled on first use into
``oracle/libfp_oracle.so`` (git-ignored) with the host C compiler.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fp_oracle.c")
_HDR = os.path.join(_HERE, "fp_oracle.h")
_LIB_PATH = os.path.join(_HERE, "libfp_oracle.so")
_lock = threading.Lock()
_lib = None

PARALLEL, LOCAL, HEA, HEA_CNOT, HEA_CZ = 0, 1, 2, 3, 4
OP_GATE2, OP_GATE1, OP_DIAG2 = 0, 1, 2


class Desc(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32),
        ("n", ctypes.c_int32),
        ("depth_min", ctypes.c_int32),
        ("depth_max", ctypes.c_int32),
        ("T_min", ctypes.c_int32),
        ("T_max", ctypes.c_int32),
        ("T_step", ctypes.c_int32),
        ("self_pair", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
    ]


class Op(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("q", ctypes.c_int32), ("m", ctypes.c_double * 32)]


def build(force: bool = False) -> str:
    """Compile the oracle shared library (idempotent)."""
    need = force or not os.path.exists(_LIB_PATH)
    if not need:
        t_lib = os.path.getmtime(_LIB_PATH)
        need = any(os.path.getmtime(p) > t_lib for p in (_SRC, _HDR))
    if need:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC,
                               "-o", tmp, "-lm", "-lpthread"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P = ctypes.POINTER
            L.orc_philox4x64.argtypes = [P(ctypes.c_uint64), P(ctypes.c_uint64), P(ctypes.c_uint64)]
            L.orc_haar_u4.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                      P(ctypes.c_double)]
            L.orc_pair_depth.argtypes = [P(Desc), ctypes.c_uint64]
            L.orc_circuit.argtypes = [P(Desc), ctypes.c_uint64, ctypes.c_int, P(Op), ctypes.c_int]
            L.orc_trace_dense.argtypes = [ctypes.c_int, ctypes.c_int, P(Op), ctypes.c_int, P(Op),
                                          P(ctypes.c_double)]
            L.orc_trace_ve.argtypes = L.orc_trace_dense.argtypes
            L.orc_trace_ve_greedy.argtypes = L.orc_trace_dense.argtypes
            L.orc_trace_pair.argtypes = [P(Desc), ctypes.c_uint64, ctypes.c_int, P(ctypes.c_double)]
            L.orc_trace_batch.argtypes = [P(Desc), ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                          ctypes.c_int, P(ctypes.c_double)]
            L.orc_moments.argtypes = [P(ctypes.c_double), ctypes.c_int64, ctypes.c_int,
                                      P(ctypes.c_double), P(ctypes.c_double)]
            L.orc_weingarten_f2_brickwork.argtypes = [ctypes.c_int, ctypes.c_int]
            L.orc_haar_uq.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                      P(ctypes.c_double)]
            L.orc_haar_uq.restype = None
            for fn in (L.orc_trace_qudit_dense, L.orc_trace_qudit_ve):
                fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                               P(ctypes.c_double)]
            L.orc_cv_estimate.argtypes = [P(ctypes.c_double), P(ctypes.c_double), ctypes.c_int64,
                                          P(ctypes.c_double), ctypes.c_int64, P(ctypes.c_double)]
            L.orc_cv_estimate.restype = None
            L.orc_bootstrap.argtypes = [P(ctypes.c_double), P(ctypes.c_int32), ctypes.c_int64, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_uint64, P(ctypes.c_double)]
            L.orc_bootstrap.restype = None
            L.orc_weingarten_f2_brickwork.restype = ctypes.c_double
            L.orc_weingarten_fk_brickwork.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
            L.orc_weingarten_fk_brickwork.restype = ctypes.c_double
            L.orc_weingarten_fkq_brickwork.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            L.orc_weingarten_fkq_brickwork.restype = ctypes.c_double
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def desc(kind, n, depth_min=1, depth_max=None, T_min=0, T_max=0, T_step=1, seed=1,
         self_pair=False):
    if depth_max is None:
        depth_max = depth_min
    return Desc(kind, n, depth_min, depth_max, T_min, T_max, T_step, int(bool(self_pair)), seed)


def philox4x64(ctr, key):
    c = (ctypes.c_uint64 * 4)(*ctr)
    k = (ctypes.c_uint64 * 2)(*key)
    o = (ctypes.c_uint64 * 4)()
    lib().orc_philox4x64(c, k, o)
    return [int(x) for x in o]


def haar_u4(seed, pair, which, gate):
    out = np.zeros(32)
    lib().orc_haar_u4(seed, pair, which, gate, _dp(out))
    return (out[0::2] + 1j * out[1::2]).reshape(4, 4)


def pair_depth(d, pair):
    return lib().orc_pair_depth(ctypes.byref(d), pair)


def circuit(d, pair, which):
    """Gate list of U (which=0) or V (which=1) of a pair, as (kind, q, matrix) tuples."""
    cap = 4 + (max(d.depth_max, d.T_max) + 1) * 3 * d.n
    ops = (Op * cap)()
    cnt = lib().orc_circuit(ctypes.byref(d), pair, which, ops, cap)
    if cnt < 0:
        raise RuntimeError(f"orc_circuit failed: {cnt}")
    out = []
    for i in range(cnt):
        m = np.array(ops[i].m[:])
        z = m[0::2] + 1j * m[1::2]
        mat = z.reshape(4, 4) if ops[i].kind == OP_GATE2 else z[:4].copy()
        if ops[i].kind == OP_GATE1:
            mat = mat.reshape(2, 2)
        out.append((ops[i].kind, ops[i].q, mat))
    return out


def _to_ops(gates):
    arr = (Op * max(1, len(gates)))()
    for i, (kind, q, mat) in enumerate(gates):
        arr[i].kind = kind
        arr[i].q = q
        flat = np.asarray(mat, dtype=complex).reshape(-1)
        buf = np.zeros(32)
        buf[0:2 * flat.size:2] = flat.real
        buf[1:2 * flat.size:2] = flat.imag
        arr[i].m[:] = list(buf)
    return arr


def trace_ops(n, U, V, method="ve"):
    """Tr(U^dagger V) for explicit gate lists (method 'dense', 've' in qubit order or
    've_greedy' in min-degree order)."""
    tr = np.zeros(2)
    fn = {"dense": lib().orc_trace_dense, "ve": lib().orc_trace_ve, "ve_greedy": lib().orc_trace_ve_greedy}[method]
    rc = fn(n, len(U), _to_ops(U), len(V), _to_ops(V), _dp(tr))
    if rc:
        raise RuntimeError(f"oracle trace failed: {rc}")
    return complex(tr[0], tr[1])


def trace_pair(d, pair, method="auto"):
    m = {"auto": -1, "dense": 0, "ve": 1, "ve_greedy": 2}[method]
    tr = np.zeros(2)
    rc = lib().orc_trace_pair(ctypes.byref(d), pair, m, _dp(tr))
    if rc:
        raise RuntimeError(f"oracle trace failed: {rc}")
    return complex(tr[0], tr[1])


def trace_batch(d, first, count, method="auto", threads=1):
    m = {"auto": -1, "dense": 0, "ve": 1, "ve_greedy": 2}[method]
    tr = np.zeros(2 * count)
    rc = lib().orc_trace_batch(ctypes.byref(d), first, count, m, threads, _dp(tr))
    if rc:
        raise RuntimeError(f"oracle trace failed: {rc}")
    return tr[0::2] + 1j * tr[1::2]


def moments(tr, kmax):
    t = np.ascontiguousarray(np.stack([np.real(tr), np.imag(tr)], axis=1).reshape(-1), dtype=np.float64)
    F = np.zeros(kmax)
    se = np.zeros(kmax)
    lib().orc_moments(_dp(t), len(tr), kmax, _dp(F), _dp(se))
    return F, se


def haar_uq(q, seed, pair, which, gate):
    """Haar U(q^2) gate g of circuit `which` of a qudit pair (orc_haar_uq), q^2 x q^2 complex."""
    d = q * q
    out = np.zeros(2 * d * d)
    lib().orc_haar_uq(q, seed, pair, which, gate, _dp(out))
    return (out[0::2] + 1j * out[1::2]).reshape(d, d)


def trace_qudit(q, n, l, seed, pair, method="ve", self_pair=False):
    """Tr(U^dagger V) of pair `pair` of the depth-l qudit brickwork ensemble (method 'dense' or 've')."""
    tr = np.zeros(2)
    fn = lib().orc_trace_qudit_dense if method == "dense" else lib().orc_trace_qudit_ve
    rc = fn(q, n, l, seed, pair, int(self_pair), _dp(tr))
    if rc:
        raise RuntimeError(f"oracle qudit trace failed: {rc}")
    return complex(tr[0], tr[1])


def cv_estimate(g_corr, f_corr, g_sur):
    """Control-variate estimate of F^(2) (orc_cv_estimate): dict with F, stderr, F_plain,
    stderr_plain, var_f, var_f_minus_g, var_g."""
    gc = np.ascontiguousarray(g_corr, dtype=np.float64)
    fc = np.ascontiguousarray(f_corr, dtype=np.float64)
    gs = np.ascontiguousarray(g_sur, dtype=np.float64)
    out = np.zeros(7)
    lib().orc_cv_estimate(_dp(gc), _dp(fc), len(gc), _dp(gs), len(gs), _dp(out))
    return dict(zip(("F", "stderr", "F_plain", "stderr_plain", "var_f", "var_f_minus_g", "var_g"), map(float, out)))


def weingarten_f2_brickwork(n, l):
    return float(lib().orc_weingarten_f2_brickwork(n, l))


def weingarten_fk_brickwork(n, l, k, q=2):
    """Exact ensemble F^(k) (k = 2, 3) of brickwork circuits of qudits of dimension q."""
    return float(lib().orc_weingarten_fkq_brickwork(n, l, k, q))


def bootstrap(tr, group, n_groups, kmax, B, seed):
    """Bootstrap distribution of F^(k): array [n_groups, kmax, B] (see orc_bootstrap)."""
    tr = np.asarray(tr)
    t = np.ascontiguousarray(np.stack([np.real(tr), np.imag(tr)], axis=1).reshape(-1), dtype=np.float64)
    g = np.ascontiguousarray(group, dtype=np.int32)
    out = np.zeros(n_groups * kmax * B)
    lib().orc_bootstrap(_dp(t), g.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), len(tr), n_groups, kmax, B,
                        seed, _dp(out))
    return out.reshape(n_groups, kmax, B)


def log10_epsilon_max(F, k, n, q=2):
    """log10 of epsilon_max = d^k sqrt(F - k!), d = q^n (Sec. "Frame potential",
    Eq. epsilonmax); NaN when F <= k!."""
    dev = F - math.factorial(k)
    if not dev > 0:
        return float("nan")
    return k * n * math.log10(q) + 0.5 * math.log10(dev)


def design_layers(depths, F, k, n, q=2, eps=0.1, dev_max=5.0):
    """Layers for an eps-approximate k-design from a depth sweep (Sec. "Frame
    potential", Eqs. exponential and layers; fitting region of the supplementary
    "Choice of curve fitting region"): keep depths with 0 < (F - k!)/k! < dev_max,
    fit log(F - k!) = a + s l by least squares, then A = exp(a/2), C = -2/s and
    l_eps = C (k n ln q + ln A + ln(1/eps)).  Returns (l_eps, A, C); NaNs if fewer
    than two depths qualify or the fitted slope is not negative."""
    fh = math.factorial(k)
    pts = [(float(l), math.log(f - fh)) for l, f in zip(depths, F) if 0 < (f - fh) / fh < dev_max]
    if len(pts) < 2:
        return float("nan"), float("nan"), float("nan")
    x = np.array([p[0] for p in pts])
    y = np.array([p[1] for p in pts])
    xm, ym = x.mean(), y.mean()
    s = float(((x - xm) * (y - ym)).sum() / ((x - xm) ** 2).sum())
    a = float(ym - s * xm)
    if not s < 0:
        return float("nan"), float("nan"), float("nan")
    C = -2.0 / s
    lnA = a / 2.0
    return C * (k * n * math.log(q) + lnA + math.log(1.0 / eps)), math.exp(lnA), C
