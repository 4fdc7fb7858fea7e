"""Pins of the FP64 CPU oracle against facts fixed outside the oracle itself.

Each test cites the passage or the mathematics that fixes the expected value.
None of these tests touches a GPU or the CUDA library.
"""
import itertools
import math

import numpy as np
import pytest

import oracle as O
from tests._golden import paper_values


# --------------------------------------------------------------------------
# Philox4x64-10: the published generator, checked against numpy's own
# implementation of it (numpy.random.Philox increments the counter before
# each block, hence the +1 on c0).
# --------------------------------------------------------------------------
@pytest.mark.parametrize("ctr,key", [((0, 0, 0, 0), (0, 0)), ((7, 3, 99, 1), (12345, 0)),
                                     ((2**64 - 2, 2**63, 5, 4), (2**64 - 1, 17))])
def test_philox_matches_numpy(ctr, key):
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64),
                          counter=np.array(ctr, dtype=np.uint64))
    ref = [int(x) for x in bg.random_raw(4)]
    c = list(ctr)
    c[0] = (c[0] + 1) % 2**64
    assert O.philox4x64(c, key) == ref


# --------------------------------------------------------------------------
# Haar U(4) sampler (Methods, "Sampling U(d^2)"): unitary, and the Haar
# moments E|U_ij|^2 = 1/d, E|U_ij|^4 = 2/(d(d+1)), E Tr U = 0, E|Tr U|^2 = 1.
# --------------------------------------------------------------------------
def test_haar_sampler_unitary_and_moments():
    N = 12000
    mats = np.array([O.haar_u4(11, p, p % 2, p // 2) for p in range(N)])
    err = np.abs(np.einsum("nji,njk->nik", mats.conj(), mats) - np.eye(4)).max()
    assert err < 1e-13
    a2 = np.abs(mats) ** 2
    m2, m4 = a2.mean(), (a2 ** 2).mean()
    # 16 correlated entries per matrix: use per-matrix means for the error bar
    se2 = a2.mean(axis=(1, 2)).std() / math.sqrt(N)
    se4 = (a2 ** 2).mean(axis=(1, 2)).std() / math.sqrt(N)
    assert abs(m2 - 0.25) < 5 * se2 + 1e-12
    assert abs(m4 - 0.1) < 5 * se4
    tr = np.trace(mats, axis1=1, axis2=2)
    assert abs(tr.mean()) < 5 / math.sqrt(N)
    t2 = np.abs(tr) ** 2
    assert abs(t2.mean() - 1) < 5 * t2.std() / math.sqrt(N)


def _lis_le(perm, d):
    best = []
    for x in perm:
        i = np.searchsorted(best, x)
        if i == len(best):
            best.append(x)
        else:
            best[i] = x
    return len(best) <= d


def haar_frame_potential(k, d):
    """E|Tr U|^{2k} over Haar U(d) = number of permutations of k elements with
    no increasing subsequence longer than d (Rains 1998); equals k! for k <= d."""
    return sum(1 for p in itertools.permutations(range(k)) if _lis_le(p, d))


def test_haar_count_reduces_to_paper_value():
    pv = paper_values()
    for k in range(1, 5):
        assert haar_frame_potential(k, 4) == pv[f"haar_F_k{k}"] == math.factorial(k)


def test_single_haar_gate_frame_potential():
    # n = 2, l = 1 is one Haar U(4) gate: F^(k) is the Haar value (Supp.,
    # "Validation of sampling Haar random two-qubit unitaries"); k! holds
    # for k <= d = 4, beyond that the exact Haar value applies.
    d = O.desc(O.PARALLEL, 2, 1, seed=2024)
    tr = O.trace_batch(d, 0, 200000, "dense", threads=8)
    F, se = O.moments(tr, 6)
    for k in range(1, 7):
        exact = haar_frame_potential(k, 4)
        assert abs(F[k - 1] - exact) < 5 * se[k - 1], (k, F[k - 1], exact, se[k - 1])


# --------------------------------------------------------------------------
# Brute force: dense 2^n matrices vs variable elimination, all ensembles.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("kind,n,dmin,dmax,extra", [
    (O.PARALLEL, 6, 1, 5, {}), (O.PARALLEL, 7, 1, 4, {}), (O.PARALLEL, 8, 4, 4, {}),
    (O.HEA, 5, 1, 4, {}), (O.HEA, 6, 2, 3, {}),
    (O.HEA_CNOT, 5, 1, 4, {}), (O.HEA_CNOT, 6, 2, 3, {}), (O.HEA_CZ, 6, 1, 4, {}),
    (O.LOCAL, 6, 1, 1, dict(T_min=4, T_max=24, T_step=4)),
    (O.LOCAL, 7, 1, 1, dict(T_min=10, T_max=30, T_step=10)),
])
def test_dense_matches_variable_elimination(kind, n, dmin, dmax, extra):
    d = O.desc(kind, n, dmin, dmax, seed=77 + n, **extra)
    for p in range(6):
        a = O.trace_pair(d, p, "dense")
        b = O.trace_pair(d, p, "ve")
        c = O.trace_pair(d, p, "ve_greedy")       # the same sums in min-degree order
        assert abs(a - b) <= 1e-12 * max(1.0, abs(a))
        assert abs(a - c) <= 1e-12 * max(1.0, abs(a))


# --------------------------------------------------------------------------
# The paper's amplitude formulation (Sec. "Algorithm description"):
# <Psi| U^dagger V |Psi> with |Psi> = M|0> and M = prod_j CNOT_{a_j,t_j} H_{a_j}
# equals Tr(U^dagger V) / 2^n.  Built here with numpy Kronecker products,
# independently of the oracle's C code.
# --------------------------------------------------------------------------
def _kron_all(ms):
    out = np.array([[1.0 + 0j]])
    for m in ms:
        out = np.kron(out, m)
    return out


def _dense_from_gates(n, gates):
    U = np.eye(2 ** n, dtype=complex)
    for kind, q, m in gates:
        if kind == O.OP_GATE1:
            full = _kron_all([np.eye(2)] * q + [m] + [np.eye(2)] * (n - q - 1))
        else:
            mm = np.diag(m) if kind == O.OP_DIAG2 else m
            full = _kron_all([np.eye(2)] * q + [mm] + [np.eye(2)] * (n - q - 2))
        U = full @ U
    return U


@pytest.mark.parametrize("kind,n,depth", [(O.PARALLEL, 3, 3), (O.PARALLEL, 4, 2), (O.HEA, 3, 2),
                                           (O.HEA_CNOT, 3, 2), (O.HEA_CZ, 4, 2)])
def test_ancilla_amplitude_identity(kind, n, depth):
    d = O.desc(kind, n, depth, seed=5)
    U = _dense_from_gates(n, O.circuit(d, 0, 0))
    V = _dense_from_gates(n, O.circuit(d, 0, 1))
    # registers ordered (a_0..a_{n-1}, t_0..t_{n-1})
    H = np.array([[1, 1], [1, -1]]) / math.sqrt(2)
    N2 = 2 * n
    psi = np.zeros(2 ** N2, dtype=complex)
    psi[0] = 1
    for j in range(n):
        psi = _kron_all([np.eye(2)] * j + [H] + [np.eye(2)] * (N2 - j - 1)) @ psi
    for j in range(n):   # CNOT control a_j (bit position n-1-j from the top half), target t_j
        idx = np.arange(2 ** N2)
        ca = (idx >> (N2 - 1 - j)) & 1
        flip = idx ^ (ca << (N2 - 1 - (n + j)))
        psi = psi[flip]
    W = np.kron(np.eye(2 ** n), U.conj().T @ V)
    amp = np.vdot(psi, W @ psi)
    tr = O.trace_pair(d, 0, "dense")
    assert abs(amp * 2 ** n - tr) < 1e-12
    assert abs(np.trace(U.conj().T @ V) - tr) < 1e-12


def test_fig3b_tensor_identity():
    # H_{m0} CNOT_{m i 0} CNOT_{m 0 j} H_{0 m} summed over m (Fig. 3b).  The
    # figure's derivation states delta_ij; with the 1/sqrt(2) of each Hadamard
    # kept it is delta_ij / 2, the per-qubit factor behind the 2^-n of the
    # amplitude identity in the same section (reading recorded with the others).
    H = np.array([[1, 1], [1, -1]]) / math.sqrt(2)
    C = np.zeros((2, 2, 2))   # C[k, i, j]: control k, target out i, target in j
    for k in range(2):
        for i in range(2):
            for j in range(2):
                C[k, i, j] = (k == 0) * (i == j) + (k == 1) * (i != j)
    T = np.einsum("m,mi,mj,m->ij", H[:, 0], C[:, :, 0], C[:, 0, :], H[0, :])
    assert np.allclose(T, np.eye(2) / 2)


# --------------------------------------------------------------------------
# Invariants and closed forms at full size (n = 50).
# --------------------------------------------------------------------------
@pytest.mark.parametrize("kind,n,depth,extra", [(O.PARALLEL, 50, 5, {}), (O.HEA, 50, 4, {}),
                                                (O.HEA_CNOT, 50, 3, {}), (O.HEA_CZ, 50, 4, {}),
                                                (O.LOCAL, 20, 1, dict(T_min=40, T_max=40))])
def test_self_pair_trace_is_dimension(kind, n, depth, extra):
    # Tr(U^dagger U) = Tr(I) = 2^n
    d = O.desc(kind, n, depth, seed=9, self_pair=True, **extra)
    tr = O.trace_pair(d, 3, "ve")
    assert abs(tr - 2.0 ** n) <= 1e-10 * 2.0 ** n


@pytest.mark.parametrize("n", [7, 8, 50])
def test_brickwork_one_layer_product_form(n):
    # l = 1: U^dagger V is a product of independent 2-qubit gates, so the trace
    # factorises into per-gate traces; an untouched qubit (odd n) gives Tr(I_2) = 2.
    d = O.desc(O.PARALLEL, n, 1, seed=31)
    for p in range(3):
        U, V = O.circuit(d, p, 0), O.circuit(d, p, 1)
        ref = np.prod([np.trace(gu[2].conj().T @ gv[2]) for gu, gv in zip(U, V)]) * 2 ** (n % 2)
        assert abs(O.trace_pair(d, p, "ve") - ref) <= 1e-12 * max(1, abs(ref))


def _hea_angles(seed, pair, which, t, q):
    x = O.philox4x64([t, q, pair, which], [seed, 0])
    return [2 * math.pi * ((v >> 11) * 2.0 ** -53) for v in x[:2]]


def test_hea_one_layer_closed_form():
    # L = 1: the CZ ladders cancel, Tr = prod_q Tr(R_q^U^dagger R_q^V) with
    # R = RY(theta) RZ(phi), whose trace is 2 cos(dtheta/2) cos(dphi/2).
    n, seed = 50, 13
    d = O.desc(O.HEA, n, 1, seed=seed)
    for p in range(3):
        ref = 1.0
        for q in range(n):
            tu, pu = _hea_angles(seed, p, 0, 0, q)
            tv, pv = _hea_angles(seed, p, 1, 0, q)
            ref *= 2 * math.cos((tv - tu) / 2) * math.cos((pv - pu) / 2)
        assert abs(O.trace_pair(d, p, "ve") - ref) <= 1e-12 * max(1, abs(ref))


@pytest.mark.parametrize("as_kind", [O.OP_GATE2, O.OP_DIAG2])
def test_diagonal_gates_transfer_matrix(as_kind):
    # Diagonal 2-qubit gates: U^dagger V is diagonal, Tr = sum_x prod_g phase_g(x),
    # a classical 1D transfer-matrix product 1^T M_0 ... M_{n-2} 1.
    rng = np.random.default_rng(3)
    n, layers = 30, 4
    U, V = [], []
    for circ in (U, V):
        for t in range(layers):
            for b in range(t % 2, n - 1, 2):
                ph = np.exp(1j * rng.uniform(0, 2 * np.pi, 4))
                circ.append((as_kind, b, np.diag(ph) if as_kind == O.OP_GATE2 else ph))
    phase = {b: np.ones(4, dtype=complex) for b in range(n - 1)}
    for (_, b, m) in U:
        phase[b] *= np.conj(np.diag(m) if as_kind == O.OP_GATE2 else m)
    for (_, b, m) in V:
        phase[b] *= np.diag(m) if as_kind == O.OP_GATE2 else m
    vec = np.ones(2, dtype=complex)
    for b in range(n - 1):
        M = phase[b].reshape(2, 2)        # M[x_b, x_{b+1}]
        vec = vec @ M
    ref = vec.sum()
    got = O.trace_ops(n, U, V, "ve")
    assert abs(got - ref) <= 1e-11 * max(1, abs(ref))


# --------------------------------------------------------------------------
# Exact ensemble F^(2) of brickwork circuits (Weingarten transfer matrix).
# --------------------------------------------------------------------------
def test_weingarten_two_qubits_is_haar():
    # n = 2: a product of independent Haar U(4) gates is Haar, F^(2) = 2! = 2.
    for l in range(1, 7):
        assert abs(O.weingarten_f2_brickwork(2, l) - 2.0) < 1e-12


def test_weingarten_one_layer_and_paper_bound():
    pv = paper_values()
    for n in range(2, 13):
        ng = n // 2
        exact_l1 = 2.0 ** ng * 16.0 ** (n % 2)
        assert abs(O.weingarten_f2_brickwork(n, 1) - exact_l1) < 1e-9 * exact_l1
    # Eq. theory_eq: F^(2) < 2 (1 + (2q/(q^2+1))^{2(l-1)})^{n_g - 1}, n_g = floor(n/2), q = 2,
    # an equality at l = 1 for even n (bound = 2^{n_g}).
    q = 2
    for n in range(4, 13, 2):
        ng = n // 2
        for l in range(1, 7):
            bound = 2 * (1 + (2 * q / (q * q + 1)) ** (2 * (l - 1))) ** (ng - 1)
            f = O.weingarten_f2_brickwork(n, l)
            if l == 1:
                assert abs(f - bound) < 1e-9 * bound
            else:
                assert f < bound
    # the paper's slope constant from the same formula: C = 1/log((q^2+1)/2q),
    # layers grow as 2 C log(q) per qubit (Eq. k=2)
    C = 1 / math.log((q * q + 1) / (2 * q))
    assert abs(2 * C * math.log(q) - pv["theory_slope_k2"]) < 0.05


def _haar_projector_k2(d=4):
    """E[G x G x conj(G) x conj(G)] for Haar G in U(d): the orthogonal projector
    onto the span of the permutation vectors |sigma> (sigma in S_2) of
    (C^d)^{x4}, built from their Gram matrix (Schur-Weyl duality), not from
    tabulated Weingarten weights.  Returned as a tensor over the two qubits'
    4-copy legs (dim 16 each): Q[out_a, out_b, in_a, in_b]."""
    vecs = []
    for sig in ((0, 1), (1, 0)):
        v = np.zeros((d,) * 4)
        for i1 in range(d):
            for i2 in range(d):
                i = (i1, i2)
                v[i1, i2, i[sig[0]], i[sig[1]]] = 1.0
        vecs.append(v.reshape(-1))
    V = np.stack(vecs, axis=1)                         # [d^4, 2]
    P = V @ np.linalg.inv(V.T @ V) @ V.T                # orthogonal projector
    # copy c's gate index (a b), a the more significant qubit -> per-qubit legs
    P = P.reshape((2, 2) * 8)                           # out c1..c4 (a, b), in c1..c4 (a, b)
    out_a, out_b = [0, 2, 4, 6], [1, 3, 5, 7]
    P = P.transpose(out_a + out_b + [8 + x for x in out_a] + [8 + x for x in out_b])
    return P.reshape(16, 16, 16, 16)


def _brickwork_f2_moment_operator(n, l):
    """F^(2) = Tr(M^dagger M) with M the second-moment operator of the depth-l
    brickwork ensemble (M = M_l ... M_1, M_t the tensor product of the Haar
    projectors of layer t, identity on idle qubits; U and V independent):
    the trace of the cyclic product P_1 P_2 ... P_l ... P_2 of projectors,
    contracted over the qubits' 4-copy legs with numpy.einsum."""
    Q = _haar_projector_k2()
    layers = list(range(1, l + 1)) + list(range(l - 1, 1, -1))
    letters = iter("abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ")
    start = [next(letters) for _ in range(n)]
    cur = list(start)
    terms = []
    for t in layers:
        for b in range((t - 1) % 2, n - 1, 2):   # layer t acts on bonds b = t-1 mod 2, b+2, ...
            oa, ob = next(letters), next(letters)
            terms.append(oa + ob + cur[b] + cur[b + 1])
            cur[b], cur[b + 1] = oa, ob
    # close the trace: the last leg of each qubit is its first
    ren = {c: s0 for c, s0 in zip(cur, start)}
    terms = ["".join(ren.get(c, c) for c in tm) for tm in terms]
    return float(np.einsum(",".join(terms) + "->", *([Q] * len(terms)), optimize="greedy"))


@pytest.mark.parametrize("n,l,value", [(4, 2, 2.64), (4, 3, 2.2048), (5, 2, 3.0112), (6, 2, None), (5, 3, None)])
def test_weingarten_exact_values(n, l, value):
    # The oracle's transfer matrix against (i) the exact values 2.64, 2.2048 and
    # 3.0112 derived from the Weingarten model behind Eq. theory_eq (Sec. "Frame
    # potential"), and (ii) the second-moment operator of the ensemble built from
    # orthogonal projectors onto permutation vectors -- no Weingarten weight and no
    # link factor of the oracle enters (ii).
    f = O.weingarten_f2_brickwork(n, l)
    direct = _brickwork_f2_moment_operator(n, l)
    assert abs(f - direct) < 1e-12 * direct, (f, direct)
    if value is not None:
        assert abs(f - value) < 1e-12, (f, value)


@pytest.mark.parametrize("n,l", [(4, 2), (4, 3), (5, 2), (6, 2)])
def test_weingarten_matches_monte_carlo(n, l):
    d = O.desc(O.PARALLEL, n, l, seed=100 + 10 * n + l)
    tr = O.trace_batch(d, 0, 120000, "dense", threads=8)
    F, se = O.moments(tr, 2)
    assert abs(F[0] - 1.0) < 5 * se[0]              # brickwork with l >= 2 is a 1-design
    exact = O.weingarten_f2_brickwork(n, l)
    assert abs(F[1] - exact) < 5 * se[1], (F[1], exact, se[1])


def test_weingarten_k3_closed_forms():
    # k = 3 over S_3 pairings: n = 2 is one Haar U(4) gate at any depth, F^(3) = 3! = 6
    # (k <= d); l = 1 is a product of floor(n/2) independent gates and, for odd n, one
    # idle qubit with Tr(I_2)^6 = 64; the k = 2 specialisation reproduces the pinned
    # F^(2) routine.
    for l in range(1, 5):
        assert abs(O.weingarten_fk_brickwork(2, l, 3) - 6.0) < 1e-12
    for n in range(2, 10):
        exact = 6.0 ** (n // 2) * 64.0 ** (n % 2)
        assert abs(O.weingarten_fk_brickwork(n, 1, 3) - exact) < 1e-9 * exact
    for n, l in [(4, 3), (5, 2), (7, 4), (50, 5)]:
        a, b = O.weingarten_fk_brickwork(n, l, 2), O.weingarten_f2_brickwork(n, l)
        assert abs(a - b) < 1e-12 * b


@pytest.mark.parametrize("q", [3, 4])
def test_weingarten_qudits_closed_forms_and_bound(q):
    # qudits of local dimension q (Haar U(q^2) gates): n = 2 is one Haar gate,
    # F^(k) = k! for k <= q^2; l = 1 is a product of floor(n/2) gates and an idle
    # qudit with Tr(I_q)^{2k} = q^{2k}; the paper's Eq. theory_eq bound
    # F^(2) <= 2 (1 + (2q/(q^2+1))^{2(l-1)})^{n_g - 1}, an equality at l = 1 for even n
    for l in range(1, 5):
        for k in (2, 3):
            assert abs(O.weingarten_fk_brickwork(2, l, k, q) - math.factorial(k)) < 1e-11
    for n in range(2, 9):
        for k in (2, 3):
            exact = math.factorial(k) ** (n // 2) * float(q) ** (2 * k * (n % 2))
            assert abs(O.weingarten_fk_brickwork(n, 1, k, q) - exact) < 1e-9 * exact
    for n in (4, 6, 8):
        ng = n // 2
        for l in range(1, 5):
            bound = 2 * (1 + (2 * q / (q * q + 1)) ** (2 * (l - 1))) ** (ng - 1)
            f = O.weingarten_fk_brickwork(n, l, 2, q)
            if l == 1:
                assert abs(f - bound) < 1e-9 * bound
            else:
                assert 2.0 < f < bound


@pytest.mark.parametrize("n,l", [(4, 2), (5, 3)])
def test_weingarten_k3_matches_monte_carlo(n, l):
    d = O.desc(O.PARALLEL, n, l, seed=300 + 10 * n + l)
    tr = O.trace_batch(d, 0, 200000, "dense", threads=8)
    F, se = O.moments(tr, 3)
    exact = O.weingarten_fk_brickwork(n, l, 3)
    assert abs(F[2] - exact) < 5 * se[2], (F[2], exact, se[2])


def test_hea_two_qubits_one_layer_moments():
    # per qubit |2 cos(a/2) cos(b/2)|^{2k} averages to (C(2k,k)/2^k)^2 / ... ->
    # E = (binom(2k,k)^2 / 4^k) per qubit; two qubits multiply.
    d = O.desc(O.HEA, 2, 1, seed=8)
    tr = O.trace_batch(d, 0, 100000, "dense", threads=8)
    F, se = O.moments(tr, 3)
    for k in range(1, 4):
        exact = (math.comb(2 * k, k) ** 2 / 4 ** k) ** 2
        assert abs(F[k - 1] - exact) < 5 * se[k - 1], (k, F[k - 1], exact)


# --------------------------------------------------------------------------
# The paper's hardware-efficient ansatz (Fig. 2c; Sec. "Hardware-efficient
# ansatze as approximate k-designs"): RY(pi/4) wall, then per layer a random
# Pauli rotation on every qubit and CNOT (or CZ) walls on the even and the
# odd bonds.
# --------------------------------------------------------------------------
_PAULI = [np.array([[0, 1], [1, 0]], dtype=complex), np.array([[0, -1j], [1j, 0]]),
          np.array([[1, 0], [0, -1]], dtype=complex)]


def _pauli_rotation_draw(seed, pair, which, t, q):
    x = O.philox4x64([t, q, pair, which], [seed, 0])
    return 2 * math.pi * ((x[0] >> 11) * 2.0 ** -53), ((x[1] >> 32) * 3) >> 32


@pytest.mark.parametrize("kind", [O.HEA_CNOT, O.HEA_CZ])
def test_paper_hea_gates_match_their_definition(kind):
    # every gate against its definition through scipy's matrix exponential:
    # RY(pi/4) = expm(-i pi/8 Y), R_P(theta) = expm(-i theta P / 2), and the
    # textbook CNOT (control = the more significant index bit) or CZ
    expm = pytest.importorskip("scipy.linalg").expm
    n, L, seed = 5, 3, 41
    d = O.desc(kind, n, L, seed=seed)
    cnot = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=complex)
    for which in (0, 1):
        g = O.circuit(d, 0, which)
        expect = [(O.OP_GATE1, q, expm(-1j * math.pi / 8 * _PAULI[1])) for q in range(n)]
        for t in range(L):
            for q in range(n):
                th, ax = _pauli_rotation_draw(seed, 0, which, t, q)
                expect.append((O.OP_GATE1, q, expm(-0.5j * th * _PAULI[ax])))
            for b in list(range(0, n - 1, 2)) + list(range(1, n - 1, 2)):
                if kind == O.HEA_CNOT:
                    expect.append((O.OP_GATE2, b, cnot))
                else:
                    expect.append((O.OP_DIAG2, b, np.array([1, 1, 1, -1], dtype=complex)))
        assert len(g) == len(expect)
        for (k1, q1, m1), (k2, q2, m2) in zip(g, expect):
            assert (k1, q1) == (k2, q2)
            assert np.abs(np.asarray(m1) - m2).max() < 1e-15


def _pauli_trace_one_layer(seed, pair, n):
    # L = 1: the entangling walls of U and V and the RY(pi/4) walls cancel in
    # Tr(U^dagger V) = Tr(R_U^dagger R_V); with R_P(t) = cos(t/2) I - i sin(t/2) P
    # and Tr(P P') = 2 delta_PP', each qubit gives 2 (c c' + delta s s').
    ref = 1.0
    for q in range(n):
        tu, au = _pauli_rotation_draw(seed, pair, 0, 0, q)
        tv, av = _pauli_rotation_draw(seed, pair, 1, 0, q)
        ref *= 2 * (math.cos(tu / 2) * math.cos(tv / 2) + (au == av) * math.sin(tu / 2) * math.sin(tv / 2))
    return ref


@pytest.mark.parametrize("kind", [O.HEA_CNOT, O.HEA_CZ])
def test_paper_hea_one_layer_product_form(kind):
    n, seed = 50, 17
    d = O.desc(kind, n, 1, seed=seed)
    for p in range(4):
        ref = _pauli_trace_one_layer(seed, p, n)
        assert abs(O.trace_pair(d, p, "ve") - ref) <= 1e-12 * max(1, abs(ref))
    d8 = O.desc(kind, 8, 1, seed=seed)
    for p in range(2):
        assert abs(O.trace_pair(d8, p, "dense") - _pauli_trace_one_layer(seed, p, 8)) < 1e-12


def test_paper_hea_two_qubits_one_layer_moments():
    # per qubit E|t|^{2k} = binom(2k,k)/3 + (2/3) binom(2k,k)^2 / 4^k (same axis
    # with probability 1/3: t = 2 cos(dtheta/2); different axes: t = 2 c c',
    # and E cos^{2k} of a uniform angle is binom(2k,k)/4^k); qubits multiply:
    # F^(1) = (4/3)^n, F^(2) = (7/2)^n, F^(3) = (65/6)^n.
    d = O.desc(O.HEA_CNOT, 2, 1, seed=23)
    tr = O.trace_batch(d, 0, 100000, "dense", threads=8)
    F, se = O.moments(tr, 3)
    for k in range(1, 4):
        c = math.comb(2 * k, k)
        exact = (c / 3 + 2 / 3 * c * c / 4 ** k) ** 2
        assert abs(F[k - 1] - exact) < 5 * se[k - 1], (k, F[k - 1], exact)


def test_moments_match_numpy():
    rng = np.random.default_rng(0)
    tr = rng.normal(size=5000) + 1j * rng.normal(size=5000)
    F, se = O.moments(tr, 3)
    for k in range(1, 4):
        x = np.abs(tr) ** (2 * k)
        assert abs(F[k - 1] - x.mean()) < 1e-12 * x.mean()
        assert abs(se[k - 1] - x.std(ddof=1) / math.sqrt(len(x))) < 1e-10 * se[k - 1]


# ---------------------------------------------------------------------------
# Bootstrap (Supplementary "Bootstrapping for uncertainty quantification") and the
# derived outputs of Sec. "Frame potential" (epsilon_max, Eqs. exponential/layers).
def test_bootstrap_resamples_follow_the_multinomial_law():
    # brute force on three samples: each resample mean is the mean of one of the
    # 10 multisets of size 3, with probability 3!/(n1! n2! n3!) / 27
    x = np.array([1.0, 10.0, 100.0])                 # |Tr|^2 values, distinct multiset means
    tr = np.sqrt(x) + 0j
    B = 40000
    Fb = O.bootstrap(tr, np.zeros(3, dtype=np.int32), 1, 1, B, seed=12)[0, 0]
    probs = {}
    for c in itertools.product(range(3), repeat=3):
        m = round(float(np.mean(x[list(c)])), 9)
        probs[m] = probs.get(m, 0) + 1 / 27
    assert len(probs) == 10
    vals, counts = np.unique(np.round(Fb, 9), return_counts=True)
    assert set(vals.tolist()) <= set(probs)
    for v, c in zip(vals, counts):
        p = probs[float(v)]
        assert abs(c / B - p) < 5 * math.sqrt(p * (1 - p) / B), (v, c / B, p)


def test_bootstrap_moments_match_plugin_standard_error():
    rng = np.random.default_rng(3)
    tr = rng.normal(size=400) + 1j * rng.normal(size=400)
    B = 3000
    Fb = O.bootstrap(tr, np.zeros(400, dtype=np.int32), 1, 2, B, seed=5)[0]
    for k in (1, 2):
        xk = np.abs(tr) ** (2 * k)
        # E[mean of a resample] = sample mean; Var = (1/N) * (1/N) sum (x - xbar)^2
        se_plug = xk.std(ddof=0) / math.sqrt(len(xk))
        assert abs(Fb[k - 1].mean() - xk.mean()) < 5 * se_plug / math.sqrt(B)
        assert abs(Fb[k - 1].std() / se_plug - 1.0) < 0.08


def test_bootstrap_groups_are_separate_and_deterministic():
    tr = np.array([1, 2, 3, 1000, 2000, 5], dtype=complex)
    grp = np.array([0, 0, 0, 1, 1, -1], dtype=np.int32)   # -1: ignored
    Fb = O.bootstrap(tr, grp, 3, 2, 200, seed=9)
    assert Fb[0, 0].min() >= 1 and Fb[0, 0].max() <= 9          # group 0: |Tr|^2 in {1, 4, 9}
    assert Fb[1, 0].min() >= 1000 ** 2 and Fb[1, 0].max() <= 2000 ** 2
    assert np.all(np.isnan(Fb[2]))                                # empty group
    assert np.array_equal(Fb, O.bootstrap(tr, grp, 3, 2, 200, seed=9), equal_nan=True)
    assert not np.array_equal(Fb, O.bootstrap(tr, grp, 3, 2, 200, seed=10), equal_nan=True)
    one = O.bootstrap(np.array([2 + 1j]), np.array([0], dtype=np.int32), 1, 3, 10, seed=1)[0]
    assert np.allclose(one, np.array([[5.0], [25.0], [125.0]]))


def test_epsilon_max_closed_form():
    # n = 2 qubits, k = 2: d^k = 16, F - 2! = 1 -> epsilon_max = 16
    assert abs(O.log10_epsilon_max(3.0, 2, 2) - math.log10(16.0)) < 1e-15
    # n = 50: 2^100 sqrt(F - 2) in log10
    assert abs(O.log10_epsilon_max(2.25, 2, 50) - (100 * math.log10(2) + math.log10(0.5))) < 1e-12
    assert math.isnan(O.log10_epsilon_max(1.9, 2, 50))


def test_design_layers_recovers_an_exact_exponential():
    # F(l) - k! = A^2 exp(-2 l / C) exactly; the first depths are pushed out of the
    # fitting region ((F - k!)/k! >= 5) and must not bias the fit
    k, n, A, C = 2, 30, 3.0, 2.5
    depths = list(range(1, 13))
    F = [math.factorial(k) + A * A * math.exp(-2 * l / C) for l in depths]
    F[0] = F[1] = 1e6
    l_eps, A_fit, C_fit = O.design_layers(depths, F, k, n)
    assert abs(A_fit - A) < 1e-9 and abs(C_fit - C) < 1e-12
    assert abs(l_eps - C * (k * n * math.log(2) + math.log(A) + math.log(10))) < 1e-9
    assert all(math.isnan(v) for v in O.design_layers([3], [2.5], k, n))


def test_design_layers_on_the_theory_bound():
    # Eq. theory_eq: F^(2) < 2 (1 + (2q/(q^2+1))^{2(l-1)})^{n_g - 1}; in the fitting
    # region the bound decays as (4/5)^{4(l-1)} for q = 2, i.e. C = -2 / ln(16/25) per
    # layer, and the layer count grows linearly in n (Eq. k=2)
    def bound(n, l):
        return 2 * (1 + (4 / 5) ** (2 * (l - 1))) ** (n // 2 - 1)
    res = {}
    for n in (20, 40, 80):
        depths = list(range(2, 80))
        l_eps, A_fit, C_fit = O.design_layers(depths, [bound(n, l) for l in depths], 2, n)
        assert abs(C_fit - (-2 / math.log(16 / 25))) < 0.02 * C_fit
        res[n] = l_eps
    slope1 = (res[40] - res[20]) / 20
    slope2 = (res[80] - res[40]) / 40
    assert abs(slope1 / slope2 - 1) < 0.05       # linear in n


# --------------------------------------------------------------------------
# Control-variate estimator of F^(2) (the estimand of Sec. "Frame potential";
# F = mean_M g + mean_N (f - g), stderr^2 = Var g / M + Var (f - g) / N).
# --------------------------------------------------------------------------
def test_cv_estimator_hand_example():
    # f - g = (1, 0, 2): mean 1, variance 1; surrogate g = (1, 3): mean 2, variance 2;
    # F = 3, stderr = sqrt(2/2 + 1/3); plain: mean f = 3, Var f = 3, stderr 1
    r = O.cv_estimate([1, 2, 3], [2, 2, 5], [1, 3])
    assert r["F"] == 3.0 and abs(r["stderr"] - math.sqrt(1 + 1 / 3)) < 1e-15
    assert r["F_plain"] == 3.0 and r["var_f"] == 3.0 and r["stderr_plain"] == 1.0
    assert r["var_f_minus_g"] == 1.0 and r["var_g"] == 2.0


def test_cv_estimator_special_cases():
    rng = np.random.default_rng(3)
    f = rng.exponential(size=1000) ** 2
    gs = rng.normal(size=500)
    # a perfect predictor on the correction pairs: the estimate is the surrogate mean
    r = O.cv_estimate(f, f, gs)
    assert abs(r["F"] - gs.mean()) < 1e-12 and abs(r["stderr"] - gs.std(ddof=1) / math.sqrt(500)) < 1e-12
    # g = 0: the plain estimator
    r = O.cv_estimate(np.zeros(1000), f, np.zeros(500))
    assert abs(r["F"] - f.mean()) < 1e-12 and abs(r["stderr"] - r["stderr_plain"]) < 1e-15
    assert abs(r["stderr_plain"] - f.std(ddof=1) / math.sqrt(1000)) < 1e-12


# --------------------------------------------------------------------------
# Qudit brickwork (local dimension q = 3, Haar U(9) gates).
# --------------------------------------------------------------------------
def test_qudit_haar_sampler_moments():
    # Haar U(d), d = 9: E|U_ij|^2 = 1/d, E|U_ij|^4 = 2/(d(d+1)); unitary to rounding
    us = [O.haar_uq(3, 5, p, w, g) for p in range(40) for w in (0, 1) for g in range(25)]
    d = 9
    for U in us[:20]:
        assert np.abs(U.conj().T @ U - np.eye(d)).max() < 1e-13
    a = np.array([np.abs(U) ** 2 for U in us])
    assert abs(a.mean() - 1 / d) < 1e-12                  # rows of a unitary: exact
    m4 = (a ** 2).mean()
    se = (a ** 2).std() / math.sqrt(a.size / d)           # entries of a row are correlated
    assert abs(m4 - 2 / (d * (d + 1))) < 5 * se


@pytest.mark.parametrize("n,l", [(2, 1), (3, 2), (4, 3), (5, 2), (6, 3), (5, 4)])
def test_qudit_dense_matches_elimination(n, l):
    for p in range(4):
        a = O.trace_qudit(3, n, l, 19, p, "dense")
        b = O.trace_qudit(3, n, l, 19, p, "ve")
        assert abs(a - b) <= 1e-12 * max(1.0, abs(a))


def test_qudit_self_pair_is_dimension():
    # V = U: Tr(U^dagger U) = q^n exactly, at the benchmark's size
    for l in (2, 3, 4):
        t = O.trace_qudit(3, 50, l, 3, 1, "ve", self_pair=True)
        assert abs(t / 3.0 ** 50 - 1) < 1e-12


@pytest.mark.parametrize("n", [4, 7, 50])
def test_qudit_one_layer_product_form(n):
    # l = 1: U and V are products of the gates on bonds 0, 2, 4, ...; Tr(U^dagger V)
    # is the product of Tr(G_U^dagger G_V) over them, times q for an idle last qudit
    for p in range(3):
        expect = 1.0 + 0j
        for g, b in enumerate(range(0, n - 1, 2)):
            gu, gv = O.haar_uq(3, 23, p, 0, g), O.haar_uq(3, 23, p, 1, g)
            expect *= np.trace(gu.conj().T @ gv)
        if n % 2:
            expect *= 3
        t = O.trace_qudit(3, n, 1, 23, p, "ve")
        assert abs(t - expect) <= 1e-11 * max(1.0, abs(expect))


def test_qudit_monte_carlo_matches_exact_weingarten():
    # the qudit traces against the oracle's exact qutrit F^(2) (Weingarten transfer
    # matrix, pinned separately): n = 4, l = 2, 20,000 dense pairs, 5 sigma
    tr = np.array([O.trace_qudit(3, 4, 2, 31, p, "dense") for p in range(20000)])
    x = np.abs(tr) ** 4
    F, se = x.mean(), x.std(ddof=1) / math.sqrt(len(x))
    assert abs(np.mean(np.abs(tr) ** 2) - 1.0) < 5 * np.std(np.abs(tr) ** 2) / math.sqrt(len(x))
    exact = O.weingarten_fk_brickwork(4, 2, 2, q=3)
    assert abs(F - exact) < 5 * se, (F, se, exact)
