/*
 * fp_oracle.h -- plain FP64 CPU oracle for the frame-potential estimator of
 * "Estimating the randomness of quantum circuit ensembles up to 50 qubits"
 * (arXiv:2205.09900).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, obviously-correct
 * reference that the GPU library is checked against.  Only the test suite,
 * the package smoke check and the benchmark's CPU-baseline leg may load it.
 * It shares no code, header, table or helper with the CUDA library: it has
 * its own counter-based generator (Philox4x64-10, Salmon et al., SC'11), its
 * own Gaussian transform (Box-Muller), its own Haar sampler (classical
 * Gram-Schmidt QR with positive-real R diagonal, Mezzadri 2007), its own
 * circuit builders, and contracts Tr(U^dagger V) either densely (n <= 12) or
 * by plain variable elimination over raw wire segments, without merging any
 * gates.
 *
 * What it computes (paper sections cited per function in fp_oracle.c):
 *   Tr(U^dagger V) = sum_{ij} conj(U_ij) V_ij                (Sec. "Frame potential")
 *   F^(k) ~= (1/N) sum |Tr(U^dagger V)|^{2k}                 (Sec. "Algorithm description")
 *   exact ensemble F^(2) and F^(3) of brickwork circuits by a
 *   Weingarten transfer matrix                                (Eq. theory_eq context)
 *   bootstrap distribution of F^(k)                           (Supplementary, "Bootstrapping
 *                                                              for uncertainty quantification")
 *
 * Conventions (the paper leaves them open; the GPU library states the same
 * conventions in its own header, written separately):
 *   - qubit 0 is the most significant bit of a basis index;
 *   - a 2-qubit gate on bond (b, b+1) has matrix index (a_b a_{b+1}) with a_b
 *     the more significant bit;
 *   - a circuit U = G_T ... G_1 (G_1 acts first);
 *   - RY(t) = exp(-i t Y / 2), RZ(p) = exp(-i p Z / 2); the HEA per-qubit gate
 *     is RY(theta) RZ(phi) (RZ acts first), followed by CZ on every bond.
 *
 * Random-number keying (the input-generator definition both sides follow):
 *   key = {seed, 0}; counter = {c0, c1, pair, stream}; one Philox4x64-10 block
 *   gives four 64-bit words x0..x3.
 *     Haar gate g of circuit w (w=0: U, w=1: V): blocks c0 = 0..7, c1 = g,
 *       stream = w.  Entry k = 4r + c of the 4x4 Gaussian Z uses block k/2,
 *       words (x0,x1) for even k and (x2,x3) for odd k, via Box-Muller:
 *       u1 = ((xa >> 11) + 1) 2^-53, u2 = (xb >> 11) 2^-53,
 *       Z_k = sqrt(-2 ln u1) (cos 2 pi u2 + i sin 2 pi u2) / sqrt 2.
 *     Local-circuit bond of gate g of circuit w: c0 = 0, c1 = g, stream = 2 + w,
 *       bond = ((x0 >> 32) (n - 1)) >> 32.
 *     Per-pair depth (l, L) or gate count T: c0 = c1 = 0, stream = 4,
 *       index = ((x0 >> 32) * choices) >> 32.
 *     HEA angles of circuit w, layer t (0-based), qubit q: c0 = t, c1 = q,
 *       stream = w; theta = 2 pi (x0 >> 11) 2^-53, phi = 2 pi (x1 >> 11) 2^-53.
 *     Paper-HEA rotation of circuit w, layer t, qubit q: the same block;
 *       theta = 2 pi (x0 >> 11) 2^-53, Pauli axis ((x1 >> 32) * 3) >> 32
 *       (0: X, 1: Y, 2: Z).
 */
#ifndef FP_ORACLE_H
#define FP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ORC_HEA_CNOT / ORC_HEA_CZ: the paper's hardware-efficient ansatz (Fig. 2c):
 * a fixed RY(pi/4) wall, then per layer exp(-i theta P / 2) on every qubit
 * (P uniform in {X, Y, Z}, theta uniform in [0, 2 pi)) and two entangling
 * walls, on the even bonds and then on the odd bonds, of CNOT (control b,
 * target b+1) or CZ. */
enum { ORC_PARALLEL = 0, ORC_LOCAL = 1, ORC_HEA = 2, ORC_HEA_CNOT = 3, ORC_HEA_CZ = 4 };
enum { ORC_OP_GATE2 = 0, ORC_OP_GATE1 = 1, ORC_OP_DIAG2 = 2 };

typedef struct {
    int32_t kind;            /* ORC_PARALLEL, ORC_LOCAL, ORC_HEA, ORC_HEA_CNOT, ORC_HEA_CZ */
    int32_t n;               /* qubits on an open chain */
    int32_t depth_min;       /* l (parallel) or L (the HEA kinds) */
    int32_t depth_max;
    int32_t T_min, T_max, T_step;   /* local circuits: gate count choices */
    int32_t self_pair;       /* nonzero: V := U (test invariant Tr = 2^n) */
    uint64_t seed;
} orc_desc;

typedef struct {
    int32_t kind;            /* ORC_OP_GATE2 on (q,q+1): m = 4x4 row-major;
                                ORC_OP_GATE1 on q: m[0..3] = 2x2 row-major;
                                ORC_OP_DIAG2 on (q,q+1): m[0..3] = diagonal */
    int32_t q;
    double m[32];            /* complex entries, (re, im) interleaved */
} orc_op;

void   orc_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);
void   orc_haar_u4(uint64_t seed, uint64_t pair, int which, int gate, double out[32]);
int    orc_pair_depth(const orc_desc *d, uint64_t pair);
int    orc_circuit(const orc_desc *d, uint64_t pair, int which, orc_op *ops, int max_ops);
int    orc_trace_dense(int n, int nU, const orc_op *U, int nV, const orc_op *V, double tr[2]);
int    orc_trace_ve(int n, int nU, const orc_op *U, int nV, const orc_op *V, double tr[2]);
/* the same elimination in min-degree order (same trace, smaller intermediates) */
int    orc_trace_ve_greedy(int n, int nU, const orc_op *U, int nV, const orc_op *V, double tr[2]);
int    orc_trace_pair(const orc_desc *d, uint64_t pair, int method, double tr[2]);
int    orc_trace_batch(const orc_desc *d, uint64_t first, uint64_t count, int method,
                       int nthreads, double *tr);
void   orc_moments(const double *tr, int64_t N, int kmax, double *F, double *se);
/* Control-variate estimate of F^(2) from g on N correction and M surrogate pairs
 * and f = |Tr|^4 on the correction pairs: out[7] = F, stderr, F_plain,
 * stderr_plain, Var f, Var (f - g), Var g (see fp_oracle.c). */
void   orc_cv_estimate(const double *g_corr, const double *f_corr, int64_t N, const double *g_sur, int64_t M,
                       double *out);
double orc_weingarten_f2_brickwork(int n, int l);
/* Exact ensemble F^(k), k = 2 or 3, of brickwork circuits (the same model
 * over S_k pairings); NaN for other k. */
double orc_weingarten_fk_brickwork(int n, int l, int k);
/* The same for qudits of local dimension q >= 2 (Haar U(q^2) gates). */
double orc_weingarten_fkq_brickwork(int n, int l, int k, int q);
/* Bootstrap distribution of F^(k) per group (Supplementary "Bootstrapping for
 * uncertainty quantification"): every group's N_g traces are resampled N_g
 * times with replacement, B times.  Draw i of resample b in group g takes
 * position ((x >> 32) N_g) >> 32 of the group's pairs listed in increasing
 * index order, x = word i mod 4 of the Philox4x64-10 block with key
 * {seed, 0} and counter {b, i / 4, g, 5}.  Pairs with group < 0 or
 * >= n_groups are ignored.  F_boot[(g * kmax + k - 1) * B + b]; NaN for an
 * empty group. */
void   orc_bootstrap(const double *tr, const int32_t *group, int64_t count, int n_groups, int kmax,
                     int B, uint64_t seed, double *F_boot);

/* Qudit brickwork (local dimension q, Haar U(q^2) gates; see fp_oracle.c):
 * the Haar sampler (out: 2 q^4 doubles), Tr(U^dagger V) of pair `pair` of
 * depth l densely (q^n <= 4096) or by variable elimination over q-ary wire
 * segments in min-degree order. */
void   orc_haar_uq(int q, uint64_t seed, uint64_t pair, int which, int gate, double *out);
int    orc_trace_qudit_dense(int q, int n, int l, uint64_t seed, uint64_t pair, int self_pair, double tr[2]);
int    orc_trace_qudit_ve(int q, int n, int l, uint64_t seed, uint64_t pair, int self_pair, double tr[2]);

#ifdef __cplusplus
}
#endif
#endif
