/*
 * fp_oracle.c -- plain FP64 CPU oracle (test infrastructure only; see
 * fp_oracle.h).  Nothing here is blocked, fused or reordered beyond what each
 * function's definition states; speed is not a goal.
 */
#define _GNU_SOURCE
#include "fp_oracle.h"

#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

static const double ORC_PI = 3.14159265358979323846;

/* ------------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11): ten rounds of two 64x64->128 multiplies with    */
/* the published multipliers and Weyl key increments.                        */
/* ------------------------------------------------------------------------ */
static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void orc_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(0xD2E7470EE14C6C93ULL, c0, &hi0, &lo0);
        mulhilo64(0xCA5A826395121157ULL, c2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B97F4A7C15ULL;
        k1 += 0xBB67AE8584CAA73BULL;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void draw(uint64_t seed, uint64_t c0, uint64_t c1, uint64_t pair, uint64_t stream,
                 uint64_t out[4])
{
    uint64_t ctr[4] = {c0, c1, pair, stream};
    uint64_t key[2] = {seed, 0};
    orc_philox4x64(ctr, key, out);
}

static double unit53(uint64_t x) { return (double)(x >> 11) * 0x1.0p-53; }

/* ------------------------------------------------------------------------ */
/* Haar U(4) (Methods, "Sampling U(d^2)"; the paper samples with a 16-phase */
/* decomposition, this oracle uses the equally Haar-distributed QR of a     */
/* complex Gaussian with R's diagonal made positive real, Mezzadri 2007).   */
/* Classical Gram-Schmidt on the columns produces exactly that Q.           */
/* ------------------------------------------------------------------------ */
void orc_haar_u4(uint64_t seed, uint64_t pair, int which, int gate, double out[32])
{
    cplx Z[16];
    for (int k = 0; k < 16; ++k) {
        uint64_t w[4];
        draw(seed, (uint64_t)(k / 2), (uint64_t)gate, pair, (uint64_t)which, w);
        uint64_t xa = (k % 2 == 0) ? w[0] : w[2];
        uint64_t xb = (k % 2 == 0) ? w[1] : w[3];
        double u1 = (double)((xa >> 11) + 1) * 0x1.0p-53;
        double u2 = (double)(xb >> 11) * 0x1.0p-53;
        double rad = sqrt(-2.0 * log(u1));
        Z[k] = (rad * cos(2.0 * ORC_PI * u2) + I * rad * sin(2.0 * ORC_PI * u2)) / sqrt(2.0);
    }
    cplx Q[16];
    for (int c = 0; c < 4; ++c) {
        cplx v[4];
        for (int r = 0; r < 4; ++r) v[r] = Z[4 * r + c];
        for (int j = 0; j < c; ++j) {
            cplx dot = 0;
            for (int r = 0; r < 4; ++r) dot += conj(Q[4 * r + j]) * Z[4 * r + c];
            for (int r = 0; r < 4; ++r) v[r] -= dot * Q[4 * r + j];
        }
        double nrm = 0;
        for (int r = 0; r < 4; ++r) nrm += creal(v[r] * conj(v[r]));
        nrm = sqrt(nrm);
        for (int r = 0; r < 4; ++r) Q[4 * r + c] = v[r] / nrm;
    }
    for (int k = 0; k < 16; ++k) { out[2 * k] = creal(Q[k]); out[2 * k + 1] = cimag(Q[k]); }
}

/* ------------------------------------------------------------------------ */
/* Ensembles (Fig. 2): (a) parallel/brickwork, (b) local, (c) HEA.          */
/* ------------------------------------------------------------------------ */
int orc_pair_depth(const orc_desc *d, uint64_t pair)
{
    uint64_t w[4];
    draw(d->seed, 0, 0, pair, 4, w);
    if (d->kind == ORC_LOCAL) {
        uint64_t choices = (uint64_t)((d->T_max - d->T_min) / d->T_step + 1);
        uint64_t idx = ((w[0] >> 32) * choices) >> 32;
        return d->T_min + (int)idx * d->T_step;
    }
    uint64_t choices = (uint64_t)(d->depth_max - d->depth_min + 1);
    uint64_t idx = ((w[0] >> 32) * choices) >> 32;
    return d->depth_min + (int)idx;
}

static void set_c(orc_op *op, int k, cplx v) { op->m[2 * k] = creal(v); op->m[2 * k + 1] = cimag(v); }

int orc_circuit(const orc_desc *d, uint64_t pair, int which, orc_op *ops, int max_ops)
{
    int n = d->n, depth = orc_pair_depth(d, pair), cnt = 0;
    int w = d->self_pair ? 0 : which;
    if (d->kind == ORC_PARALLEL) {
        int g = 0;
        for (int t = 1; t <= depth; ++t)
            for (int b = (t - 1) % 2; b <= n - 2; b += 2) {
                if (cnt >= max_ops) return -1;
                ops[cnt].kind = ORC_OP_GATE2; ops[cnt].q = b;
                orc_haar_u4(d->seed, pair, w, g, ops[cnt].m);
                ++cnt; ++g;
            }
    } else if (d->kind == ORC_LOCAL) {
        for (int g = 0; g < depth; ++g) {
            uint64_t x[4];
            if (cnt >= max_ops) return -1;
            draw(d->seed, 0, (uint64_t)g, pair, (uint64_t)(2 + w), x);
            ops[cnt].kind = ORC_OP_GATE2;
            ops[cnt].q = (int)(((x[0] >> 32) * (uint64_t)(n - 1)) >> 32);
            orc_haar_u4(d->seed, pair, w, g, ops[cnt].m);
            ++cnt;
        }
    } else if (d->kind == ORC_HEA) {
        for (int t = 0; t < depth; ++t) {
            for (int q = 0; q < n; ++q) {
                uint64_t x[4];
                if (cnt >= max_ops) return -1;
                draw(d->seed, (uint64_t)t, (uint64_t)q, pair, (uint64_t)w, x);
                double th = 2.0 * ORC_PI * unit53(x[0]);
                double ph = 2.0 * ORC_PI * unit53(x[1]);
                double c = cos(th / 2), s = sin(th / 2);
                cplx em = cexp(-I * ph / 2), ep = cexp(I * ph / 2);
                /* RY(th) RZ(ph): RZ acts first */
                orc_op *op = &ops[cnt++];
                memset(op, 0, sizeof *op);
                op->kind = ORC_OP_GATE1; op->q = q;
                set_c(op, 0, c * em);  set_c(op, 1, -s * ep);
                set_c(op, 2, s * em);  set_c(op, 3, c * ep);
            }
            for (int b = 0; b <= n - 2; ++b) {
                if (cnt >= max_ops) return -1;
                orc_op *op = &ops[cnt++];
                memset(op, 0, sizeof *op);
                op->kind = ORC_OP_DIAG2; op->q = b;
                set_c(op, 0, 1); set_c(op, 1, 1); set_c(op, 2, 1); set_c(op, 3, -1);
            }
        }
    } else if (d->kind == ORC_HEA_CNOT || d->kind == ORC_HEA_CZ) {
        /* the wall of RY(pi/4) = cos(pi/8) I - i sin(pi/8) Y */
        for (int q = 0; q < n; ++q) {
            if (cnt >= max_ops) return -1;
            orc_op *op = &ops[cnt++];
            memset(op, 0, sizeof *op);
            op->kind = ORC_OP_GATE1; op->q = q;
            double c = cos(ORC_PI / 8), s = sin(ORC_PI / 8);
            set_c(op, 0, c);  set_c(op, 1, -s);
            set_c(op, 2, s);  set_c(op, 3, c);
        }
        const cplx pauli[3][4] = {{0, 1, 1, 0}, {0, -I, I, 0}, {1, 0, 0, -1}};
        for (int t = 0; t < depth; ++t) {
            for (int q = 0; q < n; ++q) {
                uint64_t x[4];
                if (cnt >= max_ops) return -1;
                draw(d->seed, (uint64_t)t, (uint64_t)q, pair, (uint64_t)w, x);
                double th = 2.0 * ORC_PI * unit53(x[0]);
                int axis = (int)(((x[1] >> 32) * 3u) >> 32);
                orc_op *op = &ops[cnt++];
                memset(op, 0, sizeof *op);
                op->kind = ORC_OP_GATE1; op->q = q;
                /* exp(-i theta P / 2) = cos(theta/2) I - i sin(theta/2) P, as P^2 = I */
                for (int k = 0; k < 4; ++k) {
                    cplx id = (k == 0 || k == 3) ? 1 : 0;
                    set_c(op, k, cos(th / 2) * id - I * sin(th / 2) * pauli[axis][k]);
                }
            }
            for (int par = 0; par < 2; ++par)
                for (int b = par; b <= n - 2; b += 2) {
                    if (cnt >= max_ops) return -1;
                    orc_op *op = &ops[cnt++];
                    memset(op, 0, sizeof *op);
                    op->q = b;
                    if (d->kind == ORC_HEA_CZ) {
                        op->kind = ORC_OP_DIAG2;
                        set_c(op, 0, 1); set_c(op, 1, 1); set_c(op, 2, 1); set_c(op, 3, -1);
                    } else {
                        /* CNOT, control b (the more significant index bit), target b+1:
                           |c t> -> |c, t xor c> */
                        op->kind = ORC_OP_GATE2;
                        for (int ct = 0; ct < 4; ++ct) {
                            int c = ct >> 1, tt = ct & 1;
                            set_c(op, 4 * ((c << 1) | (tt ^ c)) + ct, 1);
                        }
                    }
                }
        }
    } else {
        return -2;
    }
    return cnt;
}

/* ------------------------------------------------------------------------ */
/* Dense trace: Tr(U^dagger V) = sum_ij conj(U_ij) V_ij (Sec. "Frame        */
/* potential": the integrand of F^(k)), with U and V built by applying each */
/* gate to the identity.  Qubit 0 is the most significant index bit.        */
/* ------------------------------------------------------------------------ */
static void dense_apply(int n, cplx *M, const orc_op *op)
{
    size_t D = (size_t)1 << n;
    const cplx *g = (const cplx *)op->m;
    if (op->kind == ORC_OP_GATE1) {
        size_t bq = (size_t)1 << (n - 1 - op->q);
        for (size_t col = 0; col < D; ++col)
            for (size_t r = 0; r < D; ++r) {
                if (r & bq) continue;
                cplx a0 = M[r * D + col], a1 = M[(r | bq) * D + col];
                M[r * D + col] = g[0] * a0 + g[1] * a1;
                M[(r | bq) * D + col] = g[2] * a0 + g[3] * a1;
            }
        return;
    }
    size_t b0 = (size_t)1 << (n - 1 - op->q);       /* qubit q   */
    size_t b1 = (size_t)1 << (n - 2 - op->q);       /* qubit q+1 */
    for (size_t col = 0; col < D; ++col)
        for (size_t r = 0; r < D; ++r) {
            if (r & (b0 | b1)) continue;
            size_t idx[4] = {r, r | b1, r | b0, r | b0 | b1};   /* (a_q a_q+1) = 00,01,10,11 */
            cplx a[4], o[4];
            for (int k = 0; k < 4; ++k) a[k] = M[idx[k] * D + col];
            for (int i = 0; i < 4; ++i) {
                if (op->kind == ORC_OP_DIAG2) { o[i] = g[i] * a[i]; continue; }
                o[i] = 0;
                for (int j = 0; j < 4; ++j) o[i] += g[4 * i + j] * a[j];
            }
            for (int k = 0; k < 4; ++k) M[idx[k] * D + col] = o[k];
        }
}

int orc_trace_dense(int n, int nU, const orc_op *U, int nV, const orc_op *V, double tr[2])
{
    if (n < 1 || n > 12) return -1;
    size_t D = (size_t)1 << n;
    cplx *MU = calloc(D * D, sizeof(cplx)), *MV = calloc(D * D, sizeof(cplx));
    if (!MU || !MV) { free(MU); free(MV); return -3; }
    for (size_t i = 0; i < D; ++i) { MU[i * D + i] = 1; MV[i * D + i] = 1; }
    for (int g = 0; g < nU; ++g) dense_apply(n, MU, &U[g]);
    for (int g = 0; g < nV; ++g) dense_apply(n, MV, &V[g]);
    cplx s = 0;
    for (size_t i = 0; i < D * D; ++i) s += conj(MU[i]) * MV[i];
    free(MU); free(MV);
    tr[0] = creal(s); tr[1] = cimag(s);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Variable-elimination trace (Sec. "Algorithm description": the trace is  */
/* the closed tensor network of the circuit with each qubit's output wire  */
/* joined to its input).  Every qubit's wire is cut into segments by the   */
/* non-diagonal operators on it; each segment is a binary variable; each   */
/* operator is a factor over the segments it touches (a diagonal operator  */
/* leaves its wire segments whole).  Tr = sum over all variables of the    */
/* product of all factors, summed out one variable at a time from qubit    */
/* n-1 down to qubit 0 (the space direction of the paper's contraction).   */
/* No gate is merged or split.                                              */
/* ------------------------------------------------------------------------ */
typedef struct { int nv; int *vars; cplx *t; } factor;

static cplx op_entry(const orc_op *op, const int *val)
{
    /* val: for GATE2 (out_q, out_q1, in_q, in_q1); GATE1 (out, in); DIAG2 (y_q, y_q1) */
    const cplx *g = (const cplx *)op->m;
    if (op->kind == ORC_OP_GATE2) return g[(val[0] * 2 + val[1]) * 4 + (val[2] * 2 + val[3])];
    if (op->kind == ORC_OP_GATE1) return g[val[0] * 2 + val[1]];
    return g[val[0] * 2 + val[1]];
}

static int build_factor(const orc_op *op, const int *slot_var, int nslots, factor *f)
{
    int dv[4], nd = 0, map[4];
    for (int s = 0; s < nslots; ++s) {
        int k;
        for (k = 0; k < nd; ++k) if (dv[k] == slot_var[s]) break;
        if (k == nd) dv[nd++] = slot_var[s];
        map[s] = k;
    }
    f->nv = nd;
    f->vars = malloc(sizeof(int) * (nd > 0 ? nd : 1));
    f->t = malloc(sizeof(cplx) << nd);
    if (!f->vars || !f->t) return -3;
    memcpy(f->vars, dv, sizeof(int) * nd);
    for (int a = 0; a < (1 << nd); ++a) {
        int val[4];
        for (int s = 0; s < nslots; ++s) val[s] = (a >> map[s]) & 1;
        f->t[a] = op_entry(op, val);
    }
    return 0;
}

static void dagger_op(const orc_op *in, orc_op *out)
{
    *out = *in;
    const cplx *g = (const cplx *)in->m;
    cplx *h = (cplx *)out->m;
    if (in->kind == ORC_OP_GATE2)
        for (int i = 0; i < 4; ++i) for (int j = 0; j < 4; ++j) h[4 * i + j] = conj(g[4 * j + i]);
    else if (in->kind == ORC_OP_GATE1)
        for (int i = 0; i < 2; ++i) for (int j = 0; j < 2; ++j) h[2 * i + j] = conj(g[2 * j + i]);
    else
        for (int i = 0; i < 4; ++i) h[i] = conj(g[i]);
}

static int trace_ve_order(int n, int nU, const orc_op *U, int nV, const orc_op *V, int greedy, double tr[2]);

int orc_trace_ve(int n, int nU, const orc_op *U, int nV, const orc_op *V, double tr[2])
{
    return trace_ve_order(n, nU, U, nV, V, 0, tr);
}

/* The same variable elimination with a min-degree order: every step sums out
 * the variable whose factors together span the fewest distinct variables
 * (ties: the lowest index).  The result is the same trace; only the order of
 * the sums, and so the sizes of the intermediate factors, differ -- local
 * circuits with many gates stay within reach of a CPU this way. */
int orc_trace_ve_greedy(int n, int nU, const orc_op *U, int nV, const orc_op *V, double tr[2])
{
    return trace_ve_order(n, nU, U, nV, V, 1, tr);
}

static int trace_ve_order(int n, int nU, const orc_op *U, int nV, const orc_op *V, int greedy, double tr[2])
{
    int T = nU + nV, rc = 0;
    orc_op *seq = malloc(sizeof(orc_op) * (T > 0 ? T : 1));
    if (!seq) return -3;
    /* time order of U^dagger V: V's gates first to last, then U's last to first, daggered */
    for (int g = 0; g < nV; ++g) seq[g] = V[g];
    for (int g = 0; g < nU; ++g) dagger_op(&U[nU - 1 - g], &seq[nV + g]);

    /* segments: s_q = number of non-diagonal operators on qubit q */
    int *s = calloc(n, sizeof(int)), *base = calloc(n + 1, sizeof(int));
    int *pos = malloc(sizeof(int) * (T > 0 ? T : 1) * 2);   /* per op, per touched qubit: index among q's splitters */
    for (int t = 0; t < T; ++t) {
        const orc_op *op = &seq[t];
        int qs[2] = {op->q, op->q + 1}, nq = op->kind == ORC_OP_GATE1 ? 1 : 2;
        for (int i = 0; i < nq; ++i) {
            if (op->kind == ORC_OP_DIAG2) pos[2 * t + i] = s[qs[i]] - 1;  /* last splitter before t (may be -1) */
            else pos[2 * t + i] = s[qs[i]]++;
        }
    }
    for (int q = 0; q < n; ++q) base[q + 1] = base[q] + (s[q] > 0 ? s[q] : 1);
    int nvars = base[n];

    int nf = 0, capf = T + 4;
    factor *fs = calloc(capf, sizeof(factor));
    for (int t = 0; t < T && rc == 0; ++t) {
        const orc_op *op = &seq[t];
        int qs[2] = {op->q, op->q + 1}, seg_in[2], seg_out[2], nq = op->kind == ORC_OP_GATE1 ? 1 : 2;
        for (int i = 0; i < nq; ++i) {
            int q = qs[i], sq = s[q] > 0 ? s[q] : 1, j = pos[2 * t + i];
            if (op->kind == ORC_OP_DIAG2) {
                int cur = j >= 0 ? j : sq - 1;       /* wraps to the segment after the last splitter */
                seg_in[i] = seg_out[i] = base[q] + cur;
            } else {
                seg_out[i] = base[q] + j;
                seg_in[i] = base[q] + (j - 1 + sq) % sq;
            }
        }
        int slot[4];
        if (op->kind == ORC_OP_GATE2) {
            slot[0] = seg_out[0]; slot[1] = seg_out[1]; slot[2] = seg_in[0]; slot[3] = seg_in[1];
            rc = build_factor(op, slot, 4, &fs[nf++]);
        } else if (op->kind == ORC_OP_GATE1) {
            slot[0] = seg_out[0]; slot[1] = seg_in[0];
            rc = build_factor(op, slot, 2, &fs[nf++]);
        } else {
            slot[0] = seg_out[0]; slot[1] = seg_out[1];
            rc = build_factor(op, slot, 2, &fs[nf++]);
        }
    }

    cplx scalar = 1;
    int *uvars = malloc(sizeof(int) * (nvars + 8));
    int *sel = malloc(sizeof(int) * (nf + 1));
    int **posf = malloc(sizeof(int *) * (nf + 1));
    /* elimination order: qubits n-1 down to 0, each qubit's segments in order;
     * or min-degree (greedy) */
    int *order = malloc(sizeof(int) * (nvars > 0 ? nvars : 1));
    char *gone = calloc(nvars > 0 ? nvars : 1, 1);
    for (int q = n - 1, k = 0; q >= 0; --q)
        for (int v = base[q]; v < base[q + 1]; ++v) order[k++] = v;
    for (int step = 0; step < nvars && rc == 0; ++step) {
        int v = order[step];
        if (greedy) {
            int best = -1, best_w = 1 << 30;
            for (int c = 0; c < nvars; ++c) {
                if (gone[c]) continue;
                int nu = 0;
                for (int f = 0; f < nf; ++f) {
                    if (!fs[f].t) continue;
                    int has = 0;
                    for (int k = 0; k < fs[f].nv; ++k) has |= fs[f].vars[k] == c;
                    if (!has) continue;
                    for (int k = 0; k < fs[f].nv; ++k) {
                        int u;
                        for (u = 0; u < nu; ++u) if (uvars[u] == fs[f].vars[k]) break;
                        if (u == nu) uvars[nu++] = fs[f].vars[k];
                    }
                }
                if (nu < best_w) { best_w = nu; best = c; }
            }
            v = best;
        }
        gone[v] = 1;
        {
            int ns = 0;
            for (int f = 0; f < nf; ++f) {
                if (!fs[f].t) continue;
                for (int k = 0; k < fs[f].nv; ++k) if (fs[f].vars[k] == v) { sel[ns++] = f; break; }
            }
            if (ns == 0) { scalar *= 2; continue; }          /* a free wire loop: Tr(I_2) */
            int nu = 0;
            uvars[nu++] = v;
            for (int i = 0; i < ns; ++i) {
                factor *f = &fs[sel[i]];
                for (int k = 0; k < f->nv; ++k) {
                    int u;
                    for (u = 0; u < nu; ++u) if (uvars[u] == f->vars[k]) break;
                    if (u == nu) uvars[nu++] = f->vars[k];
                }
            }
            for (int i = 0; i < ns; ++i) {
                factor *f = &fs[sel[i]];
                posf[i] = malloc(sizeof(int) * (f->nv > 0 ? f->nv : 1));
                for (int k = 0; k < f->nv; ++k)
                    for (int u = 0; u < nu; ++u) if (uvars[u] == f->vars[k]) posf[i][k] = u;
            }
            int nr = nu - 1;
            cplx *res = malloc(sizeof(cplx) << nr);
            if (!res) { rc = -3; break; }
            for (size_t r = 0; r < ((size_t)1 << nr); ++r) {
                cplx acc = 0;
                for (size_t x = 0; x < 2; ++x) {
                    size_t u = (r << 1) | x;
                    cplx p = 1;
                    for (int i = 0; i < ns; ++i) {
                        factor *f = &fs[sel[i]];
                        size_t idx = 0;
                        for (int k = 0; k < f->nv; ++k) idx |= ((u >> posf[i][k]) & 1) << k;
                        p *= f->t[idx];
                    }
                    acc += p;
                }
                res[r] = acc;
            }
            for (int i = 0; i < ns; ++i) {
                free(posf[i]);
                free(fs[sel[i]].t); fs[sel[i]].t = NULL;
                free(fs[sel[i]].vars); fs[sel[i]].vars = NULL;
            }
            if (nf >= capf) {
                capf *= 2;
                fs = realloc(fs, sizeof(factor) * capf);
            }
            factor *nfac = &fs[nf++];
            nfac->nv = nr;
            nfac->vars = malloc(sizeof(int) * (nr > 0 ? nr : 1));
            memcpy(nfac->vars, uvars + 1, sizeof(int) * nr);
            nfac->t = res;
        }
    }
    free(order); free(gone);
    for (int f = 0; f < nf; ++f) {
        if (fs[f].t) {
            if (rc == 0) scalar *= fs[f].t[0];   /* every variable is summed: scalars remain */
            free(fs[f].t); free(fs[f].vars);
        }
    }
    free(fs); free(uvars); free(sel); free(posf); free(s); free(base); free(pos); free(seq);
    tr[0] = creal(scalar); tr[1] = cimag(scalar);
    return rc;
}

/* ------------------------------------------------------------------------ */
int orc_trace_pair(const orc_desc *d, uint64_t pair, int method, double tr[2])
{
    int depth = orc_pair_depth(d, pair);
    int cap;
    if (d->kind == ORC_PARALLEL) cap = depth * d->n;
    else if (d->kind == ORC_LOCAL) cap = depth;
    else if (d->kind == ORC_HEA) cap = depth * 2 * d->n;
    else cap = (depth + 1) * 3 * d->n;
    cap += 4;
    orc_op *U = malloc(sizeof(orc_op) * cap), *V = malloc(sizeof(orc_op) * cap);
    if (!U || !V) { free(U); free(V); return -3; }
    int nU = orc_circuit(d, pair, 0, U, cap), nV = orc_circuit(d, pair, 1, V, cap), rc;
    if (nU < 0 || nV < 0) rc = -2;
    else if (method == 0 || (method < 0 && d->n <= 10)) rc = orc_trace_dense(d->n, nU, U, nV, V, tr);
    else if (method == 2) rc = orc_trace_ve_greedy(d->n, nU, U, nV, V, tr);
    else rc = orc_trace_ve(d->n, nU, U, nV, V, tr);
    free(U); free(V);
    return rc;
}

typedef struct {
    const orc_desc *d; uint64_t first, count; int method, stride, tid; double *tr; int rc;
} batch_job;

static void *batch_worker(void *arg)
{
    batch_job *j = arg;
    for (uint64_t i = (uint64_t)j->tid; i < j->count; i += (uint64_t)j->stride) {
        int rc = orc_trace_pair(j->d, j->first + i, j->method, &j->tr[2 * i]);
        if (rc) j->rc = rc;
    }
    return NULL;
}

int orc_trace_batch(const orc_desc *d, uint64_t first, uint64_t count, int method,
                    int nthreads, double *tr)
{
    if (nthreads < 1) nthreads = 1;
    pthread_t *th = malloc(sizeof(pthread_t) * nthreads);
    batch_job *jobs = malloc(sizeof(batch_job) * nthreads);
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = (batch_job){d, first, count, method, nthreads, t, tr, 0};
        pthread_create(&th[t], NULL, batch_worker, &jobs[t]);
    }
    int rc = 0;
    for (int t = 0; t < nthreads; ++t) {
        pthread_join(th[t], NULL);
        if (jobs[t].rc) rc = jobs[t].rc;
    }
    free(th); free(jobs);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Monte Carlo estimate F^(k) ~= mean of |Tr|^{2k} (Sec. "Algorithm         */
/* description") with its standard error s/sqrt(N), s the N-1 sample        */
/* deviation (the paper's error bars are standard errors, Fig. 4).          */
/* Two-pass: mean first, then squared deviations; Neumaier sums.            */
/* ------------------------------------------------------------------------ */
static void neumaier_add(double *sum, double *comp, double x)
{
    double t = *sum + x;
    if (fabs(*sum) >= fabs(x)) *comp += (*sum - t) + x;
    else *comp += (x - t) + *sum;
    *sum = t;
}

void orc_moments(const double *tr, int64_t N, int kmax, double *F, double *se)
{
    for (int k = 1; k <= kmax; ++k) {
        double s = 0, c = 0;
        for (int64_t i = 0; i < N; ++i) {
            double a2 = tr[2 * i] * tr[2 * i] + tr[2 * i + 1] * tr[2 * i + 1];
            neumaier_add(&s, &c, pow(a2, k));
        }
        double mean = (s + c) / (double)N;
        double v = 0, vc = 0;
        for (int64_t i = 0; i < N; ++i) {
            double a2 = tr[2 * i] * tr[2 * i] + tr[2 * i + 1] * tr[2 * i + 1];
            double dlt = pow(a2, k) - mean;
            neumaier_add(&v, &vc, dlt * dlt);
        }
        F[k - 1] = mean;
        se[k - 1] = N > 1 ? sqrt((v + vc) / (double)(N - 1) / (double)N) : 0.0;
    }
}

/* ------------------------------------------------------------------------ */
/* Control-variate estimate of F^(2) = E f, f = |Tr|^4 (the paper's estimand, */
/* Sec. "Frame potential"; the control variate itself is not in the paper):  */
/* with a predictor g evaluated on M surrogate pairs and on the N correction  */
/* pairs (where f is also known),                                            */
/*     F = mean_M g + mean_N (f - g),                                        */
/*     stderr^2 = Var_M(g) / M + Var_N(f - g) / N,                           */
/* sample variances with N - 1 (M - 1); the plain estimate mean_N f and its   */
/* standard error beside it.  Two passes (mean, then centred squares), both   */
/* Neumaier-compensated.                                                     */
/* out: F, stderr, F_plain, stderr_plain, Var f, Var (f - g), Var g.         */
/* ------------------------------------------------------------------------ */
static void mean_var(const double *a, const double *b, int64_t n, double *mean, double *var)
{
    /* the values are a[i] - b[i] (b may be NULL) */
    double s = 0, c = 0;
    for (int64_t i = 0; i < n; ++i) neumaier_add(&s, &c, a[i] - (b ? b[i] : 0.0));
    *mean = (s + c) / (double)n;
    double v = 0, vc = 0;
    for (int64_t i = 0; i < n; ++i) {
        double d = a[i] - (b ? b[i] : 0.0) - *mean;
        neumaier_add(&v, &vc, d * d);
    }
    *var = n > 1 ? (v + vc) / (double)(n - 1) : 0.0;
}

void orc_cv_estimate(const double *g_corr, const double *f_corr, int64_t N, const double *g_sur, int64_t M,
                     double *out)
{
    double mfg, vfg, mf, vf, mg, vg;
    mean_var(f_corr, g_corr, N, &mfg, &vfg);
    mean_var(f_corr, NULL, N, &mf, &vf);
    mean_var(g_sur, NULL, M, &mg, &vg);
    out[0] = mg + mfg;
    out[1] = sqrt(vg / (double)M + vfg / (double)N);
    out[2] = mf;
    out[3] = sqrt(vf / (double)N);
    out[4] = vf;
    out[5] = vfg;
    out[6] = vg;
}

/* ------------------------------------------------------------------------ */
/* Bootstrap of the frame-potential estimator (Supplementary, "Bootstrapping */
/* for uncertainty quantification"): a resample draws N samples with         */
/* replacement from the N stored traces and evaluates F^(k) on them; the     */
/* paper uses 300 resamples.  Written as the definition: one draw at a time. */
/* ------------------------------------------------------------------------ */
void orc_bootstrap(const double *tr, const int32_t *group, int64_t count, int n_groups, int kmax,
                   int B, uint64_t seed, double *F_boot)
{
    for (int g = 0; g < n_groups; ++g) {
        int64_t Ng = 0;
        for (int64_t i = 0; i < count; ++i) Ng += group[i] == g;
        int64_t *members = malloc((size_t)(Ng > 0 ? Ng : 1) * sizeof(int64_t));
        int64_t m = 0;
        for (int64_t i = 0; i < count; ++i)
            if (group[i] == g) members[m++] = i;
        for (int b = 0; b < B; ++b) {
            for (int k = 1; k <= kmax; ++k) F_boot[((int64_t)g * kmax + k - 1) * B + b] = NAN;
            if (Ng == 0) continue;
            double *s = calloc((size_t)kmax, sizeof(double)), *c = calloc((size_t)kmax, sizeof(double));
            for (int64_t i = 0; i < Ng; ++i) {
                const uint64_t ctr[4] = {(uint64_t)b, (uint64_t)(i / 4), (uint64_t)g, 5};
                const uint64_t key[2] = {seed, 0};
                uint64_t x[4];
                orc_philox4x64(ctr, key, x);
                const uint64_t pos = ((x[i % 4] >> 32) * (uint64_t)Ng) >> 32;
                const int64_t j = members[pos];
                const double a2 = tr[2 * j] * tr[2 * j] + tr[2 * j + 1] * tr[2 * j + 1];
                double p = 1.0;
                for (int k = 1; k <= kmax; ++k) {
                    p *= a2;
                    neumaier_add(&s[k - 1], &c[k - 1], p);
                }
            }
            for (int k = 1; k <= kmax; ++k)
                F_boot[((int64_t)g * kmax + k - 1) * B + b] = (s[k - 1] + c[k - 1]) / (double)Ng;
            free(s);
            free(c);
        }
        free(members);
    }
}

/* ------------------------------------------------------------------------ */
/* Exact ensemble F^(k), k = 2 or 3, of brickwork circuits of qudits of      */
/* local dimension q (Sec. "Frame potential": the paper's qudit remark): the */
/* same statistical-mechanics model as orc_weingarten_f2_brickwork with the  */
/* pairings running over the permutation group S_k.  Averaging a Haar U(d)   */
/* gate, d = q^2, over k copies of U and k of U^* gives                      */
/*   sum_{sigma, tau in S_k} Wg(sigma^-1 tau, d) |sigma>><<tau|              */
/* with the Weingarten function of U(d) (Collins 2003):                       */
/*   k = 2: Wg(e) = 1/(d^2-1), Wg(2-cycle) = -1/(d(d^2-1));                  */
/*   k = 3: Wg(e) = (d^2-2)/(d(d^2-1)(d^2-4)), Wg(2-cycle) =                 */
/*          -1/((d^2-1)(d^2-4)), Wg(3-cycle) = 2/(d(d^2-1)(d^2-4)).          */
/* Along a qubit wire, the output pairing sigma_a of a gate meets the input  */
/* pairing tau_b of the next gate on the wire: q^{#cycles(sigma_a^-1 tau_b)};*/
/* a qudit touched by no gate gives q^{2k}.  Summed with the                 */
/* same explicit transfer matrix over bonds as the k = 2 routine.            */
/* ------------------------------------------------------------------------ */
static int perms_of(int k, int P[6][3])
{
    int np = 0;
    for (int a = 0; a < k; ++a)
        for (int b = 0; b < k; ++b)
            for (int c = 0; c < k; ++c) {
                int v[3] = {a, b, c};
                int ok = 1;
                for (int i = 0; i < k; ++i)
                    for (int j = i + 1; j < k; ++j) if (v[i] == v[j]) ok = 0;
                if (k < 3 && c != 0) ok = 0;
                if (k < 2 && b != 0) ok = 0;
                if (!ok) continue;
                for (int i = 0; i < 3; ++i) P[np][i] = v[i];
                ++np;
            }
    return np;
}

static int cycles_of(const int *a, const int *b, int k)   /* #cycles of a^-1 b */
{
    int ainv[3], seen[3] = {0, 0, 0}, c = 0;
    for (int i = 0; i < k; ++i) ainv[a[i]] = i;
    for (int i = 0; i < k; ++i) {
        if (seen[i]) continue;
        ++c;
        for (int j = i; !seen[j]; j = ainv[b[j]]) seen[j] = 1;
    }
    return c;
}

double orc_weingarten_fkq_brickwork(int n, int l, int k, int q)
{
    if (n < 2 || l < 1 || k < 2 || k > 3 || q < 2) return NAN;
    const double d = (double)q * q;
    int Pm[6][3];
    const int np = perms_of(k, Pm), sg = np * np;   /* (sigma, tau) states per gate */
    double wg_by_cycles[4] = {0, 0, 0, 0};
    if (k == 2) {
        wg_by_cycles[2] = 1.0 / (d * d - 1);
        wg_by_cycles[1] = -1.0 / (d * (d * d - 1));
    } else {
        wg_by_cycles[3] = (d * d - 2) / (d * (d * d - 1) * (d * d - 4));
        wg_by_cycles[2] = -1.0 / ((d * d - 1) * (d * d - 4));
        wg_by_cycles[1] = 2.0 / (d * (d * d - 1) * (d * d - 4));
    }
    double wg[36], link[6][6];
    for (int s = 0; s < np; ++s)
        for (int t = 0; t < np; ++t) {
            int c = cycles_of(Pm[s], Pm[t], k);
            wg[s * np + t] = wg_by_cycles[c];
            link[s][t] = pow((double)q, c);
        }
    const double idle = pow((double)q, 2 * k);
    int P = (l == 1) ? 1 : 2 * (l - 1), nb = n - 1;
    int *g_of_bond = calloc(nb, sizeof(int));
    int **times = calloc(nb, sizeof(int *));
    for (int b = 0; b < nb; ++b) {
        times[b] = malloc(sizeof(int) * P);
        for (int t = 0; t < P; ++t) {
            int par = (l == 1) ? 0 : (t + 1) % 2;
            if (b % 2 == par) times[b][g_of_bond[b]++] = t;
        }
    }
    int gmax = 0;
    for (int b = 0; b < nb; ++b) if (g_of_bond[b] > gmax) gmax = g_of_bond[b];
    size_t S = 1;
    for (int j = 0; j < gmax; ++j) S *= (size_t)sg;
    double *v = malloc(sizeof(double) * S), *w = malloc(sizeof(double) * S);
    /* configuration c of a bond: digit j (base sg) = sigma_j * np + tau_j of gate j */
#define DIGIT(c, j) ((int)(((c) / pw[j]) % (size_t)sg))
    size_t pw[16];
    pw[0] = 1;
    for (int j = 1; j < 16; ++j) pw[j] = pw[j - 1] * (size_t)sg;
    {   /* qubit 0: links among bond-0 gates */
        int g0 = g_of_bond[0];
        for (size_t c = 0; c < pw[g0]; ++c) {
            double p = g0 == 0 ? idle : 1.0;
            for (int j = 0; j < g0; ++j) {
                int dj = DIGIT(c, j), dn = DIGIT(c, (j + 1) % g0);
                p *= wg[dj] * link[dj / np][dn % np];
            }
            v[c] = p;
        }
    }
    for (int b = 1; b < nb; ++b) {
        int ga = g_of_bond[b - 1], gb = g_of_bond[b], tot = ga + gb;
        int *who = malloc(sizeof(int) * (tot > 0 ? tot : 1)), *idx = malloc(sizeof(int) * (tot > 0 ? tot : 1));
        int ia = 0, ib = 0, kk = 0;
        while (ia < ga || ib < gb) {
            if (ib >= gb || (ia < ga && times[b - 1][ia] < times[b][ib])) { who[kk] = 0; idx[kk++] = ia++; }
            else { who[kk] = 1; idx[kk++] = ib++; }
        }
        for (size_t cb = 0; cb < pw[gb]; ++cb) {
            double gw = 1;
            for (int j = 0; j < gb; ++j) gw *= wg[DIGIT(cb, j)];
            double acc = 0;
            for (size_t ca = 0; ca < pw[ga]; ++ca) {
                double p = v[ca];
                if (tot == 0) p *= idle;
                for (int j = 0; j < tot; ++j) {
                    int jn = (j + 1) % tot;
                    int dj = who[j] ? DIGIT(cb, idx[j]) : DIGIT(ca, idx[j]);
                    int dn = who[jn] ? DIGIT(cb, idx[jn]) : DIGIT(ca, idx[jn]);
                    p *= link[dj / np][dn % np];
                }
                acc += p;
            }
            w[cb] = acc * gw;
        }
        double *tmp = v; v = w; w = tmp;
        free(who); free(idx);
    }
    double result = 0;
    {   /* qubit n-1: links among bond n-2 gates */
        int g = g_of_bond[nb - 1];
        for (size_t c = 0; c < pw[g]; ++c) {
            double p = v[c];
            if (g == 0) p *= idle;
            for (int j = 0; j < g; ++j) {
                int dj = DIGIT(c, j), dn = DIGIT(c, (j + 1) % g);
                p *= link[dj / np][dn % np];
            }
            result += p;
        }
    }
#undef DIGIT
    for (int b = 0; b < nb; ++b) free(times[b]);
    free(times); free(g_of_bond); free(v); free(w);
    return result;
}

double orc_weingarten_fk_brickwork(int n, int l, int k) { return orc_weingarten_fkq_brickwork(n, l, k, 2); }

/* ------------------------------------------------------------------------ */
/* Exact ensemble F^(2) of brickwork circuits (the statistical-mechanics    */
/* model behind Eq. theory_eq).  After averaging each Haar U(4) gate g of  */
/* the cyclic U^dagger V circuit over the Haar measure, g becomes           */
/*   sum_{sigma_g, tau_g in S_2} Wg(sigma_g tau_g^-1) |sigma_g>><<tau_g|     */
/* with Wg(e) = 1/(d^2-1), Wg(swap) = -1/(d(d^2-1)), d = 4; along each      */
/* qubit wire, the output pairing sigma_a of a gate meets the input pairing */
/* tau_b of the next gate on that wire and gives q^{#cycles(sigma_a^-1      */
/* tau_b)} = 4 (equal) or 2 (different); a qubit touched by no gate gives   */
/* q^{2k} = 16.  U^dagger V is, after the middle and cyclic merges of       */
/* independent Haar gates, a cyclic brickwork of 2l-2 layers (l >= 2), or   */
/* one layer (l = 1).  The sum over all pairings is evaluated exactly with  */
/* a transfer matrix over the bonds.                                        */
/* ------------------------------------------------------------------------ */
double orc_weingarten_f2_brickwork(int n, int l)
{
    if (n < 2 || l < 1) return NAN;
    int P = (l == 1) ? 1 : 2 * (l - 1);             /* cyclic positions */
    /* position tau holds bonds of parity (tau+1) mod 2 for l >= 2; even bonds for l = 1 */
    int nb = n - 1;
    int *g_of_bond = calloc(nb, sizeof(int));
    int **times = calloc(nb, sizeof(int *));
    for (int b = 0; b < nb; ++b) {
        times[b] = malloc(sizeof(int) * P);
        for (int t = 0; t < P; ++t) {
            int par = (l == 1) ? 0 : (t + 1) % 2;
            if (b % 2 == par) times[b][g_of_bond[b]++] = t;
        }
    }
    const double W_same = 1.0 / 15.0, W_diff = -1.0 / 60.0;
    /* link weight between output pairing s_a and input pairing t_b */
#define LINK(sa, tb) ((sa) == (tb) ? 4.0 : 2.0)

    /* the links on qubit q: consecutive gates in cyclic time order among bonds q-1 and q.
       Encode a gate as (bond, index within bond). */
    double result;
    /* v over configurations of bond b: 2 bits per gate: bit 2j = sigma, bit 2j+1 = tau */
    int gmax = 0;
    for (int b = 0; b < nb; ++b) if (g_of_bond[b] > gmax) gmax = g_of_bond[b];
    size_t S = (size_t)1 << (2 * gmax);
    double *v = malloc(sizeof(double) * S), *w = malloc(sizeof(double) * S);

    /* qubit 0: links among bond-0 gates only */
    {
        int g0 = g_of_bond[0];
        size_t S0 = (size_t)1 << (2 * g0);
        for (size_t c = 0; c < S0; ++c) {
            double p = 1;
            for (int j = 0; j < g0; ++j) {
                int sg = (c >> (2 * j)) & 1, tg = (c >> (2 * j + 1)) & 1;
                p *= (sg == tg) ? W_same : W_diff;
                int nx = (j + 1) % g0;              /* next gate on qubit 0, cyclically */
                int tn = (c >> (2 * nx + 1)) & 1;
                p *= LINK(sg, tn);
            }
            if (g0 == 0) p = 16.0;
            v[c] = p;
        }
    }
    for (int b = 1; b < nb; ++b) {
        /* qubit b sits between bond b-1 and bond b: merge the two time lists */
        int ga = g_of_bond[b - 1], gb = g_of_bond[b];
        int tot = ga + gb;
        int *who = malloc(sizeof(int) * (tot > 0 ? tot : 1)), *idx = malloc(sizeof(int) * (tot > 0 ? tot : 1));
        int ia = 0, ib = 0, k = 0;
        while (ia < ga || ib < gb) {
            if (ib >= gb || (ia < ga && times[b - 1][ia] < times[b][ib])) { who[k] = 0; idx[k++] = ia++; }
            else { who[k] = 1; idx[k++] = ib++; }
        }
        size_t Sa = (size_t)1 << (2 * ga), Sb = (size_t)1 << (2 * gb);
        for (size_t cb = 0; cb < Sb; ++cb) {
            double gw = 1;
            for (int j = 0; j < gb; ++j) {
                int sg = (cb >> (2 * j)) & 1, tg = (cb >> (2 * j + 1)) & 1;
                gw *= (sg == tg) ? W_same : W_diff;
            }
            double acc = 0;
            for (size_t ca = 0; ca < Sa; ++ca) {
                double p = v[ca];
                if (tot == 0) p *= 16.0;
                for (int j = 0; j < tot; ++j) {
                    int jn = (j + 1) % tot;
                    size_t cj = who[j] ? cb : ca, cn = who[jn] ? cb : ca;
                    int sa = (cj >> (2 * idx[j])) & 1, tb = (cn >> (2 * idx[jn] + 1)) & 1;
                    p *= LINK(sa, tb);
                }
                acc += p;
            }
            w[cb] = acc * gw;
        }
        double *tmp = v; v = w; w = tmp;
        free(who); free(idx);
    }
    /* last qubit n-1: links among bond n-2 gates */
    {
        int g = g_of_bond[nb - 1];
        size_t Sg = (size_t)1 << (2 * g);
        double acc = 0;
        for (size_t c = 0; c < Sg; ++c) {
            double p = v[c];
            if (g == 0) p *= 16.0;
            for (int j = 0; j < g; ++j) {
                int nx = (j + 1) % g;
                int sg = (c >> (2 * j)) & 1, tn = (c >> (2 * nx + 1)) & 1;
                p *= LINK(sg, tn);
            }
            acc += p;
        }
        result = acc;
    }
#undef LINK
    for (int b = 0; b < nb; ++b) free(times[b]);
    free(times); free(g_of_bond); free(v); free(w);
    return result;
}

/* ======================================================================== */
/* Qudit brickwork (the paper states its method for local dimension q: Sec.  */
/* "Frame potential" and the qudit paragraph of Sec. "Algorithm             */
/* description"; the Haar gates are U(q^2)).  Open chain of n qudits, layer  */
/* t acting on bonds b = (t-1) mod 2, b+2, ...; qudit 0 is the most         */
/* significant digit; a gate on (b, b+1) has matrix index a_b q + a_{b+1}.   */
/* Gate g of circuit w of a pair: the d x d complex Gaussian (d = q^2),      */
/* entry k = d r + c from Philox block c0 = k/2, c1 = g, stream = w, words   */
/* (x0, x1) for even k and (x2, x3) for odd k (the qubit rule for d = 4),    */
/* then classical Gram-Schmidt QR with positive-real R diagonal.             */
/* ======================================================================== */
void orc_haar_uq(int q, uint64_t seed, uint64_t pair, int which, int gate, double *out)
{
    const int d = q * q;
    cplx *Z = malloc(sizeof(cplx) * d * d), *Q = malloc(sizeof(cplx) * d * d), *v = malloc(sizeof(cplx) * d);
    for (int k = 0; k < d * d; ++k) {
        uint64_t w[4];
        draw(seed, (uint64_t)(k / 2), (uint64_t)gate, pair, (uint64_t)which, w);
        uint64_t xa = (k % 2 == 0) ? w[0] : w[2];
        uint64_t xb = (k % 2 == 0) ? w[1] : w[3];
        double u1 = (double)((xa >> 11) + 1) * 0x1.0p-53;
        double u2 = (double)(xb >> 11) * 0x1.0p-53;
        double rad = sqrt(-2.0 * log(u1));
        Z[k] = (rad * cos(2.0 * ORC_PI * u2) + I * rad * sin(2.0 * ORC_PI * u2)) / sqrt(2.0);
    }
    for (int c = 0; c < d; ++c) {
        for (int r = 0; r < d; ++r) v[r] = Z[d * r + c];
        for (int j = 0; j < c; ++j) {
            cplx dot = 0;
            for (int r = 0; r < d; ++r) dot += conj(Q[d * r + j]) * Z[d * r + c];
            for (int r = 0; r < d; ++r) v[r] -= dot * Q[d * r + j];
        }
        double nrm = 0;
        for (int r = 0; r < d; ++r) nrm += creal(v[r] * conj(v[r]));
        nrm = sqrt(nrm);
        for (int r = 0; r < d; ++r) Q[d * r + c] = v[r] / nrm;
    }
    for (int k = 0; k < d * d; ++k) { out[2 * k] = creal(Q[k]); out[2 * k + 1] = cimag(Q[k]); }
    free(Z); free(Q); free(v);
}

/* the gates of one circuit: bonds[g] and matrices gates[g * 2 d^2 ...] */
static int qudit_circuit(int q, int n, int l, uint64_t seed, uint64_t pair, int which, int *bonds, double *gates)
{
    const int d = q * q;
    int g = 0;
    for (int t = 1; t <= l; ++t)
        for (int b = (t - 1) % 2; b <= n - 2; b += 2) {
            bonds[g] = b;
            orc_haar_uq(q, seed, pair, which, g, gates + (size_t)g * 2 * d * d);
            ++g;
        }
    return g;
}

static int qudit_gate_count(int n, int l)
{
    int g = 0;
    for (int t = 1; t <= l; ++t)
        for (int b = (t - 1) % 2; b <= n - 2; b += 2) ++g;
    return g;
}

/* Tr(U^dagger V) = sum_ij conj(U_ij) V_ij with U, V built densely (q^n x q^n). */
int orc_trace_qudit_dense(int q, int n, int l, uint64_t seed, uint64_t pair, int self_pair, double tr[2])
{
    size_t D = 1;
    for (int i = 0; i < n; ++i) D *= (size_t)q;
    if (D > 4096) return -1;
    const int d = q * q, G = qudit_gate_count(n, l);
    int *bonds = malloc(sizeof(int) * (G > 0 ? G : 1));
    double *gates = malloc(sizeof(double) * 2 * d * d * (G > 0 ? G : 1));
    cplx *M[2];
    for (int w = 0; w < 2; ++w) {
        M[w] = calloc(D * D, sizeof(cplx));
        for (size_t i = 0; i < D; ++i) M[w][i * D + i] = 1;
        qudit_circuit(q, n, l, seed, pair, self_pair ? 0 : w, bonds, gates);
        for (int g = 0; g < G; ++g) {
            const cplx *U = (const cplx *)(gates + (size_t)g * 2 * d * d);
            size_t s1 = 1;                                 /* place value of qudit b+1 */
            for (int i = bonds[g] + 2; i < n; ++i) s1 *= (size_t)q;
            size_t s0 = s1 * (size_t)q;                    /* qudit b */
            cplx *a = malloc(sizeof(cplx) * d);
            for (size_t col = 0; col < D; ++col)
                for (size_t r = 0; r < D; ++r) {
                    if ((r / s0) % q != 0 || (r / s1) % q != 0) continue;   /* r: both digits zero */
                    for (int e = 0; e < d; ++e) a[e] = M[w][(r + (e / q) * s0 + (e % q) * s1) * D + col];
                    for (int o = 0; o < d; ++o) {
                        cplx acc = 0;
                        for (int e = 0; e < d; ++e) acc += U[o * d + e] * a[e];
                        M[w][(r + (o / q) * s0 + (o % q) * s1) * D + col] = acc;
                    }
                }
            free(a);
        }
    }
    cplx s = 0;
    for (size_t i = 0; i < D * D; ++i) s += conj(M[0][i]) * M[1][i];
    tr[0] = creal(s); tr[1] = cimag(s);
    free(M[0]); free(M[1]); free(bonds); free(gates);
    return 0;
}

/* Variable elimination over q-ary wire segments (the qubit elimination with   */
/* digits in place of bits): every gate of U^dagger V cuts the wires of its    */
/* two qudits; a segment is a q-ary variable; a gate is a factor over its two  */
/* output and two input segments; the sums run in min-degree order.            */
typedef struct { int nv; int *vars; cplx *t; } qfactor;

static size_t ipow(int q, int e) { size_t r = 1; while (e-- > 0) r *= (size_t)q; return r; }

int orc_trace_qudit_ve(int q, int n, int l, uint64_t seed, uint64_t pair, int self_pair, double tr[2])
{
    const int d = q * q, G = qudit_gate_count(n, l), T = 2 * G;
    int *bonds[2];
    double *gates[2];
    for (int w = 0; w < 2; ++w) {
        bonds[w] = malloc(sizeof(int) * (G > 0 ? G : 1));
        gates[w] = malloc(sizeof(double) * 2 * d * d * (G > 0 ? G : 1));
        qudit_circuit(q, n, l, seed, pair, self_pair ? 0 : w, bonds[w], gates[w]);
    }
    /* time order of U^dagger V: V's gates, then U's gates last to first, daggered */
    int *sb = malloc(sizeof(int) * (T > 0 ? T : 1));
    cplx *sg = malloc(sizeof(cplx) * d * d * (T > 0 ? T : 1));
    for (int g = 0; g < G; ++g) {
        sb[g] = bonds[1][g];
        memcpy(&sg[(size_t)g * d * d], gates[1] + (size_t)g * 2 * d * d, sizeof(cplx) * d * d);
        const cplx *u = (const cplx *)(gates[0] + (size_t)(G - 1 - g) * 2 * d * d);
        sb[G + g] = bonds[0][G - 1 - g];
        for (int r = 0; r < d; ++r)
            for (int c = 0; c < d; ++c) sg[(size_t)(G + g) * d * d + r * d + c] = conj(u[c * d + r]);
    }
    int *s = calloc(n, sizeof(int)), *base = calloc(n + 1, sizeof(int)), *pos = malloc(sizeof(int) * 2 * (T > 0 ? T : 1));
    for (int t = 0; t < T; ++t) { pos[2 * t] = s[sb[t]]++; pos[2 * t + 1] = s[sb[t] + 1]++; }
    for (int i = 0; i < n; ++i) base[i + 1] = base[i] + (s[i] > 0 ? s[i] : 1);
    const int nvars = base[n];
    int nf = T, capf = T + 8;
    qfactor *fs = calloc(capf, sizeof(qfactor));
    for (int t = 0; t < T; ++t) {
        int vo[2], vi[2];
        for (int i = 0; i < 2; ++i) {
            int qq = sb[t] + i, sq = s[qq];
            vo[i] = base[qq] + pos[2 * t + i];
            vi[i] = base[qq] + (pos[2 * t + i] - 1 + sq) % sq;
        }
        /* factor over (out_b, out_b1, in_b, in_b1): entry = G[(o_b q + o_b1), (i_b q + i_b1)];  */
        /* a segment that is both input and output of the gate (a qudit with one gate) is one  */
        /* variable: the factor then keeps the diagonal                                        */
        int all[4] = {vo[0], vo[1], vi[0], vi[1]}, uv[4], nu = 0, map[4];
        for (int k = 0; k < 4; ++k) {
            int j;
            for (j = 0; j < nu; ++j) if (uv[j] == all[k]) break;
            if (j == nu) uv[nu++] = all[k];
            map[k] = j;
        }
        fs[t].nv = nu;
        fs[t].vars = malloc(sizeof(int) * nu);
        memcpy(fs[t].vars, uv, sizeof(int) * nu);
        size_t sz = ipow(q, nu);
        fs[t].t = malloc(sizeof(cplx) * sz);
        for (size_t x = 0; x < sz; ++x) {
            int val[4], dv[4];
            size_t y = x;
            for (int j = 0; j < nu; ++j) { dv[j] = (int)(y % q); y /= q; }
            for (int k = 0; k < 4; ++k) val[k] = dv[map[k]];
            fs[t].t[x] = sg[(size_t)t * d * d + (val[0] * q + val[1]) * d + (val[2] * q + val[3])];
        }
    }
    cplx scalar = 1;
    char *gone = calloc(nvars > 0 ? nvars : 1, 1);
    int *uvars = malloc(sizeof(int) * (nvars + 8)), *sel = malloc(sizeof(int) * (capf + 1));
    for (int step = 0; step < nvars; ++step) {
        int best = -1, best_w = 1 << 30;
        for (int c = 0; c < nvars; ++c) {
            if (gone[c]) continue;
            int nu = 0;
            for (int f = 0; f < nf; ++f) {
                if (!fs[f].t) continue;
                int has = 0;
                for (int k = 0; k < fs[f].nv; ++k) has |= fs[f].vars[k] == c;
                if (!has) continue;
                for (int k = 0; k < fs[f].nv; ++k) {
                    int u;
                    for (u = 0; u < nu; ++u) if (uvars[u] == fs[f].vars[k]) break;
                    if (u == nu) uvars[nu++] = fs[f].vars[k];
                }
            }
            if (nu < best_w) { best_w = nu; best = c; }
        }
        const int v = best;
        gone[v] = 1;
        int ns = 0;
        for (int f = 0; f < nf; ++f) {
            if (!fs[f].t) continue;
            for (int k = 0; k < fs[f].nv; ++k) if (fs[f].vars[k] == v) { sel[ns++] = f; break; }
        }
        if (ns == 0) { scalar *= q; continue; }        /* a free wire loop: Tr(I_q) */
        int nu = 0;
        uvars[nu++] = v;
        for (int i = 0; i < ns; ++i)
            for (int k = 0; k < fs[sel[i]].nv; ++k) {
                int u;
                for (u = 0; u < nu; ++u) if (uvars[u] == fs[sel[i]].vars[k]) break;
                if (u == nu) uvars[nu++] = fs[sel[i]].vars[k];
            }
        const int nr = nu - 1;
        const size_t rsz = ipow(q, nr);
        cplx *res = malloc(sizeof(cplx) * rsz);
        int *dig = malloc(sizeof(int) * nu);
        for (size_t r = 0; r < rsz; ++r) {
            size_t y = r;
            for (int j = 1; j < nu; ++j) { dig[j] = (int)(y % q); y /= q; }
            cplx acc = 0;
            for (int x = 0; x < q; ++x) {
                dig[0] = x;
                cplx p = 1;
                for (int i = 0; i < ns; ++i) {
                    const qfactor *f = &fs[sel[i]];
                    size_t idx = 0, pw = 1;
                    for (int k = 0; k < f->nv; ++k) {
                        int u;
                        for (u = 0; u < nu; ++u) if (uvars[u] == f->vars[k]) break;
                        idx += (size_t)dig[u] * pw;
                        pw *= (size_t)q;
                    }
                    p *= f->t[idx];
                }
                acc += p;
            }
            res[r] = acc;
        }
        free(dig);
        for (int i = 0; i < ns; ++i) {
            free(fs[sel[i]].t); fs[sel[i]].t = NULL;
            free(fs[sel[i]].vars); fs[sel[i]].vars = NULL;
        }
        if (nf >= capf) {
            capf *= 2;
            fs = realloc(fs, sizeof(qfactor) * capf);
            sel = realloc(sel, sizeof(int) * (capf + 1));
        }
        qfactor *nfac = &fs[nf++];
        nfac->nv = nr;
        nfac->vars = malloc(sizeof(int) * (nr > 0 ? nr : 1));
        memcpy(nfac->vars, uvars + 1, sizeof(int) * nr);
        nfac->t = res;
    }
    for (int f = 0; f < nf; ++f)
        if (fs[f].t) { scalar *= fs[f].t[0]; free(fs[f].t); free(fs[f].vars); }
    tr[0] = creal(scalar); tr[1] = cimag(scalar);
    free(fs); free(gone); free(uvars); free(sel); free(s); free(base); free(pos); free(sb); free(sg);
    for (int w = 0; w < 2; ++w) { free(bonds[w]); free(gates[w]); }
    return 0;
}
