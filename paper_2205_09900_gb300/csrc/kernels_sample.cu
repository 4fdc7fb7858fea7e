// kernels_sample.cu -- gate sampler (K1), gate merging and op-table builder (K2).
#include <cuda_runtime.h>

#include "kernels.h"
#include "sample_tables.h"

namespace fpk {
namespace {

// sinpi(t), cospi(t) for t in [0, 2) a multiple of 2^-52: t = k/256 + r exactly,
// r in [0, 1/256); angle addition with the tabulated sinpi, cospi(k/256) and the
// Taylor polynomials of sin and cos at x = pi r (|x| < 0.0123: the first omitted
// terms, x^9/9! and x^10/10!, are below 2e-23).
__device__ __forceinline__ void sincospi_tab(double t, double *sn, double *cs) {
    const int k = (int)(t * 256.0);
    const double r = t - (double)k * (1.0 / 256.0);
    const double x = r * kPi, x2 = x * x;
    const double sx = x * fma(x2, fma(x2, fma(x2, -1.0 / 5040.0, 1.0 / 120.0), -1.0 / 6.0), 1.0);
    const double cx = fma(x2, fma(x2, fma(x2, fma(x2, 1.0 / 40320.0, -1.0 / 720.0), 1.0 / 24.0), -0.5), 1.0);
    const double sk = __ldg(kSinCosPi + 2 * k), ck = __ldg(kSinCosPi + 2 * k + 1);
    *sn = fma(sk, cx, ck * sx);
    *cs = fma(ck, cx, -(sk * sx));
}

// log(u) for normal u in (0, 1]: u = m 2^e with m in [0.75, 1.5); with c_j the
// nearest of the points 0.75 + j/128 and r_j the tabulated double near 1/c_j,
// log u = e ln2 - log r_j + log1p(m r_j - 1), |m r_j - 1| <= 2^-7.4, log1p by its
// series to y^9 (relative truncation below 1e-20); -log r_j and ln2 in two
// parts.  At the point c = 1 (r = 1, log r = 0) y = m - 1 exactly, so log u keeps
// its relative accuracy as u -> 1.
__device__ __forceinline__ double log_tab(double u) {
    const long long b = __double_as_longlong(u);
    int e = (int)((b >> 52) & 0x7FF) - 1023;
    double m = __longlong_as_double((b & 0x000FFFFFFFFFFFFFLL) | 0x3FF0000000000000LL);
    if (m >= 1.5) {
        m *= 0.5;
        ++e;
    }
    const int j = __double2int_rn((m - 0.75) * 128.0);
    const double r = __ldg(kLogTab + 3 * j), lh = __ldg(kLogTab + 3 * j + 1), ll = __ldg(kLogTab + 3 * j + 2);
    const double y = fma(m, r, -1.0);
    double p = fma(y, -1.0 / 9.0, 1.0 / 8.0);
    p = fma(y, p, -1.0 / 7.0);
    p = fma(y, p, 1.0 / 6.0);
    p = fma(y, p, -1.0 / 5.0);
    p = fma(y, p, 1.0 / 4.0);
    p = fma(y, p, -1.0 / 3.0);
    p = fma(y, p, 0.5);
    p = fma(y, p, -1.0);
    p = -(y * p);   // y - y^2/2 + y^3/3 - ... + y^9/9
    const double ed = (double)e;
    return fma(ed, kLn2Hi, lh) + (fma(ed, kLn2Lo, ll) + p);
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

// Haar U(4): QR of a 4x4 complex Gaussian by Householder reflections, then
// the columns of Q rotated so that R's diagonal is positive real (the Haar
// sampler of the Methods section, "Sampling U(d^2)", realised as in Mezzadri
// 2007).  Gaussian entries by Box-Muller from Philox words (keying in fp.h):
// block j of the gate gives entries 2j and 2j+1 (row-major).
__device__ __forceinline__ void gauss_pair(uint64_t seed, uint64_t pair, int w, int g, int j, double2 *out) {
    U64x4 x = philox(seed, (uint64_t)j, (uint64_t)g, pair, (uint64_t)w);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint64_t xa = x.x[2 * h], xb = x.x[2 * h + 1];
        double u1 = (double)((xa >> 11) + 1) * 0x1.0p-53;
        double u2 = (double)(xb >> 11) * 0x1.0p-53;
        double rad = sqrt(-2.0 * log_tab(u1)) * 0.70710678118654752440;
        double s, c;
        sincospi_tab(2.0 * u2, &s, &c);
        out[2 * j + h] = make_double2(rad * c, rad * s);
    }
}

// In place: the 16 Gaussian entries at g (row-major) become the Haar unitary.
// Householder step k maps column k to (alpha, 0, ..) with alpha = -ph |col|,
// ph = a_kk / |a_kk|; with v = col - alpha e_k, |v|^2 = 2 nrm (nrm + |a_kk|), so
// the reflection I - f v v^H takes f = 1 / (nrm (nrm + |a_kk|)).  Only the
// columns right of k change (column k becomes alpha e_k, the ones left of it
// are already reduced); R's diagonal phase for k < 3 is then alpha / |alpha| =
// -ph, and Q's columns are rotated by those phases (the phase fix).  The
// first reflection is applied to the identity in closed form.
__device__ void haar_qr(double2 *g) {
    double2 A[4][4];
#pragma unroll
    for (int k = 0; k < 16; ++k) A[k / 4][k % 4] = g[k];
    double2 Q[4][4];
    double2 dph[4];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double nrm2 = 0;
#pragma unroll
        for (int r = k; r < 4; ++r) nrm2 += A[r][k].x * A[r][k].x + A[r][k].y * A[r][k].y;
        const double a2 = A[k][k].x * A[k][k].x + A[k][k].y * A[k][k].y;
        const double ia = a2 > 0 ? rsqrt(a2) : 0.0, a0 = a2 * ia;   // |a_kk|
        const double2 ph = a2 > 0 ? make_double2(A[k][k].x * ia, A[k][k].y * ia) : make_double2(1.0, 0.0);
        const double nrm = sqrt(nrm2);
        dph[k] = make_double2(-ph.x, -ph.y);
        double2 v[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) v[r] = r < k ? make_double2(0, 0) : A[r][k];
        v[k].x += ph.x * nrm;
        v[k].y += ph.y * nrm;
        if (nrm == 0) {   // a zero column (probability 0): no reflection
            if (k == 0)
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) Q[r][c] = make_double2(r == c ? 1.0 : 0.0, 0.0);
            continue;
        }
        const double f = 1.0 / (nrm * (nrm + a0));
        // A <- (I - f v v^H) A, columns k+1 .. 3
#pragma unroll
        for (int c = k + 1; c < 4; ++c) {
            double2 sv = make_double2(0, 0);
#pragma unroll
            for (int r = k; r < 4; ++r) { double2 t = cmul(cconj(v[r]), A[r][c]); sv.x += t.x; sv.y += t.y; }
            sv.x *= f;
            sv.y *= f;
#pragma unroll
            for (int r = k; r < 4; ++r) { double2 t = cmul(v[r], sv); A[r][c].x -= t.x; A[r][c].y -= t.y; }
        }
        if (k == 0) {   // Q = I - f v v^H
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const double2 t = cmul(v[r], cconj(v[j]));
                    Q[r][j] = make_double2((r == j ? 1.0 : 0.0) - f * t.x, -f * t.y);
                }
        } else {        // Q <- Q (I - f v v^H)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                double2 sv = make_double2(0, 0);
#pragma unroll
                for (int j = k; j < 4; ++j) { double2 t = cmul(Q[r][j], v[j]); sv.x += t.x; sv.y += t.y; }
                sv.x *= f;
                sv.y *= f;
#pragma unroll
                for (int j = k; j < 4; ++j) { double2 t = cmul(sv, cconj(v[j])); Q[r][j].x -= t.x; Q[r][j].y -= t.y; }
            }
        }
    }
    {
        const double a2 = A[3][3].x * A[3][3].x + A[3][3].y * A[3][3].y;
        const double ia = a2 > 0 ? rsqrt(a2) : 0.0;
        dph[3] = a2 > 0 ? make_double2(A[3][3].x * ia, A[3][3].y * ia) : make_double2(1.0, 0.0);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int r = 0; r < 4; ++r) g[4 * r + c] = cmul(Q[r][c], dph[c]);
}

// Haar gates in two passes, so that the transcendental-heavy Gaussian draws
// run at full occupancy: one thread per Philox block (8 per gate) writes the
// gate's Gaussian entries into its raw record, then one thread per gate
// factorises them in place.
__global__ void gauss_kernel(SampleParams sp, const PairInfo *__restrict__ pairs, double2 *__restrict__ raw) {
    const PairInfo pi = pairs[blockIdx.y];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int idx = t >> 3, j = t & 7;
    if (idx >= 2 * pi.n_raw) return;
    const int w = idx / pi.n_raw, g = idx % pi.n_raw;
    gauss_pair(sp.seed, pi.pair, sp.self_pair ? 0 : w, g, j, raw + (pi.raw_off + idx) * 16);
}

__global__ void haar_qr_kernel(const PairInfo *__restrict__ pairs, double2 *__restrict__ raw) {
    const PairInfo pi = pairs[blockIdx.y];
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 2 * pi.n_raw) return;
    haar_qr(raw + (pi.raw_off + idx) * 16);
}

__global__ void sample_kernel(SampleParams sp, const PairInfo *__restrict__ pairs, double2 *__restrict__ raw) {
    const PairInfo pi = pairs[blockIdx.y];
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 2 * pi.n_raw) return;
    int w = idx / pi.n_raw, g = idx % pi.n_raw;
    int wr = sp.self_pair ? 0 : w;
    double2 *out = raw + (pi.raw_off + idx) * 16;
    if (sp.raw_kind == RAW_DIAG4) {
        U64x4 x = philox(sp.seed, 0, (uint64_t)g, pi.pair, (uint64_t)wr);
#pragma unroll
        for (int k = 0; k < 16; ++k) out[k] = make_double2(0, 0);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            double s, c;
            sincospi(2.0 * ((double)(x.x[k] >> 11) * 0x1.0p-53), &s, &c);
            out[5 * k] = make_double2(c, s);
        }
    } else if (sp.raw_kind == RAW_PAULI) {
        // the paper's HEA (Fig. 2c): H, the RY(pi/4) wall, Pauli rotations
#pragma unroll
        for (int k = 0; k < 16; ++k) out[k] = make_double2(0, 0);
        if (g == 0) {
            const double h = 0.70710678118654752440;
            out[0] = make_double2(h, 0); out[1] = make_double2(h, 0);
            out[2] = make_double2(h, 0); out[3] = make_double2(-h, 0);
        } else if (g <= sp.n) {
            // RY(pi/4) = [[c, -s], [s, c]], c = cos(pi/8), s = sin(pi/8)
            double s, c;
            sincospi(0.125, &s, &c);
            out[0] = make_double2(c, 0); out[1] = make_double2(-s, 0);
            out[2] = make_double2(s, 0); out[3] = make_double2(c, 0);
        } else {
            const int r = g - 1 - sp.n, t = r / sp.n, q = r % sp.n;
            U64x4 x = philox(sp.seed, (uint64_t)t, (uint64_t)q, pi.pair, (uint64_t)wr);
            const double th = (double)(x.x[0] >> 11) * 0x1.0p-53;   // theta in turns of 2 pi
            const uint32_t axis = pick(x.x[1], 3u);
            double s, c;
            sincospi(th, &s, &c);                // sin, cos of theta/2
            // exp(-i theta P/2) = c I - i s P
            if (axis == 0) {        // X
                out[0] = make_double2(c, 0); out[1] = make_double2(0, -s);
                out[2] = make_double2(0, -s); out[3] = make_double2(c, 0);
            } else if (axis == 1) { // Y
                out[0] = make_double2(c, 0); out[1] = make_double2(-s, 0);
                out[2] = make_double2(s, 0); out[3] = make_double2(c, 0);
            } else {                // Z
                out[0] = make_double2(c, -s); out[3] = make_double2(c, s);
            }
        }
    } else {   // RAW_ROT2: HEA rotation RY(theta) RZ(phi), raw index g = t*n + q
        int t = g / sp.n, q = g % sp.n;
        U64x4 x = philox(sp.seed, (uint64_t)t, (uint64_t)q, pi.pair, (uint64_t)wr);
        double th = (double)(x.x[0] >> 11) * 0x1.0p-53;   // in turns of 2 pi
        double ph = (double)(x.x[1] >> 11) * 0x1.0p-53;
        double sth, cth, sph, cph;
        sincospi(th, &sth, &cth);            // sin, cos of theta/2 = pi * th
        sincospi(ph, &sph, &cph);            // sin, cos of phi/2
        double2 em = make_double2(cph, -sph), ep = make_double2(cph, sph);
#pragma unroll
        for (int k = 4; k < 16; ++k) out[k] = make_double2(0, 0);
        out[0] = make_double2(cth * em.x, cth * em.y);
        out[1] = make_double2(-sth * ep.x, -sth * ep.y);
        out[2] = make_double2(sth * em.x, sth * em.y);
        out[3] = make_double2(cth * ep.x, cth * ep.y);
    }
}

__global__ void merge_kernel(const PairInfo *__restrict__ pairs, const DevPlan *__restrict__ plans,
                             const MergeItem *__restrict__ items, const MergeRef *__restrict__ refs,
                             const double2 *__restrict__ raw, double2 *__restrict__ merged) {
    const PairInfo pi = pairs[blockIdx.y];
    const DevPlan &pl = plans[pi.plan];
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= pl.n_merged) return;
    MergeItem it = items[pl.merge_off + m];
    double2 M[16];
    int dim = refs[pl.ref_off + it.first].dim;
#pragma unroll
    for (int k = 0; k < 16; ++k) M[k] = make_double2(0, 0);
    for (int r = 0; r < dim; ++r) M[r * dim + r] = make_double2(1, 0);
    for (int c = 0; c < it.count; ++c) {
        MergeRef rf = refs[pl.ref_off + it.first + c];
        const double2 *A = raw + (pi.raw_off + (int64_t)rf.which * pi.n_raw + rf.gate) * 16;
        double2 G[16], N[16];
        for (int r = 0; r < dim; ++r)
            for (int s = 0; s < dim; ++s)
                G[r * dim + s] = rf.dagger ? cconj(A[s * dim + r]) : A[r * dim + s];
        for (int r = 0; r < dim; ++r)
            for (int s = 0; s < dim; ++s) {
                double2 acc = make_double2(0, 0);
                for (int k = 0; k < dim; ++k) {
                    double2 t = cmul(G[r * dim + k], M[k * dim + s]);
                    acc.x += t.x; acc.y += t.y;
                }
                N[r * dim + s] = acc;
            }
        for (int k = 0; k < dim * dim; ++k) M[k] = N[k];
    }
    double2 *out = merged + (pi.merged_off + m) * 16;
#pragma unroll
    for (int k = 0; k < 16; ++k) out[k] = M[k];
}

template <typename C>
__device__ __forceinline__ C to_c(double re, double im);
template <>
__device__ __forceinline__ double2 to_c<double2>(double re, double im) { return make_double2(re, im); }
template <>
__device__ __forceinline__ float2 to_c<float2>(double re, double im) { return make_float2((float)re, (float)im); }

template <typename C>
__global__ void table_kernel(const PairInfo *__restrict__ pairs, const DevPlan *__restrict__ plans,
                             const DevRecipe *__restrict__ recipes, const double2 *__restrict__ merged,
                             C *__restrict__ tables) {
    const PairInfo pi = pairs[blockIdx.y];
    const DevPlan &pl = plans[pi.plan];
    int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= pl.n_left + pl.n_right) return;
    const DevRecipe &r = recipes[pl.rec_off + o];
    C *out = tables + (pi.table_off + o) * 16;
    const double2 *M = r.merged >= 0 ? merged + (pi.merged_off + r.merged) * 16 : nullptr;
    for (int e = 0; e < 16; ++e) {
        double re = 0, im = 0;
        if (e < r.nent) {
            if (M) {
                for (int s = 0; s < 4; ++s) {
                    int k = r.src[e][s];
                    if (k >= 0) { re += r.sgn[e][s] * M[k].x; im += r.sgn[e][s] * M[k].y; }
                }
            } else {
                re = r.cre[e];
                im = r.cim[e];
            }
        }
        out[e] = to_c<C>(re, im);
    }
}

}  // namespace

int sample_launch_count(int raw_kind) { return raw_kind == RAW_HAAR4 ? 2 : 1; }

cudaError_t launch_sample(const SampleParams &sp, const PairInfo *pairs, int npairs, int max_raw,
                          double2 *raw, cudaStream_t st) {
    if (npairs <= 0) return cudaSuccess;
    if (sp.raw_kind == RAW_HAAR4) {
        gauss_kernel<<<dim3((16 * max_raw + 255) / 256, npairs), 256, 0, st>>>(sp, pairs, raw);
        haar_qr_kernel<<<dim3((2 * max_raw + 127) / 128, npairs), 128, 0, st>>>(pairs, raw);
        return cudaGetLastError();
    }
    dim3 grid((2 * max_raw + 127) / 128, npairs);
    sample_kernel<<<grid, 128, 0, st>>>(sp, pairs, raw);
    return cudaGetLastError();
}

cudaError_t launch_merge(const PairInfo *pairs, int npairs, int max_merged, const DevPlan *plans,
                         const MergeItem *items, const MergeRef *refs, const double2 *raw,
                         double2 *merged, cudaStream_t st) {
    if (npairs <= 0 || max_merged <= 0) return cudaSuccess;
    dim3 grid((max_merged + 127) / 128, npairs);
    merge_kernel<<<grid, 128, 0, st>>>(pairs, plans, items, refs, raw, merged);
    return cudaGetLastError();
}

cudaError_t launch_tables(const PairInfo *pairs, int npairs, int max_ops, const DevPlan *plans,
                          const DevRecipe *recipes, const double2 *merged, void *tables, bool fp32,
                          cudaStream_t st) {
    if (npairs <= 0 || max_ops <= 0) return cudaSuccess;
    dim3 grid((max_ops + 127) / 128, npairs);
    if (fp32)
        table_kernel<float2><<<grid, 128, 0, st>>>(pairs, plans, recipes, merged, (float2 *)tables);
    else
        table_kernel<double2><<<grid, 128, 0, st>>>(pairs, plans, recipes, merged, (double2 *)tables);
    return cudaGetLastError();
}

}  // namespace fpk
