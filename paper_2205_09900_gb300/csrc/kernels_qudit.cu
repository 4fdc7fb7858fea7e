// kernels_qudit.cu -- brickwork circuits of qudits (local dimension q = 3, 4):
// the dual-circuit sweep of the qubit path (brick.h) with q-ary segment
// variables.  The paper states its method for general local dimension (Sec.
// "Frame potential", and the qudit paragraph of Sec. "Algorithm description");
// its generalised-Hadamard formula serves only the ancilla form, which this
// direct trace contraction does not use.
//
// K1q  qudit_sample:  Haar U(q^2) gates, one thread per gate: q^4 complex
//                     Gaussians (Philox block k/2 for entry k, Box-Muller),
//                     Householder QR, columns rotated so that R's diagonal is
//                     positive real.
// K2q  qudit_maps:    per (bond, position) the merged gate realigned into the
//                     q^2 x q^2 map the sweep applies (FP64, stored FP32/FP64).
// K3q  qudit_sweep:   one CTA per pair: the boundary over the 2m segment digits
//                     of one qudit (q^{2m} amplitudes, in shared memory when it
//                     fits, else in a per-pair global slot), both chain halves,
//                     then the FP64 meet with the cancellation ratio and the
//                     error estimate.
#include <cuda_runtime.h>

#include "brick.h"
#include "kernels.h"

namespace fpk {
namespace {

__device__ __forceinline__ double2 qmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 qconj(double2 a) { return make_double2(a.x, -a.y); }

template <int Q>
__global__ void __launch_bounds__(64) qudit_sample_kernel(uint64_t seed, const PairInfo *__restrict__ pairs, int npairs,
                                                           int n_raw, int self_pair, double2 *__restrict__ raw) {
    constexpr int D = Q * Q;
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= npairs * 2 * n_raw) return;
    const int p = id / (2 * n_raw), w = (id / n_raw) % 2, g = id % n_raw;
    const uint64_t pair = pairs[p].pair;
    const int ws = self_pair ? 0 : w;
    double2 A[D][D], Qm[D][D];
    for (int k = 0; k < D * D; k += 2) {
        U64x4 x = philox(seed, (uint64_t)(k / 2), (uint64_t)g, pair, (uint64_t)ws);
        for (int h = 0; h < 2 && k + h < D * D; ++h) {
            const uint64_t xa = x.x[2 * h], xb = x.x[2 * h + 1];
            const double u1 = (double)((xa >> 11) + 1) * 0x1.0p-53;
            const double u2 = (double)(xb >> 11) * 0x1.0p-53;
            const double rad = sqrt(-2.0 * log(u1)) * 0.70710678118654752440;
            double s, c;
            sincospi(2.0 * u2, &s, &c);
            A[(k + h) / D][(k + h) % D] = make_double2(rad * c, rad * s);
        }
    }
    for (int r = 0; r < D; ++r)
        for (int c = 0; c < D; ++c) Qm[r][c] = make_double2(r == c ? 1.0 : 0.0, 0.0);
    for (int k = 0; k < D - 1; ++k) {
        double nrm2 = 0;
        for (int r = k; r < D; ++r) nrm2 += A[r][k].x * A[r][k].x + A[r][k].y * A[r][k].y;
        const double nrm = sqrt(nrm2), a0 = hypot(A[k][k].x, A[k][k].y);
        const double2 ph = a0 > 0 ? make_double2(A[k][k].x / a0, A[k][k].y / a0) : make_double2(1.0, 0.0);
        double2 v[D];
        for (int r = 0; r < D; ++r) v[r] = r < k ? make_double2(0, 0) : A[r][k];
        v[k].x += ph.x * nrm;
        v[k].y += ph.y * nrm;
        double vn2 = 0;
        for (int r = k; r < D; ++r) vn2 += v[r].x * v[r].x + v[r].y * v[r].y;
        if (vn2 == 0) continue;
        const double f = 2.0 / vn2;
        for (int c = 0; c < D; ++c) {   // A <- (I - f v v^H) A
            double2 s = make_double2(0, 0);
            for (int r = k; r < D; ++r) { const double2 t = qmul(qconj(v[r]), A[r][c]); s.x += t.x; s.y += t.y; }
            for (int r = k; r < D; ++r) { const double2 t = qmul(v[r], s); A[r][c].x -= f * t.x; A[r][c].y -= f * t.y; }
        }
        for (int r = 0; r < D; ++r) {   // Q <- Q (I - f v v^H)
            double2 s = make_double2(0, 0);
            for (int j = k; j < D; ++j) { const double2 t = qmul(Qm[r][j], v[j]); s.x += t.x; s.y += t.y; }
            for (int j = k; j < D; ++j) { const double2 t = qmul(s, qconj(v[j])); Qm[r][j].x -= f * t.x; Qm[r][j].y -= f * t.y; }
        }
    }
    // Z = Q R: rotate column j of Q by the phase of R_jj so that R's diagonal is positive real
    double2 *out = raw + (size_t)id * D * D;
    for (int j = 0; j < D; ++j) {
        const double m = hypot(A[j][j].x, A[j][j].y);
        const double2 ph = m > 0 ? make_double2(A[j][j].x / m, A[j][j].y / m) : make_double2(1.0, 0.0);
        for (int r = 0; r < D; ++r) out[r * D + j] = qmul(Qm[r][j], ph);
    }
}

template <typename C> __device__ __forceinline__ C to_c(double2 z);
template <> __device__ __forceinline__ double2 to_c<double2>(double2 z) { return z; }
template <> __device__ __forceinline__ float2 to_c<float2>(double2 z) { return make_float2((float)z.x, (float)z.y); }

// one map per thread: (pair, side, layer t, gate j)
template <int Q, typename C>
__global__ void qudit_maps_kernel(BrickDev d, int npairs, int n_raw, const double2 *__restrict__ raw,
                                  C *__restrict__ maps) {
    constexpr int D = Q * Q;
    const int per = maps_per_pair(d);
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= npairs * per) return;
    const int p = id / per, mi = id % per, g = mi / d.m, j = mi % d.m, l = d.l;
    const int side = g < d.n_layers[0] ? 0 : 1, t = side ? g - d.n_layers[0] : g;
    const double2 *U = raw + (size_t)p * 2 * n_raw * D * D, *V = U + (size_t)n_raw * D * D;
    const int b = brick_bond(d, side, t);
    const int tau = 2 * j + (b + 1) % 2;
    const int c0 = d.n / 2, c1 = (d.n - 1) / 2;
    auto gidx = [&](int tl) {   // circuit gate index of layer tl (1-based) on bond b
        const int tm = tl - 1;
        return ((tm + 1) / 2) * c0 + (tm / 2) * c1 + (b - tm % 2) / 2;
    };
    // the merged gate at position tau (as for qubits: V's layers, the middle and
    // cyclic merges, U's layers daggered), computed entry by entry
    auto G = [&](int r, int c) -> double2 {
        if (tau <= l - 3) return V[(size_t)gidx(tau + 2) * D * D + r * D + c];
        if (tau == l - 2 || tau == 2 * l - 3) {
            const int tl = tau == l - 2 ? l : 1;
            const double2 *A = U + (size_t)gidx(tl) * D * D, *B = V + (size_t)gidx(tl) * D * D;
            double2 acc = make_double2(0, 0);
            for (int k = 0; k < D; ++k) {   // tau = l-2: U_l^dagger V_l ; tau = 2l-3: V_1 U_1^dagger
                const double2 x = tau == l - 2 ? qmul(qconj(A[k * D + r]), B[k * D + c]) : qmul(B[r * D + k], qconj(A[c * D + k]));
                acc.x += x.x;
                acc.y += x.y;
            }
            return acc;
        }
        return qconj(U[(size_t)gidx(2 * l - 2 - tau) * D * D + c * D + r]);
    };
    C *out = maps + (size_t)id * D * D;
    const bool left = side == 0;
    // gate index (a_b q + a_{b+1}); segment tau (in) and tau+1 (out) of qudits y = b, x = b+1;
    // map index e = w_tau + q w_{tau+1}: left M[ex][ey], right M[ey][ex]
    for (int yt = 0; yt < Q; ++yt)
        for (int xt = 0; xt < Q; ++xt)
            for (int yt1 = 0; yt1 < Q; ++yt1)
                for (int xt1 = 0; xt1 < Q; ++xt1) {
                    const double2 gv = G(yt1 * Q + xt1, yt * Q + xt);
                    const int ex = xt + Q * xt1, ey = yt + Q * yt1;
                    out[left ? ex * D + ey : ey * D + ex] = to_c<C>(gv);
                }
}

template <typename C>
__device__ __forceinline__ C cfmaq(C t, C x, C acc) {
    acc.x = fma(t.x, x.x, acc.x);
    acc.x = fma(-t.y, x.y, acc.x);
    acc.y = fma(t.x, x.y, acc.y);
    acc.y = fma(t.y, x.x, acc.y);
    return acc;
}

__device__ __forceinline__ double qsum(double v) {
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
    return v;
}

// One CTA per pair.  The state lives at `st` (shared memory or the pair's
// global slot), the left boundary at `lb`.  Maps are applied one at a time:
// every thread takes groups of q^2 amplitudes that differ only in digits
// (tau, tau+1 mod N), one barrier per map.
template <int Q, typename C>
__global__ void __launch_bounds__(256) qudit_sweep_kernel(BrickDev d, const PairInfo *__restrict__ pairs,
                                                           const C *__restrict__ maps, C *__restrict__ gstate,
                                                           int in_smem, double err_scale, double *__restrict__ tr,
                                                           double *__restrict__ kappa, double *__restrict__ err) {
    constexpr int D = Q * Q;
    extern __shared__ __align__(16) unsigned char qsm[];
    __shared__ double red[4][8];
    __shared__ C T[D * D];
    const int p = blockIdx.x, N = d.N;
    uint32_t S = 1;
    for (int i = 0; i < N; ++i) S *= Q;
    C *st = in_smem ? (C *)qsm : gstate + (size_t)p * 2 * S;
    C *lb = in_smem ? (C *)qsm + S : gstate + (size_t)p * 2 * S + S;
    const C *mp = maps + (size_t)p * maps_per_pair(d) * D * D;
    uint32_t pw[32];
    pw[0] = 1;
    for (int i = 1; i <= N; ++i) pw[i] = pw[i - 1] * Q;
    for (int side = 0; side < 2; ++side) {
        // chain end: prod over tau of parity delta_par[side] of delta(w_tau, w_tau+1 mod N)
        const int par = d.delta_par[side];
        for (uint32_t w = threadIdx.x; w < S; w += blockDim.x) {
            bool ok = true;
            for (int tau = par; tau < N; tau += 2) {
                const uint32_t a = (w / pw[tau]) % Q, b = (w / pw[(tau + 1) % N]) % Q;
                ok = ok && a == b;
            }
            C v;
            v.x = ok ? 1 : 0;
            v.y = 0;
            st[w] = v;
        }
        __syncthreads();
        for (int t = 0; t < d.n_layers[side]; ++t) {
            const int par_t = layer_parity(d, side, t);
            for (int j = 0; j < d.m; ++j) {
                const C *src = mp + (size_t)map_index(d, side, t, j) * D * D;
                for (int i = threadIdx.x; i < D * D; i += blockDim.x) T[i] = src[i];
                __syncthreads();
                const int pa = 2 * j + par_t, pb = (pa + 1) % N;
                const uint32_t sa = pw[pa], sb = pw[pb];
                const int lo = pa < pb ? pa : pb, hi = pa < pb ? pb : pa;
                for (uint32_t gq = threadIdx.x; gq < S / D; gq += blockDim.x) {
                    // insert zero digits at positions lo and hi
                    const uint32_t a1 = gq % pw[lo], r1 = gq / pw[lo];
                    const uint32_t x1 = a1 + r1 * pw[lo + 1];
                    const uint32_t a2 = x1 % pw[hi], r2 = x1 / pw[hi];
                    const uint32_t base = a2 + r2 * pw[hi + 1];
                    C x[D], y[D];
#pragma unroll
                    for (int e = 0; e < D; ++e) x[e] = st[base + (e % Q) * sa + (e / Q) * sb];
#pragma unroll
                    for (int o = 0; o < D; ++o) {
                        C acc;
                        acc.x = 0;
                        acc.y = 0;
#pragma unroll
                        for (int e = 0; e < D; ++e) acc = cfmaq(T[o * D + e], x[e], acc);
                        y[o] = acc;
                    }
#pragma unroll
                    for (int e = 0; e < D; ++e) st[base + (e % Q) * sa + (e / Q) * sb] = y[e];
                }
                __syncthreads();
            }
        }
        if (side == 0) {
            for (uint32_t w = threadIdx.x; w < S; w += blockDim.x) lb[w] = st[w];
            __syncthreads();
        }
    }
    double sr = 0, si = 0, sa = 0, s2 = 0;
    for (uint32_t w = threadIdx.x; w < S; w += blockDim.x) {
        const C l = lb[w], r = st[w];
        const double px = (double)l.x * r.x - (double)l.y * r.y, py = (double)l.x * r.y + (double)l.y * r.x;
        sr += px;
        si += py;
        sa += sqrt(px * px + py * py);
        s2 += px * px + py * py;
    }
    sr = qsum(sr); si = qsum(si); sa = qsum(sa); s2 = qsum(s2);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { red[0][wid] = sr; red[1][wid] = si; red[2][wid] = sa; red[3][wid] = s2; }
    __syncthreads();
    if (threadIdx.x == 0) {
        sr = si = sa = s2 = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { sr += red[0][w]; si += red[1][w]; sa += red[2][w]; s2 += red[3][w]; }
        const int64_t o = pairs[p].out;
        tr[2 * o] = sr;
        tr[2 * o + 1] = si;
        const double mag = sqrt(sr * sr + si * si);
        if (kappa) kappa[o] = mag > 0 ? sa / mag : __longlong_as_double(0x7ff0000000000000LL);
        if (err) err[o] = err_scale * (sqrt(s2) + mag);
    }
}

template <int Q>
cudaError_t run_qudit_t(const BrickDev &d, uint64_t seed, const PairInfo *pairs, int npairs, int n_raw, int self_pair,
                        bool fp32, void *ws, double err_scale, double *tr, double *kappa, double *err, cudaStream_t st) {
    constexpr int D = Q * Q;
    size_t S = 1;
    for (int i = 0; i < d.N; ++i) S *= Q;
    const size_t celem = fp32 ? sizeof(float2) : sizeof(double2);
    double2 *raw = (double2 *)ws;
    unsigned char *maps = (unsigned char *)(raw + (size_t)npairs * 2 * n_raw * D * D);
    const size_t nmaps = (size_t)npairs * maps_per_pair(d);
    unsigned char *gstate = maps + nmaps * D * D * celem;
    const int total = npairs * 2 * n_raw;
    qudit_sample_kernel<Q><<<(total + 63) / 64, 64, 0, st>>>(seed, pairs, npairs, n_raw, self_pair, raw);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const unsigned mb = (unsigned)((nmaps + 127) / 128);
    if (fp32) qudit_maps_kernel<Q, float2><<<mb, 128, 0, st>>>(d, npairs, n_raw, raw, (float2 *)maps);
    else qudit_maps_kernel<Q, double2><<<mb, 128, 0, st>>>(d, npairs, n_raw, raw, (double2 *)maps);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t smem = 2 * S * celem;
    const int in_smem = smem <= (size_t)200 * 1024 ? 1 : 0;
    const size_t dyn = in_smem ? smem : 0;
    if (fp32) {
        if ((e = cudaFuncSetAttribute(qudit_sweep_kernel<Q, float2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)dyn)) != cudaSuccess)
            return e;
        qudit_sweep_kernel<Q, float2><<<npairs, 256, dyn, st>>>(d, pairs, (const float2 *)maps, (float2 *)gstate,
                                                               in_smem, err_scale, tr, kappa, err);
    } else {
        if ((e = cudaFuncSetAttribute(qudit_sweep_kernel<Q, double2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)dyn)) != cudaSuccess)
            return e;
        qudit_sweep_kernel<Q, double2><<<npairs, 256, dyn, st>>>(d, pairs, (const double2 *)maps,
                                                                (double2 *)gstate, in_smem, err_scale, tr, kappa, err);
    }
    return cudaGetLastError();
}

}  // namespace

size_t qudit_workspace_per_pair(int q, const BrickDev &d, int n_raw, bool fp32) {
    const size_t D = (size_t)q * q, celem = fp32 ? sizeof(float2) : sizeof(double2);
    size_t S = 1;
    for (int i = 0; i < d.N; ++i) S *= (size_t)q;
    const bool in_smem = 2 * S * celem <= (size_t)200 * 1024;
    return (size_t)2 * n_raw * D * D * sizeof(double2) + (size_t)maps_per_pair(d) * D * D * celem +
           (in_smem ? 0 : 2 * S * celem);
}

cudaError_t launch_qudit(int q, const BrickDev &d, uint64_t seed, const PairInfo *pairs, int npairs, int n_raw, int self_pair,
                         bool fp32, void *ws, double err_scale, double *tr, double *kappa, double *err,
                         cudaStream_t st) {
    if (npairs <= 0) return cudaSuccess;
    switch (q) {
        case 3: return run_qudit_t<3>(d, seed, pairs, npairs, n_raw, self_pair, fp32, ws, err_scale, tr, kappa, err, st);
        case 4: return run_qudit_t<4>(d, seed, pairs, npairs, n_raw, self_pair, fp32, ws, err_scale, tr, kappa, err, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fpk
