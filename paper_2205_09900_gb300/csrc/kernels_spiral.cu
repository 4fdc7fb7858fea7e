// kernels_spiral.cu -- spiral sweep of the paper's hardware-efficient ansatz.
//
// The planner (make_spiral_plan) turns Tr(U^dagger V) of an ensemble whose
// wires are rings of segments, each tapped by one CZ, into a sequence of
// in-place 4x4 maps on a state of 2^bits amplitudes (one bit per CZ of a bond
// plus an auxiliary bit).  Per pair:
//   spiral_maps_kernel   builds every map from the pair's merged 1-qubit
//                        operators (FP64 products, stored in C);
//   spiral_sweep_kernel  one CTA per pair: start state delta(aux, first bit),
//                        the maps in order (one barrier each), then the FP64
//                        sum of the state = Tr, its cancellation ratio and
//                        rounding-error estimate.
// The state lives in shared memory when it fits, else in a per-pair global
// (L2-resident) slice.
#include <cuda_runtime.h>

#include "kernels.h"

namespace fpk {
namespace {

__device__ __forceinline__ uint32_t ins0s(uint32_t x, int p) {   // insert a zero bit at position p
    return (x & ((1u << p) - 1u)) | ((x >> p) << (p + 1));
}

template <typename C> __device__ __forceinline__ C mk(double re, double im);
template <> __device__ __forceinline__ double2 mk<double2>(double re, double im) { return make_double2(re, im); }
template <> __device__ __forceinline__ float2 mk<float2>(double re, double im) { return make_float2((float)re, (float)im); }

__device__ __forceinline__ double2 zm(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// entries of one map, T[4 o + f], o = o_a + 2 o_b, f = i_a + 2 i_b (SpiralType)
template <typename C>
__global__ void spiral_maps_kernel(const PairInfo *__restrict__ pairs, const SpiralMap *__restrict__ sm, int nmaps,
                                   const double2 *__restrict__ merged, C *__restrict__ maps) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= nmaps) return;
    const PairInfo pi = pairs[blockIdx.y];
    const SpiralMap s = sm[m];
    const double2 one = make_double2(1, 0), zero = make_double2(0, 0);
    double2 F[4] = {one, zero, zero, one}, G[4] = {one, zero, zero, one};
    if (s.f >= 0)
        for (int e = 0; e < 4; ++e) F[e] = merged[(pi.merged_off + s.f) * 16 + e];
    if (s.g >= 0)
        for (int e = 0; e < 4; ++e) G[e] = merged[(pi.merged_off + s.g) * 16 + e];
    C *out = maps + ((size_t)blockIdx.y * nmaps + m) * 16;
    for (int o = 0; o < 4; ++o)
        for (int f = 0; f < 4; ++f) {
            const int oa = o & 1, ob = o >> 1, ia = f & 1, ib = f >> 1;
            const double h = (ob & ib) ? -1.0 : 1.0;   // H[o_b][i_b] = (-1)^{o_b i_b}
            double2 v = zero;
            switch (s.type) {
                case SP_DIAG_BA: if (o == f) v = G[2 * ib + ia]; break;
                case SP_START: if (oa == ob) v = make_double2(h, 0); break;
                case SP_MID: v = zm(F[2 * oa + ia], G[2 * ob + oa]); v.x *= h; v.y *= h; break;
                case SP_MID_AUX: if (ob == ib) v = zm(F[2 * oa + ia], G[2 * ob + oa]); break;
                case SP_RL: if (oa == ia) { v = G[2 * ob + ia]; v.x *= h; v.y *= h; } break;
                case SP_MID_RR: if (ib == 0) v = zm(F[2 * oa + ia], G[2 * ob + oa]); break;
                case SP_RR: if (oa == ia && ib == 0) v = G[2 * ob + ia]; break;
                case SP_LL: if (oa == 0) { v = G[2 * ob + ia]; v.x *= h; v.y *= h; } break;
                case SP_LL_AUX: if (oa == 0 && ob == ib) v = G[2 * ib + ia]; break;
                default: break;
            }
            out[4 * o + f] = mk<C>(v.x, v.y);
        }
}

template <typename C>
__device__ __forceinline__ C cmac(C t, C x, C acc) {
    acc.x = fma(t.x, x.x, acc.x);
    acc.x = fma(-t.y, x.y, acc.x);
    acc.y = fma(t.x, x.y, acc.y);
    acc.y = fma(t.y, x.x, acc.y);
    return acc;
}

__device__ __forceinline__ double wsum_s(double v) {
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
    return v;
}

template <typename C, bool SMEM>
__global__ void __launch_bounds__(512) spiral_sweep_kernel(const PairInfo *__restrict__ pairs, const SpiralMap *__restrict__ sm,
                                                           int nmaps, int bits, int first_bit,
                                                           const C *__restrict__ maps, C *__restrict__ scratch,
                                                           double err_scale, double *__restrict__ tr,
                                                           double *__restrict__ kappa, double *__restrict__ err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[4][16];
    const uint32_t S = 1u << bits;
    C *st = SMEM ? (C *)smem_raw : scratch + (size_t)blockIdx.x * S;
    const int aux = bits - 1;
    for (uint32_t x = threadIdx.x; x < S; x += blockDim.x)
        st[x] = mk<C>((((x >> aux) ^ (x >> first_bit)) & 1u) ? 0.0 : 1.0, 0.0);
    __syncthreads();
    const C *mp = maps + (size_t)blockIdx.x * nmaps * 16;
    for (int k = 0; k < nmaps; ++k) {
        const SpiralMap s = sm[k];
        C T[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) T[e] = mp[(size_t)k * 16 + e];
        const int lo = s.a < s.b ? s.a : s.b, hi = s.a < s.b ? s.b : s.a;
        const uint32_t ia = 1u << s.a, ib = 1u << s.b;
        for (uint32_t q = threadIdx.x; q < (S >> 2); q += blockDim.x) {
            const uint32_t i0 = ins0s(ins0s(q, lo), hi);
            const C x0 = st[i0], x1 = st[i0 | ia], x2 = st[i0 | ib], x3 = st[i0 | ia | ib];
            C y[4];
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                C acc = mk<C>(0, 0);
                acc = cmac(T[4 * o + 0], x0, acc);
                acc = cmac(T[4 * o + 1], x1, acc);
                acc = cmac(T[4 * o + 2], x2, acc);
                acc = cmac(T[4 * o + 3], x3, acc);
                y[o] = acc;
            }
            st[i0] = y[0];
            st[i0 | ia] = y[1];
            st[i0 | ib] = y[2];
            st[i0 | ia | ib] = y[3];
        }
        __syncthreads();
    }
    // Tr = sum of the state (FP64), with sum |t| (cancellation ratio) and sum |t|^2 (error estimate)
    double sr = 0, si = 0, sa = 0, s2 = 0;
    for (uint32_t x = threadIdx.x; x < S; x += blockDim.x) {
        const double re = (double)st[x].x, im = (double)st[x].y, q = re * re + im * im;
        sr += re; si += im; sa += sqrt(q); s2 += q;
    }
    sr = wsum_s(sr); si = wsum_s(si); sa = wsum_s(sa); s2 = wsum_s(s2);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { red[0][wid] = sr; red[1][wid] = si; red[2][wid] = sa; red[3][wid] = s2; }
    __syncthreads();
    if (threadIdx.x == 0) {
        sr = si = sa = s2 = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { sr += red[0][w]; si += red[1][w]; sa += red[2][w]; s2 += red[3][w]; }
        const PairInfo pi = pairs[blockIdx.x];
        tr[2 * pi.out] = sr;
        tr[2 * pi.out + 1] = si;
        const double mag = sqrt(sr * sr + si * si);
        if (kappa) kappa[pi.out] = mag > 0 ? sa / mag : __longlong_as_double(0x7ff0000000000000LL);
        if (err) err[pi.out] = err_scale * (sqrt(s2) + mag);
    }
}

template <typename C>
cudaError_t sweep_t(const PairInfo *pairs, int npairs, const SpiralMap *sm, int nmaps, int bits, int first_bit,
                    const void *maps, void *scratch, double err_scale, double *tr, double *kappa, double *err,
                    cudaStream_t st) {
    const size_t bytes = ((size_t)1 << bits) * sizeof(C);
    const int threads = bits >= 11 ? 512 : (bits >= 9 ? 128 : 32);
    if (bytes <= (size_t)128 * 1024) {
        auto k = spiral_sweep_kernel<C, true>;
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return e;
        k<<<npairs, threads, bytes, st>>>(pairs, sm, nmaps, bits, first_bit, (const C *)maps, nullptr, err_scale, tr,
                                          kappa, err);
    } else {
        spiral_sweep_kernel<C, false><<<npairs, threads, 0, st>>>(pairs, sm, nmaps, bits, first_bit, (const C *)maps,
                                                                 (C *)scratch, err_scale, tr, kappa, err);
    }
    return cudaGetLastError();
}

}  // namespace

size_t spiral_scratch_elems(int bits, bool fp32) {
    const size_t bytes = ((size_t)1 << bits) * (fp32 ? sizeof(float2) : sizeof(double2));
    return bytes <= (size_t)128 * 1024 ? 0 : ((size_t)1 << bits);
}

cudaError_t launch_spiral(const PairInfo *pairs, int npairs, const SpiralMap *sm, int nmaps, int bits, int first_bit,
                          const double2 *merged, void *maps, void *scratch, bool fp32, double err_scale, double *tr,
                          double *kappa, double *err, cudaStream_t st) {
    if (npairs <= 0) return cudaSuccess;
    dim3 gm((nmaps + 127) / 128, npairs);
    if (fp32) spiral_maps_kernel<float2><<<gm, 128, 0, st>>>(pairs, sm, nmaps, merged, (float2 *)maps);
    else spiral_maps_kernel<double2><<<gm, 128, 0, st>>>(pairs, sm, nmaps, merged, (double2 *)maps);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return fp32 ? sweep_t<float2>(pairs, npairs, sm, nmaps, bits, first_bit, maps, scratch, err_scale, tr, kappa, err, st)
                : sweep_t<double2>(pairs, npairs, sm, nmaps, bits, first_bit, maps, scratch, err_scale, tr, kappa, err, st);
}

}  // namespace fpk
