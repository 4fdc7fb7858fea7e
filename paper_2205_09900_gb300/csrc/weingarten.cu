// weingarten.cu -- exact ensemble F^(k) (k = 2, 3) of brickwork circuits of qubits
// or of qudits of local dimension q (Haar U(q^2) gates).
//
// Averaging every Haar U(4) gate of the cyclic U^dagger V circuit over the
// Haar measure turns the k-th moment |Tr(U^dagger V)|^{2k} into a classical
// statistical-mechanics sum (the mapping behind the paper's Eq. theory_eq,
// Sec. "Frame potential"): each gate carries an output and an input pairing
// sigma, tau in S_k with weight Wg(sigma^-1 tau) (the Weingarten function of
// U(4)), and consecutive gates on a qubit wire, output pairing sigma_a then
// input pairing tau_b, meet with weight q^{#cycles(sigma_a^-1 tau_b)}.
//
// After the middle and cyclic merges a depth-l brickwork pair is a cyclic
// brickwork of P = 2(l-1) time positions; bond b holds the gates at the
// positions t with t = b+1 (mod 2).  Give the wire links of any qubit the
// indices t = 0..P-1 (link t joins the gate at position t to the one at t+1).
// Storing a gate's output pairing in slot t and its input pairing in slot
// t-1 (mod P), the variables of one bond occupy every slot exactly once, and
// the transfer across qubit b is
//   (1) the q^{#cycles} link matrix applied to every slot (each link of the
//       qubit pairs one slot of bond b-1 with the same slot of bond b), then
//   (2) the Wg factors of bond b's gates, a diagonal over slot pairs (t, t-1).
// The chain ends close with the links among one bond's gates, slots (t, t+1).
// The state of a bond is a (k!)^P-entry FP64 vector; it is renormalised by a
// power of two after every bond (exact), the exponents summed at the end.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "kernels.h"

namespace fpk {
namespace {

constexpr int kMaxSlots = 22;   // k = 2: l <= 12; k = 3 is limited to 12 slots (l <= 7)

struct WgTab {
    int P;                  // slots
    double link[36];        // link[x * s + y] = q^{#cycles(x^-1 y)}
    double wg[36];          // wg[sigma * s + tau] = Wg(sigma^-1 tau)
};

template <int S>
__device__ __forceinline__ void decode(uint64_t c, int P, int *d) {
    if (S == 2) {
        for (int t = 0; t < P; ++t) d[t] = (int)((c >> t) & 1u);
    } else {
        for (int t = 0; t < P; ++t) {
            d[t] = (int)(c % S);
            c /= S;
        }
    }
}

__device__ __forceinline__ void block_max_to(double v, double *dst) {
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = fmax(m, red[i]);
        // non-negative doubles order like their bit patterns
        atomicMax((unsigned long long *)dst, (unsigned long long)__double_as_longlong(m));
    }
}

__device__ __forceinline__ double unscale(const double *maxes, int b) {
    const double m = maxes[b];
    return m > 0 ? ldexp(1.0, -ilogb(m)) : 1.0;
}

// qubit 0: Wg of the bond-0 gates (positions t = 1 mod 2) and the links among them
template <int S>
__global__ void wg_init_kernel(WgTab T, uint64_t N, double *__restrict__ v, double *__restrict__ maxes) {
    double mx = 0;
    for (uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; c < N; c += (uint64_t)gridDim.x * blockDim.x) {
        int d[kMaxSlots];
        decode<S>(c, T.P, d);
        double p = 1.0;
        for (int t = 1; t < T.P; t += 2) {
            p *= T.wg[d[t] * S + d[t - 1]];
            p *= T.link[d[t] * S + d[(t + 1) % T.P]];
        }
        v[c] = p;
        mx = fmax(mx, fabs(p));
    }
    block_max_to(mx, maxes);
}

// the link matrix on slot i (stride s^i), in place
template <int S>
__global__ void wg_slot_kernel(WgTab T, uint64_t N, uint64_t stride, double *__restrict__ v) {
    const uint64_t cols = N / S;
    for (uint64_t col = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; col < cols;
         col += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t hi = col / stride, lo = col - hi * stride;
        double *p = v + hi * stride * S + lo;
        double x[S];
#pragma unroll
        for (int j = 0; j < S; ++j) x[j] = p[j * stride];
#pragma unroll
        for (int y = 0; y < S; ++y) {
            double acc = 0;
#pragma unroll
            for (int j = 0; j < S; ++j) acc = fma(T.link[j * S + y], x[j], acc);
            p[y * stride] = acc;
        }
    }
}

// Wg of bond b's gates (positions t = par mod 2), after undoing the previous scale
template <int S>
__global__ void wg_gate_kernel(WgTab T, uint64_t N, int par, int b, double *__restrict__ v, double *__restrict__ maxes) {
    const double sc = unscale(maxes, b - 1);
    double mx = 0;
    for (uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; c < N; c += (uint64_t)gridDim.x * blockDim.x) {
        int d[kMaxSlots];
        decode<S>(c, T.P, d);
        double p = sc;
        for (int t = par; t < T.P; t += 2) p *= T.wg[d[t] * S + d[(t + T.P - 1) % T.P]];
        const double x = v[c] * p;
        v[c] = x;
        mx = fmax(mx, fabs(x));
    }
    block_max_to(mx, maxes + b);
}

// last qubit: links among the last bond's gates; one partial sum per block
template <int S>
__global__ void wg_final_kernel(WgTab T, uint64_t N, int par, int blast, const double *__restrict__ v,
                                const double *__restrict__ maxes, double *__restrict__ partial) {
    const double sc = unscale(maxes, blast);
    double acc = 0;
    for (uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; c < N; c += (uint64_t)gridDim.x * blockDim.x) {
        int d[kMaxSlots];
        decode<S>(c, T.P, d);
        double p = v[c] * sc;
        for (int t = par; t < T.P; t += 2) p *= T.link[d[t] * S + d[(t + 1) % T.P]];
        acc += p;
    }
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
        partial[blockIdx.x] = s;
    }
}

// fixed-order sum of the partials, times 2^{sum of the per-bond exponents}
__global__ void wg_sum_kernel(const double *__restrict__ partial, int nparts, const double *__restrict__ maxes,
                              int nmax, double *__restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0;
    for (int i = 0; i < nparts; ++i) s += partial[i];
    int e = 0;
    for (int b = 0; b < nmax; ++b)
        if (maxes[b] > 0) e += ilogb(maxes[b]);
    *out = ldexp(s, e);
}

// host: permutations of S_k and their cycle counts
int perms(int k, int (*p)[3]) {
    int np = 0, v[3];
    for (v[0] = 0; v[0] < k; ++v[0])
        for (v[1] = 0; v[1] < (k > 1 ? k : 1); ++v[1])
            for (v[2] = 0; v[2] < (k > 2 ? k : 1); ++v[2]) {
                bool ok = true;
                for (int i = 0; i < k; ++i)
                    for (int j = 0; j < i; ++j) ok = ok && v[i] != v[j];
                if (!ok) continue;
                for (int i = 0; i < 3; ++i) p[np][i] = v[i];
                ++np;
            }
    return np;
}

int cycles(const int *a, const int *b, int k) {   // #cycles of a^-1 b
    int inv[3], seen[3] = {0, 0, 0}, c = 0;
    for (int i = 0; i < k; ++i) inv[a[i]] = i;
    for (int i = 0; i < k; ++i) {
        if (seen[i]) continue;
        ++c;
        for (int j = i; !seen[j]; j = inv[b[j]]) seen[j] = 1;
    }
    return c;
}

template <int S>
cudaError_t run_sweep(const WgTab &T, int n, uint64_t N, double *v, double *maxes, double *partial, int nparts,
                      double *out, cudaStream_t st) {
    const int threads = 256;
    const unsigned grid = (unsigned)std::min<uint64_t>((N + threads - 1) / threads, 152u * 16u);
    wg_init_kernel<S><<<grid, threads, 0, st>>>(T, N, v, maxes);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    for (int b = 1; b <= n - 2; ++b) {
        uint64_t stride = 1;
        for (int i = 0; i < T.P; ++i, stride *= S) {
            const unsigned g2 = (unsigned)std::min<uint64_t>((N / S + threads - 1) / threads, 152u * 16u);
            wg_slot_kernel<S><<<g2, threads, 0, st>>>(T, N, stride, v);
        }
        wg_gate_kernel<S><<<grid, threads, 0, st>>>(T, N, (b + 1) & 1, b, v, maxes);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    wg_final_kernel<S><<<nparts, threads, 0, st>>>(T, N, (n - 1) & 1, n - 2, v, maxes, partial);
    wg_sum_kernel<<<1, 32, 0, st>>>(partial, nparts, maxes, n - 1, out);
    return cudaGetLastError();
}

}  // namespace
}  // namespace fpk

extern "C" fp_status fp_exact_brickwork_fkq(int32_t n, int32_t l, int32_t k, int32_t q, void *cuda_stream,
                                             double *F) {
    using namespace fpk;
    if (!F) return api_fail(FP_ERR_ARG, "F is NULL");
    if (n < 2 || n > 1 << 20) return api_fail(FP_ERR_ARG, "n outside [2, 2^20]");
    if (q < 2 || q > 64) return api_fail(FP_ERR_ARG, "local dimension q outside [2, 64]");
    if (k != 2 && k != 3) return api_fail(FP_ERR_ARG, "k must be 2 or 3");
    if (l < 2 || (k == 2 && l > 12) || (k == 3 && l > 7))
        return api_fail(FP_ERR_ARG, "depth l outside [2, 12] (k = 2) or [2, 7] (k = 3)");
    WgTab T;
    T.P = 2 * (l - 1);
    int p[6][3];
    const int s = perms(k, p);
    const double d = (double)q * q;   // Haar U(q^2) gates on neighbouring qudits
    for (int a = 0; a < s; ++a)
        for (int b = 0; b < s; ++b) {
            const int c = cycles(p[a], p[b], k);
            T.link[a * s + b] = std::pow((double)q, c);
            double w;
            if (k == 2) w = c == 2 ? 1.0 / (d * d - 1) : -1.0 / (d * (d * d - 1));
            else w = c == 3 ? (d * d - 2) / (d * (d * d - 1) * (d * d - 4))
                   : c == 2 ? -1.0 / ((d * d - 1) * (d * d - 4))
                            : 2.0 / (d * (d * d - 1) * (d * d - 4));
            T.wg[a * s + b] = w;
        }
    uint64_t N = 1;
    for (int i = 0; i < T.P; ++i) N *= (uint64_t)s;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    size_t freeb = 0, totb = 0;
    cudaError_t e = cudaMemGetInfo(&freeb, &totb);
    if (e != cudaSuccess) return api_fail(FP_ERR_CUDA, cudaGetErrorString(e));
    const int nparts = 152 * 4;
    const size_t bytes = N * sizeof(double) + ((size_t)n + nparts + 1) * sizeof(double);
    if (bytes > freeb) return api_fail(FP_ERR_OOM, "transfer-matrix state does not fit in free device memory");
    double *buf = nullptr;
    if ((e = cudaMalloc(&buf, bytes)) != cudaSuccess) return api_fail(FP_ERR_OOM, cudaGetErrorString(e));
    double *v = buf, *maxes = buf + N, *partial = maxes + n, *out = partial + nparts;
    e = cudaMemsetAsync(maxes, 0, (size_t)n * sizeof(double), st);
    if (e == cudaSuccess) e = k == 2 ? run_sweep<2>(T, n, N, v, maxes, partial, nparts, out, st)
                                     : run_sweep<6>(T, n, N, v, maxes, partial, nparts, out, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(F, out, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(buf);
    if (e != cudaSuccess) return api_fail(FP_ERR_CUDA, cudaGetErrorString(e));
    return FP_OK;
}

extern "C" fp_status fp_exact_brickwork_fk(int32_t n, int32_t l, int32_t k, void *cuda_stream, double *F) {
    return fp_exact_brickwork_fkq(n, l, k, 2, cuda_stream, F);
}
