// kernels_reduce.cu -- FP64 Monte Carlo moments (K7).
//
// x = |Tr|^2 per pair; per group g: N_g, S_k = sum x^k, Q_k = sum x^{2k},
// k = 1..k_max, from which F^(k) = S_k / N and its standard error
// sqrt((Q_k - S_k^2/N) / (N-1) / N) follow (paper: Sec. "Algorithm
// description" for the estimator, Fig. 4 caption for standard errors).
// Deterministic: block b owns a fixed contiguous range of pairs, threads
// stride it in a fixed order, partials are combined by a fixed tree and the
// block partials by one thread in block order with Neumaier compensation.
#include <cuda_runtime.h>

#include "kernels.h"

namespace fpk {
namespace {

constexpr int RT = 256;
constexpr int MAXV = 2 * FP_MAX_KMAX + 1;

__global__ void __launch_bounds__(RT) moments_pass1(const double *__restrict__ tr, const int32_t *__restrict__ group,
                                                    uint64_t count, int k_max, int n_groups, double *__restrict__ partials) {
    __shared__ double sh[RT];
    const int nv = 2 * k_max + 1;
    const uint64_t per = (count + gridDim.x - 1) / gridDim.x;
    const uint64_t lo = (uint64_t)blockIdx.x * per;
    const uint64_t hi = lo + per < count ? lo + per : count;
    for (int g = 0; g < n_groups; ++g) {
        double acc[MAXV];
#pragma unroll
        for (int v = 0; v < MAXV; ++v) acc[v] = 0;
        for (uint64_t i = lo + threadIdx.x; i < hi; i += RT) {
            if (group && group[i] != g) continue;
            if (!group && g != 0) continue;
            double a = tr[2 * i], b = tr[2 * i + 1];
            double x = a * a + b * b, p = 1.0;
            acc[0] += 1.0;
#pragma unroll
            for (int k = 1; k <= FP_MAX_KMAX; ++k) {
                if (k > k_max) break;
                p *= x;
                acc[k] += p;
                acc[k_max + k] += p * p;
            }
        }
        for (int v = 0; v < nv; ++v) {
            sh[threadIdx.x] = acc[v];
            __syncthreads();
            for (int s = RT / 2; s > 0; s >>= 1) {
                if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
                __syncthreads();
            }
            if (threadIdx.x == 0) partials[((size_t)blockIdx.x * n_groups + g) * nv + v] = sh[0];
            __syncthreads();
        }
    }
}

__global__ void moments_pass2(const double *__restrict__ partials, int nblocks, int k_max, int n_groups,
                              double *__restrict__ out) {
    const int nv = 2 * k_max + 1;
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_groups * nv) return;
    int g = t / nv, v = t % nv;
    double s = 0, c = 0;
    for (int b = 0; b < nblocks; ++b) {
        double x = partials[((size_t)b * n_groups + g) * nv + v];
        double y = s + x;
        c += fabs(s) >= fabs(x) ? (s - y) + x : (x - y) + s;
        s = y;
    }
    out[t] = s + c;
}

}  // namespace

int moments_blocks(uint64_t count) {
    uint64_t b = (count + 4095) / 4096;
    if (b < 1) b = 1;
    if (b > 1024) b = 1024;
    return (int)b;
}

cudaError_t launch_moments(const double *tr, const int32_t *group, uint64_t count, int k_max,
                           int n_groups, double *partials, int nblocks, double *out,
                           cudaStream_t st) {
    moments_pass1<<<nblocks, RT, 0, st>>>(tr, group, count, k_max, n_groups, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int tot = n_groups * (2 * k_max + 1);
    moments_pass2<<<(tot + 127) / 128, 128, 0, st>>>(partials, nblocks, k_max, n_groups, out);
    return cudaGetLastError();
}

}  // namespace fpk
