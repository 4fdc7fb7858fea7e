// kernels_reduce.cu -- FP64 Monte Carlo moments (K7) and their bootstrap.
//
// x = |Tr|^2 per pair; per group g: N_g, S_k = sum x^k, Q_k = sum x^{2k},
// k = 1..k_max, from which F^(k) = S_k / N and its standard error
// sqrt((Q_k - S_k^2/N) / (N-1) / N) follow (paper: Sec. "Algorithm
// description" for the estimator, Fig. 4 caption for standard errors).
// Deterministic: block b owns a fixed contiguous range of pairs, threads
// stride it in a fixed order, partials are combined by a fixed tree and the
// block partials by one thread in block order with Neumaier compensation.
// The bootstrap (paper: Supplementary, "Bootstrapping for uncertainty
// quantification") resamples each group's stored |Tr|^2 with replacement and
// evaluates F^(k) on every resample, one CTA per (resample, group).
#include <cuda_runtime.h>

#include <algorithm>

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

// xs[j] = |Tr|^2 of pair members[j] (pairs listed group by group)
__global__ void abs2_gather_kernel(const double *__restrict__ tr, const uint32_t *__restrict__ members, uint64_t n,
                                   double *__restrict__ xs) {
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < n; j += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i = members[j];
        xs[j] = tr[2 * i] * tr[2 * i] + tr[2 * i + 1] * tr[2 * i + 1];
    }
}

// Block (b, g): resample b of group g.  Draw i takes position
// ((x >> 32) N_g) >> 32 of the group, x = word i % 4 of Philox block
// {b, i / 4, g, 5} (key {seed, 0}); F^(k) of the resample = mean of a^k over
// the draws.  Fixed thread-to-draw mapping and tree: deterministic.
constexpr int BT = 256;
__global__ void __launch_bounds__(BT) bootstrap_kernel(const double *__restrict__ xs,
                                                       const uint64_t *__restrict__ goff, int k_max, int B,
                                                       uint64_t seed, double *__restrict__ out) {
    __shared__ double sh[FP_MAX_KMAX][BT / 32];
    const int b = blockIdx.x, g = blockIdx.y;
    const uint64_t off = goff[g], N = goff[g + 1] - off;
    double s[FP_MAX_KMAX];
#pragma unroll
    for (int k = 0; k < FP_MAX_KMAX; ++k) s[k] = 0.0;
    const uint64_t nq = (N + 3) / 4;
    for (uint64_t q = threadIdx.x; q < nq; q += BT) {
        const U64x4 x = philox(seed, (uint64_t)b, q, (uint64_t)g, 5);
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            if (4 * q + w >= N) break;
            const uint64_t pos = ((x.x[w] >> 32) * N) >> 32;
            const double a2 = xs[off + pos];
            double p = 1.0;
#pragma unroll
            for (int k = 0; k < FP_MAX_KMAX; ++k) {
                if (k < k_max) {
                    p *= a2;
                    s[k] += p;
                }
            }
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < FP_MAX_KMAX; ++k) {
        double v = s[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sh[k][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < k_max) {
        const int k = threadIdx.x;
        double v = 0;
        for (int w = 0; w < BT / 32; ++w) v += sh[k][w];
        out[((size_t)g * k_max + k) * B + b] = N ? v / (double)N : __longlong_as_double(0x7ff8000000000000LL);
    }
}

}  // namespace

cudaError_t launch_bootstrap(const double *tr, const uint32_t *members, uint64_t n_members, const uint64_t *goff,
                             int n_groups, int k_max, int B, uint64_t seed, double *xs, double *out,
                             cudaStream_t st) {
    if (n_members > 0) {
        abs2_gather_kernel<<<(unsigned)std::min<uint64_t>((n_members + 255) / 256, 4096), 256, 0, st>>>(
            tr, members, n_members, xs);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    bootstrap_kernel<<<dim3((unsigned)B, (unsigned)n_groups), BT, 0, st>>>(xs, goff, k_max, B, seed, out);
    return cudaGetLastError();
}

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
