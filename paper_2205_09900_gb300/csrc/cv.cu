// cv.cu -- learned control variate for F^(2) of single-depth HEA ensembles.
//
// A small MLP maps periodic features of a pair's circuit angles to a
// prediction of log |Tr|^2; g = beta exp(2 prediction) predicts |Tr|^4, with
// beta = Cov(f, g) / Var(g) fitted on the training pairs.  The MLP is trained
// on exactly contracted pairs, g is evaluated on many cheap surrogate pairs and
// corrected on fresh exactly contracted pairs:
//     F^(2) ~= mean_M g(x) + mean_N (f(x) - g(x)),   f = |Tr(U^dagger V)|^4,
// with the three pair ranges disjoint, so the estimate stays unbiased for any
// g; its variance is Var(g)/M + Var(f - g)/N.  The plain estimator mean_N f on
// the correction pairs is reported beside it (it judges the variance
// reduction).  The paper has no control variate; F^(2) itself is the paper's
// (Sec. "Frame potential", Sec. "Algorithm description").
//
// Precision: the three hidden layers (forward, and both backward products)
// run as BF16 GEMMs with FP32 accumulation on the tensor cores (tc_gemm.cu);
// the weights are kept in FP32 for Adam and cast to BF16 copies after every
// step; the 1-wide output layer, the loss and the estimator sums are FP32 /
// FP64 SIMT kernels.  The steps of one training epoch are captured once as a
// CUDA graph and replayed; the data are reshuffled (a gather on the device)
// between epochs.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <random>
#include <vector>

#include "fp.h"
#include "kernels.h"

namespace {

using bf16 = __nv_bfloat16;
using fpk::U64x4;
using fpk::philox;

// features of one pair, 12 per (layer t, qubit q), column 12 (t n + q) + f:
// cos and sin of U's theta and phi, of V's theta and phi, and of the
// differences theta_U - theta_V, phi_U - phi_V (the trace depends on the angles
// periodically; at one layer |Tr|^2 is a product over qubits of
// (1 + cos dtheta)(1 + cos dphi)), into the row-major [count x ldx] BF16 matrix
// X (columns >= 12 n L untouched)
__global__ void features_kernel(uint64_t seed, uint64_t first, int count, int n, int L, bf16 *X, int ldx) {
    const long long total = (long long)count * L * n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int p = (int)(i / (L * n));
        const int r = (int)(i % (L * n));
        const int t = r / n, q = r % n;
        float ang[2][2];
        for (int w = 0; w < 2; ++w) {
            U64x4 x = philox(seed, (uint64_t)t, (uint64_t)q, first + p, (uint64_t)w);
            ang[w][0] = (float)((double)(x.x[0] >> 11) * 0x1.0p-53);   // theta / (2 pi)
            ang[w][1] = (float)((double)(x.x[1] >> 11) * 0x1.0p-53);   // phi / (2 pi)
        }
        float f[12];
        for (int w = 0; w < 2; ++w)
            for (int a = 0; a < 2; ++a) sincospif(2.0f * ang[w][a], &f[4 * w + 2 * a + 1], &f[4 * w + 2 * a]);
        for (int a = 0; a < 2; ++a) sincospif(2.0f * (ang[0][a] - ang[1][a]), &f[8 + 2 * a + 1], &f[8 + 2 * a]);
        bf16 *row = X + (size_t)p * ldx + 12 * r;
#pragma unroll
        for (int k = 0; k < 12; ++k) row[k] = __float2bfloat16(f[k]);
    }
}

// training target: (log(|Tr|^2 + 1e-6) - mu) / sigma
__global__ void logt_kernel(const double *tr, int count, double mu, double inv_sigma, float *y) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const double a2 = tr[2 * i] * tr[2 * i] + tr[2 * i + 1] * tr[2 * i + 1];
    y[i] = (float)((log(a2 + 1e-6) - mu) * inv_sigma);
}

// model output -> prediction of |Tr|^4: exp(2 (sigma out + mu))
__global__ void gtrans_kernel(int count, float *g, float mu, float sigma) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) g[i] = expf(fminf(2.0f * (sigma * g[i] + mu), 80.0f));
}

// sums over the training pairs for the control-variate coefficient:
// (g, g^2, f g, f), f = |Tr|^4 from the traces
__global__ void beta_sums_kernel(int count, const float *g, const double *tr, double *sums) {
    __shared__ double sh[4][256];
    double s[4] = {0, 0, 0, 0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const double a2 = tr[2 * i] * tr[2 * i] + tr[2 * i + 1] * tr[2 * i + 1], f = a2 * a2, gv = g[i];
        s[0] += gv; s[1] += gv * gv; s[2] += f * gv; s[3] += f;
    }
    for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] = s[k];
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if (threadIdx.x < st)
            for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) atomicAdd(&sums[k], sh[k][0]);
}

__global__ void abs4_kernel(const double *tr, int count, double scale, float *y, double *f) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    double a2 = tr[2 * i] * tr[2 * i] + tr[2 * i + 1] * tr[2 * i + 1];
    if (f) f[i] = a2 * a2;
    if (y) y[i] = (float)(a2 * a2 * scale);
}

// rows of a [rows x ld] BF16 matrix gathered by perm (16-byte chunks), and the
// matching targets
__global__ void gather_rows_kernel(int rows, int ld, const int *perm, const bf16 *src, bf16 *dst, const float *y,
                                   float *ye) {
    const int cpr = ld / 8;
    const long long total = (long long)rows * cpr;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / cpr), c = (int)(i % cpr);
        const int s = perm[r];
        ((uint4 *)(dst + (size_t)r * ld))[c] = ((const uint4 *)(src + (size_t)s * ld))[c];
        if (c == 0) ye[r] = y[s];
    }
}

// dst[c * ldd + r] = src[r * lds + c] for r < rows, c < cols; 32 x 32 tiles,
// blockIdx.x over row tiles, blockIdx.y over column tiles, 32 x 8 threads
__global__ void transpose_bf16_kernel(int rows, int cols, const bf16 *src, int lds, bf16 *dst, int ldd) {
    __shared__ bf16 t[32][33];
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int r = r0 + k, c = c0 + threadIdx.x;
        if (r < rows && c < cols) t[k][threadIdx.x] = src[(size_t)r * lds + c];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int c = c0 + k, r = r0 + threadIdx.x;
        if (r < rows && c < cols) dst[(size_t)c * ldd + r] = t[threadIdx.x][k];
    }
}

// output layer (H -> 1): out[i] = A[i] . w + b, one warp per row.  With
// targets y: dY[i] = 2 (out - y) / rows and the loss accumulates; the first
// thread also counts the step (Adam's bias correction reads the counter).
__global__ void out_kernel(int rows, int H, const bf16 *__restrict__ A, const float *__restrict__ w,
                           const float *__restrict__ b, const float *__restrict__ y, float *__restrict__ out,
                           float *__restrict__ dY, double *loss, int *step) {
    const int warp = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (step && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(step, 1);
    if (warp >= rows) return;
    const bf16 *a = A + (size_t)warp * H;
    float s = 0.f;
    for (int k = 2 * lane; k < H; k += 64) {
        const float2 v = __bfloat1622float2(*(const __nv_bfloat162 *)(a + k));
        s = fmaf(v.x, w[k], fmaf(v.y, w[k + 1], s));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        const float v = s + b[0];
        if (out) out[warp] = v;
        if (y) {
            const float e = v - y[warp];
            dY[warp] = 2.0f * e / (float)rows;
            atomicAdd(loss, (double)e * (double)e / (double)rows);
        }
    }
}

// output-layer gradients: dW[k] = sum_i AT[k][i] dY[i] (k < H), db = sum_i dY[i]
// (block H); one block of 128 threads per k
__global__ void out_grad_kernel(int B, int H, const bf16 *__restrict__ AT, const float *__restrict__ dY,
                                float *__restrict__ dW, float *__restrict__ db) {
    __shared__ float sh[4];
    const int k = blockIdx.x;
    float s = 0.f;
    for (int i = threadIdx.x; i < B; i += blockDim.x)
        s += (k < H ? __bfloat162float(AT[(size_t)k * B + i]) : 1.0f) * dY[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        const float t = sh[0] + sh[1] + sh[2] + sh[3];
        if (k < H) dW[k] = t; else db[0] = t;
    }
}

__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678f)) + z * 0.39894228f * expf(-0.5f * z * z);
}

// dZ[i][k] = dY[i] w[k] GELU'(Z[i][k]) into BF16 row-major dZ [B x H] and
// transposed dZT [H x B]; 32 x 32 tiles as in transpose_bf16_kernel
__global__ void dz_out_kernel(int B, int H, const float *__restrict__ dY, const float *__restrict__ w,
                              const float *__restrict__ Z, bf16 *__restrict__ dZ, bf16 *__restrict__ dZT) {
    __shared__ bf16 t[32][33];
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int r = r0 + k, c = c0 + threadIdx.x;
        if (r < B && c < H) {
            const bf16 v = __float2bfloat16(dY[r] * w[c] * gelu_grad(Z[(size_t)r * H + c]));
            dZ[(size_t)r * H + c] = v;
            t[k][threadIdx.x] = v;
        }
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int c = c0 + k, r = r0 + threadIdx.x;
        if (r < B && c < H) dZT[(size_t)c * B + r] = t[threadIdx.x][k];
    }
}

// db[k] = sum_i dZT[k][i], one warp per row k
__global__ void rowsum_kernel(int H, int B, const bf16 *__restrict__ dZT, float *__restrict__ db) {
    const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (k >= H) return;
    float s = 0.f;
    for (int i = lane; i < B; i += 32) s += __bfloat162float(dZT[(size_t)k * B + i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) db[k] = s;
}

// BF16 copies of the hidden layers' weights: Wb[l] = W_l [fin x fout] (if
// non-null) and Wtb[l] = W_l^T [fout x finp] (columns fin..finp-1 stay zero)
struct WCast {
    long long woff[3];
    int fin[3], fout[3], finp[3];
    bf16 *Wb[3], *Wtb[3];
};

__device__ __forceinline__ void cast_weight(const WCast &c, long long i, float w) {
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        const long long o = i - c.woff[l];
        if (o >= 0 && o < (long long)c.fin[l] * c.fout[l]) {
            const int k = (int)(o / c.fout[l]), j = (int)(o % c.fout[l]);
            const bf16 v = __float2bfloat16(w);
            if (c.Wb[l]) c.Wb[l][o] = v;
            c.Wtb[l][(size_t)j * c.finp[l] + k] = v;
        }
    }
}

// Adam step (bias corrections from the device step counter), then the BF16
// casts; update = 0 casts only (the initial weights)
__global__ void adam_kernel(long long n, float *w, const float *g, float *m, float *v, float lr, float b1, float b2,
                            const int *step, int update, WCast c) {
    float c1 = 1.f, c2 = 1.f;
    if (update) {
        const float t = (float)*step;
        c1 = 1.f - powf(b1, t);
        c2 = 1.f - powf(b2, t);
    }
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float wi = w[i];
        if (update) {
            const float gi = g[i];
            const float mi = b1 * m[i] + (1.f - b1) * gi, vi = b2 * v[i] + (1.f - b2) * gi * gi;
            m[i] = mi;
            v[i] = vi;
            wi -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
            w[i] = wi;
        }
        cast_weight(c, i, wi);
    }
}

// g in units of |Tr|^4 (FP64) for export
__global__ void gexport_kernel(int count, const float *g, double gscale, double *out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) out[i] = (double)g[i] * gscale;
}

// sums over a batch of (g, g^2) or (f - g, (f - g)^2, f, f^2) in FP64
__global__ void cv_sums_kernel(int count, const float *g, double gscale, const double *f, double *sums) {
    __shared__ double sh[4][256];
    double s[4] = {0, 0, 0, 0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        double gv = (double)g[i] * gscale;
        double v = f ? f[i] - gv : gv;
        s[0] += v;
        s[1] += v * v;
        if (f) { s[2] += f[i]; s[3] += f[i] * f[i]; }
    }
    for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] = s[k];
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if (threadIdx.x < st)
            for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) atomicAdd(&sums[k], sh[k][0]);
}

struct Buf {
    void *p = nullptr;
    ~Buf() { if (p) cudaFree(p); }
    cudaError_t alloc(size_t b) { return cudaMalloc(&p, std::max<size_t>(b, 16)); }
    float *f() const { return (float *)p; }
    double *d() const { return (double *)p; }
    bf16 *h() const { return (bf16 *)p; }
    int *i() const { return (int *)p; }
};

size_t up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Mlp {
    int D, Dp, H;
    // layers: 0: D->H, 1: H->H, 2: H->H, 3: H->1; FP32 master copy [fin x fout]
    // row-major, each weight block and bias 16-byte aligned
    int fin[4], fout[4];
    size_t woff[4], boff[4], total;
    // BF16 copies of layers 0..2: W (row-major) and W^T (inputs padded to Dp for layer 0)
    size_t wboff[3], wtoff[3], btotal;
};

Mlp make_mlp(int D, int H) {
    Mlp m;
    m.D = D;
    m.Dp = (int)up(D, 8);
    m.H = H;
    int in[4] = {D, H, H, H}, out[4] = {H, H, H, 1};
    size_t o = 0, ob = 0;
    for (int l = 0; l < 4; ++l) {
        m.fin[l] = in[l];
        m.fout[l] = out[l];
        m.woff[l] = o;
        o += up((size_t)in[l] * out[l], 4);
        m.boff[l] = o;
        o += up(out[l], 4);
        if (l < 3) {
            m.wboff[l] = ob;
            ob += up((size_t)in[l] * out[l], 8);
            m.wtoff[l] = ob;
            ob += (size_t)out[l] * (l == 0 ? m.Dp : in[l]);
        }
    }
    m.total = o;
    m.btotal = ob;
    return m;
}

// forward through the three hidden layers: act = GELU(in W + b) in BF16,
// optionally keeping the pre-activations Z (FP32) and transposed activations
cudaError_t hidden_forward(cudaStream_t st, const Mlp &m, const float *W, const bf16 *Wbf, const bf16 *X, int rows,
                           bf16 *const *act, float *const *Z, bf16 *const *actT, int *err) {
    const bf16 *in = X;
    int ld = m.Dp;
    for (int l = 0; l < 3; ++l) {
        fpk::TcGemm g{};
        g.M = rows, g.N = m.H, g.K = l == 0 ? m.Dp : m.H;   // layer 0: zero-padded inputs
        g.A = in, g.lda = ld;
        g.Bt = Wbf + m.wtoff[l], g.ldb = g.K;
        g.bias = W + m.boff[l];
        g.mode = 1;
        g.Z = Z ? Z[l] : nullptr, g.ldz = m.H;
        g.Cb = act[l], g.ldcb = m.H;
        g.Cbt = actT ? actT[l] : nullptr, g.ldct = rows;
        g.err = err;
        cudaError_t e = fpk::launch_tc_gemm(g, st);
        if (e != cudaSuccess) return e;
        in = act[l];
        ld = m.H;
    }
    return cudaSuccess;
}

}  // namespace

extern "C" fp_status fp_cv_frame_potential(fp_ensemble *ens, const fp_cv_config *cfg, fp_cv_result *res) {
    using namespace fpk;
    if (!ens || !cfg || !res) return fpk::api_fail(FP_ERR_ARG, "null argument");
    const fp_ensemble_desc d = fpk::ens_desc(ens);
    if (d.kind != FP_HEA || d.depth_min != d.depth_max)
        return fpk::api_fail(FP_ERR_ARG, "the control variate needs a single-depth HEA ensemble");
    const int n = d.n, L = d.depth_min, D = 12 * n * L;
    const int H = cfg->hidden > 0 ? cfg->hidden : 256;
    const int epochs = cfg->epochs > 0 ? cfg->epochs : 20;
    const int B = cfg->batch > 0 ? cfg->batch : 512;
    const float lr = cfg->lr > 0 ? (float)cfg->lr : 1e-3f;
    const uint64_t NT = cfg->n_train, NC = cfg->n_correct, MS = cfg->m_surrogate;
    if (NT < (uint64_t)B || NC < 2 || MS < 2 || H > 1024 || H % 16 != 0 || B % 8 != 0 || NT > (1u << 30))
        return fpk::api_fail(FP_ERR_ARG, "need n_train >= batch, n_correct >= 2, m_surrogate >= 2, hidden a multiple "
                                         "of 16 up to 1024, batch a multiple of 8");
    cudaStream_t ust = fpk::ens_stream(ens);
    std::memset(res, 0, sizeof *res);
    // the work runs on a private stream (capturable), ordered after and before the caller's stream
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr, ord = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    auto cleanup = [&]() {
        if (st) {
            if (ord && cudaEventRecord(ord, st) == cudaSuccess) cudaStreamWaitEvent(ust, ord, 0);
            cudaStreamSynchronize(st);
        }
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
        if (st) cudaStreamDestroy(st);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (ord) cudaEventDestroy(ord);
    };
#define CKC(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) {                                                                   \
            cleanup();                                                                             \
            return fpk::api_fail(e_ == cudaErrorMemoryAllocation ? FP_ERR_OOM : FP_ERR_CUDA,       \
                                 cudaGetErrorString(e_));                                          \
        }                                                                                          \
    } while (0)
#define CKS(call)                                  \
    do {                                           \
        fp_status s_ = (call);                     \
        if (s_ != FP_OK) { cleanup(); return s_; } \
    } while (0)
    CKC(cudaEventCreate(&e0));
    CKC(cudaEventCreate(&e1));
    CKC(cudaEventCreateWithFlags(&ord, cudaEventDisableTiming));
    CKC(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    auto join_user = [&]() -> cudaError_t {   // st waits for everything queued on the caller's stream
        cudaError_t e = cudaEventRecord(ord, ust);
        return e == cudaSuccess ? cudaStreamWaitEvent(st, ord, 0) : e;
    };
    auto elapsed = [&]() {
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms * 1e-3;
    };
    Buf derr;
    CKC(derr.alloc(sizeof(int)));
    CKC(cudaMemsetAsync(derr.p, 0, sizeof(int), st));
    auto check_err = [&]() -> fp_status {
        int h = 0;
        if (cudaMemcpyAsync(&h, derr.p, sizeof h, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return fpk::api_fail(FP_ERR_CUDA, "control variate: device error");
        return h ? fpk::api_fail(FP_ERR_TIMEOUT, "tcgen05 GEMM: an mbarrier wait ran out") : FP_OK;
    };

    const uint64_t f_train = cfg->first, f_corr = f_train + NT, f_sur = f_corr + NC;
    Mlp m = make_mlp(D, H);
    double t_mu = 0, t_sigma = 1;   // the log-scale target's normalisation
    // ---- 1. exact contractions of the training pairs -> targets
    Buf X, y;
    CKC(X.alloc(NT * m.Dp * sizeof(bf16)));
    CKC(y.alloc(NT * sizeof(float)));
    float ms_trace = 0;
    double *dtr = nullptr;
    CKS(fpk::cv_trace(ens, f_train, NT, &dtr, &ms_trace));
    res->gpu_seconds_exact += ms_trace * 1e-3;
    CKC(join_user());
    CKC(cudaEventRecord(e0, st));
    {
        std::vector<double> h(2 * NT);
        CKC(cudaMemcpyAsync(h.data(), dtr, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        CKC(cudaStreamSynchronize(st));
        double mean = 0, lm = 0, lv = 0;
        for (uint64_t i = 0; i < NT; ++i) {
            double a2 = h[2 * i] * h[2 * i] + h[2 * i + 1] * h[2 * i + 1];
            mean += a2 * a2;
            lm += std::log(a2 + 1e-6);
        }
        mean /= (double)NT;
        lm /= (double)NT;
        for (uint64_t i = 0; i < NT; ++i) {
            double a2 = h[2 * i] * h[2 * i] + h[2 * i + 1] * h[2 * i + 1], dl = std::log(a2 + 1e-6) - lm;
            lv += dl * dl;
        }
        res->target_scale = mean > 0 ? mean : 1.0;
        t_mu = lm;
        t_sigma = NT > 1 ? std::sqrt(lv / (double)(NT - 1)) : 1.0;
        if (!(t_sigma > 0)) t_sigma = 1.0;
    }
    logt_kernel<<<(unsigned)((NT + 255) / 256), 256, 0, st>>>(dtr, (int)NT, t_mu, 1.0 / t_sigma, y.f());
    CKC(cudaGetLastError());
    CKC(cudaMemsetAsync(X.p, 0, NT * m.Dp * sizeof(bf16), st));
    features_kernel<<<1024, 256, 0, st>>>(d.seed, f_train, (int)NT, n, L, X.h(), m.Dp);
    CKC(cudaGetLastError());
    // ---- 2. training (Adam on the mean squared error of |Tr|^4 / mean)
    Buf W, Wbf, G, Mm, Vv, Xe, XeT, ye, Z[3], act[3], actT[3], dZ[2], dZT[2], out, dY, loss, step, perm;
    CKC(W.alloc(m.total * sizeof(float)));
    CKC(Wbf.alloc(m.btotal * sizeof(bf16)));
    CKC(G.alloc(m.total * sizeof(float)));
    CKC(Mm.alloc(m.total * sizeof(float)));
    CKC(Vv.alloc(m.total * sizeof(float)));
    CKC(cudaMemsetAsync(Mm.p, 0, m.total * sizeof(float), st));
    CKC(cudaMemsetAsync(Vv.p, 0, m.total * sizeof(float), st));
    CKC(cudaMemsetAsync(G.p, 0, m.total * sizeof(float), st));
    CKC(cudaMemsetAsync(Wbf.p, 0, m.btotal * sizeof(bf16), st));
    WCast wc;
    for (int l = 0; l < 3; ++l) {
        wc.woff[l] = (long long)m.woff[l];
        wc.fin[l] = m.fin[l];
        wc.fout[l] = m.fout[l];
        wc.finp[l] = l == 0 ? m.Dp : m.fin[l];
        wc.Wb[l] = l == 0 ? nullptr : Wbf.h() + m.wboff[l];   // layer 0 needs no input gradient
        wc.Wtb[l] = Wbf.h() + m.wtoff[l];
    }
    std::vector<float> hw(m.total, 0.f);
    {
        std::mt19937_64 rng(d.seed ^ 0x5DEECE66DULL);
        for (int l = 0; l < 4; ++l) {
            std::normal_distribution<float> nd(0.f, std::sqrt(2.0f / (float)m.fin[l]));
            for (size_t i = 0; i < (size_t)m.fin[l] * m.fout[l]; ++i) hw[m.woff[l] + i] = nd(rng);
        }
        CKC(cudaMemcpyAsync(W.p, hw.data(), hw.size() * sizeof(float), cudaMemcpyHostToDevice, st));
    }
    adam_kernel<<<1024, 256, 0, st>>>((long long)m.total, W.f(), G.f(), Mm.f(), Vv.f(), lr, 0.9f, 0.999f, nullptr, 0,
                                      wc);
    CKC(cudaGetLastError());
    const int nb = (int)(NT / B);
    const size_t NE = (size_t)nb * B;   // rows used per epoch
    CKC(Xe.alloc(NE * m.Dp * sizeof(bf16)));
    CKC(XeT.alloc((size_t)m.D * NE * sizeof(bf16)));
    CKC(ye.alloc(NE * sizeof(float)));
    for (int l = 0; l < 3; ++l) {
        CKC(Z[l].alloc((size_t)B * H * sizeof(float)));
        CKC(act[l].alloc((size_t)B * H * sizeof(bf16)));
        CKC(actT[l].alloc((size_t)H * B * sizeof(bf16)));
    }
    for (int i = 0; i < 2; ++i) {
        CKC(dZ[i].alloc((size_t)B * H * sizeof(bf16)));
        CKC(dZT[i].alloc((size_t)H * B * sizeof(bf16)));
    }
    CKC(out.alloc((size_t)B * sizeof(float)));
    CKC(dY.alloc((size_t)B * sizeof(float)));
    CKC(loss.alloc(sizeof(double)));
    CKC(step.alloc(sizeof(int)));
    CKC(perm.alloc(NT * sizeof(int)));
    CKC(cudaMemsetAsync(step.p, 0, sizeof(int), st));
    bf16 *ap[3] = {act[0].h(), act[1].h(), act[2].h()}, *apT[3] = {actT[0].h(), actT[1].h(), actT[2].h()};
    float *zp[3] = {Z[0].f(), Z[1].f(), Z[2].f()};
    // one training step on rows [b*B, (b+1)*B) of the shuffled epoch data
    auto train_step = [&](int b) -> cudaError_t {
        cudaError_t e;
        const bf16 *xb = Xe.h() + (size_t)b * B * m.Dp;
        if ((e = hidden_forward(st, m, W.f(), Wbf.h(), xb, B, ap, zp, apT, derr.i())) != cudaSuccess) return e;
        out_kernel<<<(B * 32 + 255) / 256, 256, 0, st>>>(B, H, ap[2], W.f() + m.woff[3], W.f() + m.boff[3],
                                                         ye.f() + (size_t)b * B, out.f(), dY.f(), loss.d(), step.i());
        out_grad_kernel<<<H + 1, 128, 0, st>>>(B, H, apT[2], dY.f(), G.f() + m.woff[3], G.f() + m.boff[3]);
        dz_out_kernel<<<dim3((B + 31) / 32, (H + 31) / 32), dim3(32, 8), 0, st>>>(
            B, H, dY.f(), W.f() + m.woff[3], zp[2], dZ[0].h(), dZT[0].h());
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        int cur = 0;
        for (int l = 2; l >= 0; --l) {
            // dW_l = act_{l-1}^T . dZ_l  (the batch is the contracted dimension)
            fpk::TcGemm g{};
            g.M = m.fin[l], g.N = H, g.K = B;
            if (l == 0) {
                g.A = XeT.h() + (size_t)b * B, g.lda = (int)NE;
            } else {
                g.A = apT[l - 1], g.lda = B;
            }
            g.Bt = dZT[cur].h(), g.ldb = B;
            g.mode = 0;
            g.Cf = G.f() + m.woff[l], g.ldcf = H;
            g.err = derr.i();
            if ((e = fpk::launch_tc_gemm(g, st)) != cudaSuccess) return e;
            rowsum_kernel<<<(H * 32 + 255) / 256, 256, 0, st>>>(H, B, dZT[cur].h(), G.f() + m.boff[l]);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            if (l > 0) {
                // dZ_{l-1} = (dZ_l . W_l^T) * GELU'(Z_{l-1})
                fpk::TcGemm h{};
                h.M = B, h.N = m.fin[l], h.K = H;
                h.A = dZ[cur].h(), h.lda = H;
                h.Bt = Wbf.h() + m.wboff[l], h.ldb = H;
                h.mode = 2;
                h.Z = zp[l - 1], h.ldz = H;
                h.Cb = dZ[cur ^ 1].h(), h.ldcb = H;
                h.Cbt = dZT[cur ^ 1].h(), h.ldct = B;
                h.err = derr.i();
                if ((e = fpk::launch_tc_gemm(h, st)) != cudaSuccess) return e;
                cur ^= 1;
            }
        }
        adam_kernel<<<1024, 256, 0, st>>>((long long)m.total, W.f(), G.f(), Mm.f(), Vv.f(), lr, 0.9f, 0.999f,
                                          step.i(), 1, wc);
        return cudaGetLastError();
    };
    std::mt19937_64 prng(d.seed ^ 0x9E3779B97F4A7C15ULL);
    std::vector<int> hperm(NT);
    double last_loss = 0;
    for (int ep = 0; ep < epochs; ++ep) {
        std::iota(hperm.begin(), hperm.end(), 0);
        std::shuffle(hperm.begin(), hperm.end(), prng);
        CKC(cudaMemcpyAsync(perm.p, hperm.data(), NT * sizeof(int), cudaMemcpyHostToDevice, st));
        gather_rows_kernel<<<1024, 256, 0, st>>>((int)NE, m.Dp, perm.i(), X.h(), Xe.h(), y.f(), ye.f());
        transpose_bf16_kernel<<<dim3((unsigned)((NE + 31) / 32), (m.D + 31) / 32), dim3(32, 8), 0, st>>>(
            (int)NE, m.D, Xe.h(), m.Dp, XeT.h(), (int)NE);
        CKC(cudaGetLastError());
        CKC(cudaMemsetAsync(loss.p, 0, sizeof(double), st));
        // step 0 runs directly (it also sets the GEMM kernel's attributes);
        // steps 1..nb-1 are captured in the first epoch and replayed after
        CKC(train_step(0));
        if (nb > 1) {
            if (!gexec) {
                CKC(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
                cudaError_t ce = cudaSuccess;
                for (int b = 1; b < nb && ce == cudaSuccess; ++b) ce = train_step(b);
                cudaError_t ee = cudaStreamEndCapture(st, &graph);
                CKC(ce);
                CKC(ee);
                CKC(cudaGraphInstantiate(&gexec, graph, 0));
            }
            CKC(cudaGraphLaunch(gexec, st));
        }
        // the host buffer holds this epoch's permutation until the copy has run
        double lh = 0;
        CKC(cudaMemcpyAsync(&lh, loss.p, sizeof(double), cudaMemcpyDeviceToHost, st));
        CKC(cudaStreamSynchronize(st));
        last_loss = lh / nb;
    }
    CKS(check_err());
    res->train_loss = last_loss;
    // ---- 3. correction pairs: exact f and the surrogate g on the same pairs
    Buf Xc, gc, fc, sums, big[3];
    const size_t chunk = 1 << 16;
    CKC(Xc.alloc(chunk * m.Dp * sizeof(bf16)));
    CKC(cudaMemsetAsync(Xc.p, 0, chunk * m.Dp * sizeof(bf16), st));
    CKC(gc.alloc(chunk * sizeof(float)));
    CKC(sums.alloc(4 * sizeof(double)));
    bf16 *cap[3];
    for (int l = 0; l < 3; ++l) {
        CKC(big[l].alloc(chunk * H * sizeof(bf16)));
        cap[l] = big[l].h();
    }
    auto surrogate = [&](uint64_t f0, int cnt) -> cudaError_t {
        features_kernel<<<1024, 256, 0, st>>>(d.seed, f0, cnt, n, L, Xc.h(), m.Dp);
        cudaError_t e = hidden_forward(st, m, W.f(), Wbf.h(), Xc.h(), cnt, cap, nullptr, nullptr, derr.i());
        if (e != cudaSuccess) return e;
        out_kernel<<<(unsigned)(((size_t)cnt * 32 + 255) / 256), 256, 0, st>>>(
            cnt, H, cap[2], W.f() + m.woff[3], W.f() + m.boff[3], nullptr, gc.f(), nullptr, nullptr, nullptr);
        gtrans_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(cnt, gc.f(), (float)t_mu, (float)t_sigma);
        return cudaGetLastError();
    };
    // the control-variate coefficient beta = Cov(f, g) / Var(g) on the training pairs
    // (their traces are still in dtr); the correction and surrogate pairs are disjoint
    // from them, so beta g is a fixed function there and the estimate stays unbiased
    double beta = 1.0;
    {
        CKC(cudaMemsetAsync(sums.p, 0, 4 * sizeof(double), st));
        for (uint64_t c0 = 0; c0 < NT; c0 += chunk) {
            const int cnt = (int)std::min<uint64_t>(chunk, NT - c0);
            CKC(surrogate(f_train + c0, cnt));
            beta_sums_kernel<<<256, 256, 0, st>>>(cnt, gc.f(), dtr + 2 * c0, sums.d());
            CKC(cudaGetLastError());
        }
        double bs[4];
        CKC(cudaMemcpyAsync(bs, sums.p, sizeof bs, cudaMemcpyDeviceToHost, st));
        CKC(cudaStreamSynchronize(st));
        const double Nt = (double)NT, vg = bs[1] - bs[0] * bs[0] / Nt, cfg_ = bs[2] - bs[0] * bs[3] / Nt;
        if (vg > 0 && std::isfinite(cfg_ / vg)) beta = cfg_ / vg;
    }
    res->target_scale = beta;
    res->gpu_seconds_train = elapsed();   // features, training and the coefficient fit
    CKS(fpk::cv_trace(ens, f_corr, NC, &dtr, &ms_trace));
    res->gpu_seconds_exact += ms_trace * 1e-3;
    CKC(join_user());
    CKC(cudaEventRecord(e0, st));
    CKC(fc.alloc(NC * sizeof(double)));
    abs4_kernel<<<(unsigned)((NC + 255) / 256), 256, 0, st>>>(dtr, (int)NC, 1.0, nullptr, fc.d());
    if (cfg->f_correct) CKC(cudaMemcpyAsync(cfg->f_correct, fc.d(), NC * sizeof(double), cudaMemcpyDefault, st));
    Buf gx;   // per-pair g for the optional exports
    if (cfg->g_correct || cfg->g_surrogate) CKC(gx.alloc(chunk * sizeof(double)));
    auto export_g = [&](double *dst, int cnt) -> cudaError_t {
        if (!dst) return cudaSuccess;
        gexport_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(cnt, gc.f(), beta, gx.d());
        cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? cudaMemcpyAsync(dst, gx.d(), cnt * sizeof(double), cudaMemcpyDefault, st) : e;
    };
    CKC(cudaMemsetAsync(sums.p, 0, 4 * sizeof(double), st));
    for (uint64_t c0 = 0; c0 < NC; c0 += chunk) {
        const int cnt = (int)std::min<uint64_t>(chunk, NC - c0);
        CKC(surrogate(f_corr + c0, cnt));
        cv_sums_kernel<<<256, 256, 0, st>>>(cnt, gc.f(), beta, fc.d() + c0, sums.d());
        CKC(cudaGetLastError());
        CKC(export_g(cfg->g_correct ? cfg->g_correct + c0 : nullptr, cnt));
    }
    double sc[4];
    CKC(cudaMemcpyAsync(sc, sums.p, sizeof sc, cudaMemcpyDeviceToHost, st));
    CKC(cudaStreamSynchronize(st));
    const double Nc = (double)NC;
    const double mean_fg = sc[0] / Nc, var_fg = (sc[1] - sc[0] * sc[0] / Nc) / (Nc - 1);
    const double mean_f = sc[2] / Nc, var_f = (sc[3] - sc[2] * sc[2] / Nc) / (Nc - 1);
    // ---- 4. surrogate pairs
    CKC(cudaMemsetAsync(sums.p, 0, 4 * sizeof(double), st));
    for (uint64_t c0 = 0; c0 < MS; c0 += chunk) {
        const int cnt = (int)std::min<uint64_t>(chunk, MS - c0);
        CKC(surrogate(f_sur + c0, cnt));
        cv_sums_kernel<<<256, 256, 0, st>>>(cnt, gc.f(), beta, nullptr, sums.d());
        CKC(cudaGetLastError());
        CKC(export_g(cfg->g_surrogate ? cfg->g_surrogate + c0 : nullptr, cnt));
    }
    CKC(cudaMemcpyAsync(sc, sums.p, sizeof sc, cudaMemcpyDeviceToHost, st));
    CKC(cudaStreamSynchronize(st));
    CKS(check_err());
    const double Ms = (double)MS;
    const double mean_g = sc[0] / Ms, var_g = (sc[1] - sc[0] * sc[0] / Ms) / (Ms - 1);
    res->gpu_seconds_surrogate = elapsed();
    res->F2 = mean_g + mean_fg;
    res->stderr_ = std::sqrt(var_g / Ms + var_fg / Nc);
    res->F2_plain = mean_f;
    res->stderr_plain = std::sqrt(var_f / Nc);
    res->var_f = var_f;
    res->var_f_minus_g = var_fg;
    res->var_g = var_g;
    cleanup();
#undef CKC
#undef CKS
    return FP_OK;
}
