// cv.cu -- learned control variate for F^(2) of single-depth HEA ensembles.
//
// A small MLP g maps a pair's circuit angles to a prediction of |Tr|^4.  It is
// trained on exactly contracted pairs, evaluated on many cheap surrogate
// pairs, and corrected on fresh exactly contracted pairs:
//     F^(2) ~= mean_M g(x) + mean_N (f(x) - g(x)),   f = |Tr(U^dagger V)|^4,
// with the three pair ranges disjoint, so the estimate stays unbiased for any
// g; its variance is Var(g)/M + Var(f - g)/N.  The plain estimator mean_N f on
// the correction pairs is reported beside it (it judges the variance
// reduction).  The paper has no control variate; F^(2) itself is the paper's
// (Sec. "Frame potential", Sec. "Algorithm description").
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <vector>

#include "fp.h"
#include "kernels.h"



namespace {

using fpk::U64x4;
using fpk::philox;

// features: u in [0,1) of every angle of both circuits, mapped to 2u - 1;
// index ((w * L + t) * n + q) * 2 + a  (a = 0: theta, 1: phi)
__global__ void features_kernel(uint64_t seed, uint64_t first, int count, int n, int L, float *X) {
    const int D = 4 * n * L;
    const long long total = (long long)count * (2 * L * n);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int p = (int)(i / (2 * L * n));
        const int r = (int)(i % (2 * L * n));
        const int w = r / (L * n), t = (r / n) % L, q = r % n;
        U64x4 x = philox(seed, (uint64_t)t, (uint64_t)q, first + p, (uint64_t)w);
        float *o = X + (size_t)p * D + (size_t)((w * L + t) * n + q) * 2;
        o[0] = 2.0f * (float)((double)(x.x[0] >> 11) * 0x1.0p-53) - 1.0f;
        o[1] = 2.0f * (float)((double)(x.x[1] >> 11) * 0x1.0p-53) - 1.0f;
    }
}

__global__ void abs4_kernel(const double *tr, int count, double scale, float *y, double *f) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    double a2 = tr[2 * i] * tr[2 * i] + tr[2 * i + 1] * tr[2 * i + 1];
    if (f) f[i] = a2 * a2;
    if (y) y[i] = (float)(a2 * a2 * scale);
}

// C[M x N] = A[M x K] B[K x N] (+ bias) with general strides; optional GELU.
// A(i,k) = A[i*sar + k*sac], B(k,j) = B[k*sbr + j*sbc].  Z (pre-activation) is
// stored when non-null.  accumulate: C += product.
constexpr int TBM = 64, TBN = 64, TBK = 16;
__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, const float *__restrict__ A, long long sar,
                                                   long long sac, const float *__restrict__ B, long long sbr,
                                                   long long sbc, float *__restrict__ C, int ldc,
                                                   const float *__restrict__ bias, int gelu, float *__restrict__ Z,
                                                   int accumulate) {
    __shared__ float As[TBK][TBM + 1], Bs[TBK][TBN + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int i0 = blockIdx.y * TBM, j0 = blockIdx.x * TBN;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += TBK) {
        for (int e = threadIdx.x; e < TBK * TBM; e += 256) {
            int kk = e / TBM, ii = e % TBM;
            int gi = i0 + ii, gk = k0 + kk;
            As[kk][ii] = (gi < M && gk < K) ? A[gi * sar + gk * sac] : 0.f;
        }
        for (int e = threadIdx.x; e < TBK * TBN; e += 256) {
            int kk = e / TBN, jj = e % TBN;
            int gj = j0 + jj, gk = k0 + kk;
            Bs[kk][jj] = (gj < N && gk < K) ? B[gk * sbr + gj * sbc] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TBK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[kk][ty * 4 + r];
#pragma unroll
            for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx * 4 + c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            int gi = i0 + ty * 4 + r, gj = j0 + tx * 4 + c;
            if (gi >= M || gj >= N) continue;
            float v = acc[r][c] + (bias ? bias[gj] : 0.f);
            if (accumulate) v += C[(size_t)gi * ldc + gj];
            if (Z) Z[(size_t)gi * ldc + gj] = v;
            if (gelu) v = 0.5f * v * (1.0f + erff(v * 0.70710678f));
            C[(size_t)gi * ldc + gj] = v;
        }
}

// dZ = dA * gelu'(Z)
__global__ void gelu_back_kernel(long long n, const float *Z, const float *dA, float *dZ) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float z = Z[i];
        float d = 0.5f * (1.0f + erff(z * 0.70710678f)) + z * 0.39894228f * expf(-0.5f * z * z);
        dZ[i] = dA[i] * d;
    }
}

// dY = 2 (Y - y) / B  for a [B x 1] output
__global__ void mse_grad_kernel(int B, const float *Y, const float *y, float *dY, double *loss) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B) return;
    float e = Y[i] - y[i];
    dY[i] = 2.0f * e / (float)B;
    atomicAdd(loss, (double)e * (double)e / (double)B);
}

// db[j] = sum_i dZ[i, j]
__global__ void colsum_kernel(int B, int N, const float *dZ, float *db) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    float s = 0.f;
    for (int i = 0; i < B; ++i) s += dZ[(size_t)i * N + j];
    db[j] = s;
}

__global__ void adam_kernel(long long n, float *w, const float *g, float *m, float *v, float lr, float b1, float b2,
                            float c1, float c2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float gi = g[i];
        float mi = b1 * m[i] + (1.f - b1) * gi, vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
    }
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
};

struct Mlp {
    int D, H;
    // layers: 0: D->H, 1: H->H, 2: H->H, 3: H->1
    int fin[4], fout[4];
    size_t woff[4], boff[4], total;
};

Mlp make_mlp(int D, int H) {
    Mlp m;
    m.D = D;
    m.H = H;
    int in[4] = {D, H, H, H}, out[4] = {H, H, H, 1};
    size_t o = 0;
    for (int l = 0; l < 4; ++l) {
        m.fin[l] = in[l];
        m.fout[l] = out[l];
        m.woff[l] = o;
        o += (size_t)in[l] * out[l];
        m.boff[l] = o;
        o += out[l];
    }
    m.total = o;
    return m;
}

cudaError_t gemm(cudaStream_t st, int M, int N, int K, const float *A, long long sar, long long sac, const float *B,
                 long long sbr, long long sbc, float *C, int ldc, const float *bias, int gelu, float *Z, int accumulate) {
    dim3 grid((N + TBN - 1) / TBN, (M + TBM - 1) / TBM);
    gemm_kernel<<<grid, 256, 0, st>>>(M, N, K, A, sar, sac, B, sbr, sbc, C, ldc, bias, gelu, Z, accumulate);
    return cudaGetLastError();
}

// forward pass of a batch: acts[l] = activation after layer l (acts[-1] = X);
// zs[l] = pre-activations (layers 0..2); out = [B x 1]
cudaError_t forward(cudaStream_t st, const Mlp &m, const float *W, const float *X, int B, float *const *acts,
                    float *const *zs, float *out) {
    const float *in = X;
    for (int l = 0; l < 4; ++l) {
        float *dst = l < 3 ? acts[l] : out;
        cudaError_t e = gemm(st, B, m.fout[l], m.fin[l], in, m.fin[l], 1, W + m.woff[l], m.fout[l], 1, dst, m.fout[l],
                             W + m.boff[l], l < 3 ? 1 : 0, l < 3 && zs ? zs[l] : nullptr, 0);
        if (e != cudaSuccess) return e;
        in = dst;
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
    const int n = d.n, L = d.depth_min, D = 4 * n * L;
    const int H = cfg->hidden > 0 ? cfg->hidden : 256;
    const int epochs = cfg->epochs > 0 ? cfg->epochs : 20;
    const int B = cfg->batch > 0 ? cfg->batch : 512;
    const float lr = cfg->lr > 0 ? (float)cfg->lr : 1e-3f;
    const uint64_t NT = cfg->n_train, NC = cfg->n_correct, MS = cfg->m_surrogate;
    if (NT < (uint64_t)B || NC < 2 || MS < 2 || H > 1024)
        return fpk::api_fail(FP_ERR_ARG, "need n_train >= batch, n_correct >= 2, m_surrogate >= 2, hidden <= 1024");
    cudaStream_t st = fpk::ens_stream(ens);
    std::memset(res, 0, sizeof *res);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto elapsed = [&]() {
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms * 1e-3;
    };
#define CKC(call)                                                                          \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            cudaEventDestroy(e0);                                                          \
            cudaEventDestroy(e1);                                                          \
            return fpk::api_fail(e_ == cudaErrorMemoryAllocation ? FP_ERR_OOM : FP_ERR_CUDA,    \
                            cudaGetErrorString(e_));                                       \
        }                                                                                  \
    } while (0)
#define CKS(call)                                                                          \
    do {                                                                                   \
        fp_status s_ = (call);                                                             \
        if (s_ != FP_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); return s_; }        \
    } while (0)

    const uint64_t f_train = cfg->first, f_corr = f_train + NT, f_sur = f_corr + NC;
    // ---- 1. exact contractions of the training pairs -> targets
    Buf X, y, f;
    CKC(X.alloc(NT * D * sizeof(float)));
    CKC(y.alloc(NT * sizeof(float)));
    float ms_trace = 0;
    double *dtr = nullptr;
    CKS(fpk::cv_trace(ens, f_train, NT, &dtr, &ms_trace));
    res->gpu_seconds_exact += ms_trace * 1e-3;
    CKC(cudaEventRecord(e0, st));
    {
        std::vector<double> h(2 * NT);
        CKC(cudaMemcpyAsync(h.data(), dtr, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        CKC(cudaStreamSynchronize(st));
        double mean = 0;
        for (uint64_t i = 0; i < NT; ++i) {
            double a2 = h[2 * i] * h[2 * i] + h[2 * i + 1] * h[2 * i + 1];
            mean += a2 * a2;
        }
        mean /= (double)NT;
        res->target_scale = mean > 0 ? mean : 1.0;
    }
    abs4_kernel<<<(unsigned)((NT + 255) / 256), 256, 0, st>>>(dtr, (int)NT, 1.0 / res->target_scale, y.f(), nullptr);
    CKC(cudaGetLastError());
    features_kernel<<<1024, 256, 0, st>>>(d.seed, f_train, (int)NT, n, L, X.f());
    CKC(cudaGetLastError());
    // ---- 2. training (Adam on the mean squared error of |Tr|^4 / mean)
    Mlp m = make_mlp(D, H);
    Buf W, G, Mm, Vv, acts[3], zs[3], dA, dZ, out, dY, loss;
    CKC(W.alloc(m.total * sizeof(float)));
    CKC(G.alloc(m.total * sizeof(float)));
    CKC(Mm.alloc(m.total * sizeof(float)));
    CKC(Vv.alloc(m.total * sizeof(float)));
    CKC(cudaMemsetAsync(Mm.p, 0, m.total * sizeof(float), st));
    CKC(cudaMemsetAsync(Vv.p, 0, m.total * sizeof(float), st));
    {
        std::mt19937_64 rng(d.seed ^ 0x5DEECE66DULL);
        std::vector<float> w(m.total, 0.f);
        for (int l = 0; l < 4; ++l) {
            std::normal_distribution<float> nd(0.f, std::sqrt(2.0f / (float)m.fin[l]));
            for (size_t i = 0; i < (size_t)m.fin[l] * m.fout[l]; ++i) w[m.woff[l] + i] = nd(rng);
        }
        CKC(cudaMemcpyAsync(W.p, w.data(), w.size() * sizeof(float), cudaMemcpyHostToDevice, st));
        CKC(cudaStreamSynchronize(st));
    }
    const int HB = std::max(H, D);
    for (int l = 0; l < 3; ++l) {
        CKC(acts[l].alloc((size_t)B * H * sizeof(float)));
        CKC(zs[l].alloc((size_t)B * H * sizeof(float)));
    }
    CKC(dA.alloc((size_t)B * HB * sizeof(float)));
    CKC(dZ.alloc((size_t)B * HB * sizeof(float)));
    CKC(out.alloc((size_t)B * sizeof(float)));
    CKC(dY.alloc((size_t)B * sizeof(float)));
    CKC(loss.alloc(sizeof(double)));
    float *ap[3] = {acts[0].f(), acts[1].f(), acts[2].f()}, *zp[3] = {zs[0].f(), zs[1].f(), zs[2].f()};
    const int nb = (int)(NT / B);
    int step = 0;
    double last_loss = 0;
    for (int ep = 0; ep < epochs; ++ep) {
        CKC(cudaMemsetAsync(loss.p, 0, sizeof(double), st));
        const int shift = (int)((ep * 7919LL) % nb);
        for (int bi = 0; bi < nb; ++bi) {
            const int b = (bi + shift) % nb;
            const float *xb = X.f() + (size_t)b * B * D;
            const float *yb = y.f() + (size_t)b * B;
            CKC(forward(st, m, W.f(), xb, B, ap, zp, out.f()));
            mse_grad_kernel<<<(B + 255) / 256, 256, 0, st>>>(B, out.f(), yb, dY.f(), loss.d());
            // layer 3 (H -> 1): dW3 = A2^T dY, db3 = sum dY, dA2 = dY W3^T
            const float *dcur = dY.f();
            int ncur = 1;
            for (int l = 3; l >= 0; --l) {
                const float *ain = l == 0 ? xb : ap[l - 1];
                const int fin = m.fin[l], fout = m.fout[l];
                // dW = ain^T [fin x B] . dcur [B x fout]
                CKC(gemm(st, fin, fout, B, ain, 1, fin, dcur, ncur, 1, G.f() + m.woff[l], fout, nullptr, 0, nullptr, 0));
                colsum_kernel<<<(fout + 127) / 128, 128, 0, st>>>(B, fout, dcur, G.f() + m.boff[l]);
                if (l > 0) {
                    // dA_{l-1} = dcur [B x fout] . W^T [fout x fin]
                    CKC(gemm(st, B, fin, fout, dcur, ncur, 1, W.f() + m.woff[l], 1, fout, dA.f(), fin, nullptr, 0,
                             nullptr, 0));
                    // dZ_{l-1} = dA * gelu'(Z_{l-1}); dZ is read again only by the next layer
                    gelu_back_kernel<<<1024, 256, 0, st>>>((long long)B * fin, zp[l - 1], dA.f(), dZ.f());
                    dcur = dZ.f();
                    ncur = fin;
                }
            }
            ++step;
            const float b1 = 0.9f, b2 = 0.999f;
            adam_kernel<<<1024, 256, 0, st>>>((long long)m.total, W.f(), G.f(), Mm.f(), Vv.f(), lr, b1, b2,
                                              1.f - std::pow(b1, (float)step), 1.f - std::pow(b2, (float)step));
            CKC(cudaGetLastError());
        }
        double lh = 0;
        CKC(cudaMemcpyAsync(&lh, loss.p, sizeof(double), cudaMemcpyDeviceToHost, st));
        CKC(cudaStreamSynchronize(st));
        last_loss = lh / nb;
    }
    res->train_loss = last_loss;
    res->gpu_seconds_train = elapsed();
    // ---- 3. correction pairs: exact f and the surrogate g on the same pairs
    Buf Xc, gc, fc, sums;
    const size_t chunk = 1 << 16;
    CKC(Xc.alloc(chunk * D * sizeof(float)));
    CKC(gc.alloc(chunk * sizeof(float)));
    CKC(sums.alloc(4 * sizeof(double)));
    float *cap[3], *dummy = nullptr;
    Buf big[3];
    for (int l = 0; l < 3; ++l) {
        CKC(big[l].alloc(chunk * H * sizeof(float)));
        cap[l] = big[l].f();
    }
    (void)dummy;
    CKS(fpk::cv_trace(ens, f_corr, NC, &dtr, &ms_trace));
    res->gpu_seconds_exact += ms_trace * 1e-3;
    CKC(cudaEventRecord(e0, st));
    CKC(fc.alloc(NC * sizeof(double)));
    abs4_kernel<<<(unsigned)((NC + 255) / 256), 256, 0, st>>>(dtr, (int)NC, 1.0, nullptr, fc.d());
    CKC(cudaMemsetAsync(sums.p, 0, 4 * sizeof(double), st));
    for (uint64_t c0 = 0; c0 < NC; c0 += chunk) {
        const int cnt = (int)std::min<uint64_t>(chunk, NC - c0);
        features_kernel<<<1024, 256, 0, st>>>(d.seed, f_corr + c0, cnt, n, L, Xc.f());
        CKC(forward(st, m, W.f(), Xc.f(), cnt, cap, nullptr, gc.f()));
        cv_sums_kernel<<<256, 256, 0, st>>>(cnt, gc.f(), res->target_scale, fc.d() + c0, sums.d());
        CKC(cudaGetLastError());
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
        features_kernel<<<1024, 256, 0, st>>>(d.seed, f_sur + c0, cnt, n, L, Xc.f());
        CKC(forward(st, m, W.f(), Xc.f(), cnt, cap, nullptr, gc.f()));
        cv_sums_kernel<<<256, 256, 0, st>>>(cnt, gc.f(), res->target_scale, nullptr, sums.d());
        CKC(cudaGetLastError());
    }
    CKC(cudaMemcpyAsync(sc, sums.p, sizeof sc, cudaMemcpyDeviceToHost, st));
    CKC(cudaStreamSynchronize(st));
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
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
#undef CKC
#undef CKS
    return FP_OK;
}
