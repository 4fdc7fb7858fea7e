// peaks.cu -- measured arithmetic peaks of the device (roofline denominators).
//
// Each microbenchmark keeps one pipe busy with independent work and nothing
// else: FP32 fused multiply-adds (scalar fma.rn.f32 and packed fma.rn.f32x2),
// FP64 fused multiply-adds, and back-to-back tcgen05.mma of kind::tf32 and
// kind::f16 (BF16) on operands resident in shared memory, accumulating in
// tensor memory.  The ALU kernels run 2048 threads per SM with 8 independent
// accumulators per thread; the tensor kernels one CTA per SM whose elected
// lane issues the MMAs.  CTA 0 samples clock64 and the global timer at both
// ends, so the SM clock during the run is reported beside the rate.
#include <cuda_runtime.h>

#include <cstdint>

#include "fp.h"
#include "kernels.h"

namespace fpk {
namespace {

constexpr uint64_t kPeakWaitNs = 2000000000ull;   // 2 s

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Poll an mbarrier phase until it completes or `limit_ns` of global time pass.
__device__ __forceinline__ bool mbar_wait_ns(uint32_t mbar, uint32_t phase, uint64_t limit_ns) {
    const uint64_t t0 = gtimer();
    for (;;) {
        uint32_t d;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(d)
            : "r"(mbar), "r"(phase)
            : "memory");
        if (d) return true;
        if (gtimer() - t0 > limit_ns) return false;
    }
}

struct ClockRec {
    unsigned long long c0, c1, t0, t1;
};

__device__ __forceinline__ void clock_begin(ClockRec *rec) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        rec->t0 = gtimer();
        rec->c0 = clock64();
    }
}
__device__ __forceinline__ void clock_end(ClockRec *rec) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        rec->c1 = clock64();
        rec->t1 = gtimer();
    }
}

__global__ void __launch_bounds__(256) ffma_kernel(int iters, float x, float y, float *sink, ClockRec *rec) {
    clock_begin(rec);
    float a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = (float)threadIdx.x * 1e-3f + (float)j;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int j = 0; j < 8; ++j) a[j] = fmaf(a[j], x, y);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += a[j];
    if (s == 1234.5f) sink[threadIdx.x] = s;   // keeps the chains alive
    __syncthreads();
    clock_end(rec);
}

__device__ __forceinline__ void ffma2_inplace(float2 &a, float2 b, float2 c) {
    asm("{\n\t.reg .b64 ra, rb, rc;\n\t"
        "mov.b64 ra, {%0, %1};\n\tmov.b64 rb, {%2, %3};\n\tmov.b64 rc, {%4, %5};\n\t"
        "fma.rn.f32x2 ra, ra, rb, rc;\n\tmov.b64 {%0, %1}, ra;\n\t}"
        : "+f"(a.x), "+f"(a.y)
        : "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
}

__global__ void __launch_bounds__(256) ffma2_kernel(int iters, float x, float y, float *sink, ClockRec *rec) {
    clock_begin(rec);
    float2 a[8];
    const float2 b = make_float2(x, x), c = make_float2(y, y);
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = make_float2((float)threadIdx.x * 1e-3f + (float)j, (float)j);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int j = 0; j < 8; ++j) ffma2_inplace(a[j], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += a[j].x + a[j].y;
    if (s == 1234.5f) sink[threadIdx.x] = s;
    __syncthreads();
    clock_end(rec);
}

__global__ void __launch_bounds__(256) dfma_kernel(int iters, double x, double y, float *sink, ClockRec *rec) {
    clock_begin(rec);
    double a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = (double)threadIdx.x * 1e-3 + (double)j;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int j = 0; j < 8; ++j) a[j] = fma(a[j], x, y);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += a[j];
    if (s == 1234.5) sink[threadIdx.x] = (float)s;
    __syncthreads();
    clock_end(rec);
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// K-major 128-byte-swizzled shared-memory descriptor (rows of 128 bytes, 8-row
// groups 1024 bytes apart, base 1024-byte aligned).
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
           (2ull << 61);
}

// Back-to-back MMAs of one shape on fixed operands: 128 x 256 outputs, one
// 128-byte row of K per operand row (K = 32 TF32 or 64 BF16 per 4 MMAs).
// tf32: kind::tf32 (A, B format 2), else kind::f16 with BF16 (format 1).
template <bool TF32>
__global__ void __launch_bounds__(128, 1) tc_peak_kernel(int iters, int *err, ClockRec *rec) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t done;
    __shared__ uint32_t taddr_sh;
    __shared__ int bad;
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x;
    // operands: A 128 rows x 128 B, B 256 rows x 128 B, small finite values
    uint32_t *w = (uint32_t *)smem;
    for (int i = tid; i < (128 + 256) * 32; i += 128)
        w[i] = TF32 ? 0x3C000000u /* 2^-7 */ : 0x3C003C00u /* BF16 pair (2^-7, 2^-7) */;
    if (tid == 0) {
        bad = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&done)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (tid < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_addr(&taddr_sh)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic-proxy writes -> MMA reads
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    clock_begin(rec);
    const uint32_t taddr = taddr_sh;
    if (tid == 0) {
        const uint32_t sa = smem_addr(smem), sb = sa + 128 * 128;
        // dtype F32 (bits 4-5), A/B format at bits 7-9 / 10-12, N >> 3 at 17, M >> 4 at 24
        const uint32_t fmt = TF32 ? 2u : 1u;
        const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((256u >> 3) << 17) | ((128u >> 4) << 24);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const uint64_t ad = desc_sw128(sa + kk * 32), bd = desc_sw128(sb + kk * 32);
                const uint32_t acc = (it > 0 || kk > 0) ? 1u : 0u;
                if (TF32)
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(taddr),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                else
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(taddr),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_addr(&done))
                     : "memory");
    }
    __syncwarp();
    // every thread waits for the last commit, bounded by the global timer; on
    // a timeout the flag is raised and a second bounded wait drains the MMAs
    // still in flight before the tensor memory is released
    bool ok = mbar_wait_ns(smem_addr(&done), 0u, kPeakWaitNs);
    if (!ok) {
        bad = 1;
        mbar_wait_ns(smem_addr(&done), 0u, kPeakWaitNs);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    clock_end(rec);
    if (bad && tid == 0) atomicExch(err, 1);
    if (tid < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(taddr));
}

}  // namespace
}  // namespace fpk

extern "C" fp_status fp_measure_peak(int32_t which, int32_t iters, void *cuda_stream, double *out) {
    using namespace fpk;
    if (!out) return api_fail(FP_ERR_ARG, "out is NULL");
    if (which < FP_PEAK_FFMA || which > FP_PEAK_TC_BF16) return api_fail(FP_ERR_ARG, "unknown peak kind");
    if (iters < 0) return api_fail(FP_ERR_ARG, "iters < 0");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return api_fail(FP_ERR_CUDA, cudaGetErrorString(e));
    const bool tc = which == FP_PEAK_TC_TF32 || which == FP_PEAK_TC_BF16;
    if (iters == 0) iters = tc ? 4096 : (which == FP_PEAK_DFMA ? 512 : 4096);
    float *sink = nullptr;
    ClockRec *rec = nullptr;
    int *derr = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ClockRec hrec{};
    int herr = 0;
    float ms = 0.f;
    double flops = 0.0;
    const size_t tc_smem = (size_t)(128 + 256) * 128 + 1024;
    e = cudaMallocAsync((void **)&sink, 256 * sizeof(float), st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&rec, sizeof(ClockRec), st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&derr, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(derr, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess && tc) {
        e = cudaFuncSetAttribute(which == FP_PEAK_TC_TF32 ? tc_peak_kernel<true> : tc_peak_kernel<false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem);
    }
    // one untimed launch (clocks up, code loaded), then the timed one
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
        if (rep == 1) e = cudaEventRecord(e0, st);
        if (e != cudaSuccess) break;
        switch (which) {
            case FP_PEAK_FFMA:
                ffma_kernel<<<sms * 8, 256, 0, st>>>(iters, 0.999999f, 1e-7f, sink, rec);
                flops = 2.0 * 128 * (double)iters * 256 * sms * 8;
                break;
            case FP_PEAK_FFMA2:
                ffma2_kernel<<<sms * 8, 256, 0, st>>>(iters, 0.999999f, 1e-7f, sink, rec);
                flops = 2.0 * 2 * 64 * (double)iters * 256 * sms * 8;
                break;
            case FP_PEAK_DFMA:
                dfma_kernel<<<sms * 8, 256, 0, st>>>(iters, 0.999999, 1e-7, sink, rec);
                flops = 2.0 * 32 * (double)iters * 256 * sms * 8;
                break;
            case FP_PEAK_TC_TF32:
                tc_peak_kernel<true><<<sms, 128, tc_smem, st>>>(iters, derr, rec);
                flops = 2.0 * 128 * 256 * 32 * (double)iters * sms;
                break;
            default:
                tc_peak_kernel<false><<<sms, 128, tc_smem, st>>>(iters, derr, rec);
                flops = 2.0 * 128 * 256 * 64 * (double)iters * sms;
                break;
        }
        e = cudaGetLastError();
        if (e == cudaSuccess && rep == 1) e = cudaEventRecord(e1, st);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hrec, rec, sizeof hrec, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, derr, sizeof herr, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (sink) cudaFreeAsync(sink, st);
    if (rec) cudaFreeAsync(rec, st);
    if (derr) cudaFreeAsync(derr, st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return api_fail(FP_ERR_CUDA, cudaGetErrorString(e));
    if (herr) return api_fail(FP_ERR_TIMEOUT, "peak microbenchmark: the tensor-core wait ran out");
    const double dt = (double)(hrec.t1 - hrec.t0), dc = (double)(hrec.c1 - hrec.c0);
    const double mhz = dt > 0 ? dc / dt * 1e3 : 0.0;
    out[0] = ms > 0 ? flops / (ms * 1e-3) / 1e12 : 0.0;
    out[1] = ms;
    out[2] = mhz;
    out[3] = mhz > 0 ? out[0] * 1e12 / (mhz * 1e6) / sms : 0.0;   // flops per clock per SM
    out[4] = sms;
    return FP_OK;
}
