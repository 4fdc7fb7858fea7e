// static_scratch.cu -- brickwork traces without any device allocation.
//
// Some callers cannot allocate device memory at the point where they want
// traces: plugins hosted by a framework whose memory pool already owns the
// device memory (a cudaMalloc there can fail or fragment the pool), and
// latency-bound loops that must never block inside the allocator.  For them
// fp_trace_brick_static runs the brickwork path (sampler, maps, shared-memory
// sweep and meet) with every intermediate buffer carved out of one fixed array
// compiled into this library.  The array is FP_STATIC_SCRATCH_BYTES large and
// every GPU that loads the library holds it until the process exits.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <mutex>

#include "brick.h"
#include "fp.h"
#include "kernels.h"

namespace {

// The scratch: raw gates, gate maps, pair records and (FP64, 12-bit
// boundaries) the left boundaries of one call.  Every kernel writes what it
// later reads, so nothing here has to start at zero; calls that overlap on the
// GPU (different streams, no ordering between them) race on it.
static __device__ __align__(256) unsigned char g_scratch[FP_STATIC_SCRATCH_BYTES];

std::mutex g_mu;
constexpr int kMaxDevices = 64;
void *g_scratch_ptr[kMaxDevices] = {};

fp_status sfail(fp_status s, const char *msg) {
    fpk::set_last_error(msg);   // reported by fp_last_error()
    return s;
}

__global__ void fill_pairs_kernel(uint64_t first, uint32_t count, int n_raw, fpk::PairInfo *out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    fpk::PairInfo p;
    p.pair = first + i;
    p.plan = 0;
    p.n_raw = n_raw;
    p.raw_off = (int64_t)i * 2 * n_raw;
    p.merged_off = 0;
    p.table_off = 0;
    p.out = i;
    out[i] = p;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

extern "C" fp_status fp_trace_brick_static(int32_t n, int32_t l, uint64_t seed, uint64_t first, uint64_t count,
                                           int32_t prec, double *tr, double *kappa, void *cuda_stream) {
    char msg[256];
    if (n < 2 || n > 64) return sfail(FP_ERR_ARG, "n outside [2, 64]");
    if (l < 2 || 2 * (l - 1) > 12) return sfail(FP_ERR_ARG, "depth l outside [2, 7] (boundary of at most 12 bits)");
    if (prec != FP_PREC_FP64 && prec != FP_PREC_FP32_RAW)
        return sfail(FP_ERR_ARG, "precision must be FP_PREC_FP64 or FP_PREC_FP32_RAW");
    if (!tr) return sfail(FP_ERR_ARG, "tr is NULL");
    if (count == 0) return FP_OK;
    // the current device: the scratch address and every launch belong to it
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return sfail(FP_ERR_CUDA, "cudaGetDevice failed");
    // outputs must be reachable from this device: nothing is staged through
    // host memory, and memory of another GPU would be an illegal address here
    for (const void *p : {(const void *)tr, (const void *)kappa}) {
        if (!p) continue;
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, p) != cudaSuccess || (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)) {
            cudaGetLastError();
            return sfail(FP_ERR_ARG, "tr and kappa must be device (or managed) memory");
        }
        if (a.type == cudaMemoryTypeDevice && a.device != dev) {
            snprintf(msg, sizeof msg, "tr and kappa must be memory of the current device %d (got device %d)", dev,
                     a.device);
            return sfail(FP_ERR_ARG, msg);
        }
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (st) {
        int sdev = -1;
        if (cudaStreamGetDevice(st, &sdev) != cudaSuccess) {
            cudaGetLastError();
            return sfail(FP_ERR_ARG, "cuda_stream is not a valid stream");
        }
        if (sdev != dev) {
            snprintf(msg, sizeof msg, "cuda_stream belongs to device %d, not the current device %d", sdev, dev);
            return sfail(FP_ERR_ARG, msg);
        }
    }
    const bool fp32 = prec == FP_PREC_FP32_RAW;
    // the brickwork sweep's uniform parameters, as fp_trace_batch builds them
    // (whole boundary in one CTA: no tile schedule; host work only)
    const fpk::BrickDev d = fpk::make_brick_plan(n, l, 0, 0, 0, 0).dev;
    int n_raw = 0;
    for (int t = 1; t <= l; ++t) n_raw += (n - (t - 1) % 2) / 2;
    bool both = false;
    fpk::brick_smem_bytes(d, fp32, &both);
    const size_t celem = fp32 ? sizeof(float2) : sizeof(double2);
    const size_t per_raw = (size_t)2 * n_raw * 16 * sizeof(double2);
    const size_t per_map = (size_t)(n - 1) * (l - 1) * 16 * celem;
    const size_t per_l = both ? 0 : ((size_t)1 << d.N) * celem;
    const size_t per_info = sizeof(fpk::PairInfo);
    auto need = [&](uint64_t c) {
        return align256(c * per_info) + align256(c * per_raw) + align256(c * per_map) + align256(c * per_l);
    };
    if (count > 65535 || need(count) > (size_t)FP_STATIC_SCRATCH_BYTES) {
        uint64_t lo = 0, hi = 65535;
        while (lo < hi) {
            uint64_t mid = (lo + hi + 1) / 2;
            if (need(mid) <= (size_t)FP_STATIC_SCRATCH_BYTES) lo = mid; else hi = mid - 1;
        }
        snprintf(msg, sizeof msg, "count %llu exceeds the static scratch: at most %llu pairs fit for n=%d, l=%d",
                 (unsigned long long)count, (unsigned long long)lo, n, l);
        return sfail(FP_ERR_ARG, msg);
    }
    // set-up, once per device, with that device current: the device address of
    // the scratch array (its host-side name is only a stand-in)
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_ptr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_scratch);
            if (e != cudaSuccess) {
                snprintf(msg, sizeof msg, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
                return sfail(FP_ERR_CUDA, msg);
            }
            g_scratch_ptr[dev] = p;
        }
        base = (unsigned char *)g_scratch_ptr[dev];
    }
    fpk::PairInfo *pairs = (fpk::PairInfo *)base;
    double2 *raw = (double2 *)(base + align256(count * per_info));
    void *maps = base + align256(count * per_info) + align256(count * per_raw);
    void *lbuf = base + align256(count * per_info) + align256(count * per_raw) + align256(count * per_map);
    fill_pairs_kernel<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(first, (uint32_t)count, n_raw, pairs);
    if ((e = cudaGetLastError()) != cudaSuccess) return sfail(FP_ERR_CUDA, cudaGetErrorString(e));
    fpk::SampleParams sp;
    sp.seed = seed;
    sp.n = n;
    sp.raw_kind = fpk::RAW_HAAR4;
    sp.self_pair = 0;
    if ((e = fpk::launch_sample(sp, pairs, (int)count, n_raw, raw, st)) != cudaSuccess)
        return sfail(FP_ERR_CUDA, cudaGetErrorString(e));
    fpk::BrickDevPlan dp;
    std::memset(&dp, 0, sizeof dp);
    int nl = 0;
    if ((e = fpk::launch_brick(d, nullptr, dp, pairs, (int)count, raw, maps, lbuf, fp32, 0.0, tr, kappa, nullptr, st,
                               &nl)) != cudaSuccess)
        return sfail(FP_ERR_CUDA, cudaGetErrorString(e));
    return FP_OK;
}
