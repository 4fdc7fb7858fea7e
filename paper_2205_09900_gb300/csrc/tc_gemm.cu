// tc_gemm.cu -- BF16 GEMM on the sm_103a tensor cores (tcgen05) with fused
// epilogues: the dense layers (forward and backward) of the control-variate MLP.
//
//   C[M x N] = A[M x K] . Bt[N x K]^T (+ bias),  BF16 operands, FP32 accumulate
//
// One CTA (128 threads) owns a 128 x NT output tile (NT <= 256 columns) whose
// FP32 accumulator lives in tensor memory (TMEM: NT columns x 128 lanes).  The
// K loop streams stages of 64 columns through a ring of TC_STAGES shared-memory
// buffers, warp-specialised: one lane issues the TMA loads
// (cp.async.bulk.tensor, completing on the stage's "full" mbarrier), one lane
// waits for them and issues four tcgen05.mma (K = 16 each) and a
// tcgen05.commit to the stage's "empty" mbarrier, which the loader waits on
// before it refills the buffer.  A last commit signals the accumulator; the
// epilogue reads it back with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31,
// i.e. tile rows 32w..32w+31), adds the bias and applies one of
//   mode 0: identity,
//   mode 1: GELU (the pre-activation optionally kept in Z),
//   mode 2: multiply by GELU'(Z) (Z read: the backward pass of a GELU layer),
// then stores FP32 row-major, BF16 row-major and/or BF16 transposed results.
// Tiles are 128-byte rows (64 BF16 of K) in the 128-byte swizzle, one TMA box
// per operand and stage; rows and columns beyond the matrices are zero-filled
// by the TMA unit.
// Every wait is bounded: on timeout the kernel raises the error flag, still
// releases its TMEM, and returns; launches that find the flag raised return at
// once.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cstdint>
#include <mutex>

#include "fp.h"
#include "kernels.h"

namespace fpk {
namespace {

constexpr int TC_BM = 128, TC_BK = 64, TC_THREADS = 128, TC_MAXN = 256, TC_STAGES = 4;
constexpr uint64_t TC_DRAIN_NS = 1000000000ull;   // waits for work already issued (after a timeout)

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor (tcgen05) of a K-major tile stored as
// 128-byte rows with the 128-byte swizzle (16-byte chunk c of row r at chunk
// c ^ (r % 8)), tile base 1024-byte aligned: start address >> 4, leading
// offset unused (1), stride offset 1024 bytes (8 rows) >> 4, version 1,
// layout type 2 (128-byte swizzle) in bits 61-63.  Advancing K by 16 BF16
// elements adds 32 bytes to the start address.
__device__ __forceinline__ uint64_t make_desc_sw128(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
           (2ull << 61);
}

// instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A
// (bits 7-9 = 1) and B (bits 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
__device__ __forceinline__ uint32_t make_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Poll an mbarrier phase until it completes or `limit_ns` of global time pass.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase, uint64_t limit_ns) {
    const uint64_t t0 = gtimer();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(mbar), "r"(phase)
            : "memory");
        if (done) return true;
        if (gtimer() - t0 > limit_ns) return false;
    }
}

__device__ __forceinline__ float gelu_f(float v) { return 0.5f * v * (1.0f + erff(v * 0.70710678f)); }
__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678f)) + z * 0.39894228f * expf(-0.5f * z * z);
}

__device__ __forceinline__ void mbar_init(uint64_t *m, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(m)), "r"(count));
}

// one TMA box (64 BF16 columns = 128 bytes x box rows, first column x, first
// row y) of a 2-D tensor map into shared memory, completing its bytes on the mbarrier
__device__ __forceinline__ void tma_load(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(mbar)
        : "memory");
}

// Shared memory per stage: the A tile [128 rows x 128 bytes] then the B tile
// [boxn rows x 128 bytes], both written by the TMA unit with the 128-byte
// swizzle that the MMA descriptors declare; stage bases 1024-byte aligned.
__global__ void __launch_bounds__(TC_THREADS, 1) tc_gemm_kernel(TcGemm g, const __grid_constant__ CUtensorMap tmA,
                                                                const __grid_constant__ CUtensorMap tmB, int boxn) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[TC_STAGES], empty[TC_STAGES], done;
    __shared__ uint32_t taddr_sh;
    __shared__ int abort_sh;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // an earlier launch timed out: do nothing (one read, so that the whole CTA agrees)
    if (tid == 0) abort_sh = g.err ? *(volatile const int *)g.err : 0;
    __syncthreads();
    if (abort_sh) return;
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int m0 = blockIdx.x * TC_BM, n0 = blockIdx.y * TC_MAXN;
    const int NT = min(TC_MAXN, g.N - n0);   // a multiple of 16
    const uint32_t ncols = NT <= 32 ? 32u : (NT <= 64 ? 64u : (NT <= 128 ? 128u : 256u));
    const uint32_t a_bytes = TC_BM * TC_BK * 2, b_bytes = (uint32_t)boxn * TC_BK * 2;
    const uint32_t stage_bytes = a_bytes + TC_MAXN * TC_BK * 2;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&taddr_sh)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 32) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmA) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmB) : "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t taddr = taddr_sh;
    const int nk = (g.K + TC_BK - 1) / TC_BK;
    const uint32_t sbase = smem_u32(smem);
    int issued = 0;   // producer: stages whose TMA loads were issued
    if (tid == 0) {
        // producer: TMA loads of stage kt once the MMAs of stage kt - S have drained the buffer
        for (int kt = 0; kt < nk; ++kt) {
            const int s = kt % TC_STAGES, u = kt / TC_STAGES;
            if (abort_sh || (u > 0 && !mbar_wait(smem_u32(&empty[s]), (uint32_t)(u - 1) & 1u, g.wait_ns))) {
                abort_sh = 1;
                break;
            }
            const uint32_t fb = smem_u32(&full[s]);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(a_bytes + b_bytes)
                         : "memory");
            const uint32_t sa = sbase + s * stage_bytes, sb = sa + a_bytes;
            tma_load(sa, &tmA, kt * TC_BK, m0, fb);
            tma_load(sb, &tmB, kt * TC_BK, n0, fb);
            ++issued;
        }
        // after a timeout: wait (bounded) for the loads still in flight, the last
        // issued phase of each stage buffer
        if (abort_sh)
            for (int kt = (issued > TC_STAGES ? issued - TC_STAGES : 0); kt < issued; ++kt)
                mbar_wait(smem_u32(&full[kt % TC_STAGES]), (uint32_t)(kt / TC_STAGES) & 1u, TC_DRAIN_NS);
    } else if (tid == 32) {
        // MMA issuer: four K = 16 steps per stage, then release the buffer
        const uint32_t idesc = make_idesc(TC_BM, NT);
        bool ok = true, any = false;
        for (int kt = 0; kt < nk; ++kt) {
            const int s = kt % TC_STAGES, u = kt / TC_STAGES;
            if (abort_sh || !mbar_wait(smem_u32(&full[s]), (uint32_t)u & 1u, g.wait_ns)) {
                ok = false;
                break;
            }
            any = true;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t sa = sbase + s * stage_bytes, sb = sa + a_bytes;
#pragma unroll
            for (int kk = 0; kk < TC_BK / 16; ++kk) {
                const uint64_t ad = make_desc_sw128(sa + kk * 32);
                const uint64_t bd = make_desc_sw128(sb + kk * 32);
                const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.u32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(taddr),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&empty[s]))
                         : "memory");
        }
        if (!ok) abort_sh = 1;
        // the last commit covers every MMA issued before it (also after a timeout,
        // so that none is in flight when the tensor memory is released)
        if (any)
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&done))
                         : "memory");
        else
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&done)) : "memory");
    }
    __syncwarp();
    // everyone: wait for the accumulator (or, after a timeout, for the MMAs in flight)
    if (!mbar_wait(smem_u32(&done), 0u, abort_sh ? TC_DRAIN_NS : g.wait_ns)) {
        abort_sh = 1;
        mbar_wait(smem_u32(&done), 0u, TC_DRAIN_NS);   // every arrival on `done` is certain: drain
    }
    __syncthreads();
    if (abort_sh) {
        if (tid == 0 && g.err) atomicExch(g.err, 1);
    } else {
        asm volatile("tcgen05.fence::after_thread_sync;");
        const int row = m0 + warp * 32 + lane;
        const bool rv = row < g.M;
        for (int c0 = 0; c0 < NT; c0 += 32) {
            uint32_t r[32];
            const uint32_t ta = taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                  "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                  "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                : "r"(ta));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (!rv) continue;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                if (c0 + 4 * q >= NT) break;   // NT is a multiple of 16: groups of 4 are whole
                const int col = n0 + c0 + 4 * q;
                float v[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) v[e] = __uint_as_float(r[4 * q + e]);
                if (g.bias) {
                    const float4 b = *(const float4 *)(g.bias + col);
                    v[0] += b.x, v[1] += b.y, v[2] += b.z, v[3] += b.w;
                }
                if (g.mode == 1) {
                    if (g.Z) *(float4 *)(g.Z + (size_t)row * g.ldz + col) = make_float4(v[0], v[1], v[2], v[3]);
#pragma unroll
                    for (int e = 0; e < 4; ++e) v[e] = gelu_f(v[e]);
                } else if (g.mode == 2) {
                    const float4 z = *(const float4 *)(g.Z + (size_t)row * g.ldz + col);
                    v[0] *= gelu_grad(z.x), v[1] *= gelu_grad(z.y), v[2] *= gelu_grad(z.z), v[3] *= gelu_grad(z.w);
                }
                if (g.Cf) *(float4 *)(g.Cf + (size_t)row * g.ldcf + col) = make_float4(v[0], v[1], v[2], v[3]);
                if (g.Cb) {
                    __nv_bfloat162 p0 = __floats2bfloat162_rn(v[0], v[1]), p1 = __floats2bfloat162_rn(v[2], v[3]);
                    uint2 u;
                    u.x = *(uint32_t *)&p0;
                    u.y = *(uint32_t *)&p1;
                    *(uint2 *)(g.Cb + (size_t)row * g.ldcb + col) = u;
                }
                if (g.Cbt) {
#pragma unroll
                    for (int e = 0; e < 4; ++e) g.Cbt[(size_t)(col + e) * g.ldct + row] = __float2bfloat16(v[e]);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

bool aligned(const void *p, uintptr_t a) { return ((uintptr_t)p & (a - 1)) == 0; }

}  // namespace

size_t tc_gemm_smem_bytes() { return (size_t)TC_STAGES * (TC_BM + TC_MAXN) * TC_BK * 2 + 1024; }

const char *tc_gemm_check(const TcGemm &g) {
    if (g.M < 0 || g.N <= 0 || g.N % 16 != 0 || g.K <= 0 || g.K % 8 != 0) return "need N % 16 == 0 and K % 8 == 0";
    if (g.M == 0) return nullptr;   // nothing is read or written
    if (!g.A || !g.Bt || g.lda < g.K || g.ldb < g.K || g.lda % 8 || g.ldb % 8 || !aligned(g.A, 16) ||
        !aligned(g.Bt, 16))
        return "A and Bt need 16-byte alignment and leading dimensions >= K that are multiples of 8";
    if (!g.Cf && !g.Cb && !g.Cbt) return "no output";
    if (g.mode < 0 || g.mode > 2 || (g.mode == 2 && !g.Z)) return "mode must be 0, 1 or 2 (mode 2 needs Z)";
    if (g.Z && (g.ldz < g.N || g.ldz % 4 || !aligned(g.Z, 16)))
        return "Z needs a leading dimension >= N that is a multiple of 4, and 16-byte alignment";
    if (g.bias && !aligned(g.bias, 16)) return "bias needs 16-byte alignment";
    if (g.Cf && (g.ldcf < g.N || g.ldcf % 4 || !aligned(g.Cf, 16)))
        return "C needs a leading dimension >= N that is a multiple of 4, and 16-byte alignment";
    if (g.Cb && (g.ldcb < g.N || g.ldcb % 4 || !aligned(g.Cb, 8)))
        return "C_bf16 needs a leading dimension >= N that is a multiple of 4, and 8-byte alignment";
    if (g.Cbt && (g.ldct < g.M || !aligned(g.Cbt, 2))) return "Ct_bf16 needs a leading dimension >= M";
    return nullptr;
}

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

// tensor map of a row-major [rows x ld] BF16 matrix whose first `cols`
// columns are valid; boxes of 64 columns (128 bytes) x box_rows rows, 128-byte swizzle
bool make_map(CUtensorMap *m, const void *base, int rows, int cols, int ld, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1u, 1u};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

cudaError_t launch_tc_gemm(const TcGemm &g, cudaStream_t st) {
    if (g.M == 0) return cudaSuccess;
    if (tc_gemm_check(g)) return cudaErrorInvalidValue;
    const int boxn = g.N < TC_MAXN ? g.N : TC_MAXN;
    CUtensorMap ma, mb;
    if (!make_map(&ma, g.A, g.M, g.K, g.lda, TC_BM) || !make_map(&mb, g.Bt, g.N, g.K, g.ldb, boxn))
        return cudaErrorInvalidValue;
    const size_t smem = tc_gemm_smem_bytes();
    // the attribute is set outside stream capture (a launch being captured
    // follows a direct launch on the same device, which has set it)
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return e;
    if (cs == cudaStreamCaptureStatusNone) {
        e = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((g.M + TC_BM - 1) / TC_BM, (g.N + TC_MAXN - 1) / TC_MAXN);
    TcGemm gk = g;
    gk.wait_ns = wait_limit_ns();
    tc_gemm_kernel<<<grid, TC_THREADS, smem, st>>>(gk, ma, mb, boxn);
    return cudaGetLastError();
}

}  // namespace fpk

extern "C" fp_status fp_gemm_bf16(int32_t M, int32_t N, int32_t K, const void *A, int32_t lda, const void *Bt,
                                  int32_t ldb, const float *bias, int32_t mode, float *Z, float *C, void *C_bf16,
                                  void *Ct_bf16, void *cuda_stream) {
    fpk::TcGemm g{};
    g.M = M, g.N = N, g.K = K;
    g.A = (const __nv_bfloat16 *)A, g.lda = lda;
    g.Bt = (const __nv_bfloat16 *)Bt, g.ldb = ldb;
    g.bias = bias, g.mode = mode;
    g.Z = Z, g.ldz = N;
    g.Cf = C, g.ldcf = N;
    g.Cb = (__nv_bfloat16 *)C_bf16, g.ldcb = N;
    g.Cbt = (__nv_bfloat16 *)Ct_bf16, g.ldct = M;
    if (const char *why = fpk::tc_gemm_check(g)) return fpk::api_fail(FP_ERR_ARG, why);
    if (M == 0) return FP_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int *derr = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&derr, sizeof(int), st);
    if (e != cudaSuccess) return fpk::api_fail(FP_ERR_OOM, cudaGetErrorString(e));
    g.err = derr;
    int herr = 0;
    e = cudaMemsetAsync(derr, 0, sizeof(int), st);
    if (e == cudaSuccess) e = fpk::launch_tc_gemm(g, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(derr, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fpk::api_fail(FP_ERR_CUDA, cudaGetErrorString(e));
    if (herr) return fpk::api_fail(FP_ERR_TIMEOUT, "tcgen05 GEMM: an mbarrier wait ran out");
    return FP_OK;
}
