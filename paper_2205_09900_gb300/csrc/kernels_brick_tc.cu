// kernels_brick_tc.cu -- brickwork tile passes on the tensor cores (tcgen05).
//
// The FFMA tile pass applies the gates of each register window (5 ring bits
// of a 12-bit tile) one 4x4 map at a time.  Here the window's gates are first
// multiplied into one dense 32 x 32 complex matrix W per (pair, window)
// (tc_wmat_kernel, FP32 products of the FP32 maps), and the tile, viewed as a
// [128 rows x 32] complex matrix whose rows are the 7 other tile bits, is
// multiplied by W^T on the tensor cores: complex numbers as real pairs (K
// columns 2j, 2j+1 hold re, im of window index j; W as the real 64 x 64 block
// matrix [[Re, -Im], [Im, Re]]), TF32 operands split into hi + lo parts
// (W: hi = rna(w), lo = rna(w - hi); the tile: hi = x truncated by the MMA
// itself, lo = rna(x - trunc(x))) and three MMAs per K step (hi.lo, lo.hi, hi.hi),
// accumulated in FP32 in tensor memory (tcgen05.mma kind::tf32, M = 128,
// N = 64, K = 8).
//
// Two kernels.  brick_tc1_pass_kernel takes one tile per CTA, two CTAs per
// SM: the tile's operands sit in shared memory (K-major, 128-byte swizzle;
// every element's address is the XOR of its bits' contributions, the TcWin
// tables), and after each window 8 drain warps read the result out of tensor
// memory (tcgen05.ld), split it and store it into the next window's operand
// layout.  brick_tcm_pass_kernel keeps the tile's operand in tensor memory
// (the A operand read from TMEM), exchanges each window's result through a
// shared-memory buffer into the next window's row order, and is persistent
// over the tiles.  In both a control warp's lane issues every MMA and the
// bulk copies (cp.async.bulk) of the window matrices, and meets the drain
// warps on mbarriers only.  The first window's operand is loaded from the
// boundary in global memory, the last window's result is written back to it.
//
// Every mbarrier wait is bounded by the global timer (1 s); on a timeout the
// CTA raises the error flag, stops issuing work, drains the MMAs and bulk
// copies it has issued (bounded again), frees its tensor memory and returns;
// later launches that find the flag raised return at once.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "brick.h"
#include "kernels.h"

namespace fpk {
namespace {

constexpr uint64_t kTcDrainNs = 1000000000ull;   // waits for work already issued (after a timeout)
constexpr int kMaxTcWins = 48;
constexpr uint32_t kAOp = 32768;                 // bytes of one A operand (hi or lo) of one tile
constexpr uint32_t kWMat = 32768;                // bytes of one window matrix (hi + lo)
constexpr uint32_t kWFloats = kWMat / 4;

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Wait for the phase of parity `phase` to complete, at most limit_ns.  The
// try_wait carries a suspend-time hint: the thread is parked until the phase
// completes (or the hint runs out) instead of spinning, so waiting warps take
// no issue slots from the working ones.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase, uint64_t limit_ns) {
    const uint64_t t0 = gtimer();
    for (;;) {
        uint32_t d;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(d)
            : "r"(mbar), "r"(phase), "r"(1000000u)
            : "memory");
        if (d) return true;
        if (gtimer() - t0 > limit_ns) return false;
    }
}

__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
           (2ull << 61);
}

// x rounded to the nearest TF32 value (10 mantissa bits), ties away from zero:
// half of the dropped 13 bits' weight added to the magnitude, then those bits
// cleared (finite x of moderate size, as the window matrices' entries are)
__device__ __forceinline__ float tf32_rna(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// ---------------------------------------------------------------------------
// Window matrices: W = G_last ... G_first of the window's gates (4x4 maps on
// window bits (k, k+1)), column j built by thread j in FP32, stored as the B
// operand of the MMA: rows n = 2o (re, -im) and 2o + 1 (im, re) of output o,
// K columns 2j, 2j + 1, K-major with the 128-byte swizzle in two regions of
// 64 rows x 128 bytes; hi part then lo part.
template <int k>
__device__ __forceinline__ void wapply(float2 (&v)[32], const float2 *__restrict__ T) {
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        if (i & (3 << k)) continue;
        const float2 x0 = v[i], x1 = v[i | (1 << k)], x2 = v[i | (2 << k)], x3 = v[i | (3 << k)];
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            const float2 t0 = T[4 * o], t1 = T[4 * o + 1], t2 = T[4 * o + 2], t3 = T[4 * o + 3];
            float2 a;
            a.x = t0.x * x0.x - t0.y * x0.y + t1.x * x1.x - t1.y * x1.y + t2.x * x2.x - t2.y * x2.y + t3.x * x3.x -
                  t3.y * x3.y;
            a.y = t0.x * x0.y + t0.y * x0.x + t1.x * x1.y + t1.y * x1.x + t2.x * x2.y + t2.y * x2.x + t3.x * x3.y +
                  t3.y * x3.x;
            v[i | (o << k)] = a;
        }
    }
}

__device__ __forceinline__ uint32_t wb_addr(uint32_t n, uint32_t kc) {   // B operand: row n, K column kc
    return (kc >> 5) * 8192u + n * 128u + ((((kc >> 2) & 7u) ^ (n & 7u)) << 4) + (kc & 3u) * 4u;
}

__global__ void __launch_bounds__(32) tc_wmat_kernel(BrickDev d, int side, BrickPass ps,
                                                     const BrickGate *__restrict__ gates,
                                                     const RegPass *__restrict__ rps, const RegGate *__restrict__ rgs,
                                                     const float2 *__restrict__ maps, float *__restrict__ wm) {
    __shared__ float2 T[kMaxTcWins][16];
    const RegPass rp = rps[ps.rp_off + blockIdx.x];
    const int ng = rp.n_gates < kMaxTcWins ? rp.n_gates : kMaxTcWins;
    const float2 *mp = maps + (size_t)blockIdx.y * maps_per_pair(d) * 16;
    for (int i = threadIdx.x; i < ng * 16; i += 32) {
        const RegGate rg = rgs[rp.gate_off + i / 16];
        const BrickGate gg = gates[ps.gate_off + rg.slot];
        const float2 v = mp[(size_t)map_index(d, side, gg.layer, gg.j) * 16 + (i % 16)];
        T[i / 16][i % 16] = v;
    }
    __syncwarp();
    const int j = threadIdx.x;
    float2 v[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = make_float2(i == j ? 1.f : 0.f, 0.f);
    for (int g = 0; g < ng; ++g) {
        switch (rgs[rp.gate_off + g].type) {
            case 0: wapply<0>(v, T[g]); break;
            case 1: wapply<1>(v, T[g]); break;
            case 2: wapply<2>(v, T[g]); break;
            default: wapply<3>(v, T[g]); break;
        }
    }
    unsigned char *out = (unsigned char *)(wm + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * kWFloats);
#pragma unroll
    for (int o = 0; o < 32; ++o) {
        const float re = v[o].x, im = v[o].y;
        const float rh = tf32_rna(re), ih = tf32_rna(im);
        const float rl = tf32_rna(re - rh), il = tf32_rna(im - ih);
        const uint32_t a0 = wb_addr(2 * o, 2 * j), a1 = wb_addr(2 * o + 1, 2 * j);
        *(float2 *)(out + a0) = make_float2(rh, -ih);
        *(float2 *)(out + a1) = make_float2(ih, rh);
        *(float2 *)(out + 16384 + a0) = make_float2(rl, -il);
        *(float2 *)(out + 16384 + a1) = make_float2(il, rl);
    }
}

// ---------------------------------------------------------------------------
// The tile pass.
__device__ __forceinline__ uint32_t tile_base_of(uint32_t t, uint32_t smask, int N) {
    uint32_t base = 0;
    for (int b = 0; b < N; ++b)
        if (!(smask & (1u << b))) { base |= (t & 1u) << b; t >>= 1; }
    return base;
}

// The two TF32 parts of an operand pair: the MMA reads an FP32 word's top 19
// bits (sign, exponent, 10 mantissa bits), so x itself serves as the high
// part (read as x with its low 13 mantissa bits cleared, i.e. truncated) and
// the rest x - trunc(x), exact in FP32 and of the same sign as x, rounded to
// the nearest TF32 value (half away from zero) as the low part.  The rest has
// at most 13 significant bits, of which TF32 keeps 11: left to the MMA's
// truncation it would lose up to 2^-21 of x, always towards zero (about
// 0.9 x 2^-23 of x on average), a bias that adds up over the windows of a
// sweep; rounded, the error is at most 2^-22 of x, and the ties that rounding
// away from zero meets leave a mean of about 0.35 x 2^-23.
__device__ __forceinline__ float tf32_rest(float x) {
    const float r = x - __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
    return __uint_as_float((__float_as_uint(r) + 0x1000u) & 0xFFFFE000u);
}
__device__ __forceinline__ void st_hilo(unsigned char *A, uint32_t a, float x, float y) {
    *(float2 *)(A + a) = make_float2(x, y);
    *(float2 *)(A + kAOp + a) = make_float2(tf32_rest(x), tf32_rest(y));
}

// 3 x 8 MMAs of one tile: D[128 x 64] (+)= A[128 x 64] . B[64 x 64]^T, the
// products of the low parts first (hi.lo, then lo.hi, over all K steps), then
// hi.hi.  The tensor core's FP32 accumulation truncates: with the small terms
// summed before the large ones they keep their bits (adding them K step by K
// step to the large partial sums instead tripled the measured error and its
// bias towards zero).
__device__ __forceinline__ void issue_tile_mmas(uint32_t dtm, uint32_t sA, uint32_t sW) {
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);
    // base descriptors once; a K step adds its byte offset / 16 to the address field
    // (shared-memory addresses stay below 256 KB, so the 14-bit field never carries)
    const uint64_t dA[3] = {desc_sw128(sA), desc_sw128(sA + kAOp), desc_sw128(sA)};
    const uint64_t dB[3] = {desc_sw128(sW + 16384), desc_sw128(sW), desc_sw128(sW)};
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            const uint64_t ad = dA[p] + (uint64_t)((((s >> 2) * 16384) + (s & 3) * 32) >> 4);
            const uint64_t bd = dB[p] + (uint64_t)((((s >> 2) * 8192) + (s & 3) * 32) >> 4);
            const uint32_t acc = (p > 0 || s > 0) ? 1u : 0u;
            asm volatile(
                "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, q;\n\t}" ::"r"(dtm),
                "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
        }
}

__device__ __forceinline__ void commit_to(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// ---------------------------------------------------------------------------
// One tile per CTA, two CTAs per SM (96 KB of operands and one window-matrix
// buffer each, 64 tensor-memory columns): 8 drain warps (16 outputs per
// thread) and a control warp.  Per window the control lane waits for the
// operand and the matrix, issues the 24 MMAs and, once they are done, loads the
// next window's matrix into the one buffer -- while the drain warps empty the
// accumulator -- so the matrix load overlaps the drain, and the other CTA on
// the SM keeps the tensor cores busy while this one loads, drains and stores.
constexpr int kTc1Drain = 256;
constexpr size_t kTc1Smem = 2 * (size_t)kAOp + (size_t)kWMat + 1024;

__device__ __forceinline__ void drain_tile16(uint32_t tm, const TcWin &cw, const uint32_t *__restrict__ cbn,
                                             unsigned char *A, float2 *gdst) {
    const int warp = (threadIdx.x >> 5) & 7, lane = threadIdx.x & 31;   // warp within its group of 8
    uint32_t v[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
          "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
          "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
          "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(tm + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(32 * (warp >> 2))));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    const uint32_t r = 32u * (warp & 3) + lane;
    uint32_t base = 0;
#pragma unroll
    for (int t = 0; t < kTcRows; ++t)
        if ((r >> t) & 1u) base ^= cbn[cw.row[t]];
    if (warp >> 2) base ^= cbn[cw.win[4]];   // window output bit 4
    const uint32_t c0 = cbn[cw.win[0]], c1 = cbn[cw.win[1]], c2 = cbn[cw.win[2]], c3 = cbn[cw.win[3]];
    // the store order of TcWin::rotm over output bits 0-2 (as in drain_tile)
    const uint32_t rm = A ? cw.rotm : 0u, l4 = (uint32_t)lane & 15u;
    const int rot = (__popc(l4 & (rm & 15u)) & 1) | ((__popc(l4 & ((rm >> 4) & 15u)) & 1) << 1) |
                    ((__popc(l4 & ((rm >> 8) & 15u)) & 1) << 2);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        if ((rot >> b) & 1) {
#pragma unroll
            for (int u = 0; u < 16; ++u)
                if (!((u >> b) & 1)) {
                    const int w2 = u | (1 << b);
                    uint32_t t0 = v[2 * u], t1 = v[2 * u + 1];
                    v[2 * u] = v[2 * w2]; v[2 * u + 1] = v[2 * w2 + 1];
                    v[2 * w2] = t0; v[2 * w2 + 1] = t1;
                }
        }
    }
    base ^= ((rot & 1) ? c0 : 0u) ^ ((rot & 2) ? c1 : 0u) ^ ((rot & 4) ? c2 : 0u);
#pragma unroll
    for (int u = 0; u < 16; ++u) {   // register u holds output u ^ rot (bits 0-2)
        const uint32_t a = base ^ ((u & 1) ? c0 : 0u) ^ ((u & 2) ? c1 : 0u) ^ ((u & 4) ? c2 : 0u) ^ ((u & 8) ? c3 : 0u);
        const float x = __uint_as_float(v[2 * u]), y = __uint_as_float(v[2 * u + 1]);
        if (A) st_hilo(A, a, x, y);
        else gdst[a] = make_float2(x, y);
    }
}

__global__ void __launch_bounds__(kTc1Drain + 32, 2)
    brick_tc1_pass_kernel(BrickDev d, int side, BrickPass ps, const TcWin *__restrict__ wins,
                          const float *__restrict__ wm, float2 *__restrict__ states, int *err, uint64_t wait_ns) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t wfull, dfull, afull, fbar;
    __shared__ uint32_t taddr_sh;
    __shared__ int abort_sh;
    __shared__ int pos[32];
    __shared__ uint32_t lut_lo[128], lut_hi[1 << (kTcTile - 7)], alo[128], ahi[1 << (kTcTile - 7)], gcb[kTcTile];
    __shared__ TcWin sw[kMaxTcWins];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool ctrl = warp == kTc1Drain / 32;
    const int nw = ps.n_rp;
    const int N = d.N;
    const uint32_t S = 1u << N;
    if (tid == 0) {
        abort_sh = *(volatile const int *)err;   // an earlier launch timed out
        int k = 0;
        for (int b = 0; b < N; ++b)
            if (ps.smask & (1u << b)) pos[k++] = b;
    }
    for (int i = tid; i < nw; i += kTc1Drain + 32) sw[i] = wins[ps.rp_off + i];
    __syncthreads();
    if (abort_sh) return;
    for (int i = tid; i < 128; i += kTc1Drain + 32) {
        uint32_t o = 0, a = 0;
        for (int k = 0; k < 7; ++k)
            if ((i >> k) & 1) { o |= 1u << pos[k]; a ^= sw[0].cb[k]; }
        lut_lo[i] = o;
        alo[i] = a;
    }
    if (tid < (1 << (kTcTile - 7))) {
        uint32_t o = 0, a = 0;
        for (int k = 0; k < kTcTile - 7; ++k)
            if ((tid >> k) & 1) { o |= 1u << pos[7 + k]; a ^= sw[0].cb[7 + k]; }
        lut_hi[tid] = o;
        ahi[tid] = a;
    }
    if (tid < kTcTile) gcb[tid] = 1u << pos[tid];
    if (tid < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(smem_u32(&taddr_sh)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 32) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&wfull)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&dfull)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&afull)), "r"(kTc1Drain / 32));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&fbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t taddr = taddr_sh;
    const uint32_t sbase = smem_u32(smem);
    const uint32_t sW = sbase + 2 * kAOp;
    const float *wp = wm + (size_t)blockIdx.y * nw * kWFloats;
    auto ab = [&]() { return *(volatile int *)&abort_sh != 0; };
    float2 *st = states + ((size_t)blockIdx.y * 2 + side) * S;
    const uint32_t gb = tile_base_of(blockIdx.x, ps.smask, N);
    if (ctrl) {
        if (lane == 0) {
            int tma_issued = 0, tma_waited = 0;
            bool any = false;
            bulk_load(sW, wp, kWMat, &wfull);
            ++tma_issued;
            for (int w = 0; w < nw && !ab(); ++w) {
                if (!mbar_wait(smem_u32(&afull), (uint32_t)w & 1u, wait_ns)) { abort_sh = 1; break; }
                if (!mbar_wait(smem_u32(&wfull), (uint32_t)w & 1u, wait_ns)) { abort_sh = 1; break; }
                ++tma_waited;
                asm volatile("tcgen05.fence::after_thread_sync;");
                issue_tile_mmas(taddr, sbase, sW);
                commit_to(&dfull);
                any = true;
                if (w + 1 < nw) {   // the buffer is free once these MMAs are done
                    if (!mbar_wait(smem_u32(&dfull), (uint32_t)w & 1u, wait_ns)) { abort_sh = 1; break; }
                    bulk_load(sW, wp + (size_t)(w + 1) * kWFloats, kWMat, &wfull);
                    ++tma_issued;
                }
            }
            if (ab()) {
                if (any) {
                    commit_to(&fbar);
                    mbar_wait(smem_u32(&fbar), 0u, kTcDrainNs);
                }
                if (tma_issued > tma_waited) mbar_wait(smem_u32(&wfull), (uint32_t)(tma_issued - 1) & 1u, kTcDrainNs);
                atomicExch(err, 1);
            }
        }
    } else {
        // the tile: boundary -> A operand of window 0 (all copies in flight at once,
        // staged in the operand's low half, converted through registers)
        constexpr int kPer = (1 << kTcTile) / kTc1Drain;
        float2 *stage = (float2 *)(smem + kAOp);
#pragma unroll
        for (int m = 0; m < kPer; ++m) {
            const uint32_t i = tid + (uint32_t)m * kTc1Drain;
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(stage + i)),
                         "l"(st + gb + (lut_lo[i & 127] | lut_hi[i >> 7]))
                         : "memory");
        }
        asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
        float2 xv[kPer];
#pragma unroll
        for (int m = 0; m < kPer; ++m) xv[m] = stage[tid + m * kTc1Drain];
        asm volatile("bar.sync 1, %0;" ::"n"(kTc1Drain));   // staging reads done
#pragma unroll
        for (int m = 0; m < kPer; ++m) {
            const uint32_t i = tid + (uint32_t)m * kTc1Drain;
            st_hilo(smem, alo[i & 127] ^ ahi[i >> 7], xv[m].x, xv[m].y);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&afull);
        for (int w = 0; w < nw; ++w) {
            if (ab()) break;
            if (!mbar_wait(smem_u32(&dfull), (uint32_t)w & 1u, wait_ns)) { abort_sh = 1; break; }
            asm volatile("tcgen05.fence::after_thread_sync;");
            if (w + 1 < nw) {
                drain_tile16(taddr, sw[w], sw[w + 1].cb, smem, nullptr);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;");
                __syncwarp();
                if (lane == 0) mbar_arrive(&afull);
            } else {
                drain_tile16(taddr, sw[w], gcb, nullptr, st + gb);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (tid < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(taddr));
}

// ---------------------------------------------------------------------------
// The tile's operand in tensor memory (the A operand of tcgen05.mma read from
// TMEM): per window the MMAs read only the window matrix from shared memory.
// Persistent: two CTAs per SM, each taking tiles t = blockIdx.x, + gridDim.x,
// ...; 8 drain warps and a control warp as above.  TMEM columns: D 0-63, A
// high parts 64-127, A low parts 128-191.  A window's result goes from D
// through registers into a 32 KB shared-memory exchange buffer (TcWin::xcb of
// the next window: both the storing and the loading half-warps hit 16
// distinct bank pairs), every drain warp arrives on an mbarrier, and each
// thread then loads its row of the next window's operand, splits it into TF32
// parts and stores them into TMEM (tcgen05.st).  Exchanges alternate between
// two buffers; the next tile's elements are copied into the free one while
// the current tile's last window is multiplied and written back.  Shared
// memory traffic per window and tile: 32 KB stored and 32 KB loaded by the
// exchange, 48 KB of window matrix read by the 24 MMAs, 32 KB of window
// matrix copied in (the shared-memory operand form: 64 KB stored, 96 + 48 KB
// read by the MMAs, 32 KB copied in).
constexpr int kTcmDrain = 256;
constexpr uint32_t kXch = 32768;
constexpr size_t kTcmSmem = 2 * (size_t)kXch + (size_t)kWMat + 1024;

// As issue_tile_mmas with the tile's operand in tensor memory (columns 64-127
// high parts, 128-191 low parts; K step s reads 8 columns from 8 s)
__device__ __forceinline__ void issue_tile_mmas_tm(uint32_t tm, uint32_t sW) {
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);
    const uint64_t dB[3] = {desc_sw128(sW + 16384), desc_sw128(sW), desc_sw128(sW)};
    const uint32_t aC[3] = {64u, 128u, 64u};
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            const uint64_t bd = dB[p] + (uint64_t)((((s >> 2) * 8192) + (s & 3) * 32) >> 4);
            const uint32_t acc = (p > 0 || s > 0) ? 1u : 0u;
            asm volatile(
                "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, q;\n\t}" ::"r"(tm),
                "r"(tm + aC[p] + 8u * s), "l"(bd), "r"(idesc), "r"(acc));
        }
}

// A thread's exchange addresses for one window and direction, from the
// window's table (TcXa): element u at base ^ (c[k] of the set bits k of u)
struct XchAddr {
    uint32_t base, c0, c1, c2, c3;
    __device__ __forceinline__ XchAddr(const uint32_t *lane_t, const uint32_t *warp_t, const uint32_t *c) {
        const int warp = (threadIdx.x >> 5) & 7, lane = threadIdx.x & 31;   // warp within its group of 8
        base = __ldg(lane_t + lane) ^ __ldg(warp_t + warp);
        const uint4 cc = __ldg(reinterpret_cast<const uint4 *>(c));
        c0 = cc.x; c1 = cc.y; c2 = cc.z; c3 = cc.w;
    }
    __device__ __forceinline__ uint32_t at(int u) const {
        return base ^ ((u & 1) ? c0 : 0u) ^ ((u & 2) ? c1 : 0u) ^ ((u & 4) ? c2 : 0u) ^ ((u & 8) ? c3 : 0u);
    }
};

// This thread's operand row (lanes 32 (warp mod 4) .., columns 64 / 128 + 32 (warp / 4) ..
// of tensor memory) from the exchange buffer, split into TF32 high and low parts.
// All 16 loads are in flight at once; the parts go out in two halves of 16 columns.
__device__ __forceinline__ void tm_load_operand(uint32_t tm, const XchAddr &xa, uint32_t xs) {
    const int warp = (threadIdx.x >> 5) & 7;   // warp within its group of 8
    const uint32_t ta = tm + ((32u * (warp & 3)) << 16) + 32u * (uint32_t)(warp >> 2);
    uint32_t h[32];
#pragma unroll
    for (int u = 0; u < 16; ++u)
        asm volatile("ld.shared.v2.b32 {%0, %1}, [%2];" : "=r"(h[2 * u]), "=r"(h[2 * u + 1]) : "r"(xs + xa.at(u)) : "memory");
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const uint32_t *hq = h + 16 * q;
        uint32_t lo[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) lo[i] = __float_as_uint(tf32_rest(__uint_as_float(hq[i])));
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15, %16};" ::"r"(ta + 64u + 16u * q),
            "r"(hq[0]), "r"(hq[1]), "r"(hq[2]), "r"(hq[3]), "r"(hq[4]), "r"(hq[5]), "r"(hq[6]), "r"(hq[7]),
            "r"(hq[8]), "r"(hq[9]), "r"(hq[10]), "r"(hq[11]), "r"(hq[12]), "r"(hq[13]), "r"(hq[14]), "r"(hq[15])
            : "memory");
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15, %16};" ::"r"(ta + 128u + 16u * q),
            "r"(lo[0]), "r"(lo[1]), "r"(lo[2]), "r"(lo[3]), "r"(lo[4]), "r"(lo[5]), "r"(lo[6]), "r"(lo[7]),
            "r"(lo[8]), "r"(lo[9]), "r"(lo[10]), "r"(lo[11]), "r"(lo[12]), "r"(lo[13]), "r"(lo[14]), "r"(lo[15])
            : "memory");
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// This thread's 16 results (D row 32 (warp mod 4) + lane, window outputs 16 (warp / 4) ..)
// into the exchange buffer
__device__ __forceinline__ void tm_store_result(uint32_t tm, const XchAddr &xa, uint32_t xs) {
    const int warp = (threadIdx.x >> 5) & 7;   // warp within its group of 8
    const uint32_t ta = tm + ((32u * (warp & 3)) << 16) + 32u * (uint32_t)(warp >> 2);
    // two halves of 16 columns: the second half's read is in flight while the first is stored
    uint32_t v[16], y[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(ta));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];"
        : "=r"(y[0]), "=r"(y[1]), "=r"(y[2]), "=r"(y[3]), "=r"(y[4]), "=r"(y[5]), "=r"(y[6]), "=r"(y[7]),
          "=r"(y[8]), "=r"(y[9]), "=r"(y[10]), "=r"(y[11]), "=r"(y[12]), "=r"(y[13]), "=r"(y[14]), "=r"(y[15])
        : "r"(ta + 16u));
#pragma unroll
    for (int u = 0; u < 8; ++u)
        asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(xs + xa.at(u)), "r"(v[2 * u]), "r"(v[2 * u + 1])
                     : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int u = 0; u < 8; ++u)
        asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(xs + xa.at(8 + u)), "r"(y[2 * u]), "r"(y[2 * u + 1])
                     : "memory");
}

__global__ void __launch_bounds__(kTcmDrain + 32, 2)
    brick_tcm_pass_kernel(BrickDev d, int side, BrickPass ps, const TcWin *__restrict__ wins,
                          const TcXa *__restrict__ xat, const float *__restrict__ wm, float2 *__restrict__ states,
                          int *err, uint64_t wait_ns, uint32_t ntiles) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t wfull, dfull, afull, xbar, fbar;
    __shared__ uint32_t taddr_sh;
    __shared__ int abort_sh;
    __shared__ int pos[32];
    // tile index -> boundary offset (lut), -> input address (a); tile bit -> boundary offset (gcb)
    __shared__ uint32_t lut_lo[128], lut_hi[1 << (kTcTile - 7)], alo[128], ahi[1 << (kTcTile - 7)], gcb[kTcTile];
    __shared__ TcWin sw[kMaxTcWins];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool ctrl = warp == kTcmDrain / 32;
    const int nw = ps.n_rp;
    const int N = d.N;
    const uint32_t S = 1u << N;
    const int tb = N - kTcTile;   // tile-index bits
    if (blockIdx.x >= ntiles) return;
    if (tid == 0) {
        abort_sh = *(volatile const int *)err;   // an earlier launch timed out
        int k = 0;
        for (int b = 0; b < N; ++b)
            if (ps.smask & (1u << b)) pos[k++] = b;
    }
    for (int i = tid; i < nw; i += kTcmDrain + 32) sw[i] = wins[ps.rp_off + i];
    __syncthreads();
    if (abort_sh) return;
    for (int i = tid; i < 128; i += kTcmDrain + 32) {
        uint32_t o = 0, a = 0;
        for (int k = 0; k < 7; ++k)
            if ((i >> k) & 1) { o |= 1u << pos[k]; a ^= sw[0].xcb[k]; }
        lut_lo[i] = o;
        alo[i] = a;
    }
    if (tid < (1 << (kTcTile - 7))) {
        uint32_t o = 0, a = 0;
        for (int k = 0; k < kTcTile - 7; ++k)
            if ((tid >> k) & 1) { o |= 1u << pos[7 + k]; a ^= sw[0].xcb[7 + k]; }
        lut_hi[tid] = o;
        ahi[tid] = a;
    }
    if (tid < kTcTile) gcb[tid] = 1u << pos[tid];
    if (tid < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(&taddr_sh)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 32) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&wfull)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&dfull)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&afull)), "r"(kTcmDrain / 32));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&xbar)), "r"(kTcmDrain / 32));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&fbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t taddr = taddr_sh;
    const uint32_t sbase = smem_u32(smem);
    const uint32_t sW = sbase + 2 * kXch;
    auto ab = [&]() { return *(volatile int *)&abort_sh != 0; };
    auto wmat = [&](uint32_t t) { return wm + (size_t)(t >> tb) * nw * kWFloats; };
    auto tile_ptr = [&](uint32_t t) {
        return states + ((size_t)(t >> tb) * 2 + side) * S + tile_base_of(t & ((1u << tb) - 1u), ps.smask, N);
    };
    if (ctrl) {
        if (lane == 0) {
            int tma_issued = 0, tma_waited = 0;
            bool any = false, stop = false;
            uint32_t g = 0;
            bulk_load(sW, wmat(blockIdx.x), kWMat, &wfull);
            ++tma_issued;
            for (uint32_t t = blockIdx.x; t < ntiles && !stop; t += gridDim.x) {
                for (int w = 0; w < nw; ++w, ++g) {
                    if (ab()) { stop = true; break; }
                    if (!mbar_wait(smem_u32(&afull), g & 1u, wait_ns)) { abort_sh = 1; stop = true; break; }
                    if (!mbar_wait(smem_u32(&wfull), g & 1u, wait_ns)) { abort_sh = 1; stop = true; break; }
                    ++tma_waited;
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    issue_tile_mmas_tm(taddr, sW);
                    commit_to(&dfull);
                    any = true;
                    // the matrix buffer is free once these MMAs are done: the next window's
                    // matrix, or window 0's of the CTA's next tile
                    const float *nxt = w + 1 < nw ? wmat(t) + (size_t)(w + 1) * kWFloats
                                                  : (t + gridDim.x < ntiles ? wmat(t + gridDim.x) : nullptr);
                    if (nxt) {
                        if (!mbar_wait(smem_u32(&dfull), g & 1u, wait_ns)) { abort_sh = 1; stop = true; break; }
                        bulk_load(sW, nxt, kWMat, &wfull);
                        ++tma_issued;
                    }
                }
            }
            if (ab()) {
                if (any) {
                    commit_to(&fbar);
                    mbar_wait(smem_u32(&fbar), 0u, kTcDrainNs);
                }
                if (tma_issued > tma_waited) mbar_wait(smem_u32(&wfull), (uint32_t)(tma_issued - 1) & 1u, kTcDrainNs);
                atomicExch(err, 1);
            }
        }
    } else {
        // every exit decision of a drain warp is warp-uniform: the tcgen05 loads
        // and stores below are warp-collective
        const unsigned full = 0xFFFFFFFFu;
        constexpr int kPer = (1 << kTcTile) / kTcmDrain;
        // copies m0 .. m1 - 1 of this thread's share of tile t's boundary elements
        // -> exchange buffer xb (window 0's map)
        auto load_tile = [&](uint32_t t, uint32_t xb, int m0, int m1) {
            const float2 *src = tile_ptr(t);
#pragma unroll
            for (int m = 0; m < kPer; ++m) {
                if (m < m0 || m >= m1) continue;
                const uint32_t i = tid + (uint32_t)m * kTcmDrain;
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(xb + (alo[i & 127] ^ ahi[i >> 7])),
                             "l"(src + (lut_lo[i & 127] | lut_hi[i >> 7]))
                             : "memory");
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        // one exchange: this warp's stores are done; wait for every drain warp's
        auto exchange = [&](uint32_t &x) {
            __syncwarp();
            if (lane == 0) mbar_arrive(&xbar);
            const bool ok = __all_sync(full, mbar_wait(smem_u32(&xbar), x & 1u, wait_ns));
            ++x;
            if (!ok) abort_sh = 1;
            return ok;
        };
        auto operand_ready = [&]() {
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) mbar_arrive(&afull);
        };
        uint32_t g = 0, x = 0;
        bool stop = false;
        load_tile(blockIdx.x, sbase, 0, kPer);   // exchange 0: buffer 0
        for (uint32_t t = blockIdx.x; t < ntiles && !stop; t += gridDim.x) {
            const uint32_t tn = t + gridDim.x;   // the CTA's next tile
            uint32_t xs = sbase + (x & 1u) * kXch;
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            if (!exchange(x)) break;
            {
                const TcXa &xa = xat[ps.rp_off];
                tm_load_operand(taddr, XchAddr(xa.ld_lane, xa.ld_warp, xa.ld_c), xs);
            }
            operand_ready();
            // exchange x (now the next tile's input) goes to the buffer whose last
            // loads (exchange x - 2) every drain warp finished before exchange x - 1
            if (nw == 1 && tn < ntiles) load_tile(tn, sbase + (x & 1u) * kXch, 0, kPer);
            for (int w = 0; w < nw; ++w, ++g) {
                if (__any_sync(full, ab())) { stop = true; break; }
                if (!__all_sync(full, mbar_wait(smem_u32(&dfull), g & 1u, wait_ns))) {
                    abort_sh = 1;
                    stop = true;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                if (w + 1 < nw) {
                    xs = sbase + (x & 1u) * kXch;
                    const TcXa &xa = xat[ps.rp_off + w], &xn = xat[ps.rp_off + w + 1];
                    tm_store_result(taddr, XchAddr(xa.st_lane, xa.st_warp, xa.st_c), xs);
                    if (!exchange(x)) { stop = true; break; }
                    tm_load_operand(taddr, XchAddr(xn.ld_lane, xn.ld_warp, xn.ld_c), xs);
                    operand_ready();
                    if (w + 2 == nw && tn < ntiles) load_tile(tn, sbase + (x & 1u) * kXch, 0, kPer);
                } else {
                    drain_tile16(taddr, sw[w], gcb, nullptr, tile_ptr(t));
                }
            }
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");   // no copy outlives the CTA
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (tid < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(taddr));
}

}  // namespace

size_t tc_wmat_bytes_per_pair(const BrickDev &d, const BrickPass *hpasses) {
    int mx = 0;
    for (int i = 0; i < d.n_passes[0] + d.n_passes[1]; ++i) mx = hpasses[i].n_rp > mx ? hpasses[i].n_rp : mx;
    return (size_t)mx * kWMat;
}

bool tc_plan_ok(const BrickDev &d, const BrickPass *hpasses, const RegPass *rps) {
    if (d.tile_bits != kTcTile || d.N < kTcTile + 1) return false;
    for (int i = 0; i < d.n_passes[0] + d.n_passes[1]; ++i) {
        const BrickPass &p = hpasses[i];
        if (p.n_rp < 1 || p.n_rp > kMaxTcWins) return false;
        for (int w = 0; w < p.n_rp; ++w)
            if (rps[p.rp_off + w].r != kMaxWin || rps[p.rp_off + w].n_gates > kMaxTcWins) return false;
    }
    return true;
}

cudaError_t run_passes_tc(const BrickDev &d, const BrickPass *hpasses, const BrickDevPlan &dp, int npairs,
                          const float2 *maps, float2 *states, float *wm, int *err, cudaStream_t st) {
    // 3: the tile's operand in shared memory, one tile per CTA; 4: in tensor memory, persistent
    const bool tm = dp.persist == 4;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = tm ? cudaFuncSetAttribute(brick_tcm_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcmSmem)
           : cudaFuncSetAttribute(brick_tc1_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTc1Smem);
    if (e != cudaSuccess) return e;
    for (int side = 0; side < 2; ++side)
        for (int p = 0; p < d.n_passes[side]; ++p) {
            const BrickPass &ps = hpasses[d.pass_off[side] + p];
            tc_wmat_kernel<<<dim3(ps.n_rp, npairs), 32, 0, st>>>(d, side, ps, dp.gates, dp.rpasses, dp.rgates, maps, wm);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            if (tm) {   // two CTAs per SM
                const uint32_t ntiles = (uint32_t)npairs << (d.N - kTcTile);
                const uint32_t grid = std::min<uint32_t>(ntiles, 2u * (uint32_t)sms);
                brick_tcm_pass_kernel<<<grid, kTcmDrain + 32, kTcmSmem, st>>>(d, side, ps, dp.tcwins, dp.tcxa, wm,
                                                                              states, err, wait_limit_ns(), ntiles);
            } else {
                brick_tc1_pass_kernel<<<dim3(1u << (d.N - kTcTile), npairs), kTc1Drain + 32, kTc1Smem, st>>>(
                    d, side, ps, dp.tcwins, wm, states, err, wait_limit_ns());
            }
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    return cudaSuccess;
}

}  // namespace fpk
