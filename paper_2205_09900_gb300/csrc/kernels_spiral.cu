// kernels_spiral.cu -- spiral sweep of the paper's hardware-efficient ansatz.
//
// The planner (make_spiral_plan) turns Tr(U^dagger V) of an ensemble whose
// wires are rings of segments, each tapped by one CZ, into a sequence of
// in-place 4x4 maps on a state of 2^bits amplitudes (one bit per CZ of a bond
// plus an auxiliary bit).  Per pair:
//   spiral_maps_kernel   builds every map from the pair's merged 1-qubit
//                        operators (FP64 products, stored in C; FP32 maps as
//                        broadcast pairs for packed FMAs);
//   spiral_win_kernel    register windows: consecutive maps on at most R
//                        state bits run on 2^R amplitudes per thread in
//                        registers, one barrier per window.  The state sits
//                        in shared memory (swizzled), in one CTA or split
//                        over a 2- or 4-CTA cluster (distributed shared memory);
//   spiral_sweep_kernel  one map per pass (small states, or states too large
//                        for four CTAs: a per-pair global slice).
// Both sweeps start from delta(aux, first bit) and end with the FP64 sum of
// the state = Tr, its cancellation ratio and rounding-error estimate.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>

#include "kernels.h"

namespace cg = cooperative_groups;

namespace fpk {
namespace {

__device__ __forceinline__ uint32_t ins0s(uint32_t x, int p) {   // insert a zero bit at position p
    return (x & ((1u << p) - 1u)) | ((x >> p) << (p + 1));
}

// Shared-memory slot of local amplitude y: y ^ fold4(y >> 4).  Linear over
// XOR, so the slot of a sum of disjoint bit groups is the XOR of their slots.
__device__ __forceinline__ uint32_t swz(uint32_t y) {
    const uint32_t q = y >> 4;
    return y ^ ((q ^ (q >> 4) ^ (q >> 8) ^ (q >> 12)) & 15u);
}

template <typename C> __device__ __forceinline__ C mk(double re, double im);
template <> __device__ __forceinline__ double2 mk<double2>(double re, double im) { return make_double2(re, im); }
template <> __device__ __forceinline__ float2 mk<float2>(double re, double im) { return make_float2((float)re, (float)im); }

__device__ __forceinline__ double2 zm(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Entries per stored map: FP64 keeps the 16 complex entries; FP32 keeps each
// entry t as the pairs (tr, tr) and (-ti, ti), so that acc += t x is two
// packed FMAs: (tr, tr) * (xr, xi) + (-ti, ti) * (xi, xr).
template <typename C> struct MapW { static constexpr int w = 16; };
template <> struct MapW<float2> { static constexpr int w = 32; };

template <typename C> __device__ __forceinline__ void put_entry(C *dst, int e, double2 t) { dst[e] = mk<C>(t.x, t.y); }
template <> __device__ __forceinline__ void put_entry<float2>(float2 *dst, int e, double2 t) {   // one 16-byte store
    *reinterpret_cast<float4 *>(dst + 2 * e) = make_float4((float)t.x, (float)t.x, (float)-t.y, (float)t.y);
}

// Entry T[4 o + f] of every map, o = o_a + 2 o_b, f = i_a + 2 i_b (SpiralType):
// one thread per entry, so the 16 threads of a map store its record contiguously.
template <typename C>
__global__ void spiral_maps_kernel(const PairInfo *__restrict__ pairs, int npairs, const SpiralMap *__restrict__ sm,
                                   int nmaps, const double2 *__restrict__ merged, C *__restrict__ maps) {
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    const int m = gid >> 4, e = gid & 15;
    if (m >= nmaps) return;
    const SpiralMap s = sm[m];
    const int o = e >> 2, f = e & 3;
    const int oa = o & 1, ob = o >> 1, ia = f & 1, ib = f >> 1;
    const double h = (ob & ib) ? -1.0 : 1.0;   // H[o_b][i_b] = (-1)^{o_b i_b}
    for (int p = blockIdx.y; p < npairs; p += gridDim.y) {   // grid.y is capped at 65535
        const int64_t mo = pairs[p].merged_off;
        // entry (r, c) of merged item k (the identity when k < 0)
        auto mat = [&](int k, int r, int c) {
            return k >= 0 ? merged[(mo + k) * 16 + 2 * r + c] : make_double2(r == c ? 1.0 : 0.0, 0.0);
        };
        double2 v = make_double2(0, 0);
        switch (s.type) {
            case SP_DIAG_BA: if (o == f) v = mat(s.g, ib, ia); break;
            case SP_START: if (oa == ob) v = make_double2(h, 0); break;
            case SP_MID: v = zm(mat(s.f, oa, ia), mat(s.g, ob, oa)); v.x *= h; v.y *= h; break;
            case SP_MID_AUX: if (ob == ib) v = zm(mat(s.f, oa, ia), mat(s.g, ob, oa)); break;
            case SP_RL: if (oa == ia) { v = mat(s.g, ob, ia); v.x *= h; v.y *= h; } break;
            case SP_MID_RR: if (ib == 0) v = zm(mat(s.f, oa, ia), mat(s.g, ob, oa)); break;
            case SP_RR: if (oa == ia && ib == 0) v = mat(s.g, ob, ia); break;
            case SP_LL: if (oa == 0) { v = mat(s.g, ob, ia); v.x *= h; v.y *= h; } break;
            case SP_LL_AUX: if (oa == 0 && ob == ib) v = mat(s.g, ib, ia); break;
            default: break;
        }
        put_entry<C>(maps + ((size_t)p * nmaps + m) * MapW<C>::w, e, v);
    }
}

__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {   // a * b + c, lane-wise
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

__device__ __forceinline__ double2 cmac(double2 t, double2 x, double2 acc) {
    acc.x = fma(t.x, x.x, acc.x);
    acc.x = fma(-t.y, x.y, acc.x);
    acc.y = fma(t.x, x.y, acc.y);
    acc.y = fma(t.y, x.x, acc.y);
    return acc;
}

// (x0, x1, x2, x3) <- T (x0, x1, x2, x3) for one stored map T
__device__ __forceinline__ void quad(double2 &x0, double2 &x1, double2 &x2, double2 &x3, const double2 (&T)[16]) {
    double2 y[4];
#pragma unroll
    for (int o = 0; o < 4; ++o) {
        double2 acc = make_double2(0, 0);
        acc = cmac(T[4 * o + 0], x0, acc);
        acc = cmac(T[4 * o + 1], x1, acc);
        acc = cmac(T[4 * o + 2], x2, acc);
        acc = cmac(T[4 * o + 3], x3, acc);
        y[o] = acc;
    }
    x0 = y[0]; x1 = y[1]; x2 = y[2]; x3 = y[3];
}
__device__ __forceinline__ void quad(float2 &x0, float2 &x1, float2 &x2, float2 &x3, const float2 (&T)[32]) {
    const float2 x[4] = {x0, x1, x2, x3};
    float2 acc[4];
#pragma unroll
    for (int o = 0; o < 4; ++o) acc[o] = make_float2(0.f, 0.f);
#pragma unroll
    for (int f = 0; f < 4; ++f) {   // the four outputs accumulate side by side
        const float2 xs = make_float2(x[f].y, x[f].x);
#pragma unroll
        for (int o = 0; o < 4; ++o) acc[o] = ffma2(T[2 * (4 * o + f)], x[f], acc[o]);
#pragma unroll
        for (int o = 0; o < 4; ++o) acc[o] = ffma2(T[2 * (4 * o + f) + 1], xs, acc[o]);
    }
    x0 = acc[0]; x1 = acc[1]; x2 = acc[2]; x3 = acc[3];
}

__device__ __forceinline__ void load_map(double2 (&T)[16], const double2 *__restrict__ src) {
#pragma unroll
    for (int e = 0; e < 16; ++e) T[e] = src[e];
}
__device__ __forceinline__ void load_map(float2 (&T)[32], const float2 *__restrict__ src) {   // 16-byte loads
    const float4 *s4 = reinterpret_cast<const float4 *>(src);
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        const float4 q = s4[e];
        T[2 * e] = make_float2(q.x, q.y);
        T[2 * e + 1] = make_float2(q.z, q.w);
    }
}

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

__device__ __forceinline__ double wsum_s(double v) {
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
    return v;
}

// Block sums of (Re, Im, |t|, |t|^2) over the amplitudes this CTA holds; the
// totals land in thread 0.
template <typename C>
__device__ __forceinline__ void block_sums(const C *st, uint32_t S, double (&red)[4][16], double (&out)[4]) {
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
        for (int c = 0; c < 4; ++c) {
            out[c] = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) out[c] += red[c][w];
        }
    }
}

__device__ __forceinline__ void write_result(const PairInfo &pi, const double (&s)[4], double err_scale, double *tr,
                                             double *kappa, double *err) {
    tr[2 * pi.out] = s[0];
    tr[2 * pi.out + 1] = s[1];
    const double mag = sqrt(s[0] * s[0] + s[1] * s[1]);
    if (kappa) kappa[pi.out] = mag > 0 ? s[2] / mag : __longlong_as_double(0x7ff0000000000000LL);
    if (err) err[pi.out] = err_scale * (sqrt(s[3]) + mag);
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
    const C *mp = maps + (size_t)blockIdx.x * nmaps * MapW<C>::w;
    for (int k = 0; k < nmaps; ++k) {
        const SpiralMap s = sm[k];
        C T[MapW<C>::w];
        load_map(T, mp + (size_t)k * MapW<C>::w);
        const int lo = s.a < s.b ? s.a : s.b, hi = s.a < s.b ? s.b : s.a;
        const uint32_t ia = 1u << s.a, ib = 1u << s.b;
        for (uint32_t q = threadIdx.x; q < (S >> 2); q += blockDim.x) {
            const uint32_t i0 = ins0s(ins0s(q, lo), hi);
            C x0 = st[i0], x1 = st[i0 | ia], x2 = st[i0 | ib], x3 = st[i0 | ia | ib];
            quad(x0, x1, x2, x3, T);
            st[i0] = x0;
            st[i0 | ia] = x1;
            st[i0 | ib] = x2;
            st[i0 | ia | ib] = x3;
        }
        __syncthreads();
    }
    double s[4];
    block_sums<C>(st, S, red, s);
    if (threadIdx.x == 0) write_result(pairs[blockIdx.x], s, err_scale, tr, kappa, err);
}

// One map on window bits (I, J) of a thread's 2^R register block.
template <typename C, int I, int J, int R>
__device__ __forceinline__ void win_map(C (&v)[1 << R], const C (&T)[MapW<C>::w]) {
#pragma unroll
    for (int x = 0; x < (1 << R); ++x) {
        if (x & ((1 << I) | (1 << J))) continue;
        quad(v[x], v[x | (1 << I)], v[x | (1 << J)], v[x | (1 << I) | (1 << J)], T);
    }
}

template <typename C, int R, int I>
__device__ __forceinline__ void win_map_j(int j, C (&v)[1 << R], const C (&T)[MapW<C>::w]) {
    switch (j) {
        case 0: if constexpr (I != 0) win_map<C, I, 0, R>(v, T); break;
        case 1: if constexpr (I != 1) win_map<C, I, 1, R>(v, T); break;
        case 2: if constexpr (I != 2 && R > 2) win_map<C, I, 2, R>(v, T); break;
        case 3: if constexpr (I != 3 && R > 3) win_map<C, I, 3, R>(v, T); break;
        case 4: if constexpr (I != 4 && R > 4) win_map<C, I, 4, R>(v, T); break;
        default: break;
    }
}

template <typename C, int R>
__device__ __forceinline__ void win_map_ij(int i, int j, C (&v)[1 << R], const C (&T)[MapW<C>::w]) {
    switch (i) {
        case 0: win_map_j<C, R, 0>(j, v, T); break;
        case 1: win_map_j<C, R, 1>(j, v, T); break;
        case 2: if constexpr (R > 2) win_map_j<C, R, 2>(j, v, T); break;
        case 3: if constexpr (R > 3) win_map_j<C, R, 3>(j, v, T); break;
        case 4: if constexpr (R > 4) win_map_j<C, R, 4>(j, v, T); break;
        default: break;
    }
}

// Distributed shared memory through 32-bit shared::cluster addresses.
__device__ __forceinline__ uint32_t cluster_addr(const void *p, uint32_t rank) {
    uint32_t a = (uint32_t)__cvta_generic_to_shared(p), r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ float2 dsm_ld(uint32_t a, float2) {
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ double2 dsm_ld(uint32_t a, double2) {
    double2 v;
    asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void dsm_st(uint32_t a, float2 v) {
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ void dsm_st(uint32_t a, double2 v) {
    asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};" ::"r"(a), "d"(v.x), "d"(v.y) : "memory");
}

template <int CL>
__device__ __forceinline__ void win_sync(bool cluster_wide) {
    if constexpr (CL > 1) {
        if (cluster_wide) { cg::this_cluster().sync(); return; }
    }
    __syncthreads();
}

__device__ __forceinline__ uint32_t del_bit(uint32_t x, int p) {   // remove bit p
    return (x & ((1u << p) - 1u)) | ((x >> (p + 1)) << p);
}

template <int CL>
__device__ __forceinline__ uint32_t pick_cta(const uint32_t (&ac)[CL], uint32_t r) {
    if constexpr (CL == 1) return ac[0];
    else if constexpr (CL == 2) return r ? ac[1] : ac[0];
    else return (r & 2) ? ((r & 1) ? ac[3] : ac[2]) : ((r & 1) ? ac[1] : ac[0]);
}

// Register windows over a state held in the shared memory of CL = 1, 2 or 4
// CTAs (one pair per CTA or per cluster).  With CL > 1 the cluster bits h0
// (and h1) of an amplitude give its CTA rank; a window holding one of them
// ("cross" window) reads and writes other CTAs' parts through distributed
// shared memory and is fenced by cluster barriers; the other windows stay in
// their own CTA.  Addressing: SpiralWin.
// Threads per CTA: the FP32 two-CTA form runs one CTA per SM (its half of the
// state fills the shared memory), so it takes as many warps as its registers allow.
template <typename C, int CL> struct WinThreads { static constexpr int n = 256; };
template <> struct WinThreads<float2, 2> { static constexpr int n = 512; };

template <typename C, int R, int CL>
__global__ void __launch_bounds__(WinThreads<C, CL>::n) spiral_win_kernel(const PairInfo *__restrict__ pairs,
                                                         const SpiralWin *__restrict__ wins, int nwins,
                                                         const uint8_t *__restrict__ ij, int nmaps, int bits,
                                                         int first_bit, int h0, int h1, const C *__restrict__ maps,
                                                         double err_scale, double *__restrict__ tr,
                                                         double *__restrict__ kappa, double *__restrict__ err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[4][16];
    __shared__ double part[3][4];   // CL > 1: ranks 1.. write their sums into rank 0
    constexpr int c = CL == 4 ? 2 : (CL == 2 ? 1 : 0);
    constexpr int MB = kSpiralWinMaxMaps * MapW<C>::w;   // elements of one staged window of maps
    C *st = (C *)smem_raw;
    const uint32_t SL = 1u << (bits - c);
    C *mbuf = st + SL;   // two windows of maps: this one and the next (cp.async)
    uint32_t rank = 0, ac[CL];   // ac[r]: rank r's part in the cluster window
    double *part0 = &part[0][0];
    if constexpr (CL > 1) {
        cg::cluster_group cl = cg::this_cluster();
        rank = cl.block_rank();
#pragma unroll
        for (int r = 0; r < CL; ++r) ac[r] = cluster_addr(st, r);
        part0 = cl.map_shared_rank(&part[0][0], 0);
    } else {
        ac[0] = 0;
    }
    const int aux = bits - 1;
    for (uint32_t y = threadIdx.x; y < SL; y += blockDim.x) {
        uint32_t x = y;
        if constexpr (c >= 1) x = ins0s(x, h0) | ((rank & 1u) << h0);
        if constexpr (c == 2) x = ins0s(x, h1) | (((rank >> 1) & 1u) << h1);
        st[swz(y)] = mk<C>((((x >> aux) ^ (x >> first_bit)) & 1u) ? 0.0 : 1.0, 0.0);
    }
    const C *mp = maps + (size_t)(blockIdx.x / CL) * nmaps * MapW<C>::w;
    // 16-byte chunks of window v's maps into buffer v & 1
    auto stage = [&](int v) {
        const int chunks = wins[v].n_maps * (int)(MapW<C>::w * sizeof(C) / 16);
        const unsigned char *src = (const unsigned char *)(mp + (size_t)wins[v].first * MapW<C>::w);
        unsigned char *dst = (unsigned char *)(mbuf + (v & 1) * MB);
        for (int q = threadIdx.x; q < chunks; q += blockDim.x) cp_async16(dst + 16 * q, src + 16 * q);
    };
    if (nwins > 0) stage(0);
    cp_async_wait_all();
    win_sync<CL>(true);   // with CL > 1 also: every part exists before any remote access
    const uint32_t G = 1u << (bits - R - c);   // groups this CTA handles per window
    for (int w = 0; w < nwins; ++w) {
        const SpiralWin &W = wins[w];   // uniform reads (read-only path)
        const int n_pos = W.n_pos, first = W.first, n_maps = W.n_maps;
        const bool cross = CL > 1 && W.cross;
        if (w + 1 < nwins) stage(w + 1);   // lands while this window computes
        const C *mw = mbuf + (w & 1) * MB;
        uint32_t off[R], ctab[R];
#pragma unroll
        for (int k = 0; k < R; ++k) { off[k] = W.off[k]; ctab[k] = W.ctab[k]; }
        for (uint32_t t = threadIdx.x; t < G; t += blockDim.x) {
            const uint32_t tt = rank * G + t;
            uint32_t b = 0;
            for (int j = 0; j < n_pos; ++j) b |= ((tt >> j) & 1u) << W.pos[j];
            uint32_t cb = 0, lb = b;
            if constexpr (c == 2) { cb = ((b >> h0) & 1u) | (((b >> h1) & 1u) << 1); lb = del_bit(del_bit(b, h1), h0); }
            if constexpr (c == 1) { cb = (b >> h0) & 1u; lb = del_bit(b, h0); }
            uint32_t pb = swz(lb);
            C v[1 << R];
            if (!cross) {
#pragma unroll
                for (int i = 0; i < (1 << R); ++i) {
                    uint32_t a = pb;
#pragma unroll
                    for (int k = 0; k < R; ++k) if ((i >> k) & 1) a ^= off[k];
                    v[i] = st[a];
                }
            } else {
#pragma unroll
                for (int i = 0; i < (1 << R); ++i) {
                    uint32_t a = pb, r = cb;
#pragma unroll
                    for (int k = 0; k < R; ++k) if ((i >> k) & 1) { a ^= off[k]; r ^= ctab[k]; }
                    v[i] = dsm_ld(pick_cta<CL>(ac, r) + a * (uint32_t)sizeof(C), C());
                }
            }
            for (int m = 0; m < n_maps; ++m) {
                C T[MapW<C>::w];
                load_map(T, mw + m * MapW<C>::w);
                const int q = ij[first + m];
                win_map_ij<C, R>(q & 15, q >> 4, v, T);
            }
            // the store addresses are rebuilt from pb (not kept live across the maps)
            asm volatile("" : "+r"(pb), "+r"(cb));
            if (!cross) {
#pragma unroll
                for (int i = 0; i < (1 << R); ++i) {
                    uint32_t a = pb;
#pragma unroll
                    for (int k = 0; k < R; ++k) if ((i >> k) & 1) a ^= off[k];
                    st[a] = v[i];
                }
            } else {
#pragma unroll
                for (int i = 0; i < (1 << R); ++i) {
                    uint32_t a = pb, r = cb;
#pragma unroll
                    for (int k = 0; k < R; ++k) if ((i >> k) & 1) { a ^= off[k]; r ^= ctab[k]; }
                    dsm_st(pick_cta<CL>(ac, r) + a * (uint32_t)sizeof(C), v[i]);
                }
            }
        }
        const bool next_cross = CL > 1 && w + 1 < nwins && wins[w + 1].cross;
        cp_async_wait_all();   // the next window's maps are in place before the barrier
        win_sync<CL>(cross || next_cross);
    }
    double s[4];
    block_sums<C>(st, SL, red, s);
    if constexpr (CL > 1) {
        if (rank > 0 && threadIdx.x == 0)
            for (int k = 0; k < 4; ++k) part0[(rank - 1) * 4 + k] = s[k];
        cg::this_cluster().sync();   // every rank's sums are in rank 0; ranks > 0 may exit after this
        if (rank == 0 && threadIdx.x == 0) {
            for (int r = 1; r < CL; ++r)
                for (int k = 0; k < 4; ++k) s[k] += part[r - 1][k];
            write_result(pairs[blockIdx.x / CL], s, err_scale, tr, kappa, err);
        }
    } else {
        if (threadIdx.x == 0) write_result(pairs[blockIdx.x], s, err_scale, tr, kappa, err);
    }
}

template <typename C, int R, int CL>
cudaError_t win_t(const PairInfo *pairs, int npairs, const SpiralWin *wins, int nwins, const uint8_t *ij, int nmaps,
                  int bits, int first_bit, const int *h, const void *maps, double err_scale, double *tr, double *kappa,
                  double *err, cudaStream_t st) {
    constexpr int c = CL == 4 ? 2 : (CL == 2 ? 1 : 0);
    const size_t bytes = (((size_t)1 << (bits - c)) + 2 * kSpiralWinMaxMaps * MapW<C>::w) * sizeof(C);
    const uint32_t G = 1u << (bits - R - c);
    const int threads = (int)std::min<uint32_t>(WinThreads<C, CL>::n, std::max<uint32_t>(32u, G));
    auto k = spiral_win_kernel<C, R, CL>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3((unsigned)(npairs * CL));
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = bytes;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, pairs, wins, nwins, ij, nmaps, bits, first_bit, h[0], h[1], (const C *)maps,
                              err_scale, tr, kappa, err);
}

template <typename C>
cudaError_t sweep_t(const PairInfo *pairs, int npairs, const SpiralMap *sm, int nmaps, int bits, int first_bit,
                    const void *maps, void *scratch, double err_scale, double *tr, double *kappa, double *err,
                    cudaStream_t st) {
    const size_t bytes = ((size_t)1 << bits) * sizeof(C);
    const int threads = bits >= 11 ? 512 : (bits >= 9 ? 128 : 32);
    if (bytes <= kSpiralSmemMax) {
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

size_t spiral_map_elems(bool fp32) { return fp32 ? MapW<float2>::w : MapW<double2>::w; }

SpiralConfig spiral_config(int bits, bool fp32, int min_split) {
    SpiralConfig c;
    const size_t bytes = ((size_t)1 << bits) * (fp32 ? sizeof(float2) : sizeof(double2));
    c.split = bytes <= kSpiralSmemMax ? 0 : bytes <= 2 * kSpiralSmemMax ? 1 : bytes <= 4 * kSpiralSmemMax ? 2 : -1;
    if (const char *ev = std::getenv("FP_SPIRAL_SPLIT")) min_split = std::max(min_split, std::atoi(ev));   // tuning
    if (c.split >= 0) c.split = std::max(c.split, std::min(min_split, 2));
    // measured on GB300 (n = 50, depths 5..8): 5-bit windows from 2^13 FP32
    // amplitudes up, else 4
    c.R = fp32 && bits >= 13 ? 5 : 4;
    if (const char *ev = std::getenv("FP_SPIRAL_WIN")) c.R = std::atoi(ev);   // tuning override: 0, 4 or 5
    if (c.R != 0 && c.R != 4 && !(c.R == 5 && fp32)) c.R = 4;
    // windows need 16 lane groups per CTA and a state in (distributed) shared memory
    if (c.split < 0 || bits - c.R - c.split < 4 || bits - c.R > kSpiralMaxPos) c.R = 0;
    if (c.R == 0) c.split = 0;
    c.scratch_elems = (c.R == 0 && bytes > kSpiralSmemMax) ? ((size_t)1 << bits) : 0;
    return c;
}

cudaError_t launch_spiral(const PairInfo *pairs, int npairs, const SpiralMap *sm, int nmaps, int bits, int first_bit,
                          const SpiralConfig &cfg, const SpiralWin *wins, int nwins, const uint8_t *ij, const int *h,
                          const double2 *merged, void *maps, void *scratch, bool fp32, double err_scale, double *tr,
                          double *kappa, double *err, cudaStream_t st) {
    if (npairs <= 0) return cudaSuccess;
    dim3 gm((16 * nmaps + 255) / 256, std::min(npairs, 65535));
    if (fp32) spiral_maps_kernel<float2><<<gm, 256, 0, st>>>(pairs, npairs, sm, nmaps, merged, (float2 *)maps);
    else spiral_maps_kernel<double2><<<gm, 256, 0, st>>>(pairs, npairs, sm, nmaps, merged, (double2 *)maps);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (wins && cfg.R > 0) {
#define FP_SPIRAL_WIN_CASE(C, R, CL)                                                                               \
    return win_t<C, R, CL>(pairs, npairs, wins, nwins, ij, nmaps, bits, first_bit, h, maps, err_scale, tr, kappa, \
                           err, st)
        const int CL = 1 << cfg.split;
        if (!fp32) {
            if (cfg.R != 4) return cudaErrorInvalidValue;
            if (CL == 1) FP_SPIRAL_WIN_CASE(double2, 4, 1);
            if (CL == 2) FP_SPIRAL_WIN_CASE(double2, 4, 2);
            if (CL == 4) FP_SPIRAL_WIN_CASE(double2, 4, 4);
        } else if (cfg.R == 4) {
            if (CL == 1) FP_SPIRAL_WIN_CASE(float2, 4, 1);
            if (CL == 2) FP_SPIRAL_WIN_CASE(float2, 4, 2);
            if (CL == 4) FP_SPIRAL_WIN_CASE(float2, 4, 4);
        } else if (cfg.R == 5) {
            if (CL == 1) FP_SPIRAL_WIN_CASE(float2, 5, 1);
            if (CL == 2) FP_SPIRAL_WIN_CASE(float2, 5, 2);
            if (CL == 4) FP_SPIRAL_WIN_CASE(float2, 5, 4);
        }
#undef FP_SPIRAL_WIN_CASE
        return cudaErrorInvalidValue;
    }
    return fp32 ? sweep_t<float2>(pairs, npairs, sm, nmaps, bits, first_bit, maps, scratch, err_scale, tr, kappa, err, st)
                : sweep_t<double2>(pairs, npairs, sm, nmaps, bits, first_bit, maps, scratch, err_scale, tr, kappa, err, st);
}

}  // namespace fpk
