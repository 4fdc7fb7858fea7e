// kernels_brick.cu -- brickwork fast path (dual-circuit boundary sweep).
//
// K2b  brick_maps:  merged gate of every (bond, position) realigned into the
//                   4x4 map the sweep applies (FP64 products, stored FP32/FP64).
// K3/5 brick_smem:  boundaries up to 2^KS amplitudes: one CTA (or one warp for
//                   tiny boundaries) sweeps both chain halves in shared memory
//                   and meets them in an FP64 dot product.
// K4   brick_pass:  larger boundaries live in global memory; each launch runs
//                   one light-cone pass: a CTA loads a 2^K-amplitude tile (a
//                   contiguous cyclic arc of the segment ring), applies every
//                   gate of the pass inside shared memory, and stores it back.
// K6   brick_dot:   FP64 meet of the two boundaries with the cancellation ratio.
#include <cuda_runtime.h>

#include <algorithm>

#include "brick.h"
#include "kernels.h"

namespace fpk {
namespace {

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }

template <typename C> __device__ __forceinline__ C from_z(double2 z);
template <> __device__ __forceinline__ double2 from_z<double2>(double2 z) { return z; }
template <> __device__ __forceinline__ float2 from_z<float2>(double2 z) { return make_float2((float)z.x, (float)z.y); }

template <typename C>
__device__ __forceinline__ C cfma2(C a, C b, C acc) {   // acc + a*b
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
    return acc;
}

__device__ __forceinline__ uint32_t ins0(uint32_t x, int p) {   // insert a zero bit at position p
    return (x & ((1u << p) - 1u)) | ((x >> p) << (p + 1));
}

// 4x4 map on bits (pa: e bit 0, pb: e bit 1) of quad q (q indexes the other bits)
template <typename C>
__device__ __forceinline__ void quad_apply(C *__restrict__ s, uint32_t q, int pa, int pb, const C (&T)[16]) {
    const int lo = pa < pb ? pa : pb, hi = pa < pb ? pb : pa;
    const uint32_t i0 = ins0(ins0(q, lo), hi);
    const uint32_t ia = 1u << pa, ib = 1u << pb;
    C x0 = s[i0], x1 = s[i0 | ia], x2 = s[i0 | ib], x3 = s[i0 | ia | ib];
    C y[4];
#pragma unroll
    for (int o = 0; o < 4; ++o) {
        C acc;
        acc.x = 0; acc.y = 0;
        acc = cfma2(T[4 * o + 0], x0, acc);
        acc = cfma2(T[4 * o + 1], x1, acc);
        acc = cfma2(T[4 * o + 2], x2, acc);
        acc = cfma2(T[4 * o + 3], x3, acc);
        y[o] = acc;
    }
    s[i0] = y[0];
    s[i0 | ia] = y[1];
    s[i0 | ib] = y[2];
    s[i0 | ia | ib] = y[3];
}

template <typename C>
__device__ __forceinline__ void load_map(const C *__restrict__ g, C (&T)[16]) {
#pragma unroll
    for (int e = 0; e < 16; ++e) T[e] = g[e];
}

// product-of-deltas start state at a chain end: delta(w_tau, w_tau+1) for tau of parity `par`
__device__ __forceinline__ bool delta_ok(uint32_t w, int N, int par) {
    uint32_t rot = (w >> 1) | ((w & 1u) << (N - 1));   // bit tau = w_{tau+1}
    uint32_t pm = (par ? 0xAAAAAAAAu : 0x55555555u) & ((N >= 32) ? 0xFFFFFFFFu : ((1u << N) - 1u));
    return ((w ^ rot) & pm) == 0;
}

template <typename C>
__device__ __forceinline__ void store_map(C *out, const double2 (&G)[16]) {
#pragma unroll
    for (int e = 0; e < 16; ++e) out[e] = from_z<C>(G[e]);
}

template <typename C>
__global__ void brick_maps_kernel(BrickDev d, const PairInfo *__restrict__ pairs, const double2 *__restrict__ raw,
                                  C *__restrict__ maps) {
    const PairInfo pi = pairs[blockIdx.y];
    const int m = d.m, l = d.l;
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= maps_per_pair(d)) return;
    const int g = id / m, j = id % m;
    const int side = g < d.n_layers[0] ? 0 : 1, t = side ? g - d.n_layers[0] : g;
    const double2 *U = raw + pi.raw_off * 16;
    const double2 *V = raw + (pi.raw_off + pi.n_raw) * 16;
    C *out = maps + ((size_t)blockIdx.y * maps_per_pair(d) + id) * 16;
    double2 M[16];
    if (d.kind == 1) {
        // HEA: rotation slot s of qubit q as a diagonal map, with H x H on odd layers
        const int q = side == 0 ? t / 2 : d.n - 1 - t / 2;
        const int half = t % 2, N = d.N, L = l;
        const int s = half == 0 ? 2 * j + 1 : (2 * j + 2) % N;
        auto rot = [&](const double2 *C0, int tl) { return C0 + ((size_t)(tl - 1) * d.n + q) * 16; };
        double2 R[4];
        if (s == 0 || s == L - 1) {
            const int tl = s == 0 ? 1 : L;
            const double2 *A = rot(U, tl), *B = rot(V, tl);
            // s = 0: R_1^V R_1^U^dagger ; s = L-1: R_L^U^dagger R_L^V
            for (int r = 0; r < 2; ++r)
                for (int c = 0; c < 2; ++c) {
                    double2 acc = make_double2(0, 0);
                    for (int k = 0; k < 2; ++k) {
                        double2 t1 = s == 0 ? zmul(B[2 * r + k], zconj(A[2 * c + k])) : zmul(zconj(A[2 * k + r]), B[2 * k + c]);
                        acc.x += t1.x; acc.y += t1.y;
                    }
                    R[2 * r + c] = acc;
                }
        } else if (s <= L - 2) {
            const double2 *A = rot(V, s + 1);
            for (int e = 0; e < 4; ++e) R[e] = A[e];
        } else {
            const double2 *A = rot(U, 2 * L - 1 - s);
            for (int r = 0; r < 2; ++r)
                for (int c = 0; c < 2; ++c) R[2 * r + c] = zconj(A[2 * c + r]);
        }
        // diagonal factor D[e], e = y_in + 2 y_out (bit 0: segment s-1, bit 1: segment s)
        const bool ladder = half == 1 && !(side == 1 && q == d.cut);
        for (int xe = 0; xe < 4; ++xe)
            for (int ye = 0; ye < 4; ++ye) {
                double2 v = make_double2(0, 0);
                if (ladder) {
                    const int sgn = ((xe & 1) & (ye & 1)) ^ ((xe >> 1) & (ye >> 1));
                    v = R[ye];
                    if (sgn) { v.x = -v.x; v.y = -v.y; }
                } else if (xe == ye) {
                    v = R[ye];
                }
                M[4 * xe + ye] = v;
            }
        store_map(out, M);
        return;
    }
    // brickwork
    const int b = brick_bond(d, side, t);
    const int tau = 2 * j + (b + 1) % 2;
    const int c0 = d.n / 2, c1 = (d.n - 1) / 2;
    auto gidx = [&](int tl) {   // raw index of layer tl (1-based) on bond b
        int tm = tl - 1;
        return ((tm + 1) / 2) * c0 + (tm / 2) * c1 + (b - tm % 2) / 2;
    };
    double2 G[16];
    if (tau <= l - 3) {
        const double2 *A = V + (size_t)gidx(tau + 2) * 16;
#pragma unroll
        for (int e = 0; e < 16; ++e) G[e] = A[e];
    } else if (tau == l - 2 || tau == 2 * l - 3) {
        const int tl = tau == l - 2 ? l : 1;
        const double2 *A = U + (size_t)gidx(tl) * 16, *B = V + (size_t)gidx(tl) * 16;
        // tau = l-2: U_l^dagger V_l ; tau = 2l-3: V_1 U_1^dagger
        for (int r = 0; r < 4; ++r)
            for (int c = 0; c < 4; ++c) {
                double2 acc = make_double2(0, 0);
                for (int k = 0; k < 4; ++k) {
                    double2 t1 = tau == l - 2 ? zmul(zconj(A[4 * k + r]), B[4 * k + c])
                                              : zmul(B[4 * r + k], zconj(A[4 * c + k]));
                    acc.x += t1.x; acc.y += t1.y;
                }
                G[4 * r + c] = acc;
            }
    } else {
        const double2 *A = U + (size_t)gidx(2 * l - 2 - tau) * 16;
        for (int r = 0; r < 4; ++r)
            for (int c = 0; c < 4; ++c) G[4 * r + c] = zconj(A[4 * c + r]);
    }
    const bool left = side == 0;
#pragma unroll
    for (int xt = 0; xt < 2; ++xt)
#pragma unroll
        for (int xt1 = 0; xt1 < 2; ++xt1)
#pragma unroll
            for (int yt = 0; yt < 2; ++yt)
#pragma unroll
                for (int yt1 = 0; yt1 < 2; ++yt1) {
                    double2 gv = G[(yt1 * 2 + xt1) * 4 + (yt * 2 + xt)];
                    int ex = xt + 2 * xt1, ey = yt + 2 * yt1;
                    M[left ? ex * 4 + ey : ey * 4 + ex] = gv;
                }
    store_map(out, M);
}

// Accumulators of the meet: the trace sum in FP64; the |t| and |t|^2 sums
// (cancellation ratio, error estimate) in the boundary precision per thread,
// combined in FP64 across threads.  A term t = L_j R_j is formed in the
// boundary's own precision (one rounding of values that carry FP32 rounding
// already); FP64 conversions and square roots are costly on this part.
template <typename C> struct MeetAcc;
template <> struct MeetAcc<float2> {
    double sr = 0, si = 0;
    float sa = 0, s2 = 0;
    float fr = 0, fi = 0;   // the current run of products, folded into sr, si by flush
    __device__ __forceinline__ void add(float2 l, float2 r) {
        const float px = fmaf(l.x, r.x, -l.y * r.y), py = fmaf(l.x, r.y, l.y * r.x);
        const float q = fmaf(px, px, py * py);
        fr += px;
        fi += py;
        sa += sqrtf(q);
        s2 += q;
    }
    __device__ __forceinline__ void flush() {
        sr += (double)fr;
        si += (double)fi;
        fr = fi = 0;
    }
};
template <> struct MeetAcc<double2> {
    double sr = 0, si = 0, sa = 0, s2 = 0;
    __device__ __forceinline__ void add(double2 l, double2 r) {
        const double px = l.x * r.x - l.y * r.y, py = l.x * r.y + l.y * r.x;
        const double q = px * px + py * py;
        sr += px; si += py; sa += sqrt(q); s2 += q;
    }
    __device__ __forceinline__ void flush() {}
};

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
    return v;
}

// Asynchronous global -> shared copies (cp.async): every element of a tile
// is requested before any is waited for, so a tile load costs about one
// memory latency instead of one per few elements.
template <int BYTES>
__device__ __forceinline__ void cp_async(void *smem_dst, const void *gmem_src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(gmem_src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// Whole boundary in shared memory.  `gt` threads per pair: 32 (warp mode,
// several pairs per CTA) or blockDim.x (one pair per CTA).  With `stage_maps`
// the pair's gate maps are copied next to the boundary (cp.async) before the
// sweep, so that every gate reads its map from shared memory.
template <typename C>
__global__ void __launch_bounds__(512) brick_smem_kernel(BrickDev d, const PairInfo *__restrict__ pairs, int npairs,
                                                         const C *__restrict__ maps, C *__restrict__ lscratch,
                                                         int gt, int both, int stage_maps, double err_scale,
                                                         double *__restrict__ tr, double *__restrict__ kappa,
                                                         double *__restrict__ err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[4][16];
    C *sm = (C *)smem_raw;
    const int N = d.N, m = d.m;
    const uint32_t S = 1u << N;
    const bool warp_mode = gt == 32;
    const int gpc = blockDim.x / gt;
    const int grp = threadIdx.x / gt, tid = threadIdx.x % gt;
    const int pidx = blockIdx.x * gpc + grp;
    if (warp_mode && pidx >= npairs) return;   // whole warps only: no block barrier in warp mode
    auto sync = [&]() {
        if (warp_mode) __syncwarp();
        else __syncthreads();
    };
    const size_t mpp = (size_t)maps_per_pair(d) * 16;
    C *A = sm + (size_t)grp * ((both ? 2 : 1) * (size_t)S + (stage_maps ? mpp : 0));
    C *Lp = both ? A + S : lscratch + (size_t)pidx * S;
    const C *mp = maps + (size_t)pidx * mpp;
    if (stage_maps) {   // visible to the group after the first sync() below
        C *ms = A + (both ? 2 : 1) * (size_t)S;
        for (size_t i = tid; i < mpp; i += gt) cp_async<sizeof(C)>(&ms[i], &mp[i]);
        cp_async_wait_all();
        mp = ms;
    }
    for (int side = 0; side < 2; ++side) {
        for (uint32_t w = tid; w < S; w += gt) {
            C v;
            v.x = (d.kind == 1 || delta_ok(w, N, d.delta_par[side])) ? 1 : 0;
            v.y = 0;
            A[w] = v;
        }
        sync();
        for (int t = 0; t < d.n_layers[side]; ++t) {
            const int par = layer_parity(d, side, t);
            for (int j = 0; j < m; ++j) {
                C T[16];
                load_map(mp + (size_t)map_index(d, side, t, j) * 16, T);
                const int tau = 2 * j + par;
                const int pa = tau, pb = (tau + 1) % N;
                for (uint32_t q = tid; q < (S >> 2); q += gt) quad_apply(A, q, pa, pb, T);
                sync();
            }
        }
        if (side == 0) {
            for (uint32_t w = tid; w < S; w += gt) Lp[w] = A[w];
            sync();
        }
    }
    MeetAcc<C> acc;   // runs of 8 products summed in FP32 (FP32 states), then in FP64
    int run = 0;
    for (uint32_t w = tid; w < S; w += gt) {
        acc.add(Lp[w], A[w]);
        if (++run == 8) {
            acc.flush();
            run = 0;
        }
    }
    acc.flush();
    double sr = acc.sr, si = acc.si, sa = (double)acc.sa, s2 = (double)acc.s2;
    sr = wsum(sr); si = wsum(si); sa = wsum(sa); s2 = wsum(s2);
    if (!warp_mode) {
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        if (lane == 0) { red[0][wid] = sr; red[1][wid] = si; red[2][wid] = sa; red[3][wid] = s2; }
        __syncthreads();
        if (threadIdx.x == 0) {
            sr = si = sa = s2 = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { sr += red[0][w]; si += red[1][w]; sa += red[2][w]; s2 += red[3][w]; }
        }
    }
    if (tid == 0) {
        const PairInfo pi = pairs[pidx];
        tr[2 * pi.out] = sr;
        tr[2 * pi.out + 1] = si;
        double mag = sqrt(sr * sr + si * si);
        if (kappa) kappa[pi.out] = mag > 0 ? sa / mag : __longlong_as_double(0x7ff0000000000000LL);
        if (err) err[pi.out] = err_scale * (sqrt(s2) + mag);
    }
}

template <typename C>
__global__ void brick_init_kernel(BrickDev d, int npairs, C *__restrict__ states) {
    const uint32_t S = 1u << d.N;
    const size_t total = (size_t)npairs * 2 * S;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int side = (int)((i >> d.N) & 1);
        C v;
        v.x = (d.kind == 1 || delta_ok((uint32_t)(i & (S - 1)), d.N, d.delta_par[side])) ? 1 : 0;
        v.y = 0;
        states[i] = v;
    }
}

// Shared-memory tile layout: the low 4 index bits are XORed with a linear
// (over GF(2)) function of the higher bits, chosen per pass on the host
// (BrickPass::swz) so that the lanes reading one register window spread over
// all banks.  Linearity makes swz(a ^ b) = swz(a) ^ swz(b), so an address
// built from disjoint bit groups is the XOR of their swizzled parts.

// Packed FP32 pair FMA (two lanes per instruction): d = a * b + c lane-wise.
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

// Map entries as staged in shared memory: FP64 keeps the complex entry; FP32
// keeps two broadcast pairs (tr, tr) and (-ti, ti) so that a complex
// multiply-add is two packed FMAs: acc += (tr,tr)*(xr,xi) + (-ti,ti)*(xi,xr).
template <typename C> struct MapSlot { static constexpr int width = 16; };
template <> struct MapSlot<float2> { static constexpr int width = 32; };

template <typename C>
__device__ __forceinline__ void stage_entry(C *dst, int e, C t) { dst[e] = t; }
template <>
__device__ __forceinline__ void stage_entry<float2>(float2 *dst, int e, float2 t) {
    dst[2 * e] = make_float2(t.x, t.x);
    dst[2 * e + 1] = make_float2(-t.y, t.y);
}

// 4x4 map on register bits (k, k+1) of a 2^R register block.
template <typename C, int k, int R>
struct WinApply {
    static __device__ __forceinline__ void run(C (&v)[1 << R], const C *__restrict__ T);
};

template <int k, int R>
struct WinApply<float2, k, R> {
    static __device__ __forceinline__ void run(float2 (&v)[1 << R], const float2 *__restrict__ T) {
        float2 t[32];
#pragma unroll
        for (int e = 0; e < 32; ++e) t[e] = T[e];
        // the four outputs of a quad accumulate side by side (inputs outer,
        // outputs inner), so consecutive packed FMAs are independent
#pragma unroll
        for (int i = 0; i < (1 << R); ++i) {
            if (i & (3 << k)) continue;
            float2 x[4], xs[4], acc[4];
            x[0] = v[i]; x[1] = v[i | (1 << k)]; x[2] = v[i | (2 << k)]; x[3] = v[i | (3 << k)];
#pragma unroll
            for (int f = 0; f < 4; ++f) xs[f] = make_float2(x[f].y, x[f].x);
#pragma unroll
            for (int o = 0; o < 4; ++o) acc[o] = make_float2(0.f, 0.f);
#pragma unroll
            for (int f = 0; f < 4; ++f) {
#pragma unroll
                for (int o = 0; o < 4; ++o) acc[o] = ffma2(t[2 * (4 * o + f)], x[f], acc[o]);
#pragma unroll
                for (int o = 0; o < 4; ++o) acc[o] = ffma2(t[2 * (4 * o + f) + 1], xs[f], acc[o]);
            }
#pragma unroll
            for (int o = 0; o < 4; ++o) v[i | (o << k)] = acc[o];
        }
    }
};

template <int k, int R>
struct WinApply<double2, k, R> {
    static __device__ __forceinline__ void run(double2 (&v)[1 << R], const double2 *__restrict__ T) {
        double2 t[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) t[e] = T[e];
#pragma unroll
        for (int i = 0; i < (1 << R); ++i) {
            if (i & (3 << k)) continue;
            double2 x0 = v[i], x1 = v[i | (1 << k)], x2 = v[i | (2 << k)], x3 = v[i | (3 << k)];
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                double2 acc = make_double2(0, 0);
                acc = cfma2(t[4 * o + 0], x0, acc);
                acc = cfma2(t[4 * o + 1], x1, acc);
                acc = cfma2(t[4 * o + 2], x2, acc);
                acc = cfma2(t[4 * o + 3], x3, acc);
                v[i | (o << k)] = acc;
            }
        }
    }
};

template <typename C, int k, int R>
__device__ __forceinline__ void win_apply(C (&v)[1 << R], const C *__restrict__ T) {
    WinApply<C, k, R>::run(v, T);
}

// (generic complex version, kept for reference by the shared-memory kernel)
template <typename C, int k, int R>
__device__ __forceinline__ void win_apply_plain(C (&v)[1 << R], const C *__restrict__ T) {
    C t[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) t[e] = T[e];
#pragma unroll
    for (int i = 0; i < (1 << R); ++i) {
        if (i & (3 << k)) continue;
        C x0 = v[i], x1 = v[i | (1 << k)], x2 = v[i | (2 << k)], x3 = v[i | (3 << k)];
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            C acc;
            acc.x = 0; acc.y = 0;
            acc = cfma2(t[4 * o + 0], x0, acc);
            acc = cfma2(t[4 * o + 1], x1, acc);
            acc = cfma2(t[4 * o + 2], x2, acc);
            acc = cfma2(t[4 * o + 3], x3, acc);
            v[i | (o << k)] = acc;
        }
    }
}

template <typename C, int R>
__device__ __forceinline__ void win_dispatch(int type, C (&v)[1 << R], const C *__restrict__ T) {
    switch (type) {
        case 0: win_apply<C, 0, R>(v, T); break;
        case 1: if constexpr (R > 2) win_apply<C, 1, R>(v, T); break;
        case 2: if constexpr (R > 3) win_apply<C, 2, R>(v, T); break;
        case 3: if constexpr (R > 4) win_apply<C, 3, R>(v, T); break;
        default: break;
    }
}

constexpr int kMaxRegPasses = 160;


// The register passes of one tile pass over a tile in shared memory: every
// thread holds 2^R amplitudes of a window in registers, applies the window's
// gates, writes them back; one barrier per window.
// The pass's tile layout (BrickPass::swz): element i at i ^ shi[i >> 4].
template <int K, int TH>
__device__ __forceinline__ void swizzle_table(const BrickPass &ps, uint8_t *shi) {
    for (int h = threadIdx.x; h < (1 << (K - 4)); h += TH) {
        uint32_t v = 0;
        for (int j = 0; j < K - 4; ++j)
            if ((h >> j) & 1) v ^= ps.swz[j];
        shi[h] = (uint8_t)v;
    }
}
__device__ __forceinline__ uint32_t swzt(const uint8_t *shi, uint32_t i) { return i ^ shi[i >> 4]; }

template <typename C, int K, int R, int TH>
__device__ __forceinline__ void tile_register_passes(C *__restrict__ tile, const C *__restrict__ smaps,
                                                     const RegPass *__restrict__ srp, const RegGate *__restrict__ srg,
                                                     int n_rp, int g0, const uint8_t *__restrict__ shi) {
    constexpr int MW = MapSlot<C>::width;
    for (int p = 0; p < n_rp; ++p) {
        const RegPass rp = srp[p];
        uint32_t sw[R];
#pragma unroll
        for (int k = 0; k < R; ++k) sw[k] = swzt(shi, 1u << rp.win[k]);
        for (uint32_t t = threadIdx.x; t < (1u << (K - R)); t += TH) {
            uint32_t b0 = t;
#pragma unroll
            for (int k = 0; k < R; ++k) b0 = ins0(b0, rp.srt[k]);
            uint32_t sb = swzt(shi, b0);
            C v[1 << R];
#pragma unroll
            for (int i = 0; i < (1 << R); ++i) {
                uint32_t a = sb;
#pragma unroll
                for (int k = 0; k < R; ++k) if ((i >> k) & 1) a ^= sw[k];
                v[i] = tile[a];
            }
            for (int g = 0; g < rp.n_gates; ++g) {
                const RegGate rg = srg[rp.gate_off - g0 + g];
                win_dispatch<C, R>(rg.type, v, smaps + rg.slot * MW);
            }
            // the store addresses are rebuilt from sb (not kept live across the gates)
            asm volatile("" : "+r"(sb));
#pragma unroll
            for (int i = 0; i < (1 << R); ++i) {
                uint32_t a = sb;
#pragma unroll
                for (int k = 0; k < R; ++k) if ((i >> k) & 1) a ^= sw[k];
                tile[a] = v[i];
            }
        }
        __syncthreads();
    }
}

// Physical bits of a tile pass (ascending) and the tile's gather tables:
// element i of the tile is amplitude base | lut_lo[i & 127] | lut_hi[i >> 7].
template <int K, int TH>
__device__ __forceinline__ void tile_tables(const BrickPass &ps, int N, int *pos, uint32_t *lut_lo, uint32_t *lut_hi) {
    if (threadIdx.x == 0) {
        int k = 0;
        for (int b = 0; b < N; ++b) if (ps.smask & (1u << b)) pos[k++] = b;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 128; i += TH) {
        uint32_t o = 0;
        for (int k = 0; k < 7; ++k) o |= ((i >> k) & 1u) << pos[k];
        lut_lo[i] = o;
    }
    for (int i = threadIdx.x; i < (1 << (K - 7)); i += TH) {
        uint32_t o = 0;
        for (int k = 0; k < K - 7; ++k) o |= ((i >> k) & 1u) << pos[7 + k];
        lut_hi[i] = o;
    }
    __syncthreads();
}

// base amplitude index of tile t: t's bits spread over the bits outside the tile
__device__ __forceinline__ uint32_t tile_base(uint32_t t, uint32_t smask, int N) {
    uint32_t base = 0;
    for (int b = 0; b < N; ++b)
        if (!(smask & (1u << b))) { base |= (t & 1u) << b; t >>= 1; }
    return base;
}

// One light-cone pass of one side over all pairs: blockIdx.x = tile, blockIdx.y = pair.
// The tile (2^K amplitudes, a contiguous cyclic arc of segment bits) is loaded
// into shared memory, the pass's gate maps and schedule are staged next to it,
// and the gates are applied window by window with 2^R amplitudes per thread
// in registers; one barrier per window.
template <typename C, int K, int R, int TH>
__global__ void __launch_bounds__(TH, (sizeof(C) == 8 && K <= 13 && TH <= 256) ? 2 : 1)   // FP32 tiles <= 2^13: 2 CTAs/SM
    brick_pass_kernel(BrickDev d, int side, BrickPass ps,
                                                        const BrickGate *__restrict__ gates,
                                                        const RegPass *__restrict__ rps,
                                                        const RegGate *__restrict__ rgs,
                                                        const C *__restrict__ maps, C *__restrict__ states) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *tile = (C *)smem_raw;
    C *smaps = tile + (1u << K);
    constexpr int MW = MapSlot<C>::width;
    __shared__ uint32_t lut_lo[128], lut_hi[1 << (K - 7)];
    __shared__ int pos[32];
    __shared__ RegPass srp[kMaxRegPasses];
    __shared__ RegGate srg[256];
    __shared__ uint8_t shi[1 << (K - 4)];
    const int N = d.N;
    const uint32_t S = 1u << N;
    swizzle_table<K, TH>(ps, shi);
    tile_tables<K, TH>(ps, N, pos, lut_lo, lut_hi);   // (its barriers publish shi too)
    const uint32_t base = tile_base(blockIdx.x, ps.smask, N);
    // the tile: all 2^K element copies in flight at once ...
    static_assert((1 << K) % TH == 0, "tile size must be a multiple of the block size");
    C *st = states + ((size_t)blockIdx.y * 2 + side) * S + base;
#pragma unroll
    for (int j = 0; j < (1 << K) / TH; ++j) {
        const uint32_t i = threadIdx.x + (uint32_t)j * TH;
        cp_async<sizeof(C)>(&tile[swzt(shi, i)], &st[lut_lo[i & 127] | lut_hi[i >> 7]]);
    }
    // ... while the register schedule and the pass's gate maps are staged
    for (int i = threadIdx.x; i < ps.n_rp; i += TH) srp[i] = rps[ps.rp_off + i];
    for (int i = threadIdx.x; i < ps.n_gates; i += TH) srg[i] = rgs[ps.rg_off + i];
    const C *mp = maps + (size_t)blockIdx.y * maps_per_pair(d) * 16;
    for (int i = threadIdx.x; i < ps.n_gates * 16; i += TH) {
        const BrickGate gg = gates[ps.gate_off + i / 16];
        stage_entry<C>(smaps + (i / 16) * MW, i % 16, mp[(size_t)map_index(d, side, gg.layer, gg.j) * 16 + (i % 16)]);
    }
    cp_async_wait_all();
    __syncthreads();
    tile_register_passes<C, K, R, TH>(tile, smaps, srp, srg, ps.n_rp, ps.rg_off, shi);
    for (uint32_t i = threadIdx.x; i < (1u << K); i += TH) st[lut_lo[i & 127] | lut_hi[i >> 7]] = tile[swzt(shi, i)];
}

// Persistent, double-buffered form of brick_pass_kernel: each CTA walks the
// (pair, tile) items of the pass with a stride of gridDim.x; while it applies
// the gates of one item, the cp.async copies of the next item's tile and raw
// gate maps fill the other buffer, so tile loads overlap compute.  Shared
// memory: two 2^K tiles, two raw map sets, one staged map set.
template <typename C, int K, int R, int TH>
__global__ void __launch_bounds__(TH) brick_pass_db_kernel(BrickDev d, int side, BrickPass ps, int npairs,
                                                           const BrickGate *__restrict__ gates,
                                                           const RegPass *__restrict__ rps,
                                                           const RegGate *__restrict__ rgs,
                                                           const C *__restrict__ maps, C *__restrict__ states) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int MW = MapSlot<C>::width;
    const int G = ps.n_gates;
    C *tiles = (C *)smem_raw;                      // [2][2^K]
    C *raw = tiles + 2 * (1u << K);                // [2][G*16]
    C *smaps = raw + 2 * G * 16;                   // [G*MW]
    __shared__ uint32_t lut_lo[128], lut_hi[1 << (K - 7)];
    __shared__ int pos[32];
    __shared__ RegPass srp[kMaxRegPasses];
    __shared__ RegGate srg[256];
    __shared__ int mslot[256];                     // map index of each gate of the pass
    __shared__ uint8_t shi[1 << (K - 4)];
    const int N = d.N;
    const uint32_t S = 1u << N;
    swizzle_table<K, TH>(ps, shi);
    tile_tables<K, TH>(ps, N, pos, lut_lo, lut_hi);
    for (int i = threadIdx.x; i < ps.n_rp; i += TH) srp[i] = rps[ps.rp_off + i];
    for (int i = threadIdx.x; i < G; i += TH) {
        srg[i] = rgs[ps.rg_off + i];
        const BrickGate gg = gates[ps.gate_off + i];
        mslot[i] = map_index(d, side, gg.layer, gg.j);
    }
    __syncthreads();
    const uint32_t ntiles = 1u << (N - K);
    const uint32_t items = (uint32_t)npairs * ntiles;
    static_assert((1 << K) % TH == 0, "tile size must be a multiple of the block size");
    auto issue = [&](uint32_t it, int buf) {
        const uint32_t pair = it / ntiles, t = it - pair * ntiles;
        const C *st = states + ((size_t)pair * 2 + side) * S + tile_base(t, ps.smask, N);
        C *dst = tiles + (size_t)buf * (1u << K);
#pragma unroll
        for (int j = 0; j < (1 << K) / TH; ++j) {
            const uint32_t i = threadIdx.x + (uint32_t)j * TH;
            cp_async<sizeof(C)>(&dst[swzt(shi, i)], &st[lut_lo[i & 127] | lut_hi[i >> 7]]);
        }
        const C *mp = maps + (size_t)pair * maps_per_pair(d) * 16;
        C *rdst = raw + (size_t)buf * G * 16;
        for (int i = threadIdx.x; i < G * 16; i += TH)
            cp_async<sizeof(C)>(&rdst[i], &mp[(size_t)mslot[i / 16] * 16 + (i % 16)]);
    };
    uint32_t it = blockIdx.x;
    if (it < items) issue(it, 0);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    for (int k = 0; it < items; it += gridDim.x, ++k) {
        const int buf = k & 1;
        const uint32_t nxt = it + gridDim.x;
        if (nxt < items) issue(nxt, buf ^ 1);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");   // this item's copies are in
        __syncthreads();
        const C *rsrc = raw + (size_t)buf * G * 16;
        for (int i = threadIdx.x; i < G * 16; i += TH) stage_entry<C>(smaps + (i / 16) * MW, i % 16, rsrc[i]);
        __syncthreads();
        C *tile = tiles + (size_t)buf * (1u << K);
        tile_register_passes<C, K, R, TH>(tile, smaps, srp, srg, ps.n_rp, ps.rg_off, shi);
        const uint32_t pair = it / ntiles, t = it - pair * ntiles;
        C *st = states + ((size_t)pair * 2 + side) * S + tile_base(t, ps.smask, N);
        for (uint32_t i = threadIdx.x; i < (1u << K); i += TH) st[lut_lo[i & 127] | lut_hi[i >> 7]] = tile[swzt(shi, i)];
        __syncthreads();   // the tile and raw maps of this buffer are free for item k + 2
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

template <typename C>
__global__ void __launch_bounds__(1024) brick_dot_kernel(BrickDev d, const PairInfo *__restrict__ pairs,
                                                         const C *__restrict__ states, double err_scale,
                                                         double *__restrict__ tr, double *__restrict__ kappa,
                                                         double *__restrict__ err) {
    __shared__ double red[4][32];
    const uint32_t S = 1u << d.N;
    const C *L = states + (size_t)blockIdx.x * 2 * S, *R = L + S;
    // in FP32, the products of a thread's runs of 8 elements are summed first and
    // each run's sum is added in FP64 (8 times fewer FP64 operations)
    MeetAcc<C> acc;
    for (uint32_t w0 = threadIdx.x; w0 < S; w0 += 8 * blockDim.x) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint32_t w = w0 + (uint32_t)k * blockDim.x;
            if (w < S) acc.add(L[w], R[w]);
        }
        acc.flush();
    }
    double sr = acc.sr, si = acc.si, sa = (double)acc.sa, s2 = (double)acc.s2;
    sr = wsum(sr); si = wsum(si); sa = wsum(sa); s2 = wsum(s2);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { red[0][wid] = sr; red[1][wid] = si; red[2][wid] = sa; red[3][wid] = s2; }
    __syncthreads();
    if (threadIdx.x == 0) {
        sr = si = sa = s2 = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { sr += red[0][w]; si += red[1][w]; sa += red[2][w]; s2 += red[3][w]; }
        const PairInfo pi = pairs[blockIdx.x];
        tr[2 * pi.out] = sr;
        tr[2 * pi.out + 1] = si;
        double mag = sqrt(sr * sr + si * si);
        if (kappa) kappa[pi.out] = mag > 0 ? sa / mag : __longlong_as_double(0x7ff0000000000000LL);
        if (err) err[pi.out] = err_scale * (sqrt(s2) + mag);
    }
}

template <typename C, int K, int R, int TH>
cudaError_t run_passes(const BrickDev &d, const BrickPass *hpasses, const BrickDevPlan &dp, int npairs,
                       const C *maps, C *states, cudaStream_t st) {
    int maxg = 0;
    for (int i = 0; i < d.n_passes[0] + d.n_passes[1]; ++i) maxg = hpasses[i].n_gates > maxg ? hpasses[i].n_gates : maxg;
    const size_t smem = (((size_t)1 << K) + (size_t)maxg * MapSlot<C>::width) * sizeof(C);
    cudaError_t e = cudaFuncSetAttribute(brick_pass_kernel<C, K, R, TH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    for (int side = 0; side < 2; ++side)
        for (int p = 0; p < d.n_passes[side]; ++p) {
            dim3 grid(1u << (d.N - K), npairs);
            brick_pass_kernel<C, K, R, TH><<<grid, TH, smem, st>>>(d, side, hpasses[d.pass_off[side] + p], dp.gates,
                                                                    dp.rpasses, dp.rgates, maps, states);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    return cudaSuccess;
}

template <typename C, int K, int R, int TH>
cudaError_t run_passes_db(const BrickDev &d, const BrickPass *hpasses, const BrickDevPlan &dp, int npairs,
                          const C *maps, C *states, cudaStream_t st) {
    int maxg = 0;
    for (int i = 0; i < d.n_passes[0] + d.n_passes[1]; ++i) maxg = hpasses[i].n_gates > maxg ? hpasses[i].n_gates : maxg;
    const size_t smem = ((size_t)2 * ((size_t)1 << K) + (size_t)maxg * (2 * 16 + MapSlot<C>::width)) * sizeof(C);
    auto kern = brick_pass_db_kernel<C, K, R, TH>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TH, smem)) != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const uint64_t items = (uint64_t)npairs << (d.N - K);
    const unsigned grid = (unsigned)std::min<uint64_t>(items, (uint64_t)sms * per_sm);
    for (int side = 0; side < 2; ++side)
        for (int p = 0; p < d.n_passes[side]; ++p) {
            kern<<<grid, TH, smem, st>>>(d, side, hpasses[d.pass_off[side] + p], npairs, dp.gates, dp.rpasses,
                                          dp.rgates, maps, states);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    return cudaSuccess;
}

}  // namespace

size_t brick_smem_bytes(const BrickDev &d, bool fp32, bool *both) {
    const size_t el = fp32 ? sizeof(float2) : sizeof(double2);
    const size_t S = (size_t)1 << d.N;
    *both = 2 * S * el <= 96 * 1024;
    return (*both ? 2 : 1) * S * el;
}

cudaError_t launch_brick(const BrickDev &d, const BrickPass *hpasses, const BrickDevPlan &dp,
                         const PairInfo *pairs, int npairs, const double2 *raw, void *maps, void *states,
                         bool fp32, double err_scale, double *tr, double *kappa, double *err, cudaStream_t st,
                         int *launches) {
    if (npairs <= 0) return cudaSuccess;
    const int nm = maps_per_pair(d);
    dim3 gm((nm + 127) / 128, npairs);
    if (fp32) brick_maps_kernel<float2><<<gm, 128, 0, st>>>(d, pairs, raw, (float2 *)maps);
    else brick_maps_kernel<double2><<<gm, 128, 0, st>>>(d, pairs, raw, (double2 *)maps);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int nl = 1;
    if (d.tile_bits == 0) {
        bool both = false;
        const size_t smem = brick_smem_bytes(d, fp32, &both);
        const uint32_t quads = (1u << d.N) >> 2;
        int gt = quads <= 32 ? 32 : (quads >= 512 ? 512 : (int)((quads + 31) / 32 * 32));
        int gpc = gt == 32 ? 8 : 1;
        // one pair per CTA: its maps go to shared memory too, when they fit
        const size_t map_bytes = (size_t)nm * 16 * (fp32 ? sizeof(float2) : sizeof(double2));
        const int stage = gt > 32 && smem + map_bytes <= (size_t)200 * 1024 ? 1 : 0;
        size_t smem_cta = (smem + (stage ? map_bytes : 0)) * gpc;
        int grid = (npairs + gpc - 1) / gpc;
        if (fp32) {
            if ((e = cudaFuncSetAttribute(brick_smem_kernel<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cta)) != cudaSuccess) return e;
            brick_smem_kernel<float2><<<grid, gt * gpc, smem_cta, st>>>(d, pairs, npairs, (const float2 *)maps,
                                                                         (float2 *)states, gt, both, stage, err_scale, tr, kappa, err);
        } else {
            if ((e = cudaFuncSetAttribute(brick_smem_kernel<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cta)) != cudaSuccess) return e;
            brick_smem_kernel<double2><<<grid, gt * gpc, smem_cta, st>>>(d, pairs, npairs, (const double2 *)maps,
                                                                          (double2 *)states, gt, both, stage, err_scale, tr, kappa, err);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        nl += 1;
    } else {
        const size_t total = (size_t)npairs * 2 * ((size_t)1 << d.N);
        int dev = 0, sms = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        int ib = (int)std::min<size_t>((total + 255) / 256, (size_t)sms * 8);   // 8 resident 256-thread CTAs per SM
        if (fp32) brick_init_kernel<float2><<<ib, 256, 0, st>>>(d, npairs, (float2 *)states);
        else brick_init_kernel<double2><<<ib, 256, 0, st>>>(d, npairs, (double2 *)states);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        const int key = dp.persist * 10000 + d.tile_bits * 100 + dp.win_bits * 10 +
                        (dp.threads == 256 ? 1 : (dp.threads == 128 ? 2 : 0));
        if (fp32 && (dp.persist == 3 || dp.persist == 4)) {
            float2 *sp = (float2 *)states;
            float *wm = (float *)(sp + (size_t)npairs * 2 * ((size_t)1 << d.N));
            e = run_passes_tc(d, hpasses, dp, npairs, (const float2 *)maps, sp, wm, dp.err_flag, st);
        } else if (fp32) {
            const float2 *mp = (const float2 *)maps;
            float2 *sp = (float2 *)states;
            switch (key) {
                case 1241: e = run_passes<float2, 12, 4, 256>(d, hpasses, dp, npairs, mp, sp, st); break;
                case 1252: e = run_passes<float2, 12, 5, 128>(d, hpasses, dp, npairs, mp, sp, st); break;
                case 1440: e = run_passes<float2, 14, 4, 512>(d, hpasses, dp, npairs, mp, sp, st); break;
                case 1451: e = run_passes<float2, 14, 5, 256>(d, hpasses, dp, npairs, mp, sp, st); break;
                case 1340: e = run_passes<float2, 13, 4, 512>(d, hpasses, dp, npairs, mp, sp, st); break;
                case 1341: e = run_passes<float2, 13, 4, 256>(d, hpasses, dp, npairs, mp, sp, st); break;
                case 1351: e = run_passes<float2, 13, 5, 256>(d, hpasses, dp, npairs, mp, sp, st); break;
                case 11340: e = run_passes_db<float2, 13, 4, 512>(d, hpasses, dp, npairs, mp, sp, st); break;
                case 11351: e = run_passes_db<float2, 13, 5, 256>(d, hpasses, dp, npairs, mp, sp, st); break;
                default: return cudaErrorInvalidValue;
            }
        } else {
            const double2 *mp = (const double2 *)maps;
            double2 *sp = (double2 *)states;
            switch (key) {
                case 1330: e = run_passes<double2, 13, 3, 512>(d, hpasses, dp, npairs, mp, sp, st); break;
                case 1341: e = run_passes<double2, 13, 4, 256>(d, hpasses, dp, npairs, mp, sp, st); break;
                default: return cudaErrorInvalidValue;
            }
        }
        if (e != cudaSuccess) return e;
        if (fp32) brick_dot_kernel<float2><<<npairs, 1024, 0, st>>>(d, pairs, (const float2 *)states, err_scale, tr, kappa, err);
        else brick_dot_kernel<double2><<<npairs, 1024, 0, st>>>(d, pairs, (const double2 *)states, err_scale, tr, kappa, err);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        nl += 1 + (dp.persist >= 2 ? 2 : 1) * (d.n_passes[0] + d.n_passes[1]) + 1;
    }
    if (launches) *launches = nl;
    return cudaSuccess;
}

}  // namespace fpk
