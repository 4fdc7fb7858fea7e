// kernels_sweep.cu -- generic boundary sweep (any ensemble) and FP64 meet.
//
// One CTA contracts one pair at a time, taking pairs from a ticket queue
// ordered by estimated cost (largest first).  The left boundary is swept
// from qubit 0 to the cut and the right boundary from qubit n-1 to the cut,
// each op multiplying the boundary by a <=16-entry factor table and summing
// the variables that factor is last for.  The two boundaries then meet in an
// FP64 dot product that also gives the cancellation ratio
// kappa = sum_j |L_j R_j| / |sum_j L_j R_j|.  Boundaries live in a per-CTA
// global workspace (3 buffers: left result + right ping-pong); at the sizes
// this path serves they stay resident in L2.
#include <cuda_runtime.h>

#include "kernels.h"

namespace fpk {
namespace {

template <typename C> struct Real;
template <> struct Real<double2> { using T = double; };
template <> struct Real<float2> { using T = float; };

template <typename C>
__device__ __forceinline__ C cfma(C a, C b, C acc) {   // acc + a*b
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
    return acc;
}

__device__ __forceinline__ uint32_t remove_bit(uint32_t x, int p) {
    uint32_t lo = x & ((1u << p) - 1u);
    return lo | ((x >> (p + 1)) << p);
}
__device__ __forceinline__ uint32_t insert_bit(uint32_t x, int p, uint32_t v) {
    uint32_t lo = x & ((1u << p) - 1u);
    return lo | (v << p) | ((x >> p) << (p + 1));
}

template <typename C>
__device__ void run_op(const DevOp &op, const C *__restrict__ T, const C *__restrict__ in, C *__restrict__ out) {
    const uint32_t nout = 1u << op.b_out;
    if (op.inplace2) {
        const int p0 = op.cons_pos[0], p1 = op.cons_pos[1];
        C t[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) t[e] = T[e];
        for (uint32_t q = threadIdx.x; q < (nout >> 2); q += blockDim.x) {
            uint32_t i00 = insert_bit(insert_bit(q, p0, 0), p1, 0);
            uint32_t idx[4] = {i00, i00 | (1u << p0), i00 | (1u << p1), i00 | (1u << p0) | (1u << p1)};
            C a[4];
#pragma unroll
            for (int b = 0; b < 4; ++b) a[b] = in[idx[b]];
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                C acc;
                acc.x = 0; acc.y = 0;
#pragma unroll
                for (int b = 0; b < 4; ++b) acc = cfma(t[b | (o << 2)], a[b], acc);
                out[idx[o]] = acc;
            }
        }
        return;
    }
    const int nc = op.nc, nk = op.nk, nn = op.nn;
    for (uint32_t o = threadIdx.x; o < nout; o += blockDim.x) {
        uint32_t nv = 0, kv = 0, r = o;
        for (int z = 0; z < nn; ++z) nv |= ((o >> op.new_pos[z]) & 1u) << z;
        for (int z = 0; z < nk; ++z) kv |= ((o >> op.keep_pos[z]) & 1u) << z;
        for (int z = nn - 1; z >= 0; --z) r = remove_bit(r, op.new_pos[z]);
        const uint32_t tb = (kv << nc) | (nv << (nc + nk));
        C acc;
        acc.x = 0; acc.y = 0;
        for (uint32_t cv = 0; cv < (1u << nc); ++cv) {
            uint32_t idx = r;
            for (int z = 0; z < nc; ++z) idx = insert_bit(idx, op.cons_pos[z], (cv >> z) & 1u);
            acc = cfma(T[cv | tb], in[idx], acc);
        }
        out[o] = acc;
    }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
    return v;
}

template <typename C>
__global__ void __launch_bounds__(256) sweep_generic(const PairInfo *__restrict__ pairs,
        const int32_t *__restrict__ order, int count, const DevPlan *__restrict__ plans,
        const DevOp *__restrict__ ops, const C *__restrict__ tables, C *__restrict__ ws,
        size_t ws_elems, int *ticket, double err_unit, double *__restrict__ tr, double *__restrict__ kappa,
        double *__restrict__ err) {
    __shared__ int item;
    __shared__ double red[4][8];
    C *buf0 = ws + (size_t)blockIdx.x * 3 * ws_elems;
    C *bufs[3] = {buf0, buf0 + ws_elems, buf0 + 2 * ws_elems};
    for (;;) {
        if (threadIdx.x == 0) item = atomicAdd(ticket, 1);
        __syncthreads();
        const int it = item;
        __syncthreads();
        if (it >= count) break;
        const int pidx = order[it];
        const PairInfo pi = pairs[pidx];
        const DevPlan &pl = plans[pi.plan];
        const C *tb = tables + pi.table_off * 16;
        const DevOp *po = ops + pl.ops_off;
        C one;
        one.x = 1; one.y = 0;
        if (threadIdx.x == 0) bufs[0][0] = one;
        __syncthreads();
        int cur = 0;
        for (int k = 0; k < pl.n_left; ++k) {
            run_op<C>(po[k], tb + (size_t)k * 16, bufs[cur], bufs[cur ^ 1]);
            cur ^= 1;
            __syncthreads();
        }
        C *L = bufs[cur];
        C *rb[2] = {bufs[2], bufs[cur ^ 1]};
        if (threadIdx.x == 0) rb[0][0] = one;
        __syncthreads();
        int rc = 0;
        for (int k = 0; k < pl.n_right; ++k) {
            run_op<C>(po[pl.n_left + k], tb + (size_t)(pl.n_left + k) * 16, rb[rc], rb[rc ^ 1]);
            rc ^= 1;
            __syncthreads();
        }
        const C *R = rb[rc];
        // FP64 meet
        double sr = 0, si = 0, sa = 0, s2 = 0;
        const uint32_t nf = 1u << pl.bits_final;
        for (uint32_t o = threadIdx.x; o < nf; o += blockDim.x) {
            uint32_t ri = 0;
            for (int k = 0; k < pl.bits_final; ++k) ri |= ((o >> k) & 1u) << pl.dot_perm[k];
            double lx = (double)L[o].x, ly = (double)L[o].y, rx = (double)R[ri].x, ry = (double)R[ri].y;
            double px = lx * rx - ly * ry, py = lx * ry + ly * rx;
            double q = px * px + py * py;
            sr += px; si += py; sa += sqrt(q); s2 += q;
        }
        sr = warp_sum(sr); si = warp_sum(si); sa = warp_sum(sa); s2 = warp_sum(s2);
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        if (lane == 0) { red[0][wid] = sr; red[1][wid] = si; red[2][wid] = sa; red[3][wid] = s2; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0, b = 0, c = 0, q2 = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += red[0][w]; b += red[1][w]; c += red[2][w]; q2 += red[3][w]; }
            if (err) err[pi.out] = err_unit * pl.sqrt_ops * pl.prefactor * (sqrt(q2) + sqrt(a * a + b * b));
            tr[2 * pi.out] = pl.prefactor * a;
            tr[2 * pi.out + 1] = pl.prefactor * b;
            double mag = sqrt(a * a + b * b);
            if (kappa) kappa[pi.out] = mag > 0 ? c / mag : __longlong_as_double(0x7ff0000000000000LL);
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_sweep_generic(const PairInfo *pairs, const int32_t *order, int count,
                                 const DevPlan *plans, const DevOp *ops, const void *tables,
                                 bool fp32, void *workspace, size_t ws_elems_per_cta, int ctas,
                                 int *ticket, double err_unit, double *tr, double *kappa, double *err,
                                 cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(ticket, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    if (fp32)
        sweep_generic<float2><<<ctas, 256, 0, st>>>(pairs, order, count, plans, ops, (const float2 *)tables,
                                                    (float2 *)workspace, ws_elems_per_cta, ticket, err_unit, tr, kappa, err);
    else
        sweep_generic<double2><<<ctas, 256, 0, st>>>(pairs, order, count, plans, ops, (const double2 *)tables,
                                                     (double2 *)workspace, ws_elems_per_cta, ticket, err_unit, tr, kappa, err);
    return cudaGetLastError();
}

}  // namespace fpk
