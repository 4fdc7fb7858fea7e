// kernels_sweep.cu -- generic boundary sweep (any ensemble) and FP64 meet.
//
// One thread-block cluster of CS CTAs (CS = 1 for small boundaries, up to 16
// for boundaries of 2^18+ amplitudes) contracts one pair at a time, taking
// pairs from a ticket queue ordered by estimated cost (largest first); the
// CTAs of a cluster split every op's outputs and meet at a cluster barrier
// between ops.  The left boundary is swept
// from qubit 0 to the cut and the right boundary from qubit n-1 to the cut,
// each op multiplying the boundary by a <=16-entry factor table and summing
// the variables that factor is last for.  The two boundaries then meet in an
// FP64 dot product that also gives the cancellation ratio
// kappa = sum_j |L_j R_j| / |sum_j L_j R_j|.  Boundaries live in a per-CTA
// global workspace (3 buffers: left result + right ping-pong); at the sizes
// this path serves they stay resident in L2.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cstdlib>

#include "kernels.h"

namespace cg = cooperative_groups;

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

// one op over the outputs assigned to this CTA: worker w of W = CS * blockDim.x
template <typename C>
__device__ void run_op(const DevOp &op, const C *__restrict__ T, const C *__restrict__ in, C *__restrict__ out,
                       uint32_t w, uint32_t W) {
    const uint32_t nout = 1u << op.b_out;
    if (op.inplace2) {
        const int p0 = op.cons_pos[0], p1 = op.cons_pos[1];
        C t[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) t[e] = T[e];
        for (uint32_t q = w; q < (nout >> 2); q += W) {
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
    for (uint32_t o = w; o < nout; o += W) {
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

// CTA-or-cluster-wide barrier (global and shared memory ordered at cluster scope)
template <int CS>
__device__ __forceinline__ void csync() {
    if constexpr (CS == 1) __syncthreads();
    else cg::this_cluster().sync();
}

template <typename C, int CS>
__global__ void __launch_bounds__(256) sweep_generic(const PairInfo *__restrict__ pairs,
        const int32_t *__restrict__ order, int count, const DevPlan *__restrict__ plans,
        const DevOp *__restrict__ ops, const C *__restrict__ tables, C *__restrict__ ws,
        size_t ws_elems, int *ticket, double err_unit, double *__restrict__ tr, double *__restrict__ kappa,
        double *__restrict__ err) {
    __shared__ int item;
    __shared__ double red[4][8];
    __shared__ double part[4];   // this CTA's share of the meet
    const uint32_t rank = CS == 1 ? 0u : cg::this_cluster().block_rank();
    const uint32_t slot = blockIdx.x / CS;   // cluster index: one workspace per cluster
    const uint32_t w0 = rank * blockDim.x + threadIdx.x, W = CS * blockDim.x;
    C *buf0 = ws + (size_t)slot * 3 * ws_elems;
    C *bufs[3] = {buf0, buf0 + ws_elems, buf0 + 2 * ws_elems};
    for (;;) {
        if (rank == 0 && threadIdx.x == 0) item = atomicAdd(ticket, 1);
        csync<CS>();
        int it;
        if constexpr (CS == 1) it = item;
        else it = *cg::this_cluster().map_shared_rank(&item, 0);
        csync<CS>();   // everyone has read the ticket before rank 0 takes the next
        if (it >= count) break;
        const int pidx = order[it];
        const PairInfo pi = pairs[pidx];
        const DevPlan &pl = plans[pi.plan];
        const C *tb = tables + pi.table_off * 16;
        const DevOp *po = ops + pl.ops_off;
        C one;
        one.x = 1; one.y = 0;
        if (w0 == 0) bufs[0][0] = one;
        csync<CS>();
        int cur = 0;
        for (int k = 0; k < pl.n_left; ++k) {
            run_op<C>(po[k], tb + (size_t)k * 16, bufs[cur], bufs[cur ^ 1], w0, W);
            cur ^= 1;
            csync<CS>();
        }
        C *L = bufs[cur];
        C *rb[2] = {bufs[2], bufs[cur ^ 1]};
        if (w0 == 0) rb[0][0] = one;
        csync<CS>();
        int rc = 0;
        for (int k = 0; k < pl.n_right; ++k) {
            run_op<C>(po[pl.n_left + k], tb + (size_t)(pl.n_left + k) * 16, rb[rc], rb[rc ^ 1], w0, W);
            rc ^= 1;
            csync<CS>();
        }
        const C *R = rb[rc];
        // FP64 meet: per-CTA partial sums, combined by rank 0 (through
        // distributed shared memory when CS > 1)
        double sr = 0, si = 0, sa = 0, s2 = 0;
        const uint32_t nf = 1u << pl.bits_final;
        for (uint32_t o = w0; o < nf; o += W) {
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
            part[0] = a; part[1] = b; part[2] = c; part[3] = q2;
        }
        csync<CS>();
        if (rank == 0 && threadIdx.x == 0) {
            double a = 0, b = 0, c = 0, q2 = 0;
            for (uint32_t r = 0; r < (uint32_t)CS; ++r) {
                const double *pp;
                if constexpr (CS == 1) pp = part;
                else pp = cg::this_cluster().map_shared_rank(part, r);
                a += pp[0]; b += pp[1]; c += pp[2]; q2 += pp[3];
            }
            if (err) err[pi.out] = err_unit * pl.sqrt_ops * pl.prefactor * (sqrt(q2) + sqrt(a * a + b * b));
            tr[2 * pi.out] = pl.prefactor * a;
            tr[2 * pi.out + 1] = pl.prefactor * b;
            double mag = sqrt(a * a + b * b);
            if (kappa) kappa[pi.out] = mag > 0 ? c / mag : __longlong_as_double(0x7ff0000000000000LL);
        }
        csync<CS>();   // rank 0 has read every CTA's partials before they are overwritten
    }
}

template <typename C, int CS>
cudaError_t launch_cs(int ctas, cudaStream_t st, const PairInfo *pairs, const int32_t *order, int count,
                      const DevPlan *plans, const DevOp *ops, const void *tables, void *workspace, size_t ws_elems,
                      int *ticket, double err_unit, double *tr, double *kappa, double *err) {
    auto kern = sweep_generic<C, CS>;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)ctas);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    int na = 0;
    if (CS > 1) {
        if (CS > 8) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            if (e != cudaSuccess) return e;
        }
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = CS;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        na = 1;
    }
    cfg.attrs = attr;
    cfg.numAttrs = na;
    return cudaLaunchKernelEx(&cfg, kern, pairs, order, count, plans, ops, (const C *)tables, (C *)workspace,
                              ws_elems, ticket, err_unit, tr, kappa, err);
}

template <typename C>
cudaError_t launch_c(int cs, int ctas, cudaStream_t st, const PairInfo *pairs, const int32_t *order, int count,
                     const DevPlan *plans, const DevOp *ops, const void *tables, void *workspace, size_t ws_elems,
                     int *ticket, double err_unit, double *tr, double *kappa, double *err) {
    switch (cs) {
        case 1: return launch_cs<C, 1>(ctas, st, pairs, order, count, plans, ops, tables, workspace, ws_elems, ticket, err_unit, tr, kappa, err);
        case 4: return launch_cs<C, 4>(ctas, st, pairs, order, count, plans, ops, tables, workspace, ws_elems, ticket, err_unit, tr, kappa, err);
        case 8: return launch_cs<C, 8>(ctas, st, pairs, order, count, plans, ops, tables, workspace, ws_elems, ticket, err_unit, tr, kappa, err);
        case 16: return launch_cs<C, 16>(ctas, st, pairs, order, count, plans, ops, tables, workspace, ws_elems, ticket, err_unit, tr, kappa, err);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

// Boundaries up to 2^13 amplitudes (64 KB in FP32) stay with one CTA; up to
// 2^17 a cluster of 4 CTAs; larger ones a cluster of 16.  The environment
// variable FP_SWEEP_CLUSTER (1, 4, 8 or 16) overrides the choice.
int sweep_cluster_size(int bits) {
    if (const char *e = getenv("FP_SWEEP_CLUSTER")) {
        const int v = atoi(e);
        if (v == 1 || v == 4 || v == 8 || v == 16) return v;
    }
    return bits <= 13 ? 1 : (bits <= 17 ? 4 : 16);
}

namespace {
template <typename C, int CS>
int max_clusters_t() {
    auto k = sweep_generic<C, CS>;
    if (CS > 8 && cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)CS);
    cfg.blockDim = dim3(256);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}
}  // namespace

int sweep_max_clusters(int cs, bool fp32) {
    switch (cs) {
        case 4: return fp32 ? max_clusters_t<float2, 4>() : max_clusters_t<double2, 4>();
        case 8: return fp32 ? max_clusters_t<float2, 8>() : max_clusters_t<double2, 8>();
        case 16: return fp32 ? max_clusters_t<float2, 16>() : max_clusters_t<double2, 16>();
        default: return 0;
    }
}

cudaError_t launch_sweep_generic(const PairInfo *pairs, const int32_t *order, int count,
                                 const DevPlan *plans, const DevOp *ops, const void *tables,
                                 bool fp32, void *workspace, size_t ws_elems_per_cta, int ctas, int cs,
                                 int *ticket, double err_unit, double *tr, double *kappa, double *err,
                                 cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    if (cs < 1 || ctas % cs) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(ticket, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    if (fp32)
        return launch_c<float2>(cs, ctas, st, pairs, order, count, plans, ops, tables, workspace, ws_elems_per_cta,
                                ticket, err_unit, tr, kappa, err);
    return launch_c<double2>(cs, ctas, st, pairs, order, count, plans, ops, tables, workspace, ws_elems_per_cta,
                             ticket, err_unit, tr, kappa, err);
}

}  // namespace fpk
