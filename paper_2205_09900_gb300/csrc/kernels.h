// kernels.h -- launch wrappers of the sm_103a kernels (host-callable).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "brick.h"
#include "fp_internal.h"

namespace fpk {

struct SampleParams {
    uint64_t seed;
    int32_t n;
    int32_t raw_kind;     // RawKind
    int32_t self_pair;
};

// Sampler: raw gates of U and V for every pair of the batch (FP64).
// kernels one launch_sample issues (Haar gates: Gaussian draws, then the QR)
int sample_launch_count(int raw_kind);
cudaError_t launch_sample(const SampleParams &sp, const PairInfo *pairs, int npairs, int max_raw,
                          double2 *raw, cudaStream_t st);
// Merged gates: ordered products of raw gates (FP64).
cudaError_t launch_merge(const PairInfo *pairs, int npairs, int max_merged, const DevPlan *plans,
                         const MergeItem *items, const MergeRef *refs, const double2 *raw,
                         double2 *merged, cudaStream_t st);
// Op tables (16 entries per op) in FP64 or FP32.
cudaError_t launch_tables(const PairInfo *pairs, int npairs, int max_ops, const DevPlan *plans,
                          const DevRecipe *recipes, const double2 *merged, void *tables, bool fp32,
                          cudaStream_t st);
// Generic boundary sweep + meet: one cluster of `cs` CTAs (1, 4, 8 or 16) per
// pair at a time, persistent over a ticket queue; `ctas` is a multiple of cs
// and the workspace holds ctas/cs slots of 3 x ws_elems amplitudes.  Writes
// tr[2*i], kappa[i] for pair i of `order`.
cudaError_t launch_sweep_generic(const PairInfo *pairs, const int32_t *order, int count,
                                 const DevPlan *plans, const DevOp *ops, const void *tables,
                                 bool fp32, void *workspace, size_t ws_elems_per_cta, int ctas, int cs,
                                 int *ticket, double err_unit, double *tr, double *kappa, double *err,
                                 cudaStream_t st);
// Cluster size for a batch whose largest boundary has `bits` bits, and how many
// such clusters can be resident (0 if clusters of that size cannot launch).
int sweep_cluster_size(int bits);
int sweep_max_clusters(int cs, bool fp32);
// FP64 moments per group (deterministic).
cudaError_t launch_moments(const double *tr, const int32_t *group, uint64_t count, int k_max,
                           int n_groups, double *partials, int nblocks, double *out,
                           cudaStream_t st);
int moments_blocks(uint64_t count);
// Bootstrap of F^(k): members lists the pairs of group g at [goff[g], goff[g+1]);
// xs (n_members doubles) is scratch; out[(g*k_max + k-1)*B + b].
cudaError_t launch_bootstrap(const double *tr, const uint32_t *members, uint64_t n_members, const uint64_t *goff,
                             int n_groups, int k_max, int B, uint64_t seed, double *xs, double *out,
                             cudaStream_t st);
// Brickwork fast path: maps, then either the shared-memory sweep (tile_bits == 0)
// or init + light-cone passes + dot.  `states` holds npairs x 2 x 2^N
// amplitudes (tiled) or npairs x 2^N (shared-memory path, left boundaries).
cudaError_t launch_brick(const BrickDev &d, const BrickPass *hpasses, const BrickDevPlan &dp,
                         const PairInfo *pairs, int npairs, const double2 *raw, void *maps, void *states,
                         bool fp32, double err_scale, double *tr, double *kappa, double *err, cudaStream_t st,
                         int *launches);
size_t brick_smem_bytes(const BrickDev &d, bool fp32, bool *both);
// Tensor-core tile passes (kernels_brick_tc.cu): whether a plan qualifies
// (kTcTile-bit tiles, kMaxWin-bit windows, boundary of more than one tile
// pair), the window-matrix workspace per pair (placed after the boundaries in
// `states`), and the launches of both sides.
bool tc_plan_ok(const BrickDev &d, const BrickPass *hpasses, const RegPass *rps);
size_t tc_wmat_bytes_per_pair(const BrickDev &d, const BrickPass *hpasses);
cudaError_t run_passes_tc(const BrickDev &d, const BrickPass *hpasses, const BrickDevPlan &dp, int npairs,
                          const float2 *maps, float2 *states, float *wm, int *err, cudaStream_t st);
// Spiral sweep (the paper's HEA): maps from merged 1-qubit operators
// (spiral_map_elems(fp32) elements of C per map), then the sweep.  The
// configuration of a state of 2^bits amplitudes: R = 0 applies one map per
// pass (shared memory when it fits, else `scratch`, scratch_elems per pair);
// R = 4 or 5 runs windows of R bits (spiral_windows with `split`; cluster bits
// h[0], h[1]) over shared memory of one CTA (split = 0) or a 2^split-CTA
// cluster (split = 1, 2).
constexpr size_t kSpiralSmemMax = 128 * 1024;
struct SpiralConfig {
    int R = 0;
    int split = 0;
    size_t scratch_elems = 0;
};
SpiralConfig spiral_config(int bits, bool fp32, int min_split = 0);   // split >= min_split (<= 2)
size_t spiral_map_elems(bool fp32);
cudaError_t launch_spiral(const PairInfo *pairs, int npairs, const SpiralMap *sm, int nmaps, int bits, int first_bit,
                          const SpiralConfig &cfg, const SpiralWin *wins, int nwins, const uint8_t *ij, const int *h,
                          const double2 *merged, void *maps, void *scratch, bool fp32, double err_scale, double *tr,
                          double *kappa, double *err, cudaStream_t st);
// Qudit brickwork (kernels_qudit.cu): sampler, maps and sweep of pairs
// pairs[0..npairs) of one depth (BrickDev of the qubit plan with N = 2(l-1)
// q-ary digits); `ws` holds qudit_workspace_per_pair bytes per pair; results
// at slot pairs[i].out of tr/kappa/err.
size_t qudit_workspace_per_pair(int q, const BrickDev &d, int n_raw, bool fp32);
cudaError_t launch_qudit(int q, const BrickDev &d, uint64_t seed, const PairInfo *pairs, int npairs, int n_raw,
                         int self_pair, bool fp32, void *ws, double err_scale, double *tr, double *kappa, double *err,
                         cudaStream_t st);
// Time limit of one bounded device wait (nanoseconds of the global timer):
// fp_set_wait_limit_ns, default 1 s.
uint64_t wait_limit_ns();
// Set the thread-local message returned by fp_last_error().
void set_last_error(const char *msg);
// Internal access for the control-variate driver (cv.cu).
fp_status api_fail(fp_status s, const char *msg);
fp_ensemble_desc ens_desc(const fp_ensemble *E);
cudaStream_t ens_stream(const fp_ensemble *E);
// FP32-policy traces of pairs [first, first+count) into the ensemble's device
// array (*tr_dev, 2*count doubles), device milliseconds into *gpu_ms.
fp_status cv_trace(fp_ensemble *E, uint64_t first, uint64_t count, double **tr_dev, float *gpu_ms);

// BF16 tensor-core GEMM (tc_gemm.cu): C[M x N] = A[M x K] . Bt[N x K]^T (+ bias),
// FP32 accumulation, epilogue mode 0 identity / 1 GELU (pre-activation to Z if
// set) / 2 times GELU'(Z); outputs FP32 row-major (Cf), BF16 row-major (Cb),
// BF16 transposed (Cbt[col * ldct + row]); any subset.  err (device int, may be
// null) is set to 1 if a bounded wait ran out.
struct TcGemm {
    int M, N, K;
    const __nv_bfloat16 *A;
    int lda;
    const __nv_bfloat16 *Bt;
    int ldb;
    const float *bias;
    int mode;
    float *Z;
    int ldz;
    float *Cf;
    int ldcf;
    __nv_bfloat16 *Cb;
    int ldcb;
    __nv_bfloat16 *Cbt;
    int ldct;
    int *err;
    uint64_t wait_ns;   // bounded-wait limit (set at launch from wait_limit_ns())
};
const char *tc_gemm_check(const TcGemm &g);   // nullptr if the arguments are valid
cudaError_t launch_tc_gemm(const TcGemm &g, cudaStream_t st);
size_t tc_gemm_smem_bytes();

}  // namespace fpk
