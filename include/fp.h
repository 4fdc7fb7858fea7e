/*
 * fp.h -- C ABI of the GB300 (sm_103a) frame-potential library.
 *
 * The library estimates the frame potential of a random-circuit ensemble,
 *     F^(k) = E_{U,V} |Tr(U^dagger V)|^{2k}        (paper: Sec. "Frame potential", Eq. for F^(k))
 * by Monte Carlo over sampled circuit pairs,
 *     F^(k) ~= (1/N) sum_pairs |Tr(U^dagger V)|^{2k} (paper: Sec. "Algorithm description")
 * where every sample is an exact contraction of the closed trace network of
 * U^dagger V along the qubit (space) direction (paper: Sec. "Algorithm
 * description", Fig. 3a).  Ensembles (paper: Fig. 2, Sec. "Results"):
 *   FP_PARALLEL  brickwork of Haar U(4) gates on an open chain, layer t acting
 *                on bonds (b, b+1) with b = (t-1) mod 2, b+2, ...;
 *   FP_LOCAL     T Haar U(4) gates, each on a uniformly random bond;
 *   FP_HEA       hardware-efficient ansatz: per layer RY(theta) RZ(phi) on every
 *                qubit (theta, phi uniform in [0, 2 pi)), then CZ on every bond;
 *   FP_HEA_PAULI the paper's hardware-efficient ansatz (Fig. 2c, Sec.
 *                "Hardware-efficient ansatze as approximate k-designs"): a
 *                fixed wall of RY(pi/4) on every qubit, then per layer a
 *                rotation R_P(theta) = exp(-i theta P/2) on every qubit with
 *                the Pauli axis P uniform in {X, Y, Z} and theta uniform in
 *                [0, 2 pi), followed by two walls of CNOTs (control b, target
 *                b+1): first on the even bonds b = 0, 2, ..., then on the odd
 *                bonds b = 1, 3, ...  FP_FLAG_HEA_CZ puts CZ in place of CNOT
 *                (the controlled-phase variant the paper compares against).
 *
 * Conventions: qubit 0 is the most significant bit of a basis index; a
 * 2-qubit gate on bond (b, b+1) has matrix index (a_b a_{b+1}) with a_b the
 * more significant bit; U = G_T ... G_1 (G_1 acts first); RY(t) =
 * exp(-i t Y/2), RZ(p) = exp(-i p Z/2), RZ acts first within a layer.
 *
 * Random numbers.  Every draw is one block of Philox4x64-10 (Salmon et al.,
 * SC'11) with key {seed, 0} and counter {c0, c1, pair, stream}, giving words
 * x0..x3:
 *   Haar gate g of circuit w (0 = U, 1 = V): c0 = 0..7, c1 = g, stream = w;
 *     entry k = 4r+c of the 4x4 complex Gaussian uses block k/2, words
 *     (x0,x1) for even k, (x2,x3) for odd k: u1 = ((xa>>11)+1) 2^-53,
 *     u2 = (xb>>11) 2^-53, Z_k = sqrt(-2 ln u1) e^{2 pi i u2} / sqrt 2; the gate
 *     is Q of Z = QR with R's diagonal made positive real (Haar measure).
 *   Local bond of gate g of circuit w: c0 = 0, c1 = g, stream = 2+w,
 *     bond = ((x0 >> 32)(n-1)) >> 32.
 *   Per-pair depth (l or L) or gate count T: c0 = c1 = 0, stream = 4,
 *     choice = ((x0 >> 32) * n_choices) >> 32.
 *   HEA angles of circuit w, layer t (0-based), qubit q: c0 = t, c1 = q,
 *     stream = w: theta = 2 pi (x0>>11) 2^-53, phi = 2 pi (x1>>11) 2^-53.
 *   FP_HEA_PAULI rotation of circuit w, layer t, qubit q: the same block;
 *     theta = 2 pi (x0>>11) 2^-53, axis = ((x1 >> 32) * 3) >> 32 (0: X,
 *     1: Y, 2: Z).
 *   FP_FLAG_DIAGONAL_GATES replaces each Haar gate g of circuit w by
 *     diag(e^{i 2 pi u_j}), u_j = (x_j >> 11) 2^-53 from c0 = 0, c1 = g, stream = w.
 * Pair p of an ensemble is therefore fully determined by (seed, p).
 *
 * Memory and ownership.  The library owns ensembles and their device
 * workspaces.  The caller owns every output array.  An output pointer may be
 * host memory (pageable or pinned) or device memory (e.g. a PyTorch tensor's
 * data_ptr()); the library detects which.  All device work is ordered on the
 * stream given at creation (NULL = the legacy default stream).  Every call
 * returns after its results are in the caller's arrays.
 *
 * Environment.  FP_AUTOTUNE_CACHE names a file in which the brickwork
 * autotuner keeps its choices; FP_SWEEP_CLUSTER (1, 4, 8 or 16) fixes the
 * number of CTAs that share one pair on the generic sweep (default: by
 * boundary size); FP_SPIRAL_WIN (0, 4 or 5) fixes the register-window width
 * of the spiral sweep of FP_HEA_PAULI (0: one map per pass; default: by
 * state size) and FP_SPIRAL_SPLIT (0, 1 or 2) the least number of cluster
 * bits its state is split over (default 0: as the state size needs); both are
 * read when an ensemble first contracts a depth.
 *
 * Errors.  Calls return an fp_status; nothing is thrown across the ABI.
 * fp_last_error() gives a thread-local message for the last failing call on
 * the calling thread.  A failed call leaves caller arrays unspecified and the
 * ensemble usable.
 */
#ifndef FP_H
#define FP_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FP_OK = 0,
    FP_ERR_ARG = -1,          /* invalid argument */
    FP_ERR_CUDA = -2,         /* CUDA runtime error (message in fp_last_error) */
    FP_ERR_OOM = -3,          /* device or host allocation failed */
    FP_ERR_TIMEOUT = -4,      /* a bounded device wait ran out */
    FP_ERR_INFEASIBLE = -5,   /* a pair's boundary exceeds FP_MAX_STATE_BITS */
    FP_ERR_CANCELLED = -6     /* fp_cancel stopped a Monte Carlo run between batches */
} fp_status;

typedef enum { FP_PARALLEL = 0, FP_LOCAL = 1, FP_HEA = 2, FP_HEA_PAULI = 3 } fp_kind;

/* Arithmetic of the contraction.  The final boundary dot product, the
 * |Tr|^{2k} powers and all Monte Carlo moments are FP64 in every mode. */
typedef enum {
    FP_PREC_FP64 = 0,         /* boundary tensors and gate maps in FP64 */
    FP_PREC_FP32 = 1,         /* boundary tensors and gate maps in FP32, FP64 meet
                                 and reduction; the brickwork autotuner takes the
                                 faster of the FFMA tile passes and the TF32 x 3
                                 tensor-core passes per depth; a pair whose
                                 estimated error exceeds fp32_tol, or whose
                                 cancellation ratio exceeds kappa_max, is
                                 recontracted in FP64 */
    FP_PREC_FP32_RAW = 2,     /* FP32 as above without the FP64 recontraction */
    FP_PREC_TF32X3 = 3        /* FP_PREC_FP32 with the brickwork tile passes on the
                                 tensor cores wherever they apply (12-bit tiles,
                                 boundaries of 2^14 amplitudes and more: brickwork
                                 l >= 8, HEA L >= 8): window matrices applied by
                                 three TF32 products with FP32 accumulation; the
                                 FP32 path elsewhere */
} fp_prec;

enum {
    FP_FLAG_SELF_PAIR = 1,        /* V := U for every pair (Tr = 2^n exactly) */
    FP_FLAG_DIAGONAL_GATES = 2,   /* FP_PARALLEL/FP_LOCAL with random diagonal gates */
    FP_FLAG_GENERIC_ONLY = 4,     /* never use the specialised brickwork kernels */
    FP_FLAG_TIMING = 8,           /* record CUDA-event time of every launch (fp_kernel_stats_get);
                                     also disables CUDA-graph replay */
    FP_FLAG_NO_GRAPHS = 16,       /* launch every kernel directly (no CUDA-graph replay) */
    FP_FLAG_SKIP_INFEASIBLE = 32, /* pairs whose boundary exceeds FP_MAX_STATE_BITS are left
                                     uncontracted instead of failing the call: NaN results,
                                     group -1, left out of the moments, counted in
                                     fp_run_stats.infeasible */
    FP_FLAG_HEA_CZ = 64           /* FP_HEA_PAULI with CZ walls instead of CNOT walls */
};

/* Kernel classes of fp_kernel_stats. */
enum {
    FP_K_SAMPLE = 0,      /* gate sampler */
    FP_K_MERGE = 1,       /* gate merging */
    FP_K_TABLES = 2,      /* factor tables */
    FP_K_SWEEP = 3,       /* generic boundary sweep + meet */
    FP_K_BRICK = 4,       /* brickwork boundary sweep + meet */
    FP_K_MOMENTS = 5,     /* Monte Carlo moments */
    FP_K_BOOTSTRAP = 6,   /* bootstrap resampling */
    FP_K_SPIRAL = 7,      /* spiral sweep of FP_HEA_PAULI (maps + sweep) */
    FP_K_CLASSES = 8
};

#define FP_MAX_STATE_BITS 24      /* largest boundary: 2^24 amplitudes per side */
#define FP_MAX_KMAX 8

typedef struct {
    int32_t kind;             /* fp_kind */
    int32_t n;                /* qubits, 2 <= n <= 64 */
    int32_t depth_min;        /* l (FP_PARALLEL) or L (FP_HEA, FP_HEA_PAULI), >= 1 */
    int32_t depth_max;        /* >= depth_min; each pair draws its depth uniformly */
    int32_t T_min, T_max, T_step;   /* FP_LOCAL: T drawn uniformly from
                                       {T_min, T_min+T_step, ..., <= T_max} */
    int32_t flags;            /* FP_FLAG_* */
    uint64_t seed;
    double kappa_max;         /* FP_PREC_FP32: recontract in FP64 when the cancellation
                                 ratio exceeds this; <= 0: no cap */
    double fp32_tol;          /* FP_PREC_FP32: recontract in FP64 when the estimated
                                 absolute error of Tr exceeds this; <= 0: 1e-4 */
    uint64_t workspace_bytes; /* device workspace cap; 0: library default, min(32 GB, free/2) */
    int32_t q;                /* local dimension: 0 or 2 = qubits; 3 or 4 = qudits (FP_PARALLEL
                                 only: Haar U(q^2) gates, gate g of circuit w drawn as the
                                 q^2 x q^2 Gaussian whose entry k takes Philox block c0 = k/2,
                                 c1 = g, stream = w, words as for qubits; depth l >= 2;
                                 boundary q^{2(l-1)} amplitudes, at most 2^FP_MAX_STATE_BITS) */
    int32_t reserved;
} fp_ensemble_desc;

/* Error estimate of one trace (the `err` output of fp_trace_batch): with
 * t_j = L_j R_j the terms of the final boundary dot product, u the unit
 * roundoff of the boundary arithmetic (2^-24 or 2^-53) and G the number of
 * gate maps applied along one chain half,
 *     err = FP_ERR_SAFETY * u * sqrt(G) * (sqrt(sum_j |t_j|^2) + |Tr|),
 * a random-walk model of the accumulated rounding (term-wise part plus the
 * coherent part from rounded gate maps), calibrated so that it bounds the
 * measured FP32-vs-FP64 difference with margin. */
#define FP_ERR_SAFETY 16.0

typedef struct fp_ensemble fp_ensemble;

/* Per-run statistics of fp_frame_potential. */
typedef struct {
    uint64_t pairs;           /* pairs contracted */
    uint64_t fp64_recontracted;   /* pairs moved to FP64 by the kappa policy */
    double gpu_seconds;       /* device time of the contraction batches */
    double max_kappa;         /* largest cancellation ratio seen */
    int32_t n_groups;         /* groups reported (depth or T values) */
    int32_t reached_target;   /* 1 if every group met target_rel_stderr on F^(2) */
    uint64_t infeasible;      /* pairs left out under FP_FLAG_SKIP_INFEASIBLE */
} fp_run_stats;

/* Per-kernel-class counters, accumulated while FP_FLAG_TIMING is set. */
typedef struct {
    double ms[FP_K_CLASSES];          /* device milliseconds (CUDA events on the ensemble's stream) */
    uint64_t launches[FP_K_CLASSES];  /* kernel launches */
    double work[FP_K_CLASSES];        /* algorithmic work: complex multiply-adds for the sweep
                                         classes, pairs for the others */
    uint64_t pairs;                   /* pairs contracted */
    uint64_t graph_replays;           /* sub-batches run by CUDA-graph replay (counted always) */
    double mma_flops;                 /* flops issued to the tensor cores by the brickwork
                                         tensor-core tile passes (2 per multiply-add; three
                                         TF32 products per operand pair) */
} fp_kernel_stats;

/* Create an ensemble.  `cuda_stream` is a cudaStream_t (NULL: default stream).
 * Validates the descriptor (FP_ERR_ARG) and allocates nothing on the device
 * until the first contraction. */
fp_status fp_ensemble_create(const fp_ensemble_desc *desc, void *cuda_stream, fp_ensemble **out);

/* Release an ensemble and all its device memory.  NULL is allowed. */
void fp_ensemble_destroy(fp_ensemble *ens);

/* Number of groups F is reported for (depth or T values) and the group value
 * of each: values[g] = depth_min + g or T_min + g*T_step.  `values` may be NULL. */
fp_status fp_groups(const fp_ensemble *ens, int32_t *n_groups, int32_t *values);

/* Group index of pairs first..first+count-1 (host array of count int32). */
fp_status fp_pair_groups(const fp_ensemble *ens, uint64_t first, uint64_t count, int32_t *group);

/* Sampled gates of circuit `which` (0 = U, 1 = V) of one pair, as they enter
 * the contraction (the circuits of the ensembles of Fig. 2, Sec. "Results";
 * the paper draws U and V independently from the ensemble, Sec. "Frame
 * potential"); an input feed for independent checks of the traces: per gate a record {int32 kind, int32 qubit, 32 doubles =
 * 16 complex entries (re,im)}, kind 0 = 4x4 on (q,q+1), 1 = 2x2 on q in the
 * first 4 entries, 2 = diagonal 2-qubit (4 entries).  FP_HEA_PAULI with CNOT
 * walls lists each CNOT as H on the target, CZ, H on the target (the form
 * the contraction uses: CZ leaves both wires uncut).  *bytes is in/out:
 * capacity of host_buf on entry, bytes needed on return.  host_buf may be
 * NULL to query the size. */
fp_status fp_export_gates(fp_ensemble *ens, uint64_t pair, int32_t which, void *host_buf,
                          size_t *bytes);

/* Contract pairs first..first+count-1: every pair's Tr(U^dagger V), the closed
 * trace network of U^dagger V contracted exactly along the qubit chain (Sec.
 * "Algorithm description", Fig. 3a; the paper's samples |Tr(U^dagger V)|^{2k}
 * of the frame potential, Sec. "Frame potential").
 *   tr     [2*count] doubles: Tr(U^dagger V) as (re, im) per pair;
 *   kappa  [count] doubles or NULL: cancellation ratio sum_j |L_j R_j| / |sum_j L_j R_j|
 *          of the final boundary dot product (1 when no cancellation);
 *   err    [count] doubles or NULL: estimated absolute rounding error of Tr
 *          in the arithmetic that produced it (see FP_ERR_SAFETY);
 *   group  [count] int32 or NULL: group index of each pair.
 * Host or device pointers.  FP_ERR_INFEASIBLE if a pair's boundary exceeds
 * FP_MAX_STATE_BITS (nothing is written then), unless FP_FLAG_SKIP_INFEASIBLE
 * is set: then such pairs get tr = kappa = err = NaN and group = -1. */
fp_status fp_trace_batch(fp_ensemble *ens, uint64_t first, uint64_t count, int32_t prec,
                         double *tr, double *kappa, double *err, int32_t *group);

/* FP64 moments of |Tr|^{2k} per group: the sums behind the Monte Carlo
 * estimate F^(k) ~= (1/N) sum |Tr|^{2k} and its standard error (Sec.
 * "Algorithm description"; the paper's error bars are standard errors):
 * moments[g*(2*k_max+1) + 0] = N_g, [.. + k] = sum |Tr|^{2k}, [.. + k_max + k] =
 * sum |Tr|^{4k}, for k = 1..k_max.  tr/group as produced by fp_trace_batch,
 * on the device; moments on host or device.  Deterministic (fixed tree). */
fp_status fp_reduce_moments(fp_ensemble *ens, const double *tr, const int32_t *group,
                            uint64_t count, int32_t k_max, double *moments);

/* Bootstrap distribution of F^(k) per group (paper: Supplementary,
 * "Bootstrapping for uncertainty quantification"; the paper takes 300
 * resamples and reports medians and the spread).  Each group's stored traces
 * are resampled with replacement, as many draws as the group has pairs, and
 * F^(k) = mean |Tr|^{2k} is evaluated on every resample.
 *   tr      [2*count] doubles (re, im), group [count] int32 (entries outside
 *           [0, n_groups) are ignored): host or device, e.g. the outputs of
 *           fp_trace_batch;
 *   F_boot  [n_groups * k_max * n_resamples] doubles, host or device:
 *           F_boot[(g*k_max + k-1)*n_resamples + b]; NaN for an empty group.
 * Draw i of resample b in group g takes position ((x >> 32) N_g) >> 32 of the
 * group's pairs in increasing index order, x = word i mod 4 of the Philox
 * block with counter {b, i / 4, g, 5} and key {seed, 0}.  Deterministic.
 * count < 2^32; 1 <= n_resamples <= 2^31 - 1. */
fp_status fp_bootstrap(fp_ensemble *ens, const double *tr, const int32_t *group, uint64_t count, int32_t k_max,
                       int32_t n_resamples, uint64_t seed, double *F_boot);

/* log10 of epsilon_max = d^k sqrt(F - k!) with d = q^n (paper: Sec. "Frame
 * potential", Eq. epsilonmax): the ensemble is at least an
 * epsilon_max-approximate k-design.  *log10_eps = NaN when F <= k!. */
fp_status fp_epsilon_max(double F, int32_t k, int32_t n, int32_t q, double *log10_eps);

/* Layers for an eps-approximate k-design from a depth sweep (paper: Sec.
 * "Frame potential", Eqs. exponential and layers; fitting region from the
 * supplementary "Choice of curve fitting region", dev_max = 5 there): depths
 * with 0 < (F - k!)/k! < dev_max are kept, log(F - k!) = a + s l is fitted by
 * least squares, then A = exp(a/2), C = -2/s and
 *     l_eps = C (k n ln q + ln A + ln(1/eps)).
 * Host arrays depths[n_depths], F[n_depths].  Outputs are NaN (status FP_OK)
 * when fewer than two depths qualify or the slope is not negative. */
fp_status fp_design_layers(int32_t n_depths, const double *depths, const double *F, int32_t k, int32_t n,
                           int32_t q, double eps, double dev_max, double *l_eps, double *A, double *C);

/* Exact ensemble frame potential F^(k), k = 2 or 3, of brickwork circuits
 * (FP_PARALLEL ensembles of one depth l), with no sampling: every Haar U(4)
 * gate of the cyclic U^dagger V circuit averaged over the Haar measure
 * becomes a sum over pairings sigma, tau in S_k weighted by the Weingarten
 * function of U(4), and consecutive gates on a qubit wire meet with weight
 * 2^{#cycles(sigma^-1 tau)} -- the statistical-mechanics model behind the
 * paper's Eq. theory_eq (Sec. "Frame potential").  The sum over all pairings
 * runs as a transfer-matrix sweep over the bonds on the device, in FP64, with
 * a state of (k!)^{2(l-1)} entries (k = 3, l = 7: 17.4 GB) allocated for the
 * call and freed before it returns.  A variance-free reference for the Monte
 * Carlo estimates of F^(2) and F^(3).
 *   n >= 2; l in [2, 12] for k = 2, [2, 7] for k = 3 (FP_ERR_ARG otherwise);
 *   F  host double: the exact F^(k) of the ensemble.
 * Ordered on cuda_stream; waits for the result.  FP_ERR_OOM when the state
 * does not fit in free device memory. */
fp_status fp_exact_brickwork_fk(int32_t n, int32_t l, int32_t k, void *cuda_stream, double *F);

/* The same for brickwork circuits of qudits of local dimension q (2 <= q <= 64):
 * Haar U(q^2) gates, Weingarten function of U(q^2), links q^{#cycles} (the paper
 * treats general q in Sec. "Frame potential"; its Eq. theory_eq bound has q).
 * fp_exact_brickwork_fk is q = 2. */
fp_status fp_exact_brickwork_fkq(int32_t n, int32_t l, int32_t k, int32_t q, void *cuda_stream, double *F);

/* Monte Carlo frame potential.  Contracts pairs first, first+1, ... in batches
 * until every group's relative standard error of F^(2) (or of F^(1) when
 * k_max = 1) is <= target_rel_stderr, or max_pairs pairs are done.  With a
 * target the batches start at 4096 pairs and double (up to 2^20); with
 * target_rel_stderr <= 0 all max_pairs pairs run, in batches of 2^20.
 *   F, stderr  [n_groups * k_max] doubles (host), F[g*k_max + k-1] = F^(k) of group g,
 *              stderr = s/sqrt(N) with s the N-1 sample deviation;
 *   stats      may be NULL. */
fp_status fp_frame_potential(fp_ensemble *ens, uint64_t first, uint64_t max_pairs, int32_t k_max,
                             double target_rel_stderr, int32_t prec, double *F, double *stderr_,
                             fp_run_stats *stats);

/* Checkpoint of a Monte Carlo run (fp_frame_potential_resume).  The paper's
 * adaptive sample sizes (Supplementary Methods, "Determination of sample
 * sizes") add samples to stored ones until the error bars are small enough;
 * this state is what such a run needs to continue later or elsewhere.
 * Before the first call: next_pair = the run's first pair, next_batch = 0,
 * sums zero.  Every completed batch updates it, so after an error or a
 * cancellation it holds the last completed batch. */
typedef struct {
    uint64_t next_pair;       /* first pair of the next batch */
    uint64_t next_batch;      /* size of the next batch (0: the run has not started) */
    uint64_t pairs_done;      /* pairs taken so far (contracted + infeasible) */
    int32_t k_max, n_groups;  /* set by the first call; a resume must use the same k_max */
    double *sums;             /* caller-owned host array of 2 * n_groups * (2*k_max+1) doubles:
                                 the FP64 moment sums per group (layout of fp_reduce_moments),
                                 then their Neumaier compensations */
    fp_run_stats stats;       /* accumulated over all calls of the run */
} fp_checkpoint;

/* The Monte Carlo driver of fp_frame_potential, resumable: continues the run
 * in *ck with batches of the same schedule (so a run split over several calls
 * gives bit-identical F and stderr to one uninterrupted call) until the target
 * is met, pairs_done reaches max_pairs, or max_batches batches (0: no limit)
 * have run in this call.  F and stderr_ as in fp_frame_potential, from all
 * batches so far.  FP_ERR_CANCELLED (checkpoint intact) when fp_cancel was
 * called; the cancellation is consumed by that return. */
fp_status fp_frame_potential_resume(fp_ensemble *ens, fp_checkpoint *ck, uint64_t max_pairs, uint64_t max_batches,
                                    int32_t k_max, double target_rel_stderr, int32_t prec, double *F,
                                    double *stderr_);

/* Ask a running (or the next) Monte Carlo run of this ensemble to stop before
 * its next batch (fp_frame_potential / fp_frame_potential_resume return
 * FP_ERR_CANCELLED).  Safe to call from another host thread. */
fp_status fp_cancel(fp_ensemble *ens);

/* Fault injection for tests of the error paths (host side; no device fault):
 * the next `count` device allocations of ensemble workspaces fail as if the
 * device were out of memory, so the call returns FP_ERR_OOM and leaves the
 * ensemble usable.  0 clears it. */
fp_status fp_inject_alloc_failures(int32_t count);

/* Time limit of every bounded device wait (mbarrier waits of the tcgen05
 * kernels), in nanoseconds of the device's global timer; 0 restores the
 * default of 1 s.  A wait that runs out makes the kernel stop issuing work,
 * drain what it issued (within a fixed 1 s), release its tensor memory and
 * raise a device flag that the call reports as FP_ERR_TIMEOUT.  Applies to
 * launches made after the call (captured CUDA graphs keep the limit they
 * were captured with). */
fp_status fp_set_wait_limit_ns(uint64_t ns);

/* The brickwork sweep variant chosen for one depth (FP_PARALLEL and FP_HEA
 * ensembles, depth l >= 2): out[0] = tile bits of a tile pass (99: the whole
 * boundary in one CTA's shared memory), out[1] = register-window bits,
 * out[2] = threads per CTA, out[3] = pass kind (0: FP32/FP64 FMA tile passes,
 * 1: persistent double-buffered FMA passes, 3: tensor-core passes with the
 * tile's operand in shared memory, 4: tensor-core passes with the tile's
 * operand in tensor memory, persistent over the tiles).  The autotuner
 * chooses it the first time the ensemble contracts that depth at that
 * precision (FP_PREC_FP32 and FP_PREC_FP32_RAW share one choice,
 * FP_PREC_TF32X3 has its own); before that the call returns FP_ERR_ARG.  `out`
 * is a host array of 4 int32. */
fp_status fp_brick_variant(const fp_ensemble *ens, int32_t depth, int32_t precision, int32_t *out);

/* Copy the ensemble's kernel counters into *out; reset them if `reset`. */
fp_status fp_kernel_stats_get(fp_ensemble *ens, fp_kernel_stats *out, int32_t reset);

/* Learned control variate for F^(2) (the paper has none; the estimate is the
 * paper's F^(2), Sec. "Frame potential").  For a single-depth HEA ensemble
 * (depth_min == depth_max == L) an MLP -- input 12 features per (layer,
 * qubit): cos and sin of both circuits' theta and phi and of their
 * differences; three hidden layers of `hidden` units with GELU; one output --
 * is trained (Adam, mean squared error) on the normalised log |Tr|^2 of
 * n_train exactly contracted pairs; g = beta exp(2 x prediction) predicts
 * |Tr|^4, beta = Cov(f, g) / Var(g) on the training pairs.  Then
 *     F^(2) = mean over m_surrogate pairs of g + mean over n_correct pairs of (|Tr|^4 - g),
 * the three pair ranges consecutive from `first` and disjoint, so the
 * estimate is unbiased for any g; stderr_ = sqrt(Var g / M + Var(f - g) / N).
 * The plain estimate on the correction pairs is returned beside it.  Exact
 * contractions use FP_PREC_FP32 (with the FP64 recontraction policy). */
typedef struct {
    int32_t hidden;           /* hidden width (<= 1024; 0: 256) */
    int32_t epochs;           /* training epochs (0: 20) */
    int32_t batch;            /* minibatch size (0: 512) */
    int32_t reserved;
    double lr;                /* Adam learning rate (0: 1e-3) */
    uint64_t first;           /* first pair of the training range */
    uint64_t n_train;         /* exactly contracted training pairs (>= batch) */
    uint64_t n_correct;       /* exactly contracted correction pairs (>= 2) */
    uint64_t m_surrogate;     /* surrogate-only pairs (>= 2) */
    double *g_correct;        /* optional [n_correct] output (host or device, NULL: none):
                                 g on the correction pairs, in units of |Tr|^4 */
    double *f_correct;        /* optional [n_correct] output: f = |Tr|^4 on the correction pairs */
    double *g_surrogate;      /* optional [m_surrogate] output: g on the surrogate pairs */
} fp_cv_config;

typedef struct {
    double F2, stderr_;               /* control-variate estimate and its standard error */
    double F2_plain, stderr_plain;    /* plain estimate on the correction pairs */
    double var_f, var_f_minus_g, var_g;   /* per-pair variances */
    double target_scale;              /* the fitted coefficient beta of g */
    double train_loss;                /* last epoch's mean squared error (scaled units) */
    double gpu_seconds_exact;         /* device time of the exact contractions */
    double gpu_seconds_train;         /* device time of feature generation and training */
    double gpu_seconds_surrogate;     /* device time of correction and surrogate evaluation */
} fp_cv_result;

fp_status fp_cv_frame_potential(fp_ensemble *ens, const fp_cv_config *cfg, fp_cv_result *res);

/* Allocation-free brickwork traces (the paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory when they need
 * traces -- plugins inside a framework whose memory pool already holds the
 * device memory, where a cudaMalloc can fail or fragment that pool; loops that
 * must not block in an allocator).  It contracts pairs first..first+count-1 of
 * the brickwork ensemble (n qubits, every pair of depth l, Philox key `seed`)
 * on the brickwork shared-memory path, with all intermediate data in one
 * scratch array of FP_STATIC_SCRATCH_BYTES compiled into the library (held by
 * every GPU that loads it until the process exits).  It calls no cudaMalloc
 * or cudaFree and no allocating library routine.
 *   l         2..7 (boundaries of at most 12 bits);
 *   prec      FP_PREC_FP64 or FP_PREC_FP32_RAW (no FP64 recontraction);
 *   tr        [2*count] doubles, kappa [count] doubles or NULL: device (or
 *             managed) memory of the current device, owned by the caller;
 *   cuda_stream  a stream of the current device (NULL: the default stream);
 *             the launches are ordered on it and the call does not wait for
 *             them (results are in tr/kappa once the stream reaches that point).
 * A count whose scratch would exceed FP_STATIC_SCRATCH_BYTES returns
 * FP_ERR_ARG with the largest count that fits (fp_last_error); so do outputs
 * or a stream of another device.  The first call on a device looks up the
 * scratch array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  All calls share
 * the one array: calls that overlap on the GPU (unordered streams) race;
 * nothing in it needs to start at zero (every kernel writes what it later
 * reads). */
#define FP_STATIC_SCRATCH_BYTES (32u << 20)
fp_status fp_trace_brick_static(int32_t n, int32_t l, uint64_t seed, uint64_t first, uint64_t count,
                                int32_t prec, double *tr, double *kappa, void *cuda_stream);

/* The dense layer of the control-variate MLP on the tensor cores (tcgen05,
 * BF16 operands, FP32 accumulation); the training and surrogate passes of
 * fp_cv_frame_potential run on the same kernel.  The paper has no control
 * variate: this is the MLP that predicts |Tr(U^dagger V)|^4 (Sec. "Frame
 * potential" defines F^(2) = E|Tr|^4).
 *   C[M x N] = A[M x K] . Bt[N x K]^T + bias,  then by `mode`:
 *     0: C as is;  1: GELU(C) (exact erf form), the pre-activation written to
 *     Z if Z is non-null;  2: C * GELU'(Z) elementwise (Z is read: the
 *     backward pass through a GELU layer).
 *   A       [M x K] BF16 row-major, leading dimension lda (>= K, multiple of 8);
 *   Bt      [N x K] BF16 row-major (the right factor transposed), ldb likewise;
 *   bias    [N] FP32 or NULL;  Z [M x N] FP32 row-major (leading dimension N);
 *   C       [M x N] FP32 row-major, C_bf16 [M x N] BF16 row-major and
 *   Ct_bf16 [N x M] BF16 (C transposed): any non-empty subset, others NULL.
 * All pointers are device memory owned by the caller, 16-byte aligned (C_bf16
 * 8-byte).  Needs N % 16 == 0 and K % 8 == 0 (FP_ERR_ARG otherwise); M may be
 * anything >= 0.  Ordered on cuda_stream; the call waits for the result and
 * returns FP_ERR_TIMEOUT if a bounded device wait ran out. */
fp_status fp_gemm_bf16(int32_t M, int32_t N, int32_t K, const void *A, int32_t lda, const void *Bt, int32_t ldb,
                       const float *bias, int32_t mode, float *Z, float *C, void *C_bf16, void *Ct_bf16,
                       void *cuda_stream);

/* Measured arithmetic peaks of the current device (the paper has no
 * counterpart: these are the denominators of the roofline fractions that the
 * benchmark reports for the contraction kernels).  One microbenchmark keeps one
 * pipe busy with independent work:
 *   FP_PEAK_FFMA     scalar FP32 fused multiply-adds (fma.rn.f32),
 *   FP_PEAK_FFMA2    packed FP32 pairs (fma.rn.f32x2, the contraction's arithmetic),
 *   FP_PEAK_DFMA     FP64 fused multiply-adds,
 *   FP_PEAK_TC_TF32  tcgen05.mma kind::tf32, 128x256 outputs, K = 8 per MMA,
 *   FP_PEAK_TC_BF16  tcgen05.mma kind::f16 with BF16 operands, K = 16 per MMA;
 * the tensor kernels keep both operands in shared memory and the accumulator
 * in tensor memory (no global traffic).  iters scales the work (0: default,
 * about 1-3 ms).  One untimed launch precedes the timed one.  Output (host):
 *   out[0] TFLOP/s (2 flops per multiply-add), out[1] kernel milliseconds,
 *   out[2] SM clock in MHz during the run (clock64 over the global timer, CTA 0),
 *   out[3] flops per clock per SM, out[4] SMs.
 * Ordered on cuda_stream; waits for the result.  FP_ERR_TIMEOUT if the
 * tensor-core completion wait (bounded at 2 s) ran out. */
enum { FP_PEAK_FFMA = 0, FP_PEAK_FFMA2 = 1, FP_PEAK_DFMA = 2, FP_PEAK_TC_TF32 = 3, FP_PEAK_TC_BF16 = 4 };
fp_status fp_measure_peak(int32_t which, int32_t iters, void *cuda_stream, double *out);

/* Thread-local message of the last failing call ("" if none). */
const char *fp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
