// api.cu -- the C ABI declared in include/fp.h.
//
// Host side of the hot path: per-pair depth draws, plan cache (one plan per
// depth for fixed-topology ensembles, one per pair for local circuits),
// batching under a device-memory budget, the launches (sampler -> merge ->
// tables -> sweep+meet), the FP32->FP64 recontraction policy and the
// Monte Carlo driver.  Every step of the path runs in the kernels; the host
// only plans, marshals and orders work.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <numeric>
#include <tuple>
#include <string>
#include <thread>
#include <vector>

#include "fp.h"
#include "kernels.h"
#include "brick.h"
#include "planner.h"

using namespace fpk;

namespace {

thread_local std::string g_err;

fp_status fail(fp_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

#define CK(call)                                                                         \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(e_ == cudaErrorMemoryAllocation ? FP_ERR_OOM : FP_ERR_CUDA,      \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

// Host-side fault injection (fp_inject_alloc_failures): the next N device
// allocations of ensemble buffers fail as if the device were out of memory.
std::atomic<int> g_alloc_failures{0};
// Time limit of every bounded device wait (fp_set_wait_limit_ns).
std::atomic<uint64_t> g_wait_ns{1000000000ull};

// Device buffer that grows on demand.
struct DBuf {
    void *p = nullptr;
    size_t bytes = 0;
    ~DBuf() { if (p) cudaFree(p); }
    cudaError_t reserve(size_t b) {
        if (b <= bytes) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        for (int f = g_alloc_failures.load(); f > 0;)
            if (g_alloc_failures.compare_exchange_weak(f, f - 1)) return cudaErrorMemoryAllocation;
        cudaError_t e = cudaMalloc(&p, b);
        if (e == cudaSuccess) bytes = b;
        return e;
    }
    template <typename T> T *as() const { return (T *)p; }
};

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

namespace fpk {
void set_last_error(const char *msg) { g_err = msg; }
uint64_t wait_limit_ns() { return g_wait_ns.load(); }
}  // namespace fpk

struct GraphKey {
    int key;
    uint64_t nb;
    const void *pairs, *raw, *maps, *states, *tr, *kappa, *err;
    bool operator<(const GraphKey &o) const {
        return std::tie(key, nb, pairs, raw, maps, states, tr, kappa, err) <
               std::tie(o.key, o.nb, o.pairs, o.raw, o.maps, o.states, o.tr, o.kappa, o.err);
    }
};

struct BrickCache {
    BrickHostPlan hp;
    DBuf d_gates, d_rpasses, d_rgates, d_tcwins, d_tcxa;
    BrickDevPlan dp;
    size_t extra_per_pair = 0;   // tensor-core window matrices (bytes per pair, after the boundaries)
    int variant[4] = {0, 0, 0, 0};   // tile bits, window bits, threads, pass kind (fp_brick_variant)
    double mma_flops_pair = 0;       // tensor-core flops issued per pair (tensor-core passes)
};

struct SpiralCache {        // one depth of the paper's HEA on the spiral sweep
    SpiralPlan sp;
    DBuf d_maps, d_items, d_refs, d_plan;
    // variants: FP64, FP32, FP64 spread over a 4-CTA cluster (small batches:
    // the FP64 recontraction of a few flagged pairs)
    SpiralConfig cfg[3];
    DBuf d_wins[3], d_ij[3];   // register windows of cfg[p]
    int nwins[3] = {0, 0, 0}, h[3][2] = {{-1, -1}, {-1, -1}, {-1, -1}};
};

struct fp_ensemble {
    fp_ensemble_desc d;
    cudaStream_t st = nullptr;
    int device = 0;
    int sms = 0;
    int raw_kind = RAW_HAAR4;
    int n_groups = 0;
    size_t ws_budget = 0;
    // fixed-topology plan cache
    std::map<int, int> plan_of_depth;
    std::vector<HostPlan> plans;
    bool dev_plans_dirty = true;
    // device plan pools (fixed topology) and per-batch pools (local)
    DBuf d_plans, d_ops, d_recipes, d_items, d_refs;
    // batch buffers
    DBuf d_pairs, d_order, d_raw, d_merged, d_tables, d_ws, d_ticket, d_tr, d_kappa, d_err, d_group;
    DBuf d_partials, d_moments;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEvent_t kev[2 * FP_K_CLASSES] = {};
    fp_kernel_stats kst{};
    uint64_t kst_requeued = 0;
    bool timing = false;
    // brickwork fast path
    std::map<int, std::unique_ptr<BrickCache>> brick_plans;   // key brick_key(l, prec)
    // spiral sweep (the paper's HEA), per depth; null: the depth is not spiral-shaped
    std::map<int, std::unique_ptr<SpiralCache>> spiral_plans;
    DBuf d_spiral_scratch;
    DBuf d_maps, d_states;
    DBuf d_flag;               // device error flag of kernels with bounded waits (zero when clear)
    std::atomic<int> cancel{0};   // fp_cancel: checked by the Monte Carlo driver between batches
    std::string gpu_name;
    // CUDA graphs of the brickwork sub-batch pipeline
    cudaStream_t gst = nullptr;
    cudaEvent_t gev[2] = {};
    std::map<GraphKey, cudaGraphExec_t> graphs;
    uint64_t graph_replays = 0;
    // FP_FLAG_SKIP_INFEASIBLE: slots (relative to the current call's first pair)
    // left uncontracted because their boundary exceeds FP_MAX_STATE_BITS
    std::vector<uint64_t> skipped;
    DBuf d_skip;
    // bootstrap buffers
    DBuf d_boot_tr, d_boot_members, d_boot_off, d_boot_xs, d_boot_out;
    // resident clusters of the generic sweep per cluster size (index log2 cs) and precision; -1 unknown
    int sweep_slots[5][2] = {{-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}};
};

namespace {

int depth_of_pair(const fp_ensemble_desc &d, uint64_t pair) {
    U64x4 x = philox(d.seed, 0, 0, pair, 4);
    if (d.kind == FP_LOCAL) {
        uint32_t choices = (uint32_t)((d.T_max - d.T_min) / d.T_step + 1);
        return d.T_min + (int)pick(x.x[0], choices) * d.T_step;
    }
    uint32_t choices = (uint32_t)(d.depth_max - d.depth_min + 1);
    return d.depth_min + (int)pick(x.x[0], choices);
}

int group_of_depth(const fp_ensemble_desc &d, int depth) {
    return d.kind == FP_LOCAL ? (depth - d.T_min) / d.T_step : depth - d.depth_min;
}

std::vector<int> local_bonds(const fp_ensemble_desc &d, uint64_t pair, int which, int T) {
    int w = (d.flags & FP_FLAG_SELF_PAIR) ? 0 : which;
    std::vector<int> b(T);
    for (int g = 0; g < T; ++g) {
        U64x4 x = philox(d.seed, 0, (uint64_t)g, pair, (uint64_t)(2 + w));
        b[g] = (int)pick(x.x[0], (uint32_t)(d.n - 1));
    }
    return b;
}

// f(i) for i in [0, count) on the host cores (at most 64 threads; serial for
// small counts).  f must be safe to run concurrently for different i.
template <typename F>
void parallel_for(uint64_t count, F f) {
    unsigned nt = std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
    if (count < 64 || nt == 1) {
        for (uint64_t i = 0; i < count; ++i) f(i);
        return;
    }
    nt = (unsigned)std::min<uint64_t>(nt, count / 16);
    std::atomic<uint64_t> next{0};
    auto work = [&]() {
        for (;;) {
            const uint64_t i0 = next.fetch_add(16);
            if (i0 >= count) return;
            for (uint64_t i = i0; i < std::min(count, i0 + 16); ++i) f(i);
        }
    };
    std::vector<std::thread> th;
    for (unsigned t = 1; t < nt; ++t) th.emplace_back(work);
    work();
    for (auto &t : th) t.join();
}

// Gate layout of circuit `which` of a pair and the number of raw gates per circuit.
std::vector<GateSlot> circuit_layout(const fp_ensemble_desc &d, uint64_t pair, int which, int depth, int *n_raw) {
    switch (d.kind) {
        case FP_PARALLEL: {
            std::vector<GateSlot> g = layout_brickwork(d.n, depth);
            *n_raw = (int)g.size();
            return g;
        }
        case FP_HEA:
            *n_raw = depth * d.n;
            return layout_hea(d.n, depth);
        case FP_HEA_PAULI:
            *n_raw = 1 + d.n + depth * d.n;
            return layout_hea_pauli(d.n, depth, (d.flags & FP_FLAG_HEA_CZ) != 0);
        default:
            *n_raw = depth;
            return layout_local(d.n, local_bonds(d, pair, which, depth));
    }
}

HostPlan build_plan(const fp_ensemble_desc &d, int raw_kind, int depth, uint64_t pair) {
    int n_raw = 0;
    std::vector<GateSlot> U = circuit_layout(d, pair, 0, depth, &n_raw);
    std::vector<GateSlot> V = circuit_layout(d, pair, 1, depth, &n_raw);
    return make_plan(d.n, U, V, raw_kind, n_raw, d.n / 2, FP_MAX_STATE_BITS);
}

// Flatten host plans into device pools.
struct PlanPools {
    std::vector<DevPlan> plans;
    std::vector<DevOp> ops;
    std::vector<DevRecipe> recipes;
    std::vector<MergeItem> items;
    std::vector<MergeRef> refs;
    void add(const HostPlan &h) {
        DevPlan p;
        std::memset(&p, 0, sizeof p);
        p.n_left = h.n_left;
        p.n_right = h.n_right;
        p.ops_off = (int)ops.size();
        p.rec_off = (int)recipes.size();
        p.merge_off = (int)items.size();
        p.n_merged = (int)h.merges.size();
        p.ref_off = (int)refs.size();
        p.n_raw = h.n_raw;
        p.raw_kind = h.raw_kind;
        p.bits_max = h.bits_max;
        p.bits_final = h.bits_final;
        p.left_final_buf = h.left_final_buf;
        for (int k = 0; k < FP_MAX_STATE_BITS; ++k) p.dot_perm[k] = h.dot_perm[k];
        p.prefactor = h.prefactor;
        p.cost = h.cost;
        p.sqrt_ops = std::sqrt((double)std::max(1, std::max(h.n_left, h.n_right)));
        ops.insert(ops.end(), h.ops.begin(), h.ops.end());
        recipes.insert(recipes.end(), h.recipes.begin(), h.recipes.end());
        items.insert(items.end(), h.merges.begin(), h.merges.end());
        refs.insert(refs.end(), h.refs.begin(), h.refs.end());
        plans.push_back(p);
    }
};

template <typename T>
cudaError_t upload(DBuf &b, const std::vector<T> &v, cudaStream_t st) {
    size_t bytes = std::max<size_t>(sizeof(T), v.size() * sizeof(T));
    cudaError_t e = b.reserve(bytes);
    if (e != cudaSuccess || v.empty()) return e;
    return cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st);
}

fp_status upload_pools(fp_ensemble *E, const PlanPools &pp) {
    CK(upload(E->d_plans, pp.plans, E->st));
    CK(upload(E->d_ops, pp.ops, E->st));
    CK(upload(E->d_recipes, pp.recipes, E->st));
    CK(upload(E->d_items, pp.items, E->st));
    CK(upload(E->d_refs, pp.refs, E->st));
    return FP_OK;
}

// Optional per-launch CUDA-event timing (FP_FLAG_TIMING).
struct KTimer {
    fp_ensemble *E;
    int cls;
    KTimer(fp_ensemble *e, int c) : E(e), cls(c) {
        if (E->timing) cudaEventRecord(E->kev[2 * cls], E->st);
    }
    cudaError_t stop(double work, int launches = 1) {
        if (!E->timing) return cudaSuccess;
        cudaError_t e = cudaEventRecord(E->kev[2 * cls + 1], E->st);
        if (e != cudaSuccess) return e;
        if ((e = cudaEventSynchronize(E->kev[2 * cls + 1])) != cudaSuccess) return e;
        float ms = 0;
        if ((e = cudaEventElapsedTime(&ms, E->kev[2 * cls], E->kev[2 * cls + 1])) != cudaSuccess) return e;
        E->kst.ms[cls] += ms;
        E->kst.launches[cls] += (uint64_t)launches;
        E->kst.work[cls] += work;
        return cudaSuccess;
    }
};

// Generic path over a subset of pairs: outputs go to slots idx[i] of the
// device arrays (pairs first + idx[i]).
fp_status run_generic(fp_ensemble *E, uint64_t first, const std::vector<uint64_t> &idx_in,
                      const std::vector<int> &depth, int prec, double *tr, double *kappa, double *err,
                      float *gpu_ms) {
    const fp_ensemble_desc &d = E->d;
    const bool local = d.kind == FP_LOCAL;
    const bool skip = (d.flags & FP_FLAG_SKIP_INFEASIBLE) != 0;
    if (idx_in.empty()) return FP_OK;
    std::vector<int> plan_idx;
    std::vector<HostPlan> local_plans;
    std::vector<uint64_t> kept;   // output slots contracted here, in batch order
    PlanPools pools;
    if (!local) {
        for (uint64_t slot : idx_in) {
            const int dep = depth[slot];
            auto it = E->plan_of_depth.find(dep);
            if (it == E->plan_of_depth.end()) {
                HostPlan h = build_plan(d, E->raw_kind, dep, first + slot);
                if (!h.error.empty() && !h.infeasible) return fail(FP_ERR_ARG, "planner: %s", h.error.c_str());
                if (h.infeasible && !skip) return fail(FP_ERR_INFEASIBLE, "depth %d: %s", dep, h.error.c_str());
                E->plans.push_back(std::move(h));
                it = E->plan_of_depth.emplace(dep, (int)E->plans.size() - 1).first;
                E->dev_plans_dirty = true;
            }
            const HostPlan &h = E->plans[it->second];
            if (h.infeasible) {
                if (!skip) return fail(FP_ERR_INFEASIBLE, "depth %d: %s", dep, h.error.c_str());
                E->skipped.push_back(slot);
                continue;
            }
            plan_idx.push_back(it->second);
            kept.push_back(slot);
        }
        if (E->dev_plans_dirty) {
            for (const auto &h : E->plans) pools.add(h);
            fp_status s = upload_pools(E, pools);
            if (s != FP_OK) return s;
            E->dev_plans_dirty = false;
        }
    } else {
        // every local-circuit pair has its own topology: plan them on the host
        // cores in parallel, then order the batch by boundary size so that the
        // memory-budgeted sub-batches below group pairs of similar workspace
        const uint64_t n_in = idx_in.size();
        std::vector<HostPlan> all(n_in);
        parallel_for(n_in, [&](uint64_t i) {
            all[i] = build_plan(d, E->raw_kind, depth[idx_in[i]], first + idx_in[i]);
        });
        std::vector<uint64_t> feas;
        for (uint64_t i = 0; i < n_in; ++i) {
            const HostPlan &h = all[i];
            if (h.infeasible) {
                if (!skip)
                    return fail(FP_ERR_INFEASIBLE, "pair %llu (T=%d): %s", (unsigned long long)(first + idx_in[i]),
                                depth[idx_in[i]], h.error.c_str());
                E->skipped.push_back(idx_in[i]);
                continue;
            }
            if (!h.error.empty()) return fail(FP_ERR_ARG, "planner: %s", h.error.c_str());
            feas.push_back(i);
        }
        std::stable_sort(feas.begin(), feas.end(),
                         [&](uint64_t a, uint64_t b) { return all[a].bits_max < all[b].bits_max; });
        for (uint64_t i : feas) {
            local_plans.push_back(std::move(all[i]));
            kept.push_back(idx_in[i]);
        }
        for (uint64_t i = 0; i < local_plans.size(); ++i) {
            pools.add(local_plans[i]);
            plan_idx.push_back((int)i);
        }
        if (!local_plans.empty()) {
            fp_status s = upload_pools(E, pools);
            if (s != FP_OK) return s;
            E->dev_plans_dirty = true;   // the fixed-topology pool was overwritten
        }
    }
    const uint64_t count = kept.size();
    if (count == 0) return FP_OK;
    const std::vector<uint64_t> &idx = kept;
    auto hp = [&](uint64_t i) -> const HostPlan & { return local ? local_plans[i] : E->plans[plan_idx[i]]; };
    const bool fp32 = prec != FP_PREC_FP64;
    const size_t celem = fp32 ? sizeof(float2) : sizeof(double2);
    // pairs with large boundaries get a cluster of CTAs each (see sweep_cluster_size)
    auto cluster_of = [&](int bits) {
        int cs = sweep_cluster_size(bits);
        while (cs > 1) {
            int lg = cs == 4 ? 2 : (cs == 8 ? 3 : 4);
            int &slots = E->sweep_slots[lg][fp32 ? 1 : 0];
            if (slots < 0) slots = sweep_max_clusters(cs, fp32);
            if (slots > 0) return std::make_pair(cs, slots);
            cs /= 2;   // clusters of this size cannot launch here: smaller ones
            if (cs == 2) cs = 1;
        }
        return std::make_pair(1, E->sms * 2);
    };
    uint64_t done = 0;
    while (done < count) {
        uint64_t nb = 0;
        size_t raw_b = 0, mer_b = 0, tab_b = 0;
        int bits_max = 0, max_raw = 0, max_mer = 0, max_ops = 0;
        while (done + nb < count && nb < 65535) {
            const HostPlan &h = hp(done + nb);
            size_t r = (size_t)2 * h.n_raw * 16 * sizeof(double2);
            size_t m = h.merges.size() * 16 * sizeof(double2);
            size_t t = h.ops.size() * 16 * sizeof(double2);
            int bm = std::max(bits_max, h.bits_max);
            const int slots_full = cluster_of(bm).second;
            size_t ws = (size_t)std::min<uint64_t>(slots_full, nb + 1) * 3 * ((size_t)1 << bm) * sizeof(double2);
            if (nb > 0 && raw_b + r + mer_b + m + tab_b + t + ws > E->ws_budget) break;
            raw_b += r; mer_b += m; tab_b += t; bits_max = bm;
            max_raw = std::max(max_raw, h.n_raw);
            max_mer = std::max<int>(max_mer, (int)h.merges.size());
            max_ops = std::max<int>(max_ops, (int)h.ops.size());
            ++nb;
        }
        std::vector<PairInfo> pinfo(nb);
        int64_t ro = 0, mo = 0, to = 0;
        double cmacs = 0;
        for (uint64_t i = 0; i < nb; ++i) {
            const HostPlan &h = hp(done + i);
            pinfo[i].pair = first + idx[done + i];
            pinfo[i].plan = plan_idx[done + i];
            pinfo[i].n_raw = h.n_raw;
            pinfo[i].raw_off = ro;
            pinfo[i].merged_off = mo;
            pinfo[i].table_off = to;
            pinfo[i].out = (int64_t)idx[done + i];
            ro += 2 * h.n_raw;
            mo += (int64_t)h.merges.size();
            to += (int64_t)h.ops.size();
            cmacs += h.cost;
        }
        std::vector<int32_t> order(nb);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return hp(done + a).cost > hp(done + b).cost; });
        const auto cl = cluster_of(bits_max);
        const int slots = (int)std::min<uint64_t>(nb, (uint64_t)cl.second);
        const int ctas = slots * cl.first;
        size_t ws_elems = (size_t)1 << bits_max;
        CK(upload(E->d_pairs, pinfo, E->st));
        CK(upload(E->d_order, order, E->st));
        CK(E->d_raw.reserve(std::max<size_t>(16, ro * 16 * sizeof(double2))));
        CK(E->d_merged.reserve(std::max<size_t>(16, mo * 16 * sizeof(double2))));
        CK(E->d_tables.reserve(std::max<size_t>(16, to * 16 * sizeof(double2))));
        CK(E->d_ws.reserve((size_t)slots * 3 * ws_elems * celem));
        SampleParams sp;
        sp.seed = d.seed;
        sp.n = d.n;
        sp.raw_kind = E->raw_kind;
        sp.self_pair = (d.flags & FP_FLAG_SELF_PAIR) ? 1 : 0;
        CK(cudaEventRecord(E->ev0, E->st));
        {
            KTimer t(E, FP_K_SAMPLE);
            CK(launch_sample(sp, E->d_pairs.as<PairInfo>(), (int)nb, max_raw, E->d_raw.as<double2>(), E->st));
            CK(t.stop((double)nb, sample_launch_count(E->raw_kind)));
        }
        {
            KTimer t(E, FP_K_MERGE);
            CK(launch_merge(E->d_pairs.as<PairInfo>(), (int)nb, max_mer, E->d_plans.as<DevPlan>(),
                            E->d_items.as<MergeItem>(), E->d_refs.as<MergeRef>(), E->d_raw.as<double2>(),
                            E->d_merged.as<double2>(), E->st));
            CK(t.stop((double)nb));
        }
        {
            KTimer t(E, FP_K_TABLES);
            CK(launch_tables(E->d_pairs.as<PairInfo>(), (int)nb, max_ops, E->d_plans.as<DevPlan>(),
                             E->d_recipes.as<DevRecipe>(), E->d_merged.as<double2>(), E->d_tables.p, fp32, E->st));
            CK(t.stop((double)nb));
        }
        {
            KTimer t(E, FP_K_SWEEP);
            CK(launch_sweep_generic(E->d_pairs.as<PairInfo>(), E->d_order.as<int32_t>(), (int)nb, E->d_plans.as<DevPlan>(),
                                    E->d_ops.as<DevOp>(), E->d_tables.p, fp32, E->d_ws.p, ws_elems, ctas,
                                    cl.first, E->d_ticket.as<int>(), FP_ERR_SAFETY * (fp32 ? 0x1.0p-24 : 0x1.0p-53), tr,
                                    kappa, err, E->st));
            CK(t.stop(cmacs));
        }
        CK(cudaEventRecord(E->ev1, E->st));
        CK(cudaEventSynchronize(E->ev1));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, E->ev0, E->ev1));
        if (gpu_ms) *gpu_ms += ms;
        E->kst.pairs += nb;
        done += nb;
    }
    return FP_OK;
}

// Build and upload one brickwork plan variant.
// The device error flag of kernels with bounded waits: a raised flag is
// reported as FP_ERR_TIMEOUT and cleared, so that the ensemble stays usable.
fp_status check_flag(fp_ensemble *E) {
    int h = 0;
    CK(cudaMemcpyAsync(&h, E->d_flag.p, sizeof h, cudaMemcpyDeviceToHost, E->st));
    CK(cudaStreamSynchronize(E->st));
    if (!h) return FP_OK;
    CK(cudaMemsetAsync(E->d_flag.p, 0, sizeof h, E->st));
    return fail(FP_ERR_TIMEOUT, "a bounded device wait ran out in the tensor-core tile pass (results discarded)");
}

// The brickwork plan cache's key: depth and precision class (FP64; FP32 with the
// autotuner's free choice; FP32 restricted to the tensor-core passes).
int brick_key(int l, int prec) {
    return 4 * l + (prec == FP_PREC_FP64 ? 0 : prec == FP_PREC_TF32X3 ? 2 : 1);
}

fp_status make_brick_cache(fp_ensemble *E, int l, bool fp32, int K, int R, int TH, int persist,
                           std::unique_ptr<BrickCache> &out) {
    auto bc = std::make_unique<BrickCache>();
    bc->variant[0] = K; bc->variant[1] = R; bc->variant[2] = TH; bc->variant[3] = persist;
    // K > N: shared-memory sweep, K == N: one tile
    // arcs hold the 5 (FP32) or 4 (FP64) lowest bits, so that tile loads read contiguous runs;
    // the tensor-core pass (12-bit tiles) holds 3: at l = 10 a 12-bit arc through the 5
    // lowest bits would need 49 passes instead of 18
    bc->hp = make_brick_plan(E->d.n, l, K, persist >= 3 ? 3 : (fp32 ? 5 : 4), R, E->d.kind == FP_HEA ? 1 : 0);
    for (const auto &ps : bc->hp.passes) {
        if (ps.n_gates > 255) return fail(FP_ERR_ARG, "tile pass with %d gates exceeds 255", ps.n_gates);
        if (ps.n_rp > 160) return fail(FP_ERR_ARG, "tile pass with %d register passes exceeds 160", ps.n_rp);
    }
    if (persist == 3 || persist == 4) {   // tensor-core windows: FP32, 12-bit tiles, 5-bit windows only
        if (!fp32 || !tc_plan_ok(bc->hp.dev, bc->hp.passes.data(), bc->hp.rpasses.data()))
            return fail(FP_ERR_ARG, "the tensor-core tile pass needs FP32, %d-bit tiles, %d-bit windows and l >= 8",
                        kTcTile, kMaxWin);
        const std::vector<TcWin> wins = make_tc_windows(bc->hp);
        CK(upload(bc->d_tcwins, wins, E->st));
        CK(upload(bc->d_tcxa, make_tc_xaddr(bc->hp, wins), E->st));
        bc->dp.tcwins = bc->d_tcwins.as<TcWin>();
        bc->dp.tcxa = bc->d_tcxa.as<TcXa>();
        bc->extra_per_pair = tc_wmat_bytes_per_pair(bc->hp.dev, bc->hp.passes.data());
        // per window and tile: 3 products x 8 K steps of a 128 x 64 x 8 MMA
        double windows = 0;
        for (const BrickPass &ps : bc->hp.passes) windows += ps.n_rp;
        bc->mma_flops_pair = windows * (double)(1u << (bc->hp.dev.N - kTcTile)) * 3.0 * 2.0 * 128.0 * 64.0 * 64.0;
        if (!E->d_flag.p) {
            CK(E->d_flag.reserve(16));
            CK(cudaMemsetAsync(E->d_flag.p, 0, 16, E->st));
        }
        bc->dp.err_flag = E->d_flag.as<int>();
    }
    CK(upload(bc->d_gates, bc->hp.gates, E->st));
    CK(upload(bc->d_rpasses, bc->hp.rpasses, E->st));
    CK(upload(bc->d_rgates, bc->hp.rgates, E->st));
    bc->dp.gates = bc->d_gates.as<BrickGate>();
    bc->dp.rpasses = bc->d_rpasses.as<RegPass>();
    bc->dp.rgates = bc->d_rgates.as<RegGate>();
    bc->dp.win_bits = R;
    bc->dp.threads = TH;
    bc->dp.persist = persist;
    out = std::move(bc);
    return FP_OK;
}

// Autotuner: time every (tile bits, window bits) variant of the tiled
// brickwork sweep on a trial batch of this depth (sampler and maps once, then
// each variant's init + passes + meet), keep the fastest.  Results persist in
// the file named by FP_AUTOTUNE_CACHE (if set), keyed by GPU name, n, l and
// precision.
fp_status tune_brick(fp_ensemble *E, uint64_t first, const std::vector<uint64_t> &idx, int l, int prec) {
    const fp_ensemble_desc &d = E->d;
    const int N = 2 * (l - 1);
    const bool fp32 = prec != FP_PREC_FP64;
    const int key = brick_key(l, prec);
    struct Cand { int K, R, TH, P; };
    // K = 99: whole boundary in one CTA's shared memory (brick_smem_kernel);
    // P = 1: persistent double-buffered tile passes (brick_pass_db_kernel)
    std::vector<Cand> cands = fp32 ? std::vector<Cand>{{14, 4, 512, 0}, {14, 5, 256, 0}, {13, 4, 512, 0},
                                                       {13, 4, 256, 0}, {13, 5, 256, 0}, {13, 4, 512, 1},
                                                       {13, 5, 256, 1}, {12, 4, 256, 0}, {12, 5, 128, 0}}
                                   : std::vector<Cand>{{13, 3, 512, 0}, {13, 4, 256, 0}};
    if (((size_t)1 << N) * (fp32 ? sizeof(float2) : sizeof(double2)) <= (size_t)200 * 1024) cands.push_back({99, 0, 0, 0});
    // P = 3, 4: tensor-core windows (TF32 x 3 tcgen05 MMAs), boundaries of more than two 12-bit tiles
    if (fp32 && N >= kTcTile + 2) {
        cands.push_back({kTcTile, kMaxWin, 256, 3});   // the tile's operand in shared memory
        cands.push_back({kTcTile, kMaxWin, 256, 4});   // in tensor memory, persistent over the tiles
    }
    const int kmin = 10;   // boundaries up to 2^10: shared-memory sweep, nothing to tune
    char ckey[256];
    // the HEA's ring has its own plans: its entries carry the kind after the precision
    snprintf(ckey, sizeof ckey, "%s n=%d l=%d %s%s", E->gpu_name.c_str(), d.n, l,
             !fp32 ? "fp64" : (prec == FP_PREC_TF32X3 && N >= kTcTile + 2) ? "tf32x3" : "fp32",
             d.kind == FP_HEA ? " hea" : "");
    int bestK = cands[0].K, bestR = cands[0].R, bestT = cands[0].TH, bestP = 0;
    bool have = false;
    const char *cache = getenv("FP_AUTOTUNE_CACHE");
    if (N <= kmin) {
        have = true;            // whole boundary in one CTA: nothing to tune
        bestK = 99;
    } else if (cache) {
        FILE *f = fopen(cache, "r");
        if (f) {
            char line[512];
            while (fgets(line, sizeof line, f)) {
                int K, R, T, Pp = 0;
                char k2[256];
                if (sscanf(line, "%255[^|]|%d %d %d %d", k2, &K, &R, &T, &Pp) >= 4 && strcmp(k2, ckey) == 0) {
                    bestK = K; bestR = R; bestT = T; bestP = Pp; have = true;
                }
            }
            fclose(f);
        }
    }
    std::unique_ptr<BrickCache> cached;
    if (have && N > kmin && make_brick_cache(E, l, fp32, bestK, bestR, bestT, bestP, cached) != FP_OK) {
        have = false;   // a cache entry this depth cannot run (another build's file): tune instead
        cached.reset();
    }
    if (!have && !idx.empty()) {
        const uint64_t nt = std::min<uint64_t>(idx.size(), 192);   // several waves of tiles per variant
        const int n_raw = d.kind == FP_HEA ? l * d.n : (int)layout_brickwork(d.n, l).size();
        const int n_maps = (d.kind == FP_HEA ? 2 * d.n : d.n - 1) * (l - 1);
        const size_t celem = fp32 ? sizeof(float2) : sizeof(double2);
        std::vector<PairInfo> pinfo(nt);
        for (uint64_t i = 0; i < nt; ++i) {
            std::memset(&pinfo[i], 0, sizeof(PairInfo));
            pinfo[i].pair = first + idx[i];
            pinfo[i].n_raw = n_raw;
            pinfo[i].raw_off = (int64_t)i * 2 * n_raw;
            pinfo[i].out = (int64_t)idx[i];
        }
        CK(upload(E->d_pairs, pinfo, E->st));
        CK(E->d_raw.reserve(nt * 2 * n_raw * 16 * sizeof(double2)));
        CK(E->d_maps.reserve(nt * n_maps * 16 * celem));
        CK(E->d_states.reserve(nt * 2 * ((size_t)1 << N) * celem));
        SampleParams sp;
        sp.seed = d.seed; sp.n = d.n; sp.raw_kind = E->raw_kind; sp.self_pair = (d.flags & FP_FLAG_SELF_PAIR) ? 1 : 0;
        CK(launch_sample(sp, E->d_pairs.as<PairInfo>(), (int)nt, n_raw, E->d_raw.as<double2>(), E->st));
        float best_ms = 1e30f;
        // FP_PREC_TF32X3: the fastest tensor-core variant when one runs, else the fastest of all
        float best_tc_ms = 1e30f;
        Cand best_tc{0, 0, 0, 0};
        for (const Cand &c : cands) {
            std::unique_ptr<BrickCache> bc;
            if (c.K != 99 && c.K > N) continue;   // tiles larger than the boundary
            fp_status s = make_brick_cache(E, l, fp32, c.K, c.R, c.TH, c.P, bc);
            if (s != FP_OK) continue;
            if (bc->extra_per_pair) CK(E->d_states.reserve(nt * (2 * ((size_t)1 << N) * celem + bc->extra_per_pair)));
            float ms_sum = 0;
            for (int rep = 0; rep < 2; ++rep) {
                CK(cudaEventRecord(E->ev0, E->st));
                int nl = 0;
                if (launch_brick(bc->hp.dev, bc->hp.passes.data(), bc->dp, E->d_pairs.as<PairInfo>(), (int)nt,
                                 E->d_raw.as<double2>(), E->d_maps.p, E->d_states.p, fp32, 0.0, E->d_tr.as<double>(),
                                 nullptr, nullptr, E->st, &nl) != cudaSuccess) {
                    cudaGetLastError();   // a variant this device cannot launch: skip it
                    ms_sum = 1e30f;
                    break;
                }
                CK(cudaEventRecord(E->ev1, E->st));
                CK(cudaEventSynchronize(E->ev1));
                float ms = 0;
                CK(cudaEventElapsedTime(&ms, E->ev0, E->ev1));
                if (rep == 1) ms_sum += ms;     // first repetition warms caches and code
                if (bc->dp.err_flag) {
                    fp_status fs = check_flag(E);
                    if (fs != FP_OK) return fs;
                }
            }
            if (ms_sum < best_ms) { best_ms = ms_sum; bestK = c.K; bestR = c.R; bestT = c.TH; bestP = c.P; }
            if (c.P >= 3 && ms_sum < best_tc_ms) { best_tc_ms = ms_sum; best_tc = c; }
        }
        if (prec == FP_PREC_TF32X3 && best_tc_ms < 1e30f) {
            bestK = best_tc.K; bestR = best_tc.R; bestT = best_tc.TH; bestP = best_tc.P;
        }
        if (cache) {
            FILE *f = fopen(cache, "a");
            if (f) { fprintf(f, "%s|%d %d %d %d\n", ckey, bestK, bestR, bestT, bestP); fclose(f); }
        }
    }
    std::unique_ptr<BrickCache> bc = std::move(cached);
    if (!bc) {
        fp_status s = make_brick_cache(E, l, fp32, bestK, bestR, bestT, bestP, bc);
        if (s != FP_OK) return s;
    }
    E->brick_plans.emplace(key, std::move(bc));
    return FP_OK;
}

// Brickwork fast path for pairs of one depth l >= 2.
fp_status run_brick(fp_ensemble *E, uint64_t first, const std::vector<uint64_t> &idx, int l, int prec,
                    double *tr, double *kappa, double *err, float *gpu_ms) {
    const fp_ensemble_desc &d = E->d;
    const uint64_t count = idx.size();
    if (count == 0) return FP_OK;
    const bool fp32 = prec != FP_PREC_FP64;
    const int N = 2 * (l - 1);
    if (N > FP_MAX_STATE_BITS)
        return fail(FP_ERR_INFEASIBLE, "depth %d: boundary of %d bits exceeds the limit of %d", l, N, FP_MAX_STATE_BITS);
    const int key = brick_key(l, prec);
    auto it = E->brick_plans.find(key);
    if (it == E->brick_plans.end()) {
        fp_status s = tune_brick(E, first, idx, l, prec);
        if (s != FP_OK) return s;
        it = E->brick_plans.find(key);
    }
    const BrickHostPlan &bp = it->second->hp;
    const BrickDev &bd = bp.dev;
    const size_t celem = fp32 ? sizeof(float2) : sizeof(double2);
    const size_t S = (size_t)1 << N;
    const int n_raw = d.kind == FP_HEA ? l * d.n : (int)layout_brickwork(d.n, l).size();
    const size_t per_raw = (size_t)2 * n_raw * 16 * sizeof(double2);
    const size_t per_map = (size_t)maps_per_pair(bd) * 16 * celem;
    bool both = false;
    if (bd.tile_bits == 0) brick_smem_bytes(bd, fp32, &both);
    const size_t per_state = bd.tile_bits ? 2 * S * celem + it->second->extra_per_pair : (both ? 0 : S * celem);
    const size_t per_pair = per_raw + per_map + per_state;
    uint64_t cap = std::max<uint64_t>(1, std::min<uint64_t>(65535, E->ws_budget / per_pair));
    // flop count of the sweep (complex multiply-adds): 4 per amplitude per gate
    const double cmac_pair = 4.0 * (double)S * (double)maps_per_pair(bd);
    SampleParams sp;
    sp.seed = d.seed;
    sp.n = d.n;
    sp.raw_kind = E->raw_kind;
    sp.self_pair = (d.flags & FP_FLAG_SELF_PAIR) ? 1 : 0;
    for (uint64_t done = 0; done < count;) {
        const uint64_t nb = std::min<uint64_t>(cap, count - done);
        std::vector<PairInfo> pinfo(nb);
        for (uint64_t i = 0; i < nb; ++i) {
            std::memset(&pinfo[i], 0, sizeof(PairInfo));
            pinfo[i].pair = first + idx[done + i];
            pinfo[i].n_raw = n_raw;
            pinfo[i].raw_off = (int64_t)i * 2 * n_raw;
            pinfo[i].out = (int64_t)idx[done + i];
        }
        CK(upload(E->d_pairs, pinfo, E->st));
        CK(E->d_raw.reserve(nb * per_raw));
        CK(E->d_maps.reserve(nb * per_map));
        CK(E->d_states.reserve(std::max<size_t>(16, nb * per_state)));
        const double G = (double)std::max(bd.n_layers[0], bd.n_layers[1]) * bd.m;
        const double err_scale = FP_ERR_SAFETY * (fp32 ? 0x1.0p-24 : 0x1.0p-53) * std::sqrt(G);
        // CUDA graph replay: the launch sequence of a sub-batch (sampler, maps,
        // init, passes, meet) is captured once per (depth, precision, size,
        // buffers) on the ensemble's internal stream and replayed with fresh
        // pair records; the first sub-batch of a shape runs directly (it also
        // sets the kernels' shared-memory attributes outside any capture).
        const bool use_graph = !E->timing && !(d.flags & FP_FLAG_NO_GRAPHS);
        GraphKey gk{key, nb, E->d_pairs.p, E->d_raw.p, E->d_maps.p, E->d_states.p, tr, kappa, err};
        auto git = use_graph ? E->graphs.find(gk) : E->graphs.end();
        CK(cudaEventRecord(E->ev0, E->st));
        if (use_graph && git != E->graphs.end() && git->second) {
            CK(cudaEventRecord(E->gev[0], E->st));
            CK(cudaStreamWaitEvent(E->gst, E->gev[0], 0));
            CK(cudaGraphLaunch(git->second, E->gst));
            CK(cudaEventRecord(E->gev[1], E->gst));
            CK(cudaStreamWaitEvent(E->st, E->gev[1], 0));
            E->graph_replays++;
        } else {
            {
                KTimer t(E, FP_K_SAMPLE);
                CK(launch_sample(sp, E->d_pairs.as<PairInfo>(), (int)nb, n_raw, E->d_raw.as<double2>(), E->st));
                CK(t.stop((double)nb, sample_launch_count(E->raw_kind)));
            }
            {
                KTimer t(E, FP_K_BRICK);
                int nl = 0;
                CK(launch_brick(bd, bp.passes.data(), it->second->dp, E->d_pairs.as<PairInfo>(), (int)nb,
                                E->d_raw.as<double2>(), E->d_maps.p, E->d_states.p, fp32, err_scale, tr, kappa, err,
                                E->st, &nl));
                CK(t.stop(cmac_pair * (double)nb));
                if (E->timing) {
                    E->kst.launches[FP_K_BRICK] += (uint64_t)(nl - 1);
                    E->kst.mma_flops += it->second->mma_flops_pair * (double)nb;
                }
            }
            if (use_graph) {
                if (E->graphs.size() > 64) {
                    for (auto &kv : E->graphs) if (kv.second) cudaGraphExecDestroy(kv.second);
                    E->graphs.clear();
                }
                cudaGraph_t graph = nullptr;
                cudaGraphExec_t exec = nullptr;
                CK(cudaStreamBeginCapture(E->gst, cudaStreamCaptureModeThreadLocal));
                cudaError_t ce = launch_sample(sp, E->d_pairs.as<PairInfo>(), (int)nb, n_raw, E->d_raw.as<double2>(), E->gst);
                int nl = 0;
                if (ce == cudaSuccess)
                    ce = launch_brick(bd, bp.passes.data(), it->second->dp, E->d_pairs.as<PairInfo>(), (int)nb,
                                      E->d_raw.as<double2>(), E->d_maps.p, E->d_states.p, fp32, err_scale, tr, kappa,
                                      err, E->gst, &nl);
                cudaError_t ee = cudaStreamEndCapture(E->gst, &graph);
                if (ce == cudaSuccess && ee == cudaSuccess && graph) {
                    ce = cudaGraphInstantiate(&exec, graph, 0);
                    if (ce != cudaSuccess) exec = nullptr;
                }
                if (graph) cudaGraphDestroy(graph);
                cudaGetLastError();           // a failed capture leaves the direct path in use
                E->graphs[gk] = exec;
            }
        }
        CK(cudaEventRecord(E->ev1, E->st));
        CK(cudaEventSynchronize(E->ev1));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, E->ev0, E->ev1));
        if (gpu_ms) *gpu_ms += ms;
        if (it->second->dp.err_flag) {
            fp_status fs = check_flag(E);
            if (fs != FP_OK) return fs;
        }
        E->kst.pairs += nb;
        done += nb;
    }
    return FP_OK;
}

// The spiral program of depth L (built and uploaded once); null when the
// circuit is not spiral-shaped (the generic sweep takes it then).
SpiralCache *spiral_plan(fp_ensemble *E, int L) {
    auto it = E->spiral_plans.find(L);
    if (it != E->spiral_plans.end()) return it->second.get();
    std::unique_ptr<SpiralCache> sc;
    int n_raw = 0;
    const std::vector<GateSlot> lay = circuit_layout(E->d, 0, 0, L, &n_raw);
    SpiralPlan sp = make_spiral_plan(E->d.n, lay, lay, E->raw_kind);
    if (sp.ok) {
        sc = std::make_unique<SpiralCache>();
        sc->sp = std::move(sp);
        DevPlan pl;
        std::memset(&pl, 0, sizeof pl);
        pl.n_merged = (int)sc->sp.merges.size();
        pl.n_raw = n_raw;
        pl.raw_kind = E->raw_kind;
        if (upload(sc->d_maps, sc->sp.maps, E->st) != cudaSuccess || upload(sc->d_items, sc->sp.merges, E->st) != cudaSuccess ||
            upload(sc->d_refs, sc->sp.refs, E->st) != cudaSuccess ||
            upload(sc->d_plan, std::vector<DevPlan>{pl}, E->st) != cudaSuccess)
            sc.reset();
        for (int p = 0; sc && p < 3; ++p) {
            sc->cfg[p] = spiral_config(sc->sp.bits, p == 1, p == 2 ? 2 : 0);
            if (sc->cfg[p].R == 0) continue;
            std::vector<SpiralWin> wins;
            std::vector<uint8_t> ij;
            spiral_windows(sc->sp, sc->cfg[p].R, sc->cfg[p].split, wins, ij, sc->h[p]);
            sc->nwins[p] = (int)wins.size();
            if (upload(sc->d_wins[p], wins, E->st) != cudaSuccess || upload(sc->d_ij[p], ij, E->st) != cudaSuccess)
                sc.reset();
        }
    }
    SpiralCache *out = sc.get();
    E->spiral_plans.emplace(L, std::move(sc));
    return out;
}

// Spiral sweep for pairs of one depth L (FP_HEA_PAULI with CNOT walls):
// sampler, merged 1-qubit operators, maps, one CTA per pair; sub-batches
// under the workspace budget.
fp_status run_spiral(fp_ensemble *E, uint64_t first, const std::vector<uint64_t> &idx, int L, SpiralCache *sc, int prec,
                     double *tr, double *kappa, double *err, float *gpu_ms) {
    const fp_ensemble_desc &d = E->d;
    const SpiralPlan &sp = sc->sp;
    const bool fp32 = prec != FP_PREC_FP64;
    const size_t celem = fp32 ? sizeof(float2) : sizeof(double2);
    const int n_raw = 1 + d.n + L * d.n;
    const int n_merged = (int)sp.merges.size(), nmaps = (int)sp.maps.size();
    const int pv = fp32 ? 1 : 0;
    const SpiralConfig &cfg = sc->cfg[pv];
    const size_t scr = cfg.scratch_elems, mw = spiral_map_elems(fp32);
    const size_t per_pair = (size_t)2 * n_raw * 16 * sizeof(double2) + (size_t)n_merged * 16 * sizeof(double2) +
                            (size_t)nmaps * mw * celem + scr * celem;
    // sub-batches of at most 65535 pairs (the sampler and merge grids index pairs by grid.y)
    const uint64_t cap = std::max<uint64_t>(1, std::min<uint64_t>(65535, E->ws_budget / per_pair));
    const double err_scale = FP_ERR_SAFETY * (fp32 ? 0x1.0p-24 : 0x1.0p-53) * std::sqrt((double)nmaps);
    const double cmac_pair = 4.0 * (double)nmaps * (double)((size_t)1 << sp.bits);
    SampleParams smp;
    smp.seed = d.seed;
    smp.n = d.n;
    smp.raw_kind = E->raw_kind;
    smp.self_pair = (d.flags & FP_FLAG_SELF_PAIR) ? 1 : 0;
    for (uint64_t done = 0; done < idx.size();) {
        const uint64_t nb = std::min<uint64_t>(cap, idx.size() - done);
        std::vector<PairInfo> pinfo(nb);
        for (uint64_t i = 0; i < nb; ++i) {
            std::memset(&pinfo[i], 0, sizeof(PairInfo));
            pinfo[i].pair = first + idx[done + i];
            pinfo[i].plan = 0;
            pinfo[i].n_raw = n_raw;
            pinfo[i].raw_off = (int64_t)i * 2 * n_raw;
            pinfo[i].merged_off = (int64_t)i * n_merged;
            pinfo[i].out = (int64_t)idx[done + i];
        }
        CK(upload(E->d_pairs, pinfo, E->st));
        CK(E->d_raw.reserve(nb * 2 * n_raw * 16 * sizeof(double2)));
        CK(E->d_merged.reserve(std::max<size_t>(16, nb * n_merged * 16 * sizeof(double2))));
        CK(E->d_maps.reserve(nb * nmaps * mw * celem));
        CK(E->d_spiral_scratch.reserve(std::max<size_t>(16, nb * scr * celem)));
        CK(cudaEventRecord(E->ev0, E->st));
        {
            KTimer t(E, FP_K_SAMPLE);
            CK(launch_sample(smp, E->d_pairs.as<PairInfo>(), (int)nb, n_raw, E->d_raw.as<double2>(), E->st));
            CK(t.stop((double)nb, sample_launch_count(E->raw_kind)));
        }
        {
            KTimer t(E, FP_K_MERGE);
            CK(launch_merge(E->d_pairs.as<PairInfo>(), (int)nb, n_merged, sc->d_plan.as<DevPlan>(),
                            sc->d_items.as<MergeItem>(), sc->d_refs.as<MergeRef>(), E->d_raw.as<double2>(),
                            E->d_merged.as<double2>(), E->st));
            CK(t.stop((double)nb));
        }
        {
            KTimer t(E, FP_K_SPIRAL);
            // too few FP64 pairs to fill the SMs: the 4-CTA form (same windows, smaller parts)
            int p = pv;
            if (!fp32 && sc->cfg[2].R > 0 && sc->cfg[2].split > cfg.split &&
                (int64_t)nb * (1 << cfg.split) < (int64_t)E->sms)
                p = 2;
            const SpiralConfig &cf = sc->cfg[p];
            const bool use_win = cf.R > 0;
            CK(launch_spiral(E->d_pairs.as<PairInfo>(), (int)nb, sc->d_maps.as<SpiralMap>(), nmaps, sp.bits,
                             sp.first_bit, cf, use_win ? sc->d_wins[p].as<SpiralWin>() : nullptr,
                             use_win ? sc->nwins[p] : 0, use_win ? sc->d_ij[p].as<uint8_t>() : nullptr, sc->h[p],
                             E->d_merged.as<double2>(), E->d_maps.p, E->d_spiral_scratch.p, fp32, err_scale, tr,
                             kappa, err, E->st));
            CK(t.stop(cmac_pair * (double)nb));
            if (E->timing) E->kst.launches[FP_K_SPIRAL] += 1;   // maps + sweep
        }
        CK(cudaEventRecord(E->ev1, E->st));
        CK(cudaEventSynchronize(E->ev1));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, E->ev0, E->ev1));
        if (gpu_ms) *gpu_ms += ms;
        E->kst.pairs += nb;
        done += nb;
    }
    return FP_OK;
}

// Route pairs first + idx[i] to the brickwork or generic path.
__global__ void mark_skipped_kernel(const uint64_t *slots, uint64_t n, double *tr, double *kappa, double *err) {
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t s = slots[i];
    tr[2 * s] = tr[2 * s + 1] = NAN;
    kappa[s] = NAN;
    err[s] = NAN;
}

// Qudit brickwork pairs of one depth l: sampler, maps, sweep and meet
// (kernels_qudit.cu), in sub-batches under the workspace budget.
fp_status run_qudit(fp_ensemble *E, uint64_t first, const std::vector<uint64_t> &idx, int l, int prec, double *tr,
                    double *kappa, double *err, float *gpu_ms) {
    const fp_ensemble_desc &d = E->d;
    const uint64_t count = idx.size();
    if (count == 0) return FP_OK;
    const bool fp32 = prec != FP_PREC_FP64;
    const BrickDev bd = make_brick_plan(d.n, l, 0, 0, 0, 0).dev;
    double S = 1;
    for (int i = 0; i < bd.N; ++i) S *= d.q;
    if (S > (double)(1u << FP_MAX_STATE_BITS))
        return fail(FP_ERR_INFEASIBLE, "qudit depth %d: boundary of %d^%d amplitudes exceeds 2^%d", l, d.q, bd.N,
                    FP_MAX_STATE_BITS);
    const int n_raw = (int)layout_brickwork(d.n, l).size();
    const size_t per_pair = qudit_workspace_per_pair(d.q, bd, n_raw, fp32);
    const uint64_t cap = std::max<uint64_t>(1, std::min<uint64_t>(65535, E->ws_budget / per_pair));
    const double G = (double)std::max(bd.n_layers[0], bd.n_layers[1]) * bd.m;
    const double err_scale = FP_ERR_SAFETY * (fp32 ? 0x1.0p-24 : 0x1.0p-53) * std::sqrt(G);
    const double cmac_pair = (double)maps_per_pair(bd) * S * d.q * d.q;   // each map: S/q^2 groups of q^4
    for (uint64_t done = 0; done < count;) {
        const uint64_t nb = std::min<uint64_t>(cap, count - done);
        std::vector<PairInfo> pinfo(nb);
        for (uint64_t i = 0; i < nb; ++i) {
            std::memset(&pinfo[i], 0, sizeof(PairInfo));
            pinfo[i].pair = first + idx[done + i];
            pinfo[i].n_raw = n_raw;
            pinfo[i].out = (int64_t)idx[done + i];
        }
        CK(upload(E->d_pairs, pinfo, E->st));
        CK(E->d_states.reserve(nb * per_pair));
        CK(cudaEventRecord(E->ev0, E->st));
        {
            KTimer t(E, FP_K_BRICK);
            CK(launch_qudit(d.q, bd, d.seed, E->d_pairs.as<PairInfo>(), (int)nb, n_raw,
                            (d.flags & FP_FLAG_SELF_PAIR) ? 1 : 0, fp32, E->d_states.p, err_scale, tr, kappa, err,
                            E->st));
            CK(t.stop(cmac_pair * (double)nb, 3));
        }
        CK(cudaEventRecord(E->ev1, E->st));
        CK(cudaEventSynchronize(E->ev1));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, E->ev0, E->ev1));
        if (gpu_ms) *gpu_ms += ms;
        E->kst.pairs += nb;
        done += nb;
    }
    return FP_OK;
}

fp_status route(fp_ensemble *E, uint64_t first, const std::vector<uint64_t> &idx, const std::vector<int> &depth,
                int prec, double *tr, double *kappa, double *err, float *gpu_ms) {
    const fp_ensemble_desc &d = E->d;
    if (d.q > 2) {   // qudit brickwork: its own sweep, per depth
        std::map<int, std::vector<uint64_t>> qd;
        for (uint64_t i : idx) qd[depth[i]].push_back(i);
        for (auto it = qd.rbegin(); it != qd.rend(); ++it) {
            fp_status s = run_qudit(E, first, it->second, it->first, prec, tr, kappa, err, gpu_ms);
            if (s != FP_OK) return s;
        }
        return FP_OK;
    }
    const bool brick = (d.kind == FP_PARALLEL || d.kind == FP_HEA) && !(d.flags & FP_FLAG_GENERIC_ONLY);
    const bool spiral = d.kind == FP_HEA_PAULI && !(d.flags & (FP_FLAG_GENERIC_ONLY | FP_FLAG_HEA_CZ));
    const bool skip = (d.flags & FP_FLAG_SKIP_INFEASIBLE) != 0;
    std::map<int, std::vector<uint64_t>> by_depth, spiral_depth;
    std::vector<uint64_t> generic;
    for (uint64_t i : idx) {
        if (spiral && depth[i] >= 2 && spiral_plan(E, depth[i])) {
            spiral_depth[depth[i]].push_back(i);
            continue;
        }
        if (brick && depth[i] >= 2) {
            if (skip && 2 * (depth[i] - 1) > FP_MAX_STATE_BITS) {   // boundary of 2(l-1) segment bits
                E->skipped.push_back(i);
                continue;
            }
            by_depth[depth[i]].push_back(i);
        } else {
            generic.push_back(i);
        }
    }
    // deepest first: the largest working sets get the memory while it is free
    for (auto it = by_depth.rbegin(); it != by_depth.rend(); ++it) {
        fp_status s = run_brick(E, first, it->second, it->first, prec, tr, kappa, err, gpu_ms);
        if (s != FP_OK) return s;
    }
    for (auto it = spiral_depth.rbegin(); it != spiral_depth.rend(); ++it) {
        fp_status s = run_spiral(E, first, it->second, it->first, E->spiral_plans[it->first].get(), prec, tr, kappa,
                                 err, gpu_ms);
        if (s != FP_OK) return s;
    }
    return run_generic(E, first, generic, depth, prec, tr, kappa, err, gpu_ms);
}

// Contract pairs [first, first+count) into device arrays E->d_tr / E->d_kappa
// / E->d_err (indices relative to `first`), groups into E->d_group.
fp_status trace_device(fp_ensemble *E, uint64_t first, uint64_t count, int prec, float *gpu_ms,
                       uint64_t *requeued, double *max_kappa) {
    const fp_ensemble_desc &d = E->d;
    std::vector<int> depth(count), grp(count);
    for (uint64_t i = 0; i < count; ++i) {
        depth[i] = depth_of_pair(d, first + i);
        grp[i] = group_of_depth(d, depth[i]);
    }
    CK(E->d_tr.reserve(count * 2 * sizeof(double)));
    CK(E->d_kappa.reserve(count * sizeof(double)));
    CK(E->d_err.reserve(count * sizeof(double)));
    CK(E->d_group.reserve(count * sizeof(int32_t)));
    CK(E->d_ticket.reserve(sizeof(int) * 4));
    CK(cudaMemcpyAsync(E->d_group.p, grp.data(), count * sizeof(int32_t), cudaMemcpyHostToDevice, E->st));
    if (gpu_ms) *gpu_ms = 0;
    std::vector<uint64_t> all(count);
    std::iota(all.begin(), all.end(), 0);
    double *tr = E->d_tr.as<double>(), *kap = E->d_kappa.as<double>(), *err = E->d_err.as<double>();
    E->skipped.clear();
    fp_status s = route(E, first, all, depth, prec, tr, kap, err, gpu_ms);
    if (s != FP_OK) return s;
    std::vector<char> skipped(count, 0);
    if (!E->skipped.empty()) {
        // uncontracted pairs: NaN results, group -1 (left out of every moment)
        for (uint64_t i : E->skipped) {
            skipped[i] = 1;
            grp[i] = -1;
        }
        CK(cudaMemcpyAsync(E->d_group.p, grp.data(), count * sizeof(int32_t), cudaMemcpyHostToDevice, E->st));
        CK(upload(E->d_skip, E->skipped, E->st));
        mark_skipped_kernel<<<(unsigned)((E->skipped.size() + 255) / 256), 256, 0, E->st>>>(
            E->d_skip.as<uint64_t>(), E->skipped.size(), tr, kap, err);
        CK(cudaGetLastError());
    }
    const bool policy = prec == FP_PREC_FP32 || prec == FP_PREC_TF32X3;   // FP64 recontraction of flagged pairs
    if (policy || max_kappa) {
        std::vector<double> k(count), e(count);
        CK(cudaMemcpyAsync(k.data(), kap, count * sizeof(double), cudaMemcpyDeviceToHost, E->st));
        CK(cudaMemcpyAsync(e.data(), err, count * sizeof(double), cudaMemcpyDeviceToHost, E->st));
        CK(cudaStreamSynchronize(E->st));
        const double tol = d.fp32_tol > 0 ? d.fp32_tol : 1e-4;
        std::vector<uint64_t> redo;
        for (uint64_t i = 0; i < count; ++i) {
            if (max_kappa && std::isfinite(k[i])) *max_kappa = std::max(*max_kappa, k[i]);
            const bool over = !(e[i] <= tol) || (d.kappa_max > 0 && !(k[i] <= d.kappa_max));
            if (policy && over && !skipped[i]) redo.push_back(i);
        }
        if (!redo.empty()) {
            if (requeued) *requeued += redo.size();
            s = route(E, first, redo, depth, FP_PREC_FP64, tr, kap, err, gpu_ms);
            if (s != FP_OK) return s;
        }
    }
    return FP_OK;
}

}  // namespace

namespace fpk {
fp_status api_fail(fp_status s, const char *msg) { return fail(s, "%s", msg); }
fp_ensemble_desc ens_desc(const fp_ensemble *E) { return E->d; }
cudaStream_t ens_stream(const fp_ensemble *E) { return E->st; }
fp_status cv_trace(fp_ensemble *E, uint64_t first, uint64_t count, double **tr_dev, float *gpu_ms) {
    fp_status s = trace_device(E, first, count, FP_PREC_FP32, gpu_ms, nullptr, nullptr);
    if (s != FP_OK) return s;
    *tr_dev = E->d_tr.as<double>();
    return FP_OK;
}
}  // namespace fpk

namespace {

fp_status copy_out(fp_ensemble *E, void *dst, const void *src, size_t bytes) {
    if (!dst) return FP_OK;
    cudaMemcpyKind k = is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CK(cudaMemcpyAsync(dst, src, bytes, k, E->st));
    return FP_OK;
}

}  // namespace

extern "C" {

const char *fp_last_error(void) { return g_err.c_str(); }

fp_status fp_ensemble_create(const fp_ensemble_desc *desc, void *cuda_stream, fp_ensemble **out) {
    if (!desc || !out) return fail(FP_ERR_ARG, "null argument");
    *out = nullptr;
    const fp_ensemble_desc &d = *desc;
    if (d.kind < FP_PARALLEL || d.kind > FP_HEA_PAULI) return fail(FP_ERR_ARG, "unknown ensemble kind %d", d.kind);
    if (d.n < 2 || d.n > 64) return fail(FP_ERR_ARG, "n = %d outside [2, 64]", d.n);
    if (d.kind == FP_LOCAL) {
        if (d.T_min < 1 || d.T_max < d.T_min || d.T_step < 1)
            return fail(FP_ERR_ARG, "bad local-circuit gate counts [%d, %d] step %d", d.T_min, d.T_max, d.T_step);
    } else if (d.depth_min < 1 || d.depth_max < d.depth_min) {
        return fail(FP_ERR_ARG, "bad depth range [%d, %d]", d.depth_min, d.depth_max);
    }
    if ((d.flags & FP_FLAG_DIAGONAL_GATES) && (d.kind == FP_HEA || d.kind == FP_HEA_PAULI))
        return fail(FP_ERR_ARG, "FP_FLAG_DIAGONAL_GATES applies to Haar-gate ensembles only");
    if ((d.flags & FP_FLAG_HEA_CZ) && d.kind != FP_HEA_PAULI)
        return fail(FP_ERR_ARG, "FP_FLAG_HEA_CZ applies to FP_HEA_PAULI only");
    if (d.q != 0 && d.q != 2 && !(d.kind == FP_PARALLEL && (d.q == 3 || d.q == 4)))
        return fail(FP_ERR_ARG, "local dimension q = %d: qudits (q = 3, 4) are supported for FP_PARALLEL only", d.q);
    if (d.q > 2 && (d.flags & (FP_FLAG_DIAGONAL_GATES | FP_FLAG_GENERIC_ONLY)))
        return fail(FP_ERR_ARG, "FP_FLAG_DIAGONAL_GATES and FP_FLAG_GENERIC_ONLY apply to qubits only");
    if (d.q > 2 && d.depth_min < 2)
        return fail(FP_ERR_ARG, "qudit brickwork needs depth >= 2 (at depth 1 the trace is the product of the gates' traces)");
    std::unique_ptr<fp_ensemble> E(new fp_ensemble());
    E->d = d;
    E->st = (cudaStream_t)cuda_stream;
    CK(cudaGetDevice(&E->device));
    CK(cudaDeviceGetAttribute(&E->sms, cudaDevAttrMultiProcessorCount, E->device));
    {
        cudaDeviceProp prop;
        CK(cudaGetDeviceProperties(&prop, E->device));
        E->gpu_name = prop.name;
    }
    E->raw_kind = d.kind == FP_HEA ? RAW_ROT2
                : d.kind == FP_HEA_PAULI ? RAW_PAULI
                : ((d.flags & FP_FLAG_DIAGONAL_GATES) ? RAW_DIAG4 : RAW_HAAR4);
    E->n_groups = d.kind == FP_LOCAL ? (d.T_max - d.T_min) / d.T_step + 1 : d.depth_max - d.depth_min + 1;
    size_t freeb = 0, totb = 0;
    CK(cudaMemGetInfo(&freeb, &totb));
    // default: 32 GB (room for as many 2^24-amplitude generic-sweep slots as 16-CTA
    // clusters can be resident), at most half the free memory
    size_t cap = d.workspace_bytes ? (size_t)d.workspace_bytes : ((size_t)32 << 30);
    E->ws_budget = std::min(cap, freeb / 2);
    CK(cudaEventCreate(&E->ev0));
    CK(cudaEventCreate(&E->ev1));
    E->timing = (d.flags & FP_FLAG_TIMING) != 0;
    CK(cudaStreamCreateWithFlags(&E->gst, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&E->gev[0], cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&E->gev[1], cudaEventDisableTiming));
    for (int k = 0; k < 2 * FP_K_CLASSES; ++k) CK(cudaEventCreate(&E->kev[k]));
    *out = E.release();
    return FP_OK;
}

void fp_ensemble_destroy(fp_ensemble *ens) {
    if (!ens) return;
    if (ens->st) cudaStreamSynchronize(ens->st);
    else cudaDeviceSynchronize();
    if (ens->ev0) cudaEventDestroy(ens->ev0);
    if (ens->ev1) cudaEventDestroy(ens->ev1);
    for (int k = 0; k < 2 * FP_K_CLASSES; ++k)
        if (ens->kev[k]) cudaEventDestroy(ens->kev[k]);
    if (ens->gst) cudaStreamSynchronize(ens->gst);
    for (auto &kv : ens->graphs) if (kv.second) cudaGraphExecDestroy(kv.second);
    for (int k = 0; k < 2; ++k) if (ens->gev[k]) cudaEventDestroy(ens->gev[k]);
    if (ens->gst) cudaStreamDestroy(ens->gst);
    delete ens;
}

fp_status fp_groups(const fp_ensemble *ens, int32_t *n_groups, int32_t *values) {
    if (!ens || !n_groups) return fail(FP_ERR_ARG, "null argument");
    *n_groups = ens->n_groups;
    if (values)
        for (int g = 0; g < ens->n_groups; ++g)
            values[g] = ens->d.kind == FP_LOCAL ? ens->d.T_min + g * ens->d.T_step : ens->d.depth_min + g;
    return FP_OK;
}

fp_status fp_pair_groups(const fp_ensemble *ens, uint64_t first, uint64_t count, int32_t *group) {
    if (!ens || (!group && count)) return fail(FP_ERR_ARG, "null argument");
    for (uint64_t i = 0; i < count; ++i) group[i] = group_of_depth(ens->d, depth_of_pair(ens->d, first + i));
    return FP_OK;
}

fp_status fp_export_gates(fp_ensemble *ens, uint64_t pair, int32_t which, void *host_buf, size_t *bytes) {
    if (!ens || !bytes || (which != 0 && which != 1)) return fail(FP_ERR_ARG, "bad argument");
    const fp_ensemble_desc &d = ens->d;
    if (d.q > 2) return fail(FP_ERR_ARG, "gates of qudit ensembles are not exported (records hold 4x4 matrices)");
    int depth = depth_of_pair(d, pair);
    int n_raw = 0;
    std::vector<GateSlot> lay = circuit_layout(d, pair, which, depth, &n_raw);
    struct Rec { int32_t kind, q; double m[32]; };
    size_t need = lay.size() * sizeof(Rec);
    if (!host_buf) { *bytes = need; return FP_OK; }
    if (*bytes < need) { *bytes = need; return fail(FP_ERR_ARG, "buffer too small: need %zu bytes", need); }
    *bytes = need;
    PairInfo pi;
    pi.pair = pair; pi.plan = 0; pi.n_raw = n_raw; pi.raw_off = 0; pi.merged_off = 0; pi.table_off = 0;
    CK(upload(ens->d_pairs, std::vector<PairInfo>{pi}, ens->st));
    CK(ens->d_raw.reserve((size_t)2 * n_raw * 16 * sizeof(double2)));
    SampleParams sp;
    sp.seed = d.seed; sp.n = d.n; sp.raw_kind = ens->raw_kind; sp.self_pair = (d.flags & FP_FLAG_SELF_PAIR) ? 1 : 0;
    CK(launch_sample(sp, ens->d_pairs.as<PairInfo>(), 1, n_raw, ens->d_raw.as<double2>(), ens->st));
    std::vector<double2> raw((size_t)2 * n_raw * 16);
    CK(cudaMemcpyAsync(raw.data(), ens->d_raw.p, raw.size() * sizeof(double2), cudaMemcpyDeviceToHost, ens->st));
    CK(cudaStreamSynchronize(ens->st));
    Rec *out = (Rec *)host_buf;
    for (size_t i = 0; i < lay.size(); ++i) {
        std::memset(&out[i], 0, sizeof(Rec));
        out[i].q = lay[i].q;
        if (lay[i].kind == 2) {
            out[i].kind = 2;
            double dg[4] = {1, 1, 1, -1};
            for (int k = 0; k < 4; ++k) out[i].m[2 * k] = dg[k];
            continue;
        }
        out[i].kind = lay[i].kind == 3 ? 1 : lay[i].kind;
        const double2 *g = &raw[((size_t)which * n_raw + lay[i].raw) * 16];
        for (int k = 0; k < 16; ++k) { out[i].m[2 * k] = g[k].x; out[i].m[2 * k + 1] = g[k].y; }
    }
    return FP_OK;
}

fp_status fp_trace_batch(fp_ensemble *ens, uint64_t first, uint64_t count, int32_t prec, double *tr,
                         double *kappa, double *err, int32_t *group) {
    if (!ens || (!tr && count)) return fail(FP_ERR_ARG, "null argument");
    if (prec < FP_PREC_FP64 || prec > FP_PREC_TF32X3) return fail(FP_ERR_ARG, "unknown precision %d", prec);
    if (count == 0) return FP_OK;
    fp_status s = trace_device(ens, first, count, prec, nullptr, nullptr, nullptr);
    if (s != FP_OK) return s;
    if ((s = copy_out(ens, tr, ens->d_tr.p, count * 2 * sizeof(double))) != FP_OK) return s;
    if ((s = copy_out(ens, kappa, ens->d_kappa.p, count * sizeof(double))) != FP_OK) return s;
    if ((s = copy_out(ens, err, ens->d_err.p, count * sizeof(double))) != FP_OK) return s;
    if ((s = copy_out(ens, group, ens->d_group.p, count * sizeof(int32_t))) != FP_OK) return s;
    CK(cudaStreamSynchronize(ens->st));
    return FP_OK;
}

fp_status fp_reduce_moments(fp_ensemble *ens, const double *tr, const int32_t *group, uint64_t count,
                            int32_t k_max, double *moments) {
    if (!ens || !tr || !moments) return fail(FP_ERR_ARG, "null argument");
    if (k_max < 1 || k_max > FP_MAX_KMAX) return fail(FP_ERR_ARG, "k_max = %d outside [1, %d]", k_max, FP_MAX_KMAX);
    if (!is_device_ptr(tr) || (group && !is_device_ptr(group)))
        return fail(FP_ERR_ARG, "tr and group must be device pointers");
    int ng = group ? ens->n_groups : 1, nb = moments_blocks(count), nv = 2 * k_max + 1;
    CK(ens->d_partials.reserve((size_t)nb * ng * nv * sizeof(double)));
    CK(ens->d_moments.reserve((size_t)ng * nv * sizeof(double)));
    {
        KTimer t(ens, FP_K_MOMENTS);
        CK(launch_moments(tr, group, count, k_max, ng, ens->d_partials.as<double>(), nb, ens->d_moments.as<double>(), ens->st));
        CK(t.stop((double)count));
    }
    fp_status s = copy_out(ens, moments, ens->d_moments.p, (size_t)ng * nv * sizeof(double));
    if (s != FP_OK) return s;
    CK(cudaStreamSynchronize(ens->st));
    return FP_OK;
}

fp_status fp_bootstrap(fp_ensemble *ens, const double *tr, const int32_t *group, uint64_t count, int32_t k_max,
                       int32_t n_resamples, uint64_t seed, double *F_boot) {
    if (!ens || !tr || !group || !F_boot) return fail(FP_ERR_ARG, "null argument");
    if (k_max < 1 || k_max > FP_MAX_KMAX) return fail(FP_ERR_ARG, "k_max = %d outside [1, %d]", k_max, FP_MAX_KMAX);
    if (n_resamples < 1) return fail(FP_ERR_ARG, "n_resamples = %d must be positive", n_resamples);
    if (count >= (1ull << 32)) return fail(FP_ERR_ARG, "count must be below 2^32");
    const int ng = ens->n_groups;
    // group lists in increasing pair order (a stable counting sort on the host)
    std::vector<int32_t> hg(count);
    if (count) CK(cudaMemcpyAsync(hg.data(), group, count * sizeof(int32_t), cudaMemcpyDefault, ens->st));
    CK(cudaStreamSynchronize(ens->st));
    std::vector<uint64_t> off(ng + 1, 0);
    for (uint64_t i = 0; i < count; ++i)
        if (hg[i] >= 0 && hg[i] < ng) ++off[hg[i] + 1];
    for (int g = 0; g < ng; ++g) off[g + 1] += off[g];
    std::vector<uint32_t> members(std::max<uint64_t>(off[ng], 1));
    {
        std::vector<uint64_t> pos(off.begin(), off.end() - 1);
        for (uint64_t i = 0; i < count; ++i)
            if (hg[i] >= 0 && hg[i] < ng) members[pos[hg[i]]++] = (uint32_t)i;
    }
    const double *dtr = tr;
    if (!is_device_ptr(tr)) {
        CK(ens->d_boot_tr.reserve(std::max<uint64_t>(count, 1) * 2 * sizeof(double)));
        if (count) CK(cudaMemcpyAsync(ens->d_boot_tr.p, tr, count * 2 * sizeof(double), cudaMemcpyHostToDevice, ens->st));
        dtr = ens->d_boot_tr.as<double>();
    }
    CK(upload(ens->d_boot_members, members, ens->st));
    CK(upload(ens->d_boot_off, off, ens->st));
    CK(ens->d_boot_xs.reserve(members.size() * sizeof(double)));
    const size_t nout = (size_t)ng * k_max * n_resamples;
    CK(ens->d_boot_out.reserve(nout * sizeof(double)));
    {
        KTimer t(ens, FP_K_BOOTSTRAP);
        CK(launch_bootstrap(dtr, ens->d_boot_members.as<uint32_t>(), off[ng], ens->d_boot_off.as<uint64_t>(), ng, k_max,
                            n_resamples, seed, ens->d_boot_xs.as<double>(), ens->d_boot_out.as<double>(), ens->st));
        CK(t.stop((double)off[ng] * n_resamples));
    }
    fp_status s = copy_out(ens, F_boot, ens->d_boot_out.p, nout * sizeof(double));
    if (s != FP_OK) return s;
    CK(cudaStreamSynchronize(ens->st));
    return FP_OK;
}

fp_status fp_frame_potential_resume(fp_ensemble *ens, fp_checkpoint *ck, uint64_t max_pairs, uint64_t max_batches,
                                    int32_t k_max, double target_rel_stderr, int32_t prec, double *F,
                                    double *stderr_) {
    if (!ens || !ck || !ck->sums || !F || !stderr_) return fail(FP_ERR_ARG, "null argument");
    if (k_max < 1 || k_max > FP_MAX_KMAX) return fail(FP_ERR_ARG, "k_max = %d outside [1, %d]", k_max, FP_MAX_KMAX);
    if (prec < FP_PREC_FP64 || prec > FP_PREC_TF32X3) return fail(FP_ERR_ARG, "unknown precision %d", prec);
    const int ng = ens->n_groups, nv = 2 * k_max + 1;
    if (ck->next_batch == 0) {   // first call of a run
        ck->k_max = k_max;
        ck->n_groups = ng;
        ck->pairs_done = 0;
        std::memset(&ck->stats, 0, sizeof ck->stats);
        // with a target: batches from 4096 pairs, doubling, so the stop can come early;
        // without one: batches as large as the workspace allows
        ck->next_batch = target_rel_stderr > 0 ? 4096 : (1u << 20);
    } else if (ck->k_max != k_max || ck->n_groups != ng) {
        return fail(FP_ERR_ARG, "checkpoint of k_max = %d, %d groups resumed with k_max = %d, %d groups", ck->k_max,
                    ck->n_groups, k_max, ng);
    }
    double *acc = ck->sums, *comp = ck->sums + (size_t)ng * nv;
    std::vector<double> part((size_t)ng * nv);
    fp_run_stats &st = ck->stats;
    st.n_groups = ng;
    const int kt = k_max >= 2 ? 2 : 1;
    auto estimate = [&]() {   // F, stderr from the sums; whether every group met the target
        bool ok = target_rel_stderr > 0;
        for (int g = 0; g < ng; ++g) {
            double N = acc[g * nv] + comp[g * nv];
            for (int k = 1; k <= k_max; ++k) {
                double S = acc[g * nv + k] + comp[g * nv + k];
                double Q = acc[g * nv + k_max + k] + comp[g * nv + k_max + k];
                double mean = N > 0 ? S / N : NAN;
                double var = N > 1 ? std::max(0.0, (Q - S * S / N) / (N - 1)) : NAN;
                F[g * k_max + k - 1] = mean;
                stderr_[g * k_max + k - 1] = N > 1 ? std::sqrt(var / N) : NAN;
            }
            double f = F[g * k_max + kt - 1], e = stderr_[g * k_max + kt - 1];
            if (!(N > 1 && f > 0 && e / f <= target_rel_stderr)) ok = false;
        }
        return ok;
    };
    bool reached = ck->pairs_done > 0 && estimate();
    for (uint64_t nbatches = 0; ck->pairs_done < max_pairs && !reached && (max_batches == 0 || nbatches < max_batches);
         ++nbatches) {
        if (ens->cancel.exchange(0)) {
            estimate();
            return fail(FP_ERR_CANCELLED, "cancelled before the batch at pair %llu (the checkpoint can be resumed)",
                        (unsigned long long)ck->next_pair);
        }
        uint64_t nb = std::min<uint64_t>(ck->next_batch, max_pairs - ck->pairs_done);
        float ms = 0;
        uint64_t recon = 0;
        double mk = 0;
        fp_status s = trace_device(ens, ck->next_pair, nb, prec, &ms, &recon, &mk);
        if (s != FP_OK) return s;
        int nb_blocks = moments_blocks(nb);
        CK(ens->d_partials.reserve((size_t)nb_blocks * ng * nv * sizeof(double)));
        CK(ens->d_moments.reserve((size_t)ng * nv * sizeof(double)));
        {
            KTimer t(ens, FP_K_MOMENTS);
            CK(launch_moments(ens->d_tr.as<double>(), ens->d_group.as<int32_t>(), nb, k_max, ng,
                              ens->d_partials.as<double>(), nb_blocks, ens->d_moments.as<double>(), ens->st));
            CK(t.stop((double)nb));
        }
        CK(cudaMemcpyAsync(part.data(), ens->d_moments.p, part.size() * sizeof(double), cudaMemcpyDeviceToHost, ens->st));
        CK(cudaStreamSynchronize(ens->st));
        // the batch is complete: fold it into the checkpoint
        for (size_t i = 0; i < part.size(); ++i) {   // Neumaier accumulation across batches
            double y = acc[i] + part[i];
            comp[i] += std::fabs(acc[i]) >= std::fabs(part[i]) ? (acc[i] - y) + part[i] : (part[i] - y) + acc[i];
            acc[i] = y;
        }
        st.fp64_recontracted += recon;
        st.max_kappa = std::max(st.max_kappa, mk);
        st.infeasible += ens->skipped.size();
        st.gpu_seconds += ms * 1e-3;
        ck->pairs_done += nb;
        ck->next_pair += nb;
        st.pairs = ck->pairs_done - st.infeasible;
        if (ck->next_batch < (1u << 20)) ck->next_batch *= 2;
        reached = estimate();
    }
    if (ck->pairs_done == 0) estimate();
    st.reached_target = reached ? 1 : 0;
    return FP_OK;
}

fp_status fp_frame_potential(fp_ensemble *ens, uint64_t first, uint64_t max_pairs, int32_t k_max,
                             double target_rel_stderr, int32_t prec, double *F, double *stderr_,
                             fp_run_stats *stats) {
    if (!ens || !F || !stderr_) return fail(FP_ERR_ARG, "null argument");
    if (k_max < 1 || k_max > FP_MAX_KMAX) return fail(FP_ERR_ARG, "k_max = %d outside [1, %d]", k_max, FP_MAX_KMAX);
    std::vector<double> sums((size_t)2 * ens->n_groups * (2 * k_max + 1), 0.0);
    fp_checkpoint ck;
    std::memset(&ck, 0, sizeof ck);
    ck.next_pair = first;
    ck.sums = sums.data();
    fp_status s = fp_frame_potential_resume(ens, &ck, max_pairs, 0, k_max, target_rel_stderr, prec, F, stderr_);
    if (s == FP_OK && stats) *stats = ck.stats;
    return s;
}

fp_status fp_cancel(fp_ensemble *ens) {
    if (!ens) return fail(FP_ERR_ARG, "null argument");
    ens->cancel.store(1);
    return FP_OK;
}

fp_status fp_inject_alloc_failures(int32_t count) {
    if (count < 0) return fail(FP_ERR_ARG, "count < 0");
    g_alloc_failures.store(count);
    return FP_OK;
}

fp_status fp_set_wait_limit_ns(uint64_t ns) {
    g_wait_ns.store(ns ? ns : 1000000000ull);
    return FP_OK;
}

fp_status fp_brick_variant(const fp_ensemble *ens, int32_t depth, int32_t precision, int32_t *out) {
    if (!ens || !out) return fail(FP_ERR_ARG, "null argument");
    if (precision < FP_PREC_FP64 || precision > FP_PREC_TF32X3) return fail(FP_ERR_ARG, "unknown precision %d", precision);
    auto it = ens->brick_plans.find(brick_key(depth, precision));
    if (it == ens->brick_plans.end())
        return fail(FP_ERR_ARG, "no brickwork sweep of depth %d at this precision has run on this ensemble", depth);
    for (int i = 0; i < 4; ++i) out[i] = it->second->variant[i];
    return FP_OK;
}

fp_status fp_kernel_stats_get(fp_ensemble *ens, fp_kernel_stats *out, int32_t reset) {
    if (!ens || !out) return fail(FP_ERR_ARG, "null argument");
    *out = ens->kst;
    out->graph_replays = ens->graph_replays;
    if (reset) {
        std::memset(&ens->kst, 0, sizeof ens->kst);
        ens->graph_replays = 0;
    }
    return FP_OK;
}

}  // extern "C"
