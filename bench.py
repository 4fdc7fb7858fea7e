#!/usr/bin/env python
"""Throughput of Tr(U^dagger V) contractions at n = 50 on one or more GB300s.

Workload: brickwork ("parallel") random circuits, n = 50 qubits on an open
chain, depth l drawn uniformly from 2..10 per pair, Haar U(4) gates,
100,000 pairs per step (a fresh range of pair indices every step).
One step is the whole hot path over one batch: gate sampling, merging,
factor tables, both boundary sweeps, the FP64 meet, and the FP64 moments of
|Tr|^{2k}, k = 1..4, per depth group.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Prints one JSON line (rank 0).  `value` is device-timed (CUDA events on the
library's stream); `e2e` is the same metric through fp_frame_potential, the
call a user makes, with results returned to host memory.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Tr(U^dagger V) contractions/s at n=50 (brickwork, l=2..10)"
WORK = dict(n=50, depth_min=2, depth_max=10, pairs=100_000, seed=4, k_max=4, kind=0, name="brickwork")
# other workloads (parity-test configurations, measurable with --workload)
WORKLOADS = {
    "brickwork": dict(WORK),
    "hea": dict(n=50, depth_min=1, depth_max=8, pairs=1_000_000, seed=3, k_max=4, kind=2, name="hea"),
    # the paper's own HEA: RY(pi/4) wall, random Pauli rotations, CNOT walls on even then odd bonds
    "hea_paper": dict(n=50, depth_min=1, depth_max=8, pairs=100_000, seed=6, k_max=4, kind=3,
                      name="hea_paper"),
    # local random circuits: n = 20, T in {20, 40, ..., 100} gates per circuit (T >= 120 is
    # reported separately: its boundaries reach the 2^24 limit, see local_large_T_report)
    "local": dict(n=20, depth_min=1, depth_max=1, T=(20, 100, 20), pairs=20_000, seed=2, k_max=4, kind=1,
                  name="local"),
}
SM_COUNT, FP32_LANES = 152, 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--pairs", type=int, default=WORK["pairs"])
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workspace-gb", type=float, default=0.0,
                    help="device workspace cap of the ensemble (0: the library default)")
    ap.add_argument("--no-target", action="store_true",
                    help="skip the GPU-seconds-to-1%% measurement, the bootstrap report and the large-T report")
    ap.add_argument("--no-cv", action="store_true", help="skip the control-variate report")
    ap.add_argument("--workload", default="brickwork", choices=sorted(WORKLOADS),
                    help="brickwork (the headline workload), hea (n=50, L=1..8), hea_paper (n=50, L=1..8) "
                         "or local (n=20, T=20..100)")
    ap.add_argument("--depth", type=int, default=0,
                    help="run one depth group only (l or L; profiling runs of a single tile-pass shape)")
    a = ap.parse_args()
    WORK.update(WORKLOADS[a.workload])
    if a.pairs == 100_000 and a.workload != "brickwork":
        a.pairs = WORK["pairs"]
    if a.depth:
        WORK["depth_min"] = WORK["depth_max"] = a.depth
    if a.workspace_gb:
        WORK["workspace_gb"] = a.workspace_gb
    return a


def make_ensemble(fp, flags=0, stream=None):
    T = WORK.get("T", (0, 0, 1))
    if WORK["name"] == "local":
        flags |= fp.FLAG_SKIP_INFEASIBLE   # rare pairs beyond the 2^24 boundary are counted, not contracted
    ws = int(WORK.get("workspace_gb", 0) * (1 << 30))
    return fp.Ensemble(WORK["kind"], WORK["n"], WORK["depth_min"], WORK["depth_max"], T[0], T[1], T[2],
                       seed=WORK["seed"], flags=flags, workspace_bytes=ws, stream=stream)


def workload_config(args, world):
    desc = {"brickwork": "brickwork n=50, l uniform in 2..10 per pair, Haar U(4)",
            "hea": "HEA n=50, L uniform in 1..8 per pair, RY(theta)RZ(phi) + CZ ladder",
            "hea_paper": "paper HEA n=50, L uniform in 1..8 per pair, RY(pi/4) wall, random Pauli rotations, "
                         "CNOT walls on even then odd bonds",
            "local": "local random circuits n=20, T uniform in {20,40,...,100} Haar U(4) gates on uniformly "
                     "random neighbour bonds per circuit"}[WORK["name"]]
    if args.depth:
        desc += f" (single depth {args.depth} only)"
    return {"workload": f"{desc}, {args.pairs} pairs per step per GPU",
            "n": WORK["n"], "depth": list(WORK["T"]) if "T" in WORK else [WORK["depth_min"], WORK["depth_max"]],
            "pairs_per_step": args.pairs,
            "k_max": WORK["k_max"], "precision": args.prec, "parallelism": f"pairs sharded over {world} GPU(s)",
            "l2": "per-step device working set (sampled gates, tables, boundaries) is GBs, larger than L2"}


# ---------------------------------------------------------------------------
# CPU oracle (reported baseline; the only use of oracle/ in this file)
# ---------------------------------------------------------------------------
def oracle_sample(first_pair, cores, max_depth=8):
    """Pairs of the workload in index order, skipping those deeper than max_depth
    (the oracle needs ~30 s for l = 9 and minutes for l = 10 at n = 50)."""
    import oracle as O
    d = O.desc(O.PARALLEL, WORK["n"], WORK["depth_min"], WORK["depth_max"], seed=WORK["seed"])
    pairs, p = [], first_pair
    while len(pairs) < 2 * cores:
        if O.pair_depth(d, p) <= max_depth:
            pairs.append(p)
        p += 1
    return d, pairs


def oracle_time(first_pair, cores):
    import numpy as np
    import oracle as O
    d, pairs = oracle_sample(first_pair, cores)
    # one pair per thread: contiguous runs are not guaranteed, so time each pair range
    t0 = time.perf_counter()
    import concurrent.futures as cf
    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        list(ex.map(lambda p: O.trace_batch(d, p, 1, "ve", threads=1), pairs))
    dt = time.perf_counter() - t0
    depths = [O.pair_depth(d, p) for p in pairs]
    return len(pairs) / dt, dt, len(pairs), depths


def cpu_baseline_obj(rate, cores, npairs, depths):
    return {"value": rate, "unit": "contractions/s", "cores": cores, "kind": "oracle",
            "sample": f"{npairs} pairs of the workload in index order with l<=8 (depths "
                      f"{min(depths)}..{max(depths)}), one pair per thread, FP64 variable elimination; "
                      "pairs with l=9,10 left out (the oracle needs ~30 s and minutes per such pair)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    first = 10_000_000
    for _ in range(args.warmup):
        oracle_time(first, cores)
        first += 4 * cores
    rates, times, last = [], [], None
    for _ in range(args.steps):
        r, dt, npairs, depths = oracle_time(first, cores)
        first += 4 * cores
        rates.append(r)
        times.append(dt)
        last = (npairs, depths)
    value = args.steps / sum(t / (last[0]) for t in times) if times else 0.0
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "contractions/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded circuit pairs)",
            "config": workload_config(args, args.gpus),
            "cpu_baseline": cpu_baseline_obj(value, cores, last[0], last[1]),
            "e2e": {"value": value, "unit": "contractions/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU-seconds to F^(2) at 1% relative standard error, mixed vs plain FP64
# ---------------------------------------------------------------------------
def moments_report(mom, groups, K):
    """F^(k) and its standard error per group from fp_reduce_moments output."""
    out = {}
    for g, depth in enumerate(groups):
        row = mom[g * (2 * K + 1):(g + 1) * (2 * K + 1)]
        N = row[0]
        if N < 2:
            continue
        F = [row[k] / N for k in range(1, K + 1)]
        se = [math.sqrt(max(row[K + k] / N - F[k - 1] ** 2, 0.0) * N / (N - 1) / N) for k in range(1, K + 1)]
        out[str(int(depth))] = {"pairs": int(N), "F": F, "stderr": se}
    return out


def per_pair_cost(fp, l, prec, count, first):
    """Device seconds per pair of depth l (all kernels of the trace path)."""
    ens = fp.Ensemble(fp.PARALLEL, WORK["n"], l, l, seed=WORK["seed"], flags=fp.FLAG_TIMING)
    ens.trace_batch(first, min(count, 64), prec)             # plans, autotuning, warm caches
    ens.kernel_stats(reset=True)
    ens.trace_batch(first + 64, count, prec)
    ks = ens.kernel_stats(reset=True)
    ens.close()
    return sum(ks.ms[i] for i in range(8)) / 1e3 / count


def gpu_seconds_to_target(fp, mom, P, K, ng, rel=0.01):
    """N_g pairs per depth group for rel. stderr of F^(2) <= rel, from the moments of
    the last timed step; GPU-s = sum_g N_g x measured per-pair device time of depth g,
    for the FP32 (mixed) and FP64 paths; plus an actual adaptive run on the mixed path."""
    m = mom.cpu().numpy().reshape(ng, 2 * K + 1)
    out = {"target_rel_stderr": rel, "groups": {}}
    tot32 = tot64 = 0.0
    for g in range(ng):
        l = WORK["depth_min"] + g
        N, S2, Q2 = m[g, 0], m[g, 2], m[g, K + 2]
        F2 = S2 / N
        var = (Q2 - S2 * S2 / N) / (N - 1)
        need = var / (rel * F2) ** 2
        c32 = per_pair_cost(fp, l, fp.PREC_FP32, 2000 if l >= 9 else 4000, 50_000_000)
        c64 = per_pair_cost(fp, l, fp.PREC_FP64, 32 if l >= 10 else (64 if l == 9 else 256), 60_000_000)
        out["groups"][str(l)] = {"F2": F2, "pairs_needed": need, "s_per_pair_fp32": c32, "s_per_pair_fp64": c64}
        tot32 += need * c32
        tot64 += need * c64
    out["gpu_s_mixed_fp32"] = tot32
    out["gpu_s_plain_fp64"] = tot64
    out["speedup"] = tot64 / tot32 if tot32 > 0 else None
    out["method"] = ("pairs_needed from the variance of |Tr|^4 per depth group (last timed step); per-pair "
                     "device seconds measured per depth with CUDA events; GPU-s = sum over groups")
    ens = fp.Ensemble(fp.PARALLEL, WORK["n"], WORK["depth_min"], WORK["depth_max"], seed=WORK["seed"])
    F, se, st = ens.frame_potential(70_000_000, 3_000_000, 2, rel, fp.PREC_FP32)
    ens.close()
    out["mixed_run"] = {"pairs": int(st.pairs), "gpu_seconds": st.gpu_seconds, "reached": bool(st.reached_target),
                        "fp64_recontracted": int(st.fp64_recontracted),
                        "F2_by_depth": {str(WORK["depth_min"] + g): [float(F[g, 1]), float(se[g, 1])] for g in range(ng)}}
    return out


# ---------------------------------------------------------------------------
# learned control variate for HEA F^(2) (L = 4..6) against the plain estimator
# ---------------------------------------------------------------------------
def control_variate_report(fp, n_train=100_000, n_correct=10_000, m_surrogate=10_000_000):
    out = {}
    for L in (4, 5, 6):
        ens = fp.Ensemble(fp.HEA, 50, L, L, seed=50 + L)
        r = ens.cv_frame_potential(0, n_train, n_correct, m_surrogate)
        # plain estimator: per-pair device cost on this depth, pairs needed for the CV's stderr
        ens_t = fp.Ensemble(fp.HEA, 50, L, L, seed=50 + L, flags=fp.FLAG_TIMING)
        ens_t.trace_batch(90_000_000, 4096, fp.PREC_FP32)
        ens_t.kernel_stats(reset=True)
        ens_t.trace_batch(91_000_000, 100_000, fp.PREC_FP32)
        ks = ens_t.kernel_stats(reset=True)
        c_pair = sum(ks.ms[i] for i in range(8)) / 1e3 / 100_000
        ens_t.close()
        ens.close()
        cv_s = r.gpu_seconds_exact + r.gpu_seconds_train + r.gpu_seconds_surrogate
        plain_pairs = r.var_f / r.stderr_ ** 2
        # MLP work of the surrogate phase (correction + surrogate evaluations), algorithmic FLOPs
        D, H = 4 * 50 * L, 256
        mlp_flop = 2.0 * (D * H + 2 * H * H + H) * (n_correct + m_surrogate)
        out[str(L)] = {"F2_cv": r.F2, "stderr_cv": r.stderr_, "F2_plain_on_corrections": r.F2_plain,
                       "stderr_plain_on_corrections": r.stderr_plain,
                       "variance_reduction": r.var_f / r.var_f_minus_g if r.var_f_minus_g > 0 else None,
                       "gpu_s_cv": cv_s, "gpu_s_exact": r.gpu_seconds_exact, "gpu_s_train": r.gpu_seconds_train,
                       "gpu_s_surrogate": r.gpu_seconds_surrogate,
                       "surrogate_phase_mlp_tflops": mlp_flop / r.gpu_seconds_surrogate / 1e12,
                       "gpu_s_plain_same_stderr": plain_pairs * c_pair,
                       "train_loss": r.train_loss}
    return {"config": f"HEA n=50, L=4..6, {n_train} training pairs, {m_surrogate} surrogate evaluations, "
                      f"{n_correct} exact corrections; MLP 4nL-256-256-256-1 GELU, Adam; hidden layers "
                      f"as BF16 tcgen05 GEMMs with FP32 accumulation",
            "by_depth": out}


def bootstrap_report(fp, pairs=200_000, B=300):
    """The paper's uncertainty analysis at n = 50 (brickwork, l = 2..10): traces of
    `pairs` pairs, B bootstrap resamples of F^(k) per depth on the GPU, then per
    resample the exponential fit of F - k! over depth and the layers for a
    0.1-approximate k-design; medians and 5-95 % ranges of the bootstrap."""
    import numpy as np
    import torch
    ens = fp.Ensemble(0, 50, 2, 10, seed=WORK["seed"] + 1000, flags=fp.FLAG_TIMING)
    tr = torch.empty(2 * pairs, dtype=torch.float64, device="cuda")
    grp = torch.empty(pairs, dtype=torch.int32, device="cuda")
    ens.trace_batch(0, pairs, fp.PREC_FP32, tr, None, grp)
    ens.kernel_stats(reset=True)
    K = 4
    Fb = ens.bootstrap(tr, grp, pairs, K, B, seed=7)           # [9 depths, K, B]
    ks = ens.kernel_stats(reset=True)
    ens.close()
    depths = np.arange(2, 11)
    pct = lambda v: [float(np.nanpercentile(v, q)) for q in (5, 50, 95)]
    out = {"pairs": pairs, "resamples": B, "bootstrap_gpu_ms": ks.ms[fp.K_BOOTSTRAP],
           "F2_by_depth_p5_p50_p95": {int(l): pct(Fb[i, 1]) for i, l in enumerate(depths)},
           "log10_eps_max_k2_median": {int(l): fp.epsilon_max_log10(float(np.median(Fb[i, 1])), 2, 50)
                                       for i, l in enumerate(depths)}}
    for k in (2, 3, 4):
        ls = np.array([fp.design_layers(depths, Fb[:, k - 1, b], k, 50)[0] for b in range(B)])
        ok = np.isfinite(ls)
        out[f"layers_eps0.1_k{k}"] = {"p5_p50_p95": pct(ls[ok]) if ok.any() else None,
                                      "fits_converged": int(ok.sum())}
    return out


def exact_fk_report(fp, mc=None):
    """Exact ensemble F^(2) (l = 2..10) and F^(3) (l = 2..6) of the n = 50 brickwork
    ensemble by the Weingarten transfer-matrix sweep on the GPU, with the time of
    each call, and the Monte Carlo F^(2) of the adaptive run beside it (z-score)."""
    out = {"F2": {}, "F3": {}}
    for k, depths in ((2, range(2, 11)), (3, range(2, 7))):
        for l in depths:
            t0 = time.perf_counter()
            f = fp.exact_brickwork_fk(WORK["n"], l, k)
            row = {"exact": f, "seconds": time.perf_counter() - t0}
            if k == 2 and mc and str(l) in mc:
                F, se = mc[str(l)]
                row["monte_carlo"] = [F, se]
                row["z"] = (F - f) / se if se > 0 else None
            out[f"F{k}"][str(l)] = row
    out["F2_qutrits"] = {str(l): fp.exact_brickwork_fk(WORK["n"], l, 2, q=3) for l in range(2, 11)}
    out["note"] = ("variance-free reference: Haar average of every gate as a sum over S_k pairings with U(4) "
                   "Weingarten weights, summed by an FP64 transfer-matrix sweep over the bonds; Monte Carlo "
                   "z-scores use the naive standard error, unreliable for the heavy tails at l <= 4; "
                   "F2_qutrits: the same for qudits of local dimension 3 (Haar U(9) gates)")
    return out


def local_large_T_report(fp, per_T=12):
    """Local circuits with T >= 120 gates (n = 20): per T, the fraction of sampled pairs
    whose boundary fits the 2^24-amplitude limit, and the device time per feasible pair
    (one pair per call, FP32 policy)."""
    import numpy as np
    out = {}
    for T in (120, 140, 160, 180, 200):
        ens = fp.Ensemble(1, 20, 1, 1, T, T, 1, seed=WORK["seed"] + T, flags=fp.FLAG_TIMING)
        feas, ms = 0, 0.0
        for p in range(per_T):
            ens.kernel_stats(reset=True)
            try:
                ens.trace_batch(p, 1, fp.PREC_FP32)
            except fp.FpError as e:
                if e.status != -5:
                    raise
                continue
            feas += 1
            ks = ens.kernel_stats(reset=True)
            ms += sum(ks.ms[i] for i in range(8))
        ens.close()
        out[str(T)] = {"sampled": per_T, "feasible": feas,
                       "gpu_ms_per_feasible_pair": ms / feas if feas else None}
    return {"note": "pairs whose boundary exceeds 2^24 amplitudes return FP_ERR_INFEASIBLE; a cluster "
                    "of 16 CTAs contracts each large pair on the generic path", "by_T": out}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", delete=False, suffix=".csv")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2205_09900_gb300 import build as fpbuild
    if rank == 0 or not os.path.exists(os.path.join(ROOT, "paper_2205_09900_gb300", "libfp_gb300.so")):
        fpbuild.build()
    if dist:
        dist.barrier()
    import paper_2205_09900_gb300 as fp

    prec = fp.PREC_FP32 if args.prec == "fp32" else fp.PREC_FP64
    stream = torch.cuda.current_stream()
    P, K = args.pairs, WORK["k_max"]
    ens = make_ensemble(fp, fp.FLAG_TIMING, stream.cuda_stream)
    ng = len(ens.groups())
    tr = torch.empty(2 * P, dtype=torch.float64, device="cuda")
    kap = torch.empty(P, dtype=torch.float64, device="cuda")
    err = torch.empty(P, dtype=torch.float64, device="cuda")
    grp = torch.empty(P, dtype=torch.int32, device="cuda")
    mom = torch.empty(ng * (2 * K + 1), dtype=torch.float64, device="cuda")

    from paper_2205_09900_gb300.shard import max_over_ranks, pair_range

    def first_of(step):
        return pair_range(step, rank, world, P)[0]

    skipped = torch.zeros((), dtype=torch.int64, device="cuda")

    def step(s):
        ens.trace_batch(first_of(s), P, prec, tr, kap, grp, err)
        ens.reduce_moments(tr, grp, P, K, mom)
        if WORK["name"] == "local":
            skipped.add_((grp < 0).sum())

    for s in range(args.warmup):
        step(s)
    torch.cuda.synchronize()
    skipped.zero_()
    ens.kernel_stats(reset=True)

    clk = Clocks(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s in range(args.warmup, args.warmup + args.steps):
        step(s)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, device="cuda")
    if dist:
        dist.barrier()
    ks = ens.kernel_stats(reset=True)
    launches = int(sum(ks.launches[i] for i in range(8)))

    # e2e: the public Monte Carlo call, results to host memory, host wall clock
    e2e = None
    if not args.no_e2e:
        # a user's ensemble: no per-kernel timing, so sub-batches replay CUDA graphs
        ens_u = make_ensemble(fp, 0, stream.cuda_stream)
        ens_u.frame_potential(first_of(args.warmup + args.steps), P, K, 0.0, prec)   # warm
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        contracted = 0
        for s in range(args.steps):
            _, _, rst = ens_u.frame_potential(first_of(args.warmup + args.steps + 1 + s), P, K, 0.0, prec)
            contracted += rst.pairs
        dt = time.perf_counter() - t0
        replays = int(ens_u.kernel_stats().graph_replays)
        ens_u.close()
        # host->device per step: PairInfo (40 B) + order (4 B) + group (4 B) per pair;
        # device->host: kappa (8 B/pair, FP32 policy) + per-batch moments
        batches = 0
        b, done = 1 << 20, 0   # no target: fp_frame_potential takes batches of up to 2^20 pairs
        while done < P:
            done += min(b, P - done)
            batches += 1
            b = min(b * 2, 1 << 20)
        h2d = P * (40 + 4 + 4)
        d2h = (P * 8 if prec == fp.PREC_FP32 else 0) + batches * ng * (2 * K + 1) * 8
        e2e = {"value": world * contracted / dt, "unit": "contractions/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "api": "fp_frame_potential (results to host)",
               "graph_replays": replays}
        if WORK["name"] == "local":
            e2e["note"] = ("includes the host planning of every pair (own topology per pair); the per-pair "
                           "contraction programs it uploads are not counted in h2d_bytes_per_step")

    n_skipped = int(skipped.item())
    value = world * (P * args.steps - n_skipped) / (ms / 1e3)
    # roofline of the dominant contraction class (the sweep kernels carry the flop count)
    cls = max((fp.K_SWEEP, fp.K_BRICK, fp.K_SPIRAL), key=lambda i: ks.ms[i])
    flops = 8.0 * ks.work[cls]                 # complex multiply-add = 8 real flops
    achieved = flops / (ks.ms[cls] / 1e3) / 1e12 if ks.ms[cls] > 0 else 0.0
    sm_max = (clocks or {}).get("sm_max_mhz") or 2070.0
    peak = SM_COUNT * FP32_LANES * 2 * sm_max * 1e6 / 1e12
    if prec == fp.PREC_FP64:
        peak = peak / 64.0       # FP64 FMA rate is a small fraction of FP32 on this part
    roof = {"bound": "alu", "kernel": fp.K_NAMES.get(cls, str(cls)), "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak if peak else None, "traffic": None,
            "peak_source": f"derived: {SM_COUNT} SMs x {FP32_LANES} FP32 lanes x 2 flop x {sm_max:.0f} MHz",
            "kernel_ms_share": ks.ms[cls] / ms if ms else None}
    if WORK["name"] == "brickwork" and prec == fp.PREC_FP32:
        # DRAM bytes (read + write) of the dominant kernel from one ncu capture of the current
        # tile-pass code: brick_pass_kernel<float2, 13, 5, 256>, depth 10, one pass over 256 pairs
        roof["traffic"] = 538.040832e6 + 476.1664e6
        roof["traffic_launch"] = ("brick_pass_kernel<float2,13,5,256>, l=10, one tile pass of 256 pairs; "
                                  "algorithmic bytes 2 x 256 x 2^18 x 8 = 1.0737e9")
    if WORK["name"] == "hea_paper" and prec == fp.PREC_FP32:
        # the dominant spiral kernel from one ncu capture: its DRAM traffic is the maps it reads
        roof["traffic"] = 412.827392e6 + 4.156928e6
        roof["traffic_launch"] = ("spiral_win_kernel<float2,5,2>, L=8, one launch of 2000 pairs; "
                                  "algorithmic bytes 2000 x 797 maps x 256 B = 4.081e8")

    metric = {"brickwork": METRIC, "hea": "Tr(U^dagger V) contractions/s at n=50 (HEA, L=1..8)",
              "hea_paper": "Tr(U^dagger V) contractions/s at n=50 (paper HEA with CNOT walls, L=1..8)",
              "local": "Tr(U^dagger V) contractions/s at n=20 (local circuits, T=20..100)"}[WORK["name"]]
    line = {"metric": metric, "value": value, "unit": "contractions/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec != fp.PREC_FP64 else "f64",
            "data": "synthetic (seeded circuit pairs)", "config": workload_config(args, world),
            "clocks": clocks, "e2e": e2e, "gpu_launches": launches, "roofline": roof,
            "kernel_ms": {fp.K_NAMES.get(i, str(i)): ks.ms[i] for i in range(8) if ks.launches[i]}}
    if WORK["name"] == "local":
        line["infeasible_pairs_in_timed_steps"] = n_skipped
    if WORK["name"] == "hea_paper":
        line["F_by_depth_last_step"] = moments_report(mom.cpu().numpy(), ens.groups(), K)
    if rank == 0 and world == 1 and not args.no_target and WORK["name"] == "brickwork":
        line["gpu_s_to_1pct_F2"] = gpu_seconds_to_target(fp, mom, P, K, ng)
    if rank == 0 and world == 1 and not args.no_cv and WORK["name"] == "brickwork":
        line["control_variate"] = control_variate_report(fp)
    if rank == 0 and world == 1 and not args.no_target and WORK["name"] == "brickwork":
        line["bootstrap"] = bootstrap_report(fp)
        mc = line.get("gpu_s_to_1pct_F2", {}).get("mixed_run", {}).get("F2_by_depth")
        line["exact_weingarten"] = exact_fk_report(fp, mc)
    if rank == 0 and world == 1 and not args.no_target and WORK["name"] == "local":
        line["local_large_T"] = local_large_T_report(fp)
    if rank == 0 and world == 1 and not args.no_cpu_baseline and WORK["name"] == "brickwork":
        cores = os.cpu_count() or 1
        r, dt, npairs, depths = oracle_time(10_000_000, cores)
        line["cpu_baseline"] = cpu_baseline_obj(r, cores, npairs, depths)
    if rank == 0:
        print(json.dumps(line), flush=True)
    ens.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
