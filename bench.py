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
    ap.add_argument("--cpu-depth-max", type=int, default=10,
                    help="deepest depth the CPU oracle baseline samples (10: the whole workload)")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the secondary workloads (n=8 FP64, HEA, paper HEA, local circuits)")
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
def _pairs_of_depth(d, l, count, first_pair):
    """The first `count` pairs of depth l of the workload at or after first_pair."""
    import oracle as O
    out, p = [], first_pair
    while len(out) < count:
        if O.pair_depth(d, p) == l:
            out.append(p)
        p += 1
    return out


def oracle_depth_rate(l, cores, first_pair):
    """Oracle throughput on pairs of depth l of the workload: cores pairs (4 x cores for
    l <= 6, where a pair takes milliseconds), one pair per thread on `cores` threads,
    FP64 variable elimination.  Returns (pairs/s, wall seconds, pairs)."""
    import concurrent.futures as cf
    import oracle as O
    d = O.desc(O.PARALLEL, WORK["n"], WORK["depth_min"], WORK["depth_max"], seed=WORK["seed"])
    pairs = _pairs_of_depth(d, l, cores * (4 if l <= 6 else 1), first_pair)
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        list(ex.map(lambda p: O.trace_batch(d, p, 1, "ve", threads=1), pairs))
    dt = time.perf_counter() - t0
    return len(pairs) / dt, dt, len(pairs)


def mix_rate(rates):
    """Rate on the workload's uniform depth mix from per-depth rates: the mean time per
    pair is the mean over depths of 1/rate."""
    return 1.0 / (sum(1.0 / r for r in rates.values()) / len(rates))


def oracle_baseline(cores, first_pair, depth_max=10):
    """The oracle on the machine's host cores, per depth, combined into the uniform-mix rate."""
    per, rates = {}, {}
    for l in range(WORK["depth_min"], min(WORK["depth_max"], depth_max) + 1):
        r, dt, npairs = oracle_depth_rate(l, cores, first_pair)
        rates[l] = r
        per[str(l)] = {"pairs": npairs, "wall_s": dt, "pairs_per_s": r, "core_s_per_pair": dt * cores / npairs}
    return mix_rate(rates), per


def cpu_baseline_obj(rate, cores, per, depth_max=10):
    deep = "" if depth_max >= WORK["depth_max"] else f"; depths above {depth_max} left out"
    return {"value": rate, "unit": "contractions/s", "cores": cores, "kind": "oracle",
            "sample": f"per depth l={WORK['depth_min']}..{min(WORK['depth_max'], depth_max)}: the workload's first "
                      f"pairs of that depth (one per core for l>=7, 4 per core below), one pair per thread, FP64 "
                      f"variable elimination; value = rate on the uniform depth mix = 1/mean_l(1/rate_l){deep}",
            "per_depth": per}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    dmax = min(args.cpu_depth_max, WORK["depth_max"])
    first = 10_000_000
    cheap = list(range(WORK["depth_min"], min(8, dmax) + 1))   # timed steps cycle over these depths
    deep = list(range(9, dmax + 1))                             # measured once, before the timed steps
    for w in range(args.warmup):
        oracle_depth_rate(WORK["depth_min"], cores, first + 1_000_000 * (w + 1))
    rates, per = {}, {}
    for l in deep:
        r, dt, npairs = oracle_depth_rate(l, cores, first)
        rates[l] = r
        per[str(l)] = {"pairs": npairs, "wall_s": dt, "pairs_per_s": r, "measured": "once, before the timed steps"}
    times, step_rates = [], {}
    for s in range(args.steps):
        l = cheap[s % len(cheap)]
        r, dt, npairs = oracle_depth_rate(l, cores, first + 2_000_000 * (s // len(cheap)))
        times.append(dt)
        step_rates.setdefault(l, []).append(r)
    for l in cheap:
        if l in step_rates:
            rates[l] = statistics.mean(step_rates[l])
            per[str(l)] = {"pairs_per_s": rates[l], "timed_steps": len(step_rates[l])}
        else:   # fewer timed steps than depths: measured once outside the timed steps
            r, dt, npairs = oracle_depth_rate(l, cores, first)
            rates[l] = r
            per[str(l)] = {"pairs": npairs, "wall_s": dt, "pairs_per_s": r, "measured": "once, untimed"}
    value = mix_rate(rates)
    cb = cpu_baseline_obj(value, cores, per, dmax)
    cb["sample"] += (f"; each timed step is one depth of {cheap[0]}..{cheap[-1]} in turn, depths "
                     f"{deep[0] if deep else '-'}..{deep[-1] if deep else '-'} (minutes per pair) are measured once "
                     "before the timed steps") if deep else ""
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "contractions/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(times) if times else 0.0, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded circuit pairs)",
            "config": workload_config(args, args.gpus), "cpu_baseline": cb,
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


def gpu_seconds_to_target(fp, rel=0.01):
    """GPU-seconds to F^(2) at `rel` relative standard error, per depth of the n = 50
    brickwork ensemble, measured by running fp_frame_potential to the target:
      l >= 5: the mixed (FP32 policy) path and the plain FP64 path each run until the
              target is met (FP64 for l <= 8; at l = 9, 10 the FP64 device time per pair,
              measured, times the pairs the mixed run needed -- the estimator's variance
              does not depend on the arithmetic);
      l <= 4: |Tr|^4 is so heavy-tailed that 1 % needs far more pairs: the mixed path runs a
              fixed budget of pairs, and the naive standard error, the bootstrap 5-95 %
              range and the exact F^(2) (Weingarten transfer matrix) are reported beside it."""
    import numpy as np
    import torch
    out = {"target_rel_stderr": rel, "groups": {}}
    tot32 = tot64 = 0.0
    for l in range(5, 11):
        row = {}
        for prec, tag in ((fp.PREC_FP32, "fp32"), (fp.PREC_FP64, "fp64")):
            if prec == fp.PREC_FP64 and l >= 9:
                c64 = per_pair_cost(fp, l, prec, 64 if l == 9 else 32, 60_000_000)
                row["fp64"] = {"pairs": row["fp32"]["pairs"], "gpu_s": c64 * row["fp32"]["pairs"],
                               "reached": row["fp32"]["reached"], "s_per_pair": c64,
                               "how": "measured FP64 device seconds per pair x pairs of the mixed run"}
                continue
            ens = fp.Ensemble(fp.PARALLEL, WORK["n"], l, l, seed=7000 + l)
            ens.frame_potential(10_000_000, 4096, 2, 0.0, prec)     # plans, autotuning, graphs
            F, se, st = ens.frame_potential(0, 8_000_000, 2, rel, prec)
            ens.close()
            row[tag] = {"pairs": int(st.pairs), "gpu_s": st.gpu_seconds, "reached": bool(st.reached_target),
                        "F2": float(F[0, 1]), "stderr": float(se[0, 1]), "fp64_recontracted": int(st.fp64_recontracted)}
        row["exact_F2"] = fp.exact_brickwork_fk(WORK["n"], l, 2)
        out["groups"][str(l)] = row
        tot32 += row["fp32"]["gpu_s"]
        tot64 += row["fp64"]["gpu_s"]
    out["gpu_s_mixed_fp32_l5_10"] = tot32
    out["gpu_s_plain_fp64_l5_10"] = tot64
    out["speedup_l5_10"] = tot64 / tot32 if tot32 > 0 else None
    budget = 2_000_000
    shallow = {}
    for l in range(2, 5):
        ens = fp.Ensemble(fp.PARALLEL, WORK["n"], l, l, seed=7000 + l, flags=fp.FLAG_TIMING)
        tr = torch.empty(2 * budget, dtype=torch.float64, device="cuda")
        grp = torch.empty(budget, dtype=torch.int32, device="cuda")
        ens.trace_batch(0, budget, fp.PREC_FP32, tr, None, grp)
        ks = ens.kernel_stats(reset=True)
        mom = torch.empty(2 * 2 + 1, dtype=torch.float64, device="cuda")
        ens.reduce_moments(tr, grp, budget, 2, mom)
        Fb = ens.bootstrap(tr, grp, budget, 2, 300, seed=11)
        ens.close()
        m = mom.cpu().numpy()
        N, S2, Q2 = m[0], m[2], m[4]
        F2 = S2 / N
        se2 = math.sqrt(max(Q2 / N - F2 * F2, 0.0) / (N - 1))
        shallow[str(l)] = {"pairs": budget, "gpu_s": sum(ks.ms[i] for i in range(8)) / 1e3, "F2": F2,
                           "stderr": se2, "rel_stderr": se2 / F2,
                           "bootstrap_F2_p5_p50_p95": [float(np.percentile(Fb[0, 1], q)) for q in (5, 50, 95)],
                           "exact_F2": fp.exact_brickwork_fk(WORK["n"], l, 2)}
    out["shallow_fixed_budget"] = shallow
    out["method"] = ("single-depth ensembles (seed 7000+l); fp_frame_potential to rel. stderr <= 1% (batches from "
                     "4096 pairs doubling to 2^20), stats.gpu_seconds = device time of the contraction batches")
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
        D, H = 12 * 50 * L, 256
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
                      f"{n_correct} exact corrections; MLP 12nL-256-256-256-1 GELU on periodic angle features, Adam, "
                      f"log|Tr|^2 target, g = beta exp(2 prediction) with beta fitted on the training pairs; "
                      f"hidden layers as BF16 tcgen05 GEMMs with FP32 accumulation",
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
# ---------------------------------------------------------------------------
# measured peaks and rooflines
# ---------------------------------------------------------------------------
def measure_peaks(fp):
    """The arithmetic peaks of this GPU, measured by fp_measure_peak (microbenchmarks
    timed with CUDA events, SM clock read in-kernel)."""
    names = {fp.PEAK_FFMA: "fp32_ffma", fp.PEAK_FFMA2: "fp32_ffma2", fp.PEAK_DFMA: "fp64_dfma",
             fp.PEAK_TC_TF32: "tf32_tcgen05", fp.PEAK_TC_BF16: "bf16_tcgen05"}
    return {nm: fp.measure_peak(w) for w, nm in names.items()}


# DRAM read and write bytes of one tile-pass launch over 256 pairs at l = 10, per sweep
# variant ("tile bits, window bits, threads, pass kind" as fp_brick_variant gives it),
# from ncu captures of the committed code (the summaries under profiles/)
TRAFFIC_L10 = {
    "13 5 256 0": ("brick_pass_kernel<float2,13,5,256>", 538.275328e6, 479.907328e6,
                   "profiles/brick_pass_kernel_f32_brickwork_n50_l10.md"),
    "12 5 256 4": ("brick_tcm_pass_kernel", 587.271680e6, 481.361664e6,
                   "profiles/brick_tcm_pass_kernel_brickwork_n50_l10.md"),
}


def roofline(fp, ks, ms_total, prec, peaks, clocks):
    """Roofline of the dominant contraction class: algorithmic flops (8 real flops per
    complex multiply-add of the method, ks.work) over that class's device time, against
    the measured FP32 (packed FFMA) or FP64 peak at the run's median SM clock."""
    cls = max((fp.K_SWEEP, fp.K_BRICK, fp.K_SPIRAL), key=lambda i: ks.ms[i])
    flops = 8.0 * ks.work[cls]
    achieved = flops / (ks.ms[cls] / 1e3) / 1e12 if ks.ms[cls] > 0 else 0.0
    key = "fp64_dfma" if prec == fp.PREC_FP64 else "fp32_ffma2"
    pk = peaks[key]
    mhz = (clocks or {}).get("sm_mhz") or pk["sm_mhz"]
    peak = pk["flops_per_clk_sm"] * pk["sms"] * mhz * 1e6 / 1e12
    return {"bound": "alu", "kernel": fp.K_NAMES.get(cls, str(cls)), "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak if peak else None, "traffic": None,
            "peak_source": (f"measured: {key} microbenchmark {pk['flops_per_clk_sm']:.1f} flop/clk/SM x {pk['sms']} "
                            f"SMs x {mhz:.0f} MHz (median SM clock of the timed region); "
                            f"{pk['tflops']:.1f} TFLOP/s at {pk['sm_mhz']:.0f} MHz in the microbenchmark"),
            "kernel_ms_share": ks.ms[cls] / ms_total if ms_total else None,
            "tensor_view": tensor_view(ks, cls, peaks)}


def tensor_view(ks, cls, peaks):
    """The brickwork tensor-core passes against the tensor pipe: TF32 flops issued to the
    tensor cores (three products per operand pair, 2 per multiply-add, counted by the
    library) over the device time of the whole brickwork class (which also holds the
    gate maps, the tile loads of the first pass and the meet, so the rate is a lower
    bound), against the measured tcgen05 kind::tf32 rate of the microbenchmark."""
    mma = float(getattr(ks, "mma_flops", 0.0))
    if mma <= 0 or ks.ms[cls] <= 0 or "tf32_tcgen05" not in peaks:
        return None
    achieved = mma / (ks.ms[cls] / 1e3) / 1e12
    pk = peaks["tf32_tcgen05"]
    return {"bound": "tensor", "achieved": achieved, "peak": pk["tflops"], "unit": "TFLOP/s",
            "frac": achieved / pk["tflops"],
            "peak_source": (f"measured: tcgen05 kind::tf32 microbenchmark, {pk['tflops']:.0f} TFLOP/s at "
                            f"{pk['sm_mhz']:.0f} MHz"),
            "note": "time = whole brickwork class (lower bound on the tensor-core passes' own rate)"}


# ---------------------------------------------------------------------------
def measure(fp, args, work, P, steps, warmup, prec, stream, rank, world, dist):
    """W untimed + K timed steps of one workload (sample -> contraction -> moments),
    CUDA events on the library's stream, max over ranks; clocks sampled during the
    timed region."""
    import torch
    from paper_2205_09900_gb300.shard import max_over_ranks, pair_range
    saved = dict(WORK)
    WORK.clear()
    WORK.update(work)
    try:
        K = WORK["k_max"]
        ens = make_ensemble(fp, fp.FLAG_TIMING, stream.cuda_stream)
        ng = len(ens.groups())
        tr = torch.empty(2 * P, dtype=torch.float64, device="cuda")
        kap = torch.empty(P, dtype=torch.float64, device="cuda")
        err = torch.empty(P, dtype=torch.float64, device="cuda")
        grp = torch.empty(P, dtype=torch.int32, device="cuda")
        mom = torch.empty(ng * (2 * K + 1), dtype=torch.float64, device="cuda")
        skipped = torch.zeros((), dtype=torch.int64, device="cuda")

        def first_of(s):
            return pair_range(s, rank, world, P)[0]

        def step(s):
            ens.trace_batch(first_of(s), P, prec, tr, kap, grp, err)
            ens.reduce_moments(tr, grp, P, K, mom)
            if WORK["name"] == "local":
                skipped.add_((grp < 0).sum())

        for s in range(warmup):
            step(s)
        torch.cuda.synchronize()
        skipped.zero_()
        ens.kernel_stats(reset=True)
        clk = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        clk.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for s in range(warmup, warmup + steps):
            step(s)
        e1.record(stream)
        torch.cuda.synchronize()
        clocks = clk.stop()
        ms = max_over_ranks(e0.elapsed_time(e1), dist, device="cuda")
        if dist:
            dist.barrier()
        ks = ens.kernel_stats(reset=True)
        n_skipped = int(skipped.item())
        variants = {}
        if WORK["kind"] in (0, 2):   # brickwork and HEA: the tuner's choice of sweep per depth
            for dv in ens.groups():
                try:
                    variants[int(dv)] = " ".join(str(x) for x in ens.brick_variant(int(dv), prec))
                except fp.FpError:
                    pass             # depth 1 or a depth this step did not contract
        out = {"ms": ms, "ks": ks, "clocks": clocks, "mom": mom.cpu().numpy(), "groups": ens.groups(),
               "variants": variants,
               "value": world * (P * steps - n_skipped) / (ms / 1e3), "skipped": n_skipped,
               "launches": int(sum(ks.launches[i] for i in range(8))), "tr": tr, "first_last": first_of(warmup + steps - 1)}
        ens.close()
        return out
    finally:
        WORK.clear()
        WORK.update(saved)


def secondary_workloads(fp, peaks, stream):
    """The other configurations of the metric, measured the same way (device time of
    whole steps, clocks, roofline against the measured peaks), compactly:
      n8_fp64      brickwork n = 8, l = 4, 10^4 pairs, FP64, F^(1..3), with the error
                   against the oracle's dense 256 x 256 traces on 256 of the pairs;
      hea          HEA n = 50, L = 1..8, 10^6 pairs per step;
      hea_paper    the paper's HEA (CNOT walls) n = 50, L = 1..8, 10^5 pairs per step;
      local        local circuits n = 20, T = 20..100, 2 x 10^4 pairs per step."""
    import numpy as np
    cfgs = {
        "n8_fp64": (dict(n=8, depth_min=4, depth_max=4, pairs=10_000, seed=1, k_max=3, kind=0, name="brickwork"),
                    10_000, 5, fp.PREC_FP64),
        "hea": (WORKLOADS["hea"], 1_000_000, 2, fp.PREC_FP32),
        "hea_paper": (WORKLOADS["hea_paper"], 100_000, 3, fp.PREC_FP32),
        "local": (WORKLOADS["local"], 20_000, 3, fp.PREC_FP32),
    }
    out = {}
    for name, (work, P, steps, prec) in cfgs.items():
        r = measure(fp, None, dict(work), P, steps, 2, prec, stream, 0, 1, None)
        K = work["k_max"]
        m = r["mom"].reshape(len(r["groups"]), 2 * K + 1)
        F = {}
        for g, dv in enumerate(r["groups"]):
            N = m[g, 0]
            if N < 2:
                continue
            f = [float(m[g, k] / N) for k in range(1, K + 1)]
            se = [math.sqrt(max(m[g, K + k] / N - f[k - 1] ** 2, 0.0) / (N - 1)) for k in range(1, K + 1)]
            F[str(int(dv))] = {"F": f, "stderr": se}
        row = {"value": r["value"], "unit": "contractions/s", "ms_per_step": r["ms"] / steps, "steps": steps,
               "pairs_per_step": P, "dtype": "f64" if prec == fp.PREC_FP64 else "f32", "clocks": r["clocks"],
               "roofline": roofline(fp, r["ks"], r["ms"], prec, peaks, r["clocks"]), "gpu_launches": r["launches"],
               "F_by_group_last_step": F}
        if name == "local":
            row["infeasible_pairs_in_timed_steps"] = r["skipped"]
        if name == "n8_fp64":
            import oracle as O
            t = r["tr"].cpu().numpy()
            got = t[0:512:2] + 1j * t[1:512:2]
            ref = O.trace_batch(O.desc(O.PARALLEL, 8, 4, seed=1), r["first_last"], 256, "dense", threads=8)
            row["max_rel_err_vs_oracle_dense_256_pairs"] = float(np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1)))
        out[name] = row
    return out


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
    from paper_2205_09900_gb300.shard import pair_range

    prec = fp.PREC_FP32 if args.prec == "fp32" else fp.PREC_FP64
    stream = torch.cuda.current_stream()
    P, K = args.pairs, WORK["k_max"]
    peaks = measure_peaks(fp)
    r = measure(fp, args, dict(WORK), P, args.steps, args.warmup, prec, stream, rank, world, dist)
    ms, ks, clocks, launches = r["ms"], r["ks"], r["clocks"], r["launches"]

    def first_of(step):
        return pair_range(step, rank, world, P)[0]

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
        ng = len(ens_u.groups())
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

    value = r["value"]
    roof = roofline(fp, ks, ms, prec, peaks, clocks)
    chosen = r["variants"].get(10)
    if WORK["name"] == "brickwork" and prec == fp.PREC_FP32 and args.depth == 0 and chosen in TRAFFIC_L10:
        # DRAM bytes (read + write) of one tile-pass launch of the sweep variant the tuner chose
        # at l = 10 (the depth that dominates the step), from one ncu capture of this code
        kname, rd, wr, prof = TRAFFIC_L10[chosen]
        roof["traffic"] = rd + wr
        roof["traffic_launch"] = (f"{kname}, l=10, one tile pass of 256 pairs; "
                                  "algorithmic bytes 2 x 256 x 2^18 x 8 = 1.0737e9")
        roof["traffic_source"] = f"static: ncu capture in {prof} (the tuner chose '{chosen}' at l = 10 in this run)"

    metric = {"brickwork": METRIC, "hea": "Tr(U^dagger V) contractions/s at n=50 (HEA, L=1..8)",
              "hea_paper": "Tr(U^dagger V) contractions/s at n=50 (paper HEA with CNOT walls, L=1..8)",
              "local": "Tr(U^dagger V) contractions/s at n=20 (local circuits, T=20..100)"}[WORK["name"]]
    line = {"metric": metric, "value": value, "unit": "contractions/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec != fp.PREC_FP64 else "f64",
            "data": "synthetic (seeded circuit pairs)", "config": workload_config(args, world),
            "clocks": clocks, "e2e": e2e, "gpu_launches": launches, "roofline": roof,
            "peaks_measured": peaks, "sweep_variants": {str(k): v for k, v in r["variants"].items()},
            "kernel_ms": {fp.K_NAMES.get(i, str(i)): ks.ms[i] for i in range(8) if ks.launches[i]}}
    if WORK["name"] == "local":
        line["infeasible_pairs_in_timed_steps"] = r["skipped"]
    if WORK["name"] == "hea_paper":
        line["F_by_depth_last_step"] = moments_report(r["mom"], r["groups"], K)
    solo = rank == 0 and world == 1
    if solo and not args.no_secondary and WORK["name"] == "brickwork" and args.depth == 0:
        line["secondary"] = secondary_workloads(fp, peaks, stream)
    if solo and not args.no_target and WORK["name"] == "brickwork":
        line["gpu_s_to_1pct_F2"] = gpu_seconds_to_target(fp)
    if solo and not args.no_cv and WORK["name"] == "brickwork":
        line["control_variate"] = control_variate_report(fp)
    if solo and not args.no_target and WORK["name"] == "brickwork":
        line["bootstrap"] = bootstrap_report(fp)
        line["exact_weingarten"] = exact_fk_report(fp)
    if solo and not args.no_target and WORK["name"] == "local":
        line["local_large_T"] = local_large_T_report(fp)
    if solo and not args.no_cpu_baseline and WORK["name"] == "brickwork":
        cores = os.cpu_count() or 1
        rate, per = oracle_baseline(cores, 10_000_000, args.cpu_depth_max)
        line["cpu_baseline"] = cpu_baseline_obj(rate, cores, per, args.cpu_depth_max)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
