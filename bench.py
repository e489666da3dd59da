#!/usr/bin/env python
"""Benchmark: SLM tree training with PSO split search on GB300.

A step is one full tree (or bagged forest) grown through libslm's C ABI
(slm_train_tree): every level's nodes searched in one batch by the particle
swarm, then partitioned. The default workload is the classification tree of
50,000 samples x 64 features, 10 Gaussian-mixture classes, depth <= 8, min
leaf 20, P=64 particles, T=100 iterations, 128 bins, Gini, FP32 projection.
The metric is particle-sample evaluations per second: sum over searched
nodes of n_node * P * (T+1), divided by the time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME] [--proj fp32|bf16] [--topk K] [--compare-fp32]

--workload selects another named setting of paper_2208_07023_gb300.workloads
(regtree_n200k_d128: the regression tree, bfloat16 projection with top-8 FP32
re-scoring by default; forest64_n100k_d32_k5: 64 bagged trees; node_n2000_d16:
one node; proposal_n1m_d256_k20: the learned swarm proposal, trained first,
then PSO iterations to the plain search's loss, seeded vs plain, over the
first four levels of a 1,000,000 x 256, 20-class mixture). --compare-fp32 also times the plain FP32 form of the same workload
and reports both forms' time and training loss.

With N > 1 (torchrun) every rank grows its own tree on its own seed (weak
scaling, no data exchange); rank 0 prints one JSON line. --impl reference
times the CPU oracle on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2208_07023_gb300 import workloads as W  # noqa: E402

METRIC = "SLM tree train time & particle-sample evals/s vs plain FP32 PSO at equal loss"
UNIT = "particle-sample evals/s"
DEFAULT_WORKLOAD = "tree_n50k_d64_k10"
# FP32 fused multiply-add peak: 152 SMs x 128 FP32 lanes x 2 flop x 2.070 GHz.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
L2_FLUSH_BYTES = 256 << 20
CPU_SAMPLE_S = 10.0  # CPU work of one oracle baseline sample


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), float(j["bf16_tflops"]), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


HBM_PEAK_GBS, BF16_PEAK_TFLOPS, PEAK_SOURCE = _measured_peaks()

# DRAM bytes per particle-sample pair from ncu captures of the default
# workload's root search (dram__bytes_read.sum + dram__bytes_write.sum of one
# launch over its pairs, profiles/), each valid only for the kernel source it
# was taken from: (bytes per pair, source file, sha256 of that file).
TRAFFIC = {
    "project": (12945152 / 3.2e6, "step_kernels.cu",
                "6f7aa4390ba6326c3a0f7e2e133cae0165c0f104276e7fc53b374ce71d178241"),
    "hist_scan": (13066496 / 3.2e6, "hist_kernels.cu",
                  "503a69c3a12c5b8fac4578b88d018a05729810e190770abfa551f1af9538117e"),
}


def _kernel_source_sha(name):
    import hashlib
    p = os.path.join(ROOT, "paper_2208_07023_gb300", "csrc", name)
    with open(p, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def traffic_per_launch(name, ks, workload):
    """Captured DRAM bytes per pair x the average pairs of a launch, or None
    for another workload or once the kernel source differs from the captured
    one."""
    if workload != DEFAULT_WORKLOAD or name not in TRAFFIC:
        return None
    per_pair, src, sha = TRAFFIC[name]
    if sha != _kernel_source_sha(src):
        return None
    return per_pair * ks["pairs"] / max(1, ks["launches"])


def config_dict(name, cfg, wl, proj, topk, extra=None, args_launch=None):
    d = {"workload": name, "n": wl.n, "d": wl.d, "classes": wl.n_classes,
         "trees": cfg["n_trees"], "bootstrap": cfg.get("bootstrap", cfg["n_trees"] > 1),
         "max_depth": cfg["max_depth"], "min_leaf": cfg["min_leaf"],
         "particles": cfg["n_particles"], "iters": cfg["n_iters"], "bins": cfg["n_bins"],
         "criterion": cfg["criterion"],
         "projection": ("bf16 tcgen05 + top-%d fp32 ffma re-scoring" % topk
                        if proj == "bf16" else "fp32 ffma"),
         "l2": "flushed between steps (256 MiB write outside the timed events)"}
    if cfg.get("top_n"):
        d["feature_prescreen_top_n"] = cfg["top_n"]
    if cfg.get("apso"):
        d["swarm"] = "adaptive PSO (evolutionary-state estimation)"
    if cfg.get("rounds"):
        kind = "SLR Boost" if wl.labels is None else "SLM Boost (%d trees a round)" % wl.n_classes
        d["boost"] = {"rounds": cfg["rounds"], "learning_rate": cfg["lr"],
                      "step": "one %s training: every round's trees, residuals, "
                              "predictions and score updates" % kind}
    if args_launch is not None:
        d["search_loop_graphs"] = args_launch.graphs
        d["projection_tile_mode"] = args_launch.tiles
        d["projection_staging"] = ("tensor-map tile copies (cp.async.bulk.tensor)"
                                   if args_launch.tma == "on" else "per-thread cp.async")
    if extra:
        d.update(extra)
    return d


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons, kept for the time
    between mark_start() and mark_end(). Sampling starts before the region
    (nvidia-smi needs a moment to print its first line) every 50 ms; each
    sample carries nvidia-smi's own timestamp."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 50

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.out = ""
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", str(self.PERIOD_MS)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
            self.proc = None

    @staticmethod
    def _stamp(text):
        import datetime
        try:
            return datetime.datetime.strptime(text.strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def summary(self):
        """Median SM clock and the throttle reasons seen in the marked region
        (with half a period of slack on each side); if no sample falls in it,
        the sample closest to its middle, flagged as such."""
        rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").strip().splitlines():
            f = [t.strip() for t in line.split(",")]
            if len(f) < 10:
                continue
            try:
                rows.append((self._stamp(f[0]), float(f[2]), float(f[3]),
                             {n for n, v in zip(names, f[6:10]) if v.lower().startswith("active")}))
            except ValueError:
                continue
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not rows:
            return out
        inside = rows
        if self.t0 is not None and self.t1 is not None:
            slack = self.PERIOD_MS / 2000.0
            inside = [r for r in rows if r[0] is not None and
                      self.t0 - slack <= r[0] <= self.t1 + slack]
            if not inside:
                mid = 0.5 * (self.t0 + self.t1)
                timed = [r for r in rows if r[0] is not None]
                if not timed:
                    return out
                inside = [min(timed, key=lambda r: abs(r[0] - mid))]
                out["nearest_sample_outside_region"] = True
        out["sm_mhz"] = statistics.median(r[1] for r in inside)
        out["sm_max_mhz"] = inside[-1][2]
        out["reasons"] = sorted(set().union(*[r[3] for r in inside]))
        out["samples"] = len(inside)
        return out


def gpu_uuid(dev: int) -> str:
    import torch
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        return vis.split(",")[dev] if vis else str(dev)


# ---------------------------------------------------------------- oracle ----

def oracle_params(cfg, wl, proj, topk, iters):
    import oracle as O
    prec = O.BF16_TOPK if proj == "bf16" else O.F32_MIRROR
    return O.make_params(cfg["criterion"], wl.n_classes, cfg["n_particles"], iters,
                         cfg["n_bins"], min_leaf=cfg["min_leaf"], seed=1, precision=prec,
                         topk=topk if proj == "bf16" else 0, top_n=cfg.get("top_n", 0))


def oracle_targets(cfg, wl):
    """(labels, y) of a root search of the workload: a boosting run's first
    root search fits residuals (y minus its mean; for classes, class 0's
    one-hot minus 1/K)."""
    if not cfg.get("rounds"):
        return wl.labels, wl.y
    if wl.labels is None:
        return None, (wl.y - np.float32(np.mean(wl.y.astype(np.float64)))).astype(np.float32)
    K = wl.n_classes
    return None, ((wl.labels == 0).astype(np.float64) - 1.0 / K).astype(np.float32)


def oracle_root_sample(cfg, wl, proj, topk, iters):
    """Times the CPU oracle's swarm search of the root node (all n samples)
    with `iters` iterations; returns (evals/s, seconds, evaluations)."""
    import oracle as O
    p = oracle_params(cfg, wl, proj, topk, iters)
    t0 = time.perf_counter()
    O.node_split(p, wl.X, *oracle_targets(cfg, wl), node_uid=0)
    dt = time.perf_counter() - t0
    evals = wl.n * cfg["n_particles"] * (iters + 1)
    return evals / dt, dt, evals


def oracle_sample_iters(cfg, wl, proj, topk, budget_s):
    """Iterations of a root-node search that take about budget_s seconds on
    the host: one initial evaluation is timed first."""
    _, dt1, _ = oracle_root_sample(cfg, wl, proj, topk, 0)
    return int(max(0, min(cfg["n_iters"], budget_s / max(dt1, 1e-6) - 1)))


def cpu_baseline(cfg, wl, proj, topk):
    """Root-node searches of the workload (other node ids after the first)
    until about CPU_SAMPLE_S seconds of host work, at most 30 searches."""
    import oracle as O
    iters = oracle_sample_iters(cfg, wl, proj, topk, CPU_SAMPLE_S)
    p = oracle_params(cfg, wl, proj, topk, iters)
    secs, reps = 0.0, 0
    while reps < 30 and (reps == 0 or secs < CPU_SAMPLE_S):
        t0 = time.perf_counter()
        O.node_split(p, wl.X, *oracle_targets(cfg, wl), node_uid=reps)
        secs += time.perf_counter() - t0
        reps += 1
    ev = wl.n * cfg["n_particles"] * (iters + 1) * reps
    mode = "bf16 top-%d" % topk if proj == "bf16" else "fp32-mirror"
    return {"value": ev / secs, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": (f"{reps} root-node swarm searches of the workload (node ids 0..{reps - 1}; "
                       f"{wl.n} samples x {cfg['n_particles']} particles x {iters + 1} "
                       f"evaluations each = {ev} evaluations, {secs:.1f} s; {mode} oracle, "
                       f"OpenMP over particles)")}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cfg = W.SETTINGS[args.workload]
    wl = cfg["builder"](1)
    proj, topk = args.proj, args.topk
    iters = 10 if args.workload == DEFAULT_WORKLOAD else \
        oracle_sample_iters(cfg, wl, proj, topk, 20.0)
    for _ in range(args.warmup):
        oracle_root_sample(cfg, wl, proj, topk, iters)
    secs = []
    for _ in range(args.steps):
        _, dt, _ = oracle_root_sample(cfg, wl, proj, topk, iters)
        secs.append(dt)
    value = wl.n * cfg["n_particles"] * (iters + 1) * len(secs) / sum(secs)
    sample = (f"root-node swarm search of the same workload: {wl.n} samples x "
              f"{cfg['n_particles']} particles x {iters + 1} evaluations per step "
              f"({'bf16 top-k' if proj == 'bf16' else 'fp32-mirror'} oracle, OpenMP over "
              "particles)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(secs) / len(secs), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16+f32" if proj == "bf16" else "f32", "data": "synthetic",
            "config": config_dict(args.workload, cfg, wl, proj, topk,
                                  {"sample": f"root node, {iters + 1} evaluations"}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------- GPU ----

def tree_loss(ctx, f, wl, X):
    """Training loss of tree 0 under its criterion (weighted leaf impurity:
    MSE for regression, Gini for classification; bootstrap weights are not
    applied) and the ensemble's training MSE / error."""
    cls, val, leaf = ctx.predict(f, X, want_leaf=True)
    lf = leaf[:, 0]
    if wl.y is not None:
        g = f.export(0)
        pred = g["leaf_value"][lf]
        return {"tree0_mse": float(np.mean((pred - wl.y) ** 2)),
                "ensemble_mse": float(np.mean((val - wl.y) ** 2))}
    return {"tree0_gini": leaf_gini(lf, wl.labels, wl.n_classes),
            "ensemble_error": float(np.mean(cls != wl.labels))}


def split_loss(f, n_trees=1):
    """Summed weighted child impurity of every split (Eq. 4: each split's
    loss times the weight of the node it splits), over the root's weight."""
    tot = 0.0
    for t in range(n_trees):
        g = f.export(t)
        inner = g["kind"] == 1
        tot += float(np.sum(g["loss"][inner] * g["weight"][inner]) / max(1, g["weight"][0]))
    return tot / n_trees


def vs_plain_fp32(ctx, S, cfg, wl, X, L, Y, flush, stream, steps, plain):
    """The default classification tree in the combined form beside plain FP32
    PSO: level-batched searches with BF16 tensor-core projections and FP32
    re-scoring of the top 8 particles, without and with the learned swarm
    proposal (trained first, on (node statistics, PSO-best direction) pairs
    from nodes of the same mixture drawn with disjoint sample seeds), at T
    and at T / 4 iterations, and the seeded FP32 form; tree time (device
    events, mean of the steps), training Gini and summed split loss of each
    beside the plain FP32 form's."""
    rng = np.random.default_rng(77)
    stats, dims, targets = [], [], []
    t0 = time.perf_counter()
    K, d = wl.n_classes, wl.d
    for i in range(160):
        w2 = W.gmm(6000, d, K, seed=1, sample_seed=900_000 + i)
        keep = rng.choice(K, rng.integers(2, K + 1), replace=False)
        m = np.isin(w2.labels, keep)
        remap = np.full(K, -1, np.int32)
        remap[np.sort(keep)] = np.arange(keep.size)
        Xs, ls = w2.X[m], remap[w2.labels[m]]
        r = ctx.node_split(S.make_params("gini", K, n_particles=cfg["n_particles"], n_iters=50,
                                         n_bins=cfg["n_bins"], min_leaf=cfg["min_leaf"],
                                         seed=i + 3), Xs, labels=ls, node_uid=i)
        stats.append(ctx.node_stats(Xs, labels=ls, n_classes=K))
        dims.append(d)
        tg = np.zeros(256, np.float32)
        tg[:d] = r["direction"]
        targets.append(tg)
    t_pairs = time.perf_counter() - t0
    prop = ctx.proposal(seed=11)
    t0 = time.perf_counter()
    prop.train(np.array(stats, np.float32), np.array(dims, np.int32),
               np.array(targets, np.float32), epochs=30, batch=64, lr=1e-3, seed=3)
    t_train = time.perf_counter() - t0
    ctx.use_proposal(prop)
    out = {"plain_fp32": plain}
    T = cfg["n_iters"]
    try:
        for key, proj, seeded, iters in (("bf16_top8", "bf16", False, T),
                                         ("seeded_bf16_top8", "bf16", True, T),
                                         ("seeded_bf16_top8_T/4", "bf16", True, T // 4),
                                         ("seeded_fp32", "fp32", True, T),
                                         ("seeded_fp32_T/4", "fp32", True, T // 4)):
            pp = make_params(S, dict(cfg, n_iters=iters), wl, proj, 8)
            pp.seeded = 1 if seeded else 0
            ctx.train_tree(pp, X, labels=L, y=Y).free()  # warm-up (tiles, graphs)
            tp, ep, _ = time_steps(ctx, pp, X, L, Y, steps, flush, stream)
            f = ctx.train_tree(pp, X, labels=L, y=Y)
            out[key] = {"tree_train_ms": sum(tp) / len(tp), "iters": iters,
                        "evaluations": ep // steps, "train_loss": tree_loss(ctx, f, wl, X),
                        "split_loss_sum": split_loss(f)}
            f.free()
    finally:
        ctx.use_proposal(None)
        prop.free()
    gini = lambda k: out[k]["train_loss"]["tree0_gini"]
    for k in out:
        if k != "plain_fp32":
            out[k]["time_vs_plain"] = out[k]["tree_train_ms"] / plain["tree_train_ms"]
            out[k]["loss_le_plain"] = bool(gini(k) <= gini("plain_fp32") + 1e-12 and
                                          out[k]["split_loss_sum"] <=
                                          plain["split_loss_sum"] + 1e-12)
    out["proposal"] = {"training_pairs": len(dims), "pair_generation_s": t_pairs,
                       "train_s": t_train,
                       "pairs": "class subsets of the tree's mixture (same means and "
                                "covariance), 6,000 samples with disjoint sample seeds"}
    return out


def vs_probabilistic(ctx, S, cfg, wl, X, L, Y, n_ids=8):
    """Root searches of the swarm (P particles, T iterations: P (T + 1)
    evaluations) beside the probabilistic search of the original SLM
    (Sec. II-B) with 1000 candidates (the count the paper quotes), the same
    P (T + 1) evaluations, and ten times that, on node ids 0..n_ids-1: wall
    time of each call (device-resident inputs, synchronised), final loss,
    and the candidates the probabilistic search needed to reach the swarm's
    final loss (None if it never did). Candidates: R = 4 of the ranked
    features, weights 0.8^(r-1), ranges floor(8 exp(-0.05 r)), batches of
    256."""
    import torch
    P, T = cfg["n_particles"], cfg["n_iters"]
    pso = make_params(S, dict(cfg, max_depth=1), wl, "fp32", 0)
    counts = {"1000": 1000, "equal_evals": P * (T + 1), "10x_evals": 10 * P * (T + 1)}
    res = {"pso": {"ms": [], "loss": []}}
    res.update({k: {"candidates": v, "ms": [], "loss": [], "to_pso_loss": []}
                for k, v in counts.items()})

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return out, (time.perf_counter() - t0) * 1e3

    ctx.node_split(pso, X, labels=L, y=Y, node_uid=0)  # warm-up
    for k, I in counts.items():
        ctx.prob_search(pso, S.make_prob(I, batch=256, q=4), X, labels=L, y=Y, node_uid=0)
    for uid in range(n_ids):
        r, ms = timed(lambda: ctx.node_split(pso, X, labels=L, y=Y, node_uid=uid))
        res["pso"]["ms"].append(ms)
        res["pso"]["loss"].append(float(r["loss"]))
        for k, I in counts.items():
            pp = S.make_prob(I, batch=256, q=4)
            g, ms = timed(lambda: ctx.prob_search(pso, pp, X, labels=L, y=Y, node_uid=uid))
            reach = np.flatnonzero(g["trace"] <= r["loss"])
            res[k]["ms"].append(ms)
            res[k]["loss"].append(float(g["loss"]))
            res[k]["to_pso_loss"].append(min(I, int(reach[0] + 1) * 256) if reach.size else None)
    out = {"searches": n_ids, "node": "root", "pso_evaluations": P * (T + 1),
           "prob_params": {"R": 4, "gamma": 0.8, "alpha0": 8.0, "alpha": 0.05,
                           "batch": 256, "q": 4, "cos": "9/10"},
           "pso": {"median_ms": float(np.median(res["pso"]["ms"])),
                   "median_loss": float(np.median(res["pso"]["loss"]))}}
    for k in counts:
        got = [h for h in res[k]["to_pso_loss"] if h is not None]
        out["prob_" + k] = {
            "candidates": counts[k], "median_ms": float(np.median(res[k]["ms"])),
            "median_loss": float(np.median(res[k]["loss"])),
            "reached_pso_loss": len(got) / n_ids,
            "median_candidates_to_pso_loss": float(np.median(got)) if got else None,
            "loss_le_pso": float(np.mean(np.array(res[k]["loss"]) <=
                                         np.array(res["pso"]["loss"])))}
    return out


def leaf_gini(leaf, labels, K):
    """Weighted Gini impurity of a partition into leaves: sum over leaves of
    n_leaf (1 - sum_k p_k^2), divided by n."""
    import numpy as np
    c = np.bincount(leaf.astype(np.int64) * K + labels, minlength=(int(leaf.max()) + 1) * K)
    c = c.reshape(-1, K).astype(np.float64)
    tot = c.sum(axis=1)
    m = tot > 0
    return float((tot[m] - (c[m] ** 2).sum(axis=1) / tot[m]).sum()) / leaf.shape[0]


def apso_quality(ctx, S, cfg, wl, proj, topk, X, L, Y, n_ids=32):
    """Root searches with adaptive and plain PSO from the same initial
    swarms (node ids 0..n_ids-1): the iteration at which adaptive PSO's gB
    loss first reaches plain PSO's final loss (None if never), and both
    final losses."""
    pa = make_params(S, dict(cfg, max_depth=1), wl, proj, topk)
    pp = make_params(S, dict(cfg, max_depth=1, apso=False), wl, proj, topk)
    hit, fa, fp = [], [], []
    for uid in range(n_ids):
        a = ctx.node_split(pa, X, labels=L, y=Y, node_uid=uid, want_trace=True)["trace"]
        b = ctx.node_split(pp, X, labels=L, y=Y, node_uid=uid, want_trace=True)["trace"]
        reach = np.flatnonzero(a <= b[-1])
        hit.append(int(reach[0]) if reach.size else None)
        fa.append(float(a[-1]))
        fp.append(float(b[-1]))
    got = [h for h in hit if h is not None]
    return {"searches": n_ids, "iters": cfg["n_iters"],
            "reached_plain_final_loss": len(got) / n_ids,
            "median_iter_to_plain_final_loss": float(np.median(got)) if got else None,
            "median_final_loss_apso": float(np.median(fa)),
            "median_final_loss_plain": float(np.median(fp)),
            "apso_lower_final_loss": float(np.mean(np.array(fa) < np.array(fp)))}


def make_params(S, cfg, wl, proj, topk):
    return S.make_params(cfg["criterion"], wl.n_classes, n_particles=cfg["n_particles"],
                         n_iters=cfg["n_iters"], n_bins=cfg["n_bins"],
                         min_leaf=cfg["min_leaf"], max_depth=cfg["max_depth"], seed=1,
                         n_trees=cfg["n_trees"],
                         bootstrap=cfg.get("bootstrap", cfg["n_trees"] > 1),
                         proj=S.SLM_PROJ_BF16_TOPK if proj == "bf16" else S.SLM_PROJ_FP32,
                         topk=topk, top_n=cfg.get("top_n", 0), apso=cfg.get("apso", False))


class BoostRun:
    """One SLR Boost training seen as a step: its rounds' evaluations."""

    def __init__(self, boost):
        self.b = boost

    def info(self):
        inf = self.b.info()
        m = inf["n_rounds"] * inf["n_outputs"]  # every tree of every round
        return {"evaluations": sum(self.b.tree(i).info()["evaluations"] for i in range(m))}

    def free(self):
        self.b.free()


def train_step(ctx, p, cfg, X, L, Y):
    """One step of the workload: a tree / forest, or a boosting run."""
    if cfg.get("rounds"):
        return BoostRun(ctx.train_boost(p, X, y=Y, labels=L, n_rounds=cfg["rounds"],
                                        learning_rate=cfg["lr"], n_classes=cfg.get("classes")))
    return ctx.train_tree(p, X, labels=L, y=Y)


def step_loss(ctx, f, wl, X):
    if isinstance(f, BoostRun):
        loss = f.b.train_loss
        by_round = [round(float(v), 6) for v in loss]
        if wl.labels is None:
            y = wl.y.astype(np.float64)
            return {"boost_train_mse": float(loss[-1]), "mse_of_mean": float(np.var(y)),
                    "train_mse_by_round": by_round}
        _, cls = f.b.predict(X, want_class=True)
        return {"boost_train_cross_entropy": float(loss[-1]),
                "cross_entropy_by_round": by_round,
                "train_error": float(np.mean(cls != wl.labels))}
    return tree_loss(ctx, f, wl, X)


def time_steps(ctx, p, X, L, Y, steps, flush, stream, cfg=None):
    """K timed steps: device time of each from events on the stream."""
    import torch
    times, evals = [], 0
    launches0 = ctx.launch_count()
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        f = train_step(ctx, p, cfg or {}, X, L, Y)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        evals += f.info()["evaluations"]
        f.free()
    return times, evals, ctx.launch_count() - launches0


def measured_roofs(device, stream):
    """FP32 FFMA and L2-read roofs from the library's microbenchmarks
    (slm_measure_peaks), or the derived FFMA rate and HBM copy when they fail."""
    from paper_2208_07023_gb300 import binding as S
    try:
        m = S.measure_peaks(device, stream)
        return {"ffma_tflops": m["ffma_tflops"], "l2_gbs": m["l2_read_gbs"],
                "ffma_source": "measured: slm_measure_peaks FFMA chains (16 per thread, "
                               "64 warps per SM), best of 3 launches",
                "l2_source": "measured: slm_measure_peaks 48 MB L2-resident buffer, "
                             "16-byte cache-global loads, best of 3 launches"}
    except Exception as e:  # noqa: BLE001
        return {"ffma_tflops": FP32_PEAK_TFLOPS, "l2_gbs": HBM_PEAK_GBS,
                "ffma_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz (%s)" % e,
                "l2_source": "HBM copy (%s)" % PEAK_SOURCE}


def rooflines(kst, wl, cfg, proj, topk, workload, roofs_in=None):
    """Per-kernel roofline from the profiled pass."""
    P, d = cfg["n_particles"], wl.d
    mr = roofs_in or {"ffma_tflops": FP32_PEAK_TFLOPS, "l2_gbs": HBM_PEAK_GBS,
                      "ffma_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz",
                      "l2_source": "HBM copy"}
    ffma, l2 = mr["ffma_tflops"], mr["l2_gbs"]
    dp = (d + 15) // 16 * 16
    roofs = {}
    kp, kh, km = kst["project"], kst["hist_scan"], kst["project_mma"]
    kn = kst.get("node_search", {"ms": 0.0})
    if kn["ms"] > 0:
        # whole searches of shared-memory-resident nodes: 2 d flop per
        # particle-sample evaluation (the kernel projects twice: range, bins)
        ach = 2.0 * d * kn["pairs"] / (kn["ms"] / 1e3) / 1e12
        roofs["node_search"] = {"kernel": "node_search", "bound": "alu", "achieved": ach,
                                "peak": ffma, "unit": "TFLOP/s",
                                "frac": ach / ffma, "traffic": None,
                                "avg_launch_ms": kn["ms"] / max(1, kn["launches"]),
                                "peak_source": mr["ffma_source"]}
    if kp["ms"] > 0:
        # FP32 FFMA: 2 d flop per particle-sample pair
        ach = 2.0 * d * kp["pairs"] / (kp["ms"] / 1e3) / 1e12
        roofs["project"] = {"kernel": "project", "bound": "alu", "achieved": ach,
                            "peak": ffma, "unit": "TFLOP/s",
                            "frac": ach / ffma,
                            "traffic": traffic_per_launch("project", kp, workload),
                            "avg_launch_ms": kp["ms"] / max(1, kp["launches"]),
                            "peak_source": mr["ffma_source"]}
    if kh["ms"] > 0:
        # z (4 B per pair) + per entry and pass its label (4 B) or, for MSE,
        # its two 8-byte fixed-point moments (+ a 4-byte multiplicity when
        # weighted); the bf16 form scans P and then k particles per entry
        per_entry = P if proj != "bf16" else (P + topk) / 2.0
        weighted = cfg.get("bootstrap", cfg["n_trees"] > 1)
        entry_b = (16.0 if cfg["criterion"] == "mse" else 4.0) + (4.0 if weighted else 0.0)
        algo = kh["pairs"] * (4.0 + entry_b / per_entry)
        ach = algo / (kh["ms"] / 1e3) / 1e9
        # the projections, labels and moments it reads are L2-resident
        roofs["hist_scan"] = {"kernel": "hist_scan", "bound": "l2", "achieved": ach,
                              "peak": l2, "unit": "GB/s", "frac": ach / l2,
                              "traffic": traffic_per_launch("hist_scan", kh, workload),
                              "avg_launch_ms": kh["ms"] / max(1, kh["launches"]),
                              "peak_source": mr["l2_source"]}
    if km["ms"] > 0:
        # bf16 rows read once per launch: dp * 2 bytes per entry = pairs / P
        algo = km["pairs"] / P * dp * 2.0
        ach = algo / (km["ms"] / 1e3) / 1e9
        tfl = 2.0 * d * km["pairs"] / (km["ms"] / 1e3) / 1e12
        roofs["project_mma"] = {"kernel": "project_mma", "bound": "hbm", "achieved": ach,
                                "peak": HBM_PEAK_GBS, "unit": "GB/s",
                                "frac": ach / HBM_PEAK_GBS, "traffic": None,
                                "avg_launch_ms": km["ms"] / max(1, km["launches"]),
                                "tensor": {"achieved_tflops": tfl, "peak": BF16_PEAK_TFLOPS,
                                           "frac": tfl / BF16_PEAK_TFLOPS},
                                "peak_source": f"{PEAK_SOURCE} (MEASURED_PEAKS.json)"}
    return roofs


def apply_launch_options(ctx, args):
    ctx.set_graphs(args.graphs == "on")
    ctx.set_projection_tma(args.tma == "on")
    ctx.set_fused_step(args.fused != "off", always=args.fused == "always")
    ctx.set_class_hist(args.class_hist == "on", args.node_step == "on")
    if args.node_search != "default":
        ctx.set_node_search(args.node_search == "on")
    if args.tiles == "fixed":
        ctx.set_tuning(False)
    elif args.tiles != "auto":
        v = [int(x) for x in args.tiles.split(":")]
        ctx.force_tiles(v[0], v[1], bool(v[2]) if len(v) > 2 else False)


def reduce_over_ranks(ms, evals, world, device):
    """(the slowest rank's time, the evaluations of all ranks): each rank
    grows its own trees, so the job's throughput is the total work over the
    time of the slowest rank."""
    if world <= 1:
        return ms, float(evals)
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms, float(evals)], dtype=torch.float64, device=device)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = t.clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return mx[0].item(), sm[1].item()


def rank_seed(rank):
    """Workload seed of a rank for single-tree workloads: every rank trains
    its own tree on its own data (independent problems, weak scaling)."""
    return 1 + rank


def rank_forest_share(n_trees, rank, world):
    """Trees of one forest that rank `rank` of `world` grows: r, r + N, ...
    as (first global tree id, stride, count). The ranks share the data; each
    tree's bootstrap draw and swarm streams are keyed by its global id, so
    the ranks' trees together are exactly the forest one rank would grow."""
    return rank, world, len(range(rank, n_trees, world))


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2208_07023_gb300 import binding as S

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    name, proj, topk = args.workload, args.proj, args.topk
    cfg = W.SETTINGS[name]
    forest_split = cfg["n_trees"] > 1 and world > 1 and not cfg.get("rounds")
    if forest_split:
        # one forest split across the ranks: the same data, trees r, r + N, ...
        wl = cfg["builder"](1)
        first, stride, count = rank_forest_share(cfg["n_trees"], rank, world)
        cfg = dict(cfg, n_trees=max(1, count))
    else:
        wl = cfg["builder"](rank_seed(rank))  # each rank: its own tree
    X = torch.from_numpy(wl.X).cuda()
    L = torch.from_numpy(wl.labels).cuda() if wl.labels is not None else None
    Y = torch.from_numpy(wl.y).cuda() if wl.y is not None else None
    stream = torch.cuda.current_stream()
    ctx = S.Context(local, stream.cuda_stream)
    apply_launch_options(ctx, args)
    if forest_split:
        ctx.set_tree_ids(first, stride)
    p = make_params(S, cfg, wl, proj, topk)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    clocks = ClockSampler(gpu_uuid(local)).start()  # running before the timed region
    roofs_measured = measured_roofs(local, stream.cuda_stream)
    for _ in range(args.warmup):
        train_step(ctx, p, cfg, X, L, Y).free()

    # timed region: K trees, device time per tree from events on the stream
    barrier()
    wall0 = time.perf_counter()
    clocks.mark_start()
    try:
        times, evals, launches = time_steps(ctx, p, X, L, Y, args.steps, flush, stream, cfg)
        barrier()
    finally:
        clocks.mark_end()
        clocks.stop()
    wall = time.perf_counter() - wall0

    # per-kernel timing: the same K trees again, every launch bracketed by
    # CUDA events on the context's stream (kept out of the timed region above,
    # whose launches it would slow)
    ctx.profile(True)
    for _ in range(args.steps):
        flush.zero_()
        train_step(ctx, p, cfg, X, L, Y).free()
    kst = ctx.kernel_stats()
    ctx.profile(False)

    tot_ms = sum(times)
    tot_ms_max, evals_all = reduce_over_ranks(tot_ms, evals, world, "cuda")
    value = evals_all / (tot_ms_max / 1e3)

    # training loss of the trees this form grows
    f = train_step(ctx, p, cfg, X, L, Y)
    loss = step_loss(ctx, f, wl, X)
    sl = None if isinstance(f, BoostRun) else split_loss(f, cfg["n_trees"])
    split_info = None
    if forest_split:
        # only the tree arrays travel: rank 0 assembles the whole forest in
        # global tree order (outside the timed region)
        mine = [(first + t * stride, f.export(t)) for t in range(count)]
        parts = [None] * world
        dist.all_gather_object(parts, mine)
        forest = dict(kv for part in parts for kv in part)
        split_info = {"ranks": world, "trees_of_rank": [len(x) for x in parts],
                      "trees_gathered": len(forest),
                      "tree_ids_complete": sorted(forest) == list(range(W.SETTINGS[name]["n_trees"])),
                      "rule": "rank r grows trees r, r + N, ... of one forest on the shared "
                              "data; tree t's bootstrap and swarm streams are keyed by t"}
    f.free()

    extra = {"tree_train_ms": tot_ms_max / args.steps, "evals_per_step": evals // args.steps,
             "wall_s": wall, "train_loss": loss,
             "search_loop": dict(ctx.graph_stats(), mode=(
                 "one CUDA graph launch per level search" if args.graphs == "on"
                 else "PDL-chained stream launches")),
             "projection_tiles": ctx.tuned_shapes(),
             "last_hist_cluster": ctx.tuning_stats()["last_hist_cluster"],
             "measured_roofs": roofs_measured}
    if split_info:
        extra["forest_split"] = split_info
    if sl is not None:
        extra["split_loss_sum"] = sl
    if (name == DEFAULT_WORKLOAD and proj == "fp32" and world == 1 and args.vs_plain == "on"):
        extra["vs_plain_fp32"] = vs_plain_fp32(
            ctx, S, cfg, wl, X, L, Y, flush, stream, args.steps,
            {"tree_train_ms": tot_ms / args.steps, "iters": cfg["n_iters"],
             "evaluations": evals // args.steps, "train_loss": loss, "split_loss_sum": sl})
    if (name == DEFAULT_WORKLOAD and proj == "fp32" and world == 1 and args.vs_prob == "on"):
        extra["vs_probabilistic"] = vs_probabilistic(ctx, S, cfg, wl, X, L, Y)
    if args.compare_plain and (cfg.get("top_n") or cfg.get("apso")):
        # the same tree without the pre-screen / adaptive PSO, same harness
        pp = make_params(S, dict(cfg, top_n=0, apso=False), wl, proj, topk)
        for _ in range(max(1, args.warmup)):
            ctx.train_tree(pp, X, labels=L, y=Y).free()
        tp, ep, _ = time_steps(ctx, pp, X, L, Y, args.steps, flush, stream)
        f = ctx.train_tree(pp, X, labels=L, y=Y)
        lossp = tree_loss(ctx, f, wl, X)
        f.free()
        extra["plain_form"] = {"tree_train_ms": sum(tp) / len(tp),
                               "value": ep / (sum(tp) / 1e3), "train_loss": lossp,
                               "speedup_of_variant": (sum(tp) / len(tp)) /
                               (tot_ms / args.steps)}
    if args.compare_plain and cfg.get("apso"):
        extra["apso_vs_plain_root"] = apso_quality(ctx, S, cfg, wl, proj, topk, X, L, Y)
    if args.compare_fp32 and proj == "bf16":
        # the plain FP32 form of the same workload, same harness
        p32 = make_params(S, cfg, wl, "fp32", topk)
        for _ in range(max(1, args.warmup)):
            ctx.train_tree(p32, X, labels=L, y=Y).free()
        t32, e32, _ = time_steps(ctx, p32, X, L, Y, args.steps, flush, stream)
        f = ctx.train_tree(p32, X, labels=L, y=Y)
        loss32 = tree_loss(ctx, f, wl, X)
        f.free()
        extra["fp32_form"] = {"tree_train_ms": sum(t32) / len(t32),
                              "value": e32 / (sum(t32) / 1e3), "train_loss": loss32,
                              "speedup_of_bf16_form": (sum(t32) / len(t32)) /
                              (tot_ms / args.steps)}

    # end to end: host (pinned) inputs in, tree arrays out, through the C ABI
    Xh = torch.from_numpy(wl.X).pin_memory()
    Lh = torch.from_numpy(wl.labels).pin_memory() if wl.labels is not None else None
    Yh = torch.from_numpy(wl.y).pin_memory() if wl.y is not None else None
    e2e_t, e2e_ev, d2h = [], 0, 0
    for _ in range(max(1, min(args.steps, 3))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        f = train_step(ctx, p, cfg, Xh, Lh, Yh)
        if isinstance(f, BoostRun):  # the per-round training MSE comes back
            d2h = f.b.train_mse.nbytes
        else:
            exports = [f.export(t) for t in range(cfg["n_trees"])]
            d2h = sum(v.nbytes for g in exports for v in g.values())
        e2e_t.append(time.perf_counter() - t0)
        e2e_ev += f.info()["evaluations"]
        f.free()
    e2e_value = e2e_ev / sum(e2e_t)
    h2d = wl.X.nbytes + (wl.labels.nbytes if wl.labels is not None else wl.y.nbytes)

    roofs = rooflines(kst, wl, cfg, proj, topk, name, roofs_measured)
    dom = max(roofs, key=lambda k: kst[k]["ms"])
    roofline = dict(roofs[dom])
    roofline["timing"] = "per-launch CUDA events in a second K-step pass"
    roofline["others"] = [v for k, v in roofs.items() if k != dom]
    share = {k: round(v["ms"] / max(1e-9, sum(x["ms"] for x in kst.values())), 4)
             for k, v in kst.items() if v["launches"]}
    extra["kernel_share"] = share
    extra["launches_per_step"] = launches / max(1, args.steps)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(cfg, wl, proj, topk)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tot_ms_max / args.steps, "higher_is_better": True,
            # one forest split across the ranks: fixed total work
            "scaling": "strong" if forest_split else "weak", "vs_baseline": None,
            "dtype": "bf16+f32" if proj == "bf16" else "f32",
            "data": "synthetic (seeded, workloads.py)",
            "config": config_dict(name, cfg, wl, proj, topk, extra, args),
            "clocks": clocks.summary(),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "roofline": roofline,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def proposal_training_pairs(ctx, S, seed0, mixture_seed):
    """(statistics, PSO-best direction) pairs: single-node pattern nodes
    (d = 16..256), mixture subsets like the classification-tree workload
    (d = 64, K = 10), and nodes of the evaluated mixture's distribution: the
    same mixture parameters (means, covariance) with independently drawn
    samples (sample seeds disjoint from the evaluated data), restricted to
    random class subsets as a tree's nodes are."""
    import numpy as np
    stats, dims, targets = [], [], []

    def add(X, lab, K, p, uid):
        r = ctx.node_split(p, X, labels=lab, node_uid=uid)
        st = ctx.node_stats(X, labels=lab, n_classes=K)
        t = np.zeros(256, np.float32)
        t[:X.shape[1]] = r["direction"]
        stats.append(st)
        dims.append(X.shape[1])
        targets.append(t)

    def subset(wl, K, rng, lo):
        keep = rng.choice(K, rng.integers(lo, K + 1), replace=False)
        m = np.isin(wl.labels, keep)
        remap = np.full(K, -1, np.int32)
        remap[np.sort(keep)] = np.arange(keep.size)
        return wl.X[m], remap[wl.labels[m]]

    rng = np.random.default_rng(seed0)
    for i in range(300):
        d = (16, 32, 64, 128, 256)[i % 5]
        wl = W.single_node(2000, d, 0.05, seed=seed0 + i)
        add(wl.X, wl.labels, 2, S.make_params("entropy", 2, n_particles=32, n_iters=50,
                                              n_bins=64, min_leaf=1, seed=i + 1), i)
    for i in range(100):
        X, lab = subset(W.gmm(6000, 64, 10, seed=seed0 + 10_000 + i), 10, rng, 2)
        add(X, lab, 10, S.make_params("gini", 10, n_particles=64, n_iters=50, n_bins=128,
                                      min_leaf=20, seed=i + 7), i)
    for i in range(600):
        wl = W.gmm(20_000, 256, 20, seed=mixture_seed, sample_seed=seed0 + 20_000 + i)
        X, lab = subset(wl, 20, rng, 12)
        add(X, lab, 20, S.make_params("gini", 20, n_particles=64, n_iters=50, n_bins=128,
                                      min_leaf=20, seed=i + 9,
                                      proj=S.SLM_PROJ_BF16_TOPK, topk=8), i)
    return (np.array(stats, np.float32), np.array(dims, np.int32),
            np.array(targets, np.float32))


def run_proposal_eval(args):
    """The learned proposal on a large mixture: PSO iterations (seeded vs
    plain) to reach the plain search's split loss, median over the internal
    nodes of the first four levels of the plain tree."""
    import numpy as np
    import torch

    from paper_2208_07023_gb300 import binding as S
    cfg = W.SETTINGS[args.workload]
    stream = torch.cuda.current_stream()
    ctx = S.Context(0, stream.cuda_stream)
    t0 = time.perf_counter()
    st, dims, tg = proposal_training_pairs(ctx, S, 500_000, mixture_seed=1)
    t_pairs = time.perf_counter() - t0
    prop = ctx.proposal(seed=11)
    t0 = time.perf_counter()
    losses = prop.train(st, dims, tg, epochs=30, batch=64, lr=1e-3, seed=3)
    t_train = time.perf_counter() - t0
    wl = cfg["builder"](1)
    X = torch.from_numpy(wl.X).cuda()
    L = torch.from_numpy(wl.labels).cuda()
    p = make_params(S, cfg, wl, args.proj, args.topk)
    f = ctx.train_tree(p, X, labels=L)
    g = f.export(0)
    _, _, leaf = ctx.predict(f, X, want_leaf=True)
    f.free()
    leaf = leaf[:, 0].astype(np.int64)
    inner = [int(h) for h in np.nonzero(g["kind"] == 1)[0] if h < 15]
    ctx.use_proposal(prop)
    rows = []
    for h in inner:
        node = leaf.copy()
        member = node == h
        while (node > h).any():
            node = np.where(node > h, (node - 1) // 2, node)
            member |= node == h
        idx = torch.from_numpy(np.nonzero(member)[0].astype(np.int32)).cuda()
        res = {}
        for seeded in (False, True):
            ps = make_params(S, cfg, wl, args.proj, args.topk)
            ps.seeded = 1 if seeded else 0
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = ctx.node_split(ps, X, labels=L, sample_idx=idx, node_uid=h, want_trace=True)
            e1.record(stream)
            e1.synchronize()
            res[seeded] = (r["trace"], e0.elapsed_time(e1))
        target = res[False][0][-1]
        it_plain = int(np.argmax(res[False][0] <= target))
        hit = np.nonzero(res[True][0] <= target)[0]
        # within 1e-3 of the plain final loss: on separable classes many
        # class-group splits score within a few 1e-4 of each other
        near_p = int(np.argmax(res[False][0] <= target + 1e-3))
        near_s = np.nonzero(res[True][0] <= target + 1e-3)[0]
        rows.append({"node": h, "n": int(idx.numel()), "iters_plain": it_plain,
                     "iters_seeded": int(hit[0]) if hit.size else None,
                     "iters_within_1e-3_plain": near_p,
                     "iters_within_1e-3_seeded": int(near_s[0]) if near_s.size else None,
                     "first_plain": float(res[False][0][0]), "first_seeded": float(res[True][0][0]),
                     "final_plain": float(target), "final_seeded": float(res[True][0][-1]),
                     "ms_plain": res[False][1], "ms_seeded": res[True][1]})
    T = cfg["n_iters"]

    def med(key):
        return float(np.median([r[key] if r[key] is not None else T + 1 for r in rows]))

    # whole trees: plain FP32 and plain BF16 against the seeded BF16 form, at
    # T iterations and at T / 4
    trees = {}
    for name, proj, seeded, iters in (("plain_fp32", "fp32", False, T),
                                      ("plain_bf16", "bf16", False, T),
                                      ("seeded_bf16", "bf16", True, T),
                                      ("seeded_bf16_T/4", "bf16", True, T // 4)):
        ps = make_params(S, dict(cfg, n_iters=iters), wl, proj, args.topk)
        ps.seeded = 1 if seeded else 0
        ctx.train_tree(ps, X, labels=L).free()  # warm-up
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ft = ctx.train_tree(ps, X, labels=L)
        e1.record(stream)
        e1.synchronize()
        trees[name] = dict(tree_loss(ctx, ft, wl, X), ms=e0.elapsed_time(e1), iters=iters,
                           evaluations=ft.info()["evaluations"])
        ft.free()
    ctx.use_proposal(None)
    prop.free()
    head = trees["seeded_bf16"]
    line = {"metric": METRIC, "value": head["evaluations"] / (head["ms"] / 1e3), "unit": UNIT,
            "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": head["ms"],
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16+f32",
            "data": "synthetic (seeded, workloads.py)",
            "config": config_dict(args.workload, cfg, wl, args.proj, args.topk, {
                "step": "one seeded bf16 tree (the value); plain trees beside it",
                "proposal": {
                    "iterations_to_plain_loss_median": {
                        "plain": med("iters_plain"), "seeded": med("iters_seeded"),
                        "nodes": "internal nodes of the plain tree's first four levels; "
                                 "T + 1 = never"},
                    "iterations_to_within_1e-3_median": {
                        "plain": med("iters_within_1e-3_plain"),
                        "seeded": med("iters_within_1e-3_seeded")},
                    "first_loss_median": {
                        "plain": float(np.median([r["first_plain"] for r in rows])),
                        "seeded": float(np.median([r["first_seeded"] for r in rows]))},
                    "final_loss_median": {
                        "plain": float(np.median([r["final_plain"] for r in rows])),
                        "seeded": float(np.median([r["final_seeded"] for r in rows]))},
                    "trees": trees,
                    "nodes": rows, "training_pairs": int(dims.size),
                    "pair_generation_s": t_pairs, "train_s": t_train,
                    "epoch_loss_first_last": [float(losses[0]), float(losses[-1])]}})}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_ncu_case(args):
    """The small case for full ncu captures of the scoring kernels: one search
    of the workload's root node with 3 iterations, a handful of launches (for
    a forest: the root level of every tree, one batched search, as the
    forest's first level runs it, tiles tuned first)."""
    import torch

    from paper_2208_07023_gb300 import binding as S
    cfg = W.SETTINGS[args.workload]
    wl = cfg["builder"](1)
    ctx = S.Context(0, torch.cuda.current_stream().cuda_stream)
    apply_launch_options(ctx, args)
    p = make_params(S, cfg, wl, args.proj, args.topk)
    p.n_iters = 3
    if cfg["n_trees"] > 1:
        p.max_depth = 1
        f = ctx.forest_begin(p, wl.X, labels=wl.labels, y=wl.y)
        n_split = f.grow_level()
        f.free()
        out = {"n_split": n_split, "tiles": ctx.tuned_shapes()}
    else:
        r = ctx.node_split(p, wl.X, labels=wl.labels, y=wl.y)
        out = {"loss": r["loss"], "bin": r["bin"]}
    print(json.dumps(dict({"ncu_case": args.workload, "proj": args.proj}, **out)), flush=True)
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(W.SETTINGS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--proj", choices=["fp32", "bf16"], default=None)
    ap.add_argument("--topk", type=int, default=8)
    ap.add_argument("--compare-fp32", action="store_true")
    ap.add_argument("--tma", choices=["on", "off"], default="on",
                    help="FP32 projection staging: tensor-map tile copies (on) or "
                         "per-thread asynchronous copies (off)")
    ap.add_argument("--fused", choices=["on", "always", "off"], default="on",
                    help="plain FP32 searches: swarm move folded into the projection "
                         "(two launches per iteration) where a level's projection is a "
                         "few waves (on), wherever possible (always), or never (off)")
    ap.add_argument("--class-hist", choices=["on", "off"], default="on",
                    help="classification histograms: latency-oriented kernel (on) or the "
                         "staged-copy kernel (off)")
    ap.add_argument("--node-step", choices=["on", "off"], default="off",
                    help="folded classification searches: gbest step and move in the last "
                         "histogram block of each node (on) or in every projection block (off)")
    ap.add_argument("--node-search", choices=["default", "on", "off"], default="default",
                    help="classification nodes whose rows fit in shared memory: the whole "
                         "search in one persistent cluster launch (on) or per-iteration kernels")
    ap.add_argument("--vs-plain", choices=["on", "off"], default="on",
                    help="default workload: also time the BF16 top-8 and learned-seeded forms "
                         "beside plain FP32 (config.vs_plain_fp32)")
    ap.add_argument("--vs-prob", choices=["on", "off"], default="on",
                    help="default workload: also run root searches of the probabilistic search "
                         "(Sec. II-B) beside the swarm (config.vs_probabilistic)")
    ap.add_argument("--apso", action="store_true",
                    help="adaptive PSO (FP32 form): the workload's searches adapt inertia "
                         "and learning factors to the swarm's evolutionary state")
    ap.add_argument("--compare-plain", action="store_true",
                    help="with a pre-screen or --apso: also time the plain tree")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--graphs", choices=["on", "off"], default=None,
                    help="run each search's iteration loop as one CUDA graph launch "
                         "(default: the workload's setting, else off)")
    ap.add_argument("--tiles", default="auto",
                    help="projection tiles: auto (tuned), fixed (16 particles, 2 CTAs/SM) "
                         "or PG:CPS[:GATHER]")
    ap.add_argument("--ncu-case", action="store_true",
                    help="one root-node search with 3 iterations (small case for ncu)")
    args = ap.parse_args()
    if args.proj is None:
        args.proj = W.SETTINGS[args.workload].get("proj", "fp32")
    if args.graphs is None:
        args.graphs = "on" if W.SETTINGS[args.workload].get("graphs") else "off"
    if args.apso:
        W.SETTINGS[args.workload]["apso"] = True
    if args.impl == "reference":
        return run_reference(args)
    if args.ncu_case:
        return run_ncu_case(args)
    if args.workload == "proposal_n1m_d256_k20":
        return run_proposal_eval(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
