#!/usr/bin/env python
"""Benchmark: SLM tree training with PSO split search on GB300.

A step is one full tree grown through libslm's C ABI (slm_train_tree): every
level's nodes searched in one batch by the particle swarm, then partitioned.
The workload is the classification tree of 50,000 samples x 64 features, 10
Gaussian-mixture classes, depth <= 8, min leaf 20, P=64 particles, T=100
iterations, 128 bins, Gini. The metric is particle-sample evaluations per
second: sum over searched nodes of n_node * P * (T+1), divided by the time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

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
WORKLOAD = "tree_n50k_d64_k10"
# FP32 fused multiply-add peak: 152 SMs x 128 FP32 lanes x 2 flop x 2.070 GHz.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
L2_FLUSH_BYTES = 256 << 20


def _measured_hbm_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except Exception:
        return 6800.0  # fallback figure for a GB300 copy


HBM_PEAK_GBS = _measured_hbm_gbs()

# DRAM bytes per particle-sample pair from ncu captures of the bench workload
# (dram__bytes_read.sum + dram__bytes_write.sum, profiles/), valid only for
# the kernel source they were taken from (sha256 of csrc/eval_kernels.cu).
TRAFFIC = {"project": 12849920 / 3.2e6, "hist_scan": 13091328 / 3.2e6}
TRAFFIC_SOURCE_SHA = "ce91b6f59265ae321156e8251a0a80b435982ce0e13bb604e2fb533d1297ceb0"


def _kernel_source_sha():
    import hashlib
    p = os.path.join(ROOT, "paper_2208_07023_gb300", "csrc", "eval_kernels.cu")
    with open(p, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def traffic_per_launch(name, ks):
    """Captured DRAM bytes per pair x the average pairs of a launch, or None
    once the kernel source differs from the captured one."""
    if name not in TRAFFIC or TRAFFIC_SOURCE_SHA != _kernel_source_sha():
        return None
    return TRAFFIC[name] * ks["pairs"] / max(1, ks["launches"])


def config_dict(cfg, extra=None):
    d = {"workload": WORKLOAD, "n": 50_000, "d": 64, "classes": 10,
         "max_depth": cfg["max_depth"], "min_leaf": cfg["min_leaf"],
         "particles": cfg["n_particles"], "iters": cfg["n_iters"], "bins": cfg["n_bins"],
         "criterion": cfg["criterion"], "projection": "fp32 ffma",
         "l2": "flushed between steps (256 MiB write outside the timed events)"}
    if extra:
        d.update(extra)
    return d


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").strip().splitlines():
            f = [t.strip() for t in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_uuid(dev: int) -> str:
    import torch
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        return vis.split(",")[dev] if vis else str(dev)


def oracle_root_sample(cfg, wl, iters):
    """Times the CPU oracle's swarm search of the root node (all n samples)
    with `iters` iterations; returns (evals/s, seconds, threads)."""
    import oracle as O
    p = O.make_params(cfg["criterion"], wl.n_classes, cfg["n_particles"], iters,
                      cfg["n_bins"], min_leaf=cfg["min_leaf"], seed=1,
                      precision=O.F32_MIRROR)
    t0 = time.perf_counter()
    O.node_split(p, wl.X, wl.labels, node_uid=0)
    dt = time.perf_counter() - t0
    evals = wl.n * cfg["n_particles"] * (iters + 1)
    return evals / dt, dt, os.cpu_count()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cfg = W.SETTINGS[WORKLOAD]
    wl = cfg["builder"](1)
    iters = 10
    for _ in range(args.warmup):
        oracle_root_sample(cfg, wl, iters)
    vals, secs = [], []
    for _ in range(args.steps):
        v, dt, cores = oracle_root_sample(cfg, wl, iters)
        vals.append(v)
        secs.append(dt)
    value = wl.n * cfg["n_particles"] * (iters + 1) * len(secs) / sum(secs)
    sample = (f"root-node swarm search of the same workload: {wl.n} samples x "
              f"{cfg['n_particles']} particles x {iters + 1} evaluations per step "
              f"(fp32-mirror oracle, OpenMP over particles)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(secs) / len(secs), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config_dict(cfg, {"sample": "root node, 11 evaluations"}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


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

    cfg = W.SETTINGS[WORKLOAD]
    wl = cfg["builder"](1 + rank)  # each rank: its own tree
    X = torch.from_numpy(wl.X).cuda()
    L = torch.from_numpy(wl.labels).cuda()
    stream = torch.cuda.current_stream()
    ctx = S.Context(local, stream.cuda_stream)
    p = S.make_params(cfg["criterion"], wl.n_classes, n_particles=cfg["n_particles"],
                      n_iters=cfg["n_iters"], n_bins=cfg["n_bins"],
                      min_leaf=cfg["min_leaf"], max_depth=cfg["max_depth"], seed=1)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def step():
        f = ctx.train_tree(p, X, labels=L)
        ev = f.info()["evaluations"]
        return f, ev

    for _ in range(args.warmup):
        f, _ = step()
        f.free()

    # timed region: K trees, device time per tree from events on the stream
    launches0 = ctx.launch_count()
    times, evals = [], 0
    clocks = ClockSampler(gpu_uuid(local))
    barrier()
    wall0 = time.perf_counter()
    with clocks:
        for k in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            f, ev = step()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            evals += ev
            f.free()
        barrier()
    wall = time.perf_counter() - wall0
    launches = ctx.launch_count() - launches0

    # per-kernel timing: the same K trees again, every launch bracketed by
    # CUDA events on the context's stream (kept out of the timed region above,
    # whose launches it would slow)
    ctx.profile(True)
    for k in range(args.steps):
        flush.zero_()
        f, _ = step()
        f.free()
    kst = ctx.kernel_stats()
    ctx.profile(False)

    tot_ms = sum(times)
    if world > 1:
        t = torch.tensor([tot_ms, float(evals)], dtype=torch.float64, device="cuda")
        mx = t.clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        sm = t.clone()
        dist.all_reduce(sm, op=dist.ReduceOp.SUM)
        tot_ms_max, evals_all = mx[0].item(), sm[1].item()
    else:
        tot_ms_max, evals_all = tot_ms, float(evals)
    value = evals_all / (tot_ms_max / 1e3)

    # end to end: host (pinned) inputs in, tree arrays out, through the C ABI
    Xh = torch.from_numpy(wl.X).pin_memory()
    Lh = torch.from_numpy(wl.labels).pin_memory()
    e2e_t, e2e_ev, d2h = [], 0, 0
    for k in range(max(1, min(args.steps, 3))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        f = ctx.train_tree(p, Xh, labels=Lh)
        g = f.export(0)
        e2e_t.append(time.perf_counter() - t0)
        e2e_ev += f.info()["evaluations"]
        d2h = sum(v.nbytes for v in g.values())
        f.free()
    e2e_value = e2e_ev / sum(e2e_t)
    h2d = wl.X.nbytes + wl.labels.nbytes

    # rooflines: k_project is FP32-FFMA bound (2 d flop per particle-sample
    # pair); k_hist_scan streams z (4 B per pair) and labels (4 B per entry,
    # i.e. 4 / P per pair) and is memory bound
    roofs = {}
    kp, kh = kst["project"], kst["hist_scan"]
    if kp["ms"] > 0:
        ach = 2.0 * wl.d * kp["pairs"] / (kp["ms"] / 1e3) / 1e12
        roofs["project"] = {"kernel": "project", "bound": "alu", "achieved": ach,
                            "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                            "frac": ach / FP32_PEAK_TFLOPS,
                            "traffic": traffic_per_launch("project", kp),
                            "avg_launch_ms": kp["ms"] / max(1, kp["launches"]),
                            "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz"}
    if kh["ms"] > 0:
        algo = kh["pairs"] * (4.0 + 4.0 / cfg["n_particles"])
        ach = algo / (kh["ms"] / 1e3) / 1e9
        roofs["hist_scan"] = {"kernel": "hist_scan", "bound": "hbm", "achieved": ach,
                              "peak": HBM_PEAK_GBS, "unit": "GB/s", "frac": ach / HBM_PEAK_GBS,
                              "traffic": traffic_per_launch("hist_scan", kh),
                              "avg_launch_ms": kh["ms"] / max(1, kh["launches"]),
                              "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"}
    dom = max(kst, key=lambda k: kst[k]["ms"])
    roofline = dict(roofs.get(dom) or next(iter(roofs.values())))
    roofline["timing"] = "per-launch CUDA events in a second K-tree pass"
    roofline["others"] = [v for k, v in roofs.items() if k != roofline["kernel"]]
    share = {k: round(v["ms"] / max(1e-9, sum(x["ms"] for x in kst.values())), 4)
             for k, v in kst.items() if v["launches"]}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, dt, cores = oracle_root_sample(cfg, wl, cfg["n_iters"])
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": (f"root-node swarm search of the workload ({wl.n} samples x "
                          f"{cfg['n_particles']} particles x {cfg['n_iters'] + 1} "
                          f"evaluations, {dt:.1f} s; fp32-mirror oracle, OpenMP over "
                          "particles)")}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tot_ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded Gaussian mixture)",
            "config": config_dict(cfg, {"tree_train_ms": tot_ms_max / args.steps,
                                        "evals_per_tree": evals // args.steps,
                                        "wall_s": wall,
                                        "kernel_share": share}),
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
