#!/usr/bin/env python3
"""Benchmark of the multi-morphology HH + Hines stepper on one GB300 (or N).

A "step" is one time step dt of the whole network: spike delivery plus the
fused gates + currents + assembly + Hines solve + spike-detection kernel.
The metric is compartment-updates per second (compartments x steps / time).

Default workload: the 10,000-neuron multi-morphology network (compartment
counts log-uniform in [50, 5000], branch probability U[0.02, 0.2], 100
synapses per neuron, dt = 0.025 ms) in compensated FP32 (FP32c), in the
launch configuration of the library's defaults (CUDA graphs of 40 steps);
the plain FP64 path is timed on the same network beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--config multi10k] [--precision fp64|fp32c]

Under torchrun (N > 1) every rank runs its own replica of the workload
(weak scaling) and rank 0 prints the aggregate.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2005_06332_gb300 import netgen  # noqa: E402

METRIC = "compartment-updates/sec (HH+Hines per dt) on 1 GB300, % HBM roofline, vs plain FP64"
UNIT = "compartment-updates/s"
L2_BYTES = 129 * 1024 * 1024

# Algorithmic bytes per compartment-update of the fused step kernel:
# FP64 state V, m, h, n read + written (64 B) and the constants area, g_axial
# read (16 B); per synaptic site g_syn read + written and its index (20 B).
BYTES_PER_UPDATE = {"fp64": (80.0, 20.0),
                    # FP32c: int32 V and three uint32 gates read + written (32 B),
                    # FP32 area and g_axial read (8 B); per site FP32 g_syn r/w + index
                    "fp32c": (40.0, 12.0)}
# FP32c splits the step over one solve kernel per work-item class (regular
# and large shared-memory items, giant items), each also updating the gates
# of its compartments; their own algorithmic bytes (V and gates read and
# written, area and g_axial read; per site the conductance read + written
# and its index): V r/w 8 + gates r/w 24 + area, g_axial 8 = 40 B (+12 B per site)
KERNEL_BYTES_FP32C = {"step": (40.0, 12.0), "big": (40.0, 12.0), "giant": (40.0, 12.0)}

# Counters of one `ncu --set full` capture of the regular-class step kernel
# (profiles/step_fp32c_multi10k.md): DRAM bytes read + written and warp
# instructions executed per launch.  They describe the kernel built from the
# sources whose SHA-256 is recorded; after any change they are not reported.
KERNEL_SOURCES = ("mm_kernels_fp32c.cu", "mm_fp32c_math.h", "mm_internal.h", "mm_tma.h")
PROFILED = {
    ("multi10k", "fp32c", "step", "soma"): {
        "sha256": "be1015ab0833dee5de0afa9af58ab0b5f1968fe65f83e3d04d589f294fd3a729",
        "dram_bytes": 298201600 + 123973888,
        "warp_instructions": 350648274,
    },
}


def _kernel_sources_sha256():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2005_06332_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.rows = []
        self.proc = None
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            if self.thread is not None:
                self.thread.join(timeout=2)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, ws: int, device: str) -> float:
    """The largest x over the ranks of the process group (every rank gets it)."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, ws: int, seconds_slowest: float) -> float:
    """Whole-job rate: the units all ranks processed (each rank the same
    replica workload) over the slowest rank's time."""
    return units_per_rank * ws / seconds_slowest


def cpu_baseline(net, seconds_hint: float = 15.0, detect: str = "soma"):
    """The FP64 CPU oracle, as it stands, on a bounded sample of the workload."""
    import oracle
    rng = np.random.default_rng(0)
    k = min(net.n_neurons, 1000)
    pick = np.sort(rng.choice(net.n_neurons, k, replace=False))
    sub = net.subset(pick, keep_synapses=True)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    oracle.simulate(sub, 4, threads=cores, detect=detect)
    probe = max(1e-3, time.perf_counter() - t0)
    steps = int(max(8, min(400, 4 * seconds_hint / probe)))
    t0 = time.perf_counter()
    oracle.simulate(sub, steps, threads=cores, detect=detect)
    el = time.perf_counter() - t0
    return {"value": sub.n_comp * steps / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{k} of {net.n_neurons} neurons ({sub.n_comp} compartments, synapses among them), "
                      f"{steps} steps from rest, FP64 C oracle with OpenMP over neurons"}


def run_reference(args, net):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    rng = np.random.default_rng(0)
    k = min(net.n_neurons, 1000)
    pick = np.sort(rng.choice(net.n_neurons, k, replace=False))
    sub = net.subset(pick, keep_synapses=True)
    cores = os.cpu_count() or 1
    oracle.simulate(sub, max(1, args.warmup), threads=cores, detect=args.detect)
    t0 = time.perf_counter()
    oracle.simulate(sub, args.steps, threads=cores, detect=args.detect)
    el = time.perf_counter() - t0
    v = sub.n_comp * args.steps / el
    sample = (f"{k} of {net.n_neurons} neurons ({sub.n_comp} compartments, synapses among them), "
              f"{args.steps} steps after {args.warmup} warm-up steps")
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": net.name, "n_neurons": net.n_neurons, "n_comp": net.n_comp, "sampled": sample},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_paper_replay(args):
    """The paper's multi- vs mono-morphology tests (Sec. 4) on one GPU.

    10,000 neurons of mean size 300 in three workloads -- one morphology
    for all, sizes from a group of 20 (at most 700 apart), F-distributed
    sizes -- each timed (FP32c, CUDA graphs, CUDA events) with the work
    queue in size order (the paper's global sorting) and in a random order
    (no sorting).  Prints one JSON line with the step times and the
    overheads of the multi-morphology workloads over the mono-morphology
    one (the paper reports them for its CPU cluster: 12 % unsorted, 2.8 %
    after sorting)."""
    import torch
    from paper_2005_06332_gb300 import mm

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    mm.load()
    stream = torch.cuda.Stream(device=local)
    rng = np.random.default_rng(2019)
    res = {}
    for cfg in ("paper_mono", "paper_multi20", "paper_fisher"):
        net = netgen.make_config(cfg)
        sizes = net.sizes()
        r = {"n_comp": int(net.n_comp), "mean_size": float(sizes.mean()), "min_size": int(sizes.min()),
             "max_size": int(sizes.max())}
        for label, cost in (("size_sorted", None), ("random_order", rng.random(net.n_neurons).astype(np.float32))):
            g = mm.Network(net, precision="fp32c", graph_steps=args.graph_steps, device=local,
                           stream=stream.cuda_stream, cost=cost, block_threads=args.block_threads,
                           group_comps=args.group_comps)
            g.step(args.warmup)
            g.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.step(args.steps)
            e1.record(stream)
            e1.synchronize()
            r[label + "_ms_per_step"] = e0.elapsed_time(e1) / args.steps
            g.close()
        res[cfg] = r
    mono = res["paper_mono"]
    over = {}
    for cfg in ("paper_multi20", "paper_fisher"):
        for label in ("size_sorted", "random_order"):
            # per compartment, so that the small differences in total size cancel
            t = res[cfg][label + "_ms_per_step"] / res[cfg]["n_comp"]
            t0 = mono["size_sorted_ms_per_step"] / mono["n_comp"]
            over[f"{cfg}_{label}"] = t / t0 - 1.0
    print(json.dumps({"paper_replay": res, "overhead_vs_mono_per_compartment": over, "steps": args.steps,
                      "warmup": args.warmup, "precision": "fp32c", "data": "synthetic"}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="multi10k")
    ap.add_argument("--precision", default=None, choices=[None, "fp64", "fp32c"])
    ap.add_argument("--graph-steps", type=int, default=40)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--learned", action="store_true",
                    help="also learn the work-queue order (MLP cost model) and time it against size-sorted")
    ap.add_argument("--n-timed", type=int, default=5000)
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--block-threads", type=int, default=0)
    ap.add_argument("--group-comps", type=int, default=0)
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip the launch-configuration autotuner (default: tune on a 2M-compartment sample)")
    ap.add_argument("--detect", default="soma", choices=["soma", "points"],
                    help="threshold test at every soma, or at the points synapses leave from (each synapse "
                         "leaving a compartment drawn uniformly over its source neuron)")
    ap.add_argument("--deterministic", action="store_true",
                    help="deterministic event delivery (each site adds its events in ascending synapse id)")
    ap.add_argument("--paper-replay", action="store_true",
                    help="the paper's load-balance tests instead: one morphology vs a group of 20 sizes vs "
                         "F-distributed sizes (same mean size), size-sorted vs random work-queue order")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.paper_replay:
        run_paper_replay(args)
        return

    net = netgen.make_config(args.config, src_points=args.detect == "points")
    precision = args.precision or "fp32c"
    if args.impl == "reference":
        run_reference(args, net)
        return

    import torch
    from paper_2005_06332_gb300 import mm

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    mm.load()
    stream = torch.cuda.Stream(device=local)
    tune = None
    if not args.no_autotune and not (args.block_threads or args.group_comps):
        t0 = time.perf_counter()
        # candidates are timed on the whole network up to 16 M compartments
        # (a small sample gives each block too few items to show the load
        # balance of the full run), else on a stratified 16 M sample
        tune = mm.autotune(net, precision=precision, sample_comps=min(int(net.n_comp), 16_000_000), warmup=3,
                           steps=20, device=local, stream=stream.cuda_stream, graph_steps=args.graph_steps,
                           detect=args.detect)
        tune["seconds"] = time.perf_counter() - t0
        args.block_threads, args.group_comps = tune["block_threads"], tune["group_comps"]
    g = mm.Network(net, precision=precision, graph_steps=args.graph_steps, device=local, stream=stream.cuda_stream,
                   block_threads=args.block_threads, group_comps=args.group_comps, detect=args.detect,
                   deterministic=args.deterministic)

    launch = g.launch_info()
    # warm-up (also captures the CUDA graph)
    g.step(args.warmup)
    g.synchronize()

    # timed region: K steps, CUDA events on the launching stream; the state
    # (> 500 MB for the default workload) is larger than L2.
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        g.step(args.steps)
        ev1.record(stream)
        ev1.synchronize()
    torch.cuda.synchronize()
    ms = max_over_ranks(ev0.elapsed_time(ev1), ws, "cuda")
    if ws > 1:
        dist.barrier()
    G = args.graph_steps
    K = args.steps
    # kernels per step: delivery, then the solve of each non-empty work-item
    # class, then (FP32c) the gate update
    n_reg = launch["work_items"] - launch["big_items"] - launch["giant_items"]
    # (giant items: phase A, solve and phase C + gates, three kernels)
    kps = 2 if precision == "fp64" else 1 + (n_reg > 0) + (launch["big_items"] > 0) + 3 * (launch["giant_items"] > 0)
    launches = (K // G) * (kps * G + 1) + ((K % G > 0) * (kps * (K % G) + 1)) if G > 0 else kps * K + 1
    value = job_throughput(net.n_comp * K, ws, ms * 1e-3)

    # per-kernel times (events around each launch, direct launches)
    kt_steps = max(10, K // 4)
    g.set_kernel_timing(True)
    g.step(kt_steps)
    kt = g.read_kernel_timing(reset=True)
    g.set_kernel_timing(False)
    step_ms = kt["step_kernel_ms"] / max(1, kt["step_kernel_launches"])
    deliver_ms = kt["deliver_kernel_ms"] / max(1, kt["deliver_kernel_launches"])

    # end to end through the public API with host buffers: per step the soma
    # stimulus goes host -> device and the soma voltages and spikes come back.
    stim = np.ascontiguousarray(net.stim_nA, np.float64)
    soma = np.empty(net.n_neurons, np.float64)
    ke = args.e2e_steps
    # bytes each call moves: the stimulus and the control block's drain
    # write-back in; the soma voltages, the control block and the first
    # spike records (16 B each: time, neuron, compartment; more when more are
    # pending) out
    ctl_b = 32  # sizeof the control block
    pre = min(4096, g.spike_capacity)
    d2h = 0
    g.synchronize()
    t0 = time.perf_counter()
    for _ in range(ke):
        g.set_stimulus(stim)
        g.step(1)
        _, (sn, _sc, _st) = g.read_outputs(soma)
        d2h += 8 * net.n_neurons + ctl_b + 16 * pre + (16 * len(sn) if len(sn) > pre else 0)
    e2e_s = max_over_ranks(time.perf_counter() - t0, ws, "cuda")
    e2e = {"value": job_throughput(net.n_comp * ke, ws, e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": 8 * net.n_neurons + ctl_b, "d2h_bytes_per_step": int(round(d2h / ke)), "steps": ke,
           "calls_per_step": "mm_set_stimulus, mm_step(1), mm_read_outputs (soma voltages and spikes)"}

    peak, peak_kind = _peaks()
    b0, bsite = BYTES_PER_UPDATE.get(precision, (80.0, 20.0))
    nsite = int(np.unique(net.syn_comp.astype(np.int64) + net.comp_offset[net.syn_dst]).size)
    kernels = {"deliver": (deliver_ms, None)}
    if precision == "fp64":
        kernels["step"] = (step_ms, b0 * net.n_comp + bsite * nsite)
    else:
        # each solve kernel moves the bytes of the compartments and sites of
        # its own class (launch info)
        for cls, name in enumerate(("step", "big", "giant")):
            if launch["comps"][cls] > 0:
                k_ms = kt[f"{name}_kernel_ms"] / max(1, kt[f"{name}_kernel_launches"])
                kb = KERNEL_BYTES_FP32C[name]
                kernels[name] = (k_ms, kb[0] * launch["comps"][cls] + kb[1] * launch["sites"][cls])
    # the kernel that moves the most algorithmic bytes (FP32c giants run on a
    # side stream beside the other classes, so their times overlap)
    dom = max((k for k in kernels if kernels[k][1] is not None), key=lambda k: kernels[k][1])
    dom_ms, dom_bytes = kernels[dom]
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9
    prof = PROFILED.get((net.name, precision, dom, args.detect))
    if prof is not None and prof["sha256"] != _kernel_sources_sha256():
        prof = None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": prof["dram_bytes"] if prof else None,
                "traffic_gbs": (prof["dram_bytes"] / 1e9 / (dom_ms * 1e-3)) if prof else None,
                "peak_kind": peak_kind, "kernel": f"{dom}_{precision}",
                "kernel_ms": dom_ms, "bytes_per_launch": dom_bytes,
                "kernels_ms": {k: v[0] for k, v in kernels.items()},
                "step_bytes_per_update": f"{b0:g} B per compartment + {bsite:g} B per synaptic site",
                "step_achieved_gbs": (b0 * net.n_comp + bsite * nsite) / (ms / K * 1e-3) / 1e9}

    clocks = clk.summary()
    # the bound the step kernel meets in practice: instruction issue (four
    # schedulers per SM, one warp instruction each per cycle, at the SM clock
    # sampled during the timed region), with the executed warp instructions
    # of the profiled launch
    roofline_issue = None
    if prof is not None and clocks.get("sm_mhz"):
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        ipeak = 4.0 * sms * clocks["sm_mhz"] * 1e6
        iach = prof["warp_instructions"] / (dom_ms * 1e-3)
        roofline_issue = {"bound": "issue", "achieved": iach, "peak": ipeak, "unit": "warp-instructions/s",
                          "frac": iach / ipeak, "warp_instructions_per_launch": prof["warp_instructions"],
                          "per_compartment": prof["warp_instructions"] / launch["comps"][0]}
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": args.warmup,
           "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64" if precision == "fp64" else "f32", "data": "synthetic",
           "config": {"workload": net.name, "precision": precision, "n_neurons": net.n_neurons,
                      "block_threads": args.block_threads, "group_comps": args.group_comps,
                      "n_comp": net.n_comp, "n_syn": net.n_syn, "dt_ms": net.dt, "graph_steps": G,
                      "spike_detection": args.detect, "deterministic_delivery": args.deterministic,
                      "l2": f"inputs larger than L2 (state + constants {((48 if precision == 'fp64' else 24) * net.n_comp) / 1e6:.0f} MB)",
                      "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
           "roofline": roofline, "roofline_issue": roofline_issue, "e2e": e2e, "gpu_launches": launches,
           "clocks": clocks,
           "launch": launch, "autotune": tune}
    g.close()
    if args.learned:
        from paper_2005_06332_gb300 import schedule
        t0 = time.perf_counter()
        lc = schedule.learn_costs(net, n_timed=args.n_timed, steps=40, epochs=600, device=local)
        learn_s = time.perf_counter() - t0
        gl = mm.Network(net, precision=precision, graph_steps=args.graph_steps, device=local,
                        stream=stream.cuda_stream, cost=lc["cost"], block_threads=args.block_threads,
                        group_comps=args.group_comps)
        gl.step(args.warmup)
        gl.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        gl.step(K)
        e1.record(stream)
        e1.synchronize()
        ms_l = e0.elapsed_time(e1) / K
        gl.close()
        out["learned_schedule"] = {"ms_per_step": ms_l, "size_sorted_ms_per_step": ms / K,
                                   "gain": (ms / K) / ms_l - 1.0, "n_timed": int(len(lc["timed"])),
                                   "r2_holdout": lc["r2_holdout"], "r2_holdout_size_only": lc["r2_holdout_size_only"],
                                   "final_loss": float(lc["losses"][-1]), "learn_seconds": learn_s,
                                   "value": net.n_comp * ws / (ms_l * 1e-3)}
    if precision != "fp64" and not args.no_fp64:
        # the plain FP64 path on the same network, same launch configuration
        try:
            g64 = mm.Network(net, precision="fp64", graph_steps=args.graph_steps, device=local,
                             stream=stream.cuda_stream)
        except mm.MMError as exc:
            g64 = None
            out["plain_fp64"] = {"unavailable": str(exc)}
    if precision != "fp64" and not args.no_fp64 and g64 is not None:
        g64.step(3)
        g64.synchronize()
        k64 = max(10, min(K, 40))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g64.step(k64)
        e1.record(stream)
        e1.synchronize()
        ms64 = e0.elapsed_time(e1) / k64
        g64.close()
        v64 = net.n_comp * ws / (ms64 * 1e-3)
        out["plain_fp64"] = {"value": v64, "unit": UNIT, "ms_per_step": ms64, "steps": k64}
        out["speedup_vs_plain_fp64"] = value / v64
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(net, detect=args.detect)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
