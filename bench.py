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
FP64_MAX_NEURON_COMPS = 8192  # MM_FP64_MAX_NEURON_COMPS of include/mm.h

# Algorithmic bytes per compartment-update of the fused step kernel:
# FP64 state V, m, h, n read + written (64 B) and the constants area, g_axial
# read (16 B); per synaptic site g_syn read + written and its index (20 B).
BYTES_PER_UPDATE = {"fp64": (80.0, 20.0),
                    # FP32c: int32 V and three uint32 gates read + written (32 B),
                    # float-pair area, g_axial and passive diagonal read (24 B);
                    # per site the float-pair conductance r/w (16 B) + index (4 B)
                    "fp32c": (56.0, 20.0)}
# FP32c splits the step over one solve kernel per work-item class (regular
# and large shared-memory items, giant items), each also updating the gates
# of its compartments; each moves the same bytes per compartment and site
KERNEL_BYTES_FP32C = {"step": (56.0, 20.0), "big": (56.0, 20.0), "giant": (56.0, 20.0)}

# Counters of one `ncu --set full` capture of the regular-class step kernel
# on multi10k: DRAM bytes read + written and warp instructions executed per
# launch, with the compartments that launch updated.  They describe the
# kernel built from the sources whose SHA-256 is recorded; after any change
# they are not reported.
KERNEL_SOURCES = ("mm_kernels_fp32c.cu", "mm_fp32c_math.h", "mm_gate_table.h", "mm_internal.h", "mm_tma.h")
PROFILED = {
    # ncu counters of one regular-class launch of the step kernel (multi10k,
    # 512 threads, 4096-compartment items, a step inside the timed window)
    ("multi10k", "fp32c", "step", "soma"): {
        "sha256": "f442347e16f327b6adfd673c0fa934f5e2714eac09b925479dac6083f08d09c0",
        "dram_bytes": 495057920 + 111741184,
        "warp_instructions": 285126986,
        "comps": 9484756,
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
    # the same oracle on one core, over a tenth of the sample's neurons
    k1 = max(1, k // 10)
    sub1 = net.subset(pick[:: max(1, k // k1)][:k1], keep_synapses=True)
    steps1 = max(8, steps // 4)
    t0 = time.perf_counter()
    oracle.simulate(sub1, steps1, threads=1, detect=detect)
    el1 = time.perf_counter() - t0
    return {"value": sub.n_comp * steps / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{k} of {net.n_neurons} neurons ({sub.n_comp} compartments, synapses among them), "
                      f"{steps} steps from rest, FP64 C oracle with OpenMP over neurons",
            "one_core": {"value": sub1.n_comp * steps1 / el1, "unit": UNIT, "cores": 1,
                         "sample": f"{sub1.n_neurons} of those neurons ({sub1.n_comp} compartments), {steps1} steps"}}


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
    queue in size order (the paper's global sorting), in a random order (no
    sorting) and in the learned order (the MLP cost model trained on timed
    neurons of the same network).  Prints one JSON line with the step times and the
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
        lc = mm.train_schedule(net, n_timed=min(2000, net.n_neurons), steps=40, epochs=600, device=local,
                               stream=stream.cuda_stream)
        r["learned_r2_holdout"] = lc["r2_holdout"]
        r["size_only_r2_holdout"] = lc["r2_holdout_size_only"]
        for label, cost in (("size_sorted", None), ("random_order", rng.random(net.n_neurons).astype(np.float32)),
                            ("learned", lc["cost"])):
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
        for label in ("size_sorted", "random_order", "learned"):
            # per compartment, so that the small differences in total size cancel
            t = res[cfg][label + "_ms_per_step"] / res[cfg]["n_comp"]
            t0 = mono["size_sorted_ms_per_step"] / mono["n_comp"]
            over[f"{cfg}_{label}"] = t / t0 - 1.0
    print(json.dumps({"paper_replay": res, "overhead_vs_mono_per_compartment": over, "steps": args.steps,
                      "warmup": args.warmup, "precision": "fp32c", "data": "synthetic"}), flush=True)


def _timed(g, stream, K, settle, local, ws):
    """Advance the network `settle` steps untimed (past the first minimum
    delay, so that events flow), then time exactly K steps with CUDA events
    on the launching stream, barriers and synchronisation on both sides,
    nvidia-smi clocks sampled during the timed region.  Returns the slowest
    rank's ms, the clock summary and the spikes detected inside the window."""
    import torch
    g.step(settle)
    g.synchronize()
    g.read_spikes(allow_overflow=True)  # drain what the settling produced
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        g.step(K)
        ev1.record(stream)
        ev1.synchronize()
    torch.cuda.synchronize()
    ms = max_over_ranks(ev0.elapsed_time(ev1), ws, "cuda")
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    sn, _ = g.read_spikes(allow_overflow=True)
    return ms, clk.summary(), sn


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="multi10k",
                    help="multi10k (default; 10,000 neurons, log-uniform [50, 5000]), lognormal100k, mixed200k, mono64, "
                         "shapes10k, paper_mono, paper_multi20, paper_fisher")
    ap.add_argument("--precision", default=None, choices=[None, "fp64", "fp32c"])
    ap.add_argument("--scale", type=float, default=1.0,
                    help="shrink the workload's neuron count (and giant sizes) by this factor, for small profiling "
                         "cases of the same distributions")
    ap.add_argument("--graph-steps", type=int, default=40)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-learned", action="store_true",
                    help="time the size-sorted work queue only (default: also learn the order with the MLP cost "
                         "model and report the learned order's throughput as the value)")
    ap.add_argument("--n-timed", type=int, default=5000)
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--block-threads", type=int, default=0)
    ap.add_argument("--group-comps", type=int, default=0)
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip the launch-configuration autotuner")
    ap.add_argument("--detect", default="soma", choices=["soma", "points"],
                    help="threshold test at every soma, or at the points synapses leave from (each synapse "
                         "leaving a compartment drawn uniformly over its source neuron)")
    ap.add_argument("--deterministic", action="store_true",
                    help="deterministic event delivery (each site adds its events in ascending synapse id)")
    ap.add_argument("--paper-replay", action="store_true",
                    help="the paper's load-balance tests instead: one morphology vs a group of 20 sizes vs "
                         "F-distributed sizes (same mean size), size-sorted vs random vs learned work-queue order")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.paper_replay:
        run_paper_replay(args)
        return

    net = netgen.make_config(args.config, scale=args.scale, src_points=args.detect == "points")
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
    learned = precision == "fp32c" and not args.no_learned
    lc = None
    if learned:
        # the learned work-queue order (the target configuration): neurons
        # timed by the solve kernel, the MLP trained by the library's own
        # kernels, costs predicted for every neuron -- before the timed region
        t0 = time.perf_counter()
        lc = mm.train_schedule(net, n_timed=args.n_timed, steps=40, epochs=600, device=local,
                               stream=stream.cuda_stream)
        lc["seconds"] = time.perf_counter() - t0
    mk = lambda cost: mm.Network(net, precision=precision, graph_steps=args.graph_steps, device=local,
                                 stream=stream.cuda_stream, cost=cost, block_threads=args.block_threads,
                                 group_comps=args.group_comps, detect=args.detect, deterministic=args.deterministic)
    min_delay = int(round(float(np.min(net.syn_delay_ms)) / net.dt)) if net.n_syn else 0
    # untimed steps before the timed region: the warm-up (which also
    # captures the CUDA graphs), then past the first two minimum delays, so
    # that spikes are recorded and events delivered inside the timed window
    settle = args.warmup + 2 * (min_delay + 1)
    K = args.steps
    G = args.graph_steps

    g = mk(None)
    launch = g.launch_info()
    ms_size, clocks_size, sn_size = _timed(g, stream, K, settle, local, ws)
    timed_order = "size_sorted"
    g_timed, ms, clocks, sn_win = g, ms_size, clocks_size, sn_size
    if learned:
        gl = mk(lc["cost"])
        ms_l, clocks_l, sn_l = _timed(gl, stream, K, settle, local, ws)
        timed_order = "learned"
        g_timed, ms, clocks, sn_win = gl, ms_l, clocks_l, sn_l
        g.close()
    launch = g_timed.launch_info()
    # kernels per step: delivery, the solve of each non-empty work-item
    # class (giant items: phase A, solve, phase C + gates); every step runs
    # inside a CUDA graph (whole batches of G steps, the rest as one-step
    # graphs), each graph replay also advancing the device step counter
    n_reg = launch["work_items"] - launch["big_items"] - launch["giant_items"]
    kps = 2 if precision == "fp64" else 1 + (n_reg > 0) + (launch["big_items"] > 0) + 3 * (launch["giant_items"] > 0)
    if G > 0:
        launches = (K // G) * (kps * G + 1) + (K % G) * (kps + 1)
        launch_path = f"CUDA graphs: {K // G} replays of the {G}-step graph + {K % G} of the one-step graph"
    else:
        launches = kps * K + 1
        launch_path = "direct launches"
    value = job_throughput(net.n_comp * K, ws, ms * 1e-3)
    out_deg = np.bincount(net.syn_src, minlength=net.n_neurons) if net.n_syn else np.zeros(net.n_neurons, np.int64)
    window = {"spikes": int(len(sn_win)),
              "events_scheduled": int(out_deg[sn_win].sum()) if len(sn_win) and args.detect == "soma" else None,
              "steps_before": settle, "note": "spikes detected inside the timed steps; each schedules one event "
                                              "per outgoing synapse (delivered one delay later)"}

    # per-kernel times (events around each launch, direct launches)
    kt_steps = max(10, K // 4)
    g_timed.set_kernel_timing(True)
    g_timed.step(kt_steps)
    kt = g_timed.read_kernel_timing(reset=True)
    g_timed.set_kernel_timing(False)
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
    pre = min(4096, g_timed.spike_capacity)
    d2h = 0
    g_timed.synchronize()
    t0 = time.perf_counter()
    for _ in range(ke):
        g_timed.set_stimulus(stim)
        g_timed.step(1)
        _, (sn, _sc, _st) = g_timed.read_outputs(soma)
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
                "traffic": prof["dram_bytes"] * launch["comps"][0] / prof["comps"] if prof else None,
                "peak_kind": peak_kind, "kernel": f"{dom}_{precision}",
                "kernel_ms": dom_ms, "bytes_per_launch": dom_bytes,
                "kernels_ms": {k: v[0] for k, v in kernels.items()},
                "step_bytes_per_update": f"{b0:g} B per compartment + {bsite:g} B per synaptic site",
                "step_achieved_gbs": (b0 * net.n_comp + bsite * nsite) / (ms / K * 1e-3) / 1e9}
    # the bound the step kernel meets in practice: instruction issue (four
    # schedulers per SM, one warp instruction each per cycle, at the SM clock
    # sampled during the timed region), with the executed warp instructions
    # per compartment of the profiled launch
    roofline_issue = None
    if prof is not None and clocks.get("sm_mhz"):
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        ipeak = 4.0 * sms * clocks["sm_mhz"] * 1e6
        winst = prof["warp_instructions"] * launch["comps"][0] / prof["comps"]
        iach = winst / (dom_ms * 1e-3)
        roofline_issue = {"bound": "issue", "achieved": iach, "peak": ipeak, "unit": "warp-instructions/s",
                          "frac": iach / ipeak, "warp_instructions_per_launch": winst,
                          "per_compartment": prof["warp_instructions"] / prof["comps"]}
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": args.warmup,
           "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64" if precision == "fp64" else "f32", "data": "synthetic",
           "config": {"workload": net.name, "precision": precision, "n_neurons": net.n_neurons,
                      "work_queue_order": timed_order,
                      "block_threads": args.block_threads, "group_comps": args.group_comps,
                      "n_comp": net.n_comp, "n_syn": net.n_syn, "dt_ms": net.dt, "graph_steps": G,
                      "launch_path": launch_path,
                      "spike_detection": args.detect, "deterministic_delivery": args.deterministic,
                      "l2": f"inputs larger than L2 (state + constants "
                            f"{((48 if precision == 'fp64' else 40) * net.n_comp) / 1e6:.0f} MB)",
                      "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
           "timed_window": window,
           "roofline": roofline, "roofline_issue": roofline_issue, "e2e": e2e, "gpu_launches": launches,
           "clocks": clocks,
           "launch": launch, "autotune": tune}
    if learned:
        out["learned_schedule"] = {"ms_per_step": ms / K, "size_sorted_ms_per_step": ms_size / K,
                                   "gain": ms_size / ms - 1.0, "size_sorted_value": job_throughput(net.n_comp * K, ws,
                                                                                                   ms_size * 1e-3),
                                   "n_timed": lc["n_timed"], "r2_holdout": lc["r2_holdout"],
                                   "r2_holdout_size_only": lc["r2_holdout_size_only"],
                                   "final_loss": lc["final_loss"], "learn_seconds": lc["seconds"],
                                   "size_sorted_clocks": clocks_size}
    g_timed.close()
    if precision != "fp64" and not args.no_fp64:
        # the plain FP64 path on the same network (its own default launch
        # configuration), timed the same way over a shorter window
        k64 = max(10, min(K, 40))
        big = net.sizes() > FP64_MAX_NEURON_COMPS
        if not big.any():
            g64 = mm.Network(net, precision="fp64", graph_steps=args.graph_steps, device=local,
                             stream=stream.cuda_stream)
            ms64, _, _ = _timed(g64, stream, k64, 3, local, ws)
            g64.close()
            v64 = job_throughput(net.n_comp * k64, ws, ms64 * 1e-3)
            out["plain_fp64"] = {"value": v64, "unit": UNIT, "ms_per_step": ms64 / k64, "steps": k64}
            out["speedup_vs_plain_fp64"] = value / v64
        else:
            # the FP64 path holds no neuron above its per-neuron limit: both
            # paths are timed on the network without those neurons (synapses
            # among the rest kept), FP32c in the launch configuration above
            sub = net.subset(np.flatnonzero(~big), keep_synapses=True)
            res = {}
            for prec in ("fp64", "fp32c"):
                kw = {} if prec == "fp64" else {"block_threads": args.block_threads, "group_comps": args.group_comps}
                gs = mm.Network(sub, precision=prec, graph_steps=args.graph_steps, device=local,
                                stream=stream.cuda_stream, **kw)
                ms_s, _, _ = _timed(gs, stream, k64, 3, local, ws)
                gs.close()
                res[prec] = (job_throughput(sub.n_comp * k64, ws, ms_s * 1e-3), ms_s / k64)
            out["plain_fp64"] = {"value": res["fp64"][0], "unit": UNIT, "ms_per_step": res["fp64"][1], "steps": k64,
                                 "workload": f"{net.name} without its {int(big.sum())} neurons above "
                                             f"{FP64_MAX_NEURON_COMPS} compartments ({sub.n_comp} of {net.n_comp} "
                                             f"compartments)",
                                 "fp32c_same_workload": {"value": res["fp32c"][0], "ms_per_step": res["fp32c"][1]}}
            out["speedup_vs_plain_fp64"] = res["fp32c"][0] / res["fp64"][0]
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(net, detect=args.detect)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
