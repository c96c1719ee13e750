"""Seeded synthetic network generator (inputs only; no simulation arithmetic).

This module draws the random inputs that both the CUDA path and the CPU
oracle consume: morphologies (compartment counts, parent arrays, cylinder
lengths and diameters), per-neuron soma stimulus amplitudes and synapses
(source, target neuron, target compartment, weight, delay).  It computes
nothing of the method itself: no geometry, no conductances, no kinetics.

Morphologies follow the paper's problem statement (Sec. 2): each neuron is a
tree of compartments numbered so that ``parent[i] < i`` with the soma at
index 0 (``parent[0] = -1``), which is the numbering that lets the Hines
algorithm (Algorithm 1) run in linear time.  Random trees are grown one
compartment at a time: with probability ``1 - p_branch`` a compartment
continues the current cable (``parent[i] = i - 1``), otherwise it starts a
new branch off a uniformly chosen earlier compartment.

Neuron-size distributions stand in for the paper's synthetic workloads (a
default size of 450 compartments and 500 synapses in Sec. 3.1, a 20-size
group in Sec. 4, F-distributed sizes in Sec. 4): see ``CONFIGS`` for the
five named workloads and ``make_network`` for arbitrary ones.

The random stream is NumPy's PCG64 seeded per workload; only ``random()``
and ``integers()`` draws are used so that the same seed gives the same
network on every platform.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence

import numpy as np

# Channel / cable / synapse parameters of the workloads (units: mS/cm^2, mV,
# uF/cm^2, ohm*cm, ms).  The paper names no channel model (Sec. 2 only says
# that the current I depends on V); these are the classic squid-axon values.
DEFAULT_PARAMS = dict(
    gNa=120.0, gK=36.0, gL=0.3,
    ENa=50.0, EK=-77.0, EL=-54.4,
    Cm=1.0, Ra=100.0,
    v_init=-65.0, threshold=0.0,
    tau_syn=2.0, e_syn=0.0,
)

SEED_BASE = 2019_0306


@dataclasses.dataclass
class Network:
    """A multi-morphology network, in user numbering.

    Arrays (all C-contiguous NumPy):
      comp_offset  int64[N+1]  neuron k owns compartments comp_offset[k]..comp_offset[k+1]-1
      parent       int32[C]    parent of each compartment, LOCAL index within its neuron;
                               -1 for the soma (local index 0), otherwise < local index
      length_um    float64[C]  cylinder length
      diam_um      float64[C]  cylinder diameter
      stim_nA      float64[N]  constant soma current injected from t = 0
      syn_src      int32[S]    presynaptic neuron
      syn_dst      int32[S]    postsynaptic neuron
      syn_comp     int32[S]    LOCAL compartment of the postsynaptic neuron
      syn_w        float64[S]  peak conductance increment (uS)
      syn_delay_ms float64[S]  axonal + synaptic delay
      syn_src_comp int32[S] or None: LOCAL compartment of the presynaptic
                   neuron the synapse leaves from (the point whose threshold
                   crossings it carries when spikes are detected at synapse
                   points); None: every synapse leaves from the soma
    """
    comp_offset: np.ndarray
    parent: np.ndarray
    length_um: np.ndarray
    diam_um: np.ndarray
    stim_nA: np.ndarray
    syn_src: np.ndarray
    syn_dst: np.ndarray
    syn_comp: np.ndarray
    syn_w: np.ndarray
    syn_delay_ms: np.ndarray
    params: dict
    dt: float = 0.025
    t_stop: float = 100.0
    name: str = "custom"
    syn_src_comp: Optional[np.ndarray] = None

    @property
    def n_neurons(self) -> int:
        return int(self.comp_offset.shape[0] - 1)

    @property
    def n_comp(self) -> int:
        return int(self.comp_offset[-1])

    @property
    def n_syn(self) -> int:
        return int(self.syn_src.shape[0])

    @property
    def n_steps(self) -> int:
        return int(round(self.t_stop / self.dt))

    def sizes(self) -> np.ndarray:
        return np.diff(self.comp_offset)

    def subset(self, neurons: Sequence[int], keep_synapses: bool = False) -> "Network":
        """Network made of the listed neurons only (renumbered 0..k-1).

        Synapses whose source and target both survive are kept when
        ``keep_synapses``; otherwise the subset has no synapses (isolated neurons).
        """
        neurons = np.asarray(neurons, dtype=np.int64)
        sizes = self.sizes()[neurons]
        off = np.zeros(len(neurons) + 1, dtype=np.int64)
        np.cumsum(sizes, out=off[1:])
        idx = np.concatenate([np.arange(self.comp_offset[k], self.comp_offset[k + 1]) for k in neurons]) \
            if len(neurons) else np.zeros(0, np.int64)
        remap = -np.ones(self.n_neurons, dtype=np.int64)
        remap[neurons] = np.arange(len(neurons))
        if keep_synapses and self.n_syn:
            keep = (remap[self.syn_src] >= 0) & (remap[self.syn_dst] >= 0)
        else:
            keep = np.zeros(self.n_syn, dtype=bool)
        return Network(
            comp_offset=off,
            parent=self.parent[idx].copy(),
            length_um=self.length_um[idx].copy(),
            diam_um=self.diam_um[idx].copy(),
            stim_nA=self.stim_nA[neurons].copy(),
            syn_src=remap[self.syn_src[keep]].astype(np.int32),
            syn_dst=remap[self.syn_dst[keep]].astype(np.int32),
            syn_comp=self.syn_comp[keep].copy(),
            syn_w=self.syn_w[keep].copy(),
            syn_delay_ms=self.syn_delay_ms[keep].copy(),
            params=dict(self.params), dt=self.dt, t_stop=self.t_stop,
            name=self.name + "-subset",
            syn_src_comp=None if self.syn_src_comp is None else self.syn_src_comp[keep].copy(),
        )


def random_tree(rng: np.random.Generator, n: int, p_branch: float) -> np.ndarray:
    """Parent array (local, int32) of an n-compartment random tree, parent[i] < i."""
    parent = np.empty(n, dtype=np.int32)
    parent[0] = -1
    if n > 1:
        i = np.arange(1, n, dtype=np.int64)
        jump = rng.random(n - 1) < p_branch
        target = np.floor(rng.random(n - 1) * i).astype(np.int64)
        target = np.minimum(target, i - 1)
        parent[1:] = np.where(jump, target, i - 1).astype(np.int32)
    return parent


def _normal(rng: np.random.Generator, k: int) -> np.ndarray:
    # Box-Muller from uniform draws (platform-stable stream).
    u1 = rng.random(k)
    u2 = rng.random(k)
    u1 = np.where(u1 <= 0.0, np.finfo(np.float64).tiny, u1)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def draw_sizes(rng: np.random.Generator, n_neurons: int, dist) -> np.ndarray:
    """Compartment counts.

    dist: ("mono", n) | ("loguniform", a, b) | ("lognormal", median, sigma, lo, hi)
          | ("choice", [sizes...])  (uniform over a fixed group of sizes)
          | ("group", k, spread, mean)  (k sizes drawn once, largest minus
            smallest = spread, group mean = mean; neurons pick among them)
          | ("fisher", d1, d2, mean, lo, hi)  (F(d1, d2)-distributed, scaled
            to the given mean, clipped)
    """
    kind = dist[0]
    if kind == "mono":
        return np.full(n_neurons, int(dist[1]), dtype=np.int64)
    if kind == "loguniform":
        a, b = float(dist[1]), float(dist[2])
        u = rng.random(n_neurons)
        return np.rint(np.exp(math.log(a) + u * (math.log(b) - math.log(a)))).astype(np.int64)
    if kind == "lognormal":
        med, sig, lo, hi = float(dist[1]), float(dist[2]), int(dist[3]), int(dist[4])
        z = _normal(rng, n_neurons)
        return np.clip(np.rint(med * np.exp(sig * z)), lo, hi).astype(np.int64)
    if kind == "choice":
        group = np.asarray(dist[1], dtype=np.int64)
        return group[rng.integers(0, len(group), size=n_neurons)]
    if kind == "group":
        # k sizes lo + spread * v^a with v uniform over [0, 1] (its smallest
        # draw mapped to 0, its largest to 1) and the exponent a chosen by
        # bisection so that the group's mean is `mean`
        k, spread, mean = int(dist[1]), float(dist[2]), float(dist[3])
        lo = 10.0
        v = np.sort(rng.random(k))
        v = (v - v[0]) / (v[-1] - v[0])
        a_lo, a_hi = 1e-3, 1e3
        for _ in range(200):
            a = math.sqrt(a_lo * a_hi)
            if lo + spread * float(np.mean(v ** a)) > mean:
                a_lo = a
            else:
                a_hi = a
        group = np.rint(lo + spread * v ** math.sqrt(a_lo * a_hi)).astype(np.int64)
        return group[rng.integers(0, k, size=n_neurons)]
    if kind == "fisher":
        # F = (X1 / d1) / (X2 / d2) with X chi-square (sums of squared normals)
        d1, d2, mean, lo, hi = int(dist[1]), int(dist[2]), float(dist[3]), int(dist[4]), int(dist[5])
        x1 = (_normal(rng, n_neurons * d1).reshape(n_neurons, d1) ** 2).sum(axis=1) / d1
        x2 = (_normal(rng, n_neurons * d2).reshape(n_neurons, d2) ** 2).sum(axis=1) / d2
        f = x1 / x2
        return np.clip(np.rint(mean * f * (d2 - 2.0) / d2), lo, hi).astype(np.int64)
    raise ValueError(f"unknown size distribution {dist!r}")


def make_network(
    n_neurons: int,
    size_dist=("mono", 255),
    p_branch=0.1,
    syn_per_neuron: int = 10,
    delay_ms=("const", 1.0),
    seed: int = SEED_BASE,
    mono_tree: bool = False,
    giants: int = 0,
    giant_size: int = 100_000,
    giant_p_branch: float = 0.05,
    length_um=(5.0, 20.0),
    diam_um=(0.5, 2.0),
    stim_nA=(0.1, 0.5),
    weight_uS=(0.0, 0.05),
    dt: float = 0.025,
    t_stop: float = 100.0,
    params: Optional[dict] = None,
    name: str = "custom",
    src_points: bool = False,
) -> Network:
    """Draw a network.

    p_branch: float, ("uniform", lo, hi) drawn per neuron, or ("choice", p1,
               p2, ...): each neuron one of the listed values, uniformly.
    mono_tree: every neuron shares one tree and one set of cylinder sizes
               (the paper's mono-morphology case, Sec. 3).
    giants:    extra neurons of ``giant_size`` compartments appended last.
    delay_ms:  ("const", d) or ("uniform", lo, hi).
    src_points: every synapse also leaves from a compartment drawn uniformly
               over its source neuron (drawn after everything else, so the
               rest of the network is the one drawn without it).
    """
    rng = np.random.default_rng(seed)
    sizes = draw_sizes(rng, n_neurons, size_dist)
    if giants:
        sizes = np.concatenate([sizes, np.full(giants, giant_size, dtype=np.int64)])
    n_tot = int(sizes.shape[0])
    off = np.zeros(n_tot + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    C = int(off[-1])

    if isinstance(p_branch, tuple):
        if p_branch[0] == "uniform":
            pb = p_branch[1] + rng.random(n_neurons) * (p_branch[2] - p_branch[1])
        elif p_branch[0] == "choice":
            vals = np.asarray(p_branch[1:], dtype=np.float64)
            pb = vals[np.minimum((rng.random(n_neurons) * len(vals)).astype(np.int64), len(vals) - 1)]
        else:
            raise ValueError(f"unknown branch-probability distribution {p_branch!r}")
    else:
        pb = np.full(n_neurons, float(p_branch))
    if giants:
        pb = np.concatenate([pb, np.full(giants, float(giant_p_branch))])

    parent = np.empty(C, dtype=np.int32)
    L = np.empty(C, dtype=np.float64)
    D = np.empty(C, dtype=np.float64)
    if mono_tree:
        n0 = int(sizes[0])
        tree = random_tree(rng, n0, float(pb[0]))
        l0 = length_um[0] + rng.random(n0) * (length_um[1] - length_um[0])
        d0 = diam_um[0] + rng.random(n0) * (diam_um[1] - diam_um[0])
        for k in range(n_tot):
            s, e = off[k], off[k + 1]
            if e - s != n0:
                raise ValueError("mono_tree needs equal sizes")
            parent[s:e] = tree
            L[s:e] = l0
            D[s:e] = d0
    else:
        for k in range(n_tot):
            s, e = int(off[k]), int(off[k + 1])
            parent[s:e] = random_tree(rng, e - s, float(pb[k]))
        L[:] = length_um[0] + rng.random(C) * (length_um[1] - length_um[0])
        D[:] = diam_um[0] + rng.random(C) * (diam_um[1] - diam_um[0])

    stim = stim_nA[0] + rng.random(n_tot) * (stim_nA[1] - stim_nA[0])

    # Synapses: syn_per_neuron incoming synapses per neuron, source uniform over
    # the other neurons, target compartment uniform over the target's compartments.
    S = n_tot * syn_per_neuron if n_tot > 1 else 0
    dst = np.repeat(np.arange(n_tot, dtype=np.int64), syn_per_neuron)[:S]
    if S:
        src = rng.integers(0, n_tot - 1, size=S, dtype=np.int64)
        src = src + (src >= dst)
        comp = np.floor(rng.random(S) * sizes[dst]).astype(np.int64)
        comp = np.minimum(comp, sizes[dst] - 1)
        w = weight_uS[0] + rng.random(S) * (weight_uS[1] - weight_uS[0])
        if delay_ms[0] == "const":
            dl = np.full(S, float(delay_ms[1]))
        else:
            dl = delay_ms[1] + rng.random(S) * (delay_ms[2] - delay_ms[1])
    else:
        src = comp = np.zeros(0, np.int64)
        w = dl = np.zeros(0, np.float64)
    src_comp = None
    if src_points:
        src_comp = np.minimum(np.floor(rng.random(S) * sizes[src]).astype(np.int64), sizes[src] - 1)
        src_comp = src_comp.astype(np.int32)

    return Network(
        comp_offset=off, parent=parent, length_um=L, diam_um=D, stim_nA=stim,
        syn_src=src.astype(np.int32), syn_dst=dst.astype(np.int32), syn_comp=comp.astype(np.int32),
        syn_w=w, syn_delay_ms=dl,
        params=dict(DEFAULT_PARAMS if params is None else params),
        dt=dt, t_stop=t_stop, name=name, syn_src_comp=src_comp,
    )


# The five named workloads.  "scale" shrinks neuron counts (and giant sizes)
# for quick runs while keeping every distribution's shape.
CONFIGS = {
    "mono64": dict(  # 64 identical 255-compartment neurons, FP64, 100 ms
        n_neurons=64, size_dist=("mono", 255), p_branch=0.1, syn_per_neuron=10,
        delay_ms=("const", 1.0), mono_tree=True, t_stop=100.0, seed_index=0, precision="fp64"),
    "multi10k": dict(  # 10k own trees, log-uniform [50, 5000], FP64 batched, 50 ms
        n_neurons=10_000, size_dist=("loguniform", 50, 5000), p_branch=("uniform", 0.02, 0.2),
        syn_per_neuron=100, delay_ms=("const", 1.0), t_stop=50.0, seed_index=1, precision="fp64"),
    "multi10k_fp32c": dict(  # the same network in compensated FP32, 100 ms
        n_neurons=10_000, size_dist=("loguniform", 50, 5000), p_branch=("uniform", 0.02, 0.2),
        syn_per_neuron=100, delay_ms=("const", 1.0), t_stop=100.0, seed_index=1, precision="fp32c"),
    "lognormal100k": dict(  # 100k lognormal(800, 1.0) in [20, 20000], 1000 syn/neuron, 50 ms
        n_neurons=100_000, size_dist=("lognormal", 800, 1.0, 20, 20000), p_branch=0.1,
        syn_per_neuron=1000, delay_ms=("const", 1.0), t_stop=50.0, seed_index=3, precision="fp32c"),
    # The paper's load-balance tests (Sec. 4): 10,000 neurons of the same
    # mean size (300) -- one morphology for all, a group of 20 sizes at most
    # 700 apart, F-distributed sizes -- FP32c, 100 synapses per neuron, 50 ms
    "paper_mono": dict(
        n_neurons=10_000, size_dist=("mono", 300), p_branch=0.1, syn_per_neuron=100,
        delay_ms=("const", 1.0), mono_tree=True, t_stop=50.0, seed_index=5, precision="fp32c"),
    "paper_multi20": dict(
        n_neurons=10_000, size_dist=("group", 20, 700, 300), p_branch=0.1, syn_per_neuron=100,
        delay_ms=("const", 1.0), t_stop=50.0, seed_index=6, precision="fp32c"),
    "paper_fisher": dict(
        n_neurons=10_000, size_dist=("fisher", 10, 40, 300, 10, 5000), p_branch=0.1, syn_per_neuron=100,
        delay_ms=("const", 1.0), t_stop=50.0, seed_index=7, precision="fp32c"),
    # Neurons whose cost is not their size: log-uniform sizes, half of them
    # unbranched chains (one long serial sweep), half bushy trees (branch
    # probability 0.5, short paths), FP32c, 100 synapses per neuron, 50 ms
    "shapes10k": dict(
        n_neurons=10_000, size_dist=("loguniform", 200, 3000), p_branch=("choice", 0.0, 0.5),
        syn_per_neuron=100, delay_ms=("const", 1.0), t_stop=50.0, seed_index=8, precision="fp32c"),
    "mixed200k": dict(  # 200k lognormal(1000, 1.0) + 64 giants of 1e5 compartments, 20 ms
        n_neurons=200_000, size_dist=("lognormal", 1000, 1.0, 20, 20000), p_branch=0.1,
        syn_per_neuron=1000, delay_ms=("uniform", 1.0, 5.0), giants=64, giant_size=100_000,
        giant_p_branch=0.05, t_stop=20.0, seed_index=4, precision="fp32c"),
}


def make_config(name: str, scale: float = 1.0, n_neurons: Optional[int] = None,
                t_stop: Optional[float] = None, syn_per_neuron: Optional[int] = None,
                src_points: bool = False) -> Network:
    """Network of a named workload (optionally scaled down in neuron count;
    src_points: synapses also leave from uniformly drawn compartments)."""
    cfg = dict(CONFIGS[name])
    precision = cfg.pop("precision")
    seed = SEED_BASE + cfg.pop("seed_index")
    if n_neurons is None:
        n_neurons = max(2, int(round(cfg["n_neurons"] * scale)))
    cfg["n_neurons"] = n_neurons
    if t_stop is not None:
        cfg["t_stop"] = t_stop
    if syn_per_neuron is not None:
        cfg["syn_per_neuron"] = syn_per_neuron
    if "giants" in cfg and scale < 1.0:
        cfg["giants"] = max(1, int(round(cfg["giants"] * scale)))
        cfg["giant_size"] = max(1000, int(round(cfg["giant_size"] * min(1.0, scale * 10))))
    cfg["syn_per_neuron"] = min(cfg["syn_per_neuron"], max(1, n_neurons - 1))
    net = make_network(seed=seed, name=name, src_points=src_points, **cfg)
    net.params["precision"] = precision
    return net
