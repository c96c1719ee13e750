"""A network split by neuron across devices or processes (orchestration only).

The paper runs its simulator on a cluster: every node holds a group of
neurons, computes several local steps (one "global step", the network delay)
without communication, then exchanges the spikes of that global step with
MPI_AllGather into a global buffer that all nodes read (Sec. 2, Algorithm 2).
How the neurons are distributed decides the balance (Sec. 4): sorting all of
them globally by size and storing the largest on the first node ("global
sorting-storing") leaves the other nodes idle, while balanced groups sorted
on each node ("local sorting-storing") do not.

Here each part is a network of its own (``mm.Network`` on one GPU, or any
object with the same methods): its neurons, the synapses that end on them,
and the remote neurons among their sources as external spike sources
(``mm_options.n_ext_sources``).  A window is the largest number of steps no
spike can cross within: round(min delay / dt) steps; a spike detected in
step m reaches its targets no earlier than step m + 1 + round(min delay/dt).
After each window every part reads the spikes its own neurons fired
(``mm_read_fired``), the parts exchange them (a count all-gather, then an
all-gather of the padded lists), and each part hands the ones of its
external sources to its network (``mm_inject_spikes``) before the next window
runs.  Every step of the neurons' dynamics runs in the parts' networks; this
module only moves neuron ids and step numbers.
"""
from __future__ import annotations

import heapq
from typing import Callable, List, Optional, Sequence

import numpy as np

from .netgen import Network


# ----------------------------------------------------------------- placement

def partition(net: Network, n_parts: int, cost: Optional[np.ndarray] = None, mode: str = "local") -> List[np.ndarray]:
    """Neurons of each part (global ids).

    cost: per-neuron cost (default: compartment count), e.g. the learned
    prediction.  mode "local" (the paper's local sorting-storing): neurons
    taken largest first, each to the part with the least total cost so far
    (longest-processing-time first), then sorted largest first within the
    part; "global" (global sorting-storing): all neurons sorted largest
    first and cut into n_parts runs of equal count, the largest neurons on
    the first part.  Giant neurons are never split: a neuron is a unit.
    """
    if n_parts < 1:
        raise ValueError("n_parts must be >= 1")
    c = np.asarray(net.sizes() if cost is None else cost, dtype=np.float64)
    if c.shape != (net.n_neurons,):
        raise ValueError("cost needs one entry per neuron")
    order = np.lexsort((np.arange(net.n_neurons), -c))  # largest first, ties by id
    if mode == "global":
        return [np.asarray(x, np.int64) for x in np.array_split(order, n_parts)]
    if mode != "local":
        raise ValueError(f"unknown placement mode {mode!r}")
    heap = [(0.0, p) for p in range(n_parts)]
    parts: List[list] = [[] for _ in range(n_parts)]
    for k in order:
        load, p = heapq.heappop(heap)
        parts[p].append(int(k))
        heapq.heappush(heap, (load + float(c[k]), p))
    return [np.asarray(sorted(x, key=lambda k: (-c[k], k)), np.int64) for x in parts]


def part_loads(net: Network, parts: Sequence[np.ndarray], cost: Optional[np.ndarray] = None) -> np.ndarray:
    """Total cost (default: compartments) of each part."""
    c = np.asarray(net.sizes() if cost is None else cost, dtype=np.float64)
    return np.array([float(c[p].sum()) for p in parts])


class Part:
    """One part of a split network: its own Network (neurons renumbered
    0..k-1 in the part's order), the global id of each local neuron, and the
    global id of each external source (local source ids k, k+1, ...)."""

    def __init__(self, net: Network, neurons: np.ndarray):
        neurons = np.asarray(neurons, np.int64)
        self.neurons = neurons
        k = len(neurons)
        local = -np.ones(net.n_neurons, np.int64)
        local[neurons] = np.arange(k)
        keep = local[net.syn_dst] >= 0 if net.n_syn else np.zeros(0, bool)
        src = net.syn_src[keep].astype(np.int64)
        remote = local[src] < 0
        self.ext_ids = np.unique(src[remote])             # external source e is global neuron ext_ids[e]
        ext_of = -np.ones(net.n_neurons, np.int64)
        ext_of[self.ext_ids] = np.arange(len(self.ext_ids))
        self.ext_of = ext_of
        new_src = np.where(remote, k + ext_of[src], local[src]).astype(np.int32)
        sizes = net.sizes()[neurons]
        off = np.zeros(k + 1, np.int64)
        np.cumsum(sizes, out=off[1:])
        idx = np.concatenate([np.arange(net.comp_offset[g], net.comp_offset[g + 1]) for g in neurons]) \
            if k else np.zeros(0, np.int64)
        # synapses keep their global order, so that the events reaching one
        # site in one step are added in the same order as in the whole network
        self.net = Network(comp_offset=off, parent=net.parent[idx].copy(), length_um=net.length_um[idx].copy(),
                           diam_um=net.diam_um[idx].copy(), stim_nA=net.stim_nA[neurons].copy(),
                           syn_src=new_src, syn_dst=local[net.syn_dst[keep]].astype(np.int32),
                           syn_comp=net.syn_comp[keep].copy(), syn_w=net.syn_w[keep].copy(),
                           syn_delay_ms=net.syn_delay_ms[keep].copy(), params=dict(net.params), dt=net.dt,
                           t_stop=net.t_stop, name=f"{net.name}-part")
        self.comp_index = idx                               # global compartment of each local one

    @property
    def n_ext(self) -> int:
        return int(len(self.ext_ids))


# ------------------------------------------------------------------ exchange

class LocalExchange:
    """All parts in this process (virtual parts, e.g. several on one GPU)."""

    def allgather(self, lists: List[np.ndarray]) -> List[np.ndarray]:
        return list(lists)


class TorchExchange:
    """One part per rank of a torch.distributed process group (NCCL on GPUs,
    gloo on CPUs): a count all-gather, then an all-gather of the lists
    padded to the longest, as the paper's MPI_AllGather of spike events."""

    def __init__(self, group=None, device: str = "cpu"):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.device = device
        self.world = dist.get_world_size(group)

    def allgather(self, lists: List[np.ndarray]) -> List[np.ndarray]:
        import torch
        if len(lists) != 1:
            raise ValueError("one part per rank")
        mine = np.ascontiguousarray(lists[0], np.int64).reshape(-1)
        n = torch.tensor([mine.size], dtype=torch.int64, device=self.device)
        counts = [torch.zeros(1, dtype=torch.int64, device=self.device) for _ in range(self.world)]
        self.dist.all_gather(counts, n, group=self.group)
        cnt = [int(c.item()) for c in counts]
        width = max(1, max(cnt))
        buf = torch.zeros(width, dtype=torch.int64, device=self.device)
        buf[:mine.size] = torch.from_numpy(mine).to(self.device)
        outs = [torch.zeros(width, dtype=torch.int64, device=self.device) for _ in range(self.world)]
        self.dist.all_gather(outs, buf, group=self.group)
        return [o[:c].cpu().numpy() for o, c in zip(outs, cnt)]


# ----------------------------------------------------------------- the run

def _pack(neuron: np.ndarray, step: np.ndarray) -> np.ndarray:
    """(global neuron, step) pairs as one int64 list: step * 2^31 + neuron."""
    return np.asarray(step, np.int64) * (1 << 31) + np.asarray(neuron, np.int64)


def _unpack(x: np.ndarray):
    x = np.asarray(x, np.int64)
    return x & ((1 << 31) - 1), x >> 31


class ShardedRun:
    """Runs the parts this process holds in windows of the minimum delay.

    parts: the Part objects of this process (all of them for virtual parts,
    one per rank for a distributed run); engines: one network per part with
    the methods step(n), read_fired(step0, n) -> (local user ids, steps),
    inject_spikes(ext_src, steps) (e.g. ``mm.Network(part.net,
    n_ext_sources=part.n_ext)``); exchange: LocalExchange or TorchExchange.
    """

    def __init__(self, net: Network, parts: List[Part], engines: list, exchange):
        if len(parts) != len(engines):
            raise ValueError("one engine per part")
        self.parts, self.engines, self.exchange = parts, engines, exchange
        self.window = int(round(float(np.min(net.syn_delay_ms)) / net.dt)) if net.n_syn else 1 << 30
        if self.window < 1:
            raise ValueError("the minimum delay must be at least one step")
        self.step_now = 0
        self.spikes: List[np.ndarray] = []   # packed (global neuron, step) of every spike seen

    def run(self, n_steps: int, on_window: Optional[Callable[[int], None]] = None):
        while n_steps > 0:
            k = min(self.window, n_steps)
            for e in self.engines:
                e.step(k)
            mine = []
            for p, e in zip(self.parts, self.engines):
                nrn, st = e.read_fired(self.step_now, k)
                mine.append(_pack(p.neurons[nrn], st))
            if isinstance(self.exchange, LocalExchange):
                got = self.exchange.allgather(mine)
            else:
                got = self.exchange.allgather([np.concatenate(mine) if mine else np.zeros(0, np.int64)])
            every = np.concatenate(got) if got else np.zeros(0, np.int64)
            self.spikes.append(every)
            g, st = _unpack(every)
            for p, e in zip(self.parts, self.engines):
                if p.n_ext == 0 or every.size == 0:
                    continue
                ext = p.ext_of[g]
                sel = ext >= 0
                if np.any(sel):
                    e.inject_spikes(ext[sel].astype(np.int32), st[sel])
            self.step_now += k
            n_steps -= k
            if on_window is not None:
                on_window(self.step_now)

    def spike_list(self):
        """Every spike of the network seen so far: (global neuron ids, steps),
        ordered by (step, neuron)."""
        every = np.concatenate(self.spikes) if self.spikes else np.zeros(0, np.int64)
        every = np.unique(every)
        return _unpack(every)
