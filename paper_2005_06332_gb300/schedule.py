"""Learned work-queue order (orchestration only).

The whole pipeline is one native call, mm_train_schedule (csrc/
mm_schedule.cpp): a sample of neurons is timed by the solve kernel itself
(each neuron its own work item, %globaltimer per item), the MLP (the
library's BF16 kernels) learns log(time) from the 16 morphology features,
and its prediction for every neuron becomes mm_options.cost, so that the
persistent kernel's queue hands out the longest items first (MM_SCHED_COST);
size-sorted order stays the fallback.  measure_neuron_times exposes the
timing step alone.
"""
from __future__ import annotations

import numpy as np

from . import mm


def measure_neuron_times(net, neurons, steps: int = 40, device: int = 0) -> np.ndarray:
    """Per-step solve time (us) of each listed neuron, timed as its own work item."""
    sub = net.subset(np.asarray(neurons), keep_synapses=False)
    with mm.Network(sub, precision="fp32c", group_comps=1, time_items=True, graph_steps=0, device=device) as g:
        g.step(steps)
        return g.read_neuron_times()


def learn_costs(net, n_timed: int = 5000, steps: int = 40, epochs: int = 600, lr: float = 3e-3, seed: int = 0,
                device: int = 0, stream=None) -> dict:
    """Learned cost of every neuron (mm_train_schedule) with its report:
    held-out R^2 of log time for the network and for log size alone."""
    return mm.train_schedule(net, n_timed=n_timed, steps=steps, epochs=epochs, lr=lr, seed=seed, device=device,
                             stream=stream)
