"""Learned work-queue order: measure, learn, predict (orchestration only).

1. measure_neuron_times: a network of the sampled neurons, each its own
   work item, runs a few FP32c steps while the solve kernel times every
   item with %globaltimer (mm_read_neuron_times);
2. the MLP (mm_mlp_*, the library's BF16 kernels) learns log(time) from
   the 16 morphology features (mm_neuron_features);
3. its predictions for every neuron become mm_options.cost, so the
   persistent kernel's queue hands out the longest items first
   (MM_SCHED_COST); size-sorted order stays the fallback.
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
                holdout: float = 0.2, device: int = 0) -> dict:
    """Train the cost model on n_timed sampled neurons; predict every neuron."""
    rng = np.random.default_rng(seed)
    k = min(n_timed, net.n_neurons)
    pick = np.sort(rng.choice(net.n_neurons, k, replace=False))
    feats = mm.neuron_features(net)
    t_us = measure_neuron_times(net, pick, steps=steps, device=device)
    y = np.log(np.maximum(t_us, 1e-3)).astype(np.float32)
    perm = rng.permutation(k)
    n_test = int(round(k * holdout)) if k >= 10 else 0
    test, train = perm[:n_test], perm[n_test:]
    model = mm.MLP(seed)
    try:
        losses = model.train(feats[pick[train]], y[train], epochs=epochs, lr=lr)
        pred_all = model.predict(feats)
        r2 = None
        if n_test:
            p = model.predict(feats[pick[test]])
            resid = y[test] - p
            r2 = float(1.0 - np.sum(resid ** 2) / np.sum((y[test] - y[test].mean()) ** 2))
    finally:
        model.close()
    # the size-only baseline of the same R^2 on the held-out neurons
    r2_size = None
    if n_test:
        ls = np.log(net.sizes()[pick]).astype(np.float64)
        A = np.vstack([ls[train], np.ones(len(train))]).T
        coef, *_ = np.linalg.lstsq(A, y[train].astype(np.float64), rcond=None)
        res = y[test] - (coef[0] * ls[test] + coef[1])
        r2_size = float(1.0 - np.sum(res ** 2) / np.sum((y[test] - y[test].mean()) ** 2))
    return {"cost": np.exp(pred_all).astype(np.float32), "timed": pick, "time_us": t_us, "losses": losses,
            "r2_holdout": r2, "r2_holdout_size_only": r2_size}
