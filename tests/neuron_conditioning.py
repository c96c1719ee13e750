"""How well a single neuron's trajectory is determined by the arithmetic
(test infrastructure: uses the oracle).

Within a network whose spike trains are known, each neuron's trajectory
depends only on its own dynamics and the events its incoming synapses
deliver.  resimulate() runs one neuron alone in the FP64 oracle (a network
part whose presynaptic neurons are external sources), handing in the recorded
spikes of those neurons window by window, so that it reproduces the neuron's
trajectory in the whole network to the bit.  Two probes of conditioning:

* twin: the oracle with its membrane sums in the opposite order -- an
  equally valid FP64 evaluation; the difference bounds what FP64 arithmetic
  itself determines of the neuron's state at the end;
* stim_scale: the soma stimulus scaled by (1 + 2^-24), one FP32 rounding of
  one model parameter; a neuron that this moves by more than the FP32c
  tolerance is not determined to that tolerance by any FP32-based arithmetic.
"""
from __future__ import annotations

import numpy as np

import oracle
from paper_2005_06332_gb300 import shard


def spike_steps(t_ms, dt):
    """The step of each recorded crossing time (t in (n dt, (n + 1) dt])."""
    return np.ceil(np.asarray(t_ms) / dt - 1e-9).astype(np.int64) - 1


def resimulate(net, k: int, spk_neuron, spk_step, n_steps: int, twin: bool = False, stim_scale: float = 1.0):
    """Voltages of neuron k after n_steps, simulated alone with its recorded inputs."""
    part = shard.Part(net, np.array([k], np.int64))
    sub = part.net
    sub.stim_nA = sub.stim_nA * stim_scale
    o = oracle.Part(sub, n_ext=part.n_ext, twin=twin)
    sn = np.asarray(spk_neuron, np.int64)
    ss = np.asarray(spk_step, np.int64)
    ext = part.ext_of[sn]
    sel = ext >= 0
    e_src, e_step = ext[sel].astype(np.int32), ss[sel]
    w = int(round(float(np.min(sub.syn_delay_ms)) / net.dt)) if sub.n_syn else n_steps
    w = max(1, w)
    done = 0
    while done < n_steps:
        kk = min(w, n_steps - done)
        o.step(kk)
        m = (e_step >= done) & (e_step < done + kk)
        if np.any(m):
            o.inject_spikes(e_src[m], e_step[m])
        done += kk
    V = o.read_voltages()
    o.close()
    return V
