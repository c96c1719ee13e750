"""Pins of the conditioning probes (test infrastructure, tests/neuron_conditioning.py):
the twin oracle build, whose membrane sums run in the opposite order, is an
equally valid FP64 evaluation -- it differs from the oracle by rounding
only, and it does differ -- and the re-simulation of one neuron alone with
its recorded inputs reproduces that neuron's trajectory in the whole network
bit for bit."""
import numpy as np

import oracle
from neuron_conditioning import resimulate, spike_steps
from paper_2005_06332_gb300 import netgen


def _net():
    return netgen.make_network(24, size_dist=("loguniform", 20, 300), p_branch=("uniform", 0.05, 0.3),
                               syn_per_neuron=8, seed=31, stim_nA=(0.2, 0.8))


def test_twin_differs_from_the_oracle_by_rounding_only():
    net = _net()
    steps = 400  # 10 ms: several spikes per neuron
    V = []
    for twin in (False, True):
        p = oracle.Part(net, twin=twin)
        p.step(steps)
        V.append(p.read_voltages())
        p.close()
    d = np.abs(V[0] - V[1])
    assert d.max() > 0.0  # the order of the sums changes the last bits somewhere
    assert d.max() < 1e-8  # and only those (spiking neurons amplify them a little)
    ref = oracle.simulate(net, steps)
    assert np.array_equal(V[0], ref.V)  # the oracle part is the oracle


def test_resimulation_reproduces_each_neuron_of_the_network():
    net = _net()
    steps = 400
    ref = oracle.simulate(net, steps)
    assert ref.n_spikes > 20
    ss = spike_steps(ref.spk_t, net.dt)
    for k in (0, 5, 17):
        sl = slice(net.comp_offset[k], net.comp_offset[k + 1])
        V0 = resimulate(net, k, ref.spk_neuron, ss, steps)
        assert np.array_equal(V0, ref.V[sl]), k
    # a dropped input spike changes the trajectory: the check has resolution
    k = int(np.argmax(np.bincount(net.syn_dst, minlength=net.n_neurons)))
    srcs = np.unique(net.syn_src[net.syn_dst == k])
    fired = np.isin(ref.spk_neuron, srcs)
    assert fired.any()
    drop = np.flatnonzero(fired)[0]
    keep = np.ones(len(ss), bool)
    keep[drop] = False
    V1 = resimulate(net, k, ref.spk_neuron[keep], ss[keep], steps)
    assert not np.array_equal(V1, ref.V[net.comp_offset[k]:net.comp_offset[k + 1]])
