"""Spike detection at synapse points (Sec. 2: the threshold test runs at every
point of a morphology where a synapse leaves) on the GPU, through the C-ABI,
against the oracle's detect="points".

FP64: the same (neuron, compartment) spikes with times within 1e-9 ms and
voltages within 1e-9 mV.  FP32c: the same spikes with times within 0.01 dt
and voltages within 1e-3 mV, on regular, large-class and giant work items.
"""
import numpy as np
import pytest

import oracle
from paper_2005_06332_gb300 import mm, netgen

pytestmark = pytest.mark.gpu

TOL_V32 = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _lib():
    mm.load(build_if_missing=True)


def _by_point(n, c, t):
    o = np.lexsort((t, c, n))
    return n[o], c[o], t[o]


def _compare_spikes(gpu, ref, tol_ms):
    gn, gc, gt = _by_point(*gpu)
    rn, rc, rt = _by_point(*ref.point_spikes_sorted())
    np.testing.assert_array_equal(gn, rn)
    np.testing.assert_array_equal(gc, rc)
    assert np.max(np.abs(gt - rt), initial=0.0) <= tol_ms
    return gn, gc


def _with_points(net, rng, per_neuron=8, w=(0.0, 0.01), delay_ms=1.0):
    """The network with per_neuron synapses leaving each neuron: the first
    from the soma, the others from compartments drawn uniformly over it,
    towards uniformly drawn other neurons and compartments."""
    sizes = net.sizes()
    N = net.n_neurons
    src = np.repeat(np.arange(N), per_neuron)
    dst = rng.integers(0, N - 1, size=len(src))
    dst = dst + (dst >= src)
    scomp = np.floor(rng.random(len(src)) * sizes[src]).astype(np.int64)
    scomp[::per_neuron] = 0
    comp = np.floor(rng.random(len(src)) * sizes[dst]).astype(np.int64)
    net.syn_src = src.astype(np.int32)
    net.syn_dst = dst.astype(np.int32)
    net.syn_comp = np.minimum(comp, sizes[dst] - 1).astype(np.int32)
    net.syn_src_comp = np.minimum(scomp, sizes[src] - 1).astype(np.int32)
    net.syn_w = w[0] + rng.random(len(src)) * (w[1] - w[0])
    net.syn_delay_ms = np.full(len(src), delay_ms)
    return net


def _three_class_network():
    """A giant neuron (beyond one block's shared memory), a large-class one
    and small ones, all driven to fire."""
    parts = [netgen.make_network(1, size_dist=("mono", 20000), p_branch=0.05, syn_per_neuron=0, seed=31,
                                 stim_nA=(2.0, 2.0)),
             netgen.make_network(1, size_dist=("mono", 6000), p_branch=0.05, syn_per_neuron=0, seed=33,
                                 stim_nA=(2.0, 2.0)),
             netgen.make_network(12, size_dist=("loguniform", 20, 400), p_branch=0.1, syn_per_neuron=0, seed=32,
                                 stim_nA=(0.3, 0.8))]
    off = [np.zeros(1, np.int64)]
    for p in parts:
        off.append(off[-1][-1] + p.comp_offset[1:])
    cat = lambda k: np.concatenate([getattr(p, k) for p in parts])
    return netgen.Network(comp_offset=np.concatenate(off), parent=cat("parent"), length_um=cat("length_um"),
                          diam_um=cat("diam_um"), stim_nA=cat("stim_nA"), syn_src=np.zeros(0, np.int32),
                          syn_dst=np.zeros(0, np.int32), syn_comp=np.zeros(0, np.int32), syn_w=np.zeros(0),
                          syn_delay_ms=np.zeros(0), params=dict(netgen.DEFAULT_PARAMS), dt=0.025)


def test_fp64_synapse_points_match_oracle():
    net = netgen.make_network(24, size_dist=("loguniform", 20, 200), p_branch=0.15, syn_per_neuron=10, seed=43,
                              stim_nA=(0.3, 0.8), src_points=True)
    steps = 600
    ref = oracle.simulate(net, steps, detect="points")
    with mm.Network(net, precision="fp64", detect="points") as g:
        g.step(steps)
        V = g.read_voltages()
        spk = g.read_spike_points()
    assert np.max(np.abs(V - ref.V)) <= 1e-9
    gn, gc = _compare_spikes(spk, ref, 1e-9)
    assert np.count_nonzero(gc) > 20          # most crossings are away from the somata


def test_fp32c_synapse_points_all_item_classes():
    net = _with_points(_three_class_network(), np.random.default_rng(44))
    steps = 400
    ref = oracle.simulate(net, steps, detect="points")
    with mm.Network(net, precision="fp32c", detect="points") as g:
        info = g.launch_info()
        assert info["giant_items"] == 1 and info["big_items"] == 1
        g.step(steps)
        V = g.read_voltages()
        spk = g.read_spike_points()
    assert np.max(np.abs(V - ref.V)) <= TOL_V32
    gn, gc = _compare_spikes(spk, ref, 0.01 * net.dt)
    # crossings away from the soma on the giant and on the large neuron
    assert np.any((gn == 0) & (gc > 0)) and np.any((gn == 1) & (gc > 0))


def test_fp32c_points_at_every_soma_are_soma_detection():
    """All synapses leaving somata: detection at synapse points gives the
    soma spikes of every neuron with an outgoing synapse."""
    net = netgen.make_network(40, size_dist=("loguniform", 20, 600), p_branch=0.1, syn_per_neuron=5, seed=45,
                              stim_nA=(0.3, 0.8))
    net.syn_src_comp = np.zeros(net.n_syn, np.int32)
    steps = 800
    with mm.Network(net, precision="fp32c") as g:
        g.step(steps)
        Va = g.read_voltages()
        na, ta = g.read_spikes()
    with mm.Network(net, precision="fp32c", detect="points") as g:
        g.step(steps)
        Vb = g.read_voltages()
        nb, cb, tb = g.read_spike_points()
    has_out = np.zeros(net.n_neurons, bool)
    has_out[net.syn_src] = True
    keep = has_out[na]
    assert len(na) > 20
    assert np.max(np.abs(Va - Vb)) <= 1e-6
    np.testing.assert_array_equal(np.sort(nb), np.sort(na[keep]))
    assert np.all(cb == 0)
    np.testing.assert_allclose(np.sort(tb), np.sort(ta[keep]), rtol=0, atol=1e-9)


def test_fp32c_points_checkpoint_resume():
    net = netgen.make_network(25, size_dist=("loguniform", 10, 300), p_branch=0.1, syn_per_neuron=6, seed=12,
                              stim_nA=(0.3, 0.9), src_points=True)
    with mm.Network(net, precision="fp32c", detect="points") as g:
        g.step(90)
        blob = g.save_state()
        g.step(150)
        ref = g.read_voltages()
        _, _, t_ref = g.read_spike_points()
    with mm.Network(net, precision="fp32c", detect="points") as g2:
        g2.load_state(blob)
        g2.step(150)
        got = g2.read_voltages()
        _, _, t_got = g2.read_spike_points()
    assert np.max(np.abs(got - ref)) <= 1e-6
    assert len(t_got) == len(t_ref)


def test_source_compartment_out_of_range_is_rejected():
    net = netgen.make_network(4, size_dist=("mono", 30), p_branch=0.1, syn_per_neuron=2, seed=46, src_points=True)
    net.syn_src_comp = net.syn_src_comp.copy()
    net.syn_src_comp[3] = 30
    with pytest.raises(mm.MMError) as e:
        mm.Network(net, precision="fp32c", detect="points")
    assert e.value.status == mm.MM_EINVAL


def test_read_outputs_matches_the_separate_reads():
    """mm_read_outputs (soma voltages and the spike drain in one round trip,
    with more pending spikes than it prefetches) gives what
    mm_read_soma_voltages and mm_read_spike_points give."""
    net = netgen.make_network(200, size_dist=("loguniform", 20, 300), p_branch=0.1, syn_per_neuron=60, seed=47,
                              stim_nA=(0.5, 0.9), src_points=True)
    steps = 400
    with mm.Network(net, precision="fp32c", detect="points", deterministic=True) as a, \
            mm.Network(net, precision="fp32c", detect="points", deterministic=True) as b:
        seen = 0
        for k in range(steps // 80):
            a.step(80)
            b.step(80)
            soma_a, (na, ca, ta) = a.read_outputs()
            soma_b = b.read_soma()
            nb, cb, tb = b.read_spike_points()
            np.testing.assert_array_equal(soma_a, soma_b)
            np.testing.assert_array_equal(na, nb)
            np.testing.assert_array_equal(ca, cb)
            np.testing.assert_array_equal(ta, tb)
            seen = max(seen, len(na))
    assert seen > 4096          # the drain went beyond the prefetched records at least once
