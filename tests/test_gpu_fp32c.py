"""FP32c CUDA path vs the FP64 CPU oracle through the C-ABI.

The FP32c step keeps V and the gates in fixed point, sums the currents and
carries the model's constants as float pairs, and solves in FP32 with the
passive part of the diagonal eliminated once in FP64.  Its bar: max |dV| <=
1e-3 mV on every compartment and identical spike counts over 100 ms against
the FP64 oracle, with the spike-time shift (in dt) reported.  The accuracy
report at the end measures max |dV| and the shift per workload and writes
them to $MM_REPORT_DIR/accuracy_fp32c.json when that variable names a folder.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2005_06332_gb300 import mm, netgen

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TOL_V = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _lib():
    mm.load(build_if_missing=True)


def _spike_match(net, sn, st, ref):
    """Match spikes by (neuron, order within the neuron); returns the max
    time shift in units of dt, or None if the trains differ in count."""
    rn, rt = ref.spikes_sorted()
    if len(rn) != len(sn):
        return None
    shift = 0.0
    for k in np.unique(rn):
        a = np.sort(st[sn == k])
        b = np.sort(rt[rn == k])
        if len(a) != len(b):
            return None
        if len(a):
            shift = max(shift, float(np.max(np.abs(a - b))) / net.dt)
    return shift


def _run(net, steps, soma_every=0, **kw):
    trace = []
    with mm.Network(net, precision="fp32c", **kw) as g:
        if soma_every:
            done = 0
            while done < steps:
                k = min(soma_every, steps - done)
                g.step(k)
                done += k
                trace.append(g.read_soma().copy())
        else:
            g.step(steps)
        V = g.read_voltages()
        gates = {k: g.read_state(k) for k in ("m", "h", "n")}
        sn, st = g.read_spikes()
    return V, gates, sn, st, (np.array(trace) if trace else None)


def test_fp32c_short_horizon_parity():
    net = netgen.make_network(30, size_dist=("loguniform", 2, 300), p_branch=("uniform", 0.02, 0.3),
                              syn_per_neuron=10, seed=21, stim_nA=(0.2, 0.8))
    steps = 400
    ref = oracle.simulate(net, steps)
    V, gates, sn, st, _ = _run(net, steps)
    assert np.max(np.abs(V - ref.V)) <= TOL_V
    for k, r in (("m", ref.m), ("h", ref.h), ("n", ref.n)):
        assert np.max(np.abs(gates[k] - r)) <= 1e-5, k
    assert _spike_match(net, sn, st, ref) is not None
    assert ref.n_spikes > 0


@pytest.mark.parametrize("dt", [0.01, 0.05])
def test_fp32c_other_time_steps(dt):
    """The gate table and the passive elimination are built for the network's
    dt: other steps than the default 0.025 ms, over 20 ms of spiking."""
    net = netgen.make_network(30, size_dist=("loguniform", 2, 300), p_branch=("uniform", 0.02, 0.3),
                              syn_per_neuron=10, seed=22, stim_nA=(0.2, 0.8))
    net.dt = dt
    steps = int(round(20.0 / dt))
    ref = oracle.simulate(net, steps)
    V, gates, sn, st, _ = _run(net, steps)
    assert ref.n_spikes > 10
    assert np.max(np.abs(V - ref.V)) <= TOL_V
    for k, r in (("m", ref.m), ("h", ref.h), ("n", ref.n)):
        assert np.max(np.abs(gates[k] - r)) <= 1e-4, k
    assert _spike_match(net, sn, st, ref) is not None


@pytest.mark.parametrize("dist", [("group", 20, 700, 300), ("fisher", 10, 40, 300, 10, 5000)])
def test_fp32c_paper_size_distributions_parity(dist):
    """The size distributions of the paper's load-balance tests (a group of 20
    sizes, F-distributed sizes), also in a random work-queue order."""
    net = netgen.make_network(40, size_dist=dist, p_branch=0.1, syn_per_neuron=10, seed=23, stim_nA=(0.2, 0.8))
    steps = 320
    ref = oracle.simulate(net, steps)
    for cost in (None, np.random.default_rng(5).random(net.n_neurons).astype(np.float32)):
        V, gates, sn, st, _ = _run(net, steps, cost=cost, group_comps=1024)
        assert np.max(np.abs(V - ref.V)) <= TOL_V
        assert _spike_match(net, sn, st, ref) is not None


def test_fp32c_single_chain_one_step_is_close():
    n = 50
    off = np.array([0, n], dtype=np.int64)
    net = netgen.Network(
        comp_offset=off, parent=np.arange(-1, n - 1, dtype=np.int32),
        length_um=np.linspace(5, 20, n), diam_um=np.linspace(2, 0.5, n), stim_nA=np.array([0.4]),
        syn_src=np.zeros(0, np.int32), syn_dst=np.zeros(0, np.int32), syn_comp=np.zeros(0, np.int32),
        syn_w=np.zeros(0), syn_delay_ms=np.zeros(0), params=dict(netgen.DEFAULT_PARAMS), dt=0.025)
    ref = oracle.simulate(net, 1)
    V, _, _, _, _ = _run(net, 1)
    # one step: the error is the rounding of one FP32 increment
    assert np.max(np.abs(V - ref.V)) <= 1e-5


def test_fp32c_mono64_100ms():
    """mono64 over the full 100 ms: identical spike trains (shift below 1e-2
    dt) and every compartment within the 1e-3 mV bar at the end."""
    net = netgen.make_config("mono64")
    ref = oracle.simulate(net, net.n_steps)
    V, _, sn, st, _ = _run(net, net.n_steps)
    shift = _spike_match(net, sn, st, ref)
    assert shift is not None, "spike trains differ"
    assert shift <= 0.01
    assert np.max(np.abs(V - ref.V)) <= TOL_V


def _three_class_network():
    """One neuron too large for any block's shared memory (giant item), one
    above the regular shared-memory budget (large class), and small ones;
    the large neurons are driven hard enough to fire."""
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


def test_fp32c_all_item_classes_match_oracle():
    """Regular, large-class and giant work items agree with the oracle on
    voltages and spikes, and on the gates too: the state after a step is the
    method's state after that step, compared here in the middle of the giant
    neuron's upstroke, where one gate update more or less is visible."""
    net = _three_class_network()
    full = oracle.simulate(net, 400, record_soma=True)
    assert full.n_spikes >= 2
    k = 40 + int(np.argmax(np.diff(full.soma_trace[0][40:]))) + 1  # giant neuron's steepest rise after 1 ms
    ref = oracle.simulate(net, k)
    with mm.Network(net, precision="fp32c") as g:
        info = g.launch_info()
        assert info["giant_items"] == 1 and info["big_items"] == 1
        assert info["comps"] == [int(net.n_comp) - 26000, 6000, 20000]
        g.step(k)
        V = g.read_voltages()
        gates = {w: g.read_state(w) for w in ("m", "h", "n")}
        g.step(400 - k)
        sn, _ = g.read_spikes()
    assert np.max(np.abs(V - ref.V)) <= TOL_V
    for w, x in gates.items():
        assert np.max(np.abs(x - getattr(ref, w))) <= 1e-4, w
    assert len(sn) == full.n_spikes


def test_fp32c_all_item_classes_100ms():
    """The three-class network (giant, large-class and regular items) over
    100 ms: identical spike trains and every compartment within the bar."""
    net = _three_class_network()
    steps = 4000
    ref = oracle.simulate(net, steps)
    with mm.Network(net, precision="fp32c") as g:
        info = g.launch_info()
        assert info["giant_items"] == 1 and info["big_items"] == 1
        g.step(steps)
        V = g.read_voltages()
        sn, st = g.read_spikes()
    assert ref.n_spikes > 10
    shift = _spike_match(net, sn, st, ref)
    assert shift is not None, "spike trains differ"
    assert shift <= 0.01
    assert np.max(np.abs(V - ref.V)) <= TOL_V


def test_fp32c_eq2_as_printed_scheme_all_item_classes():
    """MM_SCHEME_CN (Eq. 2 as printed) in FP32c on regular, large-class and
    giant work items against the oracle's scheme "cn"."""
    net = _three_class_network()
    steps = 200
    ref = oracle.simulate(net, steps, scheme="cn")
    with mm.Network(net, precision="fp32c", scheme="cn") as g:
        info = g.launch_info()
        assert info["giant_items"] == 1 and info["big_items"] == 1
        g.step(steps)
        V = g.read_voltages()
        sn, st = g.read_spikes()
    assert np.max(np.abs(V - ref.V)) <= TOL_V
    assert _spike_match(net, sn, st, ref) is not None


def test_fp32c_checkpoint_resume():
    net = netgen.make_network(25, size_dist=("loguniform", 10, 300), p_branch=0.1, syn_per_neuron=6, seed=12,
                              stim_nA=(0.3, 0.9))
    with mm.Network(net, precision="fp32c") as g:
        g.step(90)
        blob = g.save_state()
        g.step(150)
        ref = g.read_voltages()
    with mm.Network(net, precision="fp32c") as g2:
        g2.load_state(blob)
        g2.step(150)
        got = g2.read_voltages()
    assert np.max(np.abs(got - ref)) <= 1e-6


def _report(name, net, steps, soma_every):
    ref = oracle.simulate(net, steps, record_soma=True)
    V, _, sn, st, trace = _run(net, steps, soma_every=soma_every)
    dv_end = float(np.max(np.abs(V - ref.V)))
    ref_soma = ref.soma_trace[:, soma_every::soma_every].T[:len(trace)]
    dv_soma = float(np.max(np.abs(trace - ref_soma)))
    shift = _spike_match(net, sn, st, ref)
    return {"workload": name, "n_neurons": net.n_neurons, "n_comp": net.n_comp, "steps": steps,
            "max_abs_dV_end_mV": dv_end, "max_abs_dV_soma_all_steps_mV": dv_soma,
            "spikes_oracle": int(ref.n_spikes), "spikes_gpu": int(len(sn)),
            "identical_spike_counts": shift is not None,
            "max_spike_shift_dt": shift}


def test_fp32c_accuracy_report():
    rows = [_report("mono64 (64 x 255 compartments), 100 ms", netgen.make_config("mono64"), 4000, 1),
            _report("multi10k distribution, 1000-neuron sample, 100 ms",
                    netgen.make_config("multi10k_fp32c", n_neurons=1000), 4000, 10)]
    out = os.environ.get("MM_REPORT_DIR", "")
    if os.path.isdir(out):
        with open(os.path.join(out, "accuracy_fp32c.json"), "w") as f:
            json.dump(rows, f, indent=1)
    print(json.dumps(rows, indent=1))
    for r in rows:
        assert r["identical_spike_counts"], r
        assert r["max_spike_shift_dt"] <= 0.01, r
        assert r["max_abs_dV_end_mV"] <= TOL_V, r


def _first_window_sampled(name, block_threads=0, group_comps=0, n_pick=40):
    """Full-size network, first min-delay window: no event can arrive before
    step round(min delay / dt) + 1, so each sampled neuron (plus the largest
    and the smallest) must follow the oracle's run of that neuron alone."""
    net = netgen.make_config(name)
    steps = int(round(float(np.min(net.syn_delay_ms)) / net.dt)) + 1
    with mm.Network(net, precision="fp32c", block_threads=block_threads, group_comps=group_comps) as g:
        info = g.launch_info()
        g.step(steps)
        V = g.read_voltages()
        gates = {k: g.read_state(k) for k in ("m", "h", "n")}
    rng = np.random.default_rng(0)
    sizes = net.sizes()
    pick = np.unique(np.concatenate([rng.choice(net.n_neurons, n_pick, replace=False),
                                     [int(np.argmax(sizes)), int(np.argmin(sizes))]]))
    sub = net.subset(pick, keep_synapses=False)
    ref = oracle.simulate(sub, steps)
    idx = np.concatenate([np.arange(net.comp_offset[k], net.comp_offset[k + 1]) for k in pick])
    assert np.max(np.abs(V[idx] - ref.V)) <= TOL_V
    for k in ("m", "h", "n"):
        assert np.max(np.abs(gates[k][idx] - getattr(ref, k))) <= 1e-5, k
    return info


def test_fp32c_multi10k_full_size_first_window_sampled():
    """multi10k (10.9 M compartments) in the launch configuration the
    benchmark's autotuner picks (512 threads, 4096-compartment items)."""
    _first_window_sampled("multi10k", block_threads=512, group_comps=4096)


def test_fp32c_lognormal100k_full_size_first_window_sampled():
    """lognormal100k (132 M compartments, 100 M synapses), library defaults:
    regular and large-class items (neurons up to 20,000 compartments)."""
    info = _first_window_sampled("lognormal100k")
    assert info["big_items"] > 0


def test_fp32c_mixed200k_full_size_first_window_sampled():
    """mixed200k (200,000 neurons and 64 giants of 100,000 compartments,
    200 M synapses with delays U[1, 5] ms), library defaults: all three item
    classes (the 64 giants and the lognormal neurons beyond the large class);
    a giant is always among the sampled neurons (the largest)."""
    info = _first_window_sampled("mixed200k")
    assert info["giant_items"] >= 64 and info["big_items"] > 0
