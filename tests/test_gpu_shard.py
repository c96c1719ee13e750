"""A network split into parts on one GPU (virtual parts, shard.ShardedRun
with the in-process exchange): each part a library network whose remote
sources are external (mm_options.n_ext_sources), their spikes handed in with
mm_inject_spikes after every window and its own read with mm_read_fired.
Against the FP64 oracle of the unsplit network; and the boundary's checks of
handed-in spikes."""
import numpy as np
import pytest

import oracle
from paper_2005_06332_gb300 import mm, netgen, shard

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    mm.load(build_if_missing=True)


def _net(n=60, seed=11):
    net = netgen.make_network(n, size_dist=("loguniform", 10, 400), p_branch=0.1, syn_per_neuron=12, seed=seed,
                              stim_nA=(0.3, 0.9), weight_uS=(0.0, 0.02), delay_ms=("uniform", 1.0, 3.0))
    net.t_stop = 30.0
    return net


def _whole(net, steps):
    w = oracle.Part(net)
    w.step(steps)
    rn, rs = w.read_fired(0, steps)
    return w.read_voltages(), rn.astype(np.int64), rs


@pytest.mark.parametrize("precision,tol,n_parts", [("fp64", 1e-9, 3), ("fp32c", 1e-3, 2)])
def test_virtual_parts_on_one_gpu_match_the_oracle(precision, tol, n_parts):
    net = _net()
    steps = net.n_steps
    Vw, rn, rs = _whole(net, steps)
    assert len(rn) > 30
    parts = [shard.Part(net, ids) for ids in shard.partition(net, n_parts)]
    assert all(p.n_ext > 0 for p in parts)
    engines = [mm.Network(p.net, precision=precision, n_ext_sources=p.n_ext) for p in parts]
    try:
        run = shard.ShardedRun(net, parts, engines, shard.LocalExchange())
        run.run(steps)
        g, st = run.spike_list()
        if precision == "fp64":
            np.testing.assert_array_equal(np.sort(g * 100000 + st), np.sort(rn * 100000 + rs))
        else:  # the same spikes; a crossing within a hair of a step boundary may change step
            assert len(g) == len(rn)
            for k in np.unique(rn):
                assert np.all(np.abs(np.sort(st[g == k]) - np.sort(rs[rn == k])) <= 1)
        V = np.full(net.n_comp, np.nan)
        for p, e in zip(parts, engines):
            V[p.comp_index] = e.read_voltages()
        assert np.max(np.abs(V - Vw)) <= tol
        # each part's own spike records (user numbering of the part) are its
        # neurons' spikes in the whole network
        for p, e in zip(parts, engines):
            sn, _ = e.read_spikes()
            assert sorted(p.neurons[sn].tolist()) == sorted(rn[np.isin(rn, p.neurons)].tolist())
    finally:
        for e in engines:
            e.close()


def test_read_fired_lists_the_steps_of_the_spike_records():
    """Every spike record (user neuron, crossing time) of the first 120
    steps (the opening volley; no more than R - 1 = 121 steps back) is one
    (neuron, step) of mm_read_fired, the time within that step."""
    net = netgen.make_network(40, size_dist=("loguniform", 10, 200), syn_per_neuron=5, seed=12, stim_nA=(0.3, 0.9),
                              delay_ms=("uniform", 1.0, 3.0))
    with mm.Network(net, precision="fp64") as g:
        g.step(120)
        nrn, st = g.read_fired(0, 120)
        sn, tt = g.read_spikes()
    assert len(sn) > 20 and len(nrn) == len(sn)
    assert np.all((st >= 0) & (st < 120)) and np.all(np.diff(st) >= 0)
    ref = sorted(zip(sn.tolist(), np.ceil(tt / net.dt - 1e-9).astype(int) - 1))
    assert sorted(zip(nrn.tolist(), st.tolist())) == ref
    for k, m in zip(nrn, st):
        t = tt[sn == k]
        assert np.any((t > m * net.dt) & (t <= (m + 1) * net.dt))


def test_inject_and_read_fired_reject_bad_requests():
    net = _net(n=20, seed=13)
    parts = [shard.Part(net, ids) for ids in shard.partition(net, 2)]
    p = parts[0]
    with mm.Network(p.net, precision="fp64", n_ext_sources=p.n_ext) as g:
        g.step(50)
        d_min = int(round(float(np.min(p.net.syn_delay_ms)) / net.dt))
        late = 50 - 2 - d_min  # its earliest delivery, step late + 1 + d_min, has already run
        for src, st in (([p.n_ext], [45]),   # source out of range
                        ([0], [50]),         # a step not yet run
                        ([0], [late]),       # handed in too late
                        ([0, 0], [45, 45])):  # the same source twice in one step
            with pytest.raises(mm.MMError) as e:
                g.inject_spikes(np.array(src), np.array(st))
            assert e.value.status == mm.MM_EINVAL
        g.inject_spikes(np.array([0, 1]), np.array([48, 48]))  # in time: accepted
        with pytest.raises(mm.MMError) as e:
            g.read_fired(40, 20)  # beyond the steps run
        assert e.value.status == mm.MM_EINVAL
    with mm.Network(net, precision="fp64") as g:
        with pytest.raises(mm.MMError) as e:
            g.inject_spikes(np.array([0]), np.array([0]))  # no external sources
        assert e.value.status == mm.MM_EINVAL
