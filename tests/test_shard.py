"""The neuron-sharded run (paper_2005_06332_gb300/shard.py) on the CPU.

Placement (local and global sorting-storing), the split of a network into
parts with external spike sources, and whole runs: virtual parts in one
process and two gloo ranks, each part a steppable FP64 oracle network
(oracle.Part), against the unsplit oracle run.  The same orchestration
drives the library's networks on GPUs (tests/test_gpu_shard.py)."""
import os

import numpy as np
import pytest

import oracle
from paper_2005_06332_gb300 import netgen, shard


def _net(n=36, seed=5, steps_ms=15.0):
    net = netgen.make_network(n, size_dist=("loguniform", 5, 120), p_branch=0.1, syn_per_neuron=8, seed=seed,
                              stim_nA=(0.4, 0.9), weight_uS=(0.0, 0.02), delay_ms=("uniform", 1.0, 2.0))
    net.t_stop = steps_ms
    return net


def test_local_placement_balances_and_sorts_each_part():
    net = netgen.make_config("multi10k", n_neurons=600)
    c = net.sizes().astype(float)
    parts = shard.partition(net, 4, mode="local")
    assert sorted(np.concatenate(parts).tolist()) == list(range(net.n_neurons))
    loads = shard.part_loads(net, parts)
    # longest-processing-time first: no part exceeds another by more than the largest neuron
    assert loads.max() - loads.min() <= c.max()
    for p in parts:
        assert np.all(np.diff(c[p]) <= 0)  # largest first within each part


def test_global_placement_puts_the_largest_on_the_first_part():
    net = netgen.make_config("multi10k", n_neurons=600)
    c = net.sizes()
    parts = shard.partition(net, 4, mode="global")
    assert [len(p) for p in parts] == [150] * 4
    assert c[parts[0]].min() >= c[parts[1]].max()
    loads = shard.part_loads(net, parts)
    assert loads[0] > 2 * loads[-1]  # the imbalance the paper measured with global sorting-storing


def test_placement_by_a_given_cost():
    net = netgen.make_config("multi10k", n_neurons=100)
    cost = np.random.default_rng(1).random(net.n_neurons)
    parts = shard.partition(net, 3, cost=cost)
    loads = shard.part_loads(net, parts, cost)
    assert loads.max() - loads.min() <= cost.max()


def test_part_maps_remote_sources_to_external_ids():
    net = _net()
    parts = shard.partition(net, 3)
    seen = 0
    for ids in parts:
        p = shard.Part(net, ids)
        k = len(ids)
        keep = np.isin(net.syn_dst, ids)
        assert p.net.n_syn == int(keep.sum())
        src_g = net.syn_src[keep]
        src_l = p.net.syn_src
        local = src_l < k
        np.testing.assert_array_equal(ids[src_l[local]], src_g[local])
        np.testing.assert_array_equal(p.ext_ids[src_l[~local] - k], src_g[~local])
        assert not np.any(np.isin(p.ext_ids, ids))
        np.testing.assert_array_equal(p.net.syn_w, net.syn_w[keep])  # global synapse order kept
        np.testing.assert_array_equal(p.net.length_um, net.length_um[p.comp_index])
        seen += p.net.n_syn
    assert seen == net.n_syn


class _OracleEngine:
    """A part simulated by the FP64 oracle (oracle.Part)."""

    def __init__(self, part):
        self.o = oracle.Part(part.net, n_ext=part.n_ext)

    def step(self, n):
        self.o.step(n)

    def read_fired(self, step0, n):
        return self.o.read_fired(step0, n)

    def inject_spikes(self, ext, steps):
        self.o.inject_spikes(ext, steps)


def _whole(net, steps):
    """The unsplit network in one oracle part: final voltages and every
    spike as (neuron, step)."""
    w = oracle.Part(net)
    w.step(steps)
    rn, rs = w.read_fired(0, steps)
    return w.read_voltages(), rn.astype(np.int64), rs


def test_oracle_part_is_the_oracle_simulation():
    """The steppable oracle part, advanced in uneven pieces, is the oracle's
    whole-run simulation to the bit, spikes included."""
    net = _net(seed=9)
    steps = net.n_steps
    ref = oracle.simulate(net, steps)
    w = oracle.Part(net)
    for k in (1, 37, 100, steps - 138):
        w.step(k)
    np.testing.assert_array_equal(w.read_voltages(), ref.V)
    rn, rs = w.read_fired(0, steps)
    assert len(rn) == ref.n_spikes
    tn, tt = ref.spikes_sorted()
    assert np.all(np.abs(np.sort(rs * net.dt) - np.sort(tt)) <= net.dt)


@pytest.mark.parametrize("n_parts,mode", [(1, "local"), (3, "local"), (4, "global")])
def test_virtual_parts_reproduce_the_whole_network(n_parts, mode):
    net = _net()
    steps = net.n_steps
    V, rn, rs = _whole(net, steps)
    assert len(rn) > 20
    parts = [shard.Part(net, ids) for ids in shard.partition(net, n_parts, mode=mode)]
    run = shard.ShardedRun(net, parts, [_OracleEngine(p) for p in parts], shard.LocalExchange())
    run.run(steps)
    g, st = run.spike_list()
    np.testing.assert_array_equal(np.sort(g * 100000 + st), np.sort(rn * 100000 + rs))
    for p, e in zip(parts, run.engines):
        np.testing.assert_array_equal(e.o.read_voltages(), V[p.comp_index])


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        net = _net(seed=7)
        ids = shard.partition(net, world)[rank]
        part = shard.Part(net, ids)
        run = shard.ShardedRun(net, [part], [_OracleEngine(part)], shard.TorchExchange(device="cpu"))
        run.run(net.n_steps)
        g, st = run.spike_list()
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), g=g, st=st, V=run.engines[0].o.read_voltages(),
                 idx=part.comp_index)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_whole_network(tmp_path):
    import socket

    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    net = _net(seed=7)
    Vw, rn, rs = _whole(net, net.n_steps)
    assert len(rn) > 20
    r0, r1 = (np.load(tmp_path / f"rank{k}.npz") for k in range(2))
    # both ranks saw every spike of the network, the same list
    np.testing.assert_array_equal(r0["g"], r1["g"])
    np.testing.assert_array_equal(r0["st"], r1["st"])
    np.testing.assert_array_equal(np.sort(r0["g"].astype(np.int64) * 100000 + r0["st"]), np.sort(rn * 100000 + rs))
    V = np.full(net.n_comp, np.nan)
    for r in (r0, r1):
        V[r["idx"]] = r["V"]
    np.testing.assert_array_equal(V, Vw)
