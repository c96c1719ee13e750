"""The seeded input generator (netgen): the workload recipes hold what they
state -- tree structure, size distributions, synapse wiring, source points,
branch-probability mixtures -- and a seed gives the same network every time
(no GPU)."""
import math

import numpy as np
import pytest

from paper_2005_06332_gb300 import netgen


def test_random_tree_parents_and_branching_rate():
    rng = np.random.default_rng(0)
    for p in (0.0, 0.1, 0.5):
        par = netgen.random_tree(rng, 20000, p)
        assert par[0] == -1 and np.all(par[1:] < np.arange(1, 20000)) and np.all(par[1:] >= 0)
        jumps = np.mean(par[1:] != np.arange(0, 19999))
        # a jump to a uniform earlier compartment lands on i-1 with probability 1/i
        assert abs(jumps - p) < 0.01, (p, jumps)


@pytest.mark.parametrize("dist,check", [
    (("mono", 255), lambda s: np.all(s == 255)),
    (("loguniform", 50, 5000), lambda s: s.min() >= 50 and s.max() <= 5000
     and abs(np.median(np.log(s)) - 0.5 * (math.log(50) + math.log(5000))) < 0.1),
    (("lognormal", 800, 1.0, 20, 20000), lambda s: s.min() >= 20 and s.max() <= 20000
     and abs(np.median(s) / 800 - 1) < 0.05),
    (("group", 20, 700, 300), lambda s: len(np.unique(s)) <= 20 and s.max() - s.min() <= 701),
    (("fisher", 10, 40, 300, 10, 5000), lambda s: s.min() >= 10 and s.max() <= 5000
     and abs(s.mean() / 300 - 1) < 0.05),
])
def test_size_distributions(dist, check):
    s = netgen.draw_sizes(np.random.default_rng(1), 20000, dist)
    assert check(s), (dist, s.min(), s.max(), s.mean())


def test_group_of_twenty_has_the_stated_spread_and_mean():
    """Sec. 4's group: 20 sizes at most 700 apart with mean 300 (reading c18).
    Every neuron picks one of the 20 uniformly, so many draws show the
    group's spread exactly and its mean to within sampling error (two of the
    rounded sizes may coincide)."""
    for seed in (5, 6, 7):
        s = netgen.draw_sizes(np.random.default_rng(seed), 200000, ("group", 20, 700, 300))
        g = np.unique(s)
        assert len(g) <= 20
        assert abs((g.max() - g.min()) - 700) <= 1
        assert abs(s.mean() - 300) < 3.0, s.mean()


def test_synapses_sources_targets_and_points():
    net = netgen.make_network(50, size_dist=("loguniform", 5, 300), syn_per_neuron=7, seed=3,
                              delay_ms=("uniform", 1.0, 5.0), src_points=True)
    sizes = net.sizes()
    assert net.n_syn == 50 * 7
    np.testing.assert_array_equal(np.bincount(net.syn_dst, minlength=50), np.full(50, 7))
    assert np.all(net.syn_src != net.syn_dst)                    # no self-synapse
    assert np.all((net.syn_comp >= 0) & (net.syn_comp < sizes[net.syn_dst]))
    assert np.all((net.syn_src_comp >= 0) & (net.syn_src_comp < sizes[net.syn_src]))
    assert np.all((net.syn_delay_ms >= 1.0) & (net.syn_delay_ms <= 5.0))
    assert np.all((net.syn_w >= 0.0) & (net.syn_w <= 0.05))


def test_source_points_leave_the_rest_of_the_network_unchanged():
    a = netgen.make_network(30, size_dist=("loguniform", 5, 300), syn_per_neuron=5, seed=4)
    b = netgen.make_network(30, size_dist=("loguniform", 5, 300), syn_per_neuron=5, seed=4, src_points=True)
    assert a.syn_src_comp is None and b.syn_src_comp is not None
    for k in ("comp_offset", "parent", "length_um", "diam_um", "stim_nA", "syn_src", "syn_dst", "syn_comp",
              "syn_w", "syn_delay_ms"):
        np.testing.assert_array_equal(getattr(a, k), getattr(b, k), err_msg=k)


def test_branch_probability_choice_gives_chains_and_bushy_trees():
    net = netgen.make_network(400, size_dist=("loguniform", 200, 3000), p_branch=("choice", 0.0, 0.5),
                              syn_per_neuron=0, seed=8)
    chains = 0
    for k in range(net.n_neurons):
        b, e = net.comp_offset[k], net.comp_offset[k + 1]
        par = net.parent[b:e]
        jumps = np.mean(par[1:] != np.arange(0, e - b - 1))
        if jumps == 0.0:
            chains += 1
        else:
            assert abs(jumps - 0.5) < 0.1
    assert 150 < chains < 250


def test_a_seed_gives_the_same_network():
    a = netgen.make_config("multi10k", n_neurons=200)
    b = netgen.make_config("multi10k", n_neurons=200)
    for k in ("comp_offset", "parent", "length_um", "diam_um", "stim_nA", "syn_src", "syn_dst", "syn_comp",
              "syn_w", "syn_delay_ms"):
        np.testing.assert_array_equal(getattr(a, k), getattr(b, k), err_msg=k)
