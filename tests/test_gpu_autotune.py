"""Launch-configuration autotuner (mm_autotune): it measures every candidate
on a sample of the network and returns the fastest, and the configuration it
picks changes no result (the per-neuron arithmetic does not depend on how
neurons are packed into work items or on the block shape)."""
import numpy as np
import pytest

from paper_2005_06332_gb300 import mm, netgen

pytestmark = pytest.mark.gpu


def _net():
    return netgen.make_network(300, size_dist=("loguniform", 50, 3000), p_branch=0.1, syn_per_neuron=10, seed=41,
                               stim_nA=(0.2, 0.5))


@pytest.mark.parametrize("precision,threads", [("fp32c", {256, 512, 1024}), ("fp64", {128, 256, 512})])
def test_autotune_returns_the_fastest_measured_candidate(precision, threads):
    net = _net()
    r = mm.autotune(net, precision=precision, sample_comps=net.n_comp // 2, warmup=2, steps=8)
    pts = r["points"]
    assert len(pts) == 12
    assert {p["block_threads"] for p in pts} == threads
    assert {p["group_comps"] for p in pts} == {1024, 2048, 4096, 8192}
    ok = [p for p in pts if p["status"] == "MM_OK"]
    assert ok and all(p["ms_per_step"] > 0 for p in ok)
    best = min(ok, key=lambda p: p["ms_per_step"])
    assert (r["block_threads"], r["group_comps"]) == (best["block_threads"], best["group_comps"])


def test_tuned_configuration_changes_no_result():
    net = _net()
    r = mm.autotune(net, precision="fp32c", sample_comps=net.n_comp // 3, warmup=2, steps=8)
    with mm.Network(net, precision="fp32c") as g:
        g.step(200)
        ref = g.read_voltages()
        ref_spk = g.read_spikes()
    for bt, gc in [(r["block_threads"], r["group_comps"]), (256, 1024), (1024, 8192)]:
        with mm.Network(net, precision="fp32c", block_threads=bt, group_comps=gc) as g:
            g.step(200)
            np.testing.assert_array_equal(g.read_voltages(), ref)
            sn, st = g.read_spikes()
            np.testing.assert_array_equal(np.sort(st), np.sort(ref_spk[1]))


def test_autotune_rejects_bad_arguments():
    net = _net()
    with pytest.raises(mm.MMError):
        mm.autotune(net, precision="fp32c", steps=0)
