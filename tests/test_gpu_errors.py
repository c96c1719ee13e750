"""The boundary's error paths on the GPU, caused on the host (no fault, no
hang): a spike buffer too small (MM_EOVERFLOW), a stimulus that drives the
voltages out of range (MM_ENUMERIC, after which the network answers
MM_ESTATE), and the bounded wait on a barrier that nothing arrives at
(MM_ETIMEOUT, after which the device runs a network normally)."""
import numpy as np
import pytest

from paper_2005_06332_gb300 import mm, netgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    mm.load(build_if_missing=True)


def _net(stim=(0.5, 0.9), n=8):
    return netgen.make_network(n, size_dist=("loguniform", 5, 60), syn_per_neuron=3, seed=71, stim_nA=stim)


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_spike_buffer_overflow_is_reported(precision):
    net = _net()
    with mm.Network(net, precision=precision, spike_capacity=1) as g:
        g.step(400)  # several spikes per neuron
        with pytest.raises(mm.MMError) as e:
            g.read_spikes()
        assert e.value.status == mm.MM_EOVERFLOW
        g.step(10)  # not poisoning: the network keeps running
        assert np.all(np.isfinite(g.read_voltages()))


@pytest.mark.parametrize("precision,stim", [("fp32c", 1e6), ("fp64", 1e308)])
def test_voltages_out_of_range_poison_the_network(precision, stim):
    net = _net(stim=(stim, stim))
    with mm.Network(net, precision=precision) as g:
        g.step(20)
        with pytest.raises(mm.MMError) as e:
            g.synchronize()
        assert e.value.status == mm.MM_ENUMERIC
        with pytest.raises(mm.MMError) as e:
            g.step(1)
        assert e.value.status == mm.MM_ESTATE


def test_bounded_wait_gives_up_and_reports_a_timeout():
    assert mm.selftest_bounded_wait(0, 1000) == mm.MM_ETIMEOUT
    assert mm.selftest_bounded_wait(0, 0) == mm.MM_EINVAL
    # the device stays usable
    net = _net()
    with mm.Network(net, precision="fp32c") as g:
        g.step(40)
        g.synchronize()
        assert np.all(np.isfinite(g.read_voltages()))
