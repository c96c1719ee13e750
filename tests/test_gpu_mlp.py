"""The learned cost model's BF16 kernels against the FP64 MLP oracle, its
training, and the learned work-queue order."""
import numpy as np
import pytest

from oracle import mlp as omlp
from paper_2005_06332_gb300 import mm, netgen, schedule

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    mm.load(build_if_missing=True)


def _theta(rng):
    t = rng.normal(scale=0.3, size=omlp.N_PARAMS).astype(np.float32)
    return t


def test_loss_and_gradient_match_fp64_oracle():
    rng = np.random.default_rng(0)
    theta = _theta(rng)
    X = rng.normal(size=(257, 16)).astype(np.float32)
    y = rng.normal(size=257).astype(np.float32)
    m = mm.MLP(1)
    try:
        m.set_params(theta)
        loss, g = m.loss_grad(X, y)
    finally:
        m.close()
    tb = omlp.bf16(theta)                     # the kernels compute with BF16 weights
    ref_loss, ref_g = omlp.loss_grad(tb, X.astype(np.float64), y.astype(np.float64))
    assert loss == pytest.approx(ref_loss, rel=1e-5)
    scale = np.max(np.abs(ref_g))
    assert np.max(np.abs(g - ref_g)) <= 1e-5 * scale


def test_prediction_matches_oracle_with_standardisation():
    rng = np.random.default_rng(3)
    theta = _theta(rng)
    X = rng.normal(loc=2.0, scale=3.0, size=(100, 16)).astype(np.float32)
    mu, sd = X.mean(0), X.std(0)
    m = mm.MLP(2)
    try:
        m.set_params(theta)
        m.set_normalisation(mu, sd, 1.5, 0.25)
        p = m.predict(X)
    finally:
        m.close()
    Xs = (X.astype(np.float64) - mu) / sd
    ref, _ = omlp.forward(omlp.bf16(theta), Xs)
    np.testing.assert_allclose(p, ref * 0.25 + 1.5, rtol=1e-4, atol=1e-4)


def test_training_fits_a_smooth_target():
    rng = np.random.default_rng(4)
    X = rng.normal(size=(2000, 16)).astype(np.float32)
    y = (np.sin(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2] + 0.3 * X[:, 3]).astype(np.float32)
    m = mm.MLP(5)
    try:
        losses = m.train(X, y, epochs=400, lr=3e-3)
    finally:
        m.close()
    assert losses[-1] < 0.15 * losses[0]


def test_cost_order_changes_no_result():
    """Any work-queue order gives the same voltages (no synapses: neurons are independent)."""
    net = netgen.make_network(60, size_dist=("loguniform", 20, 600), p_branch=("uniform", 0.02, 0.2),
                              syn_per_neuron=0, seed=8, stim_nA=(0.3, 0.8))
    with mm.Network(net, precision="fp32c") as a:
        a.step(200)
        va = a.read_voltages()
    rng = np.random.default_rng(9)
    with mm.Network(net, precision="fp32c", cost=rng.random(net.n_neurons).astype(np.float32)) as b:
        b.step(200)
        vb = b.read_voltages()
    np.testing.assert_array_equal(va, vb)


def test_learned_costs_predict_measured_solve_times():
    net = netgen.make_config("lognormal100k", n_neurons=1500, syn_per_neuron=10)
    r = schedule.learn_costs(net, n_timed=1200, steps=30, epochs=500)
    assert r["cost"].shape == (net.n_neurons,)
    assert r["mean_time_us"] > 0
    assert r["r2_holdout"] > 0.5, r
    t = schedule.measure_neuron_times(net, np.arange(50), steps=10)
    assert t.shape == (50,) and np.all(t > 0)


def test_native_train_schedule_learns_solve_times():
    """mm_train_schedule, the same pipeline as one native call: costs for
    every neuron, positive and finite, ordering the neurons like their
    measured solve times (held-out R^2 of log time) and, for this size
    distribution, nearly like their sizes; a network built with them runs."""
    net = netgen.make_config("lognormal100k", n_neurons=1500, syn_per_neuron=10)
    r = mm.train_schedule(net, n_timed=1200, steps=30, epochs=500, seed=3)
    c = r["cost"]
    assert c.shape == (net.n_neurons,) and np.all(np.isfinite(c)) and np.all(c > 0)
    assert r["n_timed"] == 1200 and r["n_holdout"] == 240
    assert r["r2_holdout"] > 0.5, r
    rank = lambda x: np.argsort(np.argsort(x))
    rho = np.corrcoef(rank(c), rank(net.sizes()))[0, 1]
    assert rho > 0.8, rho
    with mm.Network(net, precision="fp32c", cost=c) as g:
        g.step(20)
        assert np.all(np.isfinite(g.read_voltages()))


def test_native_train_schedule_rejects_bad_arguments():
    net = netgen.make_network(20, size_dist=("mono", 30), syn_per_neuron=0, seed=4)
    with pytest.raises(mm.MMError) as e:
        mm.train_schedule(net, n_timed=5)
    assert e.value.status == mm.MM_EINVAL


def _ms_per_step(net, cost, group_comps, steps=200):
    import torch
    s = torch.cuda.Stream()
    with mm.Network(net, precision="fp32c", cost=cost, block_threads=512, group_comps=group_comps,
                    stream=s.cuda_stream) as g:
        g.step(45)
        g.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        g.step(steps)
        e1.record(s)
        e1.synchronize()
        return e0.elapsed_time(e1) / steps


def test_learned_model_predicts_solve_time_where_size_does_not():
    """shapes10k: half the neurons unbranched chains, half bushy trees, sizes
    log-uniform, so size alone predicts a neuron's solve time poorly.  The
    trained network predicts it (held-out R^2 of log time) far better than
    the least-squares fit on log size."""
    net = netgen.make_config("shapes10k")
    r = mm.train_schedule(net, n_timed=5000, steps=30, epochs=600, seed=1)
    print(f"R2 learned {r['r2_holdout']:.3f}, size only {r['r2_holdout_size_only']:.3f}")
    assert r["r2_holdout"] > 0.85 and r["r2_holdout"] > r["r2_holdout_size_only"] + 0.15, r


def test_learned_order_gains_on_the_papers_f_distributed_sizes():
    """paper_fisher (Sec. 4's realistic case: 10,000 neurons, F-distributed
    sizes of mean 300): the work queue in the learned order makes the step
    faster than in size order at the library's default work-item budget.
    The two orders are timed three times each, interleaved, and the best of
    each compared; the gain must exceed twice the run-to-run spread.
    (Measured: +2.5 %, spread 0.2 %; on other workloads and item budgets
    the two orders are within a few per cent either way.)"""
    net = netgen.make_config("paper_fisher")
    r = mm.train_schedule(net, n_timed=5000, steps=30, epochs=600, seed=1)
    t_size, t_learned = [], []
    for _ in range(3):
        t_size.append(_ms_per_step(net, None, 2048))
        t_learned.append(_ms_per_step(net, r["cost"], 2048))
    gain = min(t_size) / min(t_learned) - 1.0
    spread = max(max(t_size) / min(t_size), max(t_learned) / min(t_learned)) - 1.0
    print(f"size order {min(t_size):.4f} ms, learned order {min(t_learned):.4f} ms, gain {gain:+.2%}, "
          f"run-to-run spread {spread:.2%}")
    assert gain > 0.01 and gain > 2 * spread
