"""Pins of the FP64 CPU oracle against things other than itself.

Every check here ties the oracle to the paper, to a closed form, to a
library routine or to a different published formulation, so that a dropped
term, a wrong sign, a transposed operand or a unit slip fails one of them.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.integrate
import scipy.linalg

import oracle
from paper_2005_06332_gb300 import netgen

GOLD = os.path.join(os.path.dirname(__file__), "golden")
P = dict(netgen.DEFAULT_PARAMS)


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _dense(a, b, c, parent):
    """Dense matrix of a Hines system in Algorithm 1's convention:
    A[i,i] = b[i], A[p(i), i] = a[i] (upper), A[i, p(i)] = c[i] (lower)."""
    n = len(b)
    A = np.diag(np.asarray(b, dtype=np.float64))
    for i in range(1, n):
        A[parent[i], i] = a[i]
        A[i, parent[i]] = c[i]
    return A


def _rand_tree(rng, n, p_branch):
    return netgen.random_tree(rng, n, p_branch)


# ---------------------------------------------------------------- Algorithm 1

@pytest.mark.parametrize("seed", range(40))
def test_hines_matches_dense_lu_on_small_random_trees(seed):
    """Algorithm 1 == Gaussian elimination with partial pivoting (LAPACK) on
    random trees of <= 16 compartments; a != c so that swapping the upper and
    lower roles is caught."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 17))
    parent = _rand_tree(rng, n, 0.4)
    a = -rng.uniform(0.1, 1.0, n)
    c = -rng.uniform(0.1, 1.0, n)
    a[0] = c[0] = 0.0
    b = rng.uniform(0.5, 2.0, n) + 2.0 * (np.abs(a) + np.abs(c)) * (n > 1)
    rhs = rng.normal(size=n)
    x = oracle.hines_solve(a, b, c, rhs, parent)
    ref = np.linalg.solve(_dense(a, b, c, parent), rhs)
    assert np.max(np.abs(x - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))


def test_hines_on_chain_matches_banded_lapack():
    """On an unbranched cable the Hines matrix is tridiagonal (Sec. 2 and
    Sec. 5: the Hines algorithm reduces to Thomas)."""
    rng = np.random.default_rng(7)
    n = 300
    parent = np.arange(-1, n - 1, dtype=np.int32)
    g = rng.uniform(0.05, 0.2, n)
    a = -g.copy(); c = -g.copy(); a[0] = c[0] = 0.0
    b = rng.uniform(0.01, 0.05, n)
    b[1:] += g[1:]
    b[:-1] += g[1:]
    rhs = rng.normal(size=n)
    x = oracle.hines_solve(a, b, c, rhs, parent)
    ab = np.zeros((3, n))
    ab[0, 1:] = a[1:]      # superdiagonal: A[i-1, i]
    ab[1, :] = b
    ab[2, :-1] = c[1:]     # subdiagonal:  A[i, i-1]
    ref = scipy.linalg.solve_banded((1, 1), ab, rhs)
    assert np.max(np.abs(x - ref)) <= 1e-11 * np.max(np.abs(ref))


@pytest.mark.parametrize("seed", range(5))
def test_hines_renumbering_invariance(seed):
    """Any relabelling that keeps parent < child solves the same system."""
    rng = np.random.default_rng(100 + seed)
    n = 60
    parent = _rand_tree(rng, n, 0.3)
    g = rng.uniform(0.1, 1.0, n); g[0] = 0
    b = rng.uniform(0.5, 1.0, n)
    for i in range(1, n):
        b[i] += g[i]; b[parent[i]] += g[i]
    rhs = rng.normal(size=n)
    x = oracle.hines_solve(-g, b, -g, rhs, parent)
    # new numbering: a random topological order (children after parents)
    children = [[] for _ in range(n)]
    for i in range(1, n):
        children[parent[i]].append(i)
    order, frontier = [], [0]
    while frontier:
        k = int(rng.integers(0, len(frontier)))
        v = frontier.pop(k)
        order.append(v)
        frontier.extend(children[v])
    new_of = np.empty(n, np.int64); new_of[order] = np.arange(n)
    p2 = np.array([-1] + [new_of[parent[v]] for v in order[1:]], dtype=np.int32)
    assert np.all(p2[1:] < np.arange(1, n))
    x2 = oracle.hines_solve(-g[order], b[order], -g[order], rhs[order], p2)
    assert np.max(np.abs(x2 - x[order])) <= 1e-13 * np.max(np.abs(x))


def test_hines_operation_count_matches_paper():
    gold = _gold("paper_hines_counts.json")
    rng = np.random.default_rng(3)
    for n in (1, 2, 17, 450):
        parent = _rand_tree(rng, n, 0.1)
        g = np.ones(n); g[0] = 0
        _, ops = oracle.hines_solve(-g, 4 * np.ones(n), -g, np.ones(n), parent, count_ops=True)
        assert ops == gold["flops_per_compartment"] * (n - 1) + 1


# ------------------------------------------------------------------ kinetics

def test_rest_steady_state_textbook_values():
    gold = _gold("hh_rest_steady_state.json")
    m, h, n = oracle.gates_inf(gold["V_mV"])
    for got, key in ((m, "m_inf"), (h, "h_inf"), (n, "n_inf")):
        assert abs(got - gold[key]) <= gold["abs_tol"], key


def _hh1952(V):
    """Rates from HH (1952) in their original sign convention."""
    gold = _gold("hh1952_original_rates.json")
    u = -(V + 65.0)
    out = []
    for key in ("alpha_m", "beta_m", "alpha_h", "beta_h", "alpha_n", "beta_n"):
        f = gold[key]
        if f["form"] == "linoid":
            z = u + f["shift"]
            out.append(f["k"] * z / math.expm1(z / f["scale"]))
        elif f["form"] == "exp":
            out.append(f["k"] * math.exp(u / f["scale"]))
        else:
            out.append(f["k"] / (math.exp((u + f["shift"]) / f["scale"]) + 1.0))
    return np.array(out)


@pytest.mark.parametrize("V", [-100.0, -80.0, -65.0, -54.9, -41.3, -20.0, 0.0, 17.5, 45.0])
def test_rates_match_hh1952_original_convention(V):
    np.testing.assert_allclose(oracle.rates(V), _hh1952(V), rtol=1e-12)


def test_rates_singular_points_take_their_limits():
    # alpha_m at V = -40 and alpha_n at V = -55 are 0/0; the limits are 1 and 0.1.
    assert oracle.rates(-40.0)[0] == pytest.approx(1.0, rel=1e-15)
    assert oracle.rates(-55.0)[4] == pytest.approx(0.1, rel=1e-15)
    # near them, the Taylor series of x/(e^x - 1) = 1 - x/2 + x^2/12 - x^4/720
    for V0, k, scale in ((-40.0, 0, 1.0), (-55.0, 4, 0.1)):
        for dv in (-1e-2, -1e-4, -1.01e-5, -9.9e-6, -1e-7, 1e-7, 9.9e-6, 1.01e-5, 1e-4, 1e-2):
            x = -dv / 10.0
            series = 1 - x / 2 + x * x / 12 - x ** 4 / 720
            assert oracle.rates(V0 + dv)[k] == pytest.approx(scale * series, rel=1e-13)


def test_gate_update_under_voltage_clamp_matches_ode():
    """Exponential Euler is exact for frozen V: compare with a tight ODE solve."""
    dt = 0.025
    for V in (-70.0, -30.0, 10.0):
        r = oracle.rates(V)
        x0 = np.array([0.05, 0.6, 0.32])
        x = x0.copy()
        for _ in range(400):
            x = np.array(oracle.gate_step(V, dt, *x))
        al, be = r[0::2], r[1::2]
        sol = scipy.integrate.solve_ivp(lambda t, y: al * (1 - y) - be * y, (0, 400 * dt), x0,
                                        method="DOP853", rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(x, sol.y[:, -1], rtol=1e-10, atol=1e-13)


# ------------------------------------------------------------- cable pieces

def _chain_net(n, L=10.0, d=1.0, stim=0.0, params=None):
    off = np.array([0, n], dtype=np.int64)
    return netgen.Network(
        comp_offset=off, parent=np.arange(-1, n - 1, dtype=np.int32),
        length_um=np.full(n, L), diam_um=np.full(n, d), stim_nA=np.array([stim]),
        syn_src=np.zeros(0, np.int32), syn_dst=np.zeros(0, np.int32), syn_comp=np.zeros(0, np.int32),
        syn_w=np.zeros(0), syn_delay_ms=np.zeros(0), params=dict(params or P), dt=0.025)


def _passive():
    q = dict(P)
    q["gNa"] = 0.0
    q["gK"] = 0.0
    return q


def test_single_passive_compartment_units_and_implicit_step():
    """One passive cylinder: the steady state obeys Ohm's law with the
    textbook membrane area, and the approach is the backward-Euler recurrence
    with time constant Cm/gL (a units check between C and g)."""
    L_um, d_um, I = 20.0, 5.0, 0.05
    net = _chain_net(1, L=L_um, d=d_um, stim=I, params=_passive())
    area_cm2 = math.pi * (d_um * 1e-4) * (L_um * 1e-4)          # cylinder side
    gL_uS = P["gL"] * 1e-3 * area_cm2 * 1e6                      # mS/cm^2 -> S -> uS
    v_ss = P["EL"] + I * 1e-9 / (gL_uS * 1e-6) * 1e3             # nA / uS -> V -> mV
    tau = (P["Cm"] * 1e-6) / (P["gL"] * 1e-3) * 1e3              # F/S -> s -> ms
    dt = 0.025
    for k in (1, 7, 200, 4000):
        V = oracle.simulate(net, k, dt=dt, params=_passive()).V[0]
        expect = v_ss + (P["v_init"] - v_ss) * (1.0 + dt / tau) ** (-k)
        assert abs(V - expect) <= 1e-10 * max(1.0, abs(expect)), k


def test_passive_cable_steady_state_closed_form():
    """Uniform sealed chain, current into compartment 0: the discrete steady
    state is u_k = A cosh(kappa (N - 1/2 - k)), 2 (cosh kappa - 1) = g_m/g_a."""
    N, L_um, d_um, I = 80, 10.0, 1.0, 0.1
    net = _chain_net(N, L=L_um, d=d_um, stim=I, params=_passive())
    V = oracle.simulate(net, 16000, params=_passive()).V
    area_cm2 = math.pi * (d_um * 1e-4) * (L_um * 1e-4)
    g_m = P["gL"] * 1e-3 * area_cm2 * 1e6                         # uS
    r_seg = P["Ra"] * (L_um * 1e-4) / (math.pi * (d_um * 1e-4) ** 2 / 4)  # ohm, one segment
    g_a = 1.0 / r_seg * 1e6                                       # uS between neighbours
    kappa = math.acosh(1.0 + g_m / (2.0 * g_a))
    k = np.arange(N)
    shape = np.cosh(kappa * (N - 0.5 - k))
    # current balance at compartment 0: I = g_m u0 + g_a (u0 - u1)
    A = I / (g_m * shape[0] + g_a * (shape[0] - shape[1]))
    u = A * shape
    np.testing.assert_allclose(V - P["EL"], u, rtol=0, atol=1e-10)


def test_discrete_cable_converges_to_continuous_cable():
    """Sealed passive cable of length l = 1 mm with a current I into its first
    segment: the potential at the first node (x = dx/2) converges, second order
    in dx, to the continuous cable's I r_a lambda cosh((l - x)/lambda) / sinh(l/lambda)
    with the textbook r_a = 4 Ra/(pi d^2), r_m = Rm/(pi d), lambda = sqrt(r_m/r_a)."""
    d_um, total_um, I = 1.0, 1000.0, 0.01
    Rm = 1.0 / (P["gL"] * 1e-3)                                  # ohm cm^2
    r_a = 4.0 * P["Ra"] / (math.pi * (d_um * 1e-4) ** 2)         # ohm / cm
    r_m = Rm / (math.pi * d_um * 1e-4)                           # ohm cm
    lam = math.sqrt(r_m / r_a)                                    # cm
    l_cm = total_um * 1e-4
    errs = []
    for n in (25, 50, 100):
        seg = total_um / n
        x = 0.5 * seg * 1e-4
        R_cont = r_a * lam * math.cosh((l_cm - x) / lam) / math.sinh(l_cm / lam) * 1e-6  # MOhm
        net = _chain_net(n, L=seg, d=d_um, stim=I, params=_passive())
        V = oracle.simulate(net, 20000, params=_passive()).V
        errs.append(abs((V[0] - P["EL"]) / I - R_cont) / R_cont)  # mV / nA = MOhm
    assert errs[-1] < 1e-4
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5


def test_assembly_conserves_charge_and_is_symmetric():
    """Axial terms only move charge between compartments: with any state,
    sum_i (C_i/dt + G_i) dV_i = sum_i (-I_i) + I_stim, where the uncoupled
    terms come from the same assembly with the axial conductances removed."""
    net = netgen.make_network(1, size_dist=("mono", 120), p_branch=0.2, syn_per_neuron=0, seed=5)
    rng = np.random.default_rng(5)
    n = net.n_comp
    area, Cn, gax = oracle.geometry(net.comp_offset, net.parent, net.length_um, net.diam_um, P)
    V = rng.uniform(-80, 30, n)
    m, h, nn = rng.uniform(0, 1, (3, n))
    gs = rng.uniform(0, 0.01, n)
    dt = 0.025
    a, b, c, rhs = oracle.assemble(net.parent, V, m, h, nn, gs, area, Cn, gax, 0.3, P, dt)
    np.testing.assert_array_equal(a, c)
    a0, b0, c0, rhs0 = oracle.assemble(net.parent, V, m, h, nn, gs, area, Cn, np.zeros(n), 0.3, P, dt)
    dV = oracle.hines_solve(a, b, c, rhs, net.parent)
    lhs = np.sum(b0 * dV)
    assert abs(lhs - np.sum(rhs0)) <= 1e-12 * np.sum(np.abs(rhs0))
    # Laplacian rows sum to zero: diagonal minus uncoupled part == sum of |off-diagonals| in the row
    A = _dense(a, b, c, net.parent)
    np.testing.assert_allclose(A.sum(axis=1), b0, rtol=1e-12, atol=1e-15)


# ------------------------------------------------------- single HH compartment

def _hh_reference_spikes(area_cm2, I_nA, t_stop):
    """Continuous single-compartment HH, integrated with DOP853 at tight tolerance."""
    s = area_cm2 * 1e3
    Cn = P["Cm"] * area_cm2 * 1e3

    def f(t, y):
        V, m, h, n = y
        r = oracle.rates(V)
        I = (P["gNa"] * s * m ** 3 * h * (V - P["ENa"]) + P["gK"] * s * n ** 4 * (V - P["EK"])
             + P["gL"] * s * (V - P["EL"]))
        return [(-I + I_nA) / Cn, r[0] * (1 - m) - r[1] * m, r[2] * (1 - h) - r[3] * h,
                r[4] * (1 - n) - r[5] * n]

    def up(t, y):
        return y[0] - P["threshold"]
    up.direction = 1
    y0 = [P["v_init"], *oracle.gates_inf(P["v_init"])]
    sol = scipy.integrate.solve_ivp(f, (0, t_stop), y0, method="DOP853", rtol=1e-10, atol=1e-12,
                                    events=up, max_step=0.05)
    return sol.t_events[0]


def _oracle_spikes(L_um, d_um, I, dt, t_stop):
    net = _chain_net(1, L=L_um, d=d_um, stim=I)
    r = oracle.simulate(net, int(round(t_stop / dt)), dt=dt)
    return np.sort(r.spk_t)


def test_single_compartment_hh_spike_times_match_tight_ode_solve():
    L_um, d_um = 30.0, 30.0
    area = math.pi * d_um * L_um * 1e-8
    I = 10.0 * area * 1e3                                       # 10 uA/cm^2 in nA
    t_stop = 100.0
    ref = _hh_reference_spikes(area, I, t_stop)
    got = _oracle_spikes(L_um, d_um, I, 0.025, t_stop)
    assert len(ref) >= 5
    assert len(got) == len(ref)
    assert abs(got[0] - ref[0]) < 0.1
    # first-order convergence of the first spike time in dt
    errs = []
    dts = (0.1, 0.05, 0.025, 0.0125)
    for dt in dts:
        errs.append(abs(_oracle_spikes(L_um, d_um, I, dt, 30.0)[0] - ref[0]))
    slope = np.polyfit(np.log(dts), np.log(errs), 1)[0]
    assert 0.7 < slope < 1.4, (errs, slope)


# ---------------------------------------------------------- events and delays

def _pair_net(delay_ms, w=0.01):
    """Neuron 0 (large stimulus) drives neuron 1 through one synapse."""
    off = np.array([0, 1, 4], dtype=np.int64)
    return netgen.Network(
        comp_offset=off, parent=np.array([-1, -1, 0, 1], dtype=np.int32),
        length_um=np.full(4, 20.0), diam_um=np.full(4, 10.0), stim_nA=np.array([0.5, 0.0]),
        syn_src=np.array([0], np.int32), syn_dst=np.array([1], np.int32), syn_comp=np.array([2], np.int32),
        syn_w=np.array([w]), syn_delay_ms=np.array([delay_ms]), params=dict(P), dt=0.025)


@pytest.mark.parametrize("delay_ms", [1.0, 1.2374, 4.99])
def test_single_event_arrival_step_and_exponential_decay(delay_ms):
    net = _pair_net(delay_ms)
    dt = net.dt
    r = oracle.simulate(net, 600, record_soma=True)
    tr = r.soma_trace[0]
    ns = int(np.nonzero((tr[:-1] < 0.0) & (tr[1:] >= 0.0))[0][0])   # crossing inside step ns
    arrival = ns + 1 + int(round(delay_ms / dt))
    tau = P["tau_syn"]
    before = oracle.simulate(net, arrival).g
    assert np.all(before == 0.0)
    for j in (1, 2, 9):
        g = oracle.simulate(net, arrival + j).g
        assert g[1 + 2] == pytest.approx(0.01 * math.exp(-j * dt / tau), rel=1e-14)
        assert np.count_nonzero(g) == 1


def test_causality_within_min_delay():
    """No event reaches another neuron sooner than the minimum delay: over the
    first round(1 ms/dt) + 1 steps every neuron of a connected network follows
    its isolated trajectory bit for bit (local vs global steps, Sec. 2)."""
    net = netgen.make_network(40, size_dist=("loguniform", 20, 200), p_branch=("uniform", 0.02, 0.2),
                              syn_per_neuron=10, seed=11, stim_nA=(2.0, 4.0), weight_uS=(0.5, 1.0))
    d = int(round(1.0 / net.dt))
    iso = net.subset(range(net.n_neurons), keep_synapses=False)
    a = oracle.simulate(net, d + 1)
    b = oracle.simulate(iso, d + 1)
    np.testing.assert_array_equal(a.V, b.V)
    # and the network is not trivially isolated: later on the synapses matter
    a2 = oracle.simulate(net, 8 * d)
    b2 = oracle.simulate(iso, 8 * d)
    assert a.n_spikes > 0
    assert np.max(np.abs(a2.V - b2.V)) > 1e-3


# ------------------------------------- Eq. 2 as printed (scheme "cn"): pins

def test_cn_single_passive_compartment_is_forward_euler_in_the_current():
    """With one compartment there is no axial coupling: Eq. 2 as printed keeps
    the membrane current explicit, so the approach to the Ohm's-law steady
    state is the forward-Euler recurrence (1 - dt/tau)^k, not (1 + dt/tau)^-k."""
    L_um, d_um, I = 20.0, 5.0, 0.05
    net = _chain_net(1, L=L_um, d=d_um, stim=I, params=_passive())
    area_cm2 = math.pi * (d_um * 1e-4) * (L_um * 1e-4)
    gL_uS = P["gL"] * 1e-3 * area_cm2 * 1e6
    v_ss = P["EL"] + I * 1e-9 / (gL_uS * 1e-6) * 1e3
    tau = (P["Cm"] * 1e-6) / (P["gL"] * 1e-3) * 1e3
    dt = 0.025
    for k in (1, 7, 200, 4000):
        V = oracle.simulate(net, k, dt=dt, params=_passive(), scheme="cn").V[0]
        expect = v_ss + (P["v_init"] - v_ss) * (1.0 - dt / tau) ** k
        assert abs(V - expect) <= 1e-10 * max(1.0, abs(expect)), k


def test_cn_passive_cable_steady_state_is_the_same_closed_form():
    """The discrete steady state does not depend on the time scheme: the
    sealed passive chain reaches the cosh profile of the backward-Euler pin."""
    N, L_um, d_um, I = 40, 10.0, 1.0, 0.1
    net = _chain_net(N, L=L_um, d=d_um, stim=I, params=_passive())
    V = oracle.simulate(net, 16000, params=_passive(), scheme="cn").V
    area_cm2 = math.pi * (d_um * 1e-4) * (L_um * 1e-4)
    g_m = P["gL"] * 1e-3 * area_cm2 * 1e6
    r_seg = P["Ra"] * (L_um * 1e-4) / (math.pi * (d_um * 1e-4) ** 2 / 4)
    g_a = 1.0 / r_seg * 1e6
    kappa = math.acosh(1.0 + g_m / (2.0 * g_a))
    k = np.arange(N)
    shape = np.cosh(kappa * (N - 0.5 - k))
    A = I / (g_m * shape[0] + g_a * (shape[0] - shape[1]))
    np.testing.assert_allclose(V - P["EL"], A * shape, rtol=0, atol=1e-10)


def test_cn_pure_diffusion_is_second_order_in_dt_backward_euler_first():
    """No membrane current (gL = 0): C dV/dt = -K V + b with K the chain's
    axial Laplacian and b the current into compartment 0 -- exactly solvable
    with a matrix exponential.  Half of each coupling implicit and half
    explicit (Eq. 2 as printed) is Crank-Nicolson: once dt resolves the
    stiffest coupling, the error at t = 2 ms falls 4x per halving of dt; the
    backward-Euler reading falls 2x."""
    N, L_um, d_um, I, T = 12, 20.0, 1.0, 0.05, 2.0
    params = dict(_passive())
    params["gL"] = 0.0
    net = _chain_net(N, L=L_um, d=d_um, stim=I, params=params)
    area, Cn, gax = oracle.geometry(net.comp_offset, net.parent, net.length_um, net.diam_um, params)
    K = np.zeros((N, N))
    for i in range(1, N):
        g = gax[i]
        K[i, i] += g
        K[i - 1, i - 1] += g
        K[i, i - 1] -= g
        K[i - 1, i] -= g
    Minv = np.diag(1.0 / Cn)
    b = np.zeros(N)
    b[0] = I
    # augmented system d/dt [V; 1] = [[-M^-1 K, M^-1 b], [0, 0]] [V; 1]
    Aug = np.zeros((N + 1, N + 1))
    Aug[:N, :N] = -Minv @ K
    Aug[:N, N] = Minv @ b
    y0 = np.append(np.full(N, params["v_init"]), 1.0)
    exact = (scipy.linalg.expm(Aug * T) @ y0)[:N]
    errs = {}
    for scheme in ("cn", "be"):
        errs[scheme] = []
        for dt in (0.05, 0.025, 0.0125):
            V = oracle.simulate(net, int(round(T / dt)), dt=dt, params=params, scheme=scheme).V
            errs[scheme].append(np.max(np.abs(V - exact)))
    e = errs["cn"]
    assert 3.6 < e[0] / e[1] < 4.4 and 3.6 < e[1] / e[2] < 4.4, e
    e = errs["be"]
    assert 1.8 < e[0] / e[1] < 2.5 and 1.8 < e[1] / e[2] < 2.5, e


def test_cn_assembly_conserves_charge_and_halves_the_couplings():
    """Eq. 2 as printed: off-diagonals are half the axial conductances, the
    diagonal is C/dt plus half the couplings of the row (rows of the coupling
    part sum to zero), and the axial terms still only move charge:
    sum_i (C_i/dt) dV_i = sum_i (-I_i) + I_stim."""
    net = netgen.make_network(1, size_dist=("mono", 90), p_branch=0.2, syn_per_neuron=0, seed=6)
    rng = np.random.default_rng(6)
    n = net.n_comp
    area, Cn, gax = oracle.geometry(net.comp_offset, net.parent, net.length_um, net.diam_um, P)
    V = rng.uniform(-80, 30, n)
    m, h, nn = rng.uniform(0, 1, (3, n))
    gs = rng.uniform(0, 0.01, n)
    dt = 0.025
    a, b, c, rhs = oracle.assemble(net.parent, V, m, h, nn, gs, area, Cn, gax, 0.3, P, dt, scheme="cn")
    np.testing.assert_array_equal(a, c)
    np.testing.assert_allclose(a[1:], -0.5 * gax[1:], rtol=1e-15)
    A = _dense(a, b, c, net.parent)
    np.testing.assert_allclose(A.sum(axis=1), Cn / dt, rtol=1e-12)
    _, _, _, rhs_be = oracle.assemble(net.parent, V, m, h, nn, gs, area, Cn, gax, 0.3, P, dt)
    np.testing.assert_array_equal(rhs, rhs_be)  # same explicit rhs in both readings
    dV = oracle.hines_solve(a, b, c, rhs, net.parent)
    lhs = np.sum(Cn / dt * dV)
    _, _, _, rhs0 = oracle.assemble(net.parent, V, m, h, nn, gs, area, Cn, np.zeros(n), 0.3, P, dt, scheme="cn")
    assert abs(lhs - np.sum(rhs0)) <= 1e-12 * np.sum(np.abs(rhs0))


# ------------------------- spike detection at synapse points (Sec. 2): pins

def _points_net(n_src, parent, L, d, stim, points, w=None, delays=None, params=None):
    """Neuron 0 (the given tree) with one synapse leaving each listed point
    towards a 3-compartment passive neuron 1 (compartment k % 3)."""
    n0 = len(parent)
    off = np.array([0, n0, n0 + 3], dtype=np.int64)
    S = len(points)
    return netgen.Network(
        comp_offset=off, parent=np.concatenate([parent, [-1, 0, 1]]).astype(np.int32),
        length_um=np.concatenate([L, np.full(3, 10.0)]), diam_um=np.concatenate([d, np.full(3, 1.0)]),
        stim_nA=np.array([stim, 0.0]),
        syn_src=np.zeros(S, np.int32), syn_dst=np.ones(S, np.int32),
        syn_comp=(np.arange(S) % 3).astype(np.int32),
        syn_w=np.zeros(S) if w is None else np.asarray(w, np.float64),
        syn_delay_ms=np.full(S, 1.0) if delays is None else np.asarray(delays, np.float64),
        params=dict(params or P), dt=0.025, syn_src_comp=np.asarray(points, np.int32))


def test_point_spike_times_match_a_dense_passive_recurrence():
    """A passive tree under a soma current rises monotonically towards its
    steady state, so each point crosses a threshold below its steady state
    exactly once.  The oracle's point spikes (compartment and interpolated
    time) must be those of the backward-Euler recurrence written as a dense
    linear system, (C/dt + G_m + K) dV = -G_m (V - E_L) - K V + b, and points
    whose steady state stays below the threshold must never fire."""
    rng = np.random.default_rng(21)
    n = 24
    parent = _rand_tree(rng, n, 0.3)
    L = rng.uniform(5.0, 20.0, n)
    d = rng.uniform(0.5, 2.0, n)
    I, dt, steps = 0.05, 0.025, 1200
    params = _passive()
    params["threshold"] = 0.0  # replaced below
    net0 = _points_net(1, parent, L, d, I, [0])
    area, Cn, gax = oracle.geometry(net0.comp_offset[:2], net0.parent[:n], L, d, params)
    Gm = params["gL"] * area * 1e3
    K = np.zeros((n, n))
    for i in range(1, n):
        g, q = gax[i], parent[i]
        K[i, i] += g
        K[q, q] += g
        K[i, q] -= g
        K[q, i] -= g
    A = np.diag(Cn / dt + Gm) + K
    b = np.zeros(n)
    b[0] = I
    V = np.full(n, params["v_init"])
    trace = [V.copy()]
    for _ in range(steps):
        V = V + np.linalg.solve(A, -Gm * (V - params["EL"]) - K @ V + b)
        trace.append(V.copy())
    trace = np.array(trace)
    assert np.all(np.diff(trace, axis=0) >= -1e-12)  # monotone rise
    final = trace[-1]
    theta = 0.5 * (final.max() + final.min())
    params["threshold"] = theta
    points = list(range(n))
    net = _points_net(1, parent, L, d, I, points, params=params)
    r = oracle.simulate(net, steps, dt=dt, params=params, detect="points")
    nrn, comp, t = r.point_spikes_sorted()
    expect = {}
    for c in points:
        k = np.nonzero((trace[:-1, c] < theta) & (trace[1:, c] >= theta))[0]
        if len(k):
            v0, v1 = trace[k[0], c], trace[k[0] + 1, c]
            expect[c] = k[0] * dt + dt * (theta - v0) / (v1 - v0)
    assert 0 < len(expect) < n
    assert np.all(nrn == 0)
    got = dict(zip(comp.tolist(), t.tolist()))
    assert sorted(got) == sorted(expect)
    for c in expect:
        assert got[c] == pytest.approx(expect[c], abs=1e-9)


def test_point_spikes_route_to_the_synapses_leaving_each_point():
    """An HH neuron firing repeatedly, with synapses of different weights and
    delays leaving the soma, a middle and a distal compartment towards a
    passive neuron: the target conductances after the run are the sum over
    the recorded spikes of each point, over the synapses leaving it, of
    w exp(-(n - arrival) dt / tau), arrival = spike step + 1 + round(delay/dt)."""
    n = 40
    parent = np.arange(-1, n - 1, dtype=np.int32)
    L, d = np.full(n, 10.0), np.full(n, 2.0)
    points = [0, 20, 39, 39, 0, 20]
    w = [0.011, 0.023, 0.037, 0.041, 0.053, 0.067]
    delays = [1.0, 2.5, 1.3, 4.0, 3.1, 1.7]
    params = dict(P)
    params["gL"] = 0.3
    net = _points_net(1, parent, L, d, 0.4, points, w=w, delays=delays, params=params)
    steps = 1600
    r = oracle.simulate(net, steps, detect="points")
    nrn, comp, t = r.point_spikes_sorted()
    assert r.n_spikes >= 6 and set(comp.tolist()) == {0, 20, 39}
    dt, tau = net.dt, P["tau_syn"]
    g = np.zeros(3)
    for c, ts in zip(comp, t):
        step = int(math.ceil(ts / dt - 1e-9)) - 1
        for s, pc in enumerate(points):
            if pc != c:
                continue
            arrival = step + 1 + int(round(delays[s] / dt))
            if arrival < steps:
                g[s % 3] += w[s] * math.exp(-(steps - arrival) * dt / tau)
    np.testing.assert_allclose(r.g[n:], g, rtol=1e-12, atol=1e-300)


def test_point_spikes_propagate_along_an_unbranched_cable():
    """The action potential that the onset of a soma current starts on a
    uniform HH cable reaches every point, later the farther the point is from
    the soma, at a constant speed away from the ends (equal delays between
    equally spaced interior points)."""
    n = 60
    parent = np.arange(-1, n - 1, dtype=np.int32)
    points = [0, 10, 20, 30, 40, 50, 59]
    net = _points_net(1, parent, np.full(n, 10.0), np.full(n, 2.0), 0.6, points)
    r = oracle.simulate(net, 400, detect="points")
    nrn, comp, t = r.point_spikes_sorted()
    first = [np.min(t[comp == c]) for c in points]
    assert np.all(np.diff(first) > 0), first
    lag = np.diff(first)[1:4]  # 10 -> 20 -> 30 -> 40
    assert np.max(lag) < 1.1 * np.min(lag), lag


def test_points_at_every_soma_are_soma_detection():
    """With every synapse leaving its source's soma, detection at synapse
    points is the soma test of every neuron that has an outgoing synapse:
    the same spikes (bit for bit) and the same final state."""
    net = netgen.make_network(16, size_dist=("loguniform", 20, 120), p_branch=0.15, syn_per_neuron=6, seed=23,
                              stim_nA=(0.3, 0.6), weight_uS=(0.0, 0.02))
    net.syn_src_comp = np.zeros(net.n_syn, np.int32)
    a = oracle.simulate(net, 1200)
    b = oracle.simulate(net, 1200, detect="points")
    np.testing.assert_array_equal(a.V, b.V)
    has_out = np.zeros(net.n_neurons, bool)
    has_out[net.syn_src] = True
    na, ta = a.spikes_sorted()
    keep = has_out[na]
    nb, cb, tb = b.point_spikes_sorted()
    assert a.n_spikes > 10
    np.testing.assert_array_equal(nb, na[keep])
    np.testing.assert_array_equal(tb, ta[keep])
    assert np.all(cb == 0)
