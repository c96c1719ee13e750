"""Host logic: the spike-source tables of the layout (mm_layout.cpp), dumped
by tests/sources_check.cpp and recomputed here from the synapse arrays (no
GPU): the sources (neurons, or the distinct (neuron, compartment) points
synapses leave from), the outgoing synapses of each source sorted by delay,
the incoming synapses of each site in ascending synapse id (deterministic
delivery), and under point detection the per-compartment point ids, the
soma point of each neuron and each point's user neuron and compartment."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2005_06332_gb300 import netgen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2005_06332_gb300", "csrc")
DT = 0.025


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    cuda_inc = None
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "include", "vector_types.h")):
            cuda_inc = os.path.join(c, "include")
    if cuda_inc is None:
        pytest.skip("CUDA headers not available")
    out = str(tmp_path_factory.mktemp("sources") / "sources_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-I" + CSRC, "-I" + os.path.join(ROOT, "include"), "-I" + cuda_inc,
                    os.path.join(ROOT, "tests", "sources_check.cpp"), os.path.join(CSRC, "mm_layout.cpp"), "-o", out],
                   check=True, capture_output=True)
    return out


def _dump(checker, tmp_path, net, points):
    S = net.n_syn
    scomp = net.syn_src_comp if net.syn_src_comp is not None else np.zeros(S, np.int32)
    f, o = tmp_path / "net.bin", tmp_path / "out.bin"
    with open(f, "wb") as fh:
        np.array([net.n_neurons], np.int32).tofile(fh)
        np.array([net.n_comp, S], np.int64).tofile(fh)
        net.comp_offset.astype(np.int64).tofile(fh)
        for a in (net.parent, net.syn_src, net.syn_dst, net.syn_comp, scomp):
            np.asarray(a, np.int32).tofile(fh)
        for a in (net.syn_w, net.syn_delay_ms):
            np.asarray(a, np.float64).tofile(fh)
    r = subprocess.run([checker, str(f), "1" if points else "0", str(o)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    b = open(o, "rb").read()
    pos = 0

    def take(dtype, n):
        nonlocal pos
        a = np.frombuffer(b, dtype=dtype, count=n, offset=pos)
        pos += a.nbytes
        return a

    n_src = int(take(np.int32, 1)[0])
    nsite = int(take(np.int64, 1)[0])
    C, N = net.n_comp, net.n_neurons
    d = dict(n_src=n_src, nsite=nsite, user2int=take(np.int64, C), internal_of=take(np.int32, N),
             site_internal=take(np.int64, nsite), out_off=take(np.int64, n_src + 1), out_site=take(np.int32, S),
             out_dsteps=take(np.int32, S), out_w=take(np.float64, S), in_off=take(np.int64, nsite + 1),
             in_src=take(np.int32, S), in_dsteps=take(np.int32, S), in_w=take(np.float64, S))
    if points:
        d.update(pt_of=take(np.int32, C), soma_src=take(np.int32, N), pt_user_nrn=take(np.int32, n_src),
                 pt_user_comp=take(np.int32, n_src))
    assert pos == len(b)
    return d, scomp


def _check(net, d, scomp, points):
    off = net.comp_offset
    src, dst = net.syn_src.astype(np.int64), net.syn_dst.astype(np.int64)
    S = len(src)
    dsteps = np.floor(net.syn_delay_ms / DT + 0.5).astype(np.int64)
    # sites: the distinct target compartments
    ic_dst = d["user2int"][off[dst] + net.syn_comp]
    assert sorted(d["site_internal"].tolist()) == sorted(set(ic_dst.tolist()))
    site_of = {c: k for k, c in enumerate(d["site_internal"].tolist())}
    site = np.array([site_of[c] for c in ic_dst.tolist()], np.int64)
    # sources
    if points:
        ic_src = d["user2int"][off[src] + scomp]
        pts = np.unique(ic_src)
        assert d["n_src"] == len(pts)
        sid = np.searchsorted(pts, ic_src)
    else:
        assert d["n_src"] == net.n_neurons
        sid = d["internal_of"][src].astype(np.int64)
    # outgoing synapses of each source: by delay, then synapse id
    for q in range(d["n_src"]):
        mine = np.nonzero(sid == q)[0]
        mine = mine[np.lexsort((mine, dsteps[mine]))]
        a, b = d["out_off"][q], d["out_off"][q + 1]
        np.testing.assert_array_equal(d["out_site"][a:b], site[mine])
        np.testing.assert_array_equal(d["out_dsteps"][a:b], dsteps[mine])
        np.testing.assert_array_equal(d["out_w"][a:b], net.syn_w[mine])
    # incoming synapses of each site: ascending synapse id
    for k in range(d["nsite"]):
        mine = np.nonzero(site == k)[0]
        a, b = d["in_off"][k], d["in_off"][k + 1]
        np.testing.assert_array_equal(d["in_src"][a:b], sid[mine])
        np.testing.assert_array_equal(d["in_dsteps"][a:b], dsteps[mine])
        np.testing.assert_array_equal(d["in_w"][a:b], net.syn_w[mine])
    if points:
        soma_internal = d["user2int"][off[:-1]]
        exp_pt_of = -np.ones(net.n_comp, np.int64)
        exp_soma = -np.ones(net.n_neurons, np.int64)
        for s in range(S):
            q = sid[s]
            assert d["pt_user_nrn"][q] == src[s] and d["pt_user_comp"][q] == scomp[s]
            if scomp[s] == 0:
                assert ic_src[s] == soma_internal[src[s]]
                exp_soma[d["internal_of"][src[s]]] = q
            else:
                exp_pt_of[ic_src[s]] = q
        np.testing.assert_array_equal(d["pt_of"], exp_pt_of)
        np.testing.assert_array_equal(d["soma_src"], exp_soma)


@pytest.mark.parametrize("case", ["soma", "points", "points_all_somata"])
def test_source_tables(checker, tmp_path, case):
    net = netgen.make_network(60, size_dist=("loguniform", 3, 300), p_branch=0.2, syn_per_neuron=9, seed=61,
                              delay_ms=("uniform", 1.0, 3.0), src_points=True)
    if case == "points_all_somata":
        net.syn_src_comp = np.zeros(net.n_syn, np.int32)
    points = case != "soma"
    d, scomp = _dump(checker, tmp_path, net, points)
    _check(net, d, scomp, points)
    if case == "points":
        assert np.count_nonzero(d["pt_of"] >= 0) > 100 and np.count_nonzero(d["soma_src"] >= 0) > 0
