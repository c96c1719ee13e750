"""Host logic: the FP32c work-item layout (mm_layout.cpp) built with g++ and
checked by tests/layout_check.cpp on seeded networks -- path-table
invariants the kernels rely on, for shared-memory (16-bit) and giant (32-bit)
items, and a float replay of the kernels' path-by-path sweeps against
Algorithm 1 in double (no GPU), serial per lane and, for long paths, as a
whole warp sweeps them (chunks combined by scans)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2005_06332_gb300 import netgen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2005_06332_gb300", "csrc")


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
    out = str(tmp_path_factory.mktemp("layout") / "layout_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-I" + CSRC, "-I" + os.path.join(ROOT, "include"), "-I" + cuda_inc,
                    os.path.join(ROOT, "tests", "layout_check.cpp"), os.path.join(CSRC, "mm_layout.cpp"), "-o", out],
                   check=True, capture_output=True)
    return out


def _run(checker, tmp_path, net, group_comps, regular, large, warp=0):
    f = tmp_path / "net.bin"
    with open(f, "wb") as fh:
        np.array([net.n_neurons], np.int32).tofile(fh)
        np.array([net.comp_offset[-1]], np.int64).tofile(fh)
        net.comp_offset.astype(np.int64).tofile(fh)
        net.parent.astype(np.int32).tofile(fh)
    r = subprocess.run([checker, str(f), str(group_comps), str(regular), str(large), str(warp)], capture_output=True,
                       text=True)
    fields = dict(kv.split("=") for kv in r.stdout.split())
    return r.returncode, fields


@pytest.mark.parametrize("warp", [0, 96, 8])
@pytest.mark.parametrize("case", ["mono", "multi", "large_and_giant", "all_giant"])
def test_path_tables_and_sweeps(checker, tmp_path, case, warp):
    """warp: paths of at least that many compartments swept as by a whole
    warp (96: the step kernel's threshold; 8: nearly every path, with chunks
    of one compartment and empty lanes)."""
    if case == "mono":
        net = netgen.make_network(64, size_dist=("mono", 255), p_branch=0.1, mono_tree=True, syn_per_neuron=0, seed=11)
        args = (4096, 110 * 1024, 224 * 1024)
    elif case == "multi":
        net = netgen.make_network(300, size_dist=("loguniform", 20, 3000), p_branch=("uniform", 0.02, 0.3),
                                  syn_per_neuron=0, seed=12)
        args = (2048, 110 * 1024, 224 * 1024)
    elif case == "large_and_giant":
        net = netgen.make_network(40, size_dist=("loguniform", 50, 2000), p_branch=0.1, giants=2,
                                  giant_size=40_000, syn_per_neuron=0, seed=13)
        args = (2048, 30 * 1024, 80 * 1024)
    else:  # every item beyond shared memory: 32-bit tables only
        net = netgen.make_network(30, size_dist=("loguniform", 20, 600), p_branch=0.2, syn_per_neuron=0, seed=14)
        args = (512, 1, 1)
    rc, f = _run(checker, tmp_path, net, *args, warp=warp)
    assert rc == 0 and int(f["bad"]) == 0, f
    assert float(f["maxrel"]) < 1e-4, f
    if warp == 8 or (warp and case in ("multi", "large_and_giant")):  # the others have no path of 96
        assert int(f["warp_paths"]) > 0, f
    if case == "large_and_giant":
        assert int(f["giant"]) >= 2 and int(f["large"]) >= 1, f
    if case == "all_giant":
        assert int(f["small"]) == 0 and int(f["large"]) == 0 and int(f["giant"]) >= 1, f
