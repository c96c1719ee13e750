"""Host logic: the FP32c gate table (csrc/mm_gate_table.h), built with g++
and evaluated exactly as the kernels evaluate it, against the Hodgkin-Huxley
functions written out here in FP64 and against the oracle's gate step."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2005_06332_gb300", "csrc")
VQ = 8388608  # fixed-point units per mV


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("gtab") / "gate_table_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I" + CSRC,
                    os.path.join(ROOT, "tests", "gate_table_check.cpp"), "-o", out], check=True)
    return out


def _run(checker, dt, vq, q):
    lines = "\n".join(f"{v} {a} {b} {c}" for v, (a, b, c) in zip(vq, q))
    r = subprocess.run([checker, repr(dt)], input=lines, capture_output=True, text=True, check=True)
    rows = np.array([l.split() for l in r.stdout.strip().splitlines()], dtype=np.float64)
    return rows[:, :6], rows[:, 6:].astype(np.uint64)


def _hh(V, dt):
    """X = a / (a + b) and E = 1 - exp(-dt (a + b)) of m, h, n, from the
    rates in their textbook form (1/ms, V in mV; 1 - e^-y as -expm1(-y), so
    that the removable singularities of alpha_m and alpha_n lose no digits)."""
    with np.errstate(invalid="ignore", divide="ignore"):
        am = 0.1 * (V + 40.0) / -np.expm1(-(V + 40.0) / 10.0)
        an = 0.01 * (V + 55.0) / -np.expm1(-(V + 55.0) / 10.0)
    am = np.where(np.abs(V + 40.0) < 1e-9, 1.0, am)
    an = np.where(np.abs(V + 55.0) < 1e-9, 0.1, an)
    bm = 4.0 * np.exp(-(V + 65.0) / 18.0)
    ah = 0.07 * np.exp(-(V + 65.0) / 20.0)
    bh = 1.0 / (1.0 + np.exp(-(V + 35.0) / 10.0))
    bn = 0.125 * np.exp(-(V + 65.0) / 80.0)
    out = []
    for a, b in ((am, bm), (ah, bh), (an, bn)):
        out += [a / (a + b), -np.expm1(-dt * (a + b))]
    return np.stack(out, axis=1)


def _voltages(rng):
    # every 0.5 mV interval of [-120, 120] mV at its centre, both ends and
    # random points, plus the removable singularities of alpha_m and alpha_n
    centres = (np.arange(481) * (VQ // 2) - 120 * VQ).astype(np.int64)
    pts = [centres, centres - VQ // 4, centres + VQ // 4 - 1]
    pts.append(rng.integers(-120 * VQ, 120 * VQ, 4000))
    pts.append(np.array([-40 * VQ, -55 * VQ, -40 * VQ + 1, -55 * VQ - 1, -65 * VQ, 120 * VQ, -120 * VQ]))
    v = np.concatenate(pts)
    return v[(v >= -120 * VQ) & (v <= 120 * VQ)]


@pytest.mark.parametrize("dt", [0.025, 0.01])
def test_table_functions_to_2e10_relative(checker, dt):
    rng = np.random.default_rng(11)
    vq = _voltages(rng)
    q = np.full((len(vq), 3), 1 << 31, np.int64)
    F, _ = _run(checker, dt, vq, q)
    want = _hh(vq / VQ, dt)
    rel = np.abs(F - want) / np.abs(want)
    assert rel.max() < 2e-10, (rel.max(axis=0), vq[np.argmax(rel.max(axis=1))])
    assert np.abs(np.mean((F - want) / want, axis=0)).max() < 1e-12  # no bias


def test_gate_step_equals_the_oracle_to_the_fixed_point_unit(checker):
    """Each stepped gate is the oracle's exponential-Euler step rounded to
    2^-32, within one unit (the oracle rounds nothing, the table's error is
    far below the unit)."""
    dt = 0.025
    rng = np.random.default_rng(12)
    vq = np.concatenate([rng.integers(-100 * VQ, 60 * VQ, 1500), rng.integers(-120 * VQ, 120 * VQ, 300)])
    q = rng.integers(0, 1 << 32, (len(vq), 3), dtype=np.uint64).astype(np.int64)
    _, Q = _run(checker, dt, vq, q)
    scale = 2.0 ** 32
    for k in range(len(vq)):
        m, h, n = oracle.gate_step(vq[k] / VQ, dt, *(q[k] / scale))
        want = np.array([m, h, n]) * scale
        assert np.all(np.abs(Q[k].astype(np.float64) - want) <= 1.0), (k, Q[k], want)


def test_planted_coefficient_error_is_caught(checker, tmp_path):
    """A table whose linear coefficient loses its low word (one plausible
    slip in the builder) fails the 2e-10 bar: the check has the resolution."""
    src = open(os.path.join(ROOT, "tests", "gate_table_check.cpp")).read()
    bad = tmp_path / "bad.cpp"
    bad.write_text(src.replace("mmf::build_gate_table(dt, tab.data());",
                               "mmf::build_gate_table(dt, tab.data());\n"
                               "    for (size_t k = 0; k < tab.size(); ++k) if ((k / mmf::kTabIntervals) % 2 == 0) tab[k].w = 0.0f;"))
    exe = str(tmp_path / "bad")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I" + CSRC, str(bad), "-o", exe], check=True)
    vq = _voltages(np.random.default_rng(13))
    F, _ = _run(exe, 0.025, vq, np.full((len(vq), 3), 1 << 31, np.int64))
    want = _hh(vq / VQ, 0.025)
    assert (np.abs(F - want) / np.abs(want)).max() > 2e-10


def test_voltages_beyond_the_range_read_the_end_intervals(checker):
    """V outside +-120 mV (which the step reports as MM_ENUMERIC) still reads
    inside the table: the first or last interval at its end."""
    lo, hi = -120 * VQ - VQ // 4, 120 * VQ + VQ // 4  # the table's outer edges
    vq = np.array([lo - 5 * VQ, lo, -2**31 + 1, hi + 5 * VQ, hi - 1, 2**31 - 1], np.int64)
    F, _ = _run(checker, 0.025, vq, np.full((len(vq), 3), 1 << 31, np.int64))
    assert np.all(np.isfinite(F))
    np.testing.assert_array_equal(F[0], F[1])
    np.testing.assert_array_equal(F[0], F[2])
    np.testing.assert_allclose(F[3], F[4], rtol=1e-7)  # one fixed-point unit apart
    np.testing.assert_array_equal(F[3], F[5])
