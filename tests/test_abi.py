"""The CUDA library builds for sm_103a, loads without a GPU and exports every
function include/*.h declares (no compute calls here)."""
import ctypes
import glob
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(mm_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2005_06332_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("mm_create_network", "mm_step", "mm_read_voltages", "mm_read_spikes", "mm_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.mm_status_string.restype = ctypes.c_char_p
    assert lib.mm_status_string(0) == b"MM_OK"
    assert lib.mm_status_string(6) == b"MM_EOVERFLOW"


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes mirrors of the boundary's structs have the C sizes and
    field offsets (compiled against include/mm.h with the host compiler)."""
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    import subprocess

    from paper_2005_06332_gb300 import mm
    checks = {"mm_options": (mm.Options, ["precision", "dt_ms", "cost", "allocator", "n_ext_sources"]),
              "mm_synapses": (mm.Synapses, ["n", "tau_ms", "src_comp"]),
              "mm_schedule_report": (mm.ScheduleReport, ["r2_holdout", "r2_holdout_size_only"]),
              "mm_launch_info": (mm.LaunchInfo, ["comps", "sites"])}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "mm.h"', "int main(void) {"]
    for t, (_, fields) in checks.items():
        lines.append(f'printf("{t} %zu\\n", sizeof({t}));')
        for f in fields:
            lines.append(f'printf("{t}.{f} %zu\\n", offsetof({t}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "sizes.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "sizes"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for t, (cls, fields) in checks.items():
        assert int(got[t]) == ctypes.sizeof(cls), t
        for f in fields:
            assert int(got[f"{t}.{f}"]) == getattr(cls, f).offset, f"{t}.{f}"
