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
