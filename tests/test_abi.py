"""CPU-side checks of the C ABI: the library builds for sm_103a, loads without a
GPU, and exports every entry point that include/*.h declares; the binding's
signature table covers the same set."""
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[\w\s\*]*?\b(als_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2107_00820_gb300 import build as b
    if not b.up_to_date():
        if not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("nvcc not available to build the library")
        b.build()
    from paper_2107_00820_gb300 import alstokes
    return alstokes.load()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["als_create", "als_destroy", "als_apply_agamma", "als_vcycle", "als_solve", "als_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in _declared():
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    from paper_2107_00820_gb300.alstokes import SIGNATURES
    assert set(SIGNATURES) == _declared()


def test_library_is_built_for_sm_103a(lib):
    from paper_2107_00820_gb300 import build as b
    assert "arch=compute_103a,code=sm_103a" in " ".join(b.ARCH)


def test_no_cpu_fallback_in_binding():
    """The binding refuses non-CUDA tensors for the device entry points."""
    import numpy as np
    from paper_2107_00820_gb300 import alstokes
    with pytest.raises(TypeError):
        alstokes._cuda_tensor(np.zeros(3))
