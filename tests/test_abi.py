"""The C-ABI library loads and exports every symbol include/eic.h declares (no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2506_19349_gb300 import build

    build.build()
    from paper_2506_19349_gb300 import binding

    return binding.load_library()


def _declared():
    text = open(os.path.join(ROOT, "include", "eic.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(eic_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_expected_entry_points():
    from paper_2506_19349_gb300 import binding

    assert set(_declared()) == set(binding.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_host_only_calls(lib):
    from paper_2506_19349_gb300 import binding

    p = binding.default_params()
    assert (p.alpha, p.beta, p.st_num, p.gap_shift, p.flags) == (3, 0.9, 1024, 0, 0)
    assert lib.eic_params_default(None) == binding.EINVAL
    for code in range(8):
        assert lib.eic_strerror(code)
    assert lib.eic_version() >= 100
    out = ctypes.c_void_p()
    # argument checks happen before any device call
    assert lib.eic_graph_create(None, None, None, 0, 10, 0, None, None) == binding.EINVAL
    assert lib.eic_graph_create(None, None, None, 0, 0, 0, None, ctypes.byref(out)) == binding.EINVAL
    assert lib.eic_graph_create(None, None, None, 5, 10, 0, None, ctypes.byref(out)) == binding.EINVAL
    assert lib.eic_graph_info(None, None, None, None, None, None, None) == binding.EINVAL
    assert lib.eic_graph_destroy(None) == binding.OK
    assert lib.eic_sssp(None, 0, None, None, None, None, None) == binding.EINVAL
    assert lib.eic_sssp_batch(None, None, 0, None, None, None, None) == binding.OK
