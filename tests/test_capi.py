"""The C ABI library builds, loads without a GPU, and exports every function that
include/ram.h declares.  No compute call is made here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ram_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2305_05362_gb300 import build, ram
    build.build()
    return ram.load()


def test_header_functions_exported(lib):
    names = _declared("ram.h")
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def test_binding_lists_every_export():
    from paper_2305_05362_gb300 import ram
    assert sorted(ram.EXPORTS) == sorted(n for n in _declared("ram.h"))


def test_status_strings_and_version(lib):
    from paper_2305_05362_gb300 import ram
    for code in ram.STATUS:
        s = lib.ram_status_string(code)
        assert isinstance(s, bytes) and s
    assert ram.version() >= 100


def test_null_arguments_rejected_without_gpu(lib):
    """Host-side argument checks run before any CUDA call."""
    assert lib.ram_plan_mesh(None, 0, None) == 1
    assert lib.ram_shift(None, 0, None, None, None, None) == 1
    assert lib.ram_step(None, 0, None, None, None, None, ctypes.c_double(0.0), None, 0,
                        None, None) == 1
    assert lib.ram_plan_destroy(None) == 0
    assert lib.ram_plan_set_wait_limit(None, 0) == 1


def test_library_is_not_the_oracle():
    """The product library and the oracle share no source files."""
    import glob
    csrc = glob.glob(os.path.join(ROOT, "paper_2305_05362_gb300", "csrc", "*"))
    for path in csrc:
        text = open(path).read()
        assert "oracle" not in text.lower(), path
    pkg = glob.glob(os.path.join(ROOT, "paper_2305_05362_gb300", "*.py"))
    for path in pkg:
        src = open(path).read()
        assert not re.search(r"^\s*(import|from)\s+oracle\b", src, re.M), path
