"""CPU-side checks of the boundary: the shared library builds, loads and
exports every entry point declared in include/cphifi.h (no compute calls)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cphifi.h")


def declared_entry_points():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"\b(cphifi_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2603_25691_gb300 import _build
    return _build.build()


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (cphifi_[a-z0-9_]+)", out))
    missing = [s for s in declared_entry_points() if s not in exported]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(libpath):
    import paper_2603_25691_gb300 as pkg
    assert sorted(pkg.exported_symbols()) == declared_entry_points()
    L = pkg.lib()  # loads without a GPU
    for s in declared_entry_points():
        assert hasattr(L, s)


def test_status_strings_without_gpu(libpath):
    import paper_2603_25691_gb300 as pkg
    assert pkg.status_string(0) == "ok"
    assert "budget" in pkg.status_string(pkg.E_ADMISSION)


def test_context_without_gpu_is_an_error(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2603_25691_gb300 as pkg
    with pytest.raises(pkg.CphifiError):
        pkg.Context(0)
