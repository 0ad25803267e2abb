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


def test_struct_layouts_match_the_header(tmp_path):
    # The binding's ctypes mirrors of cphifi_params / cphifi_stats must have the
    # header's size and field offsets (a C program compiled from the header
    # prints them).
    import ctypes

    import paper_2603_25691_gb300 as pkg
    fields = {"cphifi_params": pkg.Params, "cphifi_stats": pkg.Stats,
              "cphifi_tuning": pkg.Tuning, "cphifi_batch_item": pkg.BatchItem,
              "cphifi_batch_info": pkg.BatchInfo}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cphifi.h"',
             "int main(void) {"]
    for cname, py in fields.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            # (a C member named like a Python keyword has a trailing _ in ctypes)
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f.rstrip("_")}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    got = {}
    for line in out.splitlines():
        c, f, v = line.split()
        got[(c, f)] = int(v)
    for cname, py in fields.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_constants_match_the_header():
    # Every enum value and flag the binding mirrors has the header's value, and
    # every operator arithmetic of the header has a name in the binding.
    import paper_2603_25691_gb300 as pkg
    text = open(HEADER).read()
    values = {m.group(1): int(m.group(2))
              for m in re.finditer(r"\bCPHIFI_([A-Z0-9_]+)\s*=\s*(\d+)", text)}
    flag = r"#define\s+CPHIFI_([A-Z0-9_]+)\s+(0x[0-9a-fA-F]+)u?"
    values.update({m.group(1): int(m.group(2), 16) for m in re.finditer(flag, text)})
    mirrored = [k for k in values if hasattr(pkg, k)]
    assert len(mirrored) >= 15, mirrored
    for k in mirrored:
        assert getattr(pkg, k) == values[k], k
    enum = re.search(r"typedef enum cphifi_precision \{(.*?)\}", text, re.S).group(1)
    precisions = {int(v) for v in re.findall(r"=\s*(\d+)", enum)}
    assert precisions == set(pkg.PRECISIONS.values())
