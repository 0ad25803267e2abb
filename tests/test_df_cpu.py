"""CPU check of the double-float primitives (csrc/df.cuh) used by the
FP64-accurate steps of the mixed solve: a host build of the same header,
compared with extended-precision references (tests/native/df_check.cpp)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_double_float_primitives(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = tmp_path / "df_check"
    subprocess.run([cxx, "-O2", "-ffp-contract=off", "-std=c++17", "-o", str(exe),
                    os.path.join(HERE, "native", "df_check.cpp")], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    worst_dot, worst_prod, worst_split = map(float, out)
    # k-term compensated dot: error <= ~k 2^-48 of sum |x_i y_i| (k <= 2000)
    assert worst_dot <= 2000 * 2.0 ** -48
    # one double-float product: a few units of 2^-48
    assert worst_prod <= 8 * 2.0 ** -48
    # split of a double into hi + lo: 2^-48 relative
    assert worst_split <= 2.0 ** -48
