"""Host pin of the bit-level double-FP32 conversions of the CUDA kernels
(csrc/df_bits.cuh): the split hi = fl32(x), lo = fl32(x - hi) and the
widening (double)f, built with integer and FP32 operations only, must give
the same bits as the host's IEEE conversions on edge cases (ties, carries,
the ends of the bit path, zeros, subnormals, non-finite values) and on
millions of random values.  The header compiles as plain C++ for this."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2107_06635_gb300", "csrc")


def test_bit_level_split_and_widen_match_ieee_conversions(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "df_bits_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC,
                    os.path.join(HERE, "df_bits_check.cpp"), "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "split mismatches 0 widen mismatches 0" in r.stdout
