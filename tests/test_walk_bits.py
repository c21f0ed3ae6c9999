"""The cell walk's integer-pipe geometry (face coordinates built from their
bits, cell coordinates read from the bits of the position, order keys for
the minimum over axes) and its FP32-pair arithmetic, checked on the CPU
against the plain FP64 expressions they stand for (Sect. 4.3 walk: the same
faces, cells and axis choices as floor / ceil / < on doubles)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2001_11252_gb300", "csrc")


def test_bits_helpers_equal_fp64_definitions(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path / "bits_check")
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-I", CSRC, os.path.join(HERE, "native", "bits_check.cpp"),
                           "-o", exe])
    r = subprocess.run([exe], stdout=subprocess.PIPE, stderr=subprocess.STDOUT, timeout=300)
    out = r.stdout.decode()
    assert r.returncode == 0 and out.startswith("ok"), out
