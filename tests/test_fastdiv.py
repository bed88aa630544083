"""Host check of the division by invariant integers used by the kernels for
teller, branch and partition ids (fastdiv.h): exact against the integer
quotient for edge dividends and a seeded sweep, over many divisors
(Granlund & Montgomery 1994, Section 4)."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_fastdiv_exact():
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "fastdiv_check")
        subprocess.run([cxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_1103_3105_gb300", "csrc"),
                        os.path.join(ROOT, "tests", "fastdiv_check.cpp"), "-o", exe], check=True)
        divisors = [1, 2, 3, 5, 7, 10, 100, 128, 641, 1000, 1024, 10000, 65535, 65536, 65537, 1 << 20,
                    999_983, 10_000_000, (1 << 31) - 1, 1 << 31, (1 << 31) + 1, 0xfffffffe, 0xffffffff]
        out = subprocess.run([exe], input="\n".join(map(str, divisors)), capture_output=True, text=True,
                             check=True).stdout.split("\n")
        rows = [list(map(int, line.split())) for line in out if line.strip()]
        assert [r[0] for r in rows] == divisors
        for d, bad, checked in rows:
            assert checked > 200_000 and bad == 0, (d, bad)
