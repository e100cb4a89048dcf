"""The double-word arithmetic of the MPCG_FP64_DW path (csrc/dw.cuh), run as
host code on the CPU against extended precision: splitting a double into a
float pair keeps 47 bits, assembling a pair gives the double within 2^-52,
and sums and products stay within 8 * 2^-48 of the exact results relative
to |x| + |y| (resp. |x y|), multiply-adds c + a b within 16 * 2^-48 of
|c| + |a b| (the product's two rounded cross terms, the dropped lo * lo term
and the rounded low-word sum), quotients within 16 * 2^-48, including sums
that cancel (the normwise bounds the solver's sums of products need)."""
import json
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = "/usr/local/cuda/include"


@pytest.fixture(scope="module")
def report(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None or not os.path.isdir(CUDA_INC):
        pytest.skip("g++ or the CUDA headers are missing")
    exe = str(tmp_path_factory.mktemp("dw") / "dw_check")
    src = os.path.join(ROOT, "tests", "native", "dw_check.cpp")
    inc = os.path.join(ROOT, "paper_2402_12833_gb300", "csrc")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", inc, "-I", CUDA_INC, src, "-o", exe],
                   check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return json.loads(out)


def test_split_and_assemble(report):
    assert report["split"] <= 1.0, report          # |hi + lo - d| <= 2^-47 |d|
    assert report["lo_norm"] <= 1.0, report        # |lo| <= 2^-23 |hi|
    assert report["assemble"] <= 1.0, report       # pair -> double within 2^-52
    assert report["exact_fails"] == 0 and report["specials"] == 1, report


def test_operations_within_their_bounds(report):
    for op in ("add", "mul", "fma", "div"):
        assert report[op] <= 1.0, (op, report)
    # and not trivially: the errors are visible at the 2^-48 level
    assert max(report["add"], report["mul"], report["fma"]) > 1e-3, report
