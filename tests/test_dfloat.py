"""CPU checks of the double-float arithmetic (csrc/dfloat.cuh) that the deflating Cholesky of
the block orthonormalisation runs in.  The header is compiled for the host (plain IEEE
operations, no FMA contraction) and checked over 200 000 seeded random operands against long
double references:

* TwoSum and TwoProd are error-free: hi + lo equals a + b and a * b exactly;
* products stay normalised (|lo| <= ulp(hi) / 2);
* multiply, w - x y, 1/d and 1/sqrt(d) are accurate to about 2^-44 relative or better (the
  pair carries about 48 bits; the Newton steps of the reciprocals start from 2^-23);
* the FP64 round trip through a pair loses at most 2^-48 relative."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(__file__)
CSRC = os.path.join(HERE, os.pardir, "paper_2211_14828_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"


@pytest.fixture(scope="module")
def report(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx or not os.path.isdir(CUDA_INC):
        pytest.skip("g++ or the CUDA headers are not available")
    exe = str(tmp_path_factory.mktemp("dfloat") / "dfloat_check")
    cmd = [gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-Wno-unknown-pragmas", "-I", CSRC, "-I", CUDA_INC,
           os.path.join(HERE, "dfloat", "dfloat_check.cpp"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    vals = {}
    for k in range(0, len(out), 2):
        vals[out[k]] = float(out[k + 1])
    return vals


def test_error_free_transformations(report):
    assert report["sum_inexact"] == 0
    assert report["prod_inexact"] == 0
    assert report["denormalised"] == 0


def test_accuracy(report):
    assert report["mul"] <= 2.0 ** -44
    assert report["fms"] <= 2.0 ** -44
    assert report["rcp"] <= 2.0 ** -44
    assert report["rsqrt"] <= 2.0 ** -43
    assert report["round"] <= 2.0 ** -48
