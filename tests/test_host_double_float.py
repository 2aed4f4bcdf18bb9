"""Host checks of the kernels' double-float helpers (kernel_bodies.cuh, compiled
for the host with g++): df_round is the IEEE double-to-float conversion bit for
bit, and df_add_prod sums eight exact float products to within 2^-44 of the
largest term (each addition into the float low part rounds; eight terms give a
few units of 2^-46).  The FP64 path's helpers, against long double: a split
of a double into a float pair within 2^-47, ten-term sums of products (its
edgesOnEdge sums) within 1.4e-13 of the largest term, product, sum, square
root and reciprocal in double-float within 2^-44, and the Newton-refined
reciprocal in double within 2^-52.  The FP32 path takes its time-level float shadows through df_round and
its in-place / correction sums of the flux products l_e F_e through
df_add_prod (Eq. trisk_thickness, Theorem 1: the two cells of an edge add the
same exact product)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2405_10505_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"


@pytest.fixture(scope="module")
def report(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.isdir(CUDA_INC):
        pytest.skip("g++ or the CUDA headers are missing")
    exe = str(tmp_path_factory.mktemp("df") / "double_float_check")
    src = os.path.join(ROOT, "tests", "host", "double_float_check.cpp")
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                    "-I", CUDA_INC, src, "-o", exe], check=True, capture_output=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return {line.split()[0]: line.split()[1:] for line in out.splitlines()}


def test_df_round_is_the_ieee_conversion(report):
    checked, bad = (int(x) for x in report["round"])
    assert checked > 5_000_000 and bad == 0


def test_df_add_prod_within_2_pow_minus_44(report):
    checked, worst = int(report["sum"][0]), float(report["sum"][1])   # worst error in units of 2^-46
    assert checked == 200_000 and worst <= 4.0, worst


def test_fp64_helpers_accuracy(report):
    split, sum10, mul, add, sqrt, rcp, newton = (float(x) for x in report["fp64"])
    assert split <= 2.0 ** -47, split
    assert sum10 <= 1.4e-13, sum10
    for name, err in (("mul", mul), ("add", add), ("sqrt", sqrt), ("rcp", rcp)):
        assert err <= 2.0 ** -44, (name, err)
    assert newton <= 2.0 ** -52, newton
