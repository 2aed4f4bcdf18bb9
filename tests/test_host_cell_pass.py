"""The FP32 cell pass against its definitions (host).

cell32_body, compiled for the host with g++, runs in its correction-sum mode
(the exact flux products l_e F_e summed in double-float and widened) on
meshes built by the library's host mesh builder, with random u and xi: K_i
against (1/A_i) sum (d_e l_e / 4) u_e^2, Psi_i against the sum of Eq.
trisk_thickness over the same float fluxes taken in double, and the mass
change sum_i A_i Psi_i, which cancels edge by edge (Theorem 1)."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

import paper_2405_10505_gb300 as fb
from synth import scenario

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2405_10505_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"

CASES = {
    "bump": lambda: scenario.gaussian_bump_case(two_level=True),
    "shelf": lambda: scenario.shelf_case(nx=64, ny=48, dc=2e3, M=4, width=10e3),
    "jittered": lambda: scenario.jittered_voronoi_case(),
}


@pytest.fixture(scope="module")
def check(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.isdir(CUDA_INC):
        pytest.skip("g++ or the CUDA headers are missing")
    so = str(tmp_path_factory.mktemp("cell") / "cell_pass_check.so")
    subprocess.run([gxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-x", "c++", "-I", os.path.join(ROOT, "include"),
                    "-I", CSRC, "-I", CUDA_INC, os.path.join(ROOT, "tests", "host", "cell_pass_check.cpp"),
                    os.path.join(CSRC, "mesh.cpp"), "-o", so], check=True, capture_output=True)
    lib = C.CDLL(so)
    lib.cell_pass_check.argtypes = [C.c_void_p, C.c_ulonglong, C.POINTER(C.c_double)]
    lib.cell_pass_check.restype = C.c_int

    def run(s, seed):
        d, keep = fb._mesh_desc(s.mesh, s.fVertex, s.level, s.M, 0, 0)
        out = (C.c_double * 4)()
        assert lib.cell_pass_check(C.addressof(d), seed, out) == 0
        return tuple(out)
    return run


@pytest.mark.parametrize("case", sorted(CASES))
def test_cell_pass_matches_definitions(check, case):
    s = CASES[case]()
    for seed in (1, 2, 3):
        k_err, psi_err, mass, cells = check(s, seed)
        assert cells > 1000
        assert k_err <= 1e-6, (case, seed, k_err)        # float sum of six to eleven products
        assert psi_err <= 2.0 ** -44, (case, seed, psi_err)   # the double-float sum, widened
        assert mass <= 1e-13, (case, seed, mass)
