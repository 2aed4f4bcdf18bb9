"""The FP32 cell-side TRiSK reformulation against the explicit form (host).

Each cell forms, in O(n), its share of the Coriolis sum of every one of its
edges from the prefix sums of its kite fractions (trisk32_body); the edge
pass adds the two cells' shares and the gradient of B = K + g xi
(phi_from_shares).  Compiled for the host with g++, both run on meshes built
by the library's host mesh builder, with random u, xi*, q and K, and are held
against the edgesOnEdge / weightsOnEdge sum of Eq. trisk_vorticity plus the
kinetic-energy and pressure gradients, in double.  Float rounding moves Phi by
at most 1.4e-6 of the size of its terms (2e-7 on hexagons); a wrong prefix
term, vertex or factor one half, planted on the host, moves it by 0.25 to 17
of them."""
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


@pytest.fixture(scope="module")
def check(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.isdir(CUDA_INC):
        pytest.skip("g++ or the CUDA headers are missing")
    so = str(tmp_path_factory.mktemp("trisk") / "trisk_share_check.so")
    subprocess.run([gxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-x", "c++", "-I", os.path.join(ROOT, "include"),
                    "-I", CSRC, "-I", CUDA_INC, os.path.join(ROOT, "tests", "host", "trisk_share_check.cpp"),
                    os.path.join(CSRC, "mesh.cpp"), "-o", so], check=True, capture_output=True)
    lib = C.CDLL(so)
    lib.trisk_share_check.argtypes = [C.c_void_p, C.c_ulonglong, C.POINTER(C.c_double)]
    lib.trisk_share_check.restype = C.c_int

    def run(s, seed):
        d, keep = fb._mesh_desc(s.mesh, s.fVertex, s.level, s.M, 0, 0)
        out = (C.c_double * 3)()
        assert lib.trisk_share_check(C.addressof(d), seed, out) == 0
        return out[0], int(out[1]), int(out[2])
    return run


CASES = {
    "bump": lambda: scenario.gaussian_bump_case(two_level=True),             # periodic hexagons
    "shelf": lambda: scenario.shelf_case(nx=64, ny=48, dc=2e3, M=4, width=10e3),   # walls: no-flow edges
    "jittered": lambda: scenario.jittered_voronoi_case(),                    # 3-11 edges, 12-slot rows
}


@pytest.mark.parametrize("case,width", [("bump", 8), ("shelf", 8), ("jittered", 12)])
def test_cell_side_trisk_equals_explicit_sum(check, case, width):
    s = CASES[case]()
    for seed in (1, 2, 3, 4, 5):
        worst, checked, rows = check(s, seed)
        assert rows == width and checked > 1000
        assert worst <= 1e-5, (case, seed, worst)
