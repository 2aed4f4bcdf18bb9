"""The launch list of one coarse step (fblts_plan_step, host only) against the
structure of the scheme, on CPU.

Counted independently from Sec. 2.2 and Eq. fbrk32: an FB-RK(3,2) step is
three stages of four passes (cell, vertex, TRiSK / edge prep, edge), or of two
(cell, edge) under the operator splitting of Sec. 3.2; an FB-LTS step of the
pair (l, l+1) is the coarse advancement, one save, and per subcycle one
prediction plus the fine step (recursing for more levels), then one
correction; a coarse step adds the forcing launch and the step end; the
splitting adds a four-pass slow block per coarse step (and per fine step in
its Sec. 4.2 variant); classical RK4 is four stages of four passes.  The
cell-updates are the metric's definition, sum_l N_l prod_{m<l} M_m."""
import numpy as np
import pytest

import paper_2405_10505_gb300 as fb
from synth import basin, scenario


def expected_ops(L, M, split):
    stage = 2 if split else 4

    def step(l):
        if l == L - 1:
            return 3 * stage
        return 3 * stage + 1 + M[l] * (1 + (4 if split == 2 else 0) + step(l + 1)) + 1

    return 1 + (4 if split else 0) + step(0) + 1


def expected_cell_updates(level, M):
    mult = np.cumprod([1] + list(M))
    return int(sum(int(np.sum(level == l)) * int(mult[l]) for l in range(len(M) + 1)))


CASES = {
    "bump_m2": lambda: scenario.gaussian_bump_case(two_level=True),
    "bump_m5": lambda: scenario.gaussian_bump_case(two_level=True, M=5),
    "nested_3level": lambda: scenario.nested_disk_case(nx=64, ny=64, radii=(190e3, 50e3)),
    "basin_1_64": lambda: basin.basin_case(Ly=150e3),
}


@pytest.mark.parametrize("name", list(CASES))
def test_launch_count_and_cell_updates(name):
    s = CASES[name]()
    L = len(s.M) + 1
    bytes_ = {}
    for split in (0, 1, 2):
        for prec in (fb.FP64, fb.FP32_TENDENCY):
            n, b, cu = fb.plan_step(s.mesh, s.fVertex, s.level, s.M, fb.make_params(s.dt, precision=prec, split=split))
            assert n == expected_ops(L, s.M, split), (split, prec)
            assert cu == expected_cell_updates(s.level, s.M)
            bytes_[split, prec] = b
    for split in (0, 1, 2):
        assert 0 < bytes_[split, fb.FP32_TENDENCY] < bytes_[split, fb.FP64]
    for prec in (fb.FP64, fb.FP32_TENDENCY):
        # the splitting drops the vertex and TRiSK passes of every stage; its
        # variant adds a slow block per fine step
        assert bytes_[1, prec] < bytes_[2, prec] < bytes_[0, prec]


def test_rk4_plan_and_its_checks():
    s = scenario.gaussian_bump_case(two_level=True)
    one = np.zeros(s.mesh.nCells, np.int32)
    n, b, cu = fb.plan_step(s.mesh, s.fVertex, one, [], fb.make_params(s.dt, scheme=fb.SCHEME_RK4))
    assert n == 1 + 4 * 4 + 1 and cu == s.mesh.nCells and b > 0
    for level, M, kw in ((s.level, s.M, {}), (one, [], dict(split=1)), (one, [], dict(scheme=9))):
        with pytest.raises(fb.FbltsError) as e:
            fb.plan_step(s.mesh, s.fVertex, level, M, fb.make_params(s.dt, **{"scheme": fb.SCHEME_RK4, **kw}))
        assert e.value.status == fb.E_ARG


def test_degenerate_meshes():
    """One level of a tiny periodic mesh (one FB-RK(3,2) step: 14 launches); an
    empty mesh and a level array that skips a level are rejected."""
    s = scenario.gaussian_bump_case(nx=4, ny=4, two_level=False)
    n, b, cu = fb.plan_step(s.mesh, s.fVertex, s.level, [], fb.make_params(s.dt))
    assert n == 1 + 12 + 1 and cu == 16 and b > 0
    d = fb.MeshDesc()
    import ctypes as C
    n_ = C.c_int64()
    assert fb.lib().fblts_plan_step(C.byref(d), C.byref(fb.make_params(1.0)), C.byref(n_), None, None) == fb.E_ARG
    two = scenario.gaussian_bump_case(two_level=True)
    skip = two.level * 2          # levels 0 and 2, none on level 1
    with pytest.raises(fb.FbltsError):
        fb.plan_step(two.mesh, two.fVertex, skip, [2, 2], fb.make_params(two.dt))
