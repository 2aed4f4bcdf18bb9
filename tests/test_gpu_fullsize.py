"""The workloads at full size, in the launch configuration bench.py times
(captured coarse step, forcing on): the 2.03M-cell basin with 3 LTS levels,
M = 8, and the 512x512 shelf channel (2 levels, M = 4) over 100 coarse steps.

One coarse step of the oracle on the full mesh (about 100 s of CPU) is the
reference for every output of both GPU paths; then properties over more
steps: mass conserved to roundoff per step, and bitwise reproducible runs.
"""
import numpy as np
import pytest

import oracle
import paper_2405_10505_gb300 as fb
from synth import basin, scenario
from tests.gpu_util import make_state, rel_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case():
    s = basin.basin_case()
    mesh = fb.mesh_create(s.mesh, s.fVertex, level=s.level, M=s.M)
    ho, uo = oracle.fblts(oracle.Mesh.from_scenario(s), oracle.scenario_params(s), s.level, s.M, s.h0, s.u0,
                          s.dt, 1)
    return s, mesh, ho, uo


def test_full_basin_one_step_matches_oracle(case):
    s, mesh, ho, uo = case
    for precision, tol_h, tol_u in ((fb.FP64, 1e-10, 1e-10), (fb.FP32_TENDENCY, 1e-6, 1e-5)):
        st = make_state(s, precision=precision, mesh=mesh)
        fb.lts_advance(st, 1)
        h, u = fb.state_read(st)
        dh, du = rel_errors(h, u, ho, uo)
        assert dh <= tol_h and du <= tol_u, (precision, dh, du)
        fb.state_destroy(st)


def test_full_basin_mass_and_reproducibility(case):
    s, mesh, _, _ = case
    runs = []
    for _ in range(2):
        st = make_state(s, precision=fb.FP32_TENDENCY, mesh=mesh)
        m0, _ = fb.diagnostics(st)
        prev = m0
        for _ in range(3):
            fb.lts_advance(st, 1)
            cur, _ = fb.diagnostics(st)
            assert abs(cur - prev) <= 1e-13 * m0
            prev = cur
        runs.append(fb.state_read(st))
        fb.state_destroy(st)
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])


@pytest.fixture(scope="module")
def shelf_case():
    s = scenario.shelf_case()            # the 512x512 shelf channel at its stated size (262k cells)
    mesh = fb.mesh_create(s.mesh, s.fVertex, level=s.level, M=s.M)
    ho, uo = oracle.fblts(oracle.Mesh.from_scenario(s), oracle.scenario_params(s), s.level, s.M, s.h0, s.u0,
                          s.dt, 100)
    return s, mesh, ho, uo


@pytest.mark.parametrize("precision,tol_h,tol_u", [(fb.FP64, 1e-10, 1e-10), (fb.FP32_TENDENCY, 1e-6, 1e-5)])
def test_full_shelf_100_steps_matches_oracle(shelf_case, precision, tol_h, tol_u):
    """The 512x512 shelf channel (2 levels, M = 4, wind stress and drag) for
    100 coarse steps, every output against one oracle run (about 70 s of CPU)."""
    s, mesh, ho, uo = shelf_case
    st = make_state(s, precision=precision, mesh=mesh)
    fb.lts_advance(st, 100)
    h, u = fb.state_read(st)
    fb.state_destroy(st)
    dh, du = rel_errors(h, u, ho, uo)
    assert dh <= tol_h and du <= tol_u, (dh, du)
