"""The basin recipe over a 100-coarse-step window: the 1/64-length sample of
the headline basin (same generator and seed, Ly = 150 km: about 32k cells of
3 to 11 edges, 3 LTS levels with M = 8, shoaling bathymetry, wind stress,
bottom drag and the moving Holland vortex), both GPU paths against one
oracle run of 100 coarse steps (about 150 s of CPU).

Bars: FP64 max_i |dh_i|/|h_i| <= 1e-10 and max_e |du_e| <= 1e-10 max_e |u_e|;
FP32 tendencies 1e-6 and 1e-5.
"""
import pytest

import oracle
import paper_2405_10505_gb300 as fb
from synth import basin
from tests.gpu_util import make_state, rel_errors

pytestmark = pytest.mark.gpu
NSTEPS = 100


@pytest.fixture(scope="module")
def case():
    s = basin.basin_case(Ly=150e3)
    assert s.nLevels == 3 and s.M == [8, 8]
    mesh = fb.mesh_create(s.mesh, s.fVertex, level=s.level, M=s.M)
    ho, uo = oracle.fblts(oracle.Mesh.from_scenario(s), oracle.scenario_params(s), s.level, s.M, s.h0, s.u0,
                          s.dt, NSTEPS)
    return s, mesh, ho, uo


@pytest.mark.parametrize("precision,tol_h,tol_u", [(fb.FP64, 1e-10, 1e-10), (fb.FP32_TENDENCY, 1e-6, 1e-5)])
def test_basin_sample_100_steps_matches_oracle(case, precision, tol_h, tol_u):
    s, mesh, ho, uo = case
    st = make_state(s, precision=precision, mesh=mesh)
    fb.lts_advance(st, NSTEPS)
    h, u = fb.state_read(st)
    fb.state_destroy(st)
    dh, du = rel_errors(h, u, ho, uo)
    assert dh <= tol_h and du <= tol_u, (dh, du)
