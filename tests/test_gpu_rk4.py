"""Classical RK4 on the GPU (the comparison integrator of Sec. 4.2, Tab. 2)
against the oracle's RK4, through the C ABI.

Every cell and edge advances with one step size (one-level meshes; on the
multi-level scenarios the finest level's step).  Bar: the FP64 path within
1e-10 of the oracle in h and u, the FP32-tendency path within 1e-6 (h) and
1e-5 (u, of max |u|), mass conserved to 1e-13 per step, and the scheme
distinguishable from FB-RK(3,2) on the same case.
"""
import numpy as np
import pytest

import oracle
import paper_2405_10505_gb300 as fb
from synth import scenario
from tests.gpu_util import make_state, rel_errors

pytestmark = pytest.mark.gpu

CASES = {
    "bump": (lambda: scenario.gaussian_bump_case(two_level=False), 100),
    "shelf_forced": (lambda: scenario.shelf_case(nx=64, ny=48, dc=2e3, M=4, width=10e3), 100),
    "shelf_vortex": (lambda: scenario.shelf_case(nx=64, ny=48, dc=2e3, M=4, width=10e3, vortex=True), 60),
    "jittered_voronoi": (lambda: scenario.jittered_voronoi_case(), 60),
}


def _one_level(s):
    """The scenario on one level at its finest step."""
    dt = s.dt / int(np.prod(s.M)) if len(s.M) else s.dt
    return np.zeros(s.mesh.nCells, np.int32), dt


def _state(s, precision, mesh=None, scheme=fb.SCHEME_RK4):
    level, dt = _one_level(s)
    return make_state(s, M=[], level=level, precision=precision, mesh=mesh, scheme=scheme, dt=dt)


@pytest.mark.parametrize("name", list(CASES))
def test_rk4_parity_with_oracle(name):
    make, nsteps = CASES[name]
    s = make()
    _, dt = _one_level(s)
    ho, uo = oracle.rk4(oracle.Mesh.from_scenario(s), oracle.scenario_params(s), s.h0, s.u0, dt, nsteps)
    level, _ = _one_level(s)
    mesh = fb.mesh_create(s.mesh, s.fVertex, level=level, M=[])
    for precision, tol_h, tol_u in ((fb.FP64, 1e-10, 1e-10), (fb.FP32_TENDENCY, 1e-6, 1e-5)):
        st = _state(s, precision, mesh=mesh)
        fb.lts_advance(st, nsteps)
        h, u = fb.state_read(st)
        fb.state_destroy(st)
        dh, du = rel_errors(h, u, ho, uo)
        assert dh <= tol_h and du <= tol_u, (precision, dh, du)


def test_rk4_conserves_mass_and_differs_from_fbrk32():
    s = scenario.shelf_case(nx=64, ny=48, dc=2e3, M=4, width=10e3, vortex=True)
    level, _ = _one_level(s)
    mesh = fb.mesh_create(s.mesh, s.fVertex, level=level, M=[])
    for precision in (fb.FP64, fb.FP32_TENDENCY):
        st = _state(s, precision, mesh=mesh)
        m0, _ = fb.diagnostics(st)
        prev = m0
        for _ in range(10):
            fb.lts_advance(st, 1)
            cur, _ = fb.diagnostics(st)
            assert abs(cur - prev) <= 1e-13 * m0
            prev = cur
        h, u = fb.state_read(st)
        fb.state_destroy(st)
        st = _state(s, precision, mesh=mesh, scheme=fb.SCHEME_FBLTS)
        fb.lts_advance(st, 10)
        hf, uf = fb.state_read(st)
        fb.state_destroy(st)
        # far above roundoff (the same scheme would agree bitwise: no atomics)
        assert np.max(np.abs(u - uf)) > 1e-6 * np.max(np.abs(u))


def test_rk4_needs_one_level_and_no_splitting():
    s = scenario.gaussian_bump_case(two_level=True)
    with pytest.raises(fb.FbltsError) as e:
        make_state(s, scheme=fb.SCHEME_RK4)
    assert e.value.status == fb.E_ARG
    s1 = scenario.gaussian_bump_case(two_level=False)
    with pytest.raises(fb.FbltsError) as e:
        make_state(s1, scheme=fb.SCHEME_RK4, split=True)
    assert e.value.status == fb.E_ARG
    with pytest.raises(fb.FbltsError) as e:
        make_state(s1, scheme=7)
    assert e.value.status == fb.E_ARG
