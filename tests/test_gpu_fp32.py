"""FP32-tendency path against the FP64 oracle, through the C ABI.

Bar: max_i |dh_i|/|h_i| <= 1e-6 (the method's target for this path is
1e-5) and max_e |du_e| <= 1e-5 max_e |u_e| after the stated steps; total
mass still conserved to double roundoff per step (the time level and the
edge-flux divergence are accumulated in double); bit-reproducible runs.
"""
import numpy as np
import pytest

import oracle
import paper_2405_10505_gb300 as fb
from synth import scenario
from tests.gpu_util import make_state, rel_errors

pytestmark = pytest.mark.gpu

CASES = {
    "bump_single": (lambda: scenario.gaussian_bump_case(two_level=False), 100, None),
    "bump_lts_m2": (lambda: scenario.gaussian_bump_case(two_level=True), 100, None),
    "shelf_forced_m4": (lambda: scenario.shelf_case(nx=64, ny=48, dc=2e3, M=4, width=10e3), 100, None),
    "nested_3level": (lambda: scenario.nested_disk_case(nx=64, ny=64, radii=(190e3, 50e3)), 100, None),
    "shelf_vortex_m4": (lambda: scenario.shelf_case(nx=64, ny=48, dc=2e3, M=4, width=10e3, vortex=True), 100, None),
    # irregular cells of 3..11 edges (12-slot rows, obtuse triangles), 2 levels
    "jittered_voronoi_m2": (lambda: scenario.jittered_voronoi_case(), 100, None),
}


@pytest.mark.parametrize("name", list(CASES))
def test_fp32_parity_with_fp64_oracle(name):
    make, nsteps, M = CASES[name]
    s = make()
    mesh = fb.mesh_create(s.mesh, s.fVertex, level=s.level, M=s.M if M is None else M)
    # these meshes carry the kite-fraction TRiSK weights: the edge pass reads the cell rows
    assert fb.mesh_get_info(mesh).flags & 1
    st = make_state(s, M=M, precision=fb.FP32_TENDENCY, mesh=mesh)
    fb.lts_advance(st, nsteps)
    h, u = fb.state_read(st)
    m = oracle.Mesh.from_scenario(s)
    ho, uo = oracle.fblts(m, oracle.scenario_params(s), s.level, s.M if M is None else M, s.h0, s.u0, s.dt, nsteps)
    dh, du = rel_errors(h, u, ho, uo)
    assert dh <= 1e-6 and du <= 1e-5, (dh, du)


def test_fp32_mass_drift_per_step():
    s = scenario.shelf_case(nx=64, ny=48, dc=2e3, M=4, width=10e3)
    st = make_state(s, precision=fb.FP32_TENDENCY)
    prev, _ = fb.diagnostics(st)
    m0 = prev
    for _ in range(10):
        fb.lts_advance(st, 1)
        cur, _ = fb.diagnostics(st)
        assert abs(cur - prev) <= 1e-13 * m0
        prev = cur


def test_fp32_reproducible_and_graph_equals_stream():
    s = scenario.nested_disk_case(nx=64, ny=64, radii=(190e3, 50e3))
    out = []
    for g in (True, True, False):
        st = make_state(s, precision=fb.FP32_TENDENCY, use_graph=g)
        fb.lts_advance(st, 10)
        out.append(fb.state_read(st))
    for o in out[1:]:
        assert np.array_equal(o[0], out[0][0]) and np.array_equal(o[1], out[0][1])


def test_fp32_explicit_neighbour_lists():
    """Weights that are not the kite-fraction form (perturbed by 1e-6
    relative) take the explicit-list edge pass; the oracle runs the same
    weights."""
    s = scenario.shelf_case(nx=64, ny=48, dc=2e3, M=4, width=10e3)
    rng = np.random.default_rng(7)
    s.mesh.weightsOnEdge = s.mesh.weightsOnEdge * (1.0 + 1e-6 * rng.uniform(-1, 1, s.mesh.weightsOnEdge.shape))
    mesh = fb.mesh_create(s.mesh, s.fVertex, level=s.level, M=s.M)
    assert not (fb.mesh_get_info(mesh).flags & 1)
    st = make_state(s, precision=fb.FP32_TENDENCY, mesh=mesh)
    fb.lts_advance(st, 60)
    h, u = fb.state_read(st)
    ho, uo = oracle.fblts(oracle.Mesh.from_scenario(s), oracle.scenario_params(s), s.level, s.M, s.h0, s.u0,
                          s.dt, 60)
    dh, du = rel_errors(h, u, ho, uo)
    assert dh <= 1e-6 and du <= 1e-5, (dh, du)


@pytest.mark.parametrize("split", [1, 2])
@pytest.mark.parametrize("name", ["bump_lts_m2", "shelf_vortex_m4", "nested_3level", "jittered_voronoi_m2"])
def test_fp32_split_parity_with_oracle(name, split):
    """Fast/slow operator splitting (Sec. 3.2; split = 2: slow terms per fine
    step, Sec. 4.2), FP32 tendencies, against the split oracle."""
    make, nsteps, M = CASES[name]
    s = make()
    st = make_state(s, M=M, precision=fb.FP32_TENDENCY, split=split)
    fb.lts_advance(st, nsteps)
    h, u = fb.state_read(st)
    ho, uo = oracle.fblts(oracle.Mesh.from_scenario(s), oracle.scenario_params(s, split=split), s.level,
                          s.M if M is None else M, s.h0, s.u0, s.dt, nsteps)
    dh, du = rel_errors(h, u, ho, uo)
    assert dh <= 1e-6 and du <= 1e-5, (dh, du)
