"""GPU FP64 path against the oracle, through the C ABI.

Bar (from the method's accuracy target): after the stated number of coarse
steps, max_i |dh_i|/|h_i| <= 1e-10 and max_e |du_e| / max_e |u_e| <= 1e-10,
mass drift per step <= 1e-13 relative, bit-reproducible runs.
"""
import numpy as np
import pytest

import oracle
import paper_2405_10505_gb300 as fb
from synth import scenario
from tests.gpu_util import make_state, rel_errors

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _oracle(s, nsteps, M=None, level=None):
    m = oracle.Mesh.from_scenario(s)
    p = oracle.scenario_params(s)
    return oracle.fblts(m, p, s.level if level is None else level, s.M if M is None else M,
                        s.h0, s.u0, s.dt, nsteps)


CASES = {
    # the 32x32 bump case for 200 coarse steps, one level and two levels (M=2)
    "bump_single": (lambda: scenario.gaussian_bump_case(two_level=False), 200, None),
    "bump_lts_m2": (lambda: scenario.gaussian_bump_case(two_level=True), 200, None),
    "bump_lts_m1": (lambda: scenario.gaussian_bump_case(two_level=True), 100, [1]),
    "bump_lts_m5": (lambda: scenario.gaussian_bump_case(two_level=True), 100, [5]),
    "shelf_forced_m4": (lambda: scenario.shelf_case(nx=64, ny=48, dc=2e3, M=4, width=10e3), 100, None),
    "nested_3level": (lambda: scenario.nested_disk_case(nx=64, ny=64, radii=(190e3, 50e3)), 100, None),
    "shelf_vortex_m4": (lambda: scenario.shelf_case(nx=64, ny=48, dc=2e3, M=4, width=10e3, vortex=True), 100, None),
    # irregular cells of 3..11 edges (12-slot rows, obtuse triangles), 2 levels
    "jittered_voronoi_m2": (lambda: scenario.jittered_voronoi_case(), 100, None),
}


@pytest.mark.parametrize("name", list(CASES))
def test_parity_with_oracle(name):
    make, nsteps, M = CASES[name]
    s = make()
    st = make_state(s, M=M)
    fb.lts_advance(st, nsteps)
    h, u = fb.state_read(st)
    ho, uo = _oracle(s, nsteps, M=M)
    dh, du = rel_errors(h, u, ho, uo)
    assert dh <= TOL and du <= TOL, (dh, du)


def test_graph_and_stream_launches_agree_bitwise():
    s = scenario.gaussian_bump_case(two_level=True)
    a = make_state(s, use_graph=True)
    b = make_state(s, use_graph=False)
    fb.lts_advance(a, 25)
    fb.lts_advance(b, 25)
    ha, ua = fb.state_read(a)
    hb, ub = fb.state_read(b)
    assert np.array_equal(ha, hb) and np.array_equal(ua, ub)


def test_bit_reproducible():
    s = scenario.shelf_case(nx=64, ny=48, dc=2e3, M=4, width=10e3)
    out = []
    for _ in range(2):
        st = make_state(s)
        fb.lts_advance(st, 40)
        out.append(fb.state_read(st))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_mass_drift_per_step_and_diagnostics():
    s = scenario.shelf_case(nx=64, ny=48, dc=2e3, M=4, width=10e3)
    st = make_state(s)
    m = oracle.Mesh.from_scenario(s)
    mass0, av0 = fb.diagnostics(st)
    om0, oa0 = oracle.diagnostics(m, s.h0, s.u0)
    assert mass0 == pytest.approx(om0, rel=1e-13)
    assert av0 == pytest.approx(oa0, rel=1e-12)
    prev = mass0
    for _ in range(10):
        fb.lts_advance(st, 1)
        cur, _ = fb.diagnostics(st)
        assert abs(cur - prev) <= 1e-13 * mass0
        prev = cur
    h, u = fb.state_read(st)
    om, oa = oracle.diagnostics(m, h, u)
    gm, ga = fb.diagnostics(st)
    assert gm == pytest.approx(om, rel=1e-13)
    assert ga == pytest.approx(oa, rel=1e-12)


def test_checkpoint_resume_is_bit_identical():
    s = scenario.gaussian_bump_case(two_level=True)
    a = make_state(s)
    fb.lts_advance(a, 30)
    ref_h, ref_u = fb.state_read(a)
    b = make_state(s)
    fb.lts_advance(b, 12)
    blob = fb.state_save(b)
    c = make_state(s)
    fb.state_load(c, blob)
    assert fb.state_time(c)[0] == 12
    fb.lts_advance(c, 18)
    h, u = fb.state_read(c)
    assert np.array_equal(h, ref_h) and np.array_equal(u, ref_u)


def test_run_host_matches_advance():
    s = scenario.gaussian_bump_case(two_level=True)
    a = make_state(s)
    fb.lts_advance(a, 7)
    ha, ua = fb.state_read(a)
    b = make_state(s)
    h = np.empty_like(s.h0)
    u = np.empty_like(s.u0)
    fb.run_host(b, np.ascontiguousarray(s.h0), np.ascontiguousarray(s.u0), 7, h, u)
    assert np.array_equal(h, ha) and np.array_equal(u, ua)


def test_write_read_roundtrip_caller_order():
    s = scenario.shelf_case(nx=32, ny=16, dc=2e3, M=4, width=10e3)
    st = make_state(s)
    rng = np.random.default_rng(5)
    h = s.h0 + rng.random(s.mesh.nCells)
    u = rng.normal(size=s.mesh.nEdges)
    u[s.mesh.boundary_edge_mask()] = 0.0
    fb.state_write(st, h, u)
    h2, u2 = fb.state_read(st)
    assert np.array_equal(h, h2) and np.array_equal(u, u2)


def test_instability_is_reported():
    s = scenario.gaussian_bump_case(two_level=False)
    st = make_state(s)
    h = s.h0.copy()
    h[10] = np.nan          # a non-finite thickness planted on the host
    fb.state_write(st, h, None)
    fb.lts_advance(st, 1)
    with pytest.raises(fb.FbltsError) as ei:
        fb.synchronize(st)
    assert ei.value.status == fb.E_UNSTABLE


def test_bad_regions_rejected():
    s = scenario.nested_disk_case(nx=64, ny=64, radii=(190e3, 50e3))
    bad = s.level.copy()
    d = scenario.graph_distance(s.mesh, s.level == 2)
    bad[(s.level == 1) & (d > 3)] = 0
    with pytest.raises(fb.FbltsError) as ei:
        fb.mesh_create(s.mesh, s.fVertex, level=bad, M=s.M)
    assert ei.value.status == fb.E_REGIONS


@pytest.mark.parametrize("precision", [fb.FP64, fb.FP32_TENDENCY])
def test_odd_sized_arrays(precision):
    """Array sizes that are not multiples of the arena alignment (37 x 22 cells)."""
    s = scenario.shelf_case(nx=37, ny=22, dc=2e3, M=4, width=10e3)
    assert (s.mesh.nCells * 8) % 256 and (s.mesh.nEdges * 8) % 256
    st = make_state(s, precision=precision)
    fb.lts_advance(st, 20)
    h, u = fb.state_read(st)
    ho, uo = _oracle(s, 20)
    dh, du = rel_errors(h, u, ho, uo)
    tol = TOL if precision == fb.FP64 else 1e-5
    assert dh <= tol and du <= tol, (dh, du)


SPLIT_CASES = ["bump_lts_m2", "shelf_forced_m4", "shelf_vortex_m4", "nested_3level", "jittered_voronoi_m2"]


@pytest.mark.parametrize("split", [1, 2])
@pytest.mark.parametrize("name", SPLIT_CASES)
def test_split_parity_with_oracle(name, split):
    """Fast/slow operator splitting (Sec. 3.2; split = 2: slow terms per fine
    step, Sec. 4.2) against the split oracle (FP64, 1e-10)."""
    make, nsteps, M = CASES[name]
    s = make()
    st = make_state(s, M=M, split=split)
    fb.lts_advance(st, nsteps)
    h, u = fb.state_read(st)
    m = oracle.Mesh.from_scenario(s)
    ho, uo = oracle.fblts(m, oracle.scenario_params(s, split=split), s.level, s.M if M is None else M, s.h0, s.u0,
                          s.dt, nsteps)
    dh, du = rel_errors(h, u, ho, uo)
    assert dh <= 1e-10 and du <= 1e-10, (dh, du)


def test_zero_steps_and_bad_counts():
    """Advancing 0 coarse steps leaves the state bitwise as it was; a negative
    count is an argument error that leaves the state usable."""
    s = scenario.gaussian_bump_case(two_level=True)
    st = make_state(s)
    fb.lts_advance(st, 3)
    h0, u0 = fb.state_read(st)
    fb.lts_advance(st, 0)
    h1, u1 = fb.state_read(st)
    assert np.array_equal(h0, h1) and np.array_equal(u0, u1)
    with pytest.raises(fb.FbltsError) as e:
        fb.lts_advance(st, -1)
    assert e.value.status == fb.E_ARG
    fb.lts_advance(st, 2)
    ref = make_state(s)
    fb.lts_advance(ref, 5)
    h2, u2 = fb.state_read(st)
    hr, ur = fb.state_read(ref)
    assert np.array_equal(h2, hr) and np.array_equal(u2, ur)


def test_mesh_destroy_refused_while_in_use():
    """A mesh whose device tables a state or a server request still reads
    cannot be destroyed (FBLTS_E_STATE, the mesh stays usable); once they are
    gone it can."""
    s = scenario.gaussian_bump_case(two_level=True)
    mesh = fb.mesh_create(s.mesh, s.fVertex, level=s.level, M=s.M)
    st = make_state(s, mesh=mesh)
    with pytest.raises(fb.FbltsError) as e:
        fb.mesh_destroy(mesh)
    assert e.value.status == fb.E_STATE and mesh.handle
    fb.lts_advance(st, 3)
    h, u = fb.state_read(st)
    ref = make_state(s)
    fb.lts_advance(ref, 3)
    hr, ur = fb.state_read(ref)
    assert np.array_equal(h, hr) and np.array_equal(u, ur)
    fb.state_destroy(st)
    srv = fb.server_create()
    fb.server_submit(srv, mesh, fb.make_params(s.dt, g=s.g), s.h0, s.u0, s.bottom, 2)
    with pytest.raises(fb.FbltsError) as e:
        fb.mesh_destroy(mesh)
    assert e.value.status == fb.E_STATE
    fb.server_destroy(srv)
    fb.mesh_destroy(mesh)
    assert mesh.handle is None


def test_promoted_levels_run_and_match_the_oracle():
    """Nested disks without the separation the band order needs: refused as
    given, accepted with FBLTS_MESH_PROMOTE_LEVELS; the run then matches the
    oracle on the levels the library reports (fblts_mesh_levels)."""
    s = scenario.nested_disk_case(nx=64, ny=64, radii=(190e3, 50e3))
    Lx, Ly = s.mesh.period
    dx = scenario._min_image(s.mesh.xCell - Lx / 2, Lx)
    dy = scenario._min_image(s.mesh.yCell - Ly / 2, Ly)
    r2 = dx ** 2 + dy ** 2
    raw = np.zeros(s.mesh.nCells, np.int32)
    raw[r2 <= 190e3 ** 2] = 1
    raw[r2 <= 50e3 ** 2] = 2
    with pytest.raises(fb.FbltsError):
        fb.mesh_create(s.mesh, s.fVertex, level=raw, M=s.M)
    mesh = fb.mesh_create(s.mesh, s.fVertex, level=raw, M=s.M, promote=True)
    lev = fb.mesh_levels(mesh)
    assert (lev >= raw).all() and not np.array_equal(lev, raw)
    st = make_state(s, mesh=mesh)
    fb.lts_advance(st, 20)
    h, u = fb.state_read(st)
    ho, uo = _oracle(s, 20, level=lev)
    dh, du = rel_errors(h, u, ho, uo)
    assert dh <= TOL and du <= TOL, (dh, du)
