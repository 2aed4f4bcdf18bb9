"""Pins of the oracle's FB-LTS (Sec. 2.2) and its region construction.

Independent facts used:
* M = 1 makes every prediction equal the data it interpolates, so FB-LTS is
  FB-RK(3,2) (Sec. 2.2, after Eq. preds) - bitwise in the oracle.
* All cells on one level is global FB-RK(3,2).
* Theorem 1: total mass sum A_i h_i is conserved to roundoff (periodic and
  no-flow meshes, any forcing that acts on momentum only).
* Theorem 2 (diagnostic form): total absolute vorticity is constant.
* Sec. 3.3: computing every coarse sub-stage on all of F^5 instead of the
  shrinking sets changes nothing (bitwise).
* Appendix A: the predictions reproduce linear-in-time data exactly.
* Sec. 2.3 / Fig. convergence: second-order convergence against RK4 with
  M = 4, separately on fine, IF-1, IF-2 and interior cells and edges; and
  with three levels (M = 2 at both pairs), separately on those sets of both
  level pairs, which pins the hand-off of the outer pair's IF-1 predictions
  of subcycle k (Eq. preds) into the inner pair's coarse advancement: a
  prediction from the wrong subcycle leaves the interface first order.
* A lake at rest over variable bathymetry stays at rest.
"""
import numpy as np
import pytest

import oracle
from synth import scenario


@pytest.fixture(scope="module")
def bump():
    return scenario.gaussian_bump_case(two_level=True)


@pytest.fixture(scope="module")
def shelf():
    return scenario.shelf_case(nx=40, ny=24, dc=2e3, M=4, width=10e3)


@pytest.fixture(scope="module")
def nested():
    return scenario.nested_disk_case()


def _run(s, M=None, nsteps=5, full_band=False, level=None):
    m = oracle.Mesh.from_scenario(s)
    p = oracle.scenario_params(s)
    return oracle.fblts(m, p, s.level if level is None else level, s.M if M is None else M,
                        s.h0, s.u0, s.dt, nsteps, full_band=full_band)


def test_m1_is_fbrk32_bitwise(bump, shelf):
    for s in (bump, shelf):
        m = oracle.Mesh.from_scenario(s)
        p = oracle.scenario_params(s)
        h1, u1 = _run(s, M=[1], nsteps=6)
        h2, u2 = oracle.fbrk32(m, p, s.h0, s.u0, s.dt, 6)
        assert np.array_equal(h1, h2) and np.array_equal(u1, u2)


def test_m1_three_levels_is_fbrk32_bitwise(nested):
    m = oracle.Mesh.from_scenario(nested)
    p = oracle.scenario_params(nested)
    h1, u1 = _run(nested, M=[1, 1], nsteps=4)
    h2, u2 = oracle.fbrk32(m, p, nested.h0, nested.u0, nested.dt, 4)
    assert np.array_equal(h1, h2) and np.array_equal(u1, u2)


def test_single_level_is_fbrk32_bitwise(bump):
    m = oracle.Mesh.from_scenario(bump)
    p = oracle.scenario_params(bump)
    lev = np.zeros_like(bump.level)
    h1, u1 = oracle.fblts(m, p, lev, [], bump.h0, bump.u0, bump.dt, 5)
    h2, u2 = oracle.fbrk32(m, p, bump.h0, bump.u0, bump.dt, 5)
    assert np.array_equal(h1, h2) and np.array_equal(u1, u2)


@pytest.mark.parametrize("M", [2, 4, 8])
def test_mass_conserved_each_step(shelf, M):
    m = oracle.Mesh.from_scenario(shelf)
    p = oracle.scenario_params(shelf)
    assert p.terms & oracle.T_FORCING
    h, u = shelf.h0.copy(), shelf.u0.copy()
    m0 = oracle.diagnostics(m, h, u)[0]
    prev = m0
    for _ in range(6):
        h, u = oracle.fblts(m, p, shelf.level, [M], h, u, shelf.dt * M / 4, 1)
        cur = oracle.diagnostics(m, h, u)[0]
        assert abs(cur - prev) <= 1e-13 * m0
        prev = cur
    assert np.abs(u).max() > 0  # the wind did move the water


def test_mass_conserved_three_levels(nested):
    m = oracle.Mesh.from_scenario(nested)
    h, u = _run(nested, nsteps=8)
    m0, w0 = oracle.diagnostics(m, nested.h0, nested.u0)
    m1, w1 = oracle.diagnostics(m, h, u)
    assert abs(m1 - m0) <= 8e-13 * m0
    assert abs(w1 - w0) <= 1e-13 * abs(w0)


def test_absolute_vorticity_constant(bump):
    m = oracle.Mesh.from_scenario(bump)
    h, u = _run(bump, nsteps=20)
    w0 = oracle.diagnostics(m, bump.h0, bump.u0)[1]
    w1 = oracle.diagnostics(m, h, u)[1]
    assert np.abs(u).max() > 1e-3
    assert abs(w1 - w0) <= 1e-13 * abs(w0)


@pytest.mark.parametrize("which", ["bump", "shelf", "nested"])
def test_full_band_equals_shrinking_sets(which, bump, shelf, nested):
    s = {"bump": bump, "shelf": shelf, "nested": nested}[which]
    h1, u1 = _run(s, nsteps=4)
    h2, u2 = _run(s, nsteps=4, full_band=True)
    assert np.array_equal(h1, h2) and np.array_equal(u1, u2)


def test_predictions_exact_for_linear_data():
    a, b, dt = 3.25, -0.75, 0.8
    X = lambda t: a + b * t
    for M in (1, 2, 3, 4, 8):
        for k in range(M + 1):
            xk, xk13, xk12 = oracle.predict(k, M, X(0), X(dt / 3), X(dt / 2), X(dt))
            assert xk == pytest.approx(X(k * dt / M), rel=1e-15, abs=1e-15)
            if k < M:
                assert xk13 == pytest.approx(X((k + 1 / 3) * dt / M), rel=1e-15, abs=1e-15)
                assert xk12 == pytest.approx(X((k + 1 / 2) * dt / M), rel=1e-15, abs=1e-15)


def test_predictions_second_order_for_smooth_data():
    """Error O(dt^2) on sin(t) data where the stage values are exact."""
    errs = []
    for dt in (0.2, 0.1, 0.05):
        X = np.sin
        e = 0.0
        for k in range(4):
            xk, xk13, xk12 = oracle.predict(k, 4, X(0), X(dt / 3), X(dt / 2), X(dt))
            e = max(e, abs(xk - X(k * dt / 4)), abs(xk13 - X((k + 1 / 3) * dt / 4)),
                    abs(xk12 - X((k + 1 / 2) * dt / 4)))
        errs.append(e)
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 1.9), orders


def test_lake_at_rest(shelf):
    m = oracle.Mesh.from_scenario(shelf)
    p = oracle.params(g=shelf.g, terms=oracle.T_FULL)   # no wind, no drag
    h, u = oracle.fblts(m, p, shelf.level, shelf.M, shelf.h0, shelf.u0, shelf.dt, 5)
    assert np.abs(u).max() < 1e-12
    assert np.abs(h - shelf.h0).max() < 1e-10


@pytest.mark.slow
def test_second_order_convergence_per_region():
    s = scenario.gaussian_bump_case(two_level=True, amp=5.0, f=0.0)
    Lx, Ly = s.mesh.period
    rx, ry = s.mesh.xCell - Lx / 2, s.mesh.yCell - Ly / 2
    s.h0 = 1000.0 + 5.0 * np.exp(-(rx ** 2 + ry ** 2) / 60e3 ** 2)
    m = oracle.Mesh.from_scenario(s)
    p = oracle.params(terms=oracle.T_PGRAD)   # Eq. grav_wave_model
    T = 1200.0
    href, uref = oracle.rk4(m, p, s.h0, s.u0, 40.0 / 64, int(T / (40.0 / 64)))
    cc, cd, ec, ed, st = oracle.regions(m, s.level)
    assert st == 0
    errs = []
    for dt in (20.0, 10.0, 5.0):
        h, u = oracle.fblts(m, p, s.level, [4], s.h0, s.u0, dt, int(T / dt))
        errs.append([np.sqrt(np.mean((h - href)[cc[0] == r] ** 2)) for r in range(4)]
                    + [np.sqrt(np.mean((u - uref)[ec[0] == r] ** 2)) for r in range(4)])
    errs = np.array(errs)
    orders = np.log2(errs[:-1] / errs[1:])
    assert np.all(np.abs(orders - 2.0) < 0.1), orders


@pytest.mark.slow
def test_second_order_convergence_three_levels_per_region():
    """Each fine subcycle of the pair (0, 1) is an FB-LTS step of the pair
    (1, 2) whose coarse advancement reads the outer IF-1 predictions of that
    subcycle as boundary data (Sec. 2.2 steps 2-3).  The scheme stays second
    order (Sec. 2.3) on every set of both pairs only if the subcycle index of
    those predictions is right; the orders are measured against RK4 on the
    linear-pressure gravity wave (Eq. grav_wave_model, f = 0)."""
    s = scenario.three_level_wave_case()
    m = oracle.Mesh.from_scenario(s)
    p = oracle.params(terms=oracle.T_PGRAD)
    T = 1600.0
    dt_ref = 40.0 / 64
    href, uref = oracle.rk4(m, p, s.h0, s.u0, dt_ref, int(round(T / dt_ref)))
    cc, cd, ec, ed, st = oracle.regions(m, s.level)
    assert st == 0 and cc.shape[0] == 2
    errs = []
    for dt in (10.0, 5.0, 2.5):
        h, u = oracle.fblts(m, p, s.level, s.M, s.h0, s.u0, dt, int(round(T / dt)))
        row = []
        for pair in (0, 1):
            for r in (oracle.RC_FINE, oracle.RC_IF1, oracle.RC_IF2, oracle.RC_INT):
                assert (cc[pair] == r).any() and (ec[pair] == r).any()
                row.append(np.sqrt(np.mean((h - href)[cc[pair] == r] ** 2)))
                row.append(np.sqrt(np.mean((u - uref)[ec[pair] == r] ** 2)))
        errs.append(row)
    errs = np.array(errs)
    orders = np.log2(errs[:-1] / errs[1:])
    assert np.all(np.abs(orders - 2.0) < 0.1), orders


def test_region_layers(bump):
    m = oracle.Mesh.from_scenario(bump)
    cc, cd, ec, ed, st = oracle.regions(m, bump.level)
    assert st == 0
    mesh = bump.mesh
    fine = bump.level == 1
    dF = scenario.graph_distance(mesh, fine)
    dC = scenario.graph_distance(mesh, ~fine)
    np.testing.assert_array_equal(cc[0][fine], oracle.RC_FINE)
    np.testing.assert_array_equal(cd[0][fine], dC[fine])
    exp = np.where(dF <= 2, oracle.RC_IF1, np.where(dF <= 4, oracle.RC_IF2, oracle.RC_INT))
    np.testing.assert_array_equal(cc[0][~fine], exp[~fine])
    # an edge belongs to the region of its cell closest to the fine region
    c0, c1 = mesh.cellsOnEdge.T
    np.testing.assert_array_equal(ec[0], np.minimum(cc[0][c0], cc[0][c1]))


def test_level_separation_is_enforced(nested):
    bad = nested.level.copy()
    d = scenario.graph_distance(nested.mesh, nested.level == 2)
    bad[(nested.level == 1) & (d > 2)] = 0
    m = oracle.Mesh.from_scenario(nested)
    _, _, _, _, st = oracle.regions(m, bad)
    assert st == oracle.OM_E_REGIONS
