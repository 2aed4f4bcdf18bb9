"""Pins of the oracle's fast/slow operator splitting (Sec. 3.2).

Eq. splitting replaces every Phi evaluation inside a coarse step by
Phi_fast(u*, h*) + Phi_slow(u^n, h^n) with Phi_fast = -g grad(h + b) (Eq.
fast_terms); the thickness equation is not split.  Independent facts used:
* the two parts add up to Phi at the same state (the split only moves the
  time level of the slow part);
* with no slow terms (pressure gradient only) the split scheme is the unsplit
  one, bitwise;
* M = 1 FB-LTS is global FB-RK(3,2) with the same splitting, bitwise;
* mass is still conserved to roundoff (Theorem 1: Psi is unsplit);
* the splitting is a Lie-Trotter splitting, first order in time: against an
  RK4 reference the split scheme converges at order 1 while the unsplit
  FB-RK(3,2) converges at order 2 on the same problem.

The variant proposed at the end of Sec. 4.2 (``split=2``) re-evaluates the
slow terms of the fine region's edges at the start of every fine step.  On an
f-plane with flat h and uniform flow the slow part is the Coriolis term alone
and the fast part vanishes, so one coarse step advances the flow by forward
Euler: (1 - i f dt) on every edge with ``split=1``, while with ``split=2`` the
fine edges away from the interface take M forward-Euler steps of dt/M,
(1 - i f dt/M)^M, and the coarse edges keep (1 - i f dt).  With M = 1, or on
one level, the variant is the plain splitting bitwise.
"""
import numpy as np
import pytest

import oracle
from synth import scenario


@pytest.fixture(scope="module")
def shelf():
    return scenario.shelf_case(nx=40, ny=24, dc=2e3, M=4, width=10e3, vortex=True)


@pytest.fixture(scope="module")
def bump():
    return scenario.gaussian_bump_case(two_level=True)


def test_fast_plus_slow_is_phi(shelf):
    m = oracle.Mesh.from_scenario(shelf)
    rng = np.random.default_rng(5)
    u = rng.normal(0.0, 0.3, shelf.mesh.nEdges)
    h = shelf.h0 * (1.0 + 1e-3 * rng.normal(size=shelf.mesh.nCells))
    p = oracle.scenario_params(shelf)
    fields = oracle.forcing_fields(m, p, 0.0)
    full = oracle.phi(m, p, u, h, fields)
    pf = oracle.scenario_params(shelf)
    pf.terms = oracle.T_PGRAD
    ps = oracle.scenario_params(shelf)
    ps.terms = p.terms & ~oracle.T_PGRAD
    parts = oracle.phi(m, pf, u, h, fields) + oracle.phi(m, ps, u, h, fields)
    assert np.max(np.abs(parts - full)) <= 1e-12 * np.max(np.abs(full))


def test_no_slow_terms_is_unsplit_bitwise(bump):
    m = oracle.Mesh.from_scenario(bump)
    for split in (False, True):
        p = oracle.scenario_params(bump, terms=oracle.T_PGRAD, split=split)
        out = oracle.fblts(m, p, bump.level, bump.M, bump.h0, bump.u0, bump.dt, 20)
        if not split:
            ref = out
    assert np.array_equal(out[0], ref[0]) and np.array_equal(out[1], ref[1])


def test_m1_split_is_split_fbrk32_bitwise(shelf):
    m = oracle.Mesh.from_scenario(shelf)
    p = oracle.scenario_params(shelf, split=True)
    h1, u1 = oracle.fblts(m, p, shelf.level, [1], shelf.h0, shelf.u0, shelf.dt, 6)
    h2, u2 = oracle.fbrk32(m, p, shelf.h0, shelf.u0, shelf.dt, 6)
    assert np.array_equal(h1, h2) and np.array_equal(u1, u2)


def test_split_conserves_mass(shelf):
    m = oracle.Mesh.from_scenario(shelf)
    p = oracle.scenario_params(shelf, split=True)
    A = shelf.mesh.areaCell
    h, u = shelf.h0, shelf.u0
    m0 = prev = float(np.sum(A * h))
    for n in range(6):
        h, u = oracle.fblts(m, p, shelf.level, shelf.M, h, u, shelf.dt, 1, t0=n * shelf.dt)
        cur = float(np.sum(A * h))
        assert abs(cur - prev) <= 1e-13 * m0
        prev = cur


def test_split_is_first_order_unsplit_second():
    # strong rotation makes the slow (Coriolis) part matter on the gravity-wave scale
    s = scenario.gaussian_bump_case(two_level=False, f=2e-3, amp=5.0)
    m = oracle.Mesh.from_scenario(s)
    T = 2400.0
    ref_p = oracle.scenario_params(s)
    hr, ur = oracle.rk4(m, ref_p, s.h0, s.u0, T / 960, 960)
    errs = {False: [], True: []}
    for split in (False, True):
        p = oracle.scenario_params(s, split=split)
        for n in (40, 80, 160):
            h, u = oracle.fbrk32(m, p, s.h0, s.u0, T / n, n)
            errs[split].append(np.max(np.abs(u - ur)))
    o_split = np.log2(np.array(errs[True][:-1]) / np.array(errs[True][1:]))
    o_full = np.log2(np.array(errs[False][:-1]) / np.array(errs[False][1:]))
    assert np.all(np.abs(o_split - 1.0) < 0.2), (o_split, errs[True])
    assert np.all(np.abs(o_full - 2.0) < 0.3), (o_full, errs[False])


def test_split2_with_m1_or_one_level_is_split1_bitwise(bump):
    m = oracle.Mesh.from_scenario(bump)
    one = np.zeros_like(bump.level)
    for level, M in ((bump.level, [1]), (one, [])):
        a = oracle.fblts(m, oracle.scenario_params(bump, split=1), level, M, bump.h0, bump.u0, bump.dt, 12)
        b = oracle.fblts(m, oracle.scenario_params(bump, split=2), level, M, bump.h0, bump.u0, bump.dt, 12)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("M", [2, 4])
def test_split2_fine_edges_take_M_euler_steps(M):
    f, H, dt = 1e-3, 1000.0, 60.0
    s = scenario.gaussian_bump_case(nx=48, ny=48, two_level=True, f=f, radius=160e3)
    m = oracle.Mesh.from_scenario(s)
    n = np.stack([np.cos(s.mesh.angleEdge), np.sin(s.mesh.angleEdge)], 1)
    U = 0.8 - 0.3j
    h0, u0 = np.full(s.mesh.nCells, H), n @ np.array([U.real, U.imag])
    _, _, ec, ed, st = oracle.regions(m, s.level)
    assert st == oracle.OM_OK

    def on_edges(W):
        return n @ np.array([W.real, W.imag])

    coarse = on_edges(U * (1 - 1j * f * dt))
    fine = on_edges(U * (1 - 1j * f * dt / M) ** M)
    deep = (ec[0] == oracle.RC_FINE) & (ed[0] >= 5)
    outer = (ec[0] == oracle.RC_INT) | (ec[0] == oracle.RC_IF1)
    h1, u1 = oracle.fblts(m, oracle.scenario_params(s, split=1), s.level, [M], h0, u0, dt, 1)
    np.testing.assert_allclose(u1, coarse, rtol=0, atol=1e-14)
    np.testing.assert_array_equal(h1, h0)
    h2, u2 = oracle.fblts(m, oracle.scenario_params(s, split=2), s.level, [M], h0, u0, dt, 1)
    np.testing.assert_allclose(u2[deep], fine[deep], rtol=0, atol=1e-14)
    np.testing.assert_allclose(u2[outer], coarse[outer], rtol=0, atol=1e-14)
    # the two differ by O((f dt)^2) on the fine edges
    assert np.max(np.abs(fine[deep] - coarse[deep])) > 1e-4


def test_split2_conserves_mass(shelf):
    m = oracle.Mesh.from_scenario(shelf)
    p = oracle.scenario_params(shelf, split=2)
    A = shelf.mesh.areaCell
    h, u = shelf.h0, shelf.u0
    m0 = prev = float(np.sum(A * h))
    for n in range(6):
        h, u = oracle.fblts(m, p, shelf.level, shelf.M, h, u, shelf.dt, 1, t0=n * shelf.dt)
        cur = float(np.sum(A * h))
        assert abs(cur - prev) <= 1e-13 * m0
        prev = cur
