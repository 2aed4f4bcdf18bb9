"""Pins of the oracle's forcing terms (Eq. hurricane_model).

The paper names the terms but not their coefficients; the closed forms used
here are those of the terms as written: wind stress C_W |u_W - u| (u_W - u)/h,
bottom drag -C_D |u| u / h, surface pressure -(1/rho0) grad p_s, with the
Holland-type vortex whose wind is in gradient-wind balance with its pressure.
"""
import numpy as np
import pytest

import oracle
from synth.mesh import hex_periodic, finalize
from synth.scenario import Forcing

DC = 1.0e4


@pytest.fixture(scope="module")
def hexm():
    return finalize(hex_periodic(12, 12, DC))


def _normals(mesh):
    n = np.stack([np.cos(mesh.angleEdge), np.sin(mesh.angleEdge)], 1)
    return n, np.stack([-n[:, 1], n[:, 0]], 1)


def test_uniform_wind_stress_and_drag(hexm):
    m = oracle.Mesh(hexm, np.zeros(hexm.nCells), np.zeros(hexm.nVertices))
    n, t = _normals(hexm)
    W = np.array([-15.0, 4.0])
    U = np.array([0.6, 0.2])
    H = 50.0
    fz = Forcing(wind_u=W[0], wind_v=W[1], cd=2.5e-3, wind_stress=True)
    p = oracle.params(terms=oracle.T_FORCING, forcing=fz)
    p.terms = oracle.T_FORCING
    fields = oracle.forcing_fields(m, p, 0.0)
    np.testing.assert_allclose(fields[0], n @ W, atol=1e-12)
    np.testing.assert_allclose(fields[1], t @ W, atol=1e-12)
    phi = oracle.phi(m, p, n @ U, np.full(hexm.nCells, H), fields)
    cw = (1.225 / 1025.0) * (0.75 + 0.067 * np.hypot(*W)) * 1e-3
    D = W - U
    exp = cw * np.hypot(*D) * (n @ D) / H - 2.5e-3 * np.hypot(*U) * (n @ U) / H
    np.testing.assert_allclose(phi, exp, rtol=1e-12, atol=1e-18)


def test_vortex_gradient_wind_balance():
    """V^2/r + f V = (1/rho_air) dp/dr at every radius."""
    mesh = finalize(hex_periodic(40, 40, 5e3))
    m = oracle.Mesh(mesh, np.zeros(mesh.nCells), np.zeros(mesh.nVertices))
    Lx, Ly = mesh.period
    f0 = 5e-5
    vt = (96000.0, 5000.0, 40e3, 1.4, Lx / 2, Ly / 2, 0.0, 0.0)
    p = oracle.params(forcing=Forcing(vortex=vt), f0=f0)
    rho = 1.225
    # sample along a ray through edges: use cell pressure and edge wind
    wn, wt, ps = oracle.forcing_fields(m, p, 0.0)
    n, t = _normals(mesh)
    Wx = wn * n[:, 0] + wt * t[:, 0]
    Wy = wn * n[:, 1] + wt * t[:, 1]
    rx, ry = mesh.xEdge - Lx / 2, mesh.yEdge - Ly / 2
    r = np.hypot(rx, ry)
    sel = (r > 10e3) & (r < 80e3)
    V = (-Wx * ry + Wy * rx)[sel] / r[sel]          # azimuthal (counter-clockwise) wind
    radial = (Wx * rx + Wy * ry)[sel] / r[sel]
    assert np.abs(radial).max() < 1e-9
    rr = r[sel]
    a = (40e3 / rr) ** 1.4
    dpdr = 5000.0 * np.exp(-a) * 1.4 * a / rr
    np.testing.assert_allclose(V ** 2 / rr + f0 * V, dpdr / rho, rtol=1e-9)
    # pressure at cell centres
    rc = np.hypot(mesh.xCell - Lx / 2, mesh.yCell - Ly / 2)
    np.testing.assert_allclose(ps, 96000.0 + 5000.0 * np.exp(-(40e3 / rc) ** 1.4), rtol=1e-14)


def test_vortex_moves_along_track():
    mesh = finalize(hex_periodic(20, 20, 5e3))
    m = oracle.Mesh(mesh, np.zeros(mesh.nCells), np.zeros(mesh.nVertices))
    vt = (96000.0, 5000.0, 20e3, 1.4, 20e3, 30e3, 5.0, -2.0)
    p = oracle.params(forcing=Forcing(vortex=vt))
    t = 3600.0
    _, _, ps = oracle.forcing_fields(m, p, t)
    i = np.argmin(ps)
    assert np.hypot(mesh.xCell[i] - (20e3 + 5.0 * t), mesh.yCell[i] - (30e3 - 2.0 * t)) < 6e3


def test_pressure_gradient_term(hexm):
    m = oracle.Mesh(hexm, np.zeros(hexm.nCells), np.zeros(hexm.nVertices))
    n, _ = _normals(hexm)
    p = oracle.params(forcing=Forcing(vortex=(0, 0, 1, 1, 0, 0, 0, 0)))
    p.terms = oracle.T_FORCING
    gx, gy = 1e-3, -2e-3
    ps = 1e5 + gx * hexm.xCell + gy * hexm.yCell
    fields = (np.zeros(hexm.nEdges), np.zeros(hexm.nEdges), ps)
    phi = oracle.phi(m, p, np.zeros(hexm.nEdges), np.full(hexm.nCells, 10.0), fields)
    Lx, Ly = hexm.period
    sel = (hexm.xEdge > 2 * DC) & (hexm.xEdge < Lx - 2 * DC) & (hexm.yEdge > 2 * DC) & (hexm.yEdge < Ly - 2 * DC)
    np.testing.assert_allclose(phi[sel], -(n[sel] @ np.array([gx, gy])) / 1025.0, rtol=1e-7)
