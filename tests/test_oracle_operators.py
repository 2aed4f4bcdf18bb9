"""Pins of the oracle's TRiSK operators (Sec. 2.3, Eq. trisk_thickness, Eq. trisk_vorticity).

Independent facts used: on a regular hexagonal mesh the TRiSK divergence,
gradient and curl are exact for linear fields and the kinetic energy and the
tangential reconstruction are exact for uniform flow; the curl of a discrete
gradient vanishes; the total relative circulation telescopes to zero
(t_{e,v1} = -t_{e,v2}); the energy-conserving Coriolis term does no work.
"""
import numpy as np
import pytest

import oracle
from synth.mesh import hex_periodic, finalize
from synth import scenario

NX, NY, DC = 16, 16, 1.0e4


@pytest.fixture(scope="module")
def hexm():
    mesh = finalize(hex_periodic(NX, NY, DC))
    return mesh


def _om(mesh, f=0.0):
    return oracle.Mesh(mesh, np.zeros(mesh.nCells), np.full(mesh.nVertices, f))


def _normals(mesh):
    n = np.stack([np.cos(mesh.angleEdge), np.sin(mesh.angleEdge)], 1)
    t = np.stack([-n[:, 1], n[:, 0]], 1)
    return n, t


def _interior(x, y, L, margin):
    return (x > margin) & (x < L[0] - margin) & (y > margin) & (y < L[1] - margin)


def test_divergence_of_linear_flux_is_exact(hexm):
    m = _om(hexm)
    p = oracle.params(terms=oracle.T_LINEAR_FLUX, H_lin=1.0)
    n, _ = _normals(hexm)
    a, b, c, d = 0.3e-3, -0.7e-3, 0.2e-3, 0.5e-3
    Fx = a * hexm.xEdge + b * hexm.yEdge + 1.0
    Fy = c * hexm.xEdge + d * hexm.yEdge - 2.0
    u = Fx * n[:, 0] + Fy * n[:, 1]
    psi = oracle.psi(m, p, u, np.ones(hexm.nCells))
    sel = _interior(hexm.xCell, hexm.yCell, hexm.period, 2 * DC)
    assert sel.sum() > 50
    np.testing.assert_allclose(psi[sel], -(a + d), rtol=1e-11, atol=0)


def test_gradient_of_linear_h_is_exact(hexm):
    m = _om(hexm)
    g = 9.80616
    p = oracle.params(g=g, terms=oracle.T_PGRAD)
    n, _ = _normals(hexm)
    ax, ay = 2e-5, -3e-5
    h = 100.0 + ax * hexm.xCell + ay * hexm.yCell
    phi = oracle.phi(m, p, np.zeros(hexm.nEdges), h)
    sel = _interior(hexm.xEdge, hexm.yEdge, hexm.period, 2 * DC)
    np.testing.assert_allclose(phi[sel], -g * (ax * n[sel, 0] + ay * n[sel, 1]), rtol=1e-9, atol=1e-15)


def test_vertex_curl_of_linear_velocity_is_exact(hexm):
    m = _om(hexm)
    n, _ = _normals(hexm)
    A = np.array([[0.1, -0.4], [0.25, 0.3]]) * 1e-4
    U = np.stack([A[0, 0] * hexm.xEdge + A[0, 1] * hexm.yEdge, A[1, 0] * hexm.xEdge + A[1, 1] * hexm.yEdge], 1)
    u = (U * n).sum(1)
    z, hv, q = oracle.vertex_fields(m, u, np.full(hexm.nCells, 50.0))
    sel = _interior(hexm.xVertex, hexm.yVertex, hexm.period, 2 * DC)
    np.testing.assert_allclose(z[sel], A[1, 0] - A[0, 1], rtol=1e-10)
    np.testing.assert_allclose(hv, 50.0, rtol=1e-14)
    np.testing.assert_allclose(q[sel], (A[1, 0] - A[0, 1]) / 50.0, rtol=1e-10)


def test_kinetic_energy_and_tangential_reconstruction_uniform_flow(hexm):
    m = _om(hexm)
    n, t = _normals(hexm)
    U = np.array([0.37, -1.21])
    u = n @ U
    np.testing.assert_allclose(oracle.ke(m, u), 0.5 * U @ U, rtol=1e-13)
    np.testing.assert_allclose(oracle.tangential(m, u), t @ U, atol=1e-14)


def test_curl_of_gradient_tendency_vanishes(hexm):
    """Mimetic property: the vertex curl of -grad(K + g(h+b)) is zero."""
    m = _om(hexm)
    rng = np.random.default_rng(1)
    u = rng.normal(size=hexm.nEdges)
    h = 100.0 + rng.normal(size=hexm.nCells)
    p = oracle.params(terms=oracle.T_PGRAD | oracle.T_KE)
    phi = oracle.phi(m, p, u, h)
    z, _, _ = oracle.vertex_fields(m, phi, h)
    assert np.abs(z).max() < 1e-12 * np.abs(phi).max() / DC


@pytest.mark.parametrize("case", ["periodic", "walls"])
def test_total_circulation_telescopes(case, hexm):
    mesh = hexm if case == "periodic" else scenario.shelf_case(nx=24, ny=16).mesh
    m = _om(mesh)
    rng = np.random.default_rng(2)
    u = rng.normal(size=mesh.nEdges)
    u[mesh.boundary_edge_mask()] = 0.0
    z, _, _ = oracle.vertex_fields(m, u, np.ones(mesh.nCells))
    Av = np.where(mesh.cellsOnVertex >= 0, mesh.kiteAreasOnVertex, 0.0).sum(1)
    scale = np.sum(np.abs(Av * z))
    assert abs(np.sum(Av * z)) < 1e-13 * scale


@pytest.mark.parametrize("case", ["periodic", "walls"])
def test_coriolis_term_does_no_work(case, hexm):
    """sum_e dc_e dv_e F_e (q F_perp)_e = 0 for antisymmetric TRiSK weights."""
    mesh = hexm if case == "periodic" else scenario.shelf_case(nx=24, ny=16).mesh
    m = _om(mesh, f=1e-4)
    rng = np.random.default_rng(3)
    u = rng.normal(size=mesh.nEdges)
    u[mesh.boundary_edge_mask()] = 0.0
    h = 100.0 + 10.0 * rng.random(mesh.nCells)
    p = oracle.params(terms=oracle.T_CORIOLIS)
    cor = oracle.phi(m, p, u, h)
    c0, c1 = mesh.cellsOnEdge.T
    inter = (c0 >= 0) & (c1 >= 0)
    F = np.where(inter, 0.5 * (h[np.maximum(c0, 0)] + h[np.maximum(c1, 0)]) * u, 0.0)
    work = mesh.dcEdge * mesh.dvEdge * F * cor
    assert abs(work.sum()) < 1e-13 * np.abs(work).sum()


def test_thickness_tendency_uniform_flow_is_zero(hexm):
    m = _om(hexm)
    n, _ = _normals(hexm)
    u = n @ np.array([1.3, 0.4])
    psi = oracle.psi(m, oracle.params(), u, np.full(hexm.nCells, 20.0))
    assert np.abs(psi).max() < 1e-15 * 20.0 * 1.3 / DC * 1e3
