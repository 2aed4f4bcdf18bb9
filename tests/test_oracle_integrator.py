"""Pins of the oracle's FB-RK(3,2) (Sec. 2.1, Eq. fbrk32) and RK4.

Independent facts used:
* A single Fourier gravity-wave mode of the linearised system on a regular
  hexagonal mesh stays a mode, with the semi-discrete frequency
  omega^2 = g H kappa^2, kappa^2 = 4/(3 dc^2) sum_{j=1..3} (1 - cos k.d_j).
  The mesh run must then follow the 2x2 scalar recursion of the scheme.
* The CFL-optimised weights (0.531, 0.531, 0.313) allow a larger stable step
  than RK(3,2) (Sec. 2.1 reports 1.6-2.2x on nonlinear cases); on the linear
  mode the ratio must exceed 2.0, which the plausible misplacements of the
  FB averages do not reach (swapped h*** terms give 1.99, reversed weights 1.73).
* With flat h the momentum equation is the inertial oscillation
  dU/dt = -f k x U, on which the scheme is RK(3,2) whose amplification is the
  textbook polynomial 1 + z + z^2/2 + z^3/6.
* Second-order (FB-RK) and fourth-order (RK4) convergence.
"""
import numpy as np
import pytest

import oracle
from synth.mesh import hex_periodic, finalize

G = 9.80616
H = 1000.0
DC = 1.0e4


@pytest.fixture(scope="module")
def mode():
    mesh = finalize(hex_periodic(16, 16, DC))
    Lx, Ly = mesh.period
    m = oracle.Mesh(mesh, np.zeros(mesh.nCells), np.zeros(mesh.nVertices))
    k = np.array([2 * np.pi * 3 / Lx, 2 * np.pi * 2 / Ly])
    phi = np.cos(k[0] * mesh.xCell + k[1] * mesh.yCell)
    c0, c1 = mesh.cellsOnEdge.T
    gphi = (phi[c1] - phi[c0]) / mesh.dcEdge
    d = [np.array([DC, 0.0]), np.array([DC / 2, DC * np.sqrt(3) / 2]), np.array([-DC / 2, DC * np.sqrt(3) / 2])]
    kap2 = 4.0 / (3.0 * DC ** 2) * sum(1 - np.cos(k @ dj) for dj in d)
    return dict(mesh=mesh, m=m, phi=phi, gphi=gphi, kap2=kap2, k=k)


def _project(mo, h, u):
    A = ((h - H) @ mo["phi"]) / (mo["phi"] @ mo["phi"])
    al = (u @ mo["gphi"]) / (mo["gphi"] @ mo["gphi"])
    rh = h - H - A * mo["phi"]
    ru = u - al * mo["gphi"]
    return A, al, np.abs(rh).max(), np.abs(ru).max()


def _lin_params(beta=oracle.BETA):
    return oracle.params(g=G, beta=beta, terms=oracle.T_PGRAD | oracle.T_LINEAR_FLUX, H_lin=H)


def _scalar_fbrk(A, al, a, b, tau, beta, n):
    """FB-RK(3,2) on al' = -a A, A' = b al, written on the 2x2 system."""
    b1, b2, b3 = beta
    for _ in range(n):
        A1 = A + tau / 3 * b * al
        al1 = al - tau / 3 * a * (b1 * A1 + (1 - b1) * A)
        A2 = A + tau / 2 * b * al1
        al2 = al - tau / 2 * a * (b2 * A2 + (1 - b2) * A)
        A3 = A + tau * b * al2
        al3 = al - tau * a * (b3 * A3 + (1 - 2 * b3) * A2 + b3 * A)
        A, al = A3, al3
    return A, al


def test_kappa_tends_to_continuous_wavenumber(mode):
    assert mode["kap2"] == pytest.approx(mode["k"] @ mode["k"], rel=0.2)
    # dispersion relation tends to g H |k|^2 as |k| dc -> 0
    k = mode["k"] / 64
    d = [np.array([DC, 0.0]), np.array([DC / 2, DC * np.sqrt(3) / 2]), np.array([-DC / 2, DC * np.sqrt(3) / 2])]
    kap2 = 4.0 / (3.0 * DC ** 2) * sum(1 - np.cos(k @ dj) for dj in d)
    assert kap2 == pytest.approx(k @ k, rel=1e-4)


def test_linear_mode_follows_closed_form_recursion(mode):
    m = mode["m"]
    w = np.sqrt(G * H * mode["kap2"])
    tau = 1.5 / w
    h0 = H + 0.7 * mode["phi"]
    u0 = 0.2 * mode["gphi"]
    h, u = oracle.fbrk32(m, _lin_params(), h0, u0, tau, 25)
    A, al, rh, ru = _project(mode, h, u)
    Aref, alref = _scalar_fbrk(0.7, 0.2, G, H * mode["kap2"], tau, oracle.BETA, 25)
    assert rh < 1e-14 * H and ru < 1e-11 * abs(alref) * np.abs(mode["gphi"]).max()
    assert A == pytest.approx(Aref, rel=1e-11)
    assert al == pytest.approx(alref, rel=1e-11)
    # below the stability limit the scheme does not amplify the wave energy
    E0 = G * 0.7 ** 2 + H * mode["kap2"] * 0.2 ** 2
    E = G * A ** 2 + H * mode["kap2"] * al ** 2
    assert E < E0


def _stability_limit(mode, beta):
    m = mode["m"]
    w = np.sqrt(G * H * mode["kap2"])
    s = np.sqrt(G / (H * mode["kap2"]))

    def rho(x):
        cols = []
        for A, al in ((1.0, 0.0), (0.0, 1.0)):
            h, u = oracle.fbrk32(m, _lin_params(beta), H + A * mode["phi"], al * s * mode["gphi"], x / w, 1)
            An, aln, _, _ = _project(mode, h, u)
            cols.append([An, aln / s])
        return max(abs(np.linalg.eigvals(np.array(cols).T)))

    lo, hi = 0.5, 6.0
    for _ in range(40):
        mid = 0.5 * (lo + hi)
        if rho(mid) <= 1 + 1e-12:
            lo = mid
        else:
            hi = mid
    return lo


def test_stability_limit_exceeds_rk32(mode):
    ratio = _stability_limit(mode, oracle.BETA) / np.sqrt(3.0)
    assert 2.0 < ratio < 2.4


def test_inertial_oscillation_is_rk3_polynomial():
    mesh = finalize(hex_periodic(12, 12, DC))
    f = 1e-4
    m = oracle.Mesh(mesh, np.zeros(mesh.nCells), np.full(mesh.nVertices, f))
    n = np.stack([np.cos(mesh.angleEdge), np.sin(mesh.angleEdge)], 1)
    U = np.array([0.8, -0.3])
    dt, nsteps = 60.0, 200
    h, u = oracle.fbrk32(m, oracle.params(), np.full(mesh.nCells, H), n @ U, dt, nsteps)
    z = -1j * f * dt
    R = 1 + z + z ** 2 / 2 + z ** 3 / 6
    W = (U[0] + 1j * U[1]) * R ** nsteps
    np.testing.assert_allclose(u, n @ np.array([W.real, W.imag]), atol=1e-12)
    # distinguishable from the exact rotation: the scheme, not the ODE, is pinned
    Wex = (U[0] + 1j * U[1]) * np.exp(z * nsteps)
    assert abs(W - Wex) > 1e-9
    np.testing.assert_allclose(h, H, rtol=1e-15)
    # clockwise rotation for f > 0
    Wp = (U[0] + 1j * U[1]) * R
    assert np.angle(Wp / (U[0] + 1j * U[1])) < 0


def test_fbrk32_and_rk4_convergence_orders(mode):
    m = mode["m"]
    w = np.sqrt(G * H * mode["kap2"])
    T = 20.0 / w
    h0 = H + 0.7 * mode["phi"]
    u0 = np.zeros_like(mode["gphi"])
    p = _lin_params()
    # exact solution of the semi-discrete linear mode
    Aex = 0.7 * np.cos(w * T)
    errs_fb, errs_rk4 = [], []
    for n in (80, 160, 320):
        h, _ = oracle.fbrk32(m, p, h0, u0, T / n, n)
        errs_fb.append(abs(_project(mode, h, np.zeros_like(u0))[0] - Aex))
        h, _ = oracle.rk4(m, p, h0, u0, T / n, n)
        errs_rk4.append(abs(_project(mode, h, np.zeros_like(u0))[0] - Aex))
    o_fb = np.log2(np.array(errs_fb[:-1]) / np.array(errs_fb[1:]))
    o_rk = np.log2(np.array(errs_rk4[:-1]) / np.array(errs_rk4[1:]))
    assert np.all(np.abs(o_fb - 2) < 0.15), o_fb
    assert np.all(np.abs(o_rk - 4) < 0.2), o_rk


def test_bench_rk4_step_ratio_matches_the_oracle_limit(mode):
    """bench.py puts RK4 at 2 sqrt(2) / (FB-RK(3,2)'s linear limit) times the
    FB-RK step; its closed-form limit is the one the oracle's mesh run shows."""
    import bench
    lim = bench.fbrk32_imag_limit(oracle.BETA)
    assert lim == pytest.approx(_stability_limit(mode, oracle.BETA), rel=1e-6)
    assert bench.RK4_IMAG_LIMIT / lim == pytest.approx(0.732, abs=1e-3)
