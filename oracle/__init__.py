"""FB-LTS oracle: a plain, slow FP64 CPU statement of the method (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library.  The arithmetic lives in ``fblts_oracle.c`` (plain C, compiled
without FMA contraction); this module only marshals numpy arrays into it.

Parity status of each function (what pins it; see the tests under
``tests/test_oracle_*``):

* ``psi``, ``phi``, ``vertex_fields``, ``ke``, ``tangential`` - operator
  exactness on regular hexagons for analytic fields, telescoping vorticity,
  Coriolis energy neutrality, inertial oscillation.
* ``fbrk32`` - linear gravity-wave mode against the closed-form 2x2
  recursion, stability-limit ratio against RK(3,2), second-order convergence.
* ``fblts`` - M=1 and single-level reductions (bitwise), mass conservation
  (Theorem 1), shrinking-set vs full-band agreement (bitwise), prediction
  exactness on linear data, second-order convergence against ``rk4``.
* ``rk4`` - fourth-order convergence on the linear mode.
* ``fblts(..., split)`` (Sec. 3.2 splitting; 2: its per-fine-step variant of
  Sec. 4.2) - fast + slow parts add up to Phi, bitwise reductions (no slow
  terms, M = 1, one level), mass conservation, first order against ``rk4``,
  forward-Euler closed forms of the slow Coriolis term on an f-plane.
* forcing terms (wind stress, bottom drag, pressure gradient) - parity
  unpinned beyond closed forms on uniform fields (the paper gives no
  coefficients).
"""
from __future__ import annotations

import ctypes as C
import numpy as np

from . import build as _build

OM_OK, OM_E_ARG, OM_E_REGIONS, OM_E_NAN, OM_E_OOM = 0, 1, 2, 3, 4
T_PGRAD, T_KE, T_CORIOLIS, T_LINEAR_FLUX, T_FORCING = 1, 2, 4, 8, 16
T_FULL = T_PGRAD | T_KE | T_CORIOLIS
RC_FINE, RC_IF1, RC_IF2, RC_INT, RC_OUT = 0, 1, 2, 3, 4
BETA = (0.531, 0.531, 0.313)   # Sec. 2.1: CFL-optimised FB weights
GRAV = 9.80616

_P_I = C.POINTER(C.c_int)
_P_D = C.POINTER(C.c_double)


class _Mesh(C.Structure):
    _fields_ = [("nC", C.c_int), ("nE", C.c_int), ("nV", C.c_int), ("maxE", C.c_int), ("maxE2", C.c_int),
                ("cellsOnEdge", _P_I), ("nEdgesOnCell", _P_I), ("edgesOnCell", _P_I),
                ("verticesOnEdge", _P_I), ("cellsOnVertex", _P_I), ("edgesOnVertex", _P_I),
                ("nEdgesOnEdge", _P_I), ("edgesOnEdge", _P_I), ("weightsOnEdge", _P_D),
                ("dcEdge", _P_D), ("dvEdge", _P_D), ("areaCell", _P_D), ("kiteAreasOnVertex", _P_D),
                ("fVertex", _P_D), ("bottom", _P_D), ("angleEdge", _P_D), ("xCell", _P_D),
                ("yCell", _P_D), ("xEdge", _P_D), ("yEdge", _P_D)]


class Params(C.Structure):
    _fields_ = [("g", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double), ("beta3", C.c_double),
                ("terms", C.c_int), ("H_lin", C.c_double), ("wind_u", C.c_double), ("wind_v", C.c_double),
                ("wind_stress", C.c_int), ("cd", C.c_double), ("rho0", C.c_double), ("rho_air", C.c_double),
                ("vortex", C.c_int), ("vx_pc", C.c_double), ("vx_dp", C.c_double), ("vx_rmax", C.c_double),
                ("vx_B", C.c_double), ("vx_x0", C.c_double), ("vx_y0", C.c_double), ("vx_vx", C.c_double),
                ("vx_vy", C.c_double), ("vx_f0", C.c_double), ("split", C.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        PM, PP = C.POINTER(_Mesh), C.POINTER(Params)
        L.om_psi.argtypes = [PM, PP, _P_D, _P_D, _P_D]
        L.om_phi.argtypes = [PM, PP, _P_D, _P_D, _P_D, _P_D, _P_D, _P_D]
        L.om_vertex_fields.argtypes = [PM, _P_D, _P_D, _P_D, _P_D, _P_D]
        L.om_ke.argtypes = [PM, _P_D, _P_D]
        L.om_tangential.argtypes = [PM, _P_D, _P_D]
        L.om_diagnostics.argtypes = [PM, _P_D, _P_D, _P_D, _P_D]
        L.om_forcing_fields.argtypes = [PM, PP, C.c_double, _P_D, _P_D, _P_D]
        L.om_fbrk32.argtypes = [PM, PP, _P_D, _P_D, C.c_double, C.c_int, C.c_double]
        L.om_rk4.argtypes = [PM, PP, _P_D, _P_D, C.c_double, C.c_int, C.c_double]
        L.om_fblts.argtypes = [PM, PP, _P_I, C.c_int, _P_I, C.c_int, C.c_int, C.c_int, _P_D, _P_D,
                               C.c_double, C.c_int, C.c_double]
        L.om_regions_build.argtypes = [PM, _P_I, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_ubyte), _P_I,
                                       C.POINTER(C.c_ubyte), _P_I]
        L.om_predict.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
                                 _P_D, _P_D, _P_D]
        for f in ("om_fbrk32", "om_rk4", "om_fblts", "om_regions_build"):
            getattr(L, f).restype = C.c_int
        _lib = L
    return _lib


def _pi(a):
    return a.ctypes.data_as(_P_I)


def _pd(a):
    return a.ctypes.data_as(_P_D) if a is not None else None


class Mesh:
    """Oracle view of a synthetic mesh plus bottom and Coriolis fields."""

    def __init__(self, mesh, bottom, fVertex):
        self.src = mesh
        keep = {}

        def I(name):
            a = np.ascontiguousarray(getattr(mesh, name), dtype=np.int32)
            keep[name] = a
            return _pi(a)

        def D(arr, name):
            a = np.ascontiguousarray(arr, dtype=np.float64)
            keep[name] = a
            return _pd(a)

        self.s = _Mesh(mesh.nCells, mesh.nEdges, mesh.nVertices, mesh.maxEdges, mesh.maxEdges2,
                       I("cellsOnEdge"), I("nEdgesOnCell"), I("edgesOnCell"), I("verticesOnEdge"),
                       I("cellsOnVertex"), I("edgesOnVertex"), I("nEdgesOnEdge"), I("edgesOnEdge"),
                       D(mesh.weightsOnEdge, "w"), D(mesh.dcEdge, "dc"), D(mesh.dvEdge, "dv"),
                       D(mesh.areaCell, "A"), D(mesh.kiteAreasOnVertex, "kite"), D(fVertex, "f"),
                       D(bottom, "b"), D(mesh.angleEdge, "ang"), D(mesh.xCell, "xc"), D(mesh.yCell, "yc"),
                       D(mesh.xEdge, "xe"), D(mesh.yEdge, "ye"))
        self._keep = keep
        self.nC, self.nE, self.nV = mesh.nCells, mesh.nEdges, mesh.nVertices

    @classmethod
    def from_scenario(cls, scn):
        return cls(scn.mesh, scn.bottom, scn.fVertex)


def params(g=GRAV, beta=BETA, terms=T_FULL, H_lin=0.0, forcing=None, f0=None, split=False):
    """Oracle parameters; ``forcing`` is a ``synth.scenario.Forcing`` or None;
    ``split`` selects the fast/slow operator splitting of Sec. 3.2 (1 or True), or
    its variant with the slow terms of the finer levels re-evaluated once per
    fine step (2, proposed in Sec. 4.2)."""
    p = Params(g, beta[0], beta[1], beta[2], terms, H_lin, 0.0, 0.0, 0, 0.0, 1025.0, 1.225,
               0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, int(split))
    if forcing is not None and forcing.any:
        p.terms |= T_FORCING
        p.wind_u, p.wind_v = forcing.wind_u, forcing.wind_v
        p.wind_stress = int(forcing.wind_stress)
        p.cd, p.rho0, p.rho_air = forcing.cd, forcing.rho0, forcing.rho_air
        if forcing.vortex is not None:
            p.vortex = 1
            (p.vx_pc, p.vx_dp, p.vx_rmax, p.vx_B, p.vx_x0, p.vx_y0, p.vx_vx, p.vx_vy) = forcing.vortex
            p.vx_f0 = 0.0 if f0 is None else f0
    return p


def _cpy(a):
    return np.ascontiguousarray(a, dtype=np.float64).copy()


def psi(m, p, u, h):
    out = np.empty(m.nC)
    u, h = _cpy(u), _cpy(h)
    lib().om_psi(C.byref(m.s), C.byref(p), _pd(u), _pd(h), _pd(out))
    return out


def phi(m, p, u, h, fields=None):
    out = np.empty(m.nE)
    u, h = _cpy(u), _cpy(h)
    wn = wt = ps = None
    if fields is not None:
        wn, wt, ps = (_cpy(x) for x in fields)
    lib().om_phi(C.byref(m.s), C.byref(p), _pd(wn), _pd(wt), _pd(ps), _pd(u), _pd(h), _pd(out))
    return out


def forcing_fields(m, p, t):
    wn, wt, ps = np.empty(m.nE), np.empty(m.nE), np.empty(m.nC)
    lib().om_forcing_fields(C.byref(m.s), C.byref(p), float(t), _pd(wn), _pd(wt), _pd(ps))
    return wn, wt, ps


def vertex_fields(m, u, h):
    z, hv, q = np.empty(m.nV), np.empty(m.nV), np.empty(m.nV)
    u, h = _cpy(u), _cpy(h)
    lib().om_vertex_fields(C.byref(m.s), _pd(u), _pd(h), _pd(z), _pd(hv), _pd(q))
    return z, hv, q


def ke(m, u):
    K = np.empty(m.nC)
    u = _cpy(u)
    lib().om_ke(C.byref(m.s), _pd(u), _pd(K))
    return K


def tangential(m, u):
    v = np.empty(m.nE)
    u = _cpy(u)
    lib().om_tangential(C.byref(m.s), _pd(u), _pd(v))
    return v


def diagnostics(m, h, u):
    a, b = C.c_double(), C.c_double()
    h, u = _cpy(h), _cpy(u)
    lib().om_diagnostics(C.byref(m.s), _pd(h), _pd(u), C.byref(a), C.byref(b))
    return a.value, b.value


class OracleError(RuntimeError):
    pass


def _check(st, what):
    if st != OM_OK:
        raise OracleError(f"{what}: status {st}")


def fbrk32(m, p, h, u, dt, nsteps, t0=0.0):
    h, u = _cpy(h), _cpy(u)
    _check(lib().om_fbrk32(C.byref(m.s), C.byref(p), _pd(h), _pd(u), float(dt), int(nsteps), float(t0)),
           "fbrk32")
    return h, u


def rk4(m, p, h, u, dt, nsteps, t0=0.0):
    h, u = _cpy(h), _cpy(u)
    _check(lib().om_rk4(C.byref(m.s), C.byref(p), _pd(h), _pd(u), float(dt), int(nsteps), float(t0)), "rk4")
    return h, u


def fblts(m, p, level, M, h, u, dt, nsteps, nIF1=2, nIF2=2, full_band=False, t0=0.0, raise_on_error=True):
    level = np.ascontiguousarray(level, dtype=np.int32)
    L = int(level.max()) + 1 if level.size else 1
    Ma = np.ascontiguousarray(list(M) + [1], dtype=np.int32)
    h, u = _cpy(h), _cpy(u)
    st = lib().om_fblts(C.byref(m.s), C.byref(p), _pi(level), L, _pi(Ma), int(nIF1), int(nIF2),
                        int(bool(full_band)), _pd(h), _pd(u), float(dt), int(nsteps), float(t0))
    if raise_on_error:
        _check(st, "fblts")
        return h, u
    return h, u, st


def predict(k, M, x0, x13, x12, x1):
    """Interface predictions (X^{n,k}, Xbar^{n,k+1/3}, Xbar^{n,k+1/2}) of one IF-1 value."""
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    lib().om_predict(int(k), int(M), float(x0), float(x13), float(x12), float(x1),
                     C.byref(a), C.byref(b), C.byref(c))
    return a.value, b.value, c.value


def regions(m, level, nIF1=2, nIF2=2):
    """Region classes per level pair: (ccls, cdist, ecls, edist, status)."""
    level = np.ascontiguousarray(level, dtype=np.int32)
    L = int(level.max()) + 1
    P = max(L - 1, 1)
    cc = np.zeros((P, m.nC), np.uint8)
    cd = np.zeros((P, m.nC), np.int32)
    ec = np.zeros((P, m.nE), np.uint8)
    ed = np.zeros((P, m.nE), np.int32)
    st = lib().om_regions_build(C.byref(m.s), _pi(level), L, int(nIF1), int(nIF2),
                                cc.ctypes.data_as(C.POINTER(C.c_ubyte)), _pi(cd),
                                ec.ctypes.data_as(C.POINTER(C.c_ubyte)), _pi(ed))
    return cc, cd, ec, ed, st


def scenario_params(scn, terms=T_FULL, beta=BETA, split=False):
    f0 = float(np.mean(scn.fVertex)) if scn.fVertex.size else 0.0
    return params(g=scn.g, beta=beta, terms=terms, forcing=scn.forcing, f0=f0, split=split)


def run_scenario(scn, nsteps, full_band=False, terms=T_FULL):
    m = Mesh.from_scenario(scn)
    p = scenario_params(scn, terms=terms)
    return fblts(m, p, scn.level, scn.M, scn.h0, scn.u0, scn.dt, nsteps, full_band=full_band)
