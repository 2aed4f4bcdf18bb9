"""Helpers shared by the GPU tests: run a synthetic scenario through the C ABI."""
import numpy as np

import paper_2405_10505_gb300 as fb


def forcing_flags(s):
    fz = s.forcing
    flags = 0
    if fz.wind_stress:
        flags |= fb.FORCE_WIND_STRESS
    if fz.cd:
        flags |= fb.FORCE_BOTTOM_DRAG
    if fz.vortex is not None:
        flags |= fb.FORCE_VORTEX
    return flags


def make_state(s, M=None, level=None, use_graph=True, precision=fb.FP64, mesh=None, split=False,
               scheme=fb.SCHEME_FBLTS, dt=None):
    lev = s.level if level is None else level
    Ms = s.M if M is None else M
    mesh = mesh or fb.mesh_create(s.mesh, s.fVertex, level=lev, M=Ms)
    fz = s.forcing
    vt = list(fz.vortex) + [float(np.mean(s.fVertex))] if fz.vortex is not None else None
    p = fb.make_params(s.dt if dt is None else dt, g=s.g, forcing=forcing_flags(s), wind=(fz.wind_u, fz.wind_v), cd=fz.cd,
                       rho0=fz.rho0, rho_air=fz.rho_air, vortex=vt, use_graph=use_graph, precision=precision,
                       split=split, scheme=scheme)
    return fb.state_init(mesh, p, s.h0, s.u0, s.bottom)


def rel_errors(h, u, ho, uo):
    dh = float(np.max(np.abs(h - ho) / np.abs(ho)))
    du = float(np.max(np.abs(u - uo)) / max(float(np.max(np.abs(uo))), 1e-300))
    return dh, du
