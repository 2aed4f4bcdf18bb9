"""Serving loop (fblts_server_*) against each request run alone.

Requests on different resident meshes, precisions and durations arrive
while others run; admission is bounded by a device-byte budget.  Each result
must be bitwise the state that fblts_state_init + fblts_lts_advance(n) +
fblts_state_read give for the same request alone.
"""
import time

import numpy as np
import pytest

import paper_2405_10505_gb300 as fb
from synth import scenario
from tests.gpu_util import forcing_flags

pytestmark = pytest.mark.gpu


def _params(s, precision):
    fz = s.forcing
    vt = list(fz.vortex) + [float(np.mean(s.fVertex))] if fz.vortex is not None else None
    return fb.make_params(s.dt, g=s.g, forcing=forcing_flags(s), wind=(fz.wind_u, fz.wind_v), cd=fz.cd,
                          rho0=fz.rho0, rho_air=fz.rho_air, vortex=vt, precision=precision)


def _alone(mesh, s, precision, n):
    st = fb.state_init(mesh, _params(s, precision), s.h0, s.u0, s.bottom)
    fb.lts_advance(st, n)
    out = fb.state_read(st)
    fb.state_destroy(st)
    return out


def test_served_requests_equal_alone_runs():
    cases = [scenario.gaussian_bump_case(two_level=True),
             scenario.shelf_case(nx=64, ny=48, dc=2e3, M=4, width=10e3, vortex=True),
             scenario.jittered_voronoi_case()]
    meshes = [fb.mesh_create(s.mesh, s.fVertex, level=s.level, M=s.M) for s in cases]
    # (case, precision, steps): uneven durations, both precisions
    reqs = [(0, fb.FP32_TENDENCY, 7), (1, fb.FP32_TENDENCY, 5), (2, fb.FP32_TENDENCY, 9),
            (1, fb.FP64, 4), (0, fb.FP64, 6), (2, fb.FP32_TENDENCY, 3), (1, fb.FP32_TENDENCY, 8)]
    sizes = [fb.state_device_bytes(meshes[c], p) for c, p, _ in reqs]
    budget = int(2.5 * max(sizes))
    srv = fb.server_create(hbm_budget=budget, steps_per_issue=2)
    ids = []
    for c, p, n in reqs[:4]:
        ids.append(fb.server_submit(srv, meshes[c], _params(cases[c], p), cases[c].h0, cases[c].u0,
                                    cases[c].bottom, n))
    for _ in range(3):
        fb.server_progress(srv)
    for c, p, n in reqs[4:]:            # arrivals while others run
        ids.append(fb.server_submit(srv, meshes[c], _params(cases[c], p), cases[c].h0, cases[c].u0,
                                    cases[c].bottom, n))
    results = {}
    t0 = time.time()
    while len(results) < len(ids):
        assert time.time() - t0 < 120
        fb.server_progress(srv)
        st = fb.server_stats(srv)
        assert st.device_bytes_in_use <= budget
        for rid in ids:
            if rid not in results and fb.server_request_info(srv, rid).status == fb.REQ_DONE:
                results[rid] = fb.server_take(srv, rid)
    st = fb.server_stats(srv)
    assert st.finished == len(ids) and st.queued == 0 and st.running == 0
    assert st.max_running >= 2 and st.device_bytes_peak <= budget
    for rid, (c, p, n) in zip(ids, reqs):
        info = fb.server_request_info(srv, rid)
        assert info.status == fb.REQ_TAKEN and info.steps_done == n
        assert info.t_submit <= info.t_admit <= info.t_done
        h0, u0 = _alone(meshes[c], cases[c], p, n)
        h, u = results[rid]
        assert np.array_equal(h, h0) and np.array_equal(u, u0)
    fb.server_destroy(srv)


def test_server_rejects_what_can_never_fit():
    s = scenario.gaussian_bump_case(two_level=True)
    mesh = fb.mesh_create(s.mesh, s.fVertex, level=s.level, M=s.M)
    need = fb.state_device_bytes(mesh, fb.FP32_TENDENCY)
    srv = fb.server_create(hbm_budget=need - 1)
    with pytest.raises(fb.FbltsError):
        fb.server_submit(srv, mesh, _params(s, fb.FP32_TENDENCY), s.h0, s.u0, s.bottom, 3)
    fb.server_destroy(srv)


def test_served_split_and_rk4_requests_equal_alone_runs():
    """Requests with the operator splitting (both variants) and RK4 beside plain
    ones share the device and each comes out bitwise as its alone run."""
    bump = scenario.gaussian_bump_case(two_level=True)
    one = np.zeros(bump.mesh.nCells, np.int32)
    m2 = fb.mesh_create(bump.mesh, bump.fVertex, level=bump.level, M=bump.M)
    m1 = fb.mesh_create(bump.mesh, bump.fVertex, level=one, M=[])
    kinds = [(m2, dict(split=1), 6), (m2, dict(split=2), 5), (m1, dict(scheme=fb.SCHEME_RK4), 7), (m2, {}, 4)]

    def params(kw, precision):
        p = _params(bump, precision)
        p.split = kw.get("split", 0)
        p.scheme = kw.get("scheme", fb.SCHEME_FBLTS)
        return p

    srv = fb.server_create(hbm_budget=0, steps_per_issue=1)
    ids, want = [], []
    for mesh, kw, n in kinds:
        for precision in (fb.FP64, fb.FP32_TENDENCY):
            ids.append(fb.server_submit(srv, mesh, params(kw, precision), bump.h0, bump.u0, bump.bottom, n))
            st = fb.state_init(mesh, params(kw, precision), bump.h0, bump.u0, bump.bottom)
            fb.lts_advance(st, n)
            want.append(fb.state_read(st))
            fb.state_destroy(st)
    results = {}
    t0 = time.time()
    while len(results) < len(ids):
        assert time.time() - t0 < 120
        fb.server_progress(srv)
        for rid in ids:
            if rid not in results and fb.server_request_info(srv, rid).status == fb.REQ_DONE:
                results[rid] = fb.server_take(srv, rid)
    assert fb.server_stats(srv).max_running >= 2
    for rid, (h0, u0) in zip(ids, want):
        h, u = results[rid]
        assert np.array_equal(h, h0) and np.array_equal(u, u0)
    fb.server_destroy(srv)


def test_served_requests_match_oracle():
    """Served requests of 100 coarse steps in both precisions, overlapping on
    the device, against the FP64 oracle's FB-LTS run of each scenario
    (Sec. 2.2): FP64 within 1e-10, FP32 tendencies within 1e-6 (h) and 1e-5
    (u)."""
    import oracle
    from tests.gpu_util import rel_errors
    cases = [scenario.gaussian_bump_case(two_level=True),
             scenario.shelf_case(nx=64, ny=48, dc=2e3, M=4, width=10e3, vortex=True),
             scenario.jittered_voronoi_case(),
             scenario.nested_disk_case(nx=64, ny=64, radii=(190e3, 50e3))]
    n = 100
    meshes = [fb.mesh_create(s.mesh, s.fVertex, level=s.level, M=s.M) for s in cases]
    srv = fb.server_create(hbm_budget=0, max_active=4, steps_per_issue=3)
    reqs = [(c, p) for c in range(len(cases)) for p in (fb.FP32_TENDENCY, fb.FP64)]
    ids = [fb.server_submit(srv, meshes[c], _params(cases[c], p), cases[c].h0, cases[c].u0, cases[c].bottom, n)
           for c, p in reqs]
    results = {}
    t0 = time.time()
    while len(results) < len(ids):
        assert time.time() - t0 < 300
        fb.server_progress(srv)
        for rid in ids:
            if rid not in results and fb.server_request_info(srv, rid).status == fb.REQ_DONE:
                results[rid] = fb.server_take(srv, rid)
    assert fb.server_stats(srv).max_running >= 2
    ref = {c: oracle.fblts(oracle.Mesh.from_scenario(s), oracle.scenario_params(s), s.level, s.M, s.h0, s.u0,
                           s.dt, n) for c, s in enumerate(cases)}
    for rid, (c, p) in zip(ids, reqs):
        h, u = results[rid]
        dh, du = rel_errors(h, u, *ref[c])
        tol_h, tol_u = (1e-10, 1e-10) if p == fb.FP64 else (1e-6, 1e-5)
        assert dh <= tol_h and du <= tol_u, (cases[c].name, p, dh, du)
    fb.server_destroy(srv)
