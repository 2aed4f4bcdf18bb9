"""Python binding of the GB300 FB-LTS library (include/fblts.h).

Argument marshalling only: every step of the time integration runs in the
CUDA library ``_build/libfblts.so`` (built by :mod:`.build` for sm_103a).  There
is no CPU fallback: if the library cannot be built or loaded, every call
raises.

The functions carry the names of the C entry points without the ``fblts_``
prefix; handles are opaque ``ctypes`` pointers wrapped in :class:`Mesh` and
:class:`State`.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

OK, E_ARG, E_MESH, E_REGIONS, E_OOM, E_CUDA, E_UNSTABLE, E_TIMEOUT, E_STATE = range(9)
FP64, FP32_TENDENCY = 0, 1
REGION_FINE, REGION_IF1, REGION_IF2, REGION_INTERIOR, REGION_OUTSIDE = range(5)
(SEG_NONE, SEG_STAGE, SEG_IN_PLACE, SEG_SUM_SET, SEG_SUM_ADD, SEG_KE_ONLY, SEG_TENDENCY, SEG_RK4_SET,
 SEG_RK4_ADD2, SEG_RK4_FINAL) = range(10)
SCHEME_FBLTS, SCHEME_RK4 = 0, 1
FORCE_WIND_STRESS, FORCE_BOTTOM_DRAG, FORCE_VORTEX = 1, 2, 4
MESH_PROMOTE_LEVELS = 1
PAPER_BETA = (0.531, 0.531, 0.313)   # Sec. 2.1, CFL-optimised FB weights

_PI = C.POINTER(C.c_int32)
_PD = C.POINTER(C.c_double)


class MeshDesc(C.Structure):
    _fields_ = [("nCells", C.c_int32), ("nEdges", C.c_int32), ("nVertices", C.c_int32),
                ("maxEdges", C.c_int32), ("maxEdges2", C.c_int32),
                ("cellsOnEdge", _PI), ("nEdgesOnCell", _PI), ("edgesOnCell", _PI),
                ("verticesOnEdge", _PI), ("cellsOnVertex", _PI), ("edgesOnVertex", _PI),
                ("nEdgesOnEdge", _PI), ("edgesOnEdge", _PI), ("weightsOnEdge", _PD),
                ("dcEdge", _PD), ("dvEdge", _PD), ("areaCell", _PD), ("kiteAreasOnVertex", _PD),
                ("fVertex", _PD), ("angleEdge", _PD), ("xCell", _PD), ("yCell", _PD),
                ("xEdge", _PD), ("yEdge", _PD), ("ltsLevel", _PI), ("nLevels", C.c_int32),
                ("M", _PI), ("nIF1Layers", C.c_int32), ("nIF2Layers", C.c_int32), ("flags", C.c_int32)]


class MeshInfo(C.Structure):
    _fields_ = [("nCells", C.c_int32), ("nEdges", C.c_int32), ("nVertices", C.c_int32),
                ("nLevels", C.c_int32), ("cells_per_level", C.c_int64 * 8),
                ("cell_updates_per_step", C.c_int64), ("band_cells", C.c_int64 * 8), ("flags", C.c_int32)]


class Params(C.Structure):
    _fields_ = [("g", C.c_double), ("dt", C.c_double), ("beta", C.c_double * 3),
                ("precision", C.c_int32), ("forcing", C.c_int32), ("wind_u", C.c_double),
                ("wind_v", C.c_double), ("cd", C.c_double), ("rho0", C.c_double),
                ("rho_air", C.c_double), ("vortex", C.c_double * 9), ("t0", C.c_double),
                ("stream", C.c_void_p), ("use_graph", C.c_int32), ("split", C.c_int32), ("scheme", C.c_int32)]


class FbltsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"fblts status {status}: {msg}")
        self.status = status


class BatchOpts(C.Structure):
    _fields_ = [("autotune", C.c_int32), ("threads_per_block", C.c_int32), ("ctas_per_sm", C.c_int32),
                ("tile_order", C.c_int32), ("mode", C.c_int32), ("stream", C.c_void_p)]


class BatchInfo(C.Structure):
    _fields_ = [("members", C.c_int32), ("groups", C.c_int32), ("threads_per_block", C.c_int32),
                ("ctas_per_sm", C.c_int32),
                ("tile_order", C.c_int32), ("mode", C.c_int32), ("tuned", C.c_int32),
                ("launches_per_round", C.c_int64),
                ("member_launches_per_round", C.c_int64), ("cell_updates_per_round", C.c_int64),
                ("rounds", C.c_int64), ("n_candidates", C.c_int32), ("candidate_ms", C.c_float * 16)]


class ServerOpts(C.Structure):
    _fields_ = [("hbm_budget", C.c_uint64), ("max_active", C.c_int32), ("steps_per_issue", C.c_int32)]


class RequestDesc(C.Structure):
    _fields_ = [("mesh", C.c_void_p), ("params", Params), ("h0", C.POINTER(C.c_double)),
                ("u0", C.POINTER(C.c_double)), ("bottom", C.POINTER(C.c_double)), ("n_steps", C.c_int64)]


class RequestInfo(C.Structure):
    _fields_ = [("status", C.c_int32), ("error", C.c_int32), ("steps_done", C.c_int64), ("n_steps", C.c_int64),
                ("device_bytes", C.c_uint64), ("t_submit", C.c_double), ("t_admit", C.c_double),
                ("t_done", C.c_double)]


class ServerStats(C.Structure):
    _fields_ = [("queued", C.c_int64), ("running", C.c_int64), ("finished", C.c_int64), ("max_running", C.c_int64),
                ("device_bytes_in_use", C.c_uint64), ("device_bytes_peak", C.c_uint64),
                ("cell_updates", C.c_int64), ("t_now", C.c_double)]


REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED, REQ_TAKEN = range(5)

_LIB = None
SYMBOLS = ("fblts_last_error", "fblts_mesh_create", "fblts_mesh_destroy", "fblts_mesh_get_info", "fblts_mesh_regions",
           "fblts_mesh_levels",
           "fblts_plan_step", "fblts_plan_op", "fblts_plan_op_bytes",
           "fblts_state_init", "fblts_state_destroy", "fblts_lts_advance", "fblts_synchronize",
           "fblts_state_read", "fblts_state_write", "fblts_run_host", "fblts_diagnostics",
           "fblts_state_time", "fblts_state_save", "fblts_state_load", "fblts_state_launches_per_step",
           "fblts_state_profile_step", "fblts_state_step_bytes", "fblts_state_bytes_by_kind",
           "fblts_diagnostics_static",
           "fblts_state_device_bytes", "fblts_batch_create", "fblts_batch_advance", "fblts_batch_synchronize", "fblts_batch_get_info",
           "fblts_batch_destroy", "fblts_server_create", "fblts_server_submit", "fblts_server_progress",
           "fblts_server_request_info", "fblts_server_take", "fblts_server_get_stats", "fblts_server_destroy")
PROFILE_KINDS = ("cell", "vertex", "edge_prep", "edge", "save", "predict", "correct", "forcing", "step_end",
                 "trisk")


def library_path():
    return _build.LIB


def lib():
    """Load (building first if stale) the CUDA library; raises if impossible."""
    global _LIB
    if _LIB is None:
        path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library missing: {path}")
        L = C.CDLL(path)
        L.fblts_last_error.restype = C.c_char_p
        V = C.c_void_p
        sig = {
            "fblts_mesh_create": [C.POINTER(MeshDesc), C.POINTER(V)],
            "fblts_mesh_destroy": [V],
            "fblts_mesh_get_info": [V, C.POINTER(MeshInfo)],
            "fblts_mesh_levels": [V, _PI],
            "fblts_mesh_regions": [C.POINTER(MeshDesc), C.c_int32, _PI, _PI, _PI, _PI],
            "fblts_plan_step": [C.POINTER(MeshDesc), C.POINTER(Params), C.POINTER(C.c_int64), _PD,
                                C.POINTER(C.c_int64)],
            "fblts_plan_op": [C.POINTER(MeshDesc), C.POINTER(Params), C.c_int64, C.POINTER(C.c_int32),
                              C.POINTER(C.c_int32), C.POINTER(C.c_uint8)],
            "fblts_plan_op_bytes": [C.POINTER(MeshDesc), C.POINTER(Params), C.c_int64, _PD, _PD],
            "fblts_state_init": [V, C.POINTER(Params), _PD, _PD, _PD, C.POINTER(V)],
            "fblts_state_destroy": [V],
            "fblts_lts_advance": [V, C.c_int64],
            "fblts_synchronize": [V],
            "fblts_state_read": [V, _PD, _PD],
            "fblts_state_write": [V, _PD, _PD],
            "fblts_run_host": [V, _PD, _PD, C.c_int64, _PD, _PD],
            "fblts_diagnostics": [V, _PD, _PD],
            "fblts_state_time": [V, C.POINTER(C.c_int64), _PD],
            "fblts_state_save": [V, V, C.POINTER(C.c_size_t)],
            "fblts_state_load": [V, V, C.c_size_t],
            "fblts_state_launches_per_step": [V, C.POINTER(C.c_int64)],
            "fblts_state_profile_step": [V, _PD, C.POINTER(C.c_int64), _PD],
            "fblts_state_step_bytes": [V, _PD, C.POINTER(C.c_int64)],
            "fblts_state_bytes_by_kind": [V, _PD, _PD],
            "fblts_diagnostics_static": [V, V, V, V, V],
            "fblts_state_device_bytes": [V, C.c_int32, C.POINTER(C.c_size_t)],
            "fblts_batch_create": [C.POINTER(V), C.c_int32, C.POINTER(BatchOpts), C.POINTER(V)],
            "fblts_batch_advance": [V, C.c_int64],
            "fblts_batch_synchronize": [V],
            "fblts_batch_get_info": [V, C.POINTER(BatchInfo)],
            "fblts_batch_destroy": [V],
            "fblts_server_create": [C.POINTER(ServerOpts), C.POINTER(V)],
            "fblts_server_submit": [V, C.POINTER(RequestDesc), C.POINTER(C.c_int64)],
            "fblts_server_progress": [V, C.POINTER(C.c_int32)],
            "fblts_server_request_info": [V, C.c_int64, C.POINTER(RequestInfo)],
            "fblts_server_take": [V, C.c_int64, _PD, _PD],
            "fblts_server_get_stats": [V, C.POINTER(ServerStats)],
            "fblts_server_destroy": [V],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        _LIB = L
    return _LIB


def last_error():
    return lib().fblts_last_error().decode()


def _check(status):
    if status != OK:
        raise FbltsError(status, last_error())


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a, t):
    return None if a is None else a.ctypes.data_as(t)


class Mesh:
    """Handle of a created mesh (owns the device metadata)."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep

    def info(self):
        return mesh_get_info(self)

    def close(self):
        if self.handle:
            mesh_destroy(self)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class State:
    """Handle of a device state; keeps its mesh alive."""

    def __init__(self, handle, mesh):
        self.handle = handle
        self.mesh = mesh

    def close(self):
        if self.handle:
            state_destroy(self)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mesh_create(m, fVertex, level=None, M=None, nIF1=0, nIF2=0, promote=False):
    """fblts_mesh_create from MPAS-named arrays on ``m`` (any object with those
    attributes); ``promote`` sets FBLTS_MESH_PROMOTE_LEVELS (the library then
    separates the levels itself; ``mesh_levels`` returns the levels in use)."""
    d, keep = _mesh_desc(m, fVertex, level, M, nIF1, nIF2, promote)
    h = C.c_void_p()
    _check(lib().fblts_mesh_create(C.byref(d), C.byref(h)))
    return Mesh(h, keep)


def mesh_regions(m, fVertex, level, M, pair, nIF1=0, nIF2=0, promote=False):
    """fblts_mesh_regions (host only): per cell and per edge, caller order, the
    region class of the level pair (pair, pair + 1) and the F^b band."""
    d, keep = _mesh_desc(m, fVertex, level, M, nIF1, nIF2, promote)
    cc = np.empty(int(m.nCells), np.int32)
    cb = np.empty(int(m.nCells), np.int32)
    ec = np.empty(int(m.nEdges), np.int32)
    eb = np.empty(int(m.nEdges), np.int32)
    _check(lib().fblts_mesh_regions(C.byref(d), int(pair), _p(cc, _PI), _p(cb, _PI), _p(ec, _PI), _p(eb, _PI)))
    return cc, cb, ec, eb


def plan_step(m, fVertex, level, M, params, nIF1=0, nIF2=0, promote=False):
    """fblts_plan_step (host only): (launches, algorithmic bytes, cell-updates)
    of one coarse step for these parameters."""
    d, keep = _mesh_desc(m, fVertex, level, M, nIF1, nIF2, promote)
    n, cu = C.c_int64(), C.c_int64()
    b = C.c_double()
    _check(lib().fblts_plan_step(C.byref(d), C.byref(params), C.byref(n), C.byref(b), C.byref(cu)))
    return int(n.value), float(b.value), int(cu.value)


def plan_op(m, fVertex, level, M, params, index, nIF1=0, nIF2=0):
    """fblts_plan_op (host only): (kind name, stage, per-element segment modes in
    caller order, or None for kinds that are not passes over cells, vertices or
    edges) of op ``index`` of the coarse step's launch list."""
    d, keep = _mesh_desc(m, fVertex, level, M, nIF1, nIF2)
    k, st = C.c_int32(), C.c_int32()
    buf = np.zeros(max(int(m.nCells), int(m.nEdges), int(m.nVertices)), np.uint8)
    _check(lib().fblts_plan_op(C.byref(d), C.byref(params), int(index), C.byref(k), C.byref(st),
                               buf.ctypes.data_as(C.POINTER(C.c_uint8))))
    name = PROFILE_KINDS[k.value]
    n = {"cell": m.nCells, "trisk": m.nCells, "vertex": m.nVertices, "edge": m.nEdges,
         "edge_prep": m.nEdges}.get(name)
    return name, int(st.value), (buf[: int(n)].copy() if n is not None else None)


def plan_op_bytes(m, fVertex, level, M, params, index, nIF1=0, nIF2=0):
    """fblts_plan_op_bytes (host only): (algorithmic, moved) bytes of op ``index``."""
    d, keep = _mesh_desc(m, fVertex, level, M, nIF1, nIF2)
    a, mv = C.c_double(), C.c_double()
    _check(lib().fblts_plan_op_bytes(C.byref(d), C.byref(params), int(index), C.byref(a), C.byref(mv)))
    return float(a.value), float(mv.value)


def _mesh_desc(m, fVertex, level, M, nIF1, nIF2, promote=False):
    keep = {}

    def I(name, arr=None):
        a = _i32(getattr(m, name) if arr is None else arr)
        keep[name] = a
        return _p(a, _PI)

    def D(name, arr=None, optional=False):
        src = getattr(m, name, None) if arr is None else arr
        if src is None:
            if optional:
                return None
            raise ValueError(f"mesh array {name} missing")
        a = _f64(src)
        keep[name] = a
        return _p(a, _PD)

    nL = 1
    lev_p = M_p = None
    if level is not None:
        lev = _i32(level)
        nL = int(lev.max()) + 1 if lev.size else 1
        keep["level"] = lev
        lev_p = _p(lev, _PI)
        Ma = _i32(list(M or []) + [1])
        keep["M"] = Ma
        M_p = _p(Ma, _PI)
    eov = getattr(m, "edgesOnVertex", None)
    d = MeshDesc(int(m.nCells), int(m.nEdges), int(m.nVertices), int(m.maxEdges), int(m.maxEdges2),
                 I("cellsOnEdge"), I("nEdgesOnCell"), I("edgesOnCell"), I("verticesOnEdge"),
                 I("cellsOnVertex"), I("edgesOnVertex") if eov is not None else None,
                 I("nEdgesOnEdge"), I("edgesOnEdge"), D("weightsOnEdge"), D("dcEdge"), D("dvEdge"),
                 D("areaCell"), D("kiteAreasOnVertex"), D("fVertex", fVertex),
                 D("angleEdge", optional=True), D("xCell", optional=True), D("yCell", optional=True),
                 D("xEdge", optional=True), D("yEdge", optional=True), lev_p, nL, M_p, int(nIF1), int(nIF2),
                 MESH_PROMOTE_LEVELS if promote else 0)
    keep["desc"] = d
    return d, keep


def mesh_destroy(mesh):
    """fblts_mesh_destroy; raises (and keeps the handle) while states or server
    requests still use the mesh."""
    h = mesh.handle
    if h:
        _check(lib().fblts_mesh_destroy(h))
        mesh.handle = None


def mesh_levels(mesh):
    """fblts_mesh_levels: the LTS level of every cell (caller order) in use."""
    info = mesh_get_info(mesh)
    out = np.empty(int(info.nCells), np.int32)
    _check(lib().fblts_mesh_levels(mesh.handle, _p(out, _PI)))
    return out


def mesh_get_info(mesh):
    info = MeshInfo()
    _check(lib().fblts_mesh_get_info(mesh.handle, C.byref(info)))
    return info


def make_params(dt, g=9.80616, beta=PAPER_BETA, precision=FP64, forcing=0, wind=(0.0, 0.0), cd=0.0,
                rho0=1025.0, rho_air=1.225, vortex=None, t0=0.0, stream=None, use_graph=True, split=False,
                scheme=0):
    p = Params()
    p.g, p.dt = g, dt
    p.beta[:] = list(beta)
    p.precision, p.forcing = precision, forcing
    p.wind_u, p.wind_v = wind
    p.cd, p.rho0, p.rho_air = cd, rho0, rho_air
    if vortex is not None:
        p.vortex[:] = list(vortex)
    p.t0 = t0
    p.stream = stream
    p.use_graph = int(bool(use_graph))
    p.split = int(split)   # False/True -> 0/1; 2: slow terms per step of every finer level
    p.scheme = int(scheme)
    return p


def state_init(mesh, params, h0, u0, bottom):
    h0, u0, bottom = _f64(h0), _f64(u0), _f64(bottom)
    h = C.c_void_p()
    _check(lib().fblts_state_init(mesh.handle, C.byref(params), _p(h0, _PD), _p(u0, _PD), _p(bottom, _PD),
                                  C.byref(h)))
    return State(h, mesh)


def state_destroy(state):
    h, state.handle = state.handle, None
    if h:
        _check(lib().fblts_state_destroy(h))


def lts_advance(state, n):
    _check(lib().fblts_lts_advance(state.handle, int(n)))


def synchronize(state):
    _check(lib().fblts_synchronize(state.handle))


def state_read(state, h_out=None, u_out=None):
    info = state.mesh.info()
    h = np.empty(info.nCells) if h_out is None else h_out
    u = np.empty(info.nEdges) if u_out is None else u_out
    _check(lib().fblts_state_read(state.handle, _p(h, _PD), _p(u, _PD)))
    return h, u


def state_write(state, h=None, u=None):
    h = None if h is None else _f64(h)
    u = None if u is None else _f64(u)
    _check(lib().fblts_state_write(state.handle, _p(h, _PD), _p(u, _PD)))


def run_host(state, h_in, u_in, n, h_out, u_out):
    """End-to-end call on host buffers (numpy arrays, ideally pinned)."""
    _check(lib().fblts_run_host(state.handle, _p(h_in, _PD), _p(u_in, _PD), int(n), _p(h_out, _PD),
                                _p(u_out, _PD)))


def diagnostics(state):
    a, b = C.c_double(), C.c_double()
    _check(lib().fblts_diagnostics(state.handle, C.byref(a), C.byref(b)))
    return a.value, b.value


def state_time(state):
    n, t = C.c_int64(), C.c_double()
    _check(lib().fblts_state_time(state.handle, C.byref(n), C.byref(t)))
    return n.value, t.value


def state_save(state):
    n = C.c_size_t(0)
    _check(lib().fblts_state_save(state.handle, None, C.byref(n)))
    buf = C.create_string_buffer(n.value)
    _check(lib().fblts_state_save(state.handle, buf, C.byref(n)))
    return bytes(buf.raw[: n.value])


def state_load(state, blob):
    buf = C.create_string_buffer(blob, len(blob))
    _check(lib().fblts_state_load(state.handle, buf, len(blob)))


def state_device_bytes(mesh, precision):
    n = C.c_size_t()
    _check(lib().fblts_state_device_bytes(mesh.handle, int(precision), C.byref(n)))
    return n.value


def launches_per_step(state):
    n = C.c_int64()
    _check(lib().fblts_state_launches_per_step(state.handle, C.byref(n)))
    return n.value


def state_profile_step(state):
    """Per-kind (ms, launches, algorithmic bytes) of one coarse step, issued launch by launch."""
    k = len(PROFILE_KINDS)
    ms = (C.c_double * k)()
    nl = (C.c_int64 * k)()
    by = (C.c_double * k)()
    _check(lib().fblts_state_profile_step(state.handle, ms, nl, by))
    return {PROFILE_KINDS[i]: (ms[i], nl[i], by[i]) for i in range(k)}


def state_step_bytes(state):
    b, cu = C.c_double(), C.c_int64()
    _check(lib().fblts_state_step_bytes(state.handle, C.byref(b), C.byref(cu)))
    return b.value, cu.value


def state_bytes_by_kind(state):
    """Per-kind (algorithmic bytes, moved bytes) of one coarse step."""
    k = len(PROFILE_KINDS)
    alg = (C.c_double * k)()
    moved = (C.c_double * k)()
    _check(lib().fblts_state_bytes_by_kind(state.handle, alg, moved))
    return {PROFILE_KINDS[i]: (alg[i], moved[i]) for i in range(k)}


def diagnostics_static(mesh, d_h, d_u, d_out, stream=None):
    """Allocation-free diagnostics on caller-order device arrays (raw device pointers).

    Writes (mass, absolute vorticity) to the device array at ``d_out`` on
    ``stream`` without waiting; see ``fblts_diagnostics_static``.
    """
    _check(lib().fblts_diagnostics_static(mesh.handle, C.c_void_p(d_h), C.c_void_p(d_u), C.c_void_p(d_out),
                                          None if stream is None else C.c_void_p(stream)))


class Batch:
    """Handle of a batched ensemble; keeps its member states alive."""

    def __init__(self, handle, members):
        self.handle = handle
        self.members = list(members)

    def close(self):
        if self.handle:
            batch_destroy(self)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_create(states, autotune=True, threads_per_block=0, ctas_per_sm=0, tile_order=0, mode=0, stream=None):
    """fblts_batch_create over FP32-tendency states on meshes with cell rows."""
    arr = (C.c_void_p * len(states))(*[s.handle for s in states])
    o = BatchOpts(int(bool(autotune)), int(threads_per_block), int(ctas_per_sm), int(tile_order), int(mode), stream)
    h = C.c_void_p()
    _check(lib().fblts_batch_create(arr, len(states), C.byref(o), C.byref(h)))
    return Batch(h, states)


def batch_advance(batch, n):
    _check(lib().fblts_batch_advance(batch.handle, int(n)))


def batch_synchronize(batch):
    _check(lib().fblts_batch_synchronize(batch.handle))


def batch_info(batch):
    info = BatchInfo()
    _check(lib().fblts_batch_get_info(batch.handle, C.byref(info)))
    return info


def batch_destroy(batch):
    h, batch.handle = batch.handle, None
    if h:
        _check(lib().fblts_batch_destroy(h))


class Server:
    """Handle of a serving loop; keeps the submitted meshes and input arrays
    alive until their requests are admitted."""

    def __init__(self, handle):
        self.handle = handle
        self._inputs = {}

    def close(self):
        if self.handle:
            server_destroy(self)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def server_create(hbm_budget=0, max_active=0, steps_per_issue=1):
    o = ServerOpts(int(hbm_budget), int(max_active), int(steps_per_issue))
    h = C.c_void_p()
    _check(lib().fblts_server_create(C.byref(o), C.byref(h)))
    return Server(h)


def server_submit(server, mesh, params, h0, u0, bottom, n_steps):
    """Queues a request; returns its id."""
    h0, u0, bottom = _f64(h0), _f64(u0), _f64(bottom)
    d = RequestDesc(mesh.handle, params, _p(h0, _PD), _p(u0, _PD), _p(bottom, _PD), int(n_steps))
    rid = C.c_int64()
    _check(lib().fblts_server_submit(server.handle, C.byref(d), C.byref(rid)))
    server._inputs[rid.value] = (mesh, h0, u0, bottom)
    return rid.value


def server_progress(server):
    n = C.c_int32()
    _check(lib().fblts_server_progress(server.handle, C.byref(n)))
    return n.value


def server_request_info(server, rid):
    info = RequestInfo()
    _check(lib().fblts_server_request_info(server.handle, int(rid), C.byref(info)))
    return info


def server_take(server, rid, read=True):
    """A finished request's (h, u) in caller order (None, None without read); frees its state."""
    mesh = server._inputs[rid][0]
    info = mesh.info()
    h = np.empty(info.nCells) if read else None
    u = np.empty(info.nEdges) if read else None
    try:
        _check(lib().fblts_server_take(server.handle, int(rid), _p(h, _PD), _p(u, _PD)))
    finally:
        server._inputs.pop(rid, None)
    return h, u


def server_stats(server):
    s = ServerStats()
    _check(lib().fblts_server_get_stats(server.handle, C.byref(s)))
    return s


def server_destroy(server):
    h, server.handle = server.handle, None
    if h:
        _check(lib().fblts_server_destroy(h))
