"""Seeded synthetic workloads shaped like the paper's test cases.

Each builder returns a :class:`Scenario`: a mesh (MPAS arrays), the bottom
``b = -H`` per cell, the Coriolis parameter per vertex, an initial state
``(h0, u0)``, an LTS level per cell (0 = coarsest), the refinement factors
``M`` between adjacent levels, the coarse time step and the forcing switches.
Only input generation happens here: no tendency or time-stepping arithmetic.

Default seed 2405 everywhere; every random draw goes through
``numpy.random.Generator(PCG64(seed))``.
"""
from __future__ import annotations

import dataclasses
import numpy as np

from .mesh import hex_periodic, apply_cell_mask, finalize, SQRT3

G = 9.80616


@dataclasses.dataclass
class Forcing:
    """Forcing switches and coefficients (all off by default).

    Wind and surface pressure are evaluated once per coarse step at its
    start time and held over all stages and subcycles; bottom drag follows
    the state.  ``vortex`` is a Holland-type pressure/wind vortex moving on a
    straight track: (pc, dp, rmax, B, x0, y0, vx, vy).
    """
    wind_u: float = 0.0
    wind_v: float = 0.0
    cd: float = 0.0            # quadratic bottom-drag coefficient C_D
    wind_stress: bool = False  # C_W |u_W - u| (u_W - u) / h
    rho0: float = 1025.0
    rho_air: float = 1.225
    vortex: tuple | None = None

    @property
    def any(self):
        return self.wind_stress or self.cd != 0.0 or self.vortex is not None


@dataclasses.dataclass
class Scenario:
    name: str
    mesh: object
    bottom: np.ndarray       # b = -H per cell
    fVertex: np.ndarray
    h0: np.ndarray
    u0: np.ndarray
    level: np.ndarray        # int32 per cell, 0 = coarsest
    M: list
    dt: float
    g: float = G
    forcing: Forcing = dataclasses.field(default_factory=Forcing)

    @property
    def nLevels(self):
        return int(self.level.max()) + 1 if self.level.size else 1


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _min_image(dx, L):
    return dx - L * np.round(dx / L)


def cell_neighbours(mesh):
    """(nCells, maxEdges) neighbour cells, -1 where absent."""
    return mesh.cellsOnCell


def graph_dilate(mesh, mask, iters=1):
    nb = mesh.cellsOnCell
    out = mask.copy()
    for _ in range(iters):
        m2 = out.copy()
        valid = nb >= 0
        m2 |= (out[np.where(valid, nb, 0)] & valid).any(1)
        out = m2
    return out


def graph_erode(mesh, mask, iters=1):
    return ~graph_dilate(mesh, ~mask, iters)


def graph_distance(mesh, seed_mask):
    """BFS layer distance (over cellsOnCell) from the seed cells; seeds have 0."""
    nb = mesh.cellsOnCell
    dist = np.full(mesh.nCells, np.iinfo(np.int32).max, np.int64)
    dist[seed_mask] = 0
    front = seed_mask.copy()
    d = 0
    valid = nb >= 0
    while front.any():
        d += 1
        reach = np.zeros(mesh.nCells, bool)
        idx = nb[front]
        reach[idx[idx >= 0]] = True
        new = reach & (dist > d)
        dist[new] = d
        front = new
    return dist


def enforce_level_separation(mesh, level, min_sep=17, max_iter=50):
    """Promote cells so that levels l-1 and l+1 are >= ``min_sep`` layers apart.

    A level-(l-1) cell closer than ``min_sep`` to a level >= l+1 cell is
    promoted to level l (the coarse-side cells nearest to the finest region
    take the intermediate step).  Repeats until stable.
    """
    level = level.copy()
    L = int(level.max()) + 1
    for _ in range(max_iter):
        changed = False
        for l in range(1, L - 1):
            dist = graph_distance(mesh, level >= l + 1)
            bad = (level <= l - 1) & (dist < min_sep)
            if bad.any():
                level[bad] = l
                changed = True
        if not changed:
            return level
    raise RuntimeError("level separation did not converge")


def gaussian_bump_case(nx=32, ny=32, dc=10e3, H=1000.0, f=1e-4, amp=1.0, efold=100e3,
                       two_level=True, M=2, radius=80e3, dt=40.0, seed=2405):
    """Doubly periodic hex mesh, flat bottom, resting fluid with a Gaussian bump.

    With ``two_level`` the cells within ``radius`` of the domain centre are the
    fine level (factor ``M``); otherwise all cells share one level.
    """
    mesh = finalize(hex_periodic(nx, ny, dc))
    Lx, Ly = mesh.period
    rng = _rng(seed)
    cx, cy = rng.uniform(0, Lx), rng.uniform(0, Ly)
    rx = _min_image(mesh.xCell - cx, Lx)
    ry = _min_image(mesh.yCell - cy, Ly)
    h0 = H + amp * np.exp(-(rx ** 2 + ry ** 2) / efold ** 2)
    u0 = np.zeros(mesh.nEdges)
    bottom = np.full(mesh.nCells, -H)
    fV = np.full(mesh.nVertices, f)
    level = np.zeros(mesh.nCells, np.int32)
    if two_level:
        dx = _min_image(mesh.xCell - Lx / 2, Lx)
        dy = _min_image(mesh.yCell - Ly / 2, Ly)
        level[(dx ** 2 + dy ** 2) <= radius ** 2] = 1
    return Scenario(name=f"bump_hex{nx}x{ny}" + ("_lts" if two_level else ""), mesh=mesh,
                    bottom=bottom, fVertex=fV, h0=h0, u0=u0, level=level,
                    M=[M] if two_level else [], dt=dt)


def shelf_case(nx=512, ny=512, dc=2e3, f=1e-4, seed=2405, M=4, wind=15.0, cd=2.5e-3,
               roughness=0.05, width=20e3, fine_frac_cfl=0.5, vortex=False):
    """Periodic-in-y hex channel with walls in x and a continental shelf.

    ``H(x) = 10 + 3990 (1 + tanh((x - x0)/width)) / 2`` with ``x0`` the
    channel centre, times ``1 + roughness U(-1, 1)`` per cell.  The fine level
    holds the cells whose gravity-wave Courant number at the coarse step
    exceeds ``fine_frac_cfl``, closed morphologically (2 iterations).  Uniform
    onshore wind (-x) of ``wind`` m/s and quadratic bottom drag ``cd``.
    """
    full = hex_periodic(nx + 1, ny, dc)           # one land column closes x
    i_col = np.round(full.xCell / dc - 0.5 * ((np.round(full.yCell / (dc * SQRT3 / 2)).astype(int)) % 2)).astype(int)
    keep = i_col != nx
    mesh = finalize(apply_cell_mask(full, keep))
    rng = _rng(seed)
    Lx = nx * dc
    x = mesh.xCell
    H = 10.0 + 3990.0 * (1.0 + np.tanh((x - 0.5 * Lx) / width)) / 2.0
    H = H * (1.0 + roughness * rng.uniform(-1.0, 1.0, size=mesh.nCells))
    c = np.sqrt(G * H)
    dt_f = np.floor(10.0 * 0.5 * dc / c.max()) / 10.0
    dt_c = M * dt_f
    fine = c * dt_c / dc > fine_frac_cfl
    fine = graph_erode(mesh, graph_dilate(mesh, fine, 2), 2)
    level = fine.astype(np.int32)
    h0 = H.copy()
    u0 = np.zeros(mesh.nEdges)
    vt = None
    if vortex:   # a Holland vortex crossing the channel (plain distances, no periodic image)
        Ly = ny * dc * SQRT3 / 2
        vt = (95000.0, 5000.0, float(rng.uniform(8.0, 12.0)) * dc, float(rng.uniform(1.2, 1.8)),
              0.3 * Lx, 0.5 * Ly, 5.0, 1.0)
    fz = Forcing(wind_u=-wind, wind_v=0.0, cd=cd, wind_stress=wind != 0.0, vortex=vt)
    return Scenario(name=f"shelf_hex{nx}x{ny}", mesh=mesh, bottom=-H,
                    fVertex=np.full(mesh.nVertices, f), h0=h0, u0=u0, level=level,
                    M=[M], dt=float(dt_c), forcing=fz)


def nested_disk_case(nx=48, ny=48, dc=10e3, H=1000.0, f=1e-4, amp=1.0, efold=60e3,
                     radii=(140e3, 50e3), M=(2, 2), dt=40.0, seed=2405):
    """Three (or more) LTS levels as nested disks about the domain centre.

    ``radii`` lists the outer radius of level 1, level 2, ...; the levels are
    then separated with :func:`enforce_level_separation`.
    """
    mesh = finalize(hex_periodic(nx, ny, dc))
    Lx, Ly = mesh.period
    rng = _rng(seed)
    dx = _min_image(mesh.xCell - Lx / 2, Lx)
    dy = _min_image(mesh.yCell - Ly / 2, Ly)
    r2 = dx ** 2 + dy ** 2
    level = np.zeros(mesh.nCells, np.int32)
    for l, rad in enumerate(radii, start=1):
        level[r2 <= rad ** 2] = l
    level = enforce_level_separation(mesh, level).astype(np.int32)
    cx, cy = Lx / 2 + rng.uniform(-0.2, 0.2) * Lx, Ly / 2 + rng.uniform(-0.2, 0.2) * Ly
    rx = _min_image(mesh.xCell - cx, Lx)
    ry = _min_image(mesh.yCell - cy, Ly)
    h0 = H + amp * np.exp(-(rx ** 2 + ry ** 2) / efold ** 2)
    return Scenario(name=f"nested_hex{nx}x{ny}", mesh=mesh, bottom=np.full(mesh.nCells, -H),
                    fVertex=np.full(mesh.nVertices, f), h0=h0, u0=np.zeros(mesh.nEdges),
                    level=level, M=list(M), dt=dt)


def three_level_wave_case(nx=48, dc=10e3, H=1000.0, amp=5.0, efold=60e3, r_inner=40e3, sep=8,
                          M=(2, 2), dt=10.0):
    """Three LTS levels for a convergence study: a doubly periodic hex mesh
    with level 2 a disk of radius ``r_inner`` about the centre, level 1 the
    cells within ``sep`` layers of it (the oracle needs levels 0 and 2 at least
    7 layers apart), level 0 the rest; f = 0, flat bottom and a Gaussian bump
    of ``amp`` metres centred on the finest disk, so the gravity wave crosses
    both interfaces."""
    mesh = finalize(hex_periodic(nx, nx, dc))
    Lx, Ly = mesh.period
    dx = _min_image(mesh.xCell - Lx / 2, Lx)
    dy = _min_image(mesh.yCell - Ly / 2, Ly)
    r2 = dx ** 2 + dy ** 2
    inner = r2 <= r_inner ** 2
    level = np.zeros(mesh.nCells, np.int32)
    level[graph_distance(mesh, inner) <= sep] = 1
    level[inner] = 2
    h0 = H + amp * np.exp(-r2 / efold ** 2)
    return Scenario(name=f"three_level_hex{nx}x{nx}", mesh=mesh, bottom=np.full(mesh.nCells, -H),
                    fVertex=np.zeros(mesh.nVertices), h0=h0, u0=np.zeros(mesh.nEdges), level=level,
                    M=list(M), dt=dt)


def jittered_voronoi_case(k=38, L=300e3, jitter=0.45, H=1000.0, f=1e-4, amp=1.0, efold=40e3,
                          fine_radius=70e3, M=2, seed=3):
    """Irregular Voronoi mesh: a k x k grid of generators in a square box,
    each moved by a seeded uniform offset of up to ``jitter`` spacings, Qhull
    Delaunay, hull cells dropped.  Cells have 3 to about 11 edges and many
    triangles are obtuse (negative kites).  Flat depth ``H``, a Gaussian bump
    at the centre; with ``fine_radius`` a central disk is level 1 (separated).
    """
    from scipy.spatial import Delaunay
    from .mesh import build_from_triangles
    rng = _rng(seed)
    dx = L / k
    x, y = np.meshgrid(np.arange(k) * dx, np.arange(k) * dx)
    pts = np.stack([x.ravel(), y.ravel()], 1) + rng.uniform(-jitter, jitter, (k * k, 2)) * dx
    full = build_from_triangles(pts, Delaunay(pts).simplices, period=None)
    mesh = finalize(apply_cell_mask(full, np.ones(full.nCells, bool)))
    r2 = (mesh.xCell - L / 2) ** 2 + (mesh.yCell - L / 2) ** 2
    h0 = H + amp * np.exp(-r2 / efold ** 2)
    level = np.zeros(mesh.nCells, np.int32)
    Ms = []
    if fine_radius:
        level[r2 < fine_radius ** 2] = 1
        level = enforce_level_separation(mesh, level).astype(np.int32)
        Ms = [M]
    interior = (mesh.cellsOnEdge >= 0).all(1)
    dt = 0.3 * float(mesh.dcEdge[interior].min()) / np.sqrt(G * H) * (M if fine_radius else 1)
    return Scenario(name=f"jittered_voronoi_{mesh.nCells}", mesh=mesh, bottom=np.full(mesh.nCells, -H),
                    fVertex=np.full(mesh.nVertices, f), h0=h0, u0=np.zeros(mesh.nEdges), level=level,
                    M=Ms, dt=float(dt), forcing=Forcing(wind_u=0.0, wind_v=0.0, cd=0.0, wind_stress=False))


def ensemble_member(i, seed=2405, n_min=20_000, n_max=800_000):
    """Member i of the batched ensemble: a shelf channel (``shelf_case``) of
    seeded size N ~ U[n_min, n_max] cells (nx ~ sqrt(N), ny even), seeded
    roughness and vortex track, M drawn from {2, 4, 8}."""
    rng = _rng(seed + 7919 * (i + 1))
    n = int(rng.integers(n_min, n_max + 1))
    nx = max(16, int(round(np.sqrt(n))))
    ny = max(4, 2 * int(round(n / nx / 2)))
    M = int(rng.choice([2, 4, 8]))
    return shelf_case(nx=nx, ny=ny, dc=2e3, M=M, seed=seed + i, vortex=True)
