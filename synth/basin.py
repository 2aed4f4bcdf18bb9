"""Variable-resolution Voronoi basin with a sinuous coast (the storm-surge workload).

A closed rectangular basin ``[0, Lx] x [0, Ly]`` with land east of the
coastline ``x_c(y) = Lx - x_off + sum_j a_j sin(2 pi k_j y / Ly + phi_j)``
(three seeded sines) and no-flow walls on the other sides.  With ``d`` the
horizontal distance ``x_c(y) - x`` from the coast:

* cell spacing ``dx(d) = dx_min`` for ``d <= d0``, then growing by ``slope``
  per metre up to ``dx_max`` offshore;
* resting depth ``H(d) = 5 + 3995 (1 - exp(-d / 150 km))``;
* generators are laid in coast-parallel rows spaced ``sqrt(3)/2 dx`` with
  ``dx`` along each row (a hexagonal pattern that follows the spacing),
  jittered (seeded) and relaxed by density-weighted Lloyd iterations
  (centroids weighted by ``dx(d)^-4``); Qhull supplies the Delaunay
  triangulation and :mod:`synth.mesh` the Voronoi C-grid and TRiSK weights;
* LTS level per cell from the gravity-wave CFL limit
  ``0.5 dc_min / sqrt(g H)``: ``dt_0`` is 0.95 times the smallest limit of the
  coarsest cells, level ``l`` holds the cells with
  ``dt_0 / 8^l <= limit < dt_0 / 8^(l-1)`` (3 levels, M = 8), then levels are
  separated so the interface bands of successive level pairs stay apart;
* a Holland-type vortex on a seeded straight track that crosses the coast.

Input generation only: no tendency or time-stepping arithmetic.
"""
from __future__ import annotations

import time

import numpy as np
from scipy.spatial import Delaunay

from .mesh import build_from_triangles, apply_cell_mask, finalize
from .scenario import Scenario, Forcing, G, enforce_level_separation, _rng


def depth(d):
    return 5.0 + 3995.0 * (1.0 - np.exp(-np.maximum(d, 0.0) / 150e3))


class Coast:
    """Sinuous coastline; the sine amplitudes scale with the basin length so the
    coast keeps the same slopes (at most about 0.5) for any Ly."""

    def __init__(self, Lx, Ly, x_off, rng):
        self.Lx, self.Ly, self.x_off = Lx, Ly, x_off
        self.a = rng.uniform(20e3, 60e3, 3) * min(1.0, Ly / 9600e3)
        self.k = rng.integers(2, 13, 3)
        self.phi = rng.uniform(0, 2 * np.pi, 3)

    def x(self, y):
        s = np.zeros_like(y, dtype=np.float64)
        for a, k, p in zip(self.a, self.k, self.phi):
            s += a * np.sin(2 * np.pi * k * y / self.Ly + p)
        return self.Lx - self.x_off + s


def spacing(d, dx_min, dx_max, d0, slope):
    return np.clip(dx_min + slope * np.maximum(d - d0, 0.0), dx_min, dx_max)


def _rows(coast, Ly, dx_min, dx_max, d0, slope, rng, jitter, margin):
    """Coast-parallel rows of generators: ocean rows (d >= -4 dx_min) follow
    dx(d); land rows east of them coarsen by 25 % per row up to dx_max until
    the frame edge, so the cloud's hull is close to a rectangle."""
    ys = np.linspace(-margin, Ly + margin, 200001)
    xs = coast.x(ys)
    ds = np.sqrt(1.0 + np.gradient(xs, ys) ** 2)
    arc = np.concatenate([[0.0], np.cumsum(0.5 * (ds[1:] + ds[:-1]) * np.diff(ys))])

    def row(d, dx, k):
        s = np.arange(0.0, arc[-1], dx) + (0.5 * dx if k % 2 else 0.0)
        y = np.interp(s, arc, ys)
        x = coast.x(y) - d
        if jitter:
            x = x + rng.uniform(-jitter, jitter, x.size) * dx
            y = y + rng.uniform(-jitter, jitter, y.size) * dx
        return np.stack([x, y], 1)

    pts = []
    d = -4.0 * dx_min
    dmax = coast.x(ys).max() + margin
    k = 0
    while d <= dmax:
        dx = float(spacing(np.array(d), dx_min, dx_max, d0, slope))
        pts.append(row(d, dx, k))
        d += np.sqrt(3.0) / 2.0 * dx
        k += 1
    # land rows
    dx = dx_min
    d = -4.0 * dx_min
    dland = coast.x_off + coast.a.sum() + margin
    k = 1
    while d > -dland:
        dx = min(dx_max, dx * 1.25)
        d -= np.sqrt(3.0) / 2.0 * dx
        pts.append(row(d, dx, k))
        k += 1
    return np.concatenate(pts)


def _lloyd(pts, coast, dx_min, dx_max, d0, slope, iters, movable):
    """Density-weighted Lloyd steps: move each movable generator to the
    centroid of its Voronoi cell under the density dx(d)^-4 (kite
    decomposition).  Generators of the surrounding frame stay fixed."""
    for _ in range(iters):
        tri = Delaunay(pts).simplices
        pa, pb, pc = pts[tri[:, 0]], pts[tri[:, 1]], pts[tri[:, 2]]
        b = pb - pa
        c = pc - pa
        dd = 2.0 * (b[:, 0] * c[:, 1] - b[:, 1] * c[:, 0])
        ok = np.abs(dd) > 0
        b2, c2 = (b ** 2).sum(1), (c ** 2).sum(1)
        o = np.zeros_like(b)
        o[ok, 0] = (c[ok, 1] * b2[ok] - b[ok, 1] * c2[ok]) / dd[ok]
        o[ok, 1] = (b[ok, 0] * c2[ok] - c[ok, 0] * b2[ok]) / dd[ok]
        o = pa + o
        acc = np.zeros((pts.shape[0], 3))
        for (p, q, r) in ((pa, pb, pc), (pb, pc, pa), (pc, pa, pb)):
            idx = {id(pa): 0, id(pb): 1, id(pc): 2}[id(p)]
            mq, mr = 0.5 * (p + q), 0.5 * (p + r)
            for (u, v) in ((mq, o), (o, mr)):
                area = np.abs(0.5 * ((u[:, 0] - p[:, 0]) * (v[:, 1] - p[:, 1]) - (u[:, 1] - p[:, 1]) * (v[:, 0] - p[:, 0])))
                cen = (p + u + v) / 3.0
                dist = coast.x(cen[:, 1]) - cen[:, 0]
                w = area * spacing(dist, dx_min, dx_max, d0, slope) ** -4
                n = pts.shape[0]
                acc[:, 0] += np.bincount(tri[:, idx], weights=w * cen[:, 0], minlength=n)
                acc[:, 1] += np.bincount(tri[:, idx], weights=w * cen[:, 1], minlength=n)
                acc[:, 2] += np.bincount(tri[:, idx], weights=w, minlength=n)
        good = (acc[:, 2] > 0) & movable
        pts = pts.copy()
        pts[good] = acc[good, :2] / acc[good, 2:3]
    return pts


def basin_case(Ly=9600e3, Lx=1500e3, x_off=150e3, dx_min=500.0, dx_max=20e3, d0=20e3, slope=0.02,
               M=8, nlevels=3, lloyd=2, jitter=0.05, f=1e-4, seed=2405, vortex_offshore=600e3,
               dt0_fit=False, verbose=False):
    """The ~2M-cell closed basin (defaults); smaller Ly gives a proportionally smaller mesh."""
    rng = _rng(seed)
    t0 = time.time()
    coast = Coast(Lx, Ly, x_off, rng)
    margin = 3 * dx_max
    pts = _rows(coast, Ly, dx_min, dx_max, d0, slope, rng, jitter, margin)
    # keep generators inside a frame around the basin (the frame closes the hull)
    keep = (pts[:, 0] > -margin) & (pts[:, 1] > -margin) & (pts[:, 1] < Ly + margin)
    pts = pts[keep]
    if verbose:
        print(f"basin: {pts.shape[0]} generators in {time.time() - t0:.1f}s")
    movable = (pts[:, 0] > 0.0) & (pts[:, 1] > 0.0) & (pts[:, 1] < Ly)
    pts = _lloyd(pts, coast, dx_min, dx_max, d0, slope, lloyd, movable)
    if verbose:
        print(f"basin: lloyd x{lloyd} {time.time() - t0:.1f}s")
    tri = Delaunay(pts).simplices
    full = build_from_triangles(pts, tri, period=None)
    if verbose:
        print(f"basin: voronoi {time.time() - t0:.1f}s")
    x, y = full.xCell, full.yCell
    ocean = (x >= 0.0) & (y >= 0.0) & (y <= Ly) & (x <= coast.x(y)) & ~full.open_cell
    # drop ocean cells without an ocean neighbour (specks cut off by the coast)
    nb = full.cellsOnCell
    wet_nb = (np.where(nb >= 0, ocean[np.maximum(nb, 0)], False)).any(1)
    ocean &= wet_nb
    # every kept vertex needs a positive area from its kept cells: drop the
    # kept cells of a vertex whose kites (obtuse triangles) sum to <= 0
    for _ in range(10):
        cov = full.cellsOnVertex
        kept = ocean[cov]
        av = np.where(kept, full.kiteAreasOnVertex, 0.0).sum(1)
        bad = kept.any(1) & (av <= 0.0)
        if not bad.any():
            break
        ocean[cov[bad][kept[bad]]] = False
    mesh = finalize(apply_cell_mask(full, ocean))
    if verbose:
        print(f"basin: {mesh.nCells} cells {mesh.nEdges} edges {mesh.nVertices} vertices, {time.time() - t0:.1f}s")
    d = coast.x(mesh.yCell) - mesh.xCell
    H = depth(d)
    # CFL limit per cell from its shortest interior edge
    coe = mesh.cellsOnEdge
    inter = (coe >= 0).all(1)
    dcmin = np.full(mesh.nCells, np.inf)
    for s_ in (0, 1):
        np.minimum.at(dcmin, coe[inter, s_], mesh.dcEdge[inter])
    lim = 0.5 * dcmin / np.sqrt(G * H)
    nominal = spacing(d, dx_min, dx_max, d0, slope)
    coarse = nominal >= 0.99 * dx_max
    dt0 = 0.95 * float(lim[coarse].min() if coarse.any() else lim.max())
    if dt0_fit:   # small test basins: the finest level takes the smallest limit
        dt0 = min(dt0, 0.95 * float(lim.min()) * float(M) ** (nlevels - 1))
    lev = np.ceil(np.log(dt0 / lim) / np.log(M) - 1e-12)
    lev = np.clip(lev, 0, nlevels - 1).astype(np.int32)
    if np.any(dt0 / float(M) ** lev > lim * (1 + 1e-12)):
        raise RuntimeError("basin: finest level too coarse for the CFL limit; add levels")
    lev = enforce_level_separation(mesh, lev).astype(np.int32)
    # Holland vortex: starts vortex_offshore (600 km) offshore at a seeded latitude, moves east at 5 m/s
    y0 = rng.uniform(0.35, 0.65) * Ly
    x0 = float(coast.x(np.array([y0]))[0]) - vortex_offshore
    vortex = (95000.0, 5000.0, float(rng.uniform(30e3, 60e3)), float(rng.uniform(1.2, 1.8)),
              x0, y0, 5.0, float(rng.uniform(-1.0, 1.0)))
    fz = Forcing(wind_u=0.0, wind_v=0.0, cd=2.5e-3, wind_stress=True, vortex=vortex)
    s = Scenario(name=f"basin_{mesh.nCells // 1000}k", mesh=mesh, bottom=-H,
                 fVertex=np.full(mesh.nVertices, f), h0=H.copy(), u0=np.zeros(mesh.nEdges),
                 level=lev, M=[M] * (nlevels - 1), dt=dt0, forcing=fz)
    s.depth = H
    s.coast = coast
    if verbose:
        print(f"basin: levels {np.bincount(lev, minlength=nlevels).tolist()} dt0={dt0:.2f}s "
              f"min kite {mesh.kiteAreasOnVertex.min():.3g} total {time.time() - t0:.1f}s")
    return s
