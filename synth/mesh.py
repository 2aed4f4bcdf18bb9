"""Seeded synthetic TRiSK C-grid meshes in the MPAS array layout.

Input generation only.  This module builds the geometry and connectivity of a
primal Voronoi mesh and its dual Delaunay triangulation, the tangential-flux
reconstruction weights that an MPAS mesh file carries (``weightsOnEdge``), and
land masks.  It evaluates neither the shallow-water tendencies nor the time
integrator; both the oracle and the CUDA library receive these arrays as
inputs.

Conventions (all indices 0-based, ``-1`` = absent):

* ``cellsOnEdge[e] = (c0, c1)``; the fixed edge normal ``n_e`` points from
  ``c0`` to ``c1``.  ``n_{e,i} = +1`` if ``i == c0`` (``n_e`` outward from
  ``i``), else ``-1`` (Sec. 2.3, Eq. trisk_thickness).
* ``t_e = k x n_e``; ``verticesOnEdge[e] = (v0, v1)`` is ordered so that
  ``t_e`` points from ``v0`` to ``v1``.  The dual-cell sign is then
  ``t_{e,v} = -1`` for ``v0`` (``t_e`` outward from the dual cell) and
  ``+1`` for ``v1`` (Eq. trisk_vorticity).
* ``edgesOnCell`` / ``verticesOnCell`` run counter-clockwise; vertex ``k`` of
  a cell is the counter-clockwise end of edge ``k``.
* ``weightsOnEdge[e, j]`` already contains the metric factor
  ``dvEdge[e'] / dcEdge[e]``, so the tangential thickness flux is
  ``F_perp_e = sum_j weightsOnEdge[e, j] * F[edgesOnEdge[e, j]]``.

Weights (derivation, TRiSK construction of Thuburn et al. 2009 / Ringler et
al. 2010, cited by the paper for the flux mapping M_e in Eq. trisk_vorticity):
inside a cell ``i`` with counter-clockwise edges ``e_1 = e, e_2, ..., e_n`` and
vertices ``v_k`` at the counter-clockwise end of ``e_k``, require that each
kite ``(i, v_k)`` receives the fraction ``R_{i,v_k} = kite / A_i`` of the
cell's net outflow.  The flux across the half dual edge from the centre of
``i`` to the midpoint of ``e`` (counter-clockwise sense) is then
``psi = sum_{j>=2} (1/2 - sum_{k<j} R_{i,v_k}) * n_{e_j,i} dv_{e_j} F_{e_j}``,
which is exact for uniform flow on regular hexagons and antisymmetric in
``(e, e')``.  ``F_perp_e = (psi^{(c0)} - psi^{(c1)}) / dc_e``.
"""
from __future__ import annotations

import numpy as np

SQRT3 = np.sqrt(3.0)


class Mesh:
    """Plain container of MPAS-style mesh arrays (numpy)."""

    INT_FIELDS = ("cellsOnEdge", "nEdgesOnCell", "edgesOnCell", "verticesOnCell",
                  "cellsOnCell", "verticesOnEdge", "cellsOnVertex", "edgesOnVertex",
                  "nEdgesOnEdge", "edgesOnEdge")
    REAL_FIELDS = ("weightsOnEdge", "dcEdge", "dvEdge", "areaCell", "areaTriangle",
                   "kiteAreasOnVertex", "xCell", "yCell", "xEdge", "yEdge", "angleEdge",
                   "xVertex", "yVertex")

    def __init__(self, **kw):
        for k, v in kw.items():
            setattr(self, k, v)

    @property
    def nCells(self):
        return int(self.nEdgesOnCell.shape[0])

    @property
    def nEdges(self):
        return int(self.cellsOnEdge.shape[0])

    @property
    def nVertices(self):
        return int(self.cellsOnVertex.shape[0])

    @property
    def maxEdges(self):
        return int(self.edgesOnCell.shape[1])

    @property
    def maxEdges2(self):
        return int(self.edgesOnEdge.shape[1])

    def boundary_edge_mask(self):
        return (self.cellsOnEdge < 0).any(axis=1)

    def arrays(self):
        return {k: getattr(self, k) for k in self.INT_FIELDS + self.REAL_FIELDS}


def _wrap(d, period):
    """Minimum-image displacement."""
    if period is None:
        return d
    out = d.copy()
    for ax in range(2):
        L = period[ax]
        if L is not None and L > 0:
            out[..., ax] -= L * np.round(out[..., ax] / L)
    return out


def _mod(x, period):
    if period is None:
        return x
    out = x.copy()
    for ax in range(2):
        L = period[ax]
        if L is not None and L > 0:
            out[..., ax] = np.mod(out[..., ax], L)
    return out


def _shoelace(*pts):
    """Signed area of the polygon through the given (n,2) point arrays."""
    a = np.zeros(pts[0].shape[0])
    k = len(pts)
    for i in range(k):
        p, q = pts[i], pts[(i + 1) % k]
        a += p[:, 0] * q[:, 1] - q[:, 0] * p[:, 1]
    return 0.5 * a


def build_from_triangles(pts, tri, period=None):
    """Voronoi/Delaunay C-grid from generator points and their triangulation.

    ``pts`` (N,2) cell centres, ``tri`` (T,3) Delaunay triangles (any
    orientation), ``period`` = (Lx, Ly) for a doubly periodic domain (entries
    may be None).  Cells whose Voronoi polygon is not closed (hull cells) are
    flagged in ``open_cell``; drop them with :func:`apply_cell_mask`.
    """
    pts = np.asarray(pts, dtype=np.float64)
    tri = np.asarray(tri, dtype=np.int64).copy()
    N = pts.shape[0]
    T = tri.shape[0]

    # counter-clockwise triangles (unwrapped about their first vertex)
    pa = pts[tri[:, 0]]
    db = _wrap(pts[tri[:, 1]] - pa, period)
    dcv = _wrap(pts[tri[:, 2]] - pa, period)
    cross = db[:, 0] * dcv[:, 1] - db[:, 1] * dcv[:, 0]
    flip = cross < 0
    tri[flip, 1], tri[flip, 2] = tri[flip, 2].copy(), tri[flip, 1].copy()
    db, dcv = np.where(flip[:, None], dcv, db), np.where(flip[:, None], db, dcv)
    scale = np.maximum((db ** 2).sum(1), (dcv ** 2).sum(1))
    if np.any(np.abs(cross) <= 1e-13 * scale):
        raise ValueError("degenerate triangle")

    # circumcentres relative to vertex a
    d = 2.0 * (db[:, 0] * dcv[:, 1] - db[:, 1] * dcv[:, 0])
    b2 = (db ** 2).sum(1)
    c2 = (dcv ** 2).sum(1)
    ox = (dcv[:, 1] * b2 - db[:, 1] * c2) / d
    oy = (db[:, 0] * c2 - dcv[:, 0] * b2) / d
    orel = np.stack([ox, oy], 1)
    xvert = _mod(pa + orel, period)

    # triangle sides (p -> q) in counter-clockwise order
    sp = np.concatenate([tri[:, 0], tri[:, 1], tri[:, 2]])
    sq = np.concatenate([tri[:, 1], tri[:, 2], tri[:, 0]])
    st = np.concatenate([np.arange(T)] * 3)
    lo = np.minimum(sp, sq)
    hi = np.maximum(sp, sq)
    key = lo * N + hi
    ukey, sedge = np.unique(key, return_inverse=True)
    E = ukey.shape[0]
    c0 = (ukey // N).astype(np.int64)
    c1 = (ukey % N).astype(np.int64)
    # side p->q with p == c0 has the triangle on the left of n_e, i.e. along +t_e: v1
    v0 = np.full(E, -1, np.int64)
    v1 = np.full(E, -1, np.int64)
    left = sp == c0[sedge]
    v1[sedge[left]] = st[left]
    v0[sedge[~left]] = st[~left]

    dce = _wrap(pts[c1] - pts[c0], period)
    dcEdge = np.sqrt((dce ** 2).sum(1))
    nvec = dce / dcEdge[:, None]
    angleEdge = np.arctan2(nvec[:, 1], nvec[:, 0])
    xedge = _mod(pts[c0] + 0.5 * dce, period)
    both = (v0 >= 0) & (v1 >= 0)
    dvv = np.zeros((E, 2))
    dvv[both] = _wrap(xvert[v1[both]] - xvert[v0[both]], period)
    dvEdge = np.sqrt((dvv ** 2).sum(1))

    # kites: triangle (a,b,c), circumcentre o; kite of cell a = (a, m_ab, o, m_ca)
    z = np.zeros_like(db)
    mab = 0.5 * db
    mbc = 0.5 * (db + dcv)
    mca = 0.5 * dcv
    ka = _shoelace(z, mab, orel, mca)
    kb = _shoelace(db, mbc, orel, mab)
    kc = _shoelace(dcv, mca, orel, mbc)
    kites = np.stack([ka, kb, kc], 1)
    cellsOnVertex = tri.copy()
    edgesOnVertex = np.stack([sedge[:T], sedge[T:2 * T], sedge[2 * T:]], 1)
    areaCell = np.bincount(tri.ravel(), weights=kites.ravel(), minlength=N)
    areaTriangle = kites.sum(1)

    # counter-clockwise edges per cell
    ec = np.concatenate([c0, c1])
    ee = np.concatenate([np.arange(E), np.arange(E)])
    ang = np.concatenate([angleEdge, np.arctan2(-nvec[:, 1], -nvec[:, 0])])
    order = np.lexsort((ang, ec))
    ec, ee = ec[order], ee[order]
    nEdgesOnCell = np.bincount(ec, minlength=N)
    maxEdges = int(nEdgesOnCell.max())
    start = np.concatenate([[0], np.cumsum(nEdgesOnCell)[:-1]])
    slot = np.arange(ec.shape[0]) - start[ec]
    edgesOnCell = np.full((N, maxEdges), -1, np.int64)
    edgesOnCell[ec, slot] = ee
    isc0 = c0[ee] == ec
    vend = np.where(isc0, v1[ee], v0[ee])
    verticesOnCell = np.full((N, maxEdges), -1, np.int64)
    verticesOnCell[ec, slot] = vend
    cellsOnCell = np.full((N, maxEdges), -1, np.int64)
    cellsOnCell[ec, slot] = np.where(isc0, c1[ee], c0[ee])

    # open cells: any edge missing a triangle
    open_cell = np.zeros(N, bool)
    bad = ~both
    open_cell[c0[bad]] = True
    open_cell[c1[bad]] = True

    # kite area of vertex verticesOnCell[i,k] inside cell i
    kiteOnCell = np.zeros((N, maxEdges))
    valid = verticesOnCell >= 0
    ii, kk = np.nonzero(valid)
    vv = verticesOnCell[ii, kk]
    cov = cellsOnVertex[vv]
    jj = np.argmax(cov == ii[:, None], axis=1)
    kiteOnCell[ii, kk] = kites[vv, jj]

    # edgesOnEdge / weightsOnEdge (see module docstring)
    slot_of = np.zeros((E, 2), np.int64)          # position of e in the lists of c0 / c1
    slot_of[ee[isc0], 0] = slot[isc0]
    slot_of[ee[~isc0], 1] = slot[~isc0]
    closed = ~open_cell
    ok = closed[c0] & closed[c1]
    mclosed = int(nEdgesOnCell[closed].max()) if closed.any() else 3
    maxEdges2 = 2 * (mclosed - 1)
    eoe = np.full((E, maxEdges2), -1, np.int64)
    woe = np.zeros((E, maxEdges2))
    neoe = np.zeros(E, np.int64)
    rows = np.arange(E)
    for side, csel, sgn_e in ((0, c0, 1.0), (1, c1, -1.0)):
        i = csel
        n = np.maximum(nEdgesOnCell[i], 1)
        p = slot_of[:, side]
        rsum = np.zeros(E)
        for m in range(1, mclosed):
            act = ok & (m < n)
            prev = (p + m - 1) % n
            rsum = rsum + np.where(act, kiteOnCell[i, prev] / areaCell[i], 0.0)
            ej = edgesOnCell[i, (p + m) % n]
            ejc = np.maximum(ej, 0)
            sgn_j = np.where(c0[ejc] == i, 1.0, -1.0)
            w = sgn_e * sgn_j * (0.5 - rsum) * dvEdge[ejc] / dcEdge
            col = neoe[act]
            eoe[rows[act], col] = ej[act]
            woe[rows[act], col] = w[act]
            neoe = neoe + act

    return Mesh(
        cellsOnEdge=np.stack([c0, c1], 1), nEdgesOnCell=nEdgesOnCell, edgesOnCell=edgesOnCell,
        verticesOnCell=verticesOnCell, cellsOnCell=cellsOnCell,
        verticesOnEdge=np.stack([v0, v1], 1), cellsOnVertex=cellsOnVertex,
        edgesOnVertex=edgesOnVertex, nEdgesOnEdge=neoe, edgesOnEdge=eoe,
        weightsOnEdge=woe, dcEdge=dcEdge, dvEdge=dvEdge, areaCell=areaCell,
        areaTriangle=areaTriangle, kiteAreasOnVertex=kites,
        xCell=pts[:, 0].copy(), yCell=pts[:, 1].copy(), xEdge=xedge[:, 0], yEdge=xedge[:, 1],
        angleEdge=angleEdge, xVertex=xvert[:, 0], yVertex=xvert[:, 1],
        open_cell=open_cell, period=period)


def apply_cell_mask(mesh, keep):
    """Keep only the cells in ``keep`` (bool per cell); open cells are dropped too.

    Edges with one kept cell become no-flow boundary edges (the other cell is
    -1).  Vertices survive if any of their cells survives.
    """
    keep = np.asarray(keep, bool) & ~mesh.open_cell
    N, E, V = mesh.nCells, mesh.nEdges, mesh.nVertices
    cmap = np.full(N + 1, -1, np.int64)
    cmap[:N][keep] = np.arange(int(keep.sum()))
    coe = mesh.cellsOnEdge
    ekeep = keep[coe[:, 0]] | keep[coe[:, 1]]
    emap = np.full(E + 1, -1, np.int64)
    emap[:E][ekeep] = np.arange(int(ekeep.sum()))
    cov = mesh.cellsOnVertex
    vkeep = keep[cov].any(1)
    vmap = np.full(V + 1, -1, np.int64)
    vmap[:V][vkeep] = np.arange(int(vkeep.sum()))

    def rm(m, a):  # remap index array with -1 passthrough
        return m[np.where(a < 0, -1, a)]

    new_coe = rm(cmap, coe[ekeep])
    interior = (new_coe >= 0).all(1)
    eoe = rm(emap, mesh.edgesOnEdge[ekeep])
    woe = mesh.weightsOnEdge[ekeep].copy()
    neoe = mesh.nEdgesOnEdge[ekeep].copy()
    eoe[~interior] = -1
    woe[~interior] = 0.0
    neoe[~interior] = 0
    mE = max(int(mesh.nEdgesOnCell[keep].max()), 3) if keep.any() else mesh.maxEdges
    mE2 = max(int(neoe.max()), 1) if neoe.size else 1
    eoe, woe = eoe[:, :mE2], woe[:, :mE2]
    out = Mesh(
        cellsOnEdge=new_coe,
        nEdgesOnCell=mesh.nEdgesOnCell[keep].copy(),
        edgesOnCell=rm(emap, mesh.edgesOnCell[keep][:, :mE]),
        verticesOnCell=rm(vmap, mesh.verticesOnCell[keep][:, :mE]),
        cellsOnCell=rm(cmap, mesh.cellsOnCell[keep][:, :mE]),
        verticesOnEdge=rm(vmap, mesh.verticesOnEdge[ekeep]),
        cellsOnVertex=rm(cmap, cov[vkeep]),
        edgesOnVertex=rm(emap, mesh.edgesOnVertex[vkeep]),
        nEdgesOnEdge=neoe, edgesOnEdge=eoe, weightsOnEdge=woe,
        dcEdge=mesh.dcEdge[ekeep].copy(), dvEdge=mesh.dvEdge[ekeep].copy(),
        areaCell=mesh.areaCell[keep].copy(), areaTriangle=mesh.areaTriangle[vkeep].copy(),
        kiteAreasOnVertex=mesh.kiteAreasOnVertex[vkeep].copy(),
        xCell=mesh.xCell[keep].copy(), yCell=mesh.yCell[keep].copy(),
        xEdge=mesh.xEdge[ekeep].copy(), yEdge=mesh.yEdge[ekeep].copy(),
        angleEdge=mesh.angleEdge[ekeep].copy(),
        xVertex=mesh.xVertex[vkeep].copy(), yVertex=mesh.yVertex[vkeep].copy(),
        open_cell=np.zeros(int(keep.sum()), bool), period=mesh.period)
    return out


def finalize(mesh):
    """Cast index arrays to int32 and real arrays to contiguous float64."""
    for k in Mesh.INT_FIELDS:
        setattr(mesh, k, np.ascontiguousarray(getattr(mesh, k), dtype=np.int32))
    for k in Mesh.REAL_FIELDS:
        setattr(mesh, k, np.ascontiguousarray(getattr(mesh, k), dtype=np.float64))
    return mesh


def hex_periodic(nx, ny, dc):
    """Doubly periodic regular-hexagon mesh of nx x ny cells (ny even).

    Cell (i, j) sits at x = dc (i + (j mod 2)/2), y = dc sqrt(3)/2 j; the
    domain is nx dc by ny dc sqrt(3)/2.
    """
    if nx < 3 or ny < 4 or ny % 2:
        raise ValueError("need nx >= 3 and an even ny >= 4")
    j, i = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    i = i.ravel()
    j = j.ravel()
    x = dc * (i + 0.5 * (j % 2))
    y = dc * SQRT3 / 2 * j
    pts = np.stack([x, y], 1)

    def cid(ii, jj):
        return (jj % ny) * nx + (ii % nx)

    odd = j % 2
    right = cid(i + 1, j)
    upright = cid(i + odd, j + 1)
    upleft = cid(i + odd - 1, j + 1)
    me = cid(i, j)
    tri = np.concatenate([np.stack([me, right, upright], 1), np.stack([me, upright, upleft], 1)])
    period = (nx * dc, ny * dc * SQRT3 / 2)
    return build_from_triangles(pts, tri, period=period)
