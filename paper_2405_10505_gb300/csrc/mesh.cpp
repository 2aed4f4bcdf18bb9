// Host side of fblts_mesh_create: validation, LTS region classification
// (Sec. 2.2, Fig. lts_regions) and the band / space-filling-curve renumbering
// that turns every region into one contiguous index range.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <numeric>

#include "fblts_internal.h"

namespace fblts {

namespace {

// Hilbert index of (x, y) on a 2^16 x 2^16 grid.
uint64_t hilbert_d(uint32_t x, uint32_t y) {
    const uint32_t n = 1u << 16;
    uint64_t d = 0;
    for (uint32_t s = n / 2; s > 0; s /= 2) {
        uint32_t rx = (x & s) ? 1u : 0u;
        uint32_t ry = (y & s) ? 1u : 0u;
        d += (uint64_t)s * s * ((3u * rx) ^ ry);
        if (ry == 0) {
            if (rx == 1) {
                x = n - 1 - x;
                y = n - 1 - y;
            }
            std::swap(x, y);
        }
    }
    return d;
}

// BFS layer distance from seed cells across edges with two cells.
void bfs(int nC, const std::vector<int> &nbr_off, const std::vector<int> &nbr,
         const std::vector<uint8_t> &seed, std::vector<int> &dist) {
    dist.assign(nC, INT32_MAX);
    std::vector<int> q;
    q.reserve(nC);
    for (int i = 0; i < nC; ++i)
        if (seed[i]) {
            dist[i] = 0;
            q.push_back(i);
        }
    for (size_t h = 0; h < q.size(); ++h) {
        int i = q[h];
        for (int k = nbr_off[i]; k < nbr_off[i + 1]; ++k) {
            int o = nbr[k];
            if (dist[o] == INT32_MAX) {
                dist[o] = dist[i] + 1;
                q.push_back(o);
            }
        }
    }
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

}  // namespace

int HostMesh::cell_lb(uint32_t k) const {
    return (int)(std::lower_bound(ckey.begin(), ckey.end(), k) - ckey.begin());
}
int HostMesh::edge_lb(uint32_t k) const {
    return (int)(std::lower_bound(ekey.begin(), ekey.end(), k) - ekey.begin());
}
int HostMesh::vert_lb(uint32_t k) const {
    return (int)(std::lower_bound(vkey.begin(), vkey.end(), k) - vkey.begin());
}

fblts_status build_host_mesh(const fblts_mesh_desc *d, HostMesh &hm) {
    if (!d) { set_error("mesh_create: desc is NULL"); return FBLTS_E_ARG; }
    const int nC = d->nCells, nE = d->nEdges, nV = d->nVertices, mE = d->maxEdges, mE2 = d->maxEdges2;
    if (nC <= 0 || nE <= 0 || nV <= 0 || mE < 3 || mE2 < 1) {
        set_error("mesh_create: bad sizes nCells=%d nEdges=%d nVertices=%d maxEdges=%d maxEdges2=%d",
                  nC, nE, nV, mE, mE2);
        return FBLTS_E_ARG;
    }
    if (!d->cellsOnEdge || !d->nEdgesOnCell || !d->edgesOnCell || !d->verticesOnEdge ||
        !d->cellsOnVertex || !d->nEdgesOnEdge || !d->edgesOnEdge || !d->weightsOnEdge ||
        !d->dcEdge || !d->dvEdge || !d->areaCell || !d->kiteAreasOnVertex || !d->fVertex) {
        set_error("mesh_create: a required array is NULL");
        return FBLTS_E_ARG;
    }
    const int L = d->nLevels <= 0 ? 1 : d->nLevels;
    if (L > 8) { set_error("mesh_create: at most 8 levels"); return FBLTS_E_ARG; }
    if (L > 1 && (!d->ltsLevel || !d->M)) {
        set_error("mesh_create: nLevels > 1 needs ltsLevel and M");
        return FBLTS_E_ARG;
    }
    hm.nC = nC; hm.nE = nE; hm.nV = nV; hm.L = L;
    hm.nIF1 = d->nIF1Layers > 0 ? d->nIF1Layers : 2;
    hm.nIF2 = d->nIF2Layers > 0 ? d->nIF2Layers : 2;
    hm.kin_cap = hm.nIF1 + hm.nIF2 + 3;
    if (hm.kin_cap > 200) { set_error("mesh_create: IF layers too large"); return FBLTS_E_ARG; }
    hm.M.assign(L > 1 ? L - 1 : 0, 1);
    for (int l = 0; l + 1 < L; ++l) {
        if (d->M[l] < 1 || d->M[l] > 4096) { set_error("mesh_create: M[%d]=%d invalid", l, d->M[l]); return FBLTS_E_ARG; }
        hm.M[l] = d->M[l];
    }

    // ---------------------------------------------------------- validation
    const int *coe = d->cellsOnEdge, *voe = d->verticesOnEdge, *cov = d->cellsOnVertex;
    std::vector<uint8_t> ebnd(nE, 0);
    for (int e = 0; e < nE; ++e) {
        int a = coe[2 * e], b = coe[2 * e + 1];
        if (a < -1 || a >= nC || b < -1 || b >= nC || (a < 0 && b < 0) || a == b) {
            set_error("mesh_create: cellsOnEdge[%d] = (%d, %d) invalid", e, a, b);
            return FBLTS_E_MESH;
        }
        ebnd[e] = (a < 0 || b < 0);
        for (int s = 0; s < 2; ++s) {
            int v = voe[2 * e + s];
            if (v < -1 || v >= nV || (!ebnd[e] && v < 0)) {
                set_error("mesh_create: verticesOnEdge[%d] = (%d, %d) invalid", e, voe[2 * e], voe[2 * e + 1]);
                return FBLTS_E_MESH;
            }
        }
        if (!ebnd[e] && !(finite_pos(d->dcEdge[e]) && finite_pos(d->dvEdge[e]))) {
            set_error("mesh_create: dcEdge/dvEdge of edge %d not positive", e);
            return FBLTS_E_MESH;
        }
        int ne = d->nEdgesOnEdge[e];
        if (ne < 0 || ne > mE2) { set_error("mesh_create: nEdgesOnEdge[%d]=%d", e, ne); return FBLTS_E_MESH; }
        for (int j = 0; j < ne; ++j) {
            int x = d->edgesOnEdge[(size_t)e * mE2 + j];
            if (x < 0 || x >= nE || !std::isfinite(d->weightsOnEdge[(size_t)e * mE2 + j])) {
                set_error("mesh_create: edgesOnEdge/weightsOnEdge of edge %d invalid", e);
                return FBLTS_E_MESH;
            }
        }
    }
    std::vector<int> listed(nE, 0);
    for (int i = 0; i < nC; ++i) {
        int n = d->nEdgesOnCell[i];
        if (n < 3 || n > mE || !finite_pos(d->areaCell[i])) {
            set_error("mesh_create: cell %d has %d edges / area %g", i, n, d->areaCell[i]);
            return FBLTS_E_MESH;
        }
        for (int j = 0; j < n; ++j) {
            int e = d->edgesOnCell[(size_t)i * mE + j];
            if (e < 0 || e >= nE || (coe[2 * e] != i && coe[2 * e + 1] != i)) {
                set_error("mesh_create: edgesOnCell[%d][%d]=%d does not touch the cell", i, j, e);
                return FBLTS_E_MESH;
            }
            listed[e]++;
        }
    }
    for (int e = 0; e < nE; ++e)
        if (listed[e] != (ebnd[e] ? 1 : 2)) {
            set_error("mesh_create: edge %d listed by %d cells", e, listed[e]);
            return FBLTS_E_MESH;
        }
    // row widths of the library's own arrays: the actual maxima (at most 12 edges per cell)
    int W = 3, W2 = 1;
    for (int i = 0; i < nC; ++i) W = std::max(W, d->nEdgesOnCell[i]);
    for (int e = 0; e < nE; ++e) W2 = std::max(W2, d->nEdgesOnEdge[e]);
    if (W > 12) { set_error("mesh_create: a cell has %d edges (at most 12)", W); return FBLTS_E_MESH; }
    W2 = std::max(W2, 2 * (W - 1));
    hm.maxE = W;
    hm.maxE2 = W2;
    std::vector<int> eov(3 * (size_t)nV, -1);
    if (d->edgesOnVertex) {
        for (size_t k = 0; k < 3 * (size_t)nV; ++k) {
            int e = d->edgesOnVertex[k];
            if (e < -1 || e >= nE) { set_error("mesh_create: edgesOnVertex invalid"); return FBLTS_E_MESH; }
            eov[k] = e;
        }
    } else {
        std::vector<int> cnt(nV, 0);
        for (int e = 0; e < nE; ++e)
            for (int s = 0; s < 2; ++s) {
                int v = voe[2 * e + s];
                if (v < 0) continue;
                if (cnt[v] >= 3) { set_error("mesh_create: vertex %d has more than 3 edges", v); return FBLTS_E_MESH; }
                eov[3 * (size_t)v + cnt[v]++] = e;
            }
    }
    std::vector<double> Av(nV, 0.0);
    for (int v = 0; v < nV; ++v) {
        int present = 0;
        for (int j = 0; j < 3; ++j) {
            int c = cov[3 * v + j];
            if (c < -1 || c >= nC) { set_error("mesh_create: cellsOnVertex[%d] invalid", v); return FBLTS_E_MESH; }
            if (c >= 0) { present++; Av[v] += d->kiteAreasOnVertex[3 * v + j]; }
        }
        if (!present || !finite_pos(Av[v])) {
            set_error("mesh_create: vertex %d has no cell or a non-positive area", v);
            return FBLTS_E_MESH;
        }
    }
    // every interior edge must be listed by its two vertices
    for (int v = 0; v < nV; ++v)
        for (int j = 0; j < 3; ++j) {
            int e = eov[3 * v + j];
            if (e >= 0 && voe[2 * e] != v && voe[2 * e + 1] != v) {
                set_error("mesh_create: edgesOnVertex[%d] lists edge %d which does not touch it", v, e);
                return FBLTS_E_MESH;
            }
        }

    // ---------------------------------------------------------- levels
    std::vector<int> lev(nC, 0);
    std::vector<int64_t> per_level(L, 0);
    for (int i = 0; i < nC; ++i) {
        int l = (L > 1) ? d->ltsLevel[i] : 0;
        if (l < 0 || l >= L) { set_error("mesh_create: ltsLevel[%d]=%d out of range", i, l); return FBLTS_E_REGIONS; }
        lev[i] = l;
        per_level[l]++;
    }
    for (int l = 0; l < L; ++l)
        if (per_level[l] == 0) { set_error("mesh_create: level %d has no cells", l); return FBLTS_E_REGIONS; }
    // neighbour lists
    std::vector<int> off(nC + 1, 0), nbr;
    for (int i = 0; i < nC; ++i) off[i + 1] = off[i] + d->nEdgesOnCell[i];
    nbr.assign(off[nC], -1);
    {
        std::vector<int> fill(nC, 0);
        for (int i = 0; i < nC; ++i)
            for (int j = 0; j < d->nEdgesOnCell[i]; ++j) {
                int e = d->edgesOnCell[(size_t)i * mE + j];
                if (ebnd[e]) continue;
                int o = coe[2 * e] == i ? coe[2 * e + 1] : coe[2 * e];
                nbr[off[i] + fill[i]++] = o;
            }
        // compact (boundary edges leave holes)
        std::vector<int> off2(nC + 1, 0), nbr2;
        nbr2.reserve(nbr.size());
        for (int i = 0; i < nC; ++i) {
            for (int k = off[i]; k < off[i] + fill[i]; ++k) nbr2.push_back(nbr[k]);
            off2[i + 1] = (int)nbr2.size();
        }
        off.swap(off2);
        nbr.swap(nbr2);
    }
    // optional promotion: level l-1 cells closer than the separation the band
    // order needs to a level >= l+1 cell move to level l, until stable
    if ((d->flags & FBLTS_MESH_PROMOTE_LEVELS) && L >= 3) {
        std::vector<uint8_t> sd(nC);
        std::vector<int> dd;
        bool changed = true;
        for (int it = 0; changed && it < 64; ++it) {
            changed = false;
            for (int l = 1; l + 1 < L; ++l) {
                for (int i = 0; i < nC; ++i) sd[i] = lev[i] >= l + 1;
                bfs(nC, off, nbr, sd, dd);
                for (int i = 0; i < nC; ++i)
                    if (lev[i] <= l - 1 && dd[i] < 10 + hm.kin_cap) {
                        per_level[lev[i]]--;
                        per_level[l]++;
                        lev[i] = l;
                        changed = true;
                    }
            }
        }
        for (int l = 0; l < L; ++l)
            if (per_level[l] == 0) { set_error("mesh_create: level %d has no cells after promotion", l); return FBLTS_E_REGIONS; }
    }
    for (int e = 0; e < nE; ++e)
        if (!ebnd[e] && std::abs(lev[coe[2 * e]] - lev[coe[2 * e + 1]]) > 1) {
            set_error("mesh_create: edge %d joins levels %d and %d", e, lev[coe[2 * e]], lev[coe[2 * e + 1]]);
            return FBLTS_E_REGIONS;
        }
    // per pair (l, l+1): inner distance of level-l cells, outer distance of level-(l+1) cells
    std::vector<int> din(nC, hm.kin_cap), dout(nC, INT32_MAX);
    std::vector<uint8_t> seed(nC);
    std::vector<int> dist;
    for (int l = 0; l + 1 < L; ++l) {
        for (int i = 0; i < nC; ++i) seed[i] = lev[i] >= l + 1;
        bfs(nC, off, nbr, seed, dist);
        for (int i = 0; i < nC; ++i)
            if (lev[i] == l) din[i] = std::min(dist[i], hm.kin_cap);
        if (l >= 1) {
            for (int i = 0; i < nC; ++i)
                if (lev[i] <= l - 1 && dist[i] < 10 + hm.kin_cap) {
                    set_error("mesh_create: level %d cell %d is %d layers from level >= %d (need >= %d)",
                              lev[i], i, dist[i], l + 1, 10 + hm.kin_cap);
                    return FBLTS_E_REGIONS;
                }
        }
        for (int i = 0; i < nC; ++i) seed[i] = lev[i] <= l;
        bfs(nC, off, nbr, seed, dist);
        for (int i = 0; i < nC; ++i)
            if (lev[i] == l + 1) dout[i] = dist[i];
    }
    std::vector<int> kin(nC), kout(nC);
    for (int i = 0; i < nC; ++i) {
        kin[i] = (lev[i] < L - 1) ? din[i] : hm.kin_cap;
        int b = 6;
        if (lev[i] > 0 && dout[i] != INT32_MAX) b = std::min(6, (dout[i] + 1) / 2);
        kout[i] = lev[i] > 0 ? 6 - b : 0;
    }

    // ---------------------------------------------------------- locality key
    std::vector<uint64_t> sfc(nC);
    if (d->xCell && d->yCell) {
        double x0 = 1e300, x1 = -1e300, y0 = 1e300, y1 = -1e300;
        for (int i = 0; i < nC; ++i) {
            x0 = std::min(x0, d->xCell[i]); x1 = std::max(x1, d->xCell[i]);
            y0 = std::min(y0, d->yCell[i]); y1 = std::max(y1, d->yCell[i]);
        }
        double s = std::max(x1 - x0, y1 - y0);
        if (!(s > 0) || !std::isfinite(s)) s = 1.0;
        for (int i = 0; i < nC; ++i) {
            double fx = (d->xCell[i] - x0) / s, fy = (d->yCell[i] - y0) / s;
            uint32_t ix = (uint32_t)std::min(65535.0, std::max(0.0, fx * 65535.0));
            uint32_t iy = (uint32_t)std::min(65535.0, std::max(0.0, fy * 65535.0));
            sfc[i] = hilbert_d(ix, iy);
        }
    } else {
        // breadth-first order from cell 0 (each component in turn)
        std::vector<int> rank(nC, -1);
        int r = 0;
        for (int s0 = 0; s0 < nC; ++s0) {
            if (rank[s0] >= 0) continue;
            std::deque<int> q{s0};
            rank[s0] = r++;
            while (!q.empty()) {
                int i = q.front();
                q.pop_front();
                for (int k = off[i]; k < off[i + 1]; ++k)
                    if (rank[nbr[k]] < 0) { rank[nbr[k]] = r++; q.push_back(nbr[k]); }
            }
        }
        for (int i = 0; i < nC; ++i) sfc[i] = (uint64_t)rank[i];
    }

    // ---------------------------------------------------------- order cells
    std::vector<uint32_t> ck(nC);
    for (int i = 0; i < nC; ++i) ck[i] = BandKey::make(L, lev[i], kin[i], kout[i]);
    hm.cell_n2o.resize(nC);
    std::iota(hm.cell_n2o.begin(), hm.cell_n2o.end(), 0);
    std::sort(hm.cell_n2o.begin(), hm.cell_n2o.end(), [&](int a, int b) {
        if (ck[a] != ck[b]) return ck[a] < ck[b];
        if (sfc[a] != sfc[b]) return sfc[a] < sfc[b];
        return a < b;
    });
    hm.cell_o2n.assign(nC, -1);
    for (int i = 0; i < nC; ++i) hm.cell_o2n[hm.cell_n2o[i]] = i;

    // edges / vertices follow the cell of their finest level that is closest
    // to the finer region (inner) and to the coarser region (outer band)
    auto owner_key = [&](const int *cells, int n, uint32_t &key, int &loc) {
        int lmax = -1;
        for (int j = 0; j < n; ++j) if (cells[j] >= 0) lmax = std::max(lmax, lev[cells[j]]);
        int ki = INT32_MAX, ko = -1;
        loc = INT32_MAX;
        for (int j = 0; j < n; ++j) {
            int c = cells[j];
            if (c < 0 || lev[c] != lmax) continue;
            ki = std::min(ki, kin[c]);
            ko = std::max(ko, kout[c]);
            loc = std::min(loc, hm.cell_o2n[c]);
        }
        key = BandKey::make(L, lmax, ki, ko);
    };
    std::vector<uint32_t> ek(nE), vk(nV);
    std::vector<int> eloc(nE), vloc(nV);
    for (int e = 0; e < nE; ++e) owner_key(coe + 2 * e, 2, ek[e], eloc[e]);
    for (int v = 0; v < nV; ++v) owner_key(cov + 3 * v, 3, vk[v], vloc[v]);
    hm.edge_n2o.resize(nE);
    std::iota(hm.edge_n2o.begin(), hm.edge_n2o.end(), 0);
    std::sort(hm.edge_n2o.begin(), hm.edge_n2o.end(), [&](int a, int b) {
        if (ek[a] != ek[b]) return ek[a] < ek[b];
        if (eloc[a] != eloc[b]) return eloc[a] < eloc[b];
        return a < b;
    });
    hm.vert_n2o.resize(nV);
    std::iota(hm.vert_n2o.begin(), hm.vert_n2o.end(), 0);
    std::sort(hm.vert_n2o.begin(), hm.vert_n2o.end(), [&](int a, int b) {
        if (vk[a] != vk[b]) return vk[a] < vk[b];
        if (vloc[a] != vloc[b]) return vloc[a] < vloc[b];
        return a < b;
    });
    hm.edge_o2n.assign(nE, -1);
    for (int i = 0; i < nE; ++i) hm.edge_o2n[hm.edge_n2o[i]] = i;
    hm.vert_o2n.assign(nV, -1);
    for (int i = 0; i < nV; ++i) hm.vert_o2n[hm.vert_n2o[i]] = i;
    hm.ckey.resize(nC); hm.ekey.resize(nE); hm.vkey.resize(nV); hm.level.resize(nC);
    for (int i = 0; i < nC; ++i) { hm.ckey[i] = ck[hm.cell_n2o[i]]; hm.level[i] = lev[hm.cell_n2o[i]]; }
    for (int i = 0; i < nE; ++i) hm.ekey[i] = ek[hm.edge_n2o[i]];
    for (int i = 0; i < nV; ++i) hm.vkey[i] = vk[hm.vert_n2o[i]];

    // ---------------------------------------------------------- new-order arrays
    const auto &c2n = hm.cell_o2n, &e2n = hm.edge_o2n, &v2n = hm.vert_o2n;
    hm.nEoC.resize(nC); hm.eoc.assign((size_t)nC * W, 0); hm.coc.assign((size_t)nC * W, 0);
    hm.cDiv.assign((size_t)nC * W, 0.0); hm.cKE.assign((size_t)nC * W, 0.0);
    hm.area.resize(nC);
    for (int i = 0; i < nC; ++i) {
        int io = hm.cell_n2o[i];
        int n = d->nEdgesOnCell[io];
        double A = d->areaCell[io];
        hm.nEoC[i] = n;
        hm.area[i] = A;
        for (int j = 0; j < n; ++j) {
            int eo = d->edgesOnCell[(size_t)io * mE + j];
            size_t k = (size_t)i * W + j;
            hm.eoc[k] = e2n[eo];
            if (ebnd[eo]) {
                hm.coc[k] = i;
                continue;  // no-flow edge: no flux, no kinetic energy (u = 0)
            }
            int other = coe[2 * eo] == io ? coe[2 * eo + 1] : coe[2 * eo];
            double sgn = coe[2 * eo] == io ? 1.0 : -1.0;   // n_{e,i}
            hm.coc[k] = c2n[other];
            hm.cDiv[k] = -sgn * d->dvEdge[eo] / A;
            hm.cKE[k] = 0.25 * d->dcEdge[eo] * d->dvEdge[eo] / A;
        }
        for (int j = n; j < W; ++j) {  // padding: harmless entries
            size_t k = (size_t)i * W + j;
            hm.eoc[k] = hm.eoc[(size_t)i * W];
            hm.coc[k] = i;
        }
    }
    hm.coe.resize(2 * (size_t)nE); hm.voe.resize(2 * (size_t)nE); hm.ebnd.resize(nE);
    hm.nEoE.resize(nE); hm.eoe.assign((size_t)nE * W2, 0); hm.woe.assign((size_t)nE * W2, 0.0);
    hm.invDc.resize(nE);
    hm.has_angle = d->angleEdge != nullptr;
    hm.has_xy_cell = d->xCell && d->yCell;
    hm.has_xy_edge = d->xEdge && d->yEdge;
    hm.cosE.assign(nE, 1.0); hm.sinE.assign(nE, 0.0); hm.xE.assign(nE, 0.0); hm.yE.assign(nE, 0.0);
    hm.xC.assign(nC, 0.0); hm.yC.assign(nC, 0.0);
    for (int e = 0; e < nE; ++e) {
        int eo = hm.edge_n2o[e];
        int a = coe[2 * eo], b = coe[2 * eo + 1];
        hm.ebnd[e] = ebnd[eo];
        if (ebnd[eo]) {
            int p = a >= 0 ? a : b;
            hm.coe[2 * e] = hm.coe[2 * e + 1] = c2n[p];
        } else {
            hm.coe[2 * e] = c2n[a];
            hm.coe[2 * e + 1] = c2n[b];
        }
        int v0 = voe[2 * eo], v1 = voe[2 * eo + 1];
        if (v0 < 0) v0 = v1;
        if (v1 < 0) v1 = v0;
        hm.voe[2 * e] = v0 >= 0 ? v2n[v0] : 0;
        hm.voe[2 * e + 1] = v1 >= 0 ? v2n[v1] : 0;
        hm.invDc[e] = ebnd[eo] ? 0.0 : 1.0 / d->dcEdge[eo];
        int ne = ebnd[eo] ? 0 : d->nEdgesOnEdge[eo];
        hm.nEoE[e] = ne;
        for (int j = 0; j < ne; ++j) {
            hm.eoe[(size_t)e * W2 + j] = e2n[d->edgesOnEdge[(size_t)eo * mE2 + j]];
            hm.woe[(size_t)e * W2 + j] = d->weightsOnEdge[(size_t)eo * mE2 + j];
        }
        for (int j = ne; j < W2; ++j) hm.eoe[(size_t)e * W2 + j] = e;
        if (hm.has_angle) { hm.cosE[e] = std::cos(d->angleEdge[eo]); hm.sinE[e] = std::sin(d->angleEdge[eo]); }
        if (hm.has_xy_edge) { hm.xE[e] = d->xEdge[eo]; hm.yE[e] = d->yEdge[eo]; }
    }
    if (hm.has_xy_cell)
        for (int i = 0; i < nC; ++i) { hm.xC[i] = d->xCell[hm.cell_n2o[i]]; hm.yC[i] = d->yCell[hm.cell_n2o[i]]; }
    hm.cov.resize(3 * (size_t)nV); hm.eov.resize(3 * (size_t)nV);
    hm.cVort.assign(3 * (size_t)nV, 0.0); hm.cKite.assign(3 * (size_t)nV, 0.0);
    hm.fV.resize(nV); hm.Av.resize(nV);
    for (int v = 0; v < nV; ++v) {
        int vo = hm.vert_n2o[v];
        double A = Av[vo];
        hm.Av[v] = A;
        hm.fV[v] = d->fVertex[vo];
        int firstc = -1, firste = -1;
        for (int j = 0; j < 3; ++j) {
            if (cov[3 * vo + j] >= 0 && firstc < 0) firstc = c2n[cov[3 * vo + j]];
            if (eov[3 * vo + j] >= 0 && firste < 0) firste = e2n[eov[3 * vo + j]];
        }
        for (int j = 0; j < 3; ++j) {
            int c = cov[3 * vo + j];
            hm.cov[3 * v + j] = c >= 0 ? c2n[c] : firstc;
            hm.cKite[3 * v + j] = c >= 0 ? d->kiteAreasOnVertex[3 * vo + j] / A : 0.0;
            int e = eov[3 * vo + j];
            if (e >= 0 && !ebnd[e]) {
                double t = voe[2 * e] == vo ? -1.0 : 1.0;   // t_{e,v}
                hm.eov[3 * v + j] = e2n[e];
                hm.cVort[3 * v + j] = t * d->dcEdge[e] / A;
            } else {
                hm.eov[3 * v + j] = e >= 0 ? e2n[e] : (firste >= 0 ? firste : 0);
                hm.cVort[3 * v + j] = 0.0;   // absent or no-flow edge: u = 0
            }
        }
    }
    // signed edge rows and per-edge metrics of the FP32 cell pass
    hm.eocS.assign((size_t)nC * W, 0);
    hm.invA.resize(nC);
    for (int i = 0; i < nC; ++i) {
        hm.invA[i] = 1.0 / hm.area[i];
        for (int j = 0; j < W; ++j) {
            const int e = hm.eoc[(size_t)i * W + j];
            hm.eocS[(size_t)i * W + j] = (j < hm.nEoC[i] && !hm.ebnd[e] && hm.coe[2 * e + 1] == i) ? ~e : e;
        }
    }
    hm.dvE.assign(nE, 0.0);
    hm.keE.assign(nE, 0.0);
    for (int e = 0; e < nE; ++e) {
        const int eo = hm.edge_n2o[e];
        if (hm.ebnd[e]) continue;
        hm.dvE[e] = d->dvEdge[eo];
        hm.keE[e] = 0.25 * d->dcEdge[eo] * d->dvEdge[eo];
    }
    // Neighbour edges of the FP32 edge pass from the two cells' edge rows, with
    // the weights re-derived from kite fractions (see HostMesh::rows_canonical).
    // R[i][k] = kite of cell i at the counter-clockwise end of its edge slot k / A_i;
    // P[i][k] = sum_{s<k} R[i][s].  For e at slot p and e' at slot j of cell i,
    // the kite sum from e counter-clockwise up to e' is P[j] - P[p] (+1 when j < p),
    // and W_{e,e'} = n_{e,i} n_{e',i} (1/2 - that sum) l_{e'} / d_e.
    hm.rowS = W <= 8 ? 8 : 12;
    hm.rows_canonical = W <= 12;
    hm.rowE.assign((size_t)nC * hm.rowS, 0);
    hm.rowP.assign((size_t)nC * hm.rowS, 0.0);
    hm.rowN.assign((size_t)nC * hm.rowS, 0);
    hm.rowV.assign((size_t)nC * hm.rowS, 0);
    for (int i = 0; i < nC && hm.rows_canonical; ++i) {
        const int io = hm.cell_n2o[i], n = hm.nEoC[i];
        double P = 0.0;
        for (int k = 0; k < hm.rowS; ++k) {
            const size_t r = (size_t)i * hm.rowS + k;
            hm.rowE[r] = k < n ? hm.eocS[(size_t)i * W + k] : hm.eoc[(size_t)i * W];
            hm.rowP[r] = k < n ? P : 0.0;
            hm.rowN[r] = k < n ? hm.coc[(size_t)i * W + k] : i;
            hm.rowV[r] = hm.rowV[(size_t)i * hm.rowS];
            if (k >= n) continue;
            const int eo = hm.edge_n2o[hm.eoc[(size_t)i * W + k]];
            const int vend = coe[2 * eo] == io ? voe[2 * eo + 1] : voe[2 * eo];
            hm.rowV[r] = vend >= 0 ? v2n[vend] : 0;
            double kite = 0.0;
            bool found = false;
            if (vend >= 0)
                for (int j = 0; j < 3; ++j)
                    if (cov[3 * vend + j] == io) { kite = d->kiteAreasOnVertex[3 * vend + j]; found = true; }
            if (!found) { hm.rows_canonical = false; break; }
            P += kite / d->areaCell[io];
        }
    }
    hm.eslot.assign(nE, 0);
    for (int e = 0; e < nE && hm.rows_canonical; ++e) {
        if (hm.ebnd[e]) continue;
        const double wscale = 1e-9;
        int matched = 0;
        int slot[2] = {0, 0}, cnt[2] = {0, 0};
        for (int side = 0; side < 2 && hm.rows_canonical; ++side) {
            const int c = hm.coe[2 * e + side];
            const int n = hm.nEoC[c];
            int p = -1;
            for (int j = 0; j < n; ++j) if (hm.eoc[(size_t)c * W + j] == e) p = j;
            if (p < 0) { hm.rows_canonical = false; break; }
            slot[side] = p;
            cnt[side] = n;
            const double *P = &hm.rowP[(size_t)c * hm.rowS];
            for (int j = 0; j < n; ++j) {
                if (j == p) continue;
                const int x = hm.eoc[(size_t)c * W + j];
                const double rs = P[j] - P[p] + (j < p ? 1.0 : 0.0);
                const int xo = hm.edge_n2o[x];
                const double sgn = (side == 0 ? 1.0 : -1.0) * (coe[2 * xo] == hm.cell_n2o[c] ? 1.0 : -1.0);
                const double w = sgn * (0.5 - rs) * d->dvEdge[xo] * hm.invDc[e];
                bool found = false;
                for (int q = 0; q < hm.nEoE[e]; ++q)
                    if (hm.eoe[(size_t)e * W2 + q] == x) {
                        found = true;
                        ++matched;
                        if (std::fabs(hm.woe[(size_t)e * W2 + q] - w) > wscale * (1.0 + std::fabs(w)))
                            hm.rows_canonical = false;
                    }
                if (!found && std::fabs(w) > wscale) hm.rows_canonical = false;
            }
        }
        if (!hm.rows_canonical) break;
        if (matched != hm.nEoE[e]) hm.rows_canonical = false;   // a neighbour outside the two cells
        hm.eslot[e] = (uint16_t)(slot[0] | (slot[1] << 4) | (cnt[0] << 8) | (cnt[1] << 12));
    }
    hm.cells_per_level = per_level;
    int64_t cu = 0, mult = 1;
    for (int l = 0; l < L; ++l) {
        cu += per_level[l] * mult;
        if (l + 1 < L) mult *= hm.M[l];
    }
    hm.cell_updates_per_step = cu;
    return FBLTS_OK;
}

}  // namespace fblts
