// Builds the launch list of one coarse FB-LTS step (Sec. 2.2) over the
// band-ordered index ranges of a HostMesh.
//
// One FB-RK(3,2) stage (Eq. fbrk32) is four passes:
//   cell  : h_s = h0 + c tau Psi(u_in, h_in), FB average, kinetic energy K
//   vertex: q = (zeta(u_in) + f) / h_v(FB average)
//   eprep : per edge F = h_e u_in and q_e
//   edge  : u_s = u0 + c tau Phi(u_in, FB average)
// Each pass covers the contiguous ranges of its step; the kinetic-energy,
// vertex and edge-prep ranges are derived from what the edge pass reads.
//
// Level pair (l, l+1) uses the paper's shrinking sets in the coarse
// advancement (cells F^5 / F^3 / F^1, edges F_E^4 / F_E^2 / IF-1, plus the
// coarse level), saves the IF-1 data, and for k = 0..M-1 writes the
// predictions on IF-1 (Eq. preds, Eq. hstar_preds) and runs the fine step
// (FB-RK on the finest level, or the next level pair).  The stage-3 passes of
// that fine step also accumulate the correction sums of IF-1 and IF-2 (Eq.
// if_correction); FINAL applies them.  Interior coarse cells and edges are
// updated in place by the coarse stage 3.
#include <algorithm>
#include <array>
#include <map>
#include <utility>

#include "fblts_internal.h"

namespace fblts {

namespace {

struct AccInfo {
    bool on = false;
    int c_lo = 0, c_hi = 0, e_lo = 0, e_hi = 0;
    bool set = false;
};

class Builder {
public:
    Builder(const HostMesh &hm, const double beta[3], Schedule &s) : hm_(hm), s_(s) {
        b_[0] = beta[0]; b_[1] = beta[1]; b_[2] = beta[2];
    }

    void top(double dt) { step(0, dt, AccInfo{}); }

private:
    const HostMesh &hm_;
    Schedule &s_;
    double b_[3];
    std::map<std::pair<int, int>, std::array<int, 6>> memo_;

    uint32_t key(int l, int kin, int kout) const { return BandKey::make(hm_.L, l, kin, kout); }
    // level block [start, end) of cells / edges / vertices
    int cblk0(int l) const { return hm_.cell_lb(key(l, 0, 0)); }
    int cblk1(int l) const { return hm_.cell_lb(key(l, 0, 0) + (1u << 16)); }
    int eblk0(int l) const { return hm_.edge_lb(key(l, 0, 0)); }
    int eblk1(int l) const { return hm_.edge_lb(key(l, 0, 0) + (1u << 16)); }
    // inner bands of level l: first index with inner distance >= d
    int cin(int l, int d) const { return hm_.cell_lb(key(l, d, 0)); }
    int ein(int l, int d) const { return hm_.edge_lb(key(l, d, 0)); }
    // outer F^b band of level f starts here (ends at the block end)
    int cband(int f, int b) const { return hm_.cell_lb(key(f, hm_.kin_cap, 6 - b)); }
    int eband(int f, int b) const { return hm_.edge_lb(key(f, hm_.kin_cap, 6 - b)); }

    // dependency ranges of an edge range [a, b): K cells, prep edges, vertices
    std::array<int, 6> deps(int a, int b) {
        auto it = memo_.find({a, b});
        if (it != memo_.end()) return it->second;
        int kmin = INT32_MAX, kmax = -1, pmin = INT32_MAX, pmax = -1;
        for (int e = a; e < b; ++e) {
            for (int s = 0; s < 2; ++s) {
                kmin = std::min(kmin, hm_.coe[2 * e + s]);
                kmax = std::max(kmax, hm_.coe[2 * e + s]);
            }
            pmin = std::min(pmin, e);
            pmax = std::max(pmax, e);
            for (int j = 0; j < hm_.nEoE[e]; ++j) {
                int x = hm_.eoe[(size_t)e * hm_.maxE2 + j];
                pmin = std::min(pmin, x);
                pmax = std::max(pmax, x);
            }
        }
        int vmin = INT32_MAX, vmax = -1;
        for (int e = pmin; e <= pmax; ++e)
            for (int s = 0; s < 2; ++s) {
                vmin = std::min(vmin, hm_.voe[2 * e + s]);
                vmax = std::max(vmax, hm_.voe[2 * e + s]);
            }
        std::array<int, 6> r{kmin, kmax + 1, pmin, pmax + 1, vmin, vmax + 1};
        memo_[{a, b}] = r;
        return r;
    }

    static void add_seg(Op &op, int b, int e, int mode) {
        if (e <= b) return;
        op.seg[op.nseg].begin = b;
        op.seg[op.nseg].end = e;
        op.seg[op.nseg].mode = mode;
        op.nseg++;
    }

    // cover [lo, hi) with the given segments, filling gaps with KONLY
    static void close_cells(Op &op, int lo, int hi) {
        std::sort(op.seg, op.seg + op.nseg, [](const Seg &x, const Seg &y) { return x.begin < y.begin; });
        Seg out[MAX_SEG];
        int n = 0, cur = lo;
        for (int i = 0; i < op.nseg; ++i) {
            if (op.seg[i].begin > cur) out[n++] = Seg{cur, op.seg[i].begin, SEG_KONLY};
            out[n++] = op.seg[i];
            cur = std::max(cur, op.seg[i].end);
        }
        if (hi > cur) out[n++] = Seg{cur, hi, SEG_KONLY};
        op.nseg = n;
        for (int i = 0; i < n; ++i) op.seg[i] = out[i];
        op.lo = lo;
        op.hi = hi;
    }

    // one FB-RK stage: cell segments, edge segments, arrays, coefficient
    void stage(int s, double tau, std::vector<Seg> csegs, std::vector<Seg> esegs) {
        const int in_u = s == 1 ? A_U : (s == 2 ? A_US1 : A_US2);
        const int in_h = s == 1 ? A_H : (s == 2 ? A_HS1 : A_HS2);
        const int hst = s == 1 ? A_HST1 : (s == 2 ? A_HST2 : A_HST3);
        const int out_h = s == 1 ? A_HS1 : (s == 2 ? A_HS2 : A_HS3);
        const int out_u = s == 1 ? A_US1 : (s == 2 ? A_US2 : A_US3);
        const double cdt = (s == 1 ? tau / 3.0 : (s == 2 ? tau / 2.0 : tau));
        // dependency ranges of the edge pass
        int elo = INT32_MAX, ehi = -1;
        for (auto &g : esegs) if (g.end > g.begin) { elo = std::min(elo, g.begin); ehi = std::max(ehi, g.end); }
        int klo = INT32_MAX, khi = -1, plo = INT32_MAX, phi = -1, vlo = INT32_MAX, vhi = -1;
        for (auto &g : esegs) {
            if (g.end <= g.begin) continue;
            auto r = deps(g.begin, g.end);
            klo = std::min(klo, r[0]); khi = std::max(khi, r[1]);
            plo = std::min(plo, r[2]); phi = std::max(phi, r[3]);
            vlo = std::min(vlo, r[4]); vhi = std::max(vhi, r[5]);
        }
        // cell pass
        Op c;
        c.kind = OP_CELL; c.stage = s; c.in_u = in_u; c.in_h = in_h; c.h0 = A_H; c.u0 = A_U;
        c.hprev = A_HS2; c.out_h = out_h; c.hst = hst; c.cdt = cdt;
        if (s == 1) { c.fb_a = b_[0]; c.fb_b = 0.0; c.fb_c = 1.0 - b_[0]; }
        if (s == 2) { c.fb_a = b_[1]; c.fb_b = 0.0; c.fb_c = 1.0 - b_[1]; }
        if (s == 3) { c.fb_a = b_[2]; c.fb_b = 1.0 - 2.0 * b_[2]; c.fb_c = b_[2]; }
        int clo = INT32_MAX, chi = -1;
        for (auto &g : csegs) {
            if (g.end <= g.begin) continue;
            add_seg(c, g.begin, g.end, g.mode);
            clo = std::min(clo, g.begin);
            chi = std::max(chi, g.end);
        }
        if (khi > 0) { clo = std::min(clo, klo); chi = std::max(chi, khi); }
        close_cells(c, clo, chi);
        s_.ops.push_back(c);
        if (ehi <= elo) return;
        // vertex pass
        Op v;
        v.kind = OP_VERT; v.stage = s; v.in_u = in_u; v.hst = hst; v.lo = vlo; v.hi = vhi;
        add_seg(v, vlo, vhi, SEG_UPD);
        s_.ops.push_back(v);
        // edge prep
        Op p;
        p.kind = OP_EPREP; p.stage = s; p.in_u = in_u; p.hst = hst; p.lo = plo; p.hi = phi;
        add_seg(p, plo, phi, SEG_UPD);
        s_.ops.push_back(p);
        // edge pass
        Op e;
        e.kind = OP_EDGE; e.stage = s; e.in_u = in_u; e.hst = hst; e.u0 = A_U; e.out_u = out_u; e.cdt = cdt;
        for (auto &g : esegs) add_seg(e, g.begin, g.end, g.mode);
        e.lo = elo; e.hi = ehi;
        s_.ops.push_back(e);
    }

    void acc_segs(const AccInfo &acc, std::vector<Seg> &cs, std::vector<Seg> &es) {
        if (!acc.on) return;
        const int m = acc.set ? SEG_ACC_SET : SEG_ACC_ADD;
        cs.push_back(Seg{acc.c_lo, acc.c_hi, m});
        es.push_back(Seg{acc.e_lo, acc.e_hi, m});
    }

    // FB-RK(3,2) on all cells of level >= f (f is the finest level)  [Eq. fine_fbrk32]
    void fbrk(int f, double tau, const AccInfo &acc) {
        const int ce = cblk1(f), ee = eblk1(f);
        stage(1, tau, {Seg{0, ce, SEG_UPD}}, {Seg{0, ee, SEG_UPD}});
        stage(2, tau, {Seg{0, ce, SEG_UPD}}, {Seg{0, ee, SEG_UPD}});
        std::vector<Seg> cs{Seg{0, ce, SEG_INPLACE}}, es{Seg{0, ee, SEG_INPLACE}};
        acc_segs(acc, cs, es);
        stage(3, tau, cs, es);
    }

    // FB-LTS step of the pair (l, l+1)  [Sec. 2.2 steps 1-4]
    void fblts(int l, double tau, const AccInfo &acc) {
        const int f = l + 1;
        const int M = hm_.M[l];
        const int nI1 = hm_.nIF1, nI12 = hm_.nIF1 + hm_.nIF2;
        const int cb0 = cblk0(l), cb1 = cblk1(l), eb0 = eblk0(l), eb1 = eblk1(l);
        const int cIF2 = cin(l, nI1 + 1), cINT = cin(l, nI12 + 1);
        const int eIF2 = ein(l, nI1 + 1), eINT = ein(l, nI12 + 1);
        // step 1: coarse advancement on the shrinking sets
        stage(1, tau, {Seg{cband(f, 5), cb1, SEG_UPD}}, {Seg{eband(f, 4), eb1, SEG_UPD}});
        stage(2, tau, {Seg{cband(f, 3), cb1, SEG_UPD}}, {Seg{eband(f, 2), eb1, SEG_UPD}});
        std::vector<Seg> cs{Seg{cband(f, 1), cINT, SEG_UPD}, Seg{cINT, cb1, SEG_INPLACE}};
        std::vector<Seg> es{Seg{eb0, eIF2, SEG_UPD}, Seg{eINT, eb1, SEG_INPLACE}};
        acc_segs(acc, cs, es);
        stage(3, tau, cs, es);
        // step 2 inputs: save h^n, u^n on IF-1 u IF-2 and the IF-1 stage data
        Op sv;
        sv.kind = OP_SAVE; sv.level = l;
        sv.c_if1_lo = cb0; sv.c_if1_hi = cIF2; sv.c_if12_hi = cINT;
        sv.e_if1_lo = eb0; sv.e_if1_hi = eIF2; sv.e_if12_hi = eINT;
        sv.lo = 0; sv.hi = std::max(cINT - cb0, eINT - eb0);
        s_.ops.push_back(sv);
        // step 3: fine advancement with the predictions of step 2
        for (int k = 0; k < M; ++k) {
            Op pr = sv;
            pr.kind = OP_PRED; pr.k = k; pr.Mk = M;
            pr.fb_a = b_[0]; pr.fb_b = b_[1]; pr.fb_c = b_[2];
            pr.hi = std::max(cIF2 - cb0, eIF2 - eb0);
            s_.ops.push_back(pr);
            AccInfo in;
            in.on = true; in.c_lo = cb0; in.c_hi = cINT; in.e_lo = eb0; in.e_hi = eINT; in.set = (k == 0);
            step(f, tau / (double)M, in);
        }
        // step 4: interface correction
        Op fi = sv;
        fi.kind = OP_FINAL; fi.cdt = tau / (double)M;
        s_.ops.push_back(fi);
    }

    void step(int l, double tau, const AccInfo &acc) {
        if (l + 1 >= hm_.L) fbrk(l, tau, acc);
        else fblts(l, tau, acc);
    }
};

}  // namespace

// Algorithmic bytes of one launch: each array element its arithmetic reads or
// writes, once, at storage size (int32 4, double 8, float 4, flag 1).
// Gathered arrays count one read per source element, from the incidence of
// the mesh: a pass over edges that gathers a cell array reads 2 nC/nE cell
// elements per edge (2 cpe, cpe = nC/nE), a vertex array 2 nV/nE (2 vpe).
// fp32: stage data, kinetic energy, PV, fluxes and coefficients in float; the
// time level, the divergence coefficients and the correction sums in double.
void schedule_bytes(const HostMesh &hm, int forcing, bool fp32, Schedule &s) {
    std::vector<double> pc(hm.nC + 1, 0.0), pe(hm.nE + 1, 0.0);
    for (int i = 0; i < hm.nC; ++i) pc[i + 1] = pc[i] + hm.nEoC[i];
    for (int e = 0; e < hm.nE; ++e) pe[e + 1] = pe[e] + hm.nEoE[e];
    const double cpe = (double)hm.nC / hm.nE, vpe = (double)hm.nV / hm.nE;
    const double R = fp32 ? 4.0 : 8.0;        // stage / scratch element
    const double C = fp32 ? 4.0 : 8.0;        // coefficient element
    for (Op &op : s.ops) {
        double b = 0.0;
        switch (op.kind) {
            case OP_CELL:
                for (int k = 0; k < op.nseg; ++k) {
                    const Seg &g = op.seg[k];
                    const double n = g.end - g.begin, slots = pc[g.end] - pc[g.begin];
                    if (fp32) {
                        // nEoC, 1/A, K | signed edge row, u_in and the 16-byte edge record
                        // {l_e, d_e l_e/4, H_e} (an edge has 2 cells)
                        b += n * (4 + 8 + 4) + slots * (4 + 2 + 8);
                        if (g.mode == SEG_KONLY) continue;
                        b += n * 4 + slots * 4;                      // xi_in | coc
                    } else {
                        // nEoC, K out | eoc, cKE, u_in (an edge is gathered by 2 cells)
                        b += n * (4 + 8) + slots * (4 + 8 + 4);
                        if (g.mode == SEG_KONLY) continue;
                        b += n * 8 + slots * (4 + 8);                // h_in | coc, cDiv
                    }
                    if (g.mode == SEG_UPD) b += n * R * (3 + (op.stage == 3 ? 1 : 0));
                    if (g.mode == SEG_INPLACE)
                        b += n * (fp32 ? (8 + 8 + 8 + 4 + 4 + 4) : (8 + 8 + 8)) + n * (op.stage == 3 ? R : 0);
                    if (g.mode == SEG_ACC_SET) b += n * 8;
                    if (g.mode == SEG_ACC_ADD) b += n * 16;
                }
                break;
            case OP_VERT:
                b = (double)(op.hi - op.lo) * (3 * (4 + 4 + C + C) + C + (fp32 ? 4 : 0) + 1.5 * R + 0.5 * R + R);
                break;
            case OP_EPREP:   // fp32 writes the 16-byte record {F, q_e, u, 0}
                b = (double)(op.hi - op.lo) * (17 + (fp32 ? 4 : 0) + R + R * 2 * cpe + R * 2 * vpe + (fp32 ? 16 : 3 * R));
                break;
            case OP_EDGE:
                for (int k = 0; k < op.nseg; ++k) {
                    const Seg &g = op.seg[k];
                    const double n = g.end - g.begin, slots = pe[g.end] - pe[g.begin];
                    // ebnd, nEoE, neighbour records (fp32: {F, q_e, u} 16 B; fp64: F, q_e, F q_e),
                    // coe, invDc, K and hst at the cells (+ bottom in double); neighbours: an
                    // index and a weight per slot, or (rows) the two cells' edge rows, each row
                    // shared by the cell's edges, plus the two slots
                    b += n * (1 + 4 + (fp32 ? 16 : 3 * R) + 8 + C + 2 * R * 2 * cpe + (fp32 ? 0 : 8 * 2 * cpe));
                    if (fp32 && hm.rows_canonical)
                        b += n * (2 + 2 * cpe * (4 + 4 * (pc[hm.nC] / hm.nC))) + slots * C;
                    else
                        b += slots * (4 + C);
                    if (g.mode == SEG_UPD) b += n * 2 * R;
                    if (g.mode == SEG_INPLACE) b += n * (fp32 ? (8 + 8 + 4) : 16);
                    if (g.mode == SEG_ACC_SET) b += n * 8;
                    if (g.mode == SEG_ACC_ADD) b += n * 16;
                    if (forcing) b += n * ((fp32 ? 0 : R) + 3 * R + (fp32 ? 4 : 0) + R * 2 * cpe);
                }
                break;
            case OP_SAVE: {
                const double big = fp32 ? (16 + 3 * 8) : 64;   // h^n copy + 3 stage copies
                b = big * (op.c_if1_hi - op.c_if1_lo) + 16.0 * (op.c_if12_hi - op.c_if1_hi) +
                    big * (op.e_if1_hi - op.e_if1_lo) + 16.0 * (op.e_if12_hi - op.e_if1_hi);
            } break;
            case OP_PRED:
                b = (fp32 ? 52.0 : 80.0) * (op.c_if1_hi - op.c_if1_lo) +
                    (fp32 ? 32.0 : 56.0) * (op.e_if1_hi - op.e_if1_lo);
                break;
            case OP_FINAL:
                b = (fp32 ? 36.0 : 24.0) * (op.c_if12_hi - op.c_if1_lo) +
                    (fp32 ? 29.0 : 25.0) * (op.e_if12_hi - op.e_if1_lo);
                break;
            case OP_FORCING:
                if (forcing)
                    b = (double)hm.nE * (16 + 3 * R + ((forcing & FBLTS_FORCE_VORTEX) ? 16 : 0)) +
                        (double)hm.nC * (R + ((forcing & FBLTS_FORCE_VORTEX) ? 16 : 0));
                break;
            case OP_STEP_END: b = 16; break;
            default: break;
        }
        op.alg_bytes = b;
    }
}

void build_schedule(const HostMesh &hm, double dt, const double beta[3], Schedule &s) {
    s.ops.clear();
    Op fz;
    fz.kind = OP_FORCING;
    s.ops.push_back(fz);
    Builder b(hm, beta, s);
    b.top(dt);
    Op se;
    se.kind = OP_STEP_END;
    s.ops.push_back(se);
    s.launches = (int64_t)s.ops.size();
}

}  // namespace fblts
