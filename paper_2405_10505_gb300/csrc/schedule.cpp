// Builds the launch list of one coarse FB-LTS step (Sec. 2.2) over the
// band-ordered index ranges of a HostMesh.
//
// One FB-RK(3,2) stage (Eq. fbrk32) is four passes:
//   cell  : h_s = h0 + c tau Psi(u_in, h_in), FB average, kinetic energy K
//   vertex: q = (zeta(u_in) + f) / h_v(FB average)
//   eprep : per edge F = h_e u_in and q_e   (or, with cell rows,
//   trisk : per cell, each of its edges' share of the TRiSK sums and the
//           cell's Bernoulli term K + g xi)
//   edge  : u_s = u0 + c tau Phi(u_in, FB average)
// Each pass covers the contiguous ranges of its step; the kinetic-energy,
// vertex and edge-prep (trisk) ranges are derived from what the edge pass reads.
// With the operator splitting of Sec. 3.2 a slow block (K-only cell pass,
// vertex pass, TRiSK / edge-prep pass, edge pass writing the slow part of Phi)
// opens the coarse step, and with its per-fine-step variant (Sec. 4.2) also
// every fine step; the stages then run only the cell and edge passes.  The
// classical RK4 comparison scheme is four stages of the same passes on a
// one-level mesh.
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
    Builder(const HostMesh &hm, const double beta[3], bool trisk_cells, int split, bool rk4, Schedule &s)
        : hm_(hm), s_(s), trisk_cells_(trisk_cells), split_(split), rk4_(rk4) {
        b_[0] = beta[0]; b_[1] = beta[1]; b_[2] = beta[2];
    }

    void top(double dt) {
        if (rk4_) {
            rk4(dt);
            return;
        }
        // the slow part of Phi at the coarse step's start time level on every edge
        if (split_) slow_block(hm_.nE);
        step(0, dt, AccInfo{});
    }

private:
    const HostMesh &hm_;
    Schedule &s_;
    bool trisk_cells_;
    int split_;   // 0: none, 1: slow terms per coarse step, 2: per step of each level
    bool rk4_;
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
        static const int U_OF[4] = {A_U, A_US1, A_US2, A_US3}, H_OF[4] = {A_H, A_HS1, A_HS2, A_HS3};
        static const int HST_OF[4] = {A_HST1, A_HST2, A_HST3, A_HST1};
        const int in_u = U_OF[s - 1], in_h = H_OF[s - 1];
        const int hst = HST_OF[s - 1];
        const int out_h = H_OF[s < 4 ? s : 0], out_u = U_OF[s < 4 ? s : 0];
        // FB-RK(3,2): c = 1/3, 1/2, 1; RK4: c = 1/2, 1/2, 1 and the final tau/6
        const double cdt = rk4_ ? (s == 1 || s == 2 ? tau / 2.0 : (s == 3 ? tau : tau / 6.0))
                                : (s == 1 ? tau / 3.0 : (s == 2 ? tau / 2.0 : tau));
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
        if (rk4_) {
            // RK4 evaluates Phi at the stage's input state: the "average" is that state
            c.hprev = in_h;
            c.fb_a = 0.0; c.fb_b = 1.0; c.fb_c = 0.0;
        }
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
        if (split_) {
            // operator splitting: Phi = -g grad(h* + b) + the slow part of the step
            Op e;
            e.kind = OP_EDGE; e.stage = s; e.in_u = in_u; e.hst = hst; e.u0 = A_U; e.out_u = out_u; e.cdt = cdt;
            e.split = 2;
            for (auto &g : esegs) add_seg(e, g.begin, g.end, g.mode);
            e.lo = elo; e.hi = ehi;
            s_.ops.push_back(e);
            return;
        }
        // vertex pass
        Op v;
        v.kind = OP_VERT; v.stage = s; v.in_u = in_u; v.hst = hst; v.lo = vlo; v.hi = vhi;
        add_seg(v, vlo, vhi, SEG_UPD);
        s_.ops.push_back(v);
        // edge prep over the edges and their neighbours, or the cell-side TRiSK
        // sums over the cells of the edges
        Op p;
        p.kind = trisk_cells_ ? OP_TRISK : OP_EPREP; p.stage = s; p.in_u = in_u; p.hst = hst;
        p.lo = trisk_cells_ ? klo : plo;
        p.hi = trisk_cells_ ? khi : phi;
        add_seg(p, p.lo, p.hi, SEG_UPD);
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
            if (split_ == 2) slow_block(eb0);   // the fine region's slow terms at t^{n,k}
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

    // The slow part of Phi (Coriolis, kinetic-energy gradient, forcing) on
    // the edges [0, ehi) from the time level (h, u) as it stands: the K-only
    // cell pass, the vertex pass and the TRiSK (edge-prep) pass over what
    // those edges read, then an edge pass writing the slow part per edge
    // [Sec. 3.2, Eq. splitting].  Before a fine step the time level of the
    // fine cells is current and IF-1 holds the predictions X^{n,k}.
    void slow_block(int ehi) {
        if (ehi <= 0) return;
        const auto r = deps(0, ehi);
        Op k;
        k.kind = OP_CELL; k.stage = 1; k.in_u = A_U; k.in_h = A_H; k.hst = A_H; k.split = 1;
        k.seg[0] = Seg{r[0], r[1], SEG_KONLY}; k.nseg = 1; k.lo = r[0]; k.hi = r[1];
        s_.ops.push_back(k);
        Op v;
        v.kind = OP_VERT; v.in_u = A_U; v.hst = A_H; v.split = 1;
        v.seg[0] = Seg{r[4], r[5], SEG_UPD}; v.nseg = 1; v.lo = r[4]; v.hi = r[5];
        s_.ops.push_back(v);
        Op p;
        p.kind = trisk_cells_ ? OP_TRISK : OP_EPREP; p.in_u = A_U; p.hst = A_H; p.split = 1;
        p.lo = trisk_cells_ ? r[0] : r[2];
        p.hi = trisk_cells_ ? r[1] : r[3];
        p.seg[0] = Seg{p.lo, p.hi, SEG_UPD}; p.nseg = 1;
        s_.ops.push_back(p);
        Op e;
        e.kind = OP_EDGE; e.in_u = A_U; e.hst = A_H; e.out_u = A_SLOW; e.split = 1;
        e.seg[0] = Seg{0, ehi, SEG_PHI}; e.nseg = 1; e.lo = 0; e.hi = ehi;
        s_.ops.push_back(e);
    }

    // Classical RK4 on every cell and edge (the comparison integrator of
    // Sec. 4.2): stage s evaluates the tendencies T_s at the state of stage
    // s-1, writes X_s = X^n + c_s tau T_s (c = 1/2, 1/2, 1) and sums
    // T_1 + 2 T_2 + 2 T_3 in the correction-sum arrays; stage 4 applies
    // X^{n+1} = X^n + (tau/6)(sum + T_4) in place.
    void rk4(double tau) {
        static const int MODE[4] = {SEG_RK_SET, SEG_RK_ADD2, SEG_RK_ADD2, SEG_RK_FIN};
        for (int s = 1; s <= 4; ++s)
            stage(s, tau, {Seg{0, hm_.nC, MODE[s - 1]}}, {Seg{0, hm_.nE, MODE[s - 1]}});
    }
};

}  // namespace

namespace {

// Distinct elements that the gathers of one launch touch, counted exactly
// over the union of its segments and memoised by segment list (the fine
// level repeats the same ranges M times per coarse step).
struct Touched {
    double self = 0, slots = 0;        // elements in the segments, row slots read
    double cells = 0, edges = 0, verts = 0;
};

class Toucher {
public:
    explicit Toucher(const HostMesh &hm)
        : hm_(hm), sc_(hm.nC, 0), se_(hm.nE, 0), sv_(hm.nV, 0) {}

    // kind: OP_CELL (cells -> their edges, their neighbour cells and themselves),
    // OP_VERT (vertices -> edges, cells), OP_EPREP (edges -> cells, vertices),
    // OP_EDGE (edges -> cells, listed neighbour edges), OP_TRISK (cells -> edges,
    // neighbour cells and themselves, vertices)
    const Touched &get(int kind, const std::vector<std::pair<int, int>> &ranges) {
        auto key = std::make_pair(kind, ranges);
        auto it = memo_.find(key);
        if (it != memo_.end()) return it->second;
        ++stamp_;
        Touched t;
        auto C = [&](int c) { if (sc_[c] != stamp_) { sc_[c] = stamp_; t.cells += 1; } };
        auto E = [&](int e) { if (se_[e] != stamp_) { se_[e] = stamp_; t.edges += 1; } };
        auto V = [&](int v) { if (sv_[v] != stamp_) { sv_[v] = stamp_; t.verts += 1; } };
        const int W = hm_.maxE, W2 = hm_.maxE2;
        for (const auto &r : ranges)
            for (int x = r.first; x < r.second; ++x) {
                t.self += 1;
                switch (kind) {
                    case OP_TRISK:
                        C(x);
                        t.slots += hm_.nEoC[x];
                        for (int j = 0; j < hm_.nEoC[x]; ++j) {
                            E(hm_.eoc[(size_t)x * W + j]);
                            C(hm_.coc[(size_t)x * W + j]);
                            V(hm_.rowV[(size_t)x * hm_.rowS + j]);
                        }
                        break;
                    case OP_CELL:
                        C(x);
                        t.slots += hm_.nEoC[x];
                        for (int j = 0; j < hm_.nEoC[x]; ++j) {
                            E(hm_.eoc[(size_t)x * W + j]);
                            C(hm_.coc[(size_t)x * W + j]);
                        }
                        break;
                    case OP_VERT:
                        for (int j = 0; j < 3; ++j) { E(hm_.eov[3 * (size_t)x + j]); C(hm_.cov[3 * (size_t)x + j]); }
                        break;
                    case OP_EPREP:
                        C(hm_.coe[2 * (size_t)x]); C(hm_.coe[2 * (size_t)x + 1]);
                        V(hm_.voe[2 * (size_t)x]); V(hm_.voe[2 * (size_t)x + 1]);
                        break;
                    case OP_EDGE:
                        if (hm_.ebnd[x]) break;
                        E(x);
                        C(hm_.coe[2 * (size_t)x]);
                        C(hm_.coe[2 * (size_t)x + 1]);
                        t.slots += hm_.nEoE[x];
                        for (int j = 0; j < hm_.nEoE[x]; ++j) E(hm_.eoe[(size_t)x * W2 + j]);
                        break;
                    default: break;
                }
            }
        return memo_.emplace(key, t).first->second;
    }

private:
    const HostMesh &hm_;
    std::vector<int> sc_, se_, sv_;
    int stamp_ = 0;
    std::map<std::pair<int, std::vector<std::pair<int, int>>>, Touched> memo_;
};

}  // namespace

// Bytes of one launch under two models, each counting every array element once
// per launch at its storage size (int32 4, double 8, float 4, flag 1), with
// gathered arrays counted over the distinct elements the launch touches
// (exact, from the mesh incidence):
//   algorithmic - the arrays the stage's arithmetic needs (Eq. trisk_thickness,
//     Eq. trisk_vorticity, Eq. fbrk32): state, stage values and the
//     intermediates K, q, h*, F, the mesh metadata at its real length (no row
//     padding, no record padding) and with the metric factors per edge and per
//     cell (d_e, l_e, 1/A_i) rather than folded into per-slot copies.  The
//     per-slot shares of the cell-side TRiSK form are an intermediate of this
//     implementation only and count nothing: the math of Phi is counted where
//     its inputs are read.
//   moved - what the kernels of this library read and write: padded rows at
//     their stored width, padded records, per-slot coefficients and the
//     shares (written by the TRiSK pass, read by the edge pass).
// FP32: stage data, kinetic energy, PV and coefficients in float; the time
// level, 1/A and the correction sums in double.
static double op_bytes(const HostMesh &hm, Toucher &tch, const Op &op, int forcing, bool fp32, bool alg) {
    const double R = fp32 ? 4.0 : 8.0;        // stage / scratch element
    const double C = fp32 ? 4.0 : 8.0;        // coefficient element
    const double REC = alg ? 12.0 : 16.0;     // {3 floats} record, padded to 16 bytes in memory
    const bool vortex = (forcing & FBLTS_FORCE_VORTEX) != 0;
    double b = 0.0;
    std::vector<std::pair<int, int>> all;
    for (int k = 0; k < op.nseg; ++k)
        if (op.seg[k].end > op.seg[k].begin) all.emplace_back(op.seg[k].begin, op.seg[k].end);
    auto per_mode = [&](double n, int mode, bool cell) {
        double x = 0.0;
        if (mode == SEG_UPD)   // stage inputs at the element, stage output (+ FB average for cells)
            x = cell ? n * R * (3 + (op.stage == 3 ? 1 : 0)) : n * 2 * R;
        if (mode == SEG_INPLACE) {
            // FP32 cells: the double time level read and written, its float
            // shadow, xi0 and the FB average out (+ the stage-2 xi in stage 3)
            if (cell) x = fp32 ? n * (16 + 4 + 4 + 4 + (op.stage == 3 ? 4 : 0)) : n * (16 + 8 + 8);
            else x = fp32 ? n * (16 + 4) : n * 16;
        }
        if (mode == SEG_ACC_SET) x = n * 8;
        if (mode == SEG_ACC_ADD) x = n * 16;
        if (mode == SEG_PHI) x = n * R;
        // RK4: as SEG_UPD (the previous stage is the element's own input) plus
        // the tendency sum (write, or read and write); the final stage as
        // SEG_INPLACE plus the sum read
        if (mode == SEG_RK_SET || mode == SEG_RK_ADD2) x = n * ((cell ? 3 : 2) * R + (mode == SEG_RK_SET ? 8 : 16));
        if (mode == SEG_RK_FIN) {
            if (cell) x = fp32 ? n * (16 + 4 + 4 + 4 + 8) : n * (16 + 8 + 8);
            else x = fp32 ? n * (16 + 4 + 8) : n * (16 + 8);
        }
        return x;
    };
    switch (op.kind) {
        case OP_CELL: {
            if (all.empty()) break;
            // cells: nEoC, K out, (alg, or fp32) 1/A; rows (signed edge,
            // neighbour cell); edges: u_in and the metrics l_e, d_e l_e / 4
            // (fp32: {l_e, H_e} and d_e l_e / 4; fp64 moved: per-slot
            // coefficients with 1/A folded in); xi / h at the cells.  FP32
            // reads 1/A as a float, and as a double too where the double
            // time level or a correction sum changes
            bool konly = true;
            double ndbl = 0;
            for (int k = 0; k < op.nseg; ++k) {
                konly = konly && op.seg[k].mode == SEG_KONLY;
                if (op.seg[k].mode != SEG_KONLY && op.seg[k].mode != SEG_UPD) ndbl += op.seg[k].end - op.seg[k].begin;
            }
            const Touched &t = tch.get(OP_CELL, all);
            // moved, FP32 with cell rows: both rows at their stored width and
            // the neighbour thickness gathered in every launch (the kernel
            // issues all its loads in one round, K-only cells included)
            const bool rows = !alg && fp32 && hm.rows_canonical;
            b += t.self * (4 + R) + (rows ? t.self * hm.rowS * 8 : t.slots * 4) + t.edges * R;
            if (fp32) b += t.self * 4 + ndbl * 8 + t.edges * 12;
            else if (alg) b += t.self * 8 + t.edges * 2 * C;
            else b += t.slots * C;                                  // cKE per slot
            if (rows) b += t.cells * R;
            else if (!konly) b += t.slots * (4 + (fp32 || alg ? 0 : C)) + t.cells * R;   // coc (+ cDiv), h_in
            if (!konly && !fp32) b += t.edges * 8;                  // H_e
            for (int k = 0; k < op.nseg; ++k)
                b += per_mode(op.seg[k].end - op.seg[k].begin, op.seg[k].mode, true);
        } break;
        case OP_VERT: {
            const std::vector<std::pair<int, int>> r = {{op.lo, op.hi}};
            const Touched &t = tch.get(OP_VERT, r);
            // eov, cov, t d / A_v, kite / A_v, f, H_v, q out | u_in, hst
            b = t.self * (3 * (4 + 4 + C + C) + C + C + R) + t.edges * R + t.cells * R;
        } break;
        case OP_EPREP: {
            const std::vector<std::pair<int, int>> r = {{op.lo, op.hi}};
            const Touched &t = tch.get(OP_EPREP, r);
            // coe, voe, u_in, (fp32) l_e, H_e and the record {l F, q_e, l u} out,
            // (fp64) ebnd, H_e and F, q_e, F q_e out | hst at cells, q at vertices
            b = t.self * (16 + R + (fp32 ? 4 + 4 + REC : 1 + 8 + 3 * R)) + t.cells * R + t.verts * R;
        } break;
        case OP_TRISK: {
            const std::vector<std::pair<int, int>> r = {{op.lo, op.hi}};
            const Touched &t = tch.get(OP_TRISK, r);
            // cells: nEoC, K, rows {signed edge, kite prefix, neighbour cell,
            // vertex} (moved: at their stored width, and one 8-byte share out
            // per slot), (vortex) p_s | edges: u_in, l_e and H_e (moved: the
            // record {l_e, H_e}) | hst at the cells and their neighbours
            // | q at the vertices
            const double rows = alg ? t.slots * 16 : t.self * hm.rowS * 16;
            b = t.self * (4 + R + (vortex ? R : 0)) + rows + t.edges * (R + (alg ? 2 * C : 8)) + t.cells * R +
                t.verts * R;
            if (!alg) b += t.slots * 8 + t.self * 8;   // shares {t, s_v}, the cell's {B, xi*}
        } break;
        case OP_EDGE: {
            if (all.empty()) break;
            if (op.split == 2) {
                // splitting stage: ebnd, coe, 1/d_e, the slow part | the FB-averaged
                // surface elevation at the cells
                const Touched &t = tch.get(OP_EPREP, all);
                b += t.self * (1 + 8 + C + R) + t.cells * R;
                for (int k = 0; k < op.nseg; ++k)
                    b += per_mode(op.seg[k].end - op.seg[k].begin, op.seg[k].mode, false);
                break;
            }
            if (fp32 && hm.rows_canonical) {
                // ebnd, 1/d_e (moved: the two cells' 8-byte shares, coe and the
                // cells' {B, xi*} records)
                for (int k = 0; k < op.nseg; ++k) {
                    const double n = op.seg[k].end - op.seg[k].begin;
                    b += n * (1 + 4 + (alg ? 0 : 16 + 8)) + per_mode(n, op.seg[k].mode, false);
                    if (forcing) b += n * (R + 4 + 3 * R);   // u_in, H_e, wind, C_W
                }
                if (!alg) b += tch.get(OP_EPREP, all).cells * 8;
                break;
            }
            const Touched &t = tch.get(OP_EDGE, all);
            // explicit neighbour lists: ebnd, coe, invDc | K, hst at cells |
            // neighbour records | nEoE, eoe, woe
            b += t.self * (1 + 8 + C) + t.cells * 2 * R;
            if (fp32) b += t.edges * REC;                 // {l F, q_e, l u} (own q_e included)
            else b += t.edges * 2 * R + t.self * R;       // F, F q_e at the neighbours, own q_e
            b += t.self * 4 + t.slots * (4 + C);
            if (forcing) {
                // u_in (fp64: at the neighbours too), H_e, wind, C_W; surface pressure at cells
                b += fp32 ? t.self * (R + 4 + 3 * R) : t.self * (3 * R + 8) + t.edges * R;
                if (vortex) b += t.cells * R;
            }
            for (int k = 0; k < op.nseg; ++k)
                b += per_mode(op.seg[k].end - op.seg[k].begin, op.seg[k].mode, false);
        } break;
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
                b = (double)hm.nE * (16 + 3 * R + (vortex ? 16 : 0)) + (double)hm.nC * (R + (vortex ? 16 : 0));
            break;
        case OP_STEP_END: b = 16; break;
        default: break;
    }
    return b;
}

void schedule_bytes(const HostMesh &hm, int forcing, bool fp32, Schedule &s) {
    Toucher tch(hm);
    for (Op &op : s.ops) {
        op.alg_bytes = op_bytes(hm, tch, op, forcing, fp32, true);
        op.moved_bytes = op_bytes(hm, tch, op, forcing, fp32, false);
    }
}

void build_schedule(const HostMesh &hm, double dt, const double beta[3], bool trisk_cells, int split, bool rk4,
                    Schedule &s) {
    s.ops.clear();
    Op fz;
    fz.kind = OP_FORCING;
    s.ops.push_back(fz);
    Builder b(hm, beta, trisk_cells, rk4 ? 0 : split, rk4, s);
    b.top(dt);
    Op se;
    se.kind = OP_STEP_END;
    s.ops.push_back(se);
    s.launches = (int64_t)s.ops.size();
}

}  // namespace fblts
