// FP32-tendency bodies: the same passes as kernel_bodies.cuh with tendency
// arithmetic and stage data in float, thickness as xi = h - H, and the time
// level (h, u), the correction sums and the global sums in double.
#pragma once

#include "kernel_bodies.cuh"

namespace fblts {

struct CellArgs32 {
    SegSet segs;
    int lo, hi;
    const float *u_in, *xi_in, *xi0, *xiprev;   // stage inputs, xi of h0, stage-2 xi
    float *xi_out, *xi_shadow, *hst_out, *K;
    double *h_state, *acc;      // the double time level (xi) and the correction sums
    double cdt;
    float cdtf;                 // c tau rounded to float (float stage values)
    float fb_a, fb_b, fb_c;
};

struct VertArgs32 {
    int lo, hi;
    const float *u_in, *hst;
    float *q;
};

struct PrepArgs32 {
    int lo, hi;
    const float *u_in, *hst, *q;
    float4 *fqu;      // per edge {F_e, q_e, u_e, 0}
};

// row slots gathered unconditionally by the FP32 row kernels (hexagon-dominated
// meshes); longer rows take a branch for the rest
constexpr int ROW_MAIN = 6;

// Cell-side TRiSK pass: per slot of each cell, the share {t, s_v} of the
// cell in its edge's momentum tendency (trisk32_body), written to
// sh[2 e + side] (side 0 = first cell of e), and per cell {B_i, xi*_i} to
// bx[i]; both live in the A_FQU area (shares first, 4 floats per edge).
struct TriskArgs32 {
    int lo, hi;
    const float *u_in, *hst, *K, *q;
    float2 *sh, *bx;
    float g, inv_rho0;
};

struct EdgeArgs32 {
    SegSet segs;
    int lo, hi;
    const float *u_in, *hst, *K, *u0;
    const float4 *fqu;
    const float2 *sh, *bx;   // the TRiSK pass's shares and per-cell {B, xi*}
    float *us_out, *u_shadow;
    double *u_state, *acc;
    const float *slow;   // splitting: the slow part of Phi per edge
    double cdt;
    float cdtf;          // c tau rounded to float (float stage values)
    float g;
    int split;           // 0, or 1: slow-term evaluation, 2: stage with Phi = fast + slow
};

struct IfArgs32 {
    int c_lo, c_if1_hi, c_if12_hi, e_lo, e_if1_hi, e_if12_hi, n;
    double *h, *u, *sh0, *su0, *acch, *accu;
    float *xi, *u32, *hs1, *hs2, *hs3, *hst1, *hst2, *hst3, *us1, *us2, *us3;
    float *sh1, *sh2, *sh3, *su1, *su2, *su3;
    int k, M;
    float b1, b2, b3;
    double cf;
};

// the float view of an array id: the time level reads its float shadow
inline const float *f_in(const DevArrays &arr, int id) {
    if (id == A_H) return arr.xi32;
    if (id == A_U) return arr.u32;
    return arr.f[id];
}

inline CellArgs32 cell_args32(const Op &op, const DevArrays &arr, const DevMesh &m) {
    CellArgs32 a;
    a.segs = segs_of(op);
    a.lo = op.lo; a.hi = op.hi;
    a.u_in = f_in(arr, op.in_u); a.xi_in = f_in(arr, op.in_h); a.xi0 = f_in(arr, op.h0);
    a.xiprev = f_in(arr, op.hprev);
    a.xi_out = arr.f[op.out_h]; a.xi_shadow = arr.xi32; a.hst_out = arr.f[op.hst]; a.K = arr.f[A_K];
    a.h_state = arr.a[A_H]; a.acc = arr.a[A_ACCH];
    a.cdt = op.cdt; a.cdtf = (float)op.cdt;
    a.fb_a = (float)op.fb_a; a.fb_b = (float)op.fb_b; a.fb_c = (float)op.fb_c;
    return a;
}

inline VertArgs32 vert_args32(const Op &op, const DevArrays &arr) {
    return VertArgs32{op.lo, op.hi, f_in(arr, op.in_u), f_in(arr, op.hst), arr.f[A_Q]};
}

inline PrepArgs32 prep_args32(const Op &op, const DevArrays &arr) {
    return PrepArgs32{op.lo, op.hi, f_in(arr, op.in_u), f_in(arr, op.hst), arr.f[A_Q], (float4 *)arr.f[A_FQU]};
}

inline TriskArgs32 trisk_args32(const Op &op, const DevArrays &arr, double g, double rho0) {
    // the slow-term evaluation of the splitting leaves the gravity term out of B
    return TriskArgs32{op.lo, op.hi, f_in(arr, op.in_u), f_in(arr, op.hst), arr.f[A_K], arr.f[A_Q],
                       (float2 *)arr.f[A_FQU], (float2 *)arr.bx32,
                       op.split == 1 ? 0.f : (float)g,
                       (float)(rho0 > 0.0 ? 1.0 / rho0 : 0.0)};
}

inline EdgeArgs32 edge_args32(const Op &op, const DevArrays &arr, double g) {
    EdgeArgs32 a;
    a.segs = segs_of(op);
    a.lo = op.lo; a.hi = op.hi;
    a.u_in = f_in(arr, op.in_u); a.hst = f_in(arr, op.hst); a.K = arr.f[A_K]; a.fqu = (const float4 *)arr.f[A_FQU];
    a.sh = (const float2 *)arr.f[A_FQU];
    a.bx = (const float2 *)arr.bx32;
    a.u0 = f_in(arr, op.u0); a.us_out = arr.f[op.out_u]; a.u_shadow = arr.u32;
    a.u_state = arr.a[A_U]; a.acc = arr.a[A_ACCU];
    a.slow = arr.f[A_SLOW];
    a.cdt = op.cdt; a.cdtf = (float)op.cdt; a.g = (float)g;
    a.split = op.split;
    return a;
}

inline IfArgs32 if_args32(const Op &op, const DevArrays &arr, const DevMesh &m) {
    IfArgs32 a;
    a.c_lo = op.c_if1_lo; a.c_if1_hi = op.c_if1_hi; a.c_if12_hi = op.c_if12_hi;
    a.e_lo = op.e_if1_lo; a.e_if1_hi = op.e_if1_hi; a.e_if12_hi = op.e_if12_hi;
    a.n = op.hi;
    a.h = arr.a[A_H]; a.u = arr.a[A_U]; a.sh0 = arr.a[A_SH0]; a.su0 = arr.a[A_SU0];
    a.acch = arr.a[A_ACCH]; a.accu = arr.a[A_ACCU];
    a.xi = arr.xi32; a.u32 = arr.u32;
    a.hs1 = arr.f[A_HS1]; a.hs2 = arr.f[A_HS2]; a.hs3 = arr.f[A_HS3];
    a.hst1 = arr.f[A_HST1]; a.hst2 = arr.f[A_HST2]; a.hst3 = arr.f[A_HST3];
    a.us1 = arr.f[A_US1]; a.us2 = arr.f[A_US2]; a.us3 = arr.f[A_US3];
    a.sh1 = arr.f[A_SH1]; a.sh2 = arr.f[A_SH2]; a.sh3 = arr.f[A_SH3];
    a.su1 = arr.f[A_SU1]; a.su2 = arr.f[A_SU2]; a.su3 = arr.f[A_SU3];
    a.k = op.k; a.M = op.Mk; a.b1 = (float)op.fb_a; a.b2 = (float)op.fb_b; a.b3 = (float)op.fb_c; a.cf = op.cdt;
    return a;
}

// Cell i, FP32 tendency: the edge flux F_e = (H_e + (xi_i + xi_nb)/2) u_e in
// float (bit-identical from both cells of the edge: H_e is per edge and the
// sum commutes) and
// Psi_i = -(1/A_i) sum_j n_{e,i} l_e F_e (Eq. trisk_thickness).  Stage values
// (xi_s = xi0 + c tau Psi) take the float sum.  Where the double time level
// or a correction sum changes, the sum is taken over the exact products
// l_e F_e (the same from both cells) in double-float, within 2^-44 of the
// largest product, and widened to double, so the fluxes of an edge cancel in
// sum_i A_i h_i far below the double roundoff of the total (Theorem 1).  K_i =
// (1/A_i) sum_j (d_e l_e / 4) u_e^2.  NMAX bounds the edges of a cell so the
// row is loaded before the dependent gathers; the static per-edge data are
// an 8-byte {l_e, H_e} and a 4-byte d_e l_e / 4 gather.
template <int NMAX, bool ROWS>
FB_HD void cell32_body(const DevMesh &m, const CellArgs32 &a, int i) {
    const int mode = seg_mode(a.segs, i);
    if (mode == SEG_NONE) return;
    const int n = m.nEoC[i];
    int er[NMAX], nb[NMAX];
    float ue[NMAX], sdv[NMAX], kw[NMAX], He[NMAX], xn[NMAX];
    // every load the cell needs is issued in one round after the row: the
    // cell's own values first, the slot gathers (u, edge record, neighbour xi)
    // together, so no gather waits on an earlier one's arithmetic
    const float xi_i = a.xi_in[i];
    const float x0 = a.xi0[i];
    const float xp = a.fb_b != 0.f ? a.xiprev[i] : 0.f;   // the stage-2 value enters stage 3 only
    const float invAf = m.invA32[i];
    // the double 1/A_i only where the double time level or a sum changes
    const bool dbl = mode != SEG_UPD && mode != SEG_KONLY;
    const double invA = dbl ? m.invA[i] : 0.0;
    if constexpr (ROWS) {
        // cell-major rows padded with valid indices: vector loads, then the
        // gathers of the first ROW_MAIN slots unconditionally (padding masked)
        static_assert(NMAX % 4 == 0, "row width");
        const int4 *e4 = reinterpret_cast<const int4 *>(m.rowE + (size_t)i * NMAX);
        const int4 *n4 = reinterpret_cast<const int4 *>(m.rowN + (size_t)i * NMAX);
        FB_UNROLL
        for (int q = 0; q < NMAX / 4; ++q) {
            const int4 te = e4[q], tn = n4[q];
            er[4 * q] = te.x; er[4 * q + 1] = te.y; er[4 * q + 2] = te.z; er[4 * q + 3] = te.w;
            nb[4 * q] = tn.x; nb[4 * q + 1] = tn.y; nb[4 * q + 2] = tn.z; nb[4 * q + 3] = tn.w;
        }
        FB_UNROLL
        for (int j = 0; j < NMAX; ++j) {
            ue[j] = 0.f;
            kw[j] = 0.f;
            He[j] = 0.f;
            sdv[j] = 0.f;
            xn[j] = 0.f;
            if (j < ROW_MAIN || n > ROW_MAIN) {   // slots past ROW_MAIN only for cells that have them
                const int e = er[j] < 0 ? ~er[j] : er[j];
                const float u = a.u_in[e];
                const float2 st = m.el2[e];   // {l_e, H_e}
                const float kwe = m.ke32[e];  // d_e l_e / 4
                xn[j] = a.xi_in[nb[j]];
                ue[j] = j < n ? u : 0.f;
                kw[j] = kwe;
                He[j] = st.y;
                sdv[j] = j < n ? (er[j] < 0 ? st.x : -st.x) : 0.f;    // -n_{e,i} l_e
            }
        }
    } else {
        const int nC = m.nC;
        FB_UNROLL
        for (int j = 0; j < NMAX; ++j) {
            er[j] = 0;
            nb[j] = i;
            if (j < n) {
                er[j] = m.eocS[j * nC + i];
                nb[j] = m.coc[j * nC + i];
            }
        }
        FB_UNROLL
        for (int j = 0; j < NMAX; ++j) {
            ue[j] = 0.f;
            sdv[j] = 0.f;
            kw[j] = 0.f;
            He[j] = 0.f;
            xn[j] = 0.f;
            if (j < n) {
                const int e = er[j] < 0 ? ~er[j] : er[j];
                ue[j] = a.u_in[e];
                xn[j] = a.xi_in[nb[j]];
                const float2 st = m.el2[e];   // {l_e, H_e}
                kw[j] = m.ke32[e];            // d_e l_e / 4
                He[j] = st.y;
                sdv[j] = er[j] < 0 ? st.x : -st.x;    // -n_{e,i} l_e
            }
        }
    }
    float ke = 0.f;
    FB_UNROLL
    for (int j = 0; j < NMAX; ++j) ke += kw[j] * ue[j] * ue[j];
    a.K[i] = ke * invAf;
    if (mode == SEG_KONLY) return;
    float F[NMAX];
    FB_UNROLL
    for (int j = 0; j < NMAX; ++j)
        F[j] = (!ROWS || j < ROW_MAIN || n > ROW_MAIN) ? (He[j] + 0.5f * (xi_i + xn[j])) * ue[j] : 0.f;
    if (mode == SEG_UPD || mode == SEG_RK_SET || mode == SEG_RK_ADD2) {
        float S = 0.f;
        FB_UNROLL
        for (int j = 0; j < NMAX; ++j) S += sdv[j] * F[j];
        const float xs = x0 + a.cdtf * (S * invAf);
        a.xi_out[i] = xs;
        a.hst_out[i] = a.fb_a * xs + a.fb_b * xp + a.fb_c * x0;
        if (mode == SEG_UPD) return;
    }
    // the products l_e F_e are exact as float pairs (Dekker's product through
    // an FMA) and are summed in double-float on the FP32 pipe (Knuth's
    // TwoSum), then widened once: the edge's two cells take the same exact
    // product, and GB300 spends no FP64 operation per slot
    float2 Sd = make_float2(0.f, 0.f);
    FB_UNROLL
    for (int j = 0; j < NMAX; ++j) df_add_prod(Sd, sdv[j], F[j]);
    const double psi = df_value(Sd) * invA;
    switch (mode) {
        case SEG_INPLACE: {
            const double hn = a.h_state[i] + a.cdt * psi;
            const float xs = df_round(hn);
            a.h_state[i] = hn;
            a.xi_shadow[i] = xs;
            a.hst_out[i] = a.fb_a * xs + a.fb_b * xp + a.fb_c * x0;
        } break;
        case SEG_ACC_SET: a.acc[i] = psi; break;
        case SEG_ACC_ADD: a.acc[i] += psi; break;
        case SEG_RK_SET: a.acc[i] = psi; break;          // RK4: the tendency sum in double
        case SEG_RK_ADD2: a.acc[i] += 2.0 * psi; break;
        case SEG_RK_FIN: {
            const double hn = a.h_state[i] + a.cdt * (a.acc[i] + psi);
            const float xs = df_round(hn);
            a.h_state[i] = hn;
            a.xi_shadow[i] = xs;
            a.hst_out[i] = a.fb_a * xs + a.fb_b * xp + a.fb_c * x0;
        } break;
        default: break;
    }
}

// Vertex v: q_v = (zeta_v + f_v) / (H_v + sum_j kite xi / A_v)  (Eq. trisk_vorticity),
// from three 16-byte and one 8-byte record per vertex.
FB_HD void vert32_body(const DevMesh &m, const VertArgs32 &a, int v) {
    const int4 ix = m.vI4[v];
    const int2 c12 = m.vI2[v];
    const float4 cf = m.vCf[v];
    const float4 kh = m.vKh[v];
    const float z = cf.x * a.u_in[ix.x] + cf.y * a.u_in[ix.y] + cf.z * a.u_in[ix.z];
    const float xv = kh.x * a.hst[ix.w] + kh.y * a.hst[c12.x] + kh.z * a.hst[c12.y];
    a.q[v] = (z + cf.w) / (kh.w + xv);
}

// Edge e: {l_e F_e, q_e, l_e u_e, 0} with F_e = (H_e + (xi_c0 + xi_c1)/2) u_e,
// one 16-byte record, so the edge pass gathers a neighbour with one load.
// The neighbour's l_{e'} of the TRiSK weight travels with its record.
FB_HD void prep32_body(const DevMesh &m, const PrepArgs32 &a, int e) {
    const int c0 = m.coe0[e], c1 = m.coe1[e];
    const float ue = a.u_in[e];
    const float lu = m.dv32[e] * ue;   // l_e = 0 on no-flow edges
    const float lF = (m.He32[e] + 0.5f * (a.hst[c0] + a.hst[c1])) * lu;
    a.fqu[e] = make_float4(lF, 0.5f * (a.q[m.voe0[e]] + a.q[m.voe1[e]]), lu, 0.f);
}

// Cell i's share in the momentum tendency of each of its edges (Sec. 2.3,
// Eq. trisk_vorticity with the TRiSK flux mapping, and the gradient of
// Eq. nonlinear_swe).  For edges e_k, e_j of the cell (slots k, j; signs
// n_k, n_j; kite-fraction prefix P) the weight is
//   W_kj d_{e_k} = n_k n_j (1/2 - (P_j - P_k + [j < k])) l_{e_j},
// and with y_j = n_j X_j the sum over j != k reduces to
//   sum_j W_kj d X_j / l_j = n_k (1/2 (T - y_k) - T_P + P_k T - C_k),
// T = sum_j y_j, T_P = sum_j P_j y_j, C_k = sum_{j<k} y_j: O(n) per cell.
// X = l F (F = h_e u from the FB-averaged thickness) gives s0, X = l F q_e
// gives s1, X = l u gives s_v.  The share of slot k is {t = q_{e_k} s0 + s1,
// s_v} and the cell writes {B_i = K_i + g xi*_i (+ p_s / rho0), xi*_i} once,
// so the edge pass forms Phi_e = [(t_0 + t_1)/2 - (B_c1 - B_c0)] / d_e from
// one coalesced 16-byte load and the two cells' records.  q_{e_k} = (q at the
// two vertices of e_k) / 2: the row's vertex k is the counter-clockwise end
// of e_k, vertex k-1 the other.
// Rows are padded to S slots with valid indices; slots >= nEoC are masked.
template <int S, bool VORTEX>
FB_HD void trisk32_body(const DevMesh &m, const TriskArgs32 &a, const DevForcing &fz, int i) {
    const int n = m.nEoC[i];
    int re[S], rn[S], rv[S];
    float P[S];
    {
        const int4 *e4 = reinterpret_cast<const int4 *>(m.rowE + (size_t)i * S);
        const int4 *n4 = reinterpret_cast<const int4 *>(m.rowN + (size_t)i * S);
        const int4 *v4 = reinterpret_cast<const int4 *>(m.rowV + (size_t)i * S);
        const float4 *p4 = reinterpret_cast<const float4 *>(m.rowP + (size_t)i * S);
        FB_UNROLL
        for (int q = 0; q < S / 4; ++q) {
            const int4 te = e4[q], tn = n4[q], tv = v4[q];
            const float4 tp = p4[q];
            re[4 * q] = te.x; re[4 * q + 1] = te.y; re[4 * q + 2] = te.z; re[4 * q + 3] = te.w;
            rn[4 * q] = tn.x; rn[4 * q + 1] = tn.y; rn[4 * q + 2] = tn.z; rn[4 * q + 3] = tn.w;
            rv[4 * q] = tv.x; rv[4 * q + 1] = tv.y; rv[4 * q + 2] = tv.z; rv[4 * q + 3] = tv.w;
            P[4 * q] = tp.x; P[4 * q + 1] = tp.y; P[4 * q + 2] = tp.z; P[4 * q + 3] = tp.w;
        }
    }
    const float xs = a.hst[i];
    float B = a.K[i] + a.g * xs;
    if (VORTEX) B += fz.ps32[i] * a.inv_rho0;
    // slots below ROW_MAIN gather unconditionally (padding reads valid entries
    // and is masked); the rest only for the rare cells with more edges
    float lF[S], lu[S], qv[S];
    FB_UNROLL
    for (int j = 0; j < S; ++j) {
        lu[j] = 0.f;
        lF[j] = 0.f;
        qv[j] = 0.f;
        if (j < ROW_MAIN || n > ROW_MAIN) {
            const int e = re[j] < 0 ? ~re[j] : re[j];
            const float2 st = m.el2[e];   // {l_e, H_e}
            const float u = a.u_in[e];
            const float xn = a.hst[rn[j]];
            qv[j] = a.q[rv[j]];
            lu[j] = j < n ? st.x * u : 0.f;
            lF[j] = (st.y + 0.5f * (xs + xn)) * lu[j];
        }
    }
    float qlast = qv[0];
    FB_UNROLL
    for (int j = 1; j < S; ++j) qlast = (j == n - 1) ? qv[j] : qlast;
    float qe[S];
    float T0 = 0.f, T1 = 0.f, Tv = 0.f, P0 = 0.f, P1 = 0.f, Pv = 0.f;
    FB_UNROLL
    for (int j = 0; j < S; ++j) {
        qe[j] = 0.5f * ((j == 0 ? qlast : qv[j - 1]) + qv[j]);
        const float sg = re[j] < 0 ? -1.f : 1.f;
        const float y0 = sg * lF[j], y1 = y0 * qe[j], yv = sg * lu[j];
        T0 += y0; T1 += y1; Tv += yv;
        P0 += P[j] * y0; P1 += P[j] * y1; Pv += P[j] * yv;
    }
    float C0 = 0.f, C1 = 0.f, Cv = 0.f;
    FB_UNROLL
    for (int k = 0; k < S; ++k) {
        const float sg = re[k] < 0 ? -1.f : 1.f;
        const float y0 = sg * lF[k], y1 = y0 * qe[k], yv = sg * lu[k];
        if (k < n) {
            const float s0 = sg * (0.5f * (T0 - y0) - P0 + P[k] * T0 - C0);
            const float s1 = sg * (0.5f * (T1 - y1) - P1 + P[k] * T1 - C1);
            const float sv = sg * (0.5f * (Tv - yv) - Pv + P[k] * Tv - Cv);
            const int e = re[k] < 0 ? ~re[k] : re[k];
            a.sh[2 * e + (re[k] < 0 ? 1 : 0)] = make_float2(qe[k] * s0 + s1, sv);
        }
        C0 += y0; C1 += y1; Cv += yv;
    }
    a.bx[i] = make_float2(B, xs);   // last: a store before the gathers would hold them back
}

// Phi_e from the two cells' shares {t, s_v} and records {B, xi*}
// (trisk32_body): Phi_e = [(t_0 + t_1)/2 - (B_1 - B_0)] / d_e plus, with
// forcing, the wind stress and quadratic drag (Eq. hurricane_model) with
// v_e = (s_v0 + s_v1) / d_e and h_e = H_e + (xi*_0 + xi*_1)/2; the surface
// pressure is inside B.
template <bool FORCING>
FB_HD float phi_from_shares(const DevMesh &m, const float *u_in, const DevForcing &fz, int e, float4 s, float2 b0,
                            float2 b1) {
    const float idc = m.invDc32[e];
    float phi = idc * (0.5f * (s.x + s.z) - (b1.x - b0.x));
    if (FORCING) {
        const float vt = idc * (s.y + s.w);
        const float ue = u_in[e];
        const float4 w = fz.wrec32[e];   // {wind normal, wind tangential, C_W, H_e}
        const float rhe = 1.f / (w.w + 0.5f * (b0.y + b1.y));
        if (fz.flags & FBLTS_FORCE_WIND_STRESS) {
            const float dn = w.x - ue, dt = w.y - vt;
            phi += w.z * sqrtf(dn * dn + dt * dt) * dn * rhe;
        }
        if (fz.flags & FBLTS_FORCE_BOTTOM_DRAG) phi -= fz.cd32 * sqrtf(ue * ue + vt * vt) * ue * rhe;
    }
    return phi;
}

// The edge's update by segment mode: stage value u0 + c tau Phi (float), in
// place u += c tau Phi (double, with the float shadow), or the correction sum.
// No-flow edges take u = 0 and contribute 0.
template <class A>
FB_HD void edge32_apply(const A &a, int mode, int e, bool bnd, float phi) {
    const double phid = df_widen(phi);   // exact, on the integer pipe (no FP64 conversion)
    switch (mode) {
        case SEG_UPD: a.us_out[e] = bnd ? 0.f : a.u0[e] + a.cdtf * phi; break;
        case SEG_INPLACE: {
            const double un = bnd ? 0.0 : a.u_state[e] + a.cdt * phid;
            a.u_state[e] = un;
            a.u_shadow[e] = df_round(un);
        } break;
        case SEG_ACC_SET: a.acc[e] = phid; break;
        case SEG_ACC_ADD: a.acc[e] += phid; break;
        case SEG_PHI: a.us_out[e] = bnd ? 0.f : phi; break;
        case SEG_RK_SET:
        case SEG_RK_ADD2:
            a.us_out[e] = bnd ? 0.f : a.u0[e] + a.cdtf * phi;
            a.acc[e] = mode == SEG_RK_SET ? phid : a.acc[e] + 2.0 * phid;
            break;
        case SEG_RK_FIN: {
            const double un = bnd ? 0.0 : a.u_state[e] + a.cdt * (a.acc[e] + phid);
            a.u_state[e] = un;
            a.u_shadow[e] = df_round(un);
        } break;
        default: break;
    }
}

// Edge e: Phi_e in float (the pressure gradient g (xi_c1 - xi_c0) / d_e needs
// no cancellation of large depths), stage value u_s = u0 + c tau Phi, in
// place u += c tau Phi in double, or the correction sum in double.  SHARES:
// from the two cells' shares of the cell-side TRiSK pass; else from the edge
// records over explicit neighbour lists.
template <bool SHARES, bool FORCING>
FB_HD void edge32_body(const DevMesh &m, const EdgeArgs32 &a, const DevForcing &fz, int e) {
    const int mode = seg_mode(a.segs, e);
    if (mode == SEG_NONE) return;
    const bool bnd = m.ebnd[e] != 0;
    float phi = 0.f;
    if (!bnd && a.split == 2) {
        // operator splitting [Sec. 3.2, Eq. splitting]: the gravity-wave term at the
        // stage state plus the slow terms of the coarse step
        phi = a.slow[e] - a.g * (a.hst[m.coe1[e]] - a.hst[m.coe0[e]]) * m.invDc32[e];
    } else if (!bnd) {
        if constexpr (SHARES) {
            const float4 s = *reinterpret_cast<const float4 *>(a.sh + 2 * (size_t)e);   // {t0, s_v0, t1, s_v1}
            phi = phi_from_shares<FORCING>(m, a.u_in, fz, e, s, a.bx[m.coe0[e]], a.bx[m.coe1[e]]);
        } else {
            // explicit neighbour list; the weights are W_{e,e'} / l_{e'}
            const float idc = m.invDc32[e];
            const int nE = m.nE, n = m.nEoE[e];
            const int c0 = m.coe0[e], c1 = m.coe1[e];
            const float qself = a.fqu[e].y;
            float cor = 0.f, vt = 0.f;
            for (int j = 0; j < n; ++j) {
                const int x = m.eoe[j * nE + e];
                const float w = m.woe32[j * nE + e];
                const float4 r = a.fqu[x];
                cor += w * r.x * (0.5f * (qself + r.y));
                if (FORCING) vt += w * r.z;
            }
            const float x0c = a.hst[c0], x1c = a.hst[c1];
            const float grad = (a.K[c1] - a.K[c0]) + (a.split == 1 ? 0.f : a.g) * (x1c - x0c);
            phi = cor - grad * idc;
            if (FORCING) {
                const float ue = a.u_in[e];
                const float4 w = fz.wrec32[e];   // {wind normal, wind tangential, C_W, H_e}
                const float he = w.w + 0.5f * (x0c + x1c);
                if (fz.flags & FBLTS_FORCE_WIND_STRESS) {
                    const float dn = w.x - ue, dt = w.y - vt;
                    phi += w.z * sqrtf(dn * dn + dt * dt) * dn / he;
                }
                if (fz.flags & FBLTS_FORCE_BOTTOM_DRAG) phi -= fz.cd32 * sqrtf(ue * ue + vt * vt) * ue / he;
                if (fz.flags & FBLTS_FORCE_VORTEX) phi -= (fz.ps32[c1] - fz.ps32[c0]) * idc / (float)fz.rho0;
            }
        }
    }
    edge32_apply(a, mode, e, bnd, phi);
}

// Saves h^n, u^n (double) on IF-1 u IF-2 and the uncorrected IF-1 stage data (float).
FB_HD void save32_body(const IfArgs32 &a, int t) {
    const int i = a.c_lo + t;
    if (i < a.c_if12_hi) {
        a.sh0[i] = a.h[i];
        if (i < a.c_if1_hi) { a.sh1[i] = a.hs1[i]; a.sh2[i] = a.hs2[i]; a.sh3[i] = a.hs3[i]; }
    }
    const int e = a.e_lo + t;
    if (e < a.e_if12_hi) {
        a.su0[e] = a.u[e];
        if (e < a.e_if1_hi) { a.su1[e] = a.us1[e]; a.su2[e] = a.us2[e]; a.su3[e] = a.us3[e]; }
    }
}

// Interface prediction on IF-1 (Eq. preds, Eq. hstar_preds) in xi; writes the
// float shadows that the fine stages read as the time level h^{n,k}, u^{n,k}.
FB_HD void pred32_body(const IfArgs32 &a, int t) {
    const float Md = (float)a.M;
    const float wk = a.k / Md, wk1 = (a.k + 1) / Md, w1 = 1.f / Md;
    const int i = a.c_lo + t;
    if (i < a.c_if1_hi) {
        const float x0 = df_round(a.sh0[i]);
        const float x13 = a.sh1[i], x12 = a.sh2[i], x1 = a.sh3[i];
        const float hk = wk * x1 + (1.f - wk) * x0;
        const float hk1 = wk1 * x1 + (1.f - wk1) * x0;
        const float h13 = wk * x1 + w1 * x13 + (1.f - wk1) * x0;
        const float h12 = wk * x1 + w1 * x12 + (1.f - wk1) * x0;
        a.xi[i] = hk;
        a.hs1[i] = h13;
        a.hs2[i] = h12;
        a.hst1[i] = a.b1 * h13 + (1.f - a.b1) * hk;
        a.hst2[i] = a.b2 * h12 + (1.f - a.b2) * hk;
        a.hst3[i] = a.b3 * hk1 + (1.f - 2.f * a.b3) * h12 + a.b3 * hk;
    }
    const int e = a.e_lo + t;
    if (e < a.e_if1_hi) {
        const float x0 = df_round(a.su0[e]), x13 = a.su1[e], x12 = a.su2[e], x1 = a.su3[e];
        a.u32[e] = wk * x1 + (1.f - wk) * x0;
        a.us1[e] = wk * x1 + w1 * x13 + (1.f - wk1) * x0;
        a.us2[e] = wk * x1 + w1 * x12 + (1.f - wk1) * x0;
    }
}

// Interface correction (Eq. if_correction) in double, with the float shadows refreshed.
FB_HD void final32_body(const IfArgs32 &a, const unsigned char *ebnd, int t) {
    const int i = a.c_lo + t;
    if (i < a.c_if12_hi) {
        const double hn = a.sh0[i] + a.cf * a.acch[i];
        a.h[i] = hn;
        a.xi[i] = df_round(hn);
    }
    const int e = a.e_lo + t;
    if (e < a.e_if12_hi) {
        const double un = ebnd[e] ? 0.0 : a.su0[e] + a.cf * a.accu[e];
        a.u[e] = un;
        a.u32[e] = df_round(un);
    }
}

// Moving Holland-type vortex in float (the FP32 path): the offset from the
// centre is formed in double, the profile p = pc + dp exp(-(R/r)^B) and the
// gradient wind V = sqrt(B dp/rho_air (R/r)^B exp(-(R/r)^B) + (r f/2)^2) - r f/2
// in float; returns p - (pc + dp), the pressure relative to ambient.  Both are
// taken in forms without cancellation where (R/r)^B is small (far from the
// centre, where neighbouring cells differ by a tiny fraction of the pressure
// anomaly): p - (pc + dp) = dp expm1(-(R/r)^B), and with X the first term
// under the root, V = X / (sqrt(X + (r f/2)^2) + r f/2).
FB_HD float vortex_at32(const DevForcing &fz, double x, double y, double t, float &wu, float &wv) {
    const float rx = (float)(x - (fz.vx[4] + fz.vx[6] * t)), ry = (float)(y - (fz.vx[5] + fz.vx[7] * t));
    const float r = sqrtf(rx * rx + ry * ry);
    wu = 0.f;
    wv = 0.f;
    if (!(r > 0.f)) return -(float)fz.vx[1];
    const float A = powf((float)fz.vx[2] / r, (float)fz.vx[3]);
    const float ex = expf(-A);
    if (ex == 0.f) return -(float)fz.vx[1];
    const float hf = 0.5f * r * (float)fz.vx[8];
    const float X = (float)fz.vx[3] * (float)fz.vx[1] / (float)fz.rho_air * A * ex;
    const float den = sqrtf(X + hf * hf) + hf;
    const float V = den > 0.f ? X / den : 0.f;
    wu = -V * ry / r;
    wv = V * rx / r;
    return (float)fz.vx[1] * expm1f(-A);
}

// Float copies of the forcing fields: ps32 relative to the ambient pc + dp.
FB_HD void forcing32_body(const DevMesh &m, const DevForcing &fz, double time, int t) {
    if (t < m.nE) {
        float wu = (float)fz.wind_u, wv = (float)fz.wind_v;
        if (fz.flags & FBLTS_FORCE_VORTEX) {
            float a, b;
            vortex_at32(fz, m.xE[t], m.yE[t], time, a, b);
            wu += a;
            wv += b;
        }
        const float c = (float)m.cosE[t], s = (float)m.sinE[t];
        const float wn = wu * c + wv * s, wt = -wu * s + wv * c;
        const float cw = (float)(fz.rho_air / fz.rho0) * (0.75f + 0.067f * sqrtf(wn * wn + wt * wt)) * 1e-3f;
        fz.wrec32[t] = make_float4(wn, wt, cw, m.He32[t]);
    }
    if (t < m.nC) {
        float a, b;
        fz.ps32[t] = (fz.flags & FBLTS_FORCE_VORTEX) ? vortex_at32(fz, m.xC[t], m.yC[t], time, a, b) : 0.f;
    }
}

}  // namespace fblts
