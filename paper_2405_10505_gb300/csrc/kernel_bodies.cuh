// Per-element bodies of the FB-LTS passes and the argument packing of one
// schedule op.  The __global__ wrappers in kernels.cu run one body per thread.
#pragma once

#include <cmath>

#include "kernels.cuh"

#ifdef __CUDACC__
#define FB_HD __host__ __device__ __forceinline__
#else
#define FB_HD inline
#endif
#ifdef __CUDA_ARCH__
#define FB_UNROLL _Pragma("unroll")
#else
#define FB_UNROLL
#endif

namespace fblts {

FB_HD int seg_mode(const SegSet &s, int i) {
    int m = SEG_NONE;
FB_UNROLL
    for (int k = 0; k < MAX_SEG; ++k)
        if (k < s.nseg && i >= s.seg[k].begin && i < s.seg[k].end) m = s.seg[k].mode;
    return m;
}

struct CellArgs {
    SegSet segs;
    int lo, hi;
    const double *u_in, *h_in, *h0, *hprev;
    double *hs_out, *h_state, *hst_out, *K, *acc;
    double cdt, fb_a, fb_b, fb_c;
};

struct VertArgs {
    int lo, hi;
    const double *u_in, *hst;
    double *q;
};

struct PrepArgs {
    int lo, hi;
    const double *u_in, *hst, *q;
    double *Fe, *qe, *FQ;
};

struct EdgeArgs {
    SegSet segs;
    int lo, hi;
    const double *u_in, *hst, *K, *Fe, *qe, *FQ, *u0;
    double *us_out, *u_state, *acc;
    const double *slow;   // splitting: the slow part of Phi per edge
    double cdt, g;
    int split;            // 0, or 1: slow-term evaluation, 2: stage with Phi = fast + slow
};

struct IfArgs {
    int c_lo, c_if1_hi, c_if12_hi, e_lo, e_if1_hi, e_if12_hi, n;
    double *h, *hs1, *hs2, *hs3, *hst1, *hst2, *hst3, *u, *us1, *us2, *us3;
    double *sh0, *sh1, *sh2, *sh3, *su0, *su1, *su2, *su3, *acch, *accu;
    int k, M;
    double b1, b2, b3, cf;
};

// ---------------------------------------------------------------- packing

inline SegSet segs_of(const Op &op) {
    SegSet s;
    s.nseg = op.nseg;
    for (int k = 0; k < MAX_SEG; ++k) s.seg[k] = op.seg[k];
    return s;
}

inline CellArgs cell_args(const Op &op, const DevArrays &arr) {
    double *const *A = arr.a;
    CellArgs a;
    a.segs = segs_of(op);
    a.lo = op.lo; a.hi = op.hi;
    a.u_in = A[op.in_u]; a.h_in = A[op.in_h]; a.h0 = A[op.h0]; a.hprev = A[op.hprev];
    a.hs_out = A[op.out_h]; a.h_state = A[A_H]; a.hst_out = A[op.hst]; a.K = A[A_K]; a.acc = A[A_ACCH];
    a.cdt = op.cdt; a.fb_a = op.fb_a; a.fb_b = op.fb_b; a.fb_c = op.fb_c;
    return a;
}

inline VertArgs vert_args(const Op &op, const DevArrays &arr) {
    return VertArgs{op.lo, op.hi, arr.a[op.in_u], arr.a[op.hst], arr.a[A_Q]};
}

inline PrepArgs prep_args(const Op &op, const DevArrays &arr) {
    return PrepArgs{op.lo, op.hi, arr.a[op.in_u], arr.a[op.hst], arr.a[A_Q], arr.a[A_FE], arr.a[A_QE], arr.a[A_FQ]};
}

inline EdgeArgs edge_args(const Op &op, const DevArrays &arr, double g) {
    double *const *A = arr.a;
    EdgeArgs a;
    a.segs = segs_of(op);
    a.lo = op.lo; a.hi = op.hi;
    a.u_in = A[op.in_u]; a.hst = A[op.hst]; a.K = A[A_K]; a.Fe = A[A_FE]; a.qe = A[A_QE]; a.FQ = A[A_FQ];
    a.u0 = A[op.u0]; a.us_out = A[op.out_u]; a.u_state = A[A_U]; a.acc = A[A_ACCU];
    a.slow = A[A_SLOW];
    a.cdt = op.cdt; a.g = g;
    a.split = op.split;
    return a;
}

inline IfArgs if_args(const Op &op, const DevArrays &arr) {
    double *const *A = arr.a;
    IfArgs a;
    a.c_lo = op.c_if1_lo; a.c_if1_hi = op.c_if1_hi; a.c_if12_hi = op.c_if12_hi;
    a.e_lo = op.e_if1_lo; a.e_if1_hi = op.e_if1_hi; a.e_if12_hi = op.e_if12_hi;
    a.n = op.hi;
    a.h = A[A_H]; a.hs1 = A[A_HS1]; a.hs2 = A[A_HS2]; a.hs3 = A[A_HS3];
    a.hst1 = A[A_HST1]; a.hst2 = A[A_HST2]; a.hst3 = A[A_HST3];
    a.u = A[A_U]; a.us1 = A[A_US1]; a.us2 = A[A_US2]; a.us3 = A[A_US3];
    a.sh0 = A[A_SH0]; a.sh1 = A[A_SH1]; a.sh2 = A[A_SH2]; a.sh3 = A[A_SH3];
    a.su0 = A[A_SU0]; a.su1 = A[A_SU1]; a.su2 = A[A_SU2]; a.su3 = A[A_SU3];
    a.acch = A[A_ACCH]; a.accu = A[A_ACCU];
    a.k = op.k; a.M = op.Mk; a.b1 = op.fb_a; a.b2 = op.fb_b; a.b3 = op.fb_c; a.cf = op.cdt;
    return a;
}

// ---------------------------------------------------------------- bodies

// Cell i: Psi_i = sum_j cDiv_ij h_e u_e (Eq. trisk_thickness with
// cDiv = -n_{e,i} l_e / A_i and h_e = H_e + (xi_i + xi_nb)/2 the mean of the
// two cells), the stage update xi_s = xi0 + c tau Psi (Eq. fbrk32), its FB
// average and the kinetic energy K_i = sum_j cKE_ij u_e^2
// (cKE = d_e l_e / (4 A_i)).  Thickness arrays hold xi = h - H.
FB_HD void cell_body(const DevMesh &m, const CellArgs &a, int i) {
    const int mode = seg_mode(a.segs, i);
    if (mode == SEG_NONE) return;
    const int n = m.nEoC[i];
    const int nC = m.nC;
    double psi = 0.0, ke = 0.0;
    const double hi_ = a.h_in[i];
    for (int j = 0; j < n; ++j) {
        const int e = m.eoc[j * nC + i];
        const double ue = a.u_in[e];
        ke += m.cKE[j * nC + i] * ue * ue;
        if (mode != SEG_KONLY) {
            const int nb = m.coc[j * nC + i];
            psi += m.cDiv[j * nC + i] * ((m.He64[e] + 0.5 * (hi_ + a.h_in[nb])) * ue);
        }
    }
    a.K[i] = ke;
    switch (mode) {
        case SEG_UPD: {
            const double h0 = a.h0[i];
            const double hn = h0 + a.cdt * psi;
            a.hs_out[i] = hn;
            a.hst_out[i] = a.fb_a * hn + a.fb_b * a.hprev[i] + a.fb_c * h0;
        } break;
        case SEG_INPLACE: {
            const double h0 = a.h_state[i];
            const double hn = h0 + a.cdt * psi;
            a.h_state[i] = hn;
            a.hst_out[i] = a.fb_a * hn + a.fb_b * a.hprev[i] + a.fb_c * h0;
        } break;
        case SEG_ACC_SET: a.acc[i] = psi; break;
        case SEG_ACC_ADD: a.acc[i] += psi; break;
        case SEG_RK_SET:
        case SEG_RK_ADD2: {
            const double h0 = a.h0[i];
            const double hn = h0 + a.cdt * psi;
            a.hs_out[i] = hn;
            a.hst_out[i] = a.fb_a * hn + a.fb_b * a.hprev[i] + a.fb_c * h0;
            a.acc[i] = mode == SEG_RK_SET ? psi : a.acc[i] + 2.0 * psi;
        } break;
        case SEG_RK_FIN: {
            const double h0 = a.h_state[i];
            const double hn = h0 + a.cdt * (a.acc[i] + psi);
            a.hst_out[i] = a.fb_a * hn + a.fb_b * a.hprev[i] + a.fb_c * h0;
            a.h_state[i] = hn;
        } break;
        default: break;
    }
}

// Vertex v: zeta_v = sum_j t_{e,v} d_e u_e / A_v, h_v = H_v + sum_j kite xi / A_v,
// q_v = (zeta_v + f_v) / h_v  (Eq. trisk_vorticity; PV q = eta / h).
FB_HD void vert_body(const DevMesh &m, const VertArgs &a, int v) {
    const int nV = m.nV;
    double z = 0.0, hv = m.Hv64[v];
FB_UNROLL
    for (int j = 0; j < 3; ++j) {
        z += m.cVort[j * nV + v] * a.u_in[m.eov[j * nV + v]];
        hv += m.cKite[j * nV + v] * a.hst[m.cov[j * nV + v]];
    }
    a.q[v] = (z + m.fV[v]) / hv;
}

// Edge e: thickness flux F_e = h_e u_e with h_e = H_e + (xi_c0 + xi_c1)/2
// (zero on no-flow edges), the edge PV q_e = (q_v0 + q_v1) / 2 and their
// product F_e q_e.
FB_HD void prep_body(const DevMesh &m, const PrepArgs &a, int e) {
    const int c0 = m.coe0[e], c1 = m.coe1[e];
    const double F = m.ebnd[e] ? 0.0 : (m.He64[e] + 0.5 * (a.hst[c0] + a.hst[c1])) * a.u_in[e];
    const double q = 0.5 * (a.q[m.voe0[e]] + a.q[m.voe1[e]]);
    a.Fe[e] = F;
    a.qe[e] = q;
    a.FQ[e] = F * q;
}

// Edge e: Phi_e = sum_j w_j F_{e_j} (q_e + q_{e_j}) / 2
//                 - [K_c1 - K_c0 + g (xi_c1 - xi_c0)] / d_e  (+ forcing)
// with xi = h + b the stored surface elevation and h_e = H_e + (xi_c0 + xi_c1)/2
// (rotating SWE, Eq. nonlinear_swe, in TRiSK form; forcing of Eq.
// hurricane_model), then the stage update u_s = u0 + c tau Phi or the
// correction sum of Eq. if_correction.  The Coriolis sum is taken as
// (q_e sum_j w_j F_j + sum_j w_j F_j q_j) / 2: two FMAs per neighbour.
template <bool FORCING>
FB_HD void edge_body(const DevMesh &m, const EdgeArgs &a, const DevForcing &fz, int e) {
    const int mode = seg_mode(a.segs, e);
    if (mode == SEG_NONE) return;
    double phi = 0.0;
    if (!m.ebnd[e] && a.split == 2) {
        // operator splitting [Sec. 3.2, Eq. splitting]: the gravity-wave term at the
        // stage state plus the slow terms of the coarse step
        const int c0 = m.coe0[e], c1 = m.coe1[e];
        phi = a.slow[e] - a.g * (a.hst[c1] - a.hst[c0]) * m.invDc[e];
    } else if (!m.ebnd[e]) {
        const int nE = m.nE;
        const int c0 = m.coe0[e], c1 = m.coe1[e];
        const int n = m.nEoE[e];
        const double qself = a.qe[e];
        double sF = 0.0, sG = 0.0, vt = 0.0;
        for (int j = 0; j < n; ++j) {
            const int x = m.eoe[j * nE + e];
            const double w = m.woe[j * nE + e];
            sF += w * a.Fe[x];
            sG += w * a.FQ[x];
            if (FORCING) vt += w * a.u_in[x];
        }
        const double cor = 0.5 * (qself * sF + sG);
        const double h0c = a.hst[c0], h1c = a.hst[c1];
        const double gg = a.split == 1 ? 0.0 : a.g;   // the slow terms leave gravity out
        const double grad = (a.K[c1] - a.K[c0]) + gg * (h1c - h0c);
        phi = cor - grad * m.invDc[e];
        if (FORCING) {
            const double ue = a.u_in[e];
            const double rhe = 1.0 / (m.He64[e] + 0.5 * (h0c + h1c));
            if (fz.flags & FBLTS_FORCE_WIND_STRESS) {
                const double dn = fz.windN[e] - ue, dt = fz.windT[e] - vt;
                phi += fz.cw[e] * sqrt(dn * dn + dt * dt) * dn * rhe;
            }
            if (fz.flags & FBLTS_FORCE_BOTTOM_DRAG) phi -= fz.cd * sqrt(ue * ue + vt * vt) * ue * rhe;
            if (fz.flags & FBLTS_FORCE_VORTEX) phi -= (fz.ps[c1] - fz.ps[c0]) * m.invDc[e] / fz.rho0;
        }
    }
    switch (mode) {
        case SEG_UPD: a.us_out[e] = m.ebnd[e] ? 0.0 : a.u0[e] + a.cdt * phi; break;
        case SEG_INPLACE: a.u_state[e] = m.ebnd[e] ? 0.0 : a.u_state[e] + a.cdt * phi; break;
        case SEG_ACC_SET: a.acc[e] = phi; break;
        case SEG_ACC_ADD: a.acc[e] += phi; break;
        case SEG_PHI: a.us_out[e] = m.ebnd[e] ? 0.0 : phi; break;
        case SEG_RK_SET:
        case SEG_RK_ADD2:
            a.us_out[e] = m.ebnd[e] ? 0.0 : a.u0[e] + a.cdt * phi;
            a.acc[e] = mode == SEG_RK_SET ? phi : a.acc[e] + 2.0 * phi;
            break;
        case SEG_RK_FIN: a.u_state[e] = m.ebnd[e] ? 0.0 : a.u_state[e] + a.cdt * (a.acc[e] + phi); break;
        default: break;
    }
}

// Saves h^n, u^n on IF-1 u IF-2 and the uncorrected IF-1 stage data (t-th element).
FB_HD void save_body(const IfArgs &a, int t) {
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

// Interface prediction on IF-1 for subcycle k (Eq. preds, Eq. hstar_preds):
// X^{n,k} = (k/M) X~^{n+1} + (1 - k/M) X^n,
// Xbar^{n,k+1/m} = (k/M) X~^{n+1} + (1/M) X~^{n+1/m} + (1 - (k+1)/M) X^n.
FB_HD void pred_body(const IfArgs &a, int t) {
    const double Md = (double)a.M;
    const double wk = a.k / Md, wk1 = (a.k + 1) / Md, w1 = 1.0 / Md;
    const int i = a.c_lo + t;
    if (i < a.c_if1_hi) {
        const double x0 = a.sh0[i], x13 = a.sh1[i], x12 = a.sh2[i], x1 = a.sh3[i];
        const double hk = wk * x1 + (1.0 - wk) * x0;
        const double hk1 = wk1 * x1 + (1.0 - wk1) * x0;
        const double h13 = wk * x1 + w1 * x13 + (1.0 - wk1) * x0;
        const double h12 = wk * x1 + w1 * x12 + (1.0 - wk1) * x0;
        a.h[i] = hk;
        a.hs1[i] = h13;
        a.hs2[i] = h12;
        a.hst1[i] = a.b1 * h13 + (1.0 - a.b1) * hk;
        a.hst2[i] = a.b2 * h12 + (1.0 - a.b2) * hk;
        a.hst3[i] = a.b3 * hk1 + (1.0 - 2.0 * a.b3) * h12 + a.b3 * hk;
    }
    const int e = a.e_lo + t;
    if (e < a.e_if1_hi) {
        const double x0 = a.su0[e], x13 = a.su1[e], x12 = a.su2[e], x1 = a.su3[e];
        a.u[e] = wk * x1 + (1.0 - wk) * x0;
        a.us1[e] = wk * x1 + w1 * x13 + (1.0 - wk1) * x0;
        a.us2[e] = wk * x1 + w1 * x12 + (1.0 - wk1) * x0;
    }
}

// Interface correction (Eq. if_correction): X^{n+1} = X^n + (tau/M) sum_k T_k.
FB_HD void final_body(const IfArgs &a, const unsigned char *ebnd, int t) {
    const int i = a.c_lo + t;
    if (i < a.c_if12_hi) a.h[i] = a.sh0[i] + a.cf * a.acch[i];
    const int e = a.e_lo + t;
    if (e < a.e_if12_hi) a.u[e] = ebnd[e] ? 0.0 : a.su0[e] + a.cf * a.accu[e];
}

// Moving Holland-type vortex: p = pc + dp exp(-(R/r)^B) and the gradient
// wind V = sqrt(B dp/rho_air (R/r)^B exp(-(R/r)^B) + (r f/2)^2) - r f/2,
// counter-clockwise about the centre (x0 + vx t, y0 + vy t).
FB_HD void vortex_at(const DevForcing &fz, double x, double y, double t, double &p, double &wu, double &wv) {
    const double cx = fz.vx[4] + fz.vx[6] * t, cy = fz.vx[5] + fz.vx[7] * t;
    const double rx = x - cx, ry = y - cy;
    const double r = sqrt(rx * rx + ry * ry);
    const double A = r > 0.0 ? pow(fz.vx[2] / r, fz.vx[3]) : INFINITY;
    const double ex = r > 0.0 ? exp(-A) : 0.0;
    p = fz.vx[0] + fz.vx[1] * ex;
    if (r <= 0.0 || ex == 0.0) { wu = 0.0; wv = 0.0; return; }
    const double hf = 0.5 * r * fz.vx[8];
    const double V = sqrt(fz.vx[3] * fz.vx[1] / fz.rho_air * A * ex + hf * hf) - hf;
    wu = -V * ry / r;
    wv = V * rx / r;
}

// Forcing fields of the coarse step starting at `time`, held for its stages.
FB_HD void forcing_body(const DevMesh &m, const DevForcing &fz, double time, int t) {
    if (t < m.nE) {
        double wu = fz.wind_u, wv = fz.wind_v;
        if (fz.flags & FBLTS_FORCE_VORTEX) {
            double p, a, b;
            vortex_at(fz, m.xE[t], m.yE[t], time, p, a, b);
            wu += a;
            wv += b;
        }
        const double c = m.cosE[t], s = m.sinE[t];
        const double wn = wu * c + wv * s, wt = -wu * s + wv * c;
        fz.windN[t] = wn;
        fz.windT[t] = wt;
        fz.cw[t] = (fz.rho_air / fz.rho0) * (0.75 + 0.067 * sqrt(wn * wn + wt * wt)) * 1e-3;
    }
    if (t < m.nC) {
        double p = 0.0, a, b;
        if (fz.flags & FBLTS_FORCE_VORTEX) vortex_at(fz, m.xC[t], m.yC[t], time, p, a, b);
        fz.ps[t] = p;
    }
}

}  // namespace fblts
