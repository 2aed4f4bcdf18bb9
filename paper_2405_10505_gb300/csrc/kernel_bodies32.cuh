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
    double *h_state, *acc;
    const double *bottom;
    double cdt;
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

struct EdgeArgs32 {
    SegSet segs;
    int lo, hi;
    const float *u_in, *hst, *K, *u0;
    const float4 *fqu;
    float *us_out, *u_shadow;
    double *u_state, *acc;
    double cdt;
    float g;
};

struct IfArgs32 {
    int c_lo, c_if1_hi, c_if12_hi, e_lo, e_if1_hi, e_if12_hi, n;
    double *h, *u, *sh0, *su0, *acch, *accu;
    const double *bottom;
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
    a.h_state = arr.a[A_H]; a.acc = arr.a[A_ACCH]; a.bottom = m.bottom;
    a.cdt = op.cdt; a.fb_a = (float)op.fb_a; a.fb_b = (float)op.fb_b; a.fb_c = (float)op.fb_c;
    return a;
}

inline VertArgs32 vert_args32(const Op &op, const DevArrays &arr) {
    return VertArgs32{op.lo, op.hi, f_in(arr, op.in_u), arr.f[op.hst], arr.f[A_Q]};
}

inline PrepArgs32 prep_args32(const Op &op, const DevArrays &arr) {
    return PrepArgs32{op.lo, op.hi, f_in(arr, op.in_u), arr.f[op.hst], arr.f[A_Q], (float4 *)arr.f[A_FQU]};
}

inline EdgeArgs32 edge_args32(const Op &op, const DevArrays &arr, double g) {
    EdgeArgs32 a;
    a.segs = segs_of(op);
    a.lo = op.lo; a.hi = op.hi;
    a.u_in = f_in(arr, op.in_u); a.hst = arr.f[op.hst]; a.K = arr.f[A_K]; a.fqu = (const float4 *)arr.f[A_FQU];
    a.u0 = f_in(arr, op.u0); a.us_out = arr.f[op.out_u]; a.u_shadow = arr.u32;
    a.u_state = arr.a[A_U]; a.acc = arr.a[A_ACCU];
    a.cdt = op.cdt; a.g = (float)g;
    return a;
}

inline IfArgs32 if_args32(const Op &op, const DevArrays &arr, const DevMesh &m) {
    IfArgs32 a;
    a.c_lo = op.c_if1_lo; a.c_if1_hi = op.c_if1_hi; a.c_if12_hi = op.c_if12_hi;
    a.e_lo = op.e_if1_lo; a.e_if1_hi = op.e_if1_hi; a.e_if12_hi = op.e_if12_hi;
    a.n = op.hi;
    a.h = arr.a[A_H]; a.u = arr.a[A_U]; a.sh0 = arr.a[A_SH0]; a.su0 = arr.a[A_SU0];
    a.acch = arr.a[A_ACCH]; a.accu = arr.a[A_ACCU]; a.bottom = m.bottom;
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
// or a correction sum changes, the sum is taken in double from the products
// l_e F_e (exact in double and the same from both cells), so the fluxes of an
// edge cancel in sum_i A_i h_i to double roundoff (Theorem 1).  K_i =
// (1/A_i) sum_j (d_e l_e / 4) u_e^2.  NMAX bounds the edges of a cell so the
// row is loaded before the dependent gathers; the static per-edge data
// {l_e, d_e l_e / 4, H_e} is one 16-byte gather.
template <int NMAX>
FB_HD void cell32_body(const DevMesh &m, const CellArgs32 &a, int i) {
    const int mode = seg_mode(a.segs, i);
    if (mode == SEG_NONE) return;
    const int n = m.nEoC[i];
    const int nC = m.nC;
    int er[NMAX], nb[NMAX];
    FB_UNROLL
    for (int j = 0; j < NMAX; ++j) {
        er[j] = 0;
        nb[j] = i;
        if (j < n) {
            er[j] = m.eocS[j * nC + i];
            nb[j] = m.coc[j * nC + i];
        }
    }
    float ue[NMAX], sdv[NMAX], kw[NMAX], He[NMAX];
    FB_UNROLL
    for (int j = 0; j < NMAX; ++j) {
        ue[j] = 0.f;
        sdv[j] = 0.f;
        kw[j] = 0.f;
        He[j] = 0.f;
        if (j < n) {
            const int e = er[j] < 0 ? ~er[j] : er[j];
            ue[j] = a.u_in[e];
            const float4 st = m.estat[e];
            kw[j] = st.y;
            He[j] = st.z;
            sdv[j] = er[j] < 0 ? st.x : -st.x;    // -n_{e,i} l_e
        }
    }
    float ke = 0.f;
    FB_UNROLL
    for (int j = 0; j < NMAX; ++j) ke += kw[j] * ue[j] * ue[j];
    const double invA = m.invA[i];
    a.K[i] = ke * (float)invA;
    if (mode == SEG_KONLY) return;
    const float xi_i = a.xi_in[i];
    float F[NMAX];
    FB_UNROLL
    for (int j = 0; j < NMAX; ++j) F[j] = (He[j] + 0.5f * (xi_i + a.xi_in[nb[j]])) * ue[j];
    if (mode == SEG_UPD) {
        float S = 0.f;
        FB_UNROLL
        for (int j = 0; j < NMAX; ++j) S += sdv[j] * F[j];
        const float x0 = a.xi0[i];
        const float xn = x0 + (float)a.cdt * (S * (float)invA);
        a.xi_out[i] = xn;
        a.hst_out[i] = a.fb_a * xn + a.fb_b * a.xiprev[i] + a.fb_c * x0;
        return;
    }
    double S = 0.0;
    FB_UNROLL
    for (int j = 0; j < NMAX; ++j) S = fma((double)sdv[j], (double)F[j], S);
    const double psi = S * invA;
    switch (mode) {
        case SEG_INPLACE: {
            const float x0 = a.xi0[i];
            const double hn = a.h_state[i] + a.cdt * psi;
            const float xn = (float)(hn + a.bottom[i]);
            a.h_state[i] = hn;
            a.xi_shadow[i] = xn;
            a.hst_out[i] = a.fb_a * xn + a.fb_b * a.xiprev[i] + a.fb_c * x0;
        } break;
        case SEG_ACC_SET: a.acc[i] = psi; break;
        case SEG_ACC_ADD: a.acc[i] += psi; break;
        default: break;
    }
}

// Vertex v: q_v = (zeta_v + f_v) / (H_v + sum_j kite xi / A_v)  (Eq. trisk_vorticity).
FB_HD void vert32_body(const DevMesh &m, const VertArgs32 &a, int v) {
    const int nV = m.nV;
    float z = 0.f, xv = 0.f;
    FB_UNROLL
    for (int j = 0; j < 3; ++j) {
        z += m.cVort32[j * nV + v] * a.u_in[m.eov[j * nV + v]];
        xv += m.cKite32[j * nV + v] * a.hst[m.cov[j * nV + v]];
    }
    a.q[v] = (z + m.fV32[v]) / (m.Hv32[v] + xv);
}

// Edge e: {F_e = (H_e + (xi_c0 + xi_c1)/2) u_e, q_e, u_e} as one 16-byte
// record, so the edge pass gathers a neighbour with one load.
FB_HD void prep32_body(const DevMesh &m, const PrepArgs32 &a, int e) {
    const int c0 = m.coe0[e], c1 = m.coe1[e];
    const float ue = a.u_in[e];
    const float F = m.ebnd[e] ? 0.f : (m.He32[e] + 0.5f * (a.hst[c0] + a.hst[c1])) * ue;
    a.fqu[e] = make_float4(F, 0.5f * (a.q[m.voe0[e]] + a.q[m.voe1[e]]), ue, 0.f);
}

// Edge e: Phi_e in float (the pressure gradient g (xi_c1 - xi_c0) / d_e needs
// no cancellation of large depths), stage value u_s = u0 + c tau Phi, in
// place u += c tau Phi in double, or the correction sum in double.
template <bool FORCING>
FB_HD void edge32_body(const DevMesh &m, const EdgeArgs32 &a, const DevForcing &fz, int e) {
    const int mode = seg_mode(a.segs, e);
    if (mode == SEG_NONE) return;
    float phi = 0.f;
    if (!m.ebnd[e]) {
        const int nE = m.nE;
        const int c0 = m.coe0[e], c1 = m.coe1[e];
        const int n = m.nEoE[e];
        const float qself = a.fqu[e].y;
        float cor = 0.f, vt = 0.f;
        if (m.rows) {
            // neighbours = the other edges of c0 then of c1, from the cells' rows
            const int nC = m.nC;
            const unsigned short sl = m.eslot[e];
            int k = 0;
            for (int side = 0; side < 2; ++side) {
                const int c = side ? c1 : c0;
                const int nc = m.nEoC[c];
                const int p = side ? (sl >> 8) : (sl & 0xff);
                for (int j = 1; j < nc; ++j) {
                    int jj = p + j;
                    if (jj >= nc) jj -= nc;
                    const int v = m.eocS[jj * nC + c];
                    const int x = v < 0 ? ~v : v;
                    const float w = m.woeC32[k * nE + e];
                    ++k;
                    const float4 r = a.fqu[x];
                    cor += w * r.x * (0.5f * (qself + r.y));
                    if (FORCING) vt += w * r.z;
                }
            }
        } else {
            for (int j = 0; j < n; ++j) {
                const int x = m.eoe[j * nE + e];
                const float w = m.woe32[j * nE + e];
                const float4 r = a.fqu[x];
                cor += w * r.x * (0.5f * (qself + r.y));
                if (FORCING) vt += w * r.z;
            }
        }
        const float x0c = a.hst[c0], x1c = a.hst[c1];
        const float grad = (a.K[c1] - a.K[c0]) + a.g * (x1c - x0c);
        phi = cor - grad * m.invDc32[e];
        if (FORCING) {
            const float ue = a.u_in[e];
            const float he = m.He32[e] + 0.5f * (x0c + x1c);
            if (fz.flags & FBLTS_FORCE_WIND_STRESS) {
                const float dn = fz.windN32[e] - ue, dt = fz.windT32[e] - vt;
                phi += fz.cw32[e] * sqrtf(dn * dn + dt * dt) * dn / he;
            }
            if (fz.flags & FBLTS_FORCE_BOTTOM_DRAG) phi -= (float)fz.cd * sqrtf(ue * ue + vt * vt) * ue / he;
            if (fz.flags & FBLTS_FORCE_VORTEX)
                phi -= (fz.ps32[c1] - fz.ps32[c0]) * m.invDc32[e] / (float)fz.rho0;
        }
    }
    switch (mode) {
        case SEG_UPD: a.us_out[e] = m.ebnd[e] ? 0.f : a.u0[e] + (float)a.cdt * phi; break;
        case SEG_INPLACE: {
            const double un = m.ebnd[e] ? 0.0 : a.u_state[e] + a.cdt * (double)phi;
            a.u_state[e] = un;
            a.u_shadow[e] = (float)un;
        } break;
        case SEG_ACC_SET: a.acc[e] = (double)phi; break;
        case SEG_ACC_ADD: a.acc[e] += (double)phi; break;
        default: break;
    }
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
        const float x0 = (float)(a.sh0[i] + a.bottom[i]);
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
        const float x0 = (float)a.su0[e], x13 = a.su1[e], x12 = a.su2[e], x1 = a.su3[e];
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
        a.xi[i] = (float)(hn + a.bottom[i]);
    }
    const int e = a.e_lo + t;
    if (e < a.e_if12_hi) {
        const double un = ebnd[e] ? 0.0 : a.su0[e] + a.cf * a.accu[e];
        a.u[e] = un;
        a.u32[e] = (float)un;
    }
}

// Moving Holland-type vortex in float (the FP32 path): the offset from the
// centre is formed in double, the profile p = pc + dp exp(-(R/r)^B) and the
// gradient wind V = sqrt(B dp/rho_air (R/r)^B exp(-(R/r)^B) + (r f/2)^2) - r f/2
// in float; returns p - (pc + dp), the pressure relative to ambient.
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
    const float V = sqrtf((float)fz.vx[3] * (float)fz.vx[1] / (float)fz.rho_air * A * ex + hf * hf) - hf;
    wu = -V * ry / r;
    wv = V * rx / r;
    return (float)fz.vx[1] * (ex - 1.f);
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
        fz.windN32[t] = wn;
        fz.windT32[t] = wt;
        fz.cw32[t] = (float)(fz.rho_air / fz.rho0) * (0.75f + 0.067f * sqrtf(wn * wn + wt * wt)) * 1e-3f;
    }
    if (t < m.nC) {
        float a, b;
        fz.ps32[t] = (fz.flags & FBLTS_FORCE_VORTEX) ? vortex_at32(fz, m.xC[t], m.yC[t], time, a, b) : 0.f;
    }
}

}  // namespace fblts
