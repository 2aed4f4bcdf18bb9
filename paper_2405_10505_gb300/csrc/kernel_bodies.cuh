// Per-element bodies of the FB-LTS passes and the argument packing of one
// schedule op.  The __global__ wrappers in kernels.cu run one body per thread.
#pragma once

#include <cmath>
#include <cstring>

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

// FP64 edge prep: per edge q_e (double) and, for the neighbour sums of the
// edge pass, {F, F q_e} and u as double-float pairs (rec, udf)
struct PrepArgs {
    int lo, hi;
    const double *u_in, *hst, *q;
    double *qe;
    float4 *rec;
    float2 *udf;
};

struct EdgeArgs {
    SegSet segs;
    int lo, hi;
    const double *u_in, *hst, *K, *qe, *u0;
    const float4 *rec;
    const float2 *udf;
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
    // the double-float records live in the A_FQU area (16 bytes per edge) and
    // the split velocity in the A_FE area (8 bytes per edge)
    return PrepArgs{op.lo, op.hi, arr.a[op.in_u], arr.a[op.hst], arr.a[A_Q], arr.a[A_QE], (float4 *)arr.a[A_FQU],
                    (float2 *)arr.a[A_FE]};
}

inline EdgeArgs edge_args(const Op &op, const DevArrays &arr, double g) {
    double *const *A = arr.a;
    EdgeArgs a;
    a.segs = segs_of(op);
    a.lo = op.lo; a.hi = op.hi;
    a.u_in = A[op.in_u]; a.hst = A[op.hst]; a.K = A[A_K]; a.qe = A[A_QE];
    a.rec = (const float4 *)A[A_FQU]; a.udf = (const float2 *)A[A_FE];
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

// ---------------------------------------------------------------- double-float
// GB300 issues FP64 at 1/64 of its FP32 rate.  The FP64 path therefore takes
// its edgesOnEdge sums on the FP32 pipe in double-float arithmetic: a value
// is the unevaluated sum hi + lo of two floats (about 48 significant bits),
// products are exact through Dekker's product with a fused multiply-add
// (the rounding error of a*b is fma(a, b, -a*b)) and sums through Knuth's
// TwoSum (the error of s = a + b is (a - (s - bb)) + (b - bb), bb = s - a).
// Conversions between double and float pairs go through the bit patterns on
// the integer pipe: GB300's float/double conversion instructions cost about
// as much as an FP64 operation.

FB_HD unsigned long long fb_bits(double x) {
#ifdef __CUDA_ARCH__
    return (unsigned long long)__double_as_longlong(x);
#else
    unsigned long long b;
    std::memcpy(&b, &x, sizeof b);
    return b;
#endif
}
FB_HD double fb_from_bits(unsigned long long b) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)b);
#else
    double x;
    std::memcpy(&x, &b, sizeof x);
    return x;
#endif
}
FB_HD unsigned fb_fbits(float x) {
#ifdef __CUDA_ARCH__
    return __float_as_uint(x);
#else
    unsigned b;
    std::memcpy(&b, &x, sizeof b);
    return b;
#endif
}
FB_HD float fb_ffrom_bits(unsigned b) {
#ifdef __CUDA_ARCH__
    return __uint_as_float(b);
#else
    float x;
    std::memcpy(&x, &b, sizeof x);
    return x;
#endif
}

// x truncated to a float (sign, exponent, top 23 mantissa bits); 0 below the
// smallest normal float; infinities and NaN stay infinite / NaN
FB_HD float df_trunc(double x) {
    const unsigned long long b = fb_bits(x);
    const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
    const int ed = (int)((hw >> 20) & 0x7FFu);
    const unsigned sign = hw & 0x80000000u;
    const unsigned m = ((hw & 0xFFFFFu) << 3) | (lw >> 29);
    if (ed == 0x7FF) return fb_ffrom_bits(sign | 0x7F800000u | (m ? 1u : 0u));
    const int e = ed - 1023 + 127;
    if (e <= 0) return fb_ffrom_bits(sign);
    if (e >= 255) return fb_ffrom_bits(sign | 0x7F800000u);
    return fb_ffrom_bits(sign | ((unsigned)e << 23) | m);
}

// x rounded to the nearest float, ties to even (the IEEE conversion), on the
// integer pipe for results in the normal float range; the rare results
// below it (|x| < 2^-126, zero included) take the conversion instruction
FB_HD float df_round(double x) {
    const unsigned long long b = fb_bits(x);
    const int ed = (int)((b >> 52) & 0x7FFu);
    const int e = ed - 1023 + 127;
    if (e <= 0 || ed == 0x7FF) return (float)x;
    if (e >= 255) return fb_ffrom_bits((unsigned)(b >> 32) & 0x80000000u ? 0xFF800000u : 0x7F800000u);
    const unsigned long long mant = b & ((1ull << 52) - 1ull);
    unsigned r = ((unsigned)(b >> 32) & 0x80000000u) | ((unsigned)e << 23) | (unsigned)(mant >> 29);
    const unsigned rem = (unsigned)(mant & ((1ull << 29) - 1ull));
    if (rem > (1u << 28) || (rem == (1u << 28) && (r & 1u))) ++r;   // a carry moves into the exponent (to infinity past the largest float)
    return fb_ffrom_bits(r);
}

// the double value of a float (exact; subnormal floats become 0)
FB_HD double df_widen(float f) {
    const unsigned u = fb_fbits(f);
    const unsigned e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
    const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
    if (e == 0) return fb_from_bits(sign);
    const unsigned long long ed = e == 0xFFu ? 0x7FFull : (unsigned long long)(e - 127 + 1023);
    return fb_from_bits(sign | (ed << 52) | ((unsigned long long)m << 29));
}

// x as hi + lo: hi is x with the low 29 mantissa bits cleared (a float
// exactly), lo = x - hi (exact in double) truncated to a float; relative
// error at most 2^-47
FB_HD float2 df_split(double x) {
    const double hi = fb_from_bits(fb_bits(x) & ~((1ull << 29) - 1ull));
    return make_float2(df_trunc(hi), df_trunc(x - hi));
}

FB_HD double df_value(float2 s) { return df_widen(s.x) + df_widen(s.y); }

// s += a * b in double-float (the lo * lo term, 2^-48 of the product, dropped)
FB_HD void df_fma(float2 &s, float2 a, float2 b) {
#ifdef __CUDA_ARCH__
    const float ph = __fmul_rn(a.x, b.x);
    float pl = fmaf(a.x, b.x, -ph);
    pl = fmaf(a.x, b.y, fmaf(a.y, b.x, pl));
    const float t = __fadd_rn(s.x, ph);
    const float bb = __fsub_rn(t, s.x);
    const float err = __fadd_rn(__fsub_rn(s.x, __fsub_rn(t, bb)), __fsub_rn(ph, bb));
    s.y = __fadd_rn(s.y, __fadd_rn(err, pl));
#else
    const float ph = a.x * b.x;
    float pl = std::fmaf(a.x, b.x, -ph);
    pl = std::fmaf(a.x, b.y, std::fmaf(a.y, b.x, pl));
    const float t = s.x + ph;
    const float bb = t - s.x;
    const float err = (s.x - (t - bb)) + (ph - bb);
    s.y = s.y + (err + pl);
#endif
    s.x = t;
}

// s += a * b for floats a, b: the product exact as ph + pl (the FMA gives the
// rounding error pl), ph added by TwoSum, the low parts in float
FB_HD void df_add_prod(float2 &s, float a, float b) {
#ifdef __CUDA_ARCH__
    const float ph = __fmul_rn(a, b);
    const float pl = fmaf(a, b, -ph);
    const float t = __fadd_rn(s.x, ph);
    const float bb = __fsub_rn(t, s.x);
    const float err = __fadd_rn(__fsub_rn(s.x, __fsub_rn(t, bb)), __fsub_rn(ph, bb));
    s.y = __fadd_rn(s.y, __fadd_rn(err, pl));
#else
    const float ph = a * b;
    const float pl = std::fmaf(a, b, -ph);
    const float t = s.x + ph;
    const float bb = t - s.x;
    const float err = (s.x - (t - bb)) + (ph - bb);
    s.y = s.y + (err + pl);
#endif
    s.x = t;
}

// 1/x for finite x > 0: a float estimate refined by two Newton steps on
// f(r) = 1/r - x (r <- r + r (1 - x r)), each about doubling the correct bits
FB_HD double rcp_nr(double x) {
#ifdef __CUDA_ARCH__
    double r = df_widen(__fdividef(1.0f, df_trunc(x)));
#else
    double r = df_widen(1.0f / df_trunc(x));
#endif
    r = fma(r, fma(-x, r, 1.0), r);
    return fma(r, fma(-x, r, 1.0), r);
}

// Double-float operations for the FP64 edge pass's forcing terms (the same
// error-free transformations; each result normalised so |lo| <= ulp(hi)/2,
// relative error about 2^-46).  Rounded float operations that the compiler
// may not contract: fadd_ / fsub_ / fmul_.
#ifdef __CUDA_ARCH__
#define FF_ADD(a, b) __fadd_rn((a), (b))
#define FF_SUB(a, b) __fsub_rn((a), (b))
#define FF_MUL(a, b) __fmul_rn((a), (b))
#else
#define FF_ADD(a, b) ((a) + (b))
#define FF_SUB(a, b) ((a) - (b))
#define FF_MUL(a, b) ((a) * (b))
#endif

// s + e with |e| small against s (Dekker's Fast2Sum)
FB_HD float2 ff_norm(float s, float e) {
    const float h = FF_ADD(s, e);
    return make_float2(h, FF_SUB(e, FF_SUB(h, s)));
}

FB_HD float2 ff_add(float2 a, float2 b) {
    const float s = FF_ADD(a.x, b.x);
    const float bb = FF_SUB(s, a.x);
    const float e = FF_ADD(FF_SUB(a.x, FF_SUB(s, bb)), FF_SUB(b.x, bb));
    return ff_norm(s, FF_ADD(e, FF_ADD(a.y, b.y)));
}

FB_HD float2 ff_neg(float2 a) { return make_float2(-a.x, -a.y); }

FB_HD float2 ff_mul(float2 a, float2 b) {
    const float p = FF_MUL(a.x, b.x);
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, fmaf(a.y, b.x, e));
    return ff_norm(p, e);
}

// sqrt(a) for a >= 0: the float root s refined by one Newton step with the
// exact residual a - s^2 (fma); 0 for a <= 0
FB_HD float2 ff_sqrt(float2 a) {
    if (!(a.x > 0.f)) return make_float2(0.f, 0.f);
#ifdef __CUDA_ARCH__
    const float s = __fsqrt_rn(a.x);
#else
    const float s = std::sqrt(a.x);
#endif
    const float r = FF_ADD(fmaf(-s, s, a.x), a.y);
    return ff_norm(s, FF_MUL(r, FF_MUL(0.5f, 1.0f / s)));
}

// 1/a for a > 0: the float reciprocal refined by one Newton step with the
// exact residual 1 - a r (fma)
FB_HD float2 ff_rcp(float2 a) {
    const float r = 1.0f / a.x;
    const float e = FF_SUB(fmaf(-a.x, r, 1.0f), FF_MUL(a.y, r));
    return ff_norm(r, FF_MUL(r, e));
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
// q_v = (zeta_v + f_v) / h_v  (Eq. trisk_vorticity; PV q = eta / h); the
// division through rcp_nr.
FB_HD void vert_body(const DevMesh &m, const VertArgs &a, int v) {
    const int nV = m.nV;
    double z = 0.0, hv = m.Hv64[v];
FB_UNROLL
    for (int j = 0; j < 3; ++j) {
        z += m.cVort[j * nV + v] * a.u_in[m.eov[j * nV + v]];
        hv += m.cKite[j * nV + v] * a.hst[m.cov[j * nV + v]];
    }
    a.q[v] = (z + m.fV[v]) * rcp_nr(hv);
}

// Edge e: thickness flux F_e = h_e u_e with h_e = H_e + (xi_c0 + xi_c1)/2
// (zero on no-flow edges), the edge PV q_e = (q_v0 + q_v1) / 2 and their
// product F_e q_e, in double; F_e, F_e q_e and u_e are stored as
// double-float pairs for the edge pass's neighbour sums.
FB_HD void prep_body(const DevMesh &m, const PrepArgs &a, int e) {
    const int c0 = m.coe0[e], c1 = m.coe1[e];
    const double u = a.u_in[e];
    const double F = m.ebnd[e] ? 0.0 : (m.He64[e] + 0.5 * (a.hst[c0] + a.hst[c1])) * u;
    const double q = 0.5 * (a.q[m.voe0[e]] + a.q[m.voe1[e]]);
    a.qe[e] = q;
    const float2 f = df_split(F), g = df_split(F * q);
    a.rec[e] = make_float4(f.x, f.y, g.x, g.y);
    a.udf[e] = df_split(u);
}

// Edge e: Phi_e = sum_j w_j F_{e_j} (q_e + q_{e_j}) / 2
//                 - [K_c1 - K_c0 + g (xi_c1 - xi_c0)] / d_e  (+ forcing)
// with xi = h + b the stored surface elevation and h_e = H_e + (xi_c0 + xi_c1)/2
// (rotating SWE, Eq. nonlinear_swe, in TRiSK form; forcing of Eq.
// hurricane_model), then the stage update u_s = u0 + c tau Phi or the
// correction sum of Eq. if_correction.  The Coriolis sum is taken as
// (q_e sum_j w_j F_j + sum_j w_j F_j q_j) / 2; the two sums over the
// edgesOnEdge list and the tangential velocity sum_j w_j u_j run in
// double-float on the FP32 pipe (df_fma), and so do the wind stress and
// drag (ff_*); the pressure, kinetic-energy and vortex-pressure gradients
// and the update stay in double.
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
        float2 sF = make_float2(0.f, 0.f), sG = sF, sv = sF;
        for (int j = 0; j < n; ++j) {
            const int x = m.eoe[j * nE + e];
            const float2 w = m.woeDF[j * nE + e];
            const float4 r = a.rec[x];
            df_fma(sF, w, make_float2(r.x, r.y));
            df_fma(sG, w, make_float2(r.z, r.w));
            if (FORCING) df_fma(sv, w, a.udf[x]);
        }
        const double cor = 0.5 * (qself * df_value(sF) + df_value(sG));
        const double h0c = a.hst[c0], h1c = a.hst[c1];
        const double gg = a.split == 1 ? 0.0 : a.g;   // the slow terms leave gravity out
        const double grad = (a.K[c1] - a.K[c0]) + gg * (h1c - h0c);
        phi = cor - grad * m.invDc[e];
        if (FORCING) {
            // wind stress and quadratic drag in double-float: u_e from the edge
            // prep's pair, v_e = sum_j w_j u_j from the sum above
            const float2 ue = a.udf[e];
            const float2 vt = ff_norm(sv.x, sv.y);
            const float2 rhe = ff_rcp(df_split(m.He64[e] + 0.5 * (h0c + h1c)));
            float2 f = make_float2(0.f, 0.f);
            if (fz.flags & FBLTS_FORCE_WIND_STRESS) {
                const float2 dn = ff_add(df_split(fz.windN[e]), ff_neg(ue));
                const float2 dt = ff_add(df_split(fz.windT[e]), ff_neg(vt));
                const float2 mag = ff_sqrt(ff_add(ff_mul(dn, dn), ff_mul(dt, dt)));
                f = ff_mul(ff_mul(df_split(fz.cw[e]), mag), ff_mul(dn, rhe));
            }
            if (fz.flags & FBLTS_FORCE_BOTTOM_DRAG) {
                const float2 sp = ff_sqrt(ff_add(ff_mul(ue, ue), ff_mul(vt, vt)));
                f = ff_add(f, ff_neg(ff_mul(ff_mul(df_split(fz.cd), sp), ff_mul(ue, rhe))));
            }
            phi += df_value(f);
            if (fz.flags & FBLTS_FORCE_VORTEX) phi -= (fz.ps[c1] - fz.ps[c0]) * m.invDc[e] * fz.inv_rho0;
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
