/*
 * FB-LTS oracle: a plain, slow FP64 CPU statement of what the library computes.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this file's library.  It shares no
 * code, header, table or constant with the CUDA path.
 *
 * Contents (paper sections in brackets):
 *   - TRiSK tendencies on a Voronoi C-grid: thickness tendency Psi
 *     [Sec. 2.3, Eq. trisk_thickness], vertex vorticity / thickness / PV and
 *     the tangential flux F_perp [Eq. trisk_vorticity], momentum tendency Phi
 *     of the rotating SWE [Eq. nonlinear_swe] with the hurricane-model wind
 *     stress, bottom drag and surface-pressure terms [Eq. hurricane_model].
 *   - FB-RK(3,2) [Sec. 2.1, Eq. fbrk32].
 *   - FB-LTS [Sec. 2.2]: coarse advancement on the shrinking sets
 *     F^5 -> F_E^4 -> F^3 -> F_E^2 -> F^1 -> IF-1 edges, interface prediction
 *     [Eq. preds, Eq. hstar_preds] stored per k, fine advancement
 *     [Eq. fine_fbrk32], and the interface correction [Eq. if_correction]
 *     re-evaluated after the fine loop with its substitution rules.
 *     More than two levels: each fine subcycle is itself an FB-LTS step of
 *     the next pair of levels (an extension; the paper treats two levels).
 *   - The fast/slow operator splitting [Sec. 3.2, Eq. splitting] and its
 *     variant with the fine region's slow terms re-evaluated once per fine
 *     step [proposed at the end of Sec. 4.2].
 *   - Classical RK4, the reference solution of the convergence experiment
 *     [Sec. 2.3, Fig. convergence] and the paper's comparison scheme
 *     [Sec. 4.2, Tab. 2].
 *   - Global diagnostics: total mass and total absolute vorticity.
 *
 * State.  The prognostic thickness is carried as the surface elevation
 * xi = h + b (b = -H, the bottom): every tendency is the same function of
 * h = xi - b, the pressure gradient g grad(h + b) is g grad(xi) [Eq.
 * nonlinear_swe], and since b does not change, d xi / dt = d h / dt = Psi and
 * every stage, average, prediction and correction formula of the scheme is the
 * same for xi as for h.  Stored this way the state rounds at the precision of
 * the surface displacement (centimetres) rather than of the full depth (up to
 * kilometres), so two correct FP64 evaluations that round differently still
 * agree to far below 1e-10 of the velocity scale over deep water.  The
 * exported calls take and return h; they convert at entry and exit.
 *
 * Every value that the scheme has not defined at a given stage is NaN, so a
 * result that consumed data outside the stated sets comes out NaN and the
 * call returns OM_E_NAN.  Sums run in the plain index order of the mesh
 * lists (edgesOnCell, edgesOnVertex, cellsOnVertex, edgesOnEdge, k).
 * Compile with -ffp-contract=off.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OM_OK 0
#define OM_E_ARG 1
#define OM_E_REGIONS 2
#define OM_E_NAN 3
#define OM_E_OOM 4

#define OM_T_PGRAD 1
#define OM_T_KE 2
#define OM_T_CORIOLIS 4
#define OM_T_LINEAR_FLUX 8
#define OM_T_FORCING 16

/* region classes per interface */
#define RC_FINE 0
#define RC_IF1 1
#define RC_IF2 2
#define RC_INT 3
#define RC_OUT 4

typedef struct {
    int nC, nE, nV, maxE, maxE2;
    const int *cellsOnEdge;     /* [nE*2] */
    const int *nEdgesOnCell;    /* [nC] */
    const int *edgesOnCell;     /* [nC*maxE] */
    const int *verticesOnEdge;  /* [nE*2] */
    const int *cellsOnVertex;   /* [nV*3] */
    const int *edgesOnVertex;   /* [nV*3] */
    const int *nEdgesOnEdge;    /* [nE] */
    const int *edgesOnEdge;     /* [nE*maxE2] */
    const double *weightsOnEdge;/* [nE*maxE2] */
    const double *dcEdge, *dvEdge, *areaCell, *kiteAreasOnVertex, *fVertex, *bottom;
    const double *angleEdge, *xCell, *yCell, *xEdge, *yEdge; /* forcing only */
} om_mesh;

typedef struct {
    double g;
    double beta1, beta2, beta3;
    int terms;
    double H_lin;
    double wind_u, wind_v;
    int wind_stress;
    double cd, rho0, rho_air;
    int vortex;
    double vx_pc, vx_dp, vx_rmax, vx_B, vx_x0, vx_y0, vx_vx, vx_vy, vx_f0;
    int split;   /* 1: fast/slow operator splitting of Phi (Sec. 3.2); 2: its slow terms
                    re-evaluated at the start of every fine step (Sec. 4.2) */
} om_params;

static const double OM_NAN = (double)NAN;

/* ------------------------------------------------------------------ */
/* forcing fields at time t (held fixed over one coarse step)          */
/* ------------------------------------------------------------------ */

/* Holland-type vortex: p(r) = pc + dp exp(-(R/r)^B) and the gradient wind
 * V(r) = sqrt(B dp/rho_air (R/r)^B exp(-(R/r)^B) + (r f0/2)^2) - r f0/2,
 * blowing counter-clockwise about the moving centre. */
static void om_vortex_at(const om_params *p, double x, double y, double t,
                         double *pres, double *wu, double *wv) {
    double cx = p->vx_x0 + p->vx_vx * t, cy = p->vx_y0 + p->vx_vy * t;
    double rx = x - cx, ry = y - cy;
    double r = sqrt(rx * rx + ry * ry);
    double a = (r > 0.0) ? pow(p->vx_rmax / r, p->vx_B) : INFINITY;
    double ex = (r > 0.0) ? exp(-a) : 0.0;
    *pres = p->vx_pc + p->vx_dp * ex;
    if (r <= 0.0 || ex == 0.0) { *wu = 0.0; *wv = 0.0; return; }
    double hf = 0.5 * r * p->vx_f0;
    double V = sqrt(p->vx_B * p->vx_dp / p->rho_air * a * ex + hf * hf) - hf;
    *wu = -V * ry / r;
    *wv = V * rx / r;
}

void om_forcing_fields(const om_mesh *m, const om_params *p, double t,
                       double *windN, double *windT, double *ps) {
    for (int e = 0; e < m->nE; ++e) {
        double wu = p->wind_u, wv = p->wind_v;
        if (p->vortex) {
            double pr, a, b;
            om_vortex_at(p, m->xEdge[e], m->yEdge[e], t, &pr, &a, &b);
            wu += a; wv += b;
        }
        double nx = cos(m->angleEdge[e]), ny = sin(m->angleEdge[e]);
        windN[e] = wu * nx + wv * ny;
        windT[e] = -wu * ny + wv * nx;
    }
    for (int i = 0; i < m->nC; ++i) {
        double pr = 0.0, a, b;
        if (p->vortex) om_vortex_at(p, m->xCell[i], m->yCell[i], t, &pr, &a, &b);
        ps[i] = pr;
    }
}

typedef struct {
    const double *windN, *windT, *ps;
} om_forcing;

/* ------------------------------------------------------------------ */
/* TRiSK operators                                                     */
/* ------------------------------------------------------------------ */

static int present2(const int *pair) { return pair[0] >= 0 && pair[1] >= 0; }

/* Thickness h_i = xi_i - b_i of cell i from the surface elevation xi. */
static double om_h(const om_mesh *m, const double *xi, int i) { return xi[i] - m->bottom[i]; }

/* Thickness flux F_e = h_e u_e with h_e the mean of the two cells (zero on
 * no-flow edges).  [Eq. trisk_thickness: F_e(u_e, h)] */
static double om_flux(const om_mesh *m, const om_params *p, const double *u, const double *xi, int e) {
    const int *ce = m->cellsOnEdge + 2 * e;
    if (!present2(ce)) return 0.0;
    if (p->terms & OM_T_LINEAR_FLUX) return p->H_lin * u[e];
    return 0.5 * (om_h(m, xi, ce[0]) + om_h(m, xi, ce[1])) * u[e];
}

/* Psi_i = -(1/A_i) sum_{e in E_i} n_{e,i} l_e F_e   [Eq. trisk_thickness] */
static double om_psi_cell(const om_mesh *m, const om_params *p, const double *u, const double *xi, int i) {
    double s = 0.0;
    for (int j = 0; j < m->nEdgesOnCell[i]; ++j) {
        int e = m->edgesOnCell[i * m->maxE + j];
        double n = (m->cellsOnEdge[2 * e] == i) ? 1.0 : -1.0;
        s += n * m->dvEdge[e] * om_flux(m, p, u, xi, e);
    }
    return -s / m->areaCell[i];
}

/* K_i = (1/A_i) sum_{e in E_i} (1/4) d_e l_e u_e^2  (TRiSK kinetic energy) */
static double om_ke_cell(const om_mesh *m, const double *u, int i) {
    double s = 0.0;
    for (int j = 0; j < m->nEdgesOnCell[i]; ++j) {
        int e = m->edgesOnCell[i * m->maxE + j];
        s += 0.25 * m->dcEdge[e] * m->dvEdge[e] * u[e] * u[e];
    }
    return s / m->areaCell[i];
}

/* Dual cell v: A_v = sum of the kites of its present cells,
 * zeta_v = (1/A_v) sum_{e in E_v} t_{e,v} d_e u_e with t_{e,v} = -1 when v is
 * the first vertex of e, h_v = (1/A_v) sum kite h_i, q_v = (zeta_v + f_v)/h_v.
 * [Eq. trisk_vorticity and the PV q = eta/h of Sec. 2.3] */
static void om_vertex(const om_mesh *m, const double *u, const double *xi, int v,
                      double *zeta, double *hv, double *q) {
    double av = 0.0, hs = 0.0, cs = 0.0;
    for (int j = 0; j < 3; ++j) {
        int c = m->cellsOnVertex[3 * v + j];
        if (c < 0) continue;
        av += m->kiteAreasOnVertex[3 * v + j];
        hs += m->kiteAreasOnVertex[3 * v + j] * om_h(m, xi, c);
    }
    for (int j = 0; j < 3; ++j) {
        int e = m->edgesOnVertex[3 * v + j];
        if (e < 0) continue;
        double t = (m->verticesOnEdge[2 * e] == v) ? -1.0 : 1.0;
        cs += t * m->dcEdge[e] * u[e];
    }
    *zeta = cs / av;
    *hv = hs / av;
    *q = (*zeta + m->fVertex[v]) / *hv;
}

/* Phi_e for one interior edge, from precomputed K (cells) and q (vertices):
 *   Phi_e = sum_j W_{e,j} F_{e_j} (q_e + q_{e_j})/2              (q F_perp)
 *           - (K_{c1} - K_{c0})/d_e - g (xi_{c1} - xi_{c0})/d_e   (xi = h + b)
 *           + forcing,
 * q_e = (q_{v0} + q_{v1})/2 and F from (u, h) with h the FB-averaged
 * thickness (given as its surface elevation xi).  [Eq. nonlinear_swe;
 * Eq. trisk_vorticity for q F_perp; Eq. hurricane_model for the forcing terms] */
static double om_phi_edge(const om_mesh *m, const om_params *p, const om_forcing *fz,
                          const double *u, const double *xi, const double *K,
                          const double *q, int e) {
    const int *ce = m->cellsOnEdge + 2 * e;
    if (!present2(ce)) return 0.0;
    int c0 = ce[0], c1 = ce[1];
    double dc = m->dcEdge[e];
    double val = 0.0;
    if (p->terms & OM_T_CORIOLIS) {
        const int *ve = m->verticesOnEdge + 2 * e;
        double qe = 0.5 * (q[ve[0]] + q[ve[1]]);
        double s = 0.0;
        for (int j = 0; j < m->nEdgesOnEdge[e]; ++j) {
            int ej = m->edgesOnEdge[e * m->maxE2 + j];
            const int *vj = m->verticesOnEdge + 2 * ej;
            double qj = 0.5 * (q[vj[0]] + q[vj[1]]);
            s += m->weightsOnEdge[e * m->maxE2 + j] * om_flux(m, p, u, xi, ej) * 0.5 * (qe + qj);
        }
        val += s;
    }
    if (p->terms & OM_T_KE) val -= (K[c1] - K[c0]) / dc;
    if (p->terms & OM_T_PGRAD)
        val -= p->g * (xi[c1] - xi[c0]) / dc;
    if ((p->terms & OM_T_FORCING) && fz) {
        double he = 0.5 * (om_h(m, xi, c0) + om_h(m, xi, c1));
        double vt = 0.0;
        for (int j = 0; j < m->nEdgesOnEdge[e]; ++j) {
            int ej = m->edgesOnEdge[e * m->maxE2 + j];
            vt += m->weightsOnEdge[e * m->maxE2 + j] * u[ej];
        }
        if (p->wind_stress) {
            double wn = fz->windN[e], wt = fz->windT[e];
            double U10 = sqrt(wn * wn + wt * wt);
            double cw = (p->rho_air / p->rho0) * (0.75 + 0.067 * U10) * 1e-3;
            double dn = wn - u[e], dt = wt - vt;
            val += cw * sqrt(dn * dn + dt * dt) * dn / he;
        }
        if (p->cd != 0.0) {
            double sp = sqrt(u[e] * u[e] + vt * vt);
            val -= p->cd * sp * u[e] / he;
        }
        if (p->vortex) val -= (fz->ps[c1] - fz->ps[c0]) / (p->rho0 * dc);
    }
    return val;
}

/* Operator splitting [Sec. 3.2, Eq. splitting, Eq. fast_terms].  With
 * p->split, a Phi evaluation inside a coarse step is
 *   Phi(u*, h*) ~ Phi_fast(u*, h*) + Phi_slow(u^n, h^n),
 * Phi_fast = -g grad(h + b) (the external gravity-wave term) and Phi_slow the
 * remaining terms (Coriolis, kinetic-energy gradient, forcing), evaluated once
 * per coarse step from its start time level; Psi is not split.  `slow` holds
 * Phi_slow per edge (NULL: no splitting).
 * p->split == 2 is the variant the paper proposes at the end of Sec. 4.2:
 * while the fine region advances, the slow terms of its edges are evaluated
 * once per fine step, at t^{n,k} (fine cells at their current state, IF-1 at
 * the predictions X^{n,k} of Eq. preds), so the slow subsystem advances with
 * the fine step there; coarse edges, the interface correction included, keep
 * the values of t^n.  With more levels this holds per level pair. */
static double om_phi_stage(const om_mesh *m, const om_params *p, const om_forcing *fz, const double *slow,
                           const double *u, const double *xi, const double *K, const double *q, int e) {
    if (!slow) return om_phi_edge(m, p, fz, u, xi, K, q, e);
    om_params pf = *p;
    pf.terms = p->terms & OM_T_PGRAD;
    return om_phi_edge(m, &pf, NULL, u, xi, K, q, e) + slow[e];
}

static void om_all_K(const om_mesh *m, const double *u, double *K);
static void om_all_q(const om_mesh *m, const double *u, const double *xi, double *q);

/* Phi_slow(u, h) on every edge (0 on no-flow edges), or NULL without splitting. */
static double *om_slow_terms(const om_mesh *m, const om_params *p, const om_forcing *fz, const double *u,
                             const double *xi) {
    if (!p->split) return NULL;
    om_params ps = *p;
    ps.terms = p->terms & ~OM_T_PGRAD;
    double *slow = (double *)malloc(sizeof(double) * (size_t)(m->nE > 0 ? m->nE : 1));
    double *K = (double *)malloc(sizeof(double) * (size_t)(m->nC > 0 ? m->nC : 1));
    double *q = (double *)malloc(sizeof(double) * (size_t)(m->nV > 0 ? m->nV : 1));
    om_all_K(m, u, K);
    om_all_q(m, u, xi, q);
    for (int e = 0; e < m->nE; ++e) slow[e] = om_phi_edge(m, &ps, fz, u, xi, K, q, e);
    free(K);
    free(q);
    return slow;
}

/* helpers computing K on all cells and q on all vertices (NaN where inputs are) */
static void om_all_K(const om_mesh *m, const double *u, double *K) {
    for (int i = 0; i < m->nC; ++i) K[i] = om_ke_cell(m, u, i);
}
static void om_all_q(const om_mesh *m, const double *u, const double *xi, double *q) {
    double z, hv;
    for (int v = 0; v < m->nV; ++v) om_vertex(m, u, xi, v, &z, &hv, &q[v]);
}

/* surface elevation xi = h + b of a thickness array (a new array), and back */
static double *om_to_xi(const om_mesh *m, const double *h) {
    double *xi = (double *)malloc(sizeof(double) * (size_t)(m->nC > 0 ? m->nC : 1));
    for (int i = 0; i < m->nC; ++i) xi[i] = h[i] + m->bottom[i];
    return xi;
}
static void om_from_xi(const om_mesh *m, const double *xi, double *h) {
    for (int i = 0; i < m->nC; ++i) h[i] = xi[i] - m->bottom[i];
}

/* ------------------------------------------------------------------ */
/* exported single-operator entry points (for the operator pins)       */
/* ------------------------------------------------------------------ */

void om_psi(const om_mesh *m, const om_params *p, const double *u, const double *h, double *out) {
    double *xi = om_to_xi(m, h);
    for (int i = 0; i < m->nC; ++i) out[i] = om_psi_cell(m, p, u, xi, i);
    free(xi);
}

void om_phi(const om_mesh *m, const om_params *p, const double *windN, const double *windT,
            const double *ps, const double *u, const double *h, double *out) {
    double *K = malloc(sizeof(double) * m->nC), *q = malloc(sizeof(double) * m->nV);
    om_forcing fz = {windN, windT, ps};
    double *xi = om_to_xi(m, h);
    om_all_K(m, u, K);
    om_all_q(m, u, xi, q);
    for (int e = 0; e < m->nE; ++e) out[e] = om_phi_edge(m, p, windN ? &fz : NULL, u, xi, K, q, e);
    free(K); free(q); free(xi);
}

void om_vertex_fields(const om_mesh *m, const double *u, const double *h,
                      double *zeta, double *hv, double *q) {
    double *xi = om_to_xi(m, h);
    for (int v = 0; v < m->nV; ++v) om_vertex(m, u, xi, v, &zeta[v], &hv[v], &q[v]);
    free(xi);
}

void om_ke(const om_mesh *m, const double *u, double *K) { om_all_K(m, u, K); }

void om_tangential(const om_mesh *m, const double *u, double *vt) {
    for (int e = 0; e < m->nE; ++e) {
        double s = 0.0;
        for (int j = 0; j < m->nEdgesOnEdge[e]; ++j)
            s += m->weightsOnEdge[e * m->maxE2 + j] * u[m->edgesOnEdge[e * m->maxE2 + j]];
        vt[e] = s;
    }
}

/* Total mass sum_i A_i h_i and total absolute vorticity sum_v A_v (zeta_v + f_v),
 * with A_v the sum of the kites of the present cells.  [Sec. 2.3] */
void om_diagnostics(const om_mesh *m, const double *h, const double *u, double *mass, double *absvort) {
    double s = 0.0;
    for (int i = 0; i < m->nC; ++i) s += m->areaCell[i] * h[i];
    *mass = s;
    double w = 0.0;
    for (int v = 0; v < m->nV; ++v) {
        double av = 0.0, cs = 0.0;
        for (int j = 0; j < 3; ++j)
            if (m->cellsOnVertex[3 * v + j] >= 0) av += m->kiteAreasOnVertex[3 * v + j];
        for (int j = 0; j < 3; ++j) {
            int e = m->edgesOnVertex[3 * v + j];
            if (e < 0) continue;
            double t = (m->verticesOnEdge[2 * e] == v) ? -1.0 : 1.0;
            cs += t * m->dcEdge[e] * u[e];
        }
        w += cs + av * m->fVertex[v];
    }
    *absvort = w;
}

/* ------------------------------------------------------------------ */
/* global FB-RK(3,2) and RK4                                           */
/* ------------------------------------------------------------------ */

static int om_has_nan(const double *a, int n) {
    for (int i = 0; i < n; ++i)
        if (a[i] != a[i]) return 1;
    return 0;
}

static double *dalloc(int n) { return (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1)); }

/* One FB-RK(3,2) step on the whole mesh  [Eq. fbrk32]; h holds the surface
 * elevation xi. */
static void om_fbrk32_once(const om_mesh *m, const om_params *p, const om_forcing *fz,
                           double *h, double *u, double dt) {
    int nC = m->nC, nE = m->nE;
    double *h1 = dalloc(nC), *h2 = dalloc(nC), *h3 = dalloc(nC), *hs = dalloc(nC);
    double *u1 = dalloc(nE), *u2 = dalloc(nE), *u3 = dalloc(nE);
    double *K = dalloc(nC), *q = dalloc(m->nV);
    const double b1 = p->beta1, b2 = p->beta2, b3 = p->beta3;
    double *slow = om_slow_terms(m, p, fz, u, h);
    /* stage 1 */
    for (int i = 0; i < nC; ++i) h1[i] = h[i] + dt / 3.0 * om_psi_cell(m, p, u, h, i);
    for (int i = 0; i < nC; ++i) hs[i] = b1 * h1[i] + (1.0 - b1) * h[i];
    om_all_K(m, u, K); om_all_q(m, u, hs, q);
    for (int e = 0; e < nE; ++e) u1[e] = u[e] + dt / 3.0 * om_phi_stage(m, p, fz, slow, u, hs, K, q, e);
    /* stage 2 */
    for (int i = 0; i < nC; ++i) h2[i] = h[i] + dt / 2.0 * om_psi_cell(m, p, u1, h1, i);
    for (int i = 0; i < nC; ++i) hs[i] = b2 * h2[i] + (1.0 - b2) * h[i];
    om_all_K(m, u1, K); om_all_q(m, u1, hs, q);
    for (int e = 0; e < nE; ++e) u2[e] = u[e] + dt / 2.0 * om_phi_stage(m, p, fz, slow, u1, hs, K, q, e);
    /* stage 3 */
    for (int i = 0; i < nC; ++i) h3[i] = h[i] + dt * om_psi_cell(m, p, u2, h2, i);
    for (int i = 0; i < nC; ++i) hs[i] = b3 * h3[i] + (1.0 - 2.0 * b3) * h2[i] + b3 * h[i];
    om_all_K(m, u2, K); om_all_q(m, u2, hs, q);
    for (int e = 0; e < nE; ++e) u3[e] = u[e] + dt * om_phi_stage(m, p, fz, slow, u2, hs, K, q, e);
    free(slow);
    memcpy(h, h3, sizeof(double) * nC);
    memcpy(u, u3, sizeof(double) * nE);
    free(h1); free(h2); free(h3); free(hs); free(u1); free(u2); free(u3); free(K); free(q);
}

static void om_make_forcing(const om_mesh *m, const om_params *p, double t,
                            double *wn, double *wt, double *ps, om_forcing *fz) {
    if (p->terms & OM_T_FORCING) {
        om_forcing_fields(m, p, t, wn, wt, ps);
        fz->windN = wn; fz->windT = wt; fz->ps = ps;
    } else {
        fz->windN = fz->windT = fz->ps = NULL;
    }
}

int om_fbrk32(const om_mesh *m, const om_params *p, double *h, double *u, double dt,
              int nsteps, double t0) {
    double *wn = dalloc(m->nE), *wt = dalloc(m->nE), *ps = dalloc(m->nC);
    double *xi = om_to_xi(m, h);
    om_forcing fz;
    for (int n = 0; n < nsteps; ++n) {
        om_make_forcing(m, p, t0 + n * dt, wn, wt, ps, &fz);
        om_fbrk32_once(m, p, (p->terms & OM_T_FORCING) ? &fz : NULL, xi, u, dt);
    }
    om_from_xi(m, xi, h);
    free(wn); free(wt); free(ps); free(xi);
    return (om_has_nan(h, m->nC) || om_has_nan(u, m->nE)) ? OM_E_NAN : OM_OK;
}

/* Classical four-stage RK4 on (u, h); tendencies Phi(u, h), Psi(u, h). */
int om_rk4(const om_mesh *m, const om_params *p, double *h_io, double *u, double dt, int nsteps, double t0) {
    int nC = m->nC, nE = m->nE;
    double *h = om_to_xi(m, h_io);   /* the surface elevation, advanced below */
    double *kh[4], *ku[4];
    for (int s = 0; s < 4; ++s) { kh[s] = dalloc(nC); ku[s] = dalloc(nE); }
    double *hh = dalloc(nC), *uu = dalloc(nE), *K = dalloc(nC), *q = dalloc(m->nV);
    double *wn = dalloc(nE), *wt = dalloc(nE), *ps = dalloc(nC);
    const double cst[4] = {0.0, 0.5, 0.5, 1.0};
    om_forcing fz;
    for (int n = 0; n < nsteps; ++n) {
        om_make_forcing(m, p, t0 + n * dt, wn, wt, ps, &fz);
        for (int s = 0; s < 4; ++s) {
            for (int i = 0; i < nC; ++i) hh[i] = s ? h[i] + cst[s] * dt * kh[s - 1][i] : h[i];
            for (int e = 0; e < nE; ++e) uu[e] = s ? u[e] + cst[s] * dt * ku[s - 1][e] : u[e];
            for (int i = 0; i < nC; ++i) kh[s][i] = om_psi_cell(m, p, uu, hh, i);
            om_all_K(m, uu, K); om_all_q(m, uu, hh, q);
            for (int e = 0; e < nE; ++e)
                ku[s][e] = om_phi_edge(m, p, (p->terms & OM_T_FORCING) ? &fz : NULL, uu, hh, K, q, e);
        }
        for (int i = 0; i < nC; ++i)
            h[i] += dt / 6.0 * (kh[0][i] + 2.0 * kh[1][i] + 2.0 * kh[2][i] + kh[3][i]);
        for (int e = 0; e < nE; ++e)
            u[e] += dt / 6.0 * (ku[0][e] + 2.0 * ku[1][e] + 2.0 * ku[2][e] + ku[3][e]);
    }
    for (int s = 0; s < 4; ++s) { free(kh[s]); free(ku[s]); }
    free(hh); free(uu); free(K); free(q); free(wn); free(wt); free(ps);
    om_from_xi(m, h, h_io);
    free(h);
    return (om_has_nan(h_io, nC) || om_has_nan(u, nE)) ? OM_E_NAN : OM_OK;
}

/* ------------------------------------------------------------------ */
/* LTS regions  [Sec. 2.2, Fig. lts_regions]                           */
/* ------------------------------------------------------------------ */

/* BFS layer distance from the seed cells across edges with two cells. */
static void om_bfs(const om_mesh *m, const unsigned char *seed, int *dist) {
    int nC = m->nC;
    int *queue = (int *)malloc(sizeof(int) * (size_t)(nC > 0 ? nC : 1));
    int qh = 0, qt = 0;
    for (int i = 0; i < nC; ++i) {
        dist[i] = seed[i] ? 0 : INT32_MAX;
        if (seed[i]) queue[qt++] = i;
    }
    while (qh < qt) {
        int i = queue[qh++];
        for (int j = 0; j < m->nEdgesOnCell[i]; ++j) {
            int e = m->edgesOnCell[i * m->maxE + j];
            const int *ce = m->cellsOnEdge + 2 * e;
            if (!present2(ce)) continue;
            int o = ce[0] == i ? ce[1] : ce[0];
            if (dist[o] == INT32_MAX) { dist[o] = dist[i] + 1; queue[qt++] = o; }
        }
    }
    free(queue);
}

typedef struct {
    int L;
    const int *level;
    int nIF1, nIF2;
    /* per interface l = 0..L-2, arrays of nC / nE */
    unsigned char *ccls, *ecls; /* RC_* */
    int *cdist;                 /* fine cells: layer distance to level <= l (1 = adjacent) */
    int *edist;                 /* fine edges: min cdist over their fine cells */
    unsigned char *in_R;        /* [L*nC]: level >= l */
    unsigned char *e_in_R;      /* [L*nE]: edge has a present cell of level >= l */
} om_regions;

static void om_regions_free(om_regions *r) {
    free(r->ccls); free(r->ecls); free(r->cdist); free(r->edist); free(r->in_R); free(r->e_in_R);
}

/* Classify cells and edges for every pair of adjacent levels:
 * fine = level >= l+1 with band distance to level <= l (F^b holds 2b layers),
 * level-l cells = IF-1 (first nIF1 layers next to the fine region), IF-2
 * (next nIF2 layers) or interior; an edge takes the class of its cell that is
 * closest to the fine region.  Also checks that levels l-1 and l+1 are at
 * least 7 layers apart, so the bands of successive level pairs never meet. */
static int om_regions_build_internal(const om_mesh *m, const int *level, int L, int nIF1, int nIF2,
                                     om_regions *r) {
    int nC = m->nC, nE = m->nE, P = L > 1 ? L - 1 : 1;
    r->L = L; r->level = level; r->nIF1 = nIF1; r->nIF2 = nIF2;
    r->ccls = calloc((size_t)P * nC + 1, 1);
    r->ecls = calloc((size_t)P * nE + 1, 1);
    r->cdist = calloc((size_t)P * nC + 1, sizeof(int));
    r->edist = calloc((size_t)P * nE + 1, sizeof(int));
    r->in_R = calloc((size_t)L * nC + 1, 1);
    r->e_in_R = calloc((size_t)L * nE + 1, 1);
    unsigned char *seed = calloc((size_t)nC + 1, 1);
    int *dF = malloc(sizeof(int) * (size_t)(nC + 1)), *dC = malloc(sizeof(int) * (size_t)(nC + 1));
    int status = OM_OK;
    for (int i = 0; i < nC; ++i)
        if (level[i] < 0 || level[i] >= L) status = OM_E_ARG;
    for (int l = 0; l < L && status == OM_OK; ++l) {
        int cnt = 0;
        for (int i = 0; i < nC; ++i) { r->in_R[l * nC + i] = level[i] >= l; cnt += level[i] == l; }
        if (cnt == 0 && l < L) status = OM_E_REGIONS; /* every level must be populated */
        for (int e = 0; e < nE; ++e) {
            const int *ce = m->cellsOnEdge + 2 * e;
            int in = 0;
            for (int s = 0; s < 2; ++s) if (ce[s] >= 0 && level[ce[s]] >= l) in = 1;
            r->e_in_R[l * nE + e] = (unsigned char)in;
        }
    }
    for (int l = 0; l + 1 < L && status == OM_OK; ++l) {
        for (int i = 0; i < nC; ++i) seed[i] = level[i] >= l + 1;
        om_bfs(m, seed, dF);
        for (int i = 0; i < nC; ++i) seed[i] = level[i] <= l;
        om_bfs(m, seed, dC);
        unsigned char *cc = r->ccls + (size_t)l * nC;
        int *cd = r->cdist + (size_t)l * nC;
        for (int i = 0; i < nC; ++i) {
            cd[i] = 0;
            if (level[i] >= l + 1) { cc[i] = RC_FINE; cd[i] = dC[i]; }
            else if (level[i] == l) cc[i] = dF[i] <= nIF1 ? RC_IF1 : (dF[i] <= nIF1 + nIF2 ? RC_IF2 : RC_INT);
            else cc[i] = RC_OUT;
        }
        unsigned char *ec = r->ecls + (size_t)l * nE;
        int *ed = r->edist + (size_t)l * nE;
        for (int e = 0; e < nE; ++e) {
            const int *ce = m->cellsOnEdge + 2 * e;
            int best = RC_OUT, bd = INT32_MAX;
            for (int s = 0; s < 2; ++s) {
                int c = ce[s];
                if (c < 0) continue;
                if (cc[c] < best) best = cc[c];
                if (cc[c] == RC_FINE && cd[c] < bd) bd = cd[c];
            }
            ec[e] = (unsigned char)best;
            ed[e] = best == RC_FINE ? bd : 0;
        }
        if (l >= 1) {
            for (int i = 0; i < nC; ++i) seed[i] = level[i] >= l + 1;
            om_bfs(m, seed, dF);
            for (int i = 0; i < nC; ++i)
                if (level[i] <= l - 1 && dF[i] < 7) status = OM_E_REGIONS;
        }
    }
    free(seed); free(dF); free(dC);
    return status;
}

/* Export of the region classification for tests: ccls/cdist [(L-1)*nC], ecls/edist [(L-1)*nE]. */
int om_regions_build(const om_mesh *m, const int *level, int L, int nIF1, int nIF2,
                     unsigned char *ccls, int *cdist, unsigned char *ecls, int *edist) {
    om_regions r;
    int st = om_regions_build_internal(m, level, L, nIF1, nIF2, &r);
    if (L > 1) {
        memcpy(ccls, r.ccls, (size_t)(L - 1) * m->nC);
        memcpy(cdist, r.cdist, sizeof(int) * (size_t)(L - 1) * m->nC);
        memcpy(ecls, r.ecls, (size_t)(L - 1) * m->nE);
        memcpy(edist, r.edist, sizeof(int) * (size_t)(L - 1) * m->nE);
    }
    om_regions_free(&r);
    return st;
}

/* ------------------------------------------------------------------ */
/* FB-LTS  [Sec. 2.2]                                                  */
/* ------------------------------------------------------------------ */

/* Below, every cell array (h, H0, HS1, ..., the predictions and the boundary
 * data) holds the surface elevation xi = h + b; om_fblts converts at entry
 * and exit. */

typedef struct {
    const om_mesh *m;
    const om_params *p;
    const om_forcing *fz;
    om_regions *r;
    const int *M;
    int full_band; /* 1: compute every coarse sub-stage on all of F^5 (Sec. 3.3 simplification) */
    int status;
    const double *slow; /* Phi_slow of the current coarse step (splitting), or NULL */
} om_ctx;

/* Interface prediction for one IF-1 value  [Eq. preds; Appendix A]:
 *   X^{n,k}       = (k/M) X~^{n+1} + (1 - k/M) X^n
 *   Xbar^{n,k+1/3} = (k/M) X~^{n+1} + (1/M) X~^{n+1/3} + (1 - (k+1)/M) X^n
 *   Xbar^{n,k+1/2} = (k/M) X~^{n+1} + (1/M) X~^{n+1/2} + (1 - (k+1)/M) X^n
 * x0 = X^n, x13 = X~^{n+1/3}, x12 = X~^{n+1/2}, x1 = X~^{n+1}; outputs may be NULL. */
void om_predict(int k, int M, double x0, double x13, double x12, double x1,
                double *xk, double *xk13, double *xk12) {
    const double Md = (double)M;
    if (xk) *xk = (k / Md) * x1 + (1.0 - k / Md) * x0;
    if (xk13) *xk13 = (k / Md) * x1 + (1.0 / Md) * x13 + (1.0 - (k + 1) / Md) * x0;
    if (xk12) *xk12 = (k / Md) * x1 + (1.0 / Md) * x12 + (1.0 - (k + 1) / Md) * x0;
}

/* Boundary data on the IF-1 cells/edges of the enclosing level pair, for the
 * current subcycle k: the predictions of Eq. preds / Eq. hstar_preds. */
typedef struct {
    const unsigned char *cmask, *emask;
    const double *h0, *u0, *hs1, *us1, *hst1, *hs2, *us2, *hst2, *hst3;
} om_bnd;

static double *nan_cells(const om_ctx *c) {
    double *a = dalloc(c->m->nC);
    for (int i = 0; i < c->m->nC; ++i) a[i] = OM_NAN;
    return a;
}
/* edge arrays start NaN except on no-flow edges, where u = 0 at every time */
static double *nan_edges(const om_ctx *c) {
    double *a = dalloc(c->m->nE);
    for (int e = 0; e < c->m->nE; ++e) a[e] = present2(c->m->cellsOnEdge + 2 * e) ? OM_NAN : 0.0;
    return a;
}
static void put_cells(const om_ctx *c, double *dst, const double *src, const unsigned char *mask) {
    for (int i = 0; i < c->m->nC; ++i) if (mask[i]) dst[i] = src[i];
}
static void put_edges(const om_ctx *c, double *dst, const double *src, const unsigned char *mask) {
    for (int e = 0; e < c->m->nE; ++e) if (mask[e] && present2(c->m->cellsOnEdge + 2 * e)) dst[e] = src[e];
}

/* Phi on the edges of `set`, writing out[e] = base[e] + cdt * Phi_e(u, hs). */
static void stage_u(const om_ctx *c, const unsigned char *set, const double *base, double cdt,
                    const double *u, const double *hs, double *out) {
    const om_mesh *m = c->m;
    double *K = dalloc(m->nC), *q = dalloc(m->nV);
    om_all_K(m, u, K);
    om_all_q(m, u, hs, q);
    for (int e = 0; e < m->nE; ++e)
        if (set[e] && present2(m->cellsOnEdge + 2 * e))
            out[e] = base[e] + cdt * om_phi_stage(m, c->p, c->fz, c->slow, u, hs, K, q, e);
    free(K); free(q);
}

static int om_advance(om_ctx *c, int l, double tau, double *h, double *u, const om_bnd *bnd,
                      double *o_hs2, double *o_us2, double *o_hst3);

/* Finest level in reach: FB-RK(3,2) on R_l with the enclosing IF-1 predictions
 * as boundary data  [Eq. fine_fbrk32]. */
static int om_fbrk_region(om_ctx *c, int l, double tau, double *h, double *u, const om_bnd *bnd,
                          double *o_hs2, double *o_us2, double *o_hst3) {
    const om_mesh *m = c->m;
    const om_params *p = c->p;
    int nC = m->nC, nE = m->nE;
    const unsigned char *Rc = c->r->in_R + (size_t)l * nC, *Re = c->r->e_in_R + (size_t)l * nE;
    double *H0 = nan_cells(c), *U0 = nan_edges(c);
    double *HS1 = nan_cells(c), *HST1 = nan_cells(c), *HS2 = nan_cells(c), *HST2 = nan_cells(c);
    double *HN = nan_cells(c), *HST3 = nan_cells(c);
    double *US1 = nan_edges(c), *US2 = nan_edges(c), *UN = nan_edges(c);
    put_cells(c, H0, h, Rc); put_edges(c, U0, u, Re);
    if (bnd) {
        put_cells(c, H0, bnd->h0, bnd->cmask); put_edges(c, U0, bnd->u0, bnd->emask);
        put_cells(c, HS1, bnd->hs1, bnd->cmask); put_cells(c, HST1, bnd->hst1, bnd->cmask);
        put_edges(c, US1, bnd->us1, bnd->emask);
        put_cells(c, HS2, bnd->hs2, bnd->cmask); put_cells(c, HST2, bnd->hst2, bnd->cmask);
        put_edges(c, US2, bnd->us2, bnd->emask);
        put_cells(c, HST3, bnd->hst3, bnd->cmask);
    }
    for (int i = 0; i < nC; ++i) if (Rc[i]) {
        HS1[i] = H0[i] + tau / 3.0 * om_psi_cell(m, p, U0, H0, i);
        HST1[i] = p->beta1 * HS1[i] + (1.0 - p->beta1) * H0[i];
    }
    stage_u(c, Re, U0, tau / 3.0, U0, HST1, US1);
    for (int i = 0; i < nC; ++i) if (Rc[i]) {
        HS2[i] = H0[i] + tau / 2.0 * om_psi_cell(m, p, US1, HS1, i);
        HST2[i] = p->beta2 * HS2[i] + (1.0 - p->beta2) * H0[i];
    }
    stage_u(c, Re, U0, tau / 2.0, US1, HST2, US2);
    for (int i = 0; i < nC; ++i) if (Rc[i]) {
        HN[i] = H0[i] + tau * om_psi_cell(m, p, US2, HS2, i);
        HST3[i] = p->beta3 * HN[i] + (1.0 - 2.0 * p->beta3) * HS2[i] + p->beta3 * H0[i];
    }
    stage_u(c, Re, U0, tau, US2, HST3, UN);
    for (int i = 0; i < nC; ++i) if (Rc[i]) {
        if (HN[i] != HN[i]) c->status = OM_E_NAN;
        h[i] = HN[i];
        if (o_hs2) { o_hs2[i] = HS2[i]; o_hst3[i] = HST3[i]; }
    }
    for (int e = 0; e < nE; ++e) if (Re[e]) {
        if (UN[e] != UN[e]) c->status = OM_E_NAN;
        u[e] = UN[e];
        if (o_us2) o_us2[e] = US2[e];
    }
    free(H0); free(U0); free(HS1); free(HST1); free(HS2); free(HST2); free(HN); free(HST3);
    free(US1); free(US2); free(UN);
    return c->status;
}

/* Two-level FB-LTS step between level l (coarse) and levels >= l+1 (fine)
 * [Sec. 2.2 steps 1-4]; the fine advancement recurses into om_advance. */
static int om_fblts_region(om_ctx *c, int l, double tau, double *h, double *u, const om_bnd *bnd,
                           double *o_hs2, double *o_us2, double *o_hst3) {
    const om_mesh *m = c->m;
    const om_params *p = c->p;
    int nC = m->nC, nE = m->nE, Mk = c->M[l];
    const unsigned char *Rc = c->r->in_R + (size_t)l * nC, *Re = c->r->e_in_R + (size_t)l * nE;
    const unsigned char *cc = c->r->ccls + (size_t)l * nC, *ec = c->r->ecls + (size_t)l * nE;
    const int *cd = c->r->cdist + (size_t)l * nC, *ed = c->r->edist + (size_t)l * nE;
    const double b1 = p->beta1, b2 = p->beta2, b3 = p->beta3;

    /* membership masks */
    unsigned char *cF5 = calloc(nC + 1, 1), *cF3 = calloc(nC + 1, 1), *cF1 = calloc(nC + 1, 1);
    unsigned char *cCo = calloc(nC + 1, 1), *cIF1 = calloc(nC + 1, 1), *cIF12 = calloc(nC + 1, 1);
    unsigned char *cINT = calloc(nC + 1, 1), *cFine = calloc(nC + 1, 1), *cIF2INT = calloc(nC + 1, 1);
    unsigned char *eF4 = calloc(nE + 1, 1), *eF2 = calloc(nE + 1, 1), *eCo = calloc(nE + 1, 1);
    unsigned char *eIF1 = calloc(nE + 1, 1), *eIF12 = calloc(nE + 1, 1), *eINT = calloc(nE + 1, 1);
    unsigned char *eS3 = calloc(nE + 1, 1), *eFine = calloc(nE + 1, 1), *eIF2INT = calloc(nE + 1, 1);
    unsigned char *cS1 = calloc(nC + 1, 1), *cS2 = calloc(nC + 1, 1), *cS3 = calloc(nC + 1, 1);
    unsigned char *eS1 = calloc(nE + 1, 1), *eS2 = calloc(nE + 1, 1);
    int fb = c->full_band;
    for (int i = 0; i < nC; ++i) {
        if (!Rc[i]) continue;
        int fine = cc[i] == RC_FINE;
        cFine[i] = fine;
        cF5[i] = fine && cd[i] <= 10;
        cF3[i] = fine && cd[i] <= (fb ? 10 : 6);
        cF1[i] = fine && cd[i] <= (fb ? 10 : 2);
        cCo[i] = cc[i] == RC_IF1 || cc[i] == RC_IF2 || cc[i] == RC_INT;
        cIF1[i] = cc[i] == RC_IF1;
        cIF12[i] = cc[i] == RC_IF1 || cc[i] == RC_IF2;
        cINT[i] = cc[i] == RC_INT;
        cIF2INT[i] = cc[i] == RC_IF2 || cc[i] == RC_INT;
        cS1[i] = cF5[i] || cCo[i];
        cS2[i] = cF3[i] || cCo[i];
        cS3[i] = cF1[i] || cCo[i];
    }
    for (int e = 0; e < nE; ++e) {
        if (!Re[e]) continue;
        int fine = ec[e] == RC_FINE;
        eFine[e] = fine;
        eF4[e] = fine && ed[e] <= (fb ? 10 : 8);
        eF2[e] = fine && ed[e] <= (fb ? 10 : 4);
        eCo[e] = ec[e] == RC_IF1 || ec[e] == RC_IF2 || ec[e] == RC_INT;
        eIF1[e] = ec[e] == RC_IF1;
        eIF12[e] = ec[e] == RC_IF1 || ec[e] == RC_IF2;
        eINT[e] = ec[e] == RC_INT;
        eIF2INT[e] = ec[e] == RC_IF2 || ec[e] == RC_INT;
        eS1[e] = eF4[e] || eCo[e];
        eS2[e] = eF2[e] || eCo[e];
        eS3[e] = (fb && fine && ed[e] <= 10) || eIF1[e] || eINT[e];
    }

    /* ---- step 1: coarse advancement (tilde on F^l, IF-1, IF-2; bar on int) */
    double *H0 = nan_cells(c), *U0 = nan_edges(c);
    double *HS1 = nan_cells(c), *HST1 = nan_cells(c), *HS2 = nan_cells(c), *HST2 = nan_cells(c);
    double *HS3 = nan_cells(c), *HST3 = nan_cells(c);
    double *US1 = nan_edges(c), *US2 = nan_edges(c), *US3 = nan_edges(c);
    put_cells(c, H0, h, Rc); put_edges(c, U0, u, Re);
    if (bnd) {
        put_cells(c, H0, bnd->h0, bnd->cmask); put_edges(c, U0, bnd->u0, bnd->emask);
        put_cells(c, HS1, bnd->hs1, bnd->cmask); put_cells(c, HST1, bnd->hst1, bnd->cmask);
        put_edges(c, US1, bnd->us1, bnd->emask);
        put_cells(c, HS2, bnd->hs2, bnd->cmask); put_cells(c, HST2, bnd->hst2, bnd->cmask);
        put_edges(c, US2, bnd->us2, bnd->emask);
        put_cells(c, HST3, bnd->hst3, bnd->cmask);
    }
    for (int i = 0; i < nC; ++i) if (cS1[i]) {           /* thickness stage 1: F^5 U C */
        HS1[i] = H0[i] + tau / 3.0 * om_psi_cell(m, p, U0, H0, i);
        HST1[i] = b1 * HS1[i] + (1.0 - b1) * H0[i];
    }
    stage_u(c, eS1, U0, tau / 3.0, U0, HST1, US1);        /* velocity stage 1: F_E^4 U C_E */
    for (int i = 0; i < nC; ++i) if (cS2[i]) {           /* thickness stage 2: F^3 U C */
        HS2[i] = H0[i] + tau / 2.0 * om_psi_cell(m, p, US1, HS1, i);
        HST2[i] = b2 * HS2[i] + (1.0 - b2) * H0[i];
    }
    stage_u(c, eS2, U0, tau / 2.0, US1, HST2, US2);       /* velocity stage 2: F_E^2 U C_E */
    for (int i = 0; i < nC; ++i) if (cS3[i]) {           /* thickness stage 3: F^1 U C */
        HS3[i] = H0[i] + tau * om_psi_cell(m, p, US2, HS2, i);
        HST3[i] = b3 * HS3[i] + (1.0 - 2.0 * b3) * HS2[i] + b3 * H0[i];
    }
    stage_u(c, eS3, U0, tau, US2, HST3, US3);             /* velocity stage 3: IF-1 and int edges */

    /* ---- step 2: interface prediction on IF-1, stored for every k */
    double **hP = malloc(sizeof(double *) * (Mk + 1));
    double **uP = malloc(sizeof(double *) * Mk), **hP13 = malloc(sizeof(double *) * Mk);
    double **uP13 = malloc(sizeof(double *) * Mk), **hP12 = malloc(sizeof(double *) * Mk);
    double **uP12 = malloc(sizeof(double *) * Mk), **sP1 = malloc(sizeof(double *) * Mk);
    double **sP2 = malloc(sizeof(double *) * Mk), **sP3 = malloc(sizeof(double *) * Mk);
    const double Md = (double)Mk;
    for (int k = 0; k <= Mk; ++k) {
        hP[k] = nan_cells(c);
        for (int i = 0; i < nC; ++i) if (cIF1[i])
            om_predict(k, Mk, H0[i], HS1[i], HS2[i], HS3[i], &hP[k][i], NULL, NULL);
    }
    for (int k = 0; k < Mk; ++k) {
        uP[k] = nan_edges(c); uP13[k] = nan_edges(c); uP12[k] = nan_edges(c);
        hP13[k] = nan_cells(c); hP12[k] = nan_cells(c);
        sP1[k] = nan_cells(c); sP2[k] = nan_cells(c); sP3[k] = nan_cells(c);
        for (int e = 0; e < nE; ++e) if (eIF1[e] && present2(m->cellsOnEdge + 2 * e))
            om_predict(k, Mk, U0[e], US1[e], US2[e], US3[e], &uP[k][e], &uP13[k][e], &uP12[k][e]);
        for (int i = 0; i < nC; ++i) if (cIF1[i]) {
            double dummy;
            om_predict(k, Mk, H0[i], HS1[i], HS2[i], HS3[i], &dummy, &hP13[k][i], &hP12[k][i]);
        }
    }
    /* predicted FB averages on IF-1  [Eq. hstar_preds] */
    for (int k = 0; k < Mk; ++k)
        for (int i = 0; i < nC; ++i) if (cIF1[i]) {
            sP1[k][i] = b1 * hP13[k][i] + (1.0 - b1) * hP[k][i];
            sP2[k][i] = b2 * hP12[k][i] + (1.0 - b2) * hP[k][i];
            sP3[k][i] = b3 * hP[k + 1][i] + (1.0 - 2.0 * b3) * hP12[k][i] + b3 * hP[k][i];
        }

    /* ---- step 3: fine advancement, M subcycles of tau/M */
    double **fH2 = malloc(sizeof(double *) * Mk), **fU2 = malloc(sizeof(double *) * Mk);
    double **fS3 = malloc(sizeof(double *) * Mk);
    for (int k = 0; k < Mk && c->status == OM_OK; ++k) {
        om_bnd in = {cIF1, eIF1, hP[k], uP[k], hP13[k], uP13[k], sP1[k], hP12[k], uP12[k], sP2[k], sP3[k]};
        fH2[k] = nan_cells(c); fU2[k] = nan_edges(c); fS3[k] = nan_cells(c);
        const double *outer = c->slow;
        double *slow_k = NULL;
        if (p->split == 2) {
            /* slow terms of the fine edges at t^{n,k}: fine cells and edges as they
             * stand after k subcycles, IF-1 at the predictions, the rest undefined */
            double *Hk = nan_cells(c), *Uk = nan_edges(c);
            put_cells(c, Hk, h, cFine); put_edges(c, Uk, u, eFine);
            put_cells(c, Hk, hP[k], cIF1); put_edges(c, Uk, uP[k], eIF1);
            double *fresh = om_slow_terms(m, p, c->fz, Uk, Hk);
            slow_k = dalloc(nE);
            for (int e = 0; e < nE; ++e) slow_k[e] = eFine[e] ? fresh[e] : outer[e];
            c->slow = slow_k;
            free(fresh); free(Hk); free(Uk);
        }
        om_advance(c, l + 1, tau / Md, h, u, &in, fH2[k], fU2[k], fS3[k]);
        c->slow = outer;
        free(slow_k);
    }

    /* ---- step 4: interface correction on IF-1 and IF-2 [Eq. if_correction] */
    if (c->status == OM_OK) {
        double *acch = dalloc(nC), *accu = dalloc(nE);
        for (int i = 0; i < nC; ++i) acch[i] = 0.0;
        for (int e = 0; e < nE; ++e) accu[e] = 0.0;
        for (int k = 0; k < Mk; ++k) {
            double *Ub = nan_edges(c), *Hb = nan_cells(c), *Hs = nan_cells(c);
            put_edges(c, Ub, fU2[k], eFine); put_edges(c, Ub, uP12[k], eIF1); put_edges(c, Ub, US2, eIF2INT);
            put_cells(c, Hb, fH2[k], cFine); put_cells(c, Hb, hP12[k], cIF1); put_cells(c, Hb, HS2, cIF2INT);
            put_cells(c, Hs, fS3[k], cFine); put_cells(c, Hs, sP3[k], cIF1); put_cells(c, Hs, HST3, cIF2INT);
            for (int i = 0; i < nC; ++i) if (cIF12[i]) acch[i] += om_psi_cell(m, p, Ub, Hb, i);
            double *K = dalloc(nC), *q = dalloc(m->nV);
            om_all_K(m, Ub, K);
            om_all_q(m, Ub, Hs, q);
            for (int e = 0; e < nE; ++e)
                if (eIF12[e] && present2(m->cellsOnEdge + 2 * e))
                    accu[e] += om_phi_stage(m, p, c->fz, c->slow, Ub, Hs, K, q, e);
            free(K); free(q); free(Ub); free(Hb); free(Hs);
        }
        for (int i = 0; i < nC; ++i) {
            if (cIF12[i]) h[i] = H0[i] + (tau / Md) * acch[i];
            else if (cINT[i]) h[i] = HS3[i];
            if ((cIF12[i] || cINT[i]) && h[i] != h[i]) c->status = OM_E_NAN;
        }
        for (int e = 0; e < nE; ++e) {
            if (!present2(m->cellsOnEdge + 2 * e)) continue;
            if (eIF12[e]) u[e] = U0[e] + (tau / Md) * accu[e];
            else if (eINT[e]) u[e] = US3[e];
            if ((eIF12[e] || eINT[e]) && u[e] != u[e]) c->status = OM_E_NAN;
        }
        free(acch); free(accu);
        /* stage data for the enclosing level pair: bar data on the interior */
        if (o_hs2) {
            for (int i = 0; i < nC; ++i) if (cINT[i]) { o_hs2[i] = HS2[i]; o_hst3[i] = HST3[i]; }
            for (int e = 0; e < nE; ++e) if (eINT[e]) o_us2[e] = US2[e];
        }
    }
    for (int k = 0; k < Mk; ++k) {
        free(uP[k]); free(uP13[k]); free(uP12[k]); free(hP13[k]); free(hP12[k]);
        free(sP1[k]); free(sP2[k]); free(sP3[k]); free(fH2[k]); free(fU2[k]); free(fS3[k]);
    }
    for (int k = 0; k <= Mk; ++k) free(hP[k]);
    free(hP); free(uP); free(uP13); free(uP12); free(hP13); free(hP12); free(sP1); free(sP2); free(sP3);
    free(fH2); free(fU2); free(fS3);
    free(H0); free(U0); free(HS1); free(HST1); free(HS2); free(HST2); free(HS3); free(HST3);
    free(US1); free(US2); free(US3);
    free(cF5); free(cF3); free(cF1); free(cCo); free(cIF1); free(cIF12); free(cINT); free(cFine); free(cIF2INT);
    free(eF4); free(eF2); free(eCo); free(eIF1); free(eIF12); free(eINT); free(eS3); free(eFine); free(eIF2INT);
    free(cS1); free(cS2); free(cS3); free(eS1); free(eS2);
    return c->status;
}

static int om_advance(om_ctx *c, int l, double tau, double *h, double *u, const om_bnd *bnd,
                      double *o_hs2, double *o_us2, double *o_hst3) {
    if (c->status != OM_OK) return c->status;
    if (l + 1 >= c->r->L) return om_fbrk_region(c, l, tau, h, u, bnd, o_hs2, o_us2, o_hst3);
    return om_fblts_region(c, l, tau, h, u, bnd, o_hs2, o_us2, o_hst3);
}

/* nsteps coarse FB-LTS steps of size dt.  level[i] in [0, L), M[l] = ratio of
 * the time steps of levels l and l+1.  full_band = 0 follows the shrinking
 * sets of Sec. 2.2 literally; 1 computes every coarse sub-stage on all of F^5. */
int om_fblts(const om_mesh *m, const om_params *p, const int *level, int L, const int *M,
             int nIF1, int nIF2, int full_band, double *h_io, double *u, double dt, int nsteps, double t0) {
    if (L < 1) return OM_E_ARG;
    for (int l = 0; l + 1 < L; ++l) if (M[l] < 1) return OM_E_ARG;
    om_regions r;
    int st = om_regions_build_internal(m, level, L, nIF1, nIF2, &r);
    if (st != OM_OK) { om_regions_free(&r); return st; }
    double *h = om_to_xi(m, h_io);   /* the surface elevation, advanced below */
    double *wn = dalloc(m->nE), *wt = dalloc(m->nE), *ps = dalloc(m->nC);
    om_ctx c = {m, p, NULL, &r, M, full_band, OM_OK, NULL};
    om_forcing fz;
    for (int n = 0; n < nsteps && c.status == OM_OK; ++n) {
        om_make_forcing(m, p, t0 + n * dt, wn, wt, ps, &fz);
        c.fz = (p->terms & OM_T_FORCING) ? &fz : NULL;
        double *slow = om_slow_terms(m, p, c.fz, u, h);
        c.slow = slow;
        om_advance(&c, 0, dt, h, u, NULL, NULL, NULL, NULL);
        free(slow);
        c.slow = NULL;
    }
    free(wn); free(wt); free(ps);
    om_regions_free(&r);
    om_from_xi(m, h, h_io);
    free(h);
    if (c.status == OM_OK && (om_has_nan(h_io, m->nC) || om_has_nan(u, m->nE))) c.status = OM_E_NAN;
    return c.status;
}
