// Host check of the FP32 cell-side TRiSK pass: trisk32_body and the edge
// pass's phi_from_shares (paper_2405_10505_gb300/csrc/kernel_bodies32.cuh,
// compiled here for the host) against the explicit edgesOnEdge /
// weightsOnEdge form of the momentum tendency (Eq. trisk_vorticity with the
// kinetic-energy and pressure gradients of Eq. nonlinear_swe), summed in
// double, on a mesh built by the library's own host mesh builder and random
// fields.  trisk_share_check returns 0 and writes {max error / scale, edges
// checked, row width} to out[3].
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <random>
#include <vector>

#include "fblts_internal.h"
#include "kernel_bodies32.cuh"

namespace fblts {
void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    std::vfprintf(stderr, fmt, ap);
    va_end(ap);
    std::fputc('\n', stderr);
}
}  // namespace fblts

using namespace fblts;

extern "C" int trisk_share_check(const fblts_mesh_desc *d, unsigned long long seed, double *out) {
    HostMesh hm;
    if (build_host_mesh(d, hm) != FBLTS_OK || !hm.rows_canonical) return 1;
    const int nC = hm.nC, nE = hm.nE, nV = hm.nV, W2 = hm.maxE2;
    const float g = 9.80616f;
    std::mt19937_64 rng(seed);
    std::uniform_real_distribution<float> U(-1.f, 1.f);
    std::vector<float> u(nE), xs(nC), q(nV), K(nC), He(nE);
    for (int e = 0; e < nE; ++e) {
        u[e] = hm.ebnd[e] ? 0.f : U(rng);              // no-flow edges carry no flow
        He[e] = 1000.f * (1.f + 0.5f * U(rng));
    }
    for (int c = 0; c < nC; ++c) {
        xs[c] = U(rng);                                 // surface elevation xi* [m]
        K[c] = 0.5f * (1.f + U(rng));
    }
    for (int v = 0; v < nV; ++v) q[v] = 1e-7f * (1.f + 0.5f * U(rng));   // PV (zeta + f) / h
    std::vector<float> rowP(hm.rowP.begin(), hm.rowP.end()), invDc32(hm.invDc.begin(), hm.invDc.end());
    std::vector<float2> el2(nE), sh(2 * (size_t)nE), bx(nC);
    for (int e = 0; e < nE; ++e) el2[e] = make_float2((float)hm.dvE[e], He[e]);
    DevMesh m{};
    m.nC = nC; m.nE = nE; m.nV = nV;
    m.nEoC = hm.nEoC.data();
    m.rowS = hm.rowS;
    m.rowE = hm.rowE.data(); m.rowN = hm.rowN.data(); m.rowV = hm.rowV.data(); m.rowP = rowP.data();
    m.el2 = el2.data();
    m.invDc32 = invDc32.data();
    TriskArgs32 a{0, nC, u.data(), xs.data(), K.data(), q.data(), sh.data(), bx.data(), g, 0.f};
    DevForcing fz{};
    for (int i = 0; i < nC; ++i) {
        if (hm.rowS == 8) trisk32_body<8, false>(m, a, fz, i);
        else trisk32_body<12, false>(m, a, fz, i);
    }
    double worst = 0.0;
    int checked = 0;
    for (int e = 0; e < nE; ++e) {
        if (hm.ebnd[e]) continue;
        const int c0 = hm.coe[2 * e], c1 = hm.coe[2 * e + 1];
        const double qe = 0.5 * ((double)q[hm.voe[2 * e]] + q[hm.voe[2 * e + 1]]);
        double cor = 0.0, mag = 0.0;
        for (int j = 0; j < hm.nEoE[e]; ++j) {
            const int x = hm.eoe[(size_t)e * W2 + j];
            const double hx = He[x] + 0.5 * ((double)xs[hm.coe[2 * x]] + xs[hm.coe[2 * x + 1]]);
            const double qx = 0.5 * ((double)q[hm.voe[2 * x]] + q[hm.voe[2 * x + 1]]);
            const double t = hm.woe[(size_t)e * W2 + j] * hx * u[x] * 0.5 * (qe + qx);
            cor += t;
            mag += std::fabs(t);
        }
        const double B0 = (double)K[c0] + (double)g * xs[c0], B1 = (double)K[c1] + (double)g * xs[c1];
        const double ref = cor - (B1 - B0) * hm.invDc[e];
        const float4 s = make_float4(sh[2 * (size_t)e].x, sh[2 * (size_t)e].y, sh[2 * (size_t)e + 1].x,
                                     sh[2 * (size_t)e + 1].y);
        const float phi = phi_from_shares<false>(m, u.data(), fz, e, s, bx[c0], bx[c1]);
        const double scale = mag + (std::fabs(B0) + std::fabs(B1)) * hm.invDc[e];
        if (scale > 0) worst = std::fmax(worst, std::fabs((double)phi - ref) / scale);
        ++checked;
    }
    out[0] = worst;
    out[1] = checked;
    out[2] = hm.rowS;
    return 0;
}
