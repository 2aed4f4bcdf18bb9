// Host check of the FP32 cell pass (cell32_body of
// paper_2405_10505_gb300/csrc/kernel_bodies32.cuh, compiled here for the host)
// on a mesh built by the library's host mesh builder, with random fields:
//   - K_i against (1/A_i) sum_j (d_e l_e / 4) u_e^2 in double;
//   - the correction-sum mode (exact flux products summed in double-float)
//     against Psi_i = -(1/A_i) sum_j n_{e,i} l_e F_e, F_e = (H_e + (xi_i +
//     xi_nb)/2) u_e with the float flux, summed in double (Eq. trisk_thickness);
//   - mass: sum_i A_i Psi_i, which cancels edge by edge (Theorem 1).
// cell_pass_check returns 0 and writes {max K error / K, max Psi error / sum
// |terms|, |sum A Psi| / sum |A terms|, cells} to out[4].
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

extern "C" int cell_pass_check(const fblts_mesh_desc *d, unsigned long long seed, double *out) {
    HostMesh hm;
    if (build_host_mesh(d, hm) != FBLTS_OK || !hm.rows_canonical) return 1;
    const int nC = hm.nC, nE = hm.nE, W = hm.maxE;
    std::mt19937_64 rng(seed);
    std::uniform_real_distribution<float> U(-1.f, 1.f);
    std::vector<float> u(nE), xi(nC), He(nE), ke32(hm.keE.begin(), hm.keE.end()), invA32(hm.invA.begin(), hm.invA.end());
    for (int e = 0; e < nE; ++e) {
        u[e] = hm.ebnd[e] ? 0.f : U(rng);
        He[e] = 1000.f * (1.f + 0.5f * U(rng));
    }
    for (int c = 0; c < nC; ++c) xi[c] = U(rng);
    std::vector<float2> el2(nE);
    for (int e = 0; e < nE; ++e) el2[e] = make_float2((float)hm.dvE[e], He[e]);
    DevMesh m{};
    m.nC = nC; m.nE = nE;
    m.nEoC = hm.nEoC.data();
    m.rowS = hm.rowS;
    m.rowE = hm.rowE.data(); m.rowN = hm.rowN.data();
    m.el2 = el2.data(); m.ke32 = ke32.data();
    m.invA32 = invA32.data(); m.invA = hm.invA.data();
    std::vector<float> K(nC), dummy(nC);
    std::vector<double> acc(nC), hstate(nC);
    CellArgs32 a{};
    a.segs.nseg = 1;
    a.segs.seg[0] = Seg{0, nC, SEG_ACC_SET};
    a.lo = 0; a.hi = nC;
    a.u_in = u.data(); a.xi_in = xi.data(); a.xi0 = xi.data(); a.xiprev = xi.data();
    a.xi_out = dummy.data(); a.xi_shadow = dummy.data(); a.hst_out = dummy.data(); a.K = K.data();
    a.h_state = hstate.data(); a.acc = acc.data();
    for (int i = 0; i < nC; ++i) {
        if (hm.rowS == 8) cell32_body<8, true>(m, a, i);
        else cell32_body<12, true>(m, a, i);
    }
    double wk = 0.0, wp = 0.0, mass = 0.0, mass_scale = 0.0;
    for (int i = 0; i < nC; ++i) {
        double k = 0.0, psi = 0.0, mag = 0.0;
        for (int j = 0; j < hm.nEoC[i]; ++j) {
            const int e = hm.eoc[(size_t)i * W + j];
            const int nb = hm.coc[(size_t)i * W + j];
            k += hm.keE[e] * (double)u[e] * u[e];
            // the float flux of the kernel, the same from both cells of the edge
            const float F = (He[e] + 0.5f * (xi[i] + xi[nb])) * u[e];
            const double n = hm.coe[2 * e] == i ? 1.0 : -1.0;      // n_{e,i}: +1 for the first cell
            const double t = -n * (double)el2[e].x * (double)F;
            psi += t;
            mag += std::fabs(t);
        }
        k *= hm.invA[i];
        if (k > 0) wk = std::fmax(wk, std::fabs((double)K[i] - k) / k);
        if (mag > 0) wp = std::fmax(wp, std::fabs(acc[i] / hm.invA[i] - psi) / mag);
        mass += acc[i] / hm.invA[i];
        mass_scale += mag;
    }
    out[0] = wk;
    out[1] = wp;
    out[2] = std::fabs(mass) / mass_scale;
    out[3] = nC;
    return 0;
}
