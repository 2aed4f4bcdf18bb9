// Device-side structures shared by the kernels and the C ABI implementation.
#pragma once

#include <cuda_runtime.h>

#include "fblts_internal.h"

namespace fblts {

// Mesh metadata on the device, structure of arrays in band order.
// Per-element lists are stored slot-major: x[j * n + i].
struct DevMesh {
    int nC, nE, nV, maxE, maxE2;
    const int *nEoC, *eoc, *coc;        // cells
    const double *cDiv, *cKE;           // -n_{e,i} l_e / A_i, d_e l_e / (4 A_i)
    const double *bottom, *area;
    const int *coe0, *coe1, *voe0, *voe1;  // edges
    const int *nEoE, *eoe;
    const double *woe, *invDc;
    const unsigned char *ebnd;
    const double *cosE, *sinE, *xE, *yE, *xC, *yC;
    const int *eov, *cov;               // vertices
    const double *cVort, *cKite, *fV, *Av;
};

struct DevForcing {
    int flags;                 // FBLTS_FORCE_* bits
    double *windN, *windT, *cw, *ps;
    double wind_u, wind_v, cd, rho0, rho_air;
    double vx[9];
    double t0, dt;
    const long long *step;     // device step counter
};

struct DevArrays {
    double *a[A_COUNT];
};

struct SegSet {
    int nseg;
    Seg seg[MAX_SEG];
};

// launches one schedule op on the stream
cudaError_t launch_op(const Op &op, const DevMesh &m, const DevArrays &arr, const DevForcing &fz,
                      double g, long long *step_counter, cudaStream_t st);

// caller-order <-> band-order copies
cudaError_t launch_gather(double *dst, const double *src, const int *idx, int n, cudaStream_t st);
cudaError_t launch_zero_boundary(double *u, const unsigned char *ebnd, int nE, cudaStream_t st);

// deterministic reductions: mass = sum A_i h_i, absolute vorticity = sum_v A_v (zeta_v + f_v)
cudaError_t launch_diagnostics(const DevMesh &m, const double *h, const double *u, double *partials,
                               int nblocks, double *out2, cudaStream_t st);
constexpr int DIAG_BLOCKS = 608;   // 4 blocks per SM of a 152-SM GB300
// non-finite or non-positive thickness check; sets *flag to 1
cudaError_t launch_check(const double *h, int nC, const double *u, int nE, int *flag, cudaStream_t st);

}  // namespace fblts
