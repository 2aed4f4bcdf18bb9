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
    const float2 *woeDF;                // FP64 path: W as a double-float pair (hi, lo), slot-major
    const unsigned char *ebnd;
    const double *cosE, *sinE, *xE, *yE, *xC, *yC;
    const int *eov, *cov;               // vertices
    const double *cVort, *cKite, *fV, *Av;
    // single-precision copies of the coefficients (FP32-tendency path)
    const float *woe32, *invDc32;
    // neighbour edges from the cells' edge rows: slots and weights in row order (FP32 path)
    const int *eocS;                    // edge rows with the sign n_{e,i} (~e for the second cell)
    const float *dv32, *ke32;           // l_e and d_e l_e / 4 per edge
    const float2 *el2;                  // per edge {l_e, H_e} (H_e per state)
    // FP32 vertex pass, one record per vertex: {eov x3, cov[0]}, {cov[1], cov[2]},
    // {t_{e,v} d_e / A_v x3, f_v}, and per state {kite / A_v x3, H_v}
    const int4 *vI4;
    const int2 *vI2;
    const float4 *vCf;
    const float4 *vKh;
    const double *invA;                 // 1 / A_i
    const float *invA32;                // 1 / A_i rounded to float (FP32 stage values and K)
    // neighbour edges from the cells' edge rows (FP32 edge pass): rowS = 8 or
    // 12 when valid, else 0 (explicit lists eoe / woe32, woe32 = W / l_{e'})
    int rowS;
    const unsigned short *eslot;        // slot in the row of c0 | of c1 << 4 | row lengths << 8, << 12
    const int *rowE;                    // [nC * rowS] signed edge rows, padded
    const float *rowP;                  // [nC * rowS] prefix sums of the kite fractions
    const int *rowN, *rowV;             // [nC * rowS] neighbour cell / counter-clockwise vertex per slot
    // resting depth H = -b as seen by the FP32 path: per cell, edge mean, vertex mean (per state)
    const float *He32;
    // FP64 path (per state): H_e = -(b_c0 + b_c1) / 2 per edge and
    // H_v = sum_j kite_j H_j / A_v per vertex, the resting thickness that the
    // flux and the vertex thickness add to the surface elevation xi
    const double *He64, *Hv64;
};

struct DevForcing {
    int flags;                 // FBLTS_FORCE_* bits
    int fp32;                  // write the single-precision fields instead
    double *windN, *windT, *cw, *ps;
    // FP32: per edge {wind normal, wind tangential, C_W, H_e}, one 16-byte record;
    // ps32 = p_s - (pc + dp), the ambient-relative pressure
    float4 *wrec32;
    float *ps32;
    double wind_u, wind_v, cd, rho0, rho_air;
    float cd32;                // cd rounded to float (FP32 edge pass)
    double inv_rho0;           // 1 / rho0 (the per-edge pressure force multiplies by it)
    double vx[9];
    double t0, dt;
    const long long *step;     // device step counter
};

// State arrays by schedule id.  Every thickness array, the double time level
// A_H included, holds the surface elevation xi = h + b = h - H (the
// deviation from the resting depth), so the state rounds at the precision of
// the displacement, not of the depth.  FP64 path: every array is double (a[]).
// FP32-tendency path: the time level A_H / A_U, the correction sums A_ACCH /
// A_ACCU and the saved time level A_SH0 / A_SU0 stay double (a[]); the stage
// arrays, K, q, F, q_e and the saved IF-1 stage data are float (f[]), with
// every thickness stored as xi = h - H (deviation from the resting depth);
// xi32 / u32 are float shadows of the double time level.
struct DevArrays {
    double *a[A_COUNT];
    float *f[A_COUNT];
    float *xi32, *u32;
    float *bx32;      // FP32 with cell rows: per cell {B, xi*} of the TRiSK pass (in the A_FQU area)
    int fp32;
};

struct SegSet {
    int nseg;
    Seg seg[MAX_SEG];
};

// launches one schedule op on the stream
cudaError_t launch_op(const Op &op, const DevMesh &m, const DevArrays &arr, const DevForcing &fz,
                      double g, long long *step_counter, cudaStream_t st);

// FP32-tendency path: resting depths seen by the float kernels, and the
// float shadows of the double time level (after any write of h, u)
cudaError_t launch_fp32_depths(const DevMesh &m, float *He32, float2 *el2,
                               float4 *vkh, cudaStream_t st);
cudaError_t launch_fp32_shadows(const DevMesh &m, const DevArrays &arr, cudaStream_t st);

// caller-order <-> band-order copies: dst[i] = src[idx[i]] + sign * b[k],
// k = i (sign +1: h in caller order to xi in band order) or idx[i] (sign -1:
// xi to h in caller order); b = NULL copies only
cudaError_t launch_gather(double *dst, const double *src, const int *idx, int n, cudaStream_t st,
                          const double *b = nullptr, int sign = 0);
// FP64 path: the resting thickness per edge and vertex (He64, Hv64) from the bottom
cudaError_t launch_fp64_depths(const DevMesh &m, double *He64, double *Hv64, cudaStream_t st);
cudaError_t launch_zero_boundary(double *u, const unsigned char *ebnd, int nE, cudaStream_t st);

// deterministic reductions: mass = sum A_i h_i (h = xi - b), absolute
// vorticity = sum_v A_v (zeta_v + f_v)
cudaError_t launch_diagnostics(const DevMesh &m, const double *xi, const double *u, double *partials,
                               int nblocks, double *out2, cudaStream_t st);
constexpr int DIAG_BLOCKS = 608;   // 4 blocks per SM of a 152-SM GB300
// non-finite state or non-positive thickness h = xi - b check; sets *flag to 1
cudaError_t launch_check(const double *xi, const double *b, int nC, const double *u, int nE, int *flag,
                         cudaStream_t st);

}  // namespace fblts
