// sm_103a kernels of the FB-LTS hot path.
//
// One thread per cell / vertex / edge of a contiguous band range; the mode of
// each index (stage update, in-place update, correction sum, kinetic energy
// only) comes from the launch's segment list.  The passes use no atomics, so
// every result is bit-reproducible run to run.
#include <utility>

#include "kernel_bodies32.cuh"

namespace fblts {

namespace {

constexpr int TPB = 256;

// Programmatic dependent launch: a kernel of the schedule may be scheduled
// while its predecessor drains; it waits here, before touching memory, until
// the predecessor's results are visible.
__device__ __forceinline__ void wait_predecessor() {
#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 900)
    cudaGridDependencySynchronize();
#endif
}

__global__ void __launch_bounds__(TPB) cell_pass(DevMesh m, CellArgs a) {
    wait_predecessor();
    const int i = a.lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (i < a.hi) cell_body(m, a, i);
}

__global__ void __launch_bounds__(TPB) vert_pass(DevMesh m, VertArgs a) {
    wait_predecessor();
    const int v = a.lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (v < a.hi) vert_body(m, a, v);
}

__global__ void __launch_bounds__(TPB) eprep_pass(DevMesh m, PrepArgs a) {
    wait_predecessor();
    const int e = a.lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (e < a.hi) prep_body(m, a, e);
}

template <bool FORCING>
__global__ void __launch_bounds__(TPB) edge_pass(DevMesh m, EdgeArgs a, DevForcing fz) {
    wait_predecessor();
    const int e = a.lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (e < a.hi) edge_body<FORCING>(m, a, fz, e);
}

__global__ void __launch_bounds__(TPB) save_pass(IfArgs a) {
    wait_predecessor();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < a.n) save_body(a, t);
}

__global__ void __launch_bounds__(TPB) pred_pass(IfArgs a) {
    wait_predecessor();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < a.n) pred_body(a, t);
}

__global__ void __launch_bounds__(TPB) final_pass(IfArgs a, const unsigned char *ebnd) {
    wait_predecessor();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < a.n) final_body(a, ebnd, t);
}

__global__ void __launch_bounds__(TPB) forcing_pass(DevMesh m, DevForcing fz) {
    wait_predecessor();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const double time = fz.t0 + (double)(*fz.step) * fz.dt;
    forcing_body(m, fz, time, t);
}

template <int NMAX, bool ROWS>
__global__ void __launch_bounds__(TPB) cell32_pass(DevMesh m, CellArgs32 a) {
    wait_predecessor();
    const int i = a.lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (i < a.hi) cell32_body<NMAX, ROWS>(m, a, i);
}

__global__ void __launch_bounds__(TPB) vert32_pass(DevMesh m, VertArgs32 a) {
    wait_predecessor();
    const int v = a.lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (v < a.hi) vert32_body(m, a, v);
}

__global__ void __launch_bounds__(TPB) eprep32_pass(DevMesh m, PrepArgs32 a) {
    wait_predecessor();
    const int e = a.lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (e < a.hi) prep32_body(m, a, e);
}

template <bool SHARES, bool FORCING>
__global__ void __launch_bounds__(TPB) edge32_pass(DevMesh m, EdgeArgs32 a, DevForcing fz) {
    wait_predecessor();
    const int e = a.lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (e < a.hi) edge32_body<SHARES, FORCING>(m, a, fz, e);
}

template <int S, bool VORTEX>
__global__ void __launch_bounds__(TPB) trisk32_pass(DevMesh m, TriskArgs32 a, DevForcing fz) {
    wait_predecessor();
    const int i = a.lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (i < a.hi) trisk32_body<S, VORTEX>(m, a, fz, i);
}


__global__ void __launch_bounds__(TPB) save32_pass(IfArgs32 a) {
    wait_predecessor();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < a.n) save32_body(a, t);
}

__global__ void __launch_bounds__(TPB) pred32_pass(IfArgs32 a) {
    wait_predecessor();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < a.n) pred32_body(a, t);
}

__global__ void __launch_bounds__(TPB) final32_pass(IfArgs32 a, const unsigned char *ebnd) {
    wait_predecessor();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < a.n) final32_body(a, ebnd, t);
}

__global__ void __launch_bounds__(TPB) forcing32_pass(DevMesh m, DevForcing fz) {
    wait_predecessor();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const double time = fz.t0 + (double)(*fz.step) * fz.dt;
    forcing32_body(m, fz, time, t);
}

// resting depth seen by the FP32 path: H_e, the mean over the two cells of an
// edge (also in the per-edge record {l_e, H_e}), and the per-vertex record
// {kite / A_v x3, H_v} with the kite-weighted mean H_v
__global__ void fp32_depths(DevMesh m, float *He32, float2 *el2, float4 *vkh) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < m.nE) {
        const float He = (float)(-0.5 * (m.bottom[m.coe0[t]] + m.bottom[m.coe1[t]]));
        He32[t] = He;
        el2[t] = make_float2(m.dv32[t], He);
    }
    if (t < m.nV) {
        double s = 0.0;
        for (int j = 0; j < 3; ++j) s += m.cKite[j * m.nV + t] * (-m.bottom[m.cov[j * m.nV + t]]);
        vkh[t] = make_float4((float)m.cKite[t], (float)m.cKite[m.nV + t], (float)m.cKite[2 * m.nV + t], (float)s);
    }
}

__global__ void fp32_shadows(const double *xi_state, const double *u, float *xi, float *u32, int nC, int nE) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nC) xi[t] = (float)xi_state[t];
    if (t < nE) u32[t] = (float)u[t];
}

// FP64 path: resting thickness H_e per edge (mean of the two cells; a no-flow
// edge's absent cell is its present one) and H_v per vertex (kite-weighted)
__global__ void fp64_depths(DevMesh m, double *He64, double *Hv64) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < m.nE) He64[t] = -0.5 * (m.bottom[m.coe0[t]] + m.bottom[m.coe1[t]]);
    if (t < m.nV) {
        double s = 0.0;
        for (int j = 0; j < 3; ++j) s += m.cKite[j * m.nV + t] * (-m.bottom[m.cov[j * m.nV + t]]);
        Hv64[t] = s;
    }
}

__global__ void step_end(long long *step) {
    wait_predecessor();
    *step += 1;
}

__global__ void gather_kernel(double *dst, const double *src, const int *idx, int n, const double *b, int sign) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int k = idx[i];
    double v = src[k];
    if (b) v = sign > 0 ? v + b[i] : v - b[k];
    dst[i] = v;
}

__global__ void zero_bnd_kernel(double *u, const unsigned char *ebnd, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && ebnd[i]) u[i] = 0.0;
}

__device__ double block_sum(double v, double *sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    return sh[0];
}

// Fixed-order partial sums (deterministic): thread t of the grid sums
// elements t, t + G, t + 2G, ...; each block reduces with a fixed tree.
__global__ void __launch_bounds__(TPB) diag_partials(DevMesh m, const double *xi, const double *u,
                                                      double *partials) {
    __shared__ double sh[TPB];
    const int G = gridDim.x * blockDim.x;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    double mass = 0.0, vort = 0.0;
    for (int i = t; i < m.nC; i += G) mass += m.area[i] * (xi[i] - m.bottom[i]);
    const int nV = m.nV;
    for (int v = t; v < nV; v += G) {
        double c = 0.0;
#pragma unroll
        for (int j = 0; j < 3; ++j) c += m.cVort[j * nV + v] * u[m.eov[j * nV + v]];
        vort += m.Av[v] * (c + m.fV[v]);
    }
    const double bm = block_sum(mass, sh);
    __syncthreads();
    const double bv = block_sum(vort, sh);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = bm;
        partials[2 * blockIdx.x + 1] = bv;
    }
}

__global__ void __launch_bounds__(TPB) diag_final(const double *partials, int nb, double *out2) {
    __shared__ double sh[TPB];
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        a += partials[2 * k];
        b += partials[2 * k + 1];
    }
    const double sa = block_sum(a, sh);
    __syncthreads();
    const double sb = block_sum(b, sh);
    if (threadIdx.x == 0) {
        out2[0] = sa;
        out2[1] = sb;
    }
}

__global__ void check_kernel(const double *xi, const double *b, int nC, const double *u, int nE, int *flag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool bad = false;
    if (i < nC) bad |= !(xi[i] - b[i] > 0.0) || !isfinite(xi[i]);
    if (i < nE) bad |= !isfinite(u[i]);
    if (bad) atomicOr(flag, 1);
}

inline int nblk(long long n) { return (int)((n + TPB - 1) / TPB); }

// launch with the programmatic-stream-serialisation attribute (see wait_predecessor)
template <typename... KArgs, typename... Args>
cudaError_t pdl(void (*kernel)(KArgs...), int grid, int block, cudaStream_t st, Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace

#define CK_L(x)                                  \
    do {                                         \
        cudaError_t e__ = (x);                   \
        if (e__ != cudaSuccess) return e__;      \
    } while (0)

static cudaError_t launch_op32(const Op &op, const DevMesh &m, const DevArrays &arr, const DevForcing &fz,
                               double g, long long *step_counter, cudaStream_t st) {
    switch (op.kind) {
        case OP_CELL: {
            if (op.hi <= op.lo) return cudaSuccess;
            const CellArgs32 a = cell_args32(op, arr, m);
            const int nb = nblk(op.hi - op.lo);
            if (m.rowS == 8) CK_L(pdl(cell32_pass<8, true>, nb, TPB, st, m, a));
            else if (m.rowS == 12) CK_L(pdl(cell32_pass<12, true>, nb, TPB, st, m, a));
            else if (m.maxE <= 6) CK_L(pdl(cell32_pass<6, false>, nb, TPB, st, m, a));
            else if (m.maxE <= 8) CK_L(pdl(cell32_pass<8, false>, nb, TPB, st, m, a));
            else CK_L(pdl(cell32_pass<12, false>, nb, TPB, st, m, a));
        } break;
        case OP_VERT:
            if (op.hi <= op.lo) return cudaSuccess;
            CK_L(pdl(vert32_pass, nblk(op.hi - op.lo), TPB, st, m, vert_args32(op, arr)));
            break;
        case OP_EPREP:
            if (op.hi <= op.lo) return cudaSuccess;
            CK_L(pdl(eprep32_pass, nblk(op.hi - op.lo), TPB, st, m, prep_args32(op, arr)));
            break;
        case OP_EDGE: {
            if (op.hi <= op.lo) return cudaSuccess;
            const EdgeArgs32 a = edge_args32(op, arr, g);
            const int nb = nblk(op.hi - op.lo);
            if (m.rowS) {
                if (fz.flags) CK_L(pdl(edge32_pass<true, true>, nb, TPB, st, m, a, fz));
                else CK_L(pdl(edge32_pass<true, false>, nb, TPB, st, m, a, fz));
            } else {
                if (fz.flags) CK_L(pdl(edge32_pass<false, true>, nb, TPB, st, m, a, fz));
                else CK_L(pdl(edge32_pass<false, false>, nb, TPB, st, m, a, fz));
            }
        } break;
        case OP_TRISK: {
            if (op.hi <= op.lo) return cudaSuccess;
            const TriskArgs32 a = trisk_args32(op, arr, g, fz.rho0);
            const int nb = nblk(op.hi - op.lo);
            const bool vx = (fz.flags & FBLTS_FORCE_VORTEX) != 0;
            if (m.rowS == 8) {
                if (vx) CK_L(pdl(trisk32_pass<8, true>, nb, TPB, st, m, a, fz));
                else CK_L(pdl(trisk32_pass<8, false>, nb, TPB, st, m, a, fz));
            } else if (m.rowS == 12) {
                if (vx) CK_L(pdl(trisk32_pass<12, true>, nb, TPB, st, m, a, fz));
                else CK_L(pdl(trisk32_pass<12, false>, nb, TPB, st, m, a, fz));
            } else {
                return cudaErrorInvalidValue;   // the schedule emits OP_TRISK only with cell rows
            }
        } break;
        case OP_SAVE:
        case OP_PRED:
        case OP_FINAL: {
            IfArgs32 a = if_args32(op, arr, m);
            if (a.n <= 0) return cudaSuccess;
            if (op.kind == OP_SAVE) CK_L(pdl(save32_pass, nblk(a.n), TPB, st, a));
            else if (op.kind == OP_PRED) CK_L(pdl(pred32_pass, nblk(a.n), TPB, st, a));
            else CK_L(pdl(final32_pass, nblk(a.n), TPB, st, a, m.ebnd));
        } break;
        case OP_FORCING:
            if (!fz.flags) return cudaSuccess;
            CK_L(pdl(forcing32_pass, nblk(m.nE > m.nC ? m.nE : m.nC), TPB, st, m, fz));
            break;
        case OP_STEP_END: step_end<<<1, 1, 0, st>>>(step_counter); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_fp32_depths(const DevMesh &m, float *He32, float2 *el2,
                               float4 *vkh, cudaStream_t st) {
    const int n = m.nE > m.nV ? (m.nE > m.nC ? m.nE : m.nC) : (m.nV > m.nC ? m.nV : m.nC);
    fp32_depths<<<nblk(n), TPB, 0, st>>>(m, He32, el2, vkh);
    return cudaGetLastError();
}

cudaError_t launch_fp32_shadows(const DevMesh &m, const DevArrays &arr, cudaStream_t st) {
    fp32_shadows<<<nblk(m.nE > m.nC ? m.nE : m.nC), TPB, 0, st>>>(arr.a[A_H], arr.a[A_U], arr.xi32, arr.u32,
                                                                   m.nC, m.nE);
    return cudaGetLastError();
}

cudaError_t launch_fp64_depths(const DevMesh &m, double *He64, double *Hv64, cudaStream_t st) {
    fp64_depths<<<nblk(m.nE > m.nV ? m.nE : m.nV), TPB, 0, st>>>(m, He64, Hv64);
    return cudaGetLastError();
}

cudaError_t launch_op(const Op &op, const DevMesh &m, const DevArrays &arr, const DevForcing &fz, double g,
                      long long *step_counter, cudaStream_t st) {
    if (arr.fp32) return launch_op32(op, m, arr, fz, g, step_counter, st);
    switch (op.kind) {
        case OP_CELL:
            if (op.hi <= op.lo) return cudaSuccess;
            CK_L(pdl(cell_pass, nblk(op.hi - op.lo), TPB, st, m, cell_args(op, arr)));
            break;
        case OP_VERT:
            if (op.hi <= op.lo) return cudaSuccess;
            CK_L(pdl(vert_pass, nblk(op.hi - op.lo), TPB, st, m, vert_args(op, arr)));
            break;
        case OP_EPREP:
            if (op.hi <= op.lo) return cudaSuccess;
            CK_L(pdl(eprep_pass, nblk(op.hi - op.lo), TPB, st, m, prep_args(op, arr)));
            break;
        case OP_EDGE:
            if (op.hi <= op.lo) return cudaSuccess;
            if (fz.flags) CK_L(pdl(edge_pass<true>, nblk(op.hi - op.lo), TPB, st, m, edge_args(op, arr, g), fz));
            else CK_L(pdl(edge_pass<false>, nblk(op.hi - op.lo), TPB, st, m, edge_args(op, arr, g), fz));
            break;
        case OP_SAVE:
        case OP_PRED:
        case OP_FINAL: {
            IfArgs a = if_args(op, arr);
            if (a.n <= 0) return cudaSuccess;
            if (op.kind == OP_SAVE) CK_L(pdl(save_pass, nblk(a.n), TPB, st, a));
            else if (op.kind == OP_PRED) CK_L(pdl(pred_pass, nblk(a.n), TPB, st, a));
            else CK_L(pdl(final_pass, nblk(a.n), TPB, st, a, m.ebnd));
        } break;
        case OP_FORCING:
            if (!fz.flags) return cudaSuccess;
            CK_L(pdl(forcing_pass, nblk(m.nE > m.nC ? m.nE : m.nC), TPB, st, m, fz));
            break;
        case OP_STEP_END: step_end<<<1, 1, 0, st>>>(step_counter); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_gather(double *dst, const double *src, const int *idx, int n, cudaStream_t st, const double *b,
                          int sign) {
    if (n <= 0) return cudaSuccess;
    gather_kernel<<<nblk(n), TPB, 0, st>>>(dst, src, idx, n, b, sign);
    return cudaGetLastError();
}

cudaError_t launch_zero_boundary(double *u, const unsigned char *ebnd, int nE, cudaStream_t st) {
    zero_bnd_kernel<<<nblk(nE), TPB, 0, st>>>(u, ebnd, nE);
    return cudaGetLastError();
}

cudaError_t launch_diagnostics(const DevMesh &m, const double *xi, const double *u, double *partials, int nblocks,
                               double *out2, cudaStream_t st) {
    diag_partials<<<nblocks, TPB, 0, st>>>(m, xi, u, partials);
    diag_final<<<1, TPB, 0, st>>>(partials, nblocks, out2);
    return cudaGetLastError();
}

cudaError_t launch_check(const double *xi, const double *b, int nC, const double *u, int nE, int *flag,
                         cudaStream_t st) {
    check_kernel<<<nblk(nE > nC ? nE : nC), TPB, 0, st>>>(xi, b, nC, u, nE, flag);
    return cudaGetLastError();
}

}  // namespace fblts
