// Allocation-free variant of the global diagnostics (total mass and total
// absolute vorticity) for callers that cannot allocate device memory.
//
// Its scratch (one pair of partial sums per block) lives in a file-scope
// static __device__ array, so the call itself never allocates.  Host code
// gets the device address of that array with cudaGetSymbolAddress, once per
// device, on the first call made with that device current.
#include <cuda_runtime.h>

#include <mutex>

#include "fblts.h"
#include "kernels.cuh"

namespace fblts {

// elements (cells, vertices) summed by one block of the static variant
constexpr int STATIC_CHUNK = 8192;
// capacity of the static scratch: this many blocks, two doubles each (64 KiB)
constexpr int STATIC_BLOCKS = 4096;
constexpr long long STATIC_MAX_ELEMENTS = (long long)STATIC_CHUNK * STATIC_BLOCKS;

namespace {

__device__ __align__(256) double g_static_partials[2 * STATIC_BLOCKS];

constexpr int TPB = 256;
constexpr int MAX_DEVICES = 64;

std::mutex g_mu;
double *g_scratch[MAX_DEVICES] = {nullptr};

__device__ double block_sum_static(double v, double *sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    return sh[0];
}

// block b sums cells and vertices [b*CHUNK, (b+1)*CHUNK) of arrays in the
// caller's order, reading the mesh tables through its permutations
__global__ void __launch_bounds__(TPB) static_partials(DevMesh m, const int *cell_n2o, const int *edge_n2o,
                                                        const double *h, const double *u, double *partials) {
    __shared__ double sh[TPB];
    const long long base = (long long)blockIdx.x * STATIC_CHUNK;
    double mass = 0.0, vort = 0.0;
    const int nV = m.nV;
    for (int k = threadIdx.x; k < STATIC_CHUNK; k += TPB) {
        const long long i = base + k;
        if (i < m.nC) mass += m.area[i] * h[cell_n2o[i]];
        if (i < nV) {
            double c = 0.0;
            for (int j = 0; j < 3; ++j) c += m.cVort[j * nV + i] * u[edge_n2o[m.eov[j * nV + i]]];
            vort += m.Av[i] * (c + m.fV[i]);
        }
    }
    const double bm = block_sum_static(mass, sh);
    __syncthreads();
    const double bv = block_sum_static(vort, sh);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = bm;
        partials[2 * blockIdx.x + 1] = bv;
    }
}

__global__ void __launch_bounds__(TPB) static_final(const double *partials, int nb, double *out2) {
    __shared__ double sh[TPB];
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < nb; k += TPB) {
        a += partials[2 * k];
        b += partials[2 * k + 1];
    }
    const double sa = block_sum_static(a, sh);
    __syncthreads();
    const double sb = block_sum_static(b, sh);
    if (threadIdx.x == 0) {
        out2[0] = sa;
        out2[1] = sb;
    }
}

}  // namespace

// device address of the static scratch on the current device (set up once per device)
static fblts_status static_scratch(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_error("diagnostics_static: no CUDA device (%s)", cudaGetErrorString(e));
        return FBLTS_E_CUDA;
    }
    if (dev < 0 || dev >= MAX_DEVICES) {
        set_error("diagnostics_static: device %d beyond the %d supported", dev, MAX_DEVICES);
        return FBLTS_E_ARG;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_partials);
        if (e != cudaSuccess || !p) {
            set_error("diagnostics_static: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return FBLTS_E_CUDA;
        }
        g_scratch[dev] = (double *)p;
    }
    *out = g_scratch[dev];
    return FBLTS_OK;
}

// exported by api.cu: the mesh's device tables
const DevMesh *mesh_dev(const fblts_mesh *m, const int **cell_n2o, const int **edge_n2o, int *device);

}  // namespace fblts

extern "C" fblts_status fblts_diagnostics_static(const fblts_mesh *mesh, const double *d_h, const double *d_u,
                                                 double *d_out, void *stream) {
    using namespace fblts;
    if (!mesh || !d_h || !d_u || !d_out) {
        set_error("diagnostics_static: NULL argument");
        return FBLTS_E_ARG;
    }
    const int *cn2o = nullptr, *en2o = nullptr;
    int mdev = 0;
    const DevMesh *dm = mesh_dev(mesh, &cn2o, &en2o, &mdev);
    long long n = dm->nC > dm->nV ? dm->nC : dm->nV;
    if (n > STATIC_MAX_ELEMENTS) {
        set_error("diagnostics_static: mesh has %lld cells/vertices, the static scratch holds at most %lld",
                  n, STATIC_MAX_ELEMENTS);
        return FBLTS_E_ARG;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != mdev) {
        set_error("diagnostics_static: the current device is not the mesh's device");
        return FBLTS_E_ARG;
    }
    double *scratch = nullptr;
    fblts_status st = static_scratch(&scratch);
    if (st != FBLTS_OK) return st;
    const int nb = (int)((n + STATIC_CHUNK - 1) / STATIC_CHUNK);
    cudaStream_t s = (cudaStream_t)stream;
    static_partials<<<nb, TPB, 0, s>>>(*dm, cn2o, en2o, d_h, d_u, scratch);
    static_final<<<1, TPB, 0, s>>>(scratch, nb, d_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("diagnostics_static: launch failed: %s", cudaGetErrorString(e));
        return FBLTS_E_CUDA;
    }
    return FBLTS_OK;
}
