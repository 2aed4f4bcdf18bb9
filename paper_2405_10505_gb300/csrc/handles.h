// Host-side handle types shared by the C ABI translation units.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "fblts.h"
#include "kernels.cuh"

// returns from an extern "C" entry point with FBLTS_E_CUDA / FBLTS_E_OOM and
// a message naming the failed call
#define CK(call)                                                                            \
    do {                                                                                    \
        cudaError_t err__ = (call);                                                         \
        if (err__ != cudaSuccess) {                                                         \
            fblts::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(err__), __FILE__, \
                             __LINE__);                                                     \
            return err__ == cudaErrorMemoryAllocation ? FBLTS_E_OOM : FBLTS_E_CUDA;         \
        }                                                                                   \
    } while (0)

struct fblts_mesh {
    fblts::HostMesh hm;
    int device = 0;
    void *dbase = nullptr;
    fblts::DevMesh dm{};
    int *cell_n2o = nullptr, *cell_o2n = nullptr, *edge_n2o = nullptr, *edge_o2n = nullptr;
    // launch lists built for states on this mesh, by (dt, beta, precision, forcing, splitting, scheme)
    struct CachedSchedule {
        double dt;
        double beta[3];
        bool f32;
        int forcing;
        int split;
        int scheme;
        fblts::Schedule sched;
    };
    mutable std::mutex cache_mu;
    mutable std::vector<CachedSchedule> sched_cache;
    // states on this mesh plus server requests that name it and are not yet
    // taken: fblts_mesh_destroy refuses while any is left, since each of them
    // reads the mesh's device tables
    mutable std::atomic<int64_t> holds{0};
};

struct fblts_state {
    const fblts_mesh *mesh = nullptr;
    fblts_params p{};
    cudaStream_t st = nullptr;
    bool own_stream = false;
    void *dbase = nullptr;
    fblts::DevArrays arr{};
    fblts::DevMesh dm{};
    fblts::DevForcing fz{};
    long long *d_step = nullptr;
    int *d_flag = nullptr;
    double *d_partials = nullptr, *d_diag = nullptr;
    double *d_stage_c = nullptr, *d_stage_e = nullptr;
    fblts::Schedule sched;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int64_t steps = 0;
};

