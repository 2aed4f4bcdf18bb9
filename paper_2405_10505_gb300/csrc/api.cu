// C ABI of the FB-LTS library (include/fblts.h): handles, device arenas,
// the captured coarse step, caller-order I/O, diagnostics and checkpoints.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "handles.h"
#include "kernels.cuh"

namespace fblts {

namespace {
thread_local char g_err[1024] = "no error";
}

const char *last_error_text() { return g_err; }

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

bool arr_is_cell(int a) {
    switch (a) {
        case A_H: case A_HS1: case A_HS2: case A_HS3: case A_HST1: case A_HST2: case A_HST3:
        case A_K: case A_ACCH: case A_SH0: case A_SH1: case A_SH2: case A_SH3: return true;
        default: return false;
    }
}
bool arr_is_vert(int a) { return a == A_Q; }

namespace {

// Bump allocator over one device allocation.
struct Arena {
    char *base = nullptr;
    size_t size = 0, used = 0;
    size_t reserve(size_t bytes) {  // sizing pass
        used = ((used + 255) & ~size_t(255)) + bytes;
        return used;
    }
    void *take(size_t bytes) {
        size_t off = (used + 255) & ~size_t(255);
        if (off + bytes > size) return nullptr;
        used = off + bytes;
        return base + off;
    }
};

// slot-major copy of a row-major [n][k] table
template <class T>
std::vector<T> slot_major(const std::vector<T> &v, int n, int k) {
    std::vector<T> out((size_t)n * k);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < k; ++j) out[(size_t)j * n + i] = v[(size_t)i * k + j];
    return out;
}

}  // namespace
}  // namespace fblts

using namespace fblts;

extern "C" const char *fblts_last_error(void) { return last_error_text(); }

namespace fblts {
// the mesh's device tables and permutations (used by the allocation-free diagnostics)
const DevMesh *mesh_dev(const fblts_mesh *m, const int **cell_n2o, const int **edge_n2o, int *device) {
    *cell_n2o = m->cell_n2o;
    *edge_n2o = m->edge_n2o;
    *device = m->device;
    return &m->dm;
}
}  // namespace fblts

// ------------------------------------------------------------------ mesh

extern "C" fblts_status fblts_mesh_create(const fblts_mesh_desc *desc, fblts_mesh **out) {
    if (!out) { set_error("mesh_create: out is NULL"); return FBLTS_E_ARG; }
    *out = nullptr;
    fblts_mesh *m = new (std::nothrow) fblts_mesh();
    if (!m) { set_error("mesh_create: host allocation failed"); return FBLTS_E_OOM; }
    fblts_status s = build_host_mesh(desc, m->hm);
    if (s != FBLTS_OK) { delete m; return s; }
    const HostMesh &hm = m->hm;
    const int nC = hm.nC, nE = hm.nE, nV = hm.nV, mE = hm.maxE, mE2 = hm.maxE2;
    if (cudaGetDevice(&m->device) != cudaSuccess) {
        set_error("mesh_create: no CUDA device (%s)", cudaGetErrorString(cudaGetLastError()));
        delete m;
        return FBLTS_E_CUDA;
    }
    // host staging of every device array, then one allocation and one copy
    struct Item { const void *src; size_t bytes; void **dst; };
    std::vector<Item> items;
    std::vector<std::vector<int>> ikeep;
    std::vector<std::vector<double>> dkeep;
    std::vector<std::vector<unsigned char>> bkeep;
    std::vector<std::vector<float>> fkeep;
    DevMesh &dm = m->dm;
    dm.nC = nC; dm.nE = nE; dm.nV = nV; dm.maxE = mE; dm.maxE2 = mE2;
    auto addi = [&](std::vector<int> v, const int **dst) {
        ikeep.push_back(std::move(v));
        items.push_back({ikeep.back().data(), ikeep.back().size() * sizeof(int), (void **)dst});
    };
    auto addd = [&](std::vector<double> v, const double **dst) {
        dkeep.push_back(std::move(v));
        items.push_back({dkeep.back().data(), dkeep.back().size() * sizeof(double), (void **)dst});
    };
    auto addf = [&](const std::vector<double> &v, const float **dst) {
        fkeep.emplace_back(v.begin(), v.end());
        items.push_back({fkeep.back().data(), fkeep.back().size() * sizeof(float), (void **)dst});
    };
    ikeep.reserve(32); dkeep.reserve(32); bkeep.reserve(4); fkeep.reserve(16);
    addi(hm.nEoC, &dm.nEoC);
    addi(slot_major(hm.eoc, nC, mE), &dm.eoc);
    addi(slot_major(hm.coc, nC, mE), &dm.coc);
    addd(slot_major(hm.cDiv, nC, mE), &dm.cDiv);
    addd(slot_major(hm.cKE, nC, mE), &dm.cKE);
    addd(hm.area, &dm.area);
    std::vector<int> c0(nE), c1(nE), v0(nE), v1(nE);
    for (int e = 0; e < nE; ++e) { c0[e] = hm.coe[2 * e]; c1[e] = hm.coe[2 * e + 1]; v0[e] = hm.voe[2 * e]; v1[e] = hm.voe[2 * e + 1]; }
    addi(c0, &dm.coe0); addi(c1, &dm.coe1); addi(v0, &dm.voe0); addi(v1, &dm.voe1);
    addi(hm.nEoE, &dm.nEoE);
    addi(slot_major(hm.eoe, nE, mE2), &dm.eoe);
    addd(slot_major(hm.woe, nE, mE2), &dm.woe);
    {   // the FP64 path's TRiSK weights as double-float pairs: hi = nearest float, lo = the rest
        std::vector<float> wdf((size_t)2 * nE * mE2);
        const std::vector<double> w = slot_major(hm.woe, nE, mE2);
        for (size_t k = 0; k < w.size(); ++k) {
            const float hi = (float)w[k];
            wdf[2 * k] = hi;
            wdf[2 * k + 1] = (float)(w[k] - (double)hi);
        }
        fkeep.emplace_back(std::move(wdf));
        items.push_back({fkeep.back().data(), fkeep.back().size() * sizeof(float), (void **)&dm.woeDF});
    }
    addd(hm.invDc, &dm.invDc);
    bkeep.push_back(hm.ebnd);
    items.push_back({bkeep.back().data(), bkeep.back().size(), (void **)&dm.ebnd});
    addd(hm.cosE, &dm.cosE); addd(hm.sinE, &dm.sinE); addd(hm.xE, &dm.xE); addd(hm.yE, &dm.yE);
    addd(hm.xC, &dm.xC); addd(hm.yC, &dm.yC);
    addi(slot_major(hm.eov, nV, 3), &dm.eov);
    addi(slot_major(hm.cov, nV, 3), &dm.cov);
    addd(slot_major(hm.cVort, nV, 3), &dm.cVort);
    addd(slot_major(hm.cKite, nV, 3), &dm.cKite);
    addd(hm.fV, &dm.fV);
    addd(hm.Av, &dm.Av);
    {   // FP32 list weights W_{e,e'} / l_{e'}: the edge records carry l_{e'}
        std::vector<double> w(hm.woe);
        for (int e = 0; e < nE; ++e)
            for (int j = 0; j < mE2; ++j) {
                const double l = hm.dvE[hm.eoe[(size_t)e * mE2 + j]];
                w[(size_t)e * mE2 + j] = l != 0.0 ? w[(size_t)e * mE2 + j] / l : 0.0;
            }
        addf(slot_major(w, nE, mE2), &dm.woe32);
    }
    addf(hm.invDc, &dm.invDc32);
    {   // FP32 vertex pass: {e0, e1, e2, c0}, {c1, c2}, {t d / A_v x3, f} per vertex
        std::vector<int> i4((size_t)nV * 4), i2((size_t)nV * 2);
        std::vector<double> f4((size_t)nV * 4);
        for (int v = 0; v < nV; ++v) {
            for (int j = 0; j < 3; ++j) {
                i4[4 * (size_t)v + j] = hm.eov[3 * (size_t)v + j];
                f4[4 * (size_t)v + j] = hm.cVort[3 * (size_t)v + j];
            }
            i4[4 * (size_t)v + 3] = hm.cov[3 * (size_t)v];
            i2[2 * (size_t)v] = hm.cov[3 * (size_t)v + 1];
            i2[2 * (size_t)v + 1] = hm.cov[3 * (size_t)v + 2];
            f4[4 * (size_t)v + 3] = hm.fV[v];
        }
        addi(i4, (const int **)&dm.vI4);
        addi(i2, (const int **)&dm.vI2);
        addf(f4, (const float **)&dm.vCf);
    }
    addi(slot_major(hm.eocS, nC, mE), &dm.eocS);
    addf(hm.dvE, &dm.dv32);
    addf(hm.keE, &dm.ke32);
    addd(hm.invA, &dm.invA);
    addf(hm.invA, &dm.invA32);
    dm.rowS = hm.rows_canonical ? hm.rowS : 0;
    if (dm.rowS) {
        addi(hm.rowE, &dm.rowE);
        addf(hm.rowP, &dm.rowP);
        addi(hm.rowN, &dm.rowN);
        addi(hm.rowV, &dm.rowV);
        std::vector<unsigned char> sl(hm.eslot.size() * 2);
        std::memcpy(sl.data(), hm.eslot.data(), sl.size());
        bkeep.push_back(std::move(sl));
        items.push_back({bkeep.back().data(), bkeep.back().size(), (void **)&dm.eslot});
    }
    addi(hm.cell_n2o, (const int **)&m->cell_n2o);
    addi(hm.cell_o2n, (const int **)&m->cell_o2n);
    addi(hm.edge_n2o, (const int **)&m->edge_n2o);
    addi(hm.edge_o2n, (const int **)&m->edge_o2n);
    Arena ar;
    for (auto &it : items) ar.reserve(it.bytes);
    ar.size = ar.used + 256;
    if (cudaMalloc(&m->dbase, ar.size) != cudaSuccess) {
        cudaGetLastError();
        set_error("mesh_create: cudaMalloc of %zu bytes failed", ar.size);
        delete m;
        return FBLTS_E_OOM;
    }
    ar.base = (char *)m->dbase;
    ar.used = 0;
    std::vector<char> host(ar.size, 0);
    for (auto &it : items) {
        char *d = (char *)ar.take(it.bytes);
        if (!d) {
            set_error("mesh_create: arena layout error");
            cudaFree(m->dbase);
            delete m;
            return FBLTS_E_OOM;
        }
        std::memcpy(host.data() + (d - ar.base), it.src, it.bytes);
        *it.dst = d;
    }
    if (cudaMemcpy(m->dbase, host.data(), ar.size, cudaMemcpyHostToDevice) != cudaSuccess) {
        set_error("mesh_create: upload failed: %s", cudaGetErrorString(cudaGetLastError()));
        cudaFree(m->dbase);
        delete m;
        return FBLTS_E_CUDA;
    }
    dm.bottom = nullptr;
    *out = m;
    return FBLTS_OK;
}

extern "C" fblts_status fblts_mesh_destroy(fblts_mesh *m) {
    if (!m) return FBLTS_OK;
    const int64_t holds = m->holds.load();
    if (holds > 0) {
        set_error("mesh_destroy: %lld states or server requests still use this mesh", (long long)holds);
        return FBLTS_E_STATE;
    }
    if (m->dbase) cudaFree(m->dbase);
    delete m;
    return FBLTS_OK;
}

extern "C" fblts_status fblts_mesh_regions(const fblts_mesh_desc *desc, int32_t pair, int32_t *cell_class,
                                          int32_t *cell_band, int32_t *edge_class, int32_t *edge_band) {
    if (!desc) { set_error("mesh_regions: desc is NULL"); return FBLTS_E_ARG; }
    HostMesh hm;
    const fblts_status st = build_host_mesh(desc, hm);
    if (st != FBLTS_OK) return st;
    if (pair < 0 || pair > hm.L - 2) {
        set_error("mesh_regions: pair %d outside [0, %d]", pair, hm.L - 2);
        return FBLTS_E_ARG;
    }
    // the band key of an element relative to the pair (pair, pair + 1)
    auto classify = [&](uint32_t key, int32_t &cls, int32_t &band) {
        const int level = hm.L - 1 - (int)(key >> 16);
        const int kin = (int)((key >> 8) & 0xff), kout = (int)(key & 0xff);
        band = 0;
        if (level > pair + 1) {
            cls = FBLTS_REGION_FINE;
            band = 6;
        } else if (level == pair + 1) {
            cls = FBLTS_REGION_FINE;
            band = 6 - kout;
        } else if (level == pair) {
            cls = kin <= hm.nIF1 ? FBLTS_REGION_IF1
                                 : (kin <= hm.nIF1 + hm.nIF2 ? FBLTS_REGION_IF2 : FBLTS_REGION_INTERIOR);
        } else {
            cls = FBLTS_REGION_OUTSIDE;
        }
    };
    for (int i = 0; i < hm.nC; ++i) {
        int32_t c, b;
        classify(hm.ckey[i], c, b);
        if (cell_class) cell_class[hm.cell_n2o[i]] = c;
        if (cell_band) cell_band[hm.cell_n2o[i]] = b;
    }
    for (int e = 0; e < hm.nE; ++e) {
        int32_t c, b;
        classify(hm.ekey[e], c, b);
        if (edge_class) edge_class[hm.edge_n2o[e]] = c;
        if (edge_band) edge_band[hm.edge_n2o[e]] = b;
    }
    return FBLTS_OK;
}

// The host mesh and the launch list of one coarse step for a description and
// parameters, with the argument checks of fblts_mesh_create / fblts_state_init.
static fblts_status plan(const fblts_mesh_desc *desc, const fblts_params *p, const char *who, HostMesh &hm,
                         Schedule &s) {
    if (!desc || !p) { set_error("%s: NULL argument", who); return FBLTS_E_ARG; }
    if (p->precision != FBLTS_FP64 && p->precision != FBLTS_FP32_TENDENCY) {
        set_error("%s: unknown precision %d", who, p->precision);
        return FBLTS_E_ARG;
    }
    if (p->split < 0 || p->split > 2) { set_error("%s: split must be 0, 1 or 2", who); return FBLTS_E_ARG; }
    if (p->scheme != FBLTS_SCHEME_FBLTS && p->scheme != FBLTS_SCHEME_RK4) {
        set_error("%s: unknown scheme %d", who, p->scheme);
        return FBLTS_E_ARG;
    }
    const fblts_status st = build_host_mesh(desc, hm);
    if (st != FBLTS_OK) return st;
    if (p->scheme == FBLTS_SCHEME_RK4 && (hm.L != 1 || p->split)) {
        set_error("%s: RK4 needs a one-level mesh and split = 0", who);
        return FBLTS_E_ARG;
    }
    const bool f32 = p->precision == FBLTS_FP32_TENDENCY;
    build_schedule(hm, p->dt, p->beta, f32 && hm.rows_canonical, p->split, p->scheme == FBLTS_SCHEME_RK4, s);
    schedule_bytes(hm, p->forcing, f32, s);
    return FBLTS_OK;
}

extern "C" fblts_status fblts_plan_step(const fblts_mesh_desc *desc, const fblts_params *p, int64_t *ops,
                                       double *alg_bytes, int64_t *cell_updates) {
    HostMesh hm;
    Schedule s;
    const fblts_status st = plan(desc, p, "plan_step", hm, s);
    if (st != FBLTS_OK) return st;
    double b = 0.0;
    for (const Op &op : s.ops) b += op.alg_bytes;
    if (ops) *ops = (int64_t)s.ops.size();
    if (alg_bytes) *alg_bytes = b;
    if (cell_updates) *cell_updates = hm.cell_updates_per_step;
    return FBLTS_OK;
}

extern "C" fblts_status fblts_mesh_levels(const fblts_mesh *m, int32_t *level_out) {
    if (!m || !level_out) { set_error("mesh_levels: NULL argument"); return FBLTS_E_ARG; }
    const HostMesh &hm = m->hm;
    for (int i = 0; i < hm.nC; ++i) level_out[hm.cell_n2o[i]] = hm.level[i];
    return FBLTS_OK;
}

extern "C" fblts_status fblts_mesh_get_info(const fblts_mesh *m, fblts_mesh_info *info) {
    if (!m || !info) { set_error("mesh_get_info: NULL argument"); return FBLTS_E_ARG; }
    std::memset(info, 0, sizeof(*info));
    const HostMesh &hm = m->hm;
    info->nCells = hm.nC; info->nEdges = hm.nE; info->nVertices = hm.nV; info->nLevels = hm.L;
    for (int l = 0; l < hm.L && l < 8; ++l) info->cells_per_level[l] = hm.cells_per_level[l];
    info->cell_updates_per_step = hm.cell_updates_per_step;
    info->flags = hm.rows_canonical ? 1 : 0;
    // band sizes: IF-1 u IF-2 cells of each level pair
    for (int l = 0; l + 1 < hm.L && l < 8; ++l) {
        uint32_t k0 = BandKey::make(hm.L, l, 0, 0);
        int b0 = hm.cell_lb(k0);
        int b1 = hm.cell_lb(BandKey::make(hm.L, l, hm.nIF1 + hm.nIF2 + 1, 0));
        info->band_cells[l] = b1 - b0;
    }
    return FBLTS_OK;
}

// ------------------------------------------------------------------ state

static fblts_status capture_graph(fblts_state *s);

static fblts_status issue_step(fblts_state *s) {
    if (s->gexec) {
        CK(cudaGraphLaunch(s->gexec, s->st));
        return FBLTS_OK;
    }
    for (const Op &op : s->sched.ops) CK(launch_op(op, s->dm, s->arr, s->fz, s->p.g, s->d_step, s->st));
    return FBLTS_OK;
}

static fblts_status capture_graph(fblts_state *s) {
    CK(cudaStreamBeginCapture(s->st, cudaStreamCaptureModeThreadLocal));
    for (const Op &op : s->sched.ops) {
        cudaError_t e = launch_op(op, s->dm, s->arr, s->fz, s->p.g, s->d_step, s->st);
        if (e != cudaSuccess) {
            cudaGraph_t g;
            cudaStreamEndCapture(s->st, &g);
            if (g) cudaGraphDestroy(g);
            set_error("graph capture: %s", cudaGetErrorString(e));
            return FBLTS_E_CUDA;
        }
    }
    CK(cudaStreamEndCapture(s->st, &s->graph));
    CK(cudaGraphInstantiate(&s->gexec, s->graph, 0));
    return FBLTS_OK;
}

extern "C" fblts_status fblts_state_destroy(fblts_state *s) {
    if (!s) return FBLTS_OK;
    if (s->gexec) cudaGraphExecDestroy(s->gexec);
    if (s->graph) cudaGraphDestroy(s->graph);
    // stream-ordered release: no device-wide synchronisation (other states keep running)
    if (s->dbase && s->st) cudaFreeAsync(s->dbase, s->st);
    if (s->st) cudaStreamSynchronize(s->st);
    if (s->own_stream && s->st) cudaStreamDestroy(s->st);
    if (s->mesh) s->mesh->holds.fetch_sub(1);
    delete s;
    return FBLTS_OK;
}

// h holds the thickness, or with raw = true the surface elevation xi = h + b
// itself (checkpoints: the state's exact bits)
static fblts_status upload_state(fblts_state *s, const double *h, const double *u, bool raw = false) {
    const fblts_mesh *m = s->mesh;
    const int nC = m->hm.nC, nE = m->hm.nE;
    if (h) {   // the time level holds the surface elevation xi = h + b
        CK(cudaMemcpyAsync(s->d_stage_c, h, sizeof(double) * nC, cudaMemcpyHostToDevice, s->st));
        CK(launch_gather(s->arr.a[A_H], s->d_stage_c, m->cell_n2o, nC, s->st, raw ? nullptr : s->dm.bottom, +1));
    }
    if (u) {
        CK(cudaMemcpyAsync(s->d_stage_e, u, sizeof(double) * nE, cudaMemcpyHostToDevice, s->st));
        CK(launch_gather(s->arr.a[A_U], s->d_stage_e, m->edge_n2o, nE, s->st));
        CK(launch_zero_boundary(s->arr.a[A_U], s->dm.ebnd, nE, s->st));
    }
    if (s->arr.fp32 && (h || u)) CK(launch_fp32_shadows(s->dm, s->arr, s->st));
    return FBLTS_OK;
}

// every device allocation of a state, in order; the sizing pass and the
// carving pass of fblts_state_init walk the same list
static std::vector<size_t> state_plan(const fblts_mesh *m, bool f32) {
    const HostMesh &hm = m->hm;
    const size_t nC = hm.nC, nE = hm.nE, nV = hm.nV;
    auto is_double = [&](int a) {
        return !f32 || a == A_H || a == A_U || a == A_ACCH || a == A_ACCU || a == A_SH0 || a == A_SU0;
    };
    auto count = [&](int a) -> size_t {
        // FP32 path: the edge records {l F, q_e, l u, 0}, or with cell rows the
        // two cells' 8-byte shares per edge and a {B, xi*} record per cell
        if (a == A_FQU) return m->dm.rowS ? 4 * nE + 2 * nC : 4 * nE;
        return arr_is_cell(a) ? nC : (arr_is_vert(a) ? nV : nE);
    };
    const size_t szc = sizeof(double) * nC, sze = sizeof(double) * nE;
    std::vector<size_t> plan;
    for (int a = 0; a < A_COUNT; ++a) plan.push_back(count(a) * (is_double(a) ? 8 : 4));
    plan.push_back(szc);                                           // bottom
    plan.push_back(sze); plan.push_back(sze); plan.push_back(sze); plan.push_back(szc);  // forcing (double)
    if (!f32) { plan.push_back(sze); plan.push_back(sizeof(double) * nV); }   // H_e, H_v
    if (f32) {
        plan.push_back(4 * nC); plan.push_back(4 * nE);            // shadows
        plan.push_back(4 * nE);                                    // H_e
        plan.push_back(8 * nE);                                    // per-edge record {l_e, H_e}
        plan.push_back(16 * nV);                                   // per-vertex record
        plan.push_back(16 * nE); plan.push_back(4 * nC);           // forcing (float): per-edge record, p_s
    }
    plan.push_back(64);                                            // step counter + flag
    plan.push_back(sizeof(double) * (2 * DIAG_BLOCKS + 2));        // diagnostics partials
    plan.push_back(szc); plan.push_back(sze);                      // caller-order staging
    return plan;
}

static size_t plan_bytes(const std::vector<size_t> &plan) {
    Arena ar;
    for (size_t b : plan) ar.reserve(b);
    return ar.used + 256;
}

// The launch list of one coarse step with its algorithmic bytes.  States on
// one mesh with the same step, coefficients, precision and forcing switches
// share it: the mesh keeps the lists it has built.
static void cached_schedule(const fblts_mesh *m, const fblts_params *p, Schedule &out) {
    const bool f32 = p->precision == FBLTS_FP32_TENDENCY;
    const bool trisk = f32 && m->dm.rowS != 0;
    std::lock_guard<std::mutex> lock(m->cache_mu);
    const int split = p->split;
    for (const auto &c : m->sched_cache)
        if (c.dt == p->dt && c.beta[0] == p->beta[0] && c.beta[1] == p->beta[1] && c.beta[2] == p->beta[2] &&
            c.f32 == f32 && c.forcing == p->forcing && c.split == split && c.scheme == p->scheme) {
            out = c.sched;
            return;
        }
    Schedule s;
    build_schedule(m->hm, p->dt, p->beta, trisk, split, p->scheme == FBLTS_SCHEME_RK4, s);
    schedule_bytes(m->hm, p->forcing, f32, s);
    if (m->sched_cache.size() < 8)
        m->sched_cache.push_back({p->dt, {p->beta[0], p->beta[1], p->beta[2]}, f32, p->forcing, split, p->scheme, s});
    out = std::move(s);
}

extern "C" fblts_status fblts_state_device_bytes(const fblts_mesh *m, int32_t precision, size_t *bytes) {
    if (!m || !bytes) { set_error("state_device_bytes: NULL argument"); return FBLTS_E_ARG; }
    if (precision != FBLTS_FP64 && precision != FBLTS_FP32_TENDENCY) {
        set_error("state_device_bytes: unknown precision %d", precision);
        return FBLTS_E_ARG;
    }
    *bytes = plan_bytes(state_plan(m, precision == FBLTS_FP32_TENDENCY));
    return FBLTS_OK;
}

extern "C" fblts_status fblts_state_init(const fblts_mesh *m, const fblts_params *p, const double *h0,
                                         const double *u0, const double *bottom, fblts_state **out) {
    if (!out) { set_error("state_init: out is NULL"); return FBLTS_E_ARG; }
    *out = nullptr;
    if (!m || !p || !h0 || !u0 || !bottom) { set_error("state_init: NULL argument"); return FBLTS_E_ARG; }
    if (!(p->dt > 0.0) || !(p->g > 0.0)) { set_error("state_init: dt and g must be positive"); return FBLTS_E_ARG; }
    if (p->precision != FBLTS_FP64 && p->precision != FBLTS_FP32_TENDENCY) {
        set_error("state_init: unknown precision %d", p->precision);
        return FBLTS_E_ARG;
    }
    if ((p->forcing & FBLTS_FORCE_WIND_STRESS) && !m->hm.has_angle) {
        set_error("state_init: wind forcing needs angleEdge in the mesh");
        return FBLTS_E_ARG;
    }
    if ((p->forcing & FBLTS_FORCE_VORTEX) && !(m->hm.has_xy_cell && m->hm.has_xy_edge && m->hm.has_angle)) {
        set_error("state_init: vortex forcing needs xCell/yCell/xEdge/yEdge/angleEdge");
        return FBLTS_E_ARG;
    }
    if (p->forcing & ~7) { set_error("state_init: unknown forcing bits"); return FBLTS_E_ARG; }
    if (p->split < 0 || p->split > 2) { set_error("state_init: split must be 0, 1 or 2"); return FBLTS_E_ARG; }
    if (p->scheme != FBLTS_SCHEME_FBLTS && p->scheme != FBLTS_SCHEME_RK4) {
        set_error("state_init: unknown scheme %d", p->scheme);
        return FBLTS_E_ARG;
    }
    if (p->scheme == FBLTS_SCHEME_RK4 && (m->hm.L != 1 || p->split)) {
        set_error("state_init: RK4 needs a one-level mesh and split = 0");
        return FBLTS_E_ARG;
    }
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev != m->device) { set_error("state_init: current device differs from the mesh's"); return FBLTS_E_ARG; }
    fblts_state *s = new (std::nothrow) fblts_state();
    if (!s) { set_error("state_init: host allocation failed"); return FBLTS_E_OOM; }
    s->mesh = m;
    m->holds.fetch_add(1);
    s->p = *p;
    const int nC = m->hm.nC;
    if (p->stream) {
        s->st = (cudaStream_t)p->stream;
    } else {
        if (cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking) != cudaSuccess) {
            set_error("state_init: stream creation failed");
            delete s;
            return FBLTS_E_CUDA;
        }
        s->own_stream = true;
    }
    // arena layout: FP64 path every array double; FP32 path the time level,
    // correction sums and saved time level double, everything else float
    const bool f32 = p->precision == FBLTS_FP32_TENDENCY;
    auto is_double = [&](int a) {
        return !f32 || a == A_H || a == A_U || a == A_ACCH || a == A_ACCU || a == A_SH0 || a == A_SU0;
    };
    // the launch list of one coarse step and its algorithmic bytes
    cached_schedule(m, p, s->sched);
    const std::vector<size_t> plan = state_plan(m, f32);
    size_t szc = sizeof(double) * (size_t)nC;
    Arena ar;
    ar.size = plan_bytes(plan);
    if (cudaMallocAsync(&s->dbase, ar.size, s->st) != cudaSuccess) {
        cudaGetLastError();
        s->dbase = nullptr;
        set_error("state_init: device allocation of %zu bytes failed", ar.size);
        fblts_state_destroy(s);
        return FBLTS_E_OOM;
    }
    ar.base = (char *)s->dbase;
    ar.used = 0;
    std::vector<void *> got;
    for (size_t b : plan) {
        void *ptr = ar.take(b);
        if (!ptr) {
            set_error("state_init: arena layout error");
            fblts_state_destroy(s);
            return FBLTS_E_OOM;
        }
        got.push_back(ptr);
    }
    size_t gi = 0;
    s->arr.fp32 = f32 ? 1 : 0;
    for (int a = 0; a < A_COUNT; ++a) {
        void *ptr = got[gi++];
        s->arr.a[a] = is_double(a) ? (double *)ptr : nullptr;
        s->arr.f[a] = is_double(a) ? nullptr : (float *)ptr;
    }
    // the TRiSK pass's per-cell records follow its per-edge shares (4 floats per edge)
    s->arr.bx32 = (f32 && m->dm.rowS) ? s->arr.f[A_FQU] + 4 * (size_t)m->hm.nE : nullptr;
    double *db = (double *)got[gi++];
    s->fz.windN = (double *)got[gi++];
    s->fz.windT = (double *)got[gi++];
    s->fz.cw = (double *)got[gi++];
    s->fz.ps = (double *)got[gi++];
    double *He64 = nullptr, *Hv64 = nullptr;
    if (!f32) {
        He64 = (double *)got[gi++];
        Hv64 = (double *)got[gi++];
    }
    float *He32 = nullptr;
    float4 *vkh = nullptr;
    float2 *el2 = nullptr;
    if (f32) {
        s->arr.xi32 = (float *)got[gi++];
        s->arr.u32 = (float *)got[gi++];
        He32 = (float *)got[gi++];
        el2 = (float2 *)got[gi++];
        vkh = (float4 *)got[gi++];
        s->fz.wrec32 = (float4 *)got[gi++];
        s->fz.ps32 = (float *)got[gi++];
    }
    s->d_step = (long long *)got[gi++];
    s->d_flag = (int *)((char *)s->d_step + 16);
    s->d_partials = (double *)got[gi++];
    s->d_diag = s->d_partials + 2 * DIAG_BLOCKS;
    s->d_stage_c = (double *)got[gi++];
    s->d_stage_e = (double *)got[gi++];
    if (cudaMemsetAsync(s->dbase, 0, ar.size, s->st) != cudaSuccess) {
        set_error("state_init: memset failed");
        fblts_state_destroy(s);
        return FBLTS_E_CUDA;
    }
    s->dm = m->dm;
    s->dm.bottom = db;
    fblts_status st = FBLTS_OK;
    // the bottom first: the time level is stored as xi = h + b
    if (cudaMemcpyAsync(s->d_stage_c, bottom, szc, cudaMemcpyHostToDevice, s->st) != cudaSuccess ||
        launch_gather(db, s->d_stage_c, m->cell_n2o, nC, s->st) != cudaSuccess) {
        set_error("state_init: bottom upload failed");
        st = FBLTS_E_CUDA;
    }
    if (st == FBLTS_OK && !f32) {
        s->dm.He64 = He64; s->dm.Hv64 = Hv64;
        if (launch_fp64_depths(s->dm, He64, Hv64, s->st) != cudaSuccess) {
            set_error("state_init: FP64 setup failed");
            st = FBLTS_E_CUDA;
        }
    }
    if (st == FBLTS_OK) st = upload_state(s, h0, u0);
    if (st == FBLTS_OK && f32) {
        s->dm.He32 = He32; s->dm.el2 = el2; s->dm.vKh = vkh;
        if (launch_fp32_depths(s->dm, He32, el2, vkh, s->st) != cudaSuccess ||
            launch_fp32_shadows(s->dm, s->arr, s->st) != cudaSuccess) {
            set_error("state_init: FP32 setup failed");
            st = FBLTS_E_CUDA;
        }
    }
    if (st != FBLTS_OK) { fblts_state_destroy(s); return st; }
    DevForcing &fz = s->fz;
    fz.fp32 = f32 ? 1 : 0;
    fz.flags = p->forcing;
    fz.wind_u = p->wind_u; fz.wind_v = p->wind_v; fz.cd = p->cd; fz.cd32 = (float)p->cd;
    fz.rho0 = p->rho0 > 0 ? p->rho0 : 1025.0;
    fz.inv_rho0 = 1.0 / fz.rho0;
    fz.rho_air = p->rho_air > 0 ? p->rho_air : 1.225;
    for (int k = 0; k < 9; ++k) fz.vx[k] = p->vortex[k];
    fz.t0 = p->t0; fz.dt = p->dt; fz.step = s->d_step;
    if (cudaStreamSynchronize(s->st) != cudaSuccess) {
        set_error("state_init: %s", cudaGetErrorString(cudaGetLastError()));
        fblts_state_destroy(s);
        return FBLTS_E_CUDA;
    }
    if (p->use_graph) {
        st = capture_graph(s);
        if (st != FBLTS_OK) { fblts_state_destroy(s); return st; }
    }
    *out = s;
    return FBLTS_OK;
}

extern "C" fblts_status fblts_lts_advance(fblts_state *s, int64_t n) {
    if (!s || n < 0) { set_error("lts_advance: bad arguments"); return FBLTS_E_ARG; }
    for (int64_t i = 0; i < n; ++i) {
        fblts_status st = issue_step(s);
        if (st != FBLTS_OK) return st;
    }
    if (n > 0)
        CK(launch_check(s->arr.a[A_H], s->dm.bottom, s->mesh->hm.nC, s->arr.a[A_U], s->mesh->hm.nE, s->d_flag,
                        s->st));
    s->steps += n;
    return FBLTS_OK;
}

static fblts_status sync_and_check(const fblts_state *s) {
    CK(cudaStreamSynchronize(s->st));
    int flag = 0;
    CK(cudaMemcpy(&flag, s->d_flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        set_error("state became non-finite or a thickness is <= 0");
        return FBLTS_E_UNSTABLE;
    }
    return FBLTS_OK;
}

extern "C" fblts_status fblts_synchronize(fblts_state *s) {
    if (!s) { set_error("synchronize: NULL state"); return FBLTS_E_ARG; }
    return sync_and_check(s);
}

// caller-order copies of h = xi - b (raw: of xi itself) and u; synchronises
static fblts_status read_state(const fblts_state *s, double *h_out, double *u_out, bool raw) {
    const fblts_mesh *m = s->mesh;
    const int nC = m->hm.nC, nE = m->hm.nE;
    if (h_out) {
        CK(launch_gather(s->d_stage_c, s->arr.a[A_H], m->cell_o2n, nC, s->st, raw ? nullptr : s->dm.bottom, -1));
        CK(cudaMemcpyAsync(h_out, s->d_stage_c, sizeof(double) * nC, cudaMemcpyDeviceToHost, s->st));
    }
    if (u_out) {
        CK(launch_gather(s->d_stage_e, s->arr.a[A_U], m->edge_o2n, nE, s->st));
        CK(cudaMemcpyAsync(u_out, s->d_stage_e, sizeof(double) * nE, cudaMemcpyDeviceToHost, s->st));
    }
    return sync_and_check(s);
}

extern "C" fblts_status fblts_state_read(const fblts_state *s, double *h_out, double *u_out) {
    if (!s) { set_error("state_read: NULL state"); return FBLTS_E_ARG; }
    return read_state(s, h_out, u_out, false);
}

extern "C" fblts_status fblts_state_write(fblts_state *s, const double *h, const double *u) {
    if (!s) { set_error("state_write: NULL state"); return FBLTS_E_ARG; }
    return upload_state(s, h, u);
}

extern "C" fblts_status fblts_run_host(fblts_state *s, const double *h_in, const double *u_in, int64_t n,
                                       double *h_out, double *u_out) {
    if (!s) { set_error("run_host: NULL state"); return FBLTS_E_ARG; }
    fblts_status st = upload_state(s, h_in, u_in);
    if (st != FBLTS_OK) return st;
    st = fblts_lts_advance(s, n);
    if (st != FBLTS_OK) return st;
    return fblts_state_read(s, h_out, u_out);
}

extern "C" fblts_status fblts_diagnostics(const fblts_state *s, double *mass, double *absvort) {
    if (!s) { set_error("diagnostics: NULL state"); return FBLTS_E_ARG; }
    CK(launch_diagnostics(s->dm, s->arr.a[A_H], s->arr.a[A_U], s->d_partials, DIAG_BLOCKS, s->d_diag, s->st));
    double out[2];
    CK(cudaMemcpyAsync(out, s->d_diag, sizeof(out), cudaMemcpyDeviceToHost, s->st));
    fblts_status st = sync_and_check(s);
    if (mass) *mass = out[0];
    if (absvort) *absvort = out[1];
    return st;
}

extern "C" fblts_status fblts_state_time(const fblts_state *s, int64_t *steps, double *time) {
    if (!s) { set_error("state_time: NULL state"); return FBLTS_E_ARG; }
    if (steps) *steps = s->steps;
    if (time) *time = s->p.t0 + (double)s->steps * s->p.dt;
    return FBLTS_OK;
}

namespace {
struct CkptHeader {
    char magic[8];
    int64_t nC, nE, steps;
    double t0, dt;
};
}  // namespace

extern "C" fblts_status fblts_state_save(const fblts_state *s, void *buf, size_t *len) {
    if (!s || !len) { set_error("state_save: NULL argument"); return FBLTS_E_ARG; }
    const int nC = s->mesh->hm.nC, nE = s->mesh->hm.nE;
    size_t need = sizeof(CkptHeader) + sizeof(double) * ((size_t)nC + nE);
    if (!buf) { *len = need; return FBLTS_OK; }
    if (*len < need) { set_error("state_save: buffer of %zu bytes, need %zu", *len, need); return FBLTS_E_ARG; }
    CkptHeader hd;
    std::memcpy(hd.magic, "FBLTSCK2", 8);
    hd.nC = nC; hd.nE = nE; hd.steps = s->steps; hd.t0 = s->p.t0; hd.dt = s->p.dt;
    std::memcpy(buf, &hd, sizeof(hd));
    // the surface elevation xi = h + b as stored (the state's exact bits), and u
    double *h = (double *)((char *)buf + sizeof(hd));
    fblts_status st = read_state(s, h, h + nC, true);
    *len = need;
    return st;
}

extern "C" fblts_status fblts_state_load(fblts_state *s, const void *buf, size_t len) {
    if (!s || !buf) { set_error("state_load: NULL argument"); return FBLTS_E_ARG; }
    const int nC = s->mesh->hm.nC, nE = s->mesh->hm.nE;
    CkptHeader hd;
    if (len < sizeof(hd)) { set_error("state_load: buffer too small"); return FBLTS_E_STATE; }
    std::memcpy(&hd, buf, sizeof(hd));
    if (std::memcmp(hd.magic, "FBLTSCK2", 8) != 0 || hd.nC != nC || hd.nE != nE ||
        len < sizeof(hd) + sizeof(double) * ((size_t)nC + nE)) {
        set_error("state_load: checkpoint does not match this mesh");
        return FBLTS_E_STATE;
    }
    const double *h = (const double *)((const char *)buf + sizeof(hd));
    fblts_status st = upload_state(s, h, h + nC, true);
    if (st != FBLTS_OK) return st;
    long long step = hd.steps;
    CK(cudaMemcpyAsync(s->d_step, &step, sizeof(step), cudaMemcpyHostToDevice, s->st));
    CK(cudaStreamSynchronize(s->st));
    s->steps = hd.steps;
    return FBLTS_OK;
}

// whether launch_op issues a kernel for this op
static bool op_launches(const fblts_state *s, const Op &op) {
    if (op.kind == OP_FORCING) return s->fz.flags != 0;
    if (op.kind == OP_CELL || op.kind == OP_VERT || op.kind == OP_EPREP || op.kind == OP_EDGE || op.kind == OP_TRISK)
        return op.hi > op.lo;
    return true;
}

extern "C" fblts_status fblts_state_launches_per_step(const fblts_state *s, int64_t *launches) {
    if (!s || !launches) { set_error("launches_per_step: NULL argument"); return FBLTS_E_ARG; }
    int64_t n = 0;
    for (const Op &op : s->sched.ops) n += op_launches(s, op) ? 1 : 0;
    *launches = n;
    return FBLTS_OK;
}

static int op_kind_profile(int kind) {
    switch (kind) {
        case OP_CELL: return FBLTS_PK_CELL;
        case OP_VERT: return FBLTS_PK_VERTEX;
        case OP_EPREP: return FBLTS_PK_EDGE_PREP;
        case OP_EDGE: return FBLTS_PK_EDGE;
        case OP_SAVE: return FBLTS_PK_SAVE;
        case OP_PRED: return FBLTS_PK_PREDICT;
        case OP_FINAL: return FBLTS_PK_CORRECT;
        case OP_FORCING: return FBLTS_PK_FORCING;
        case OP_TRISK: return FBLTS_PK_TRISK;
        default: return FBLTS_PK_STEP_END;
    }
}

static_assert(FBLTS_SEG_NONE == SEG_NONE && FBLTS_SEG_STAGE == SEG_UPD && FBLTS_SEG_IN_PLACE == SEG_INPLACE &&
                  FBLTS_SEG_SUM_SET == SEG_ACC_SET && FBLTS_SEG_SUM_ADD == SEG_ACC_ADD &&
                  FBLTS_SEG_KE_ONLY == SEG_KONLY && FBLTS_SEG_TENDENCY == SEG_PHI && FBLTS_SEG_RK4_SET == SEG_RK_SET &&
                  FBLTS_SEG_RK4_ADD2 == SEG_RK_ADD2 && FBLTS_SEG_RK4_FINAL == SEG_RK_FIN,
              "public segment modes");

extern "C" fblts_status fblts_plan_op(const fblts_mesh_desc *desc, const fblts_params *p, int64_t index,
                                     int32_t *kind, int32_t *stage, uint8_t *mode) {
    HostMesh hm;
    Schedule s;
    const fblts_status st = plan(desc, p, "plan_op", hm, s);
    if (st != FBLTS_OK) return st;
    if (index < 0 || index >= (int64_t)s.ops.size()) {
        set_error("plan_op: index %lld outside [0, %zu)", (long long)index, s.ops.size());
        return FBLTS_E_ARG;
    }
    const Op &op = s.ops[(size_t)index];
    const bool pass = op.kind == OP_CELL || op.kind == OP_VERT || op.kind == OP_EPREP || op.kind == OP_EDGE ||
                      op.kind == OP_TRISK;
    if (kind) *kind = op_kind_profile(op.kind);
    if (stage) *stage = pass ? op.stage : 0;
    if (mode && pass) {
        const bool cells = op.kind == OP_CELL || op.kind == OP_TRISK, verts = op.kind == OP_VERT;
        const int n = cells ? hm.nC : (verts ? hm.nV : hm.nE);
        const std::vector<int> &n2o = cells ? hm.cell_n2o : (verts ? hm.vert_n2o : hm.edge_n2o);
        for (int x = 0; x < n; ++x) mode[n2o[x]] = SEG_NONE;
        // the last segment containing an element decides its mode, as in the kernels
        for (int x = std::max(op.lo, 0); x < std::min(op.hi, n); ++x) {
            int m = SEG_NONE;
            for (int k = 0; k < op.nseg; ++k)
                if (x >= op.seg[k].begin && x < op.seg[k].end) m = op.seg[k].mode;
            mode[n2o[x]] = (uint8_t)m;
        }
    }
    return FBLTS_OK;
}

extern "C" fblts_status fblts_plan_op_bytes(const fblts_mesh_desc *desc, const fblts_params *p, int64_t index,
                                           double *alg_bytes, double *moved_bytes) {
    HostMesh hm;
    Schedule s;
    const fblts_status st = plan(desc, p, "plan_op_bytes", hm, s);
    if (st != FBLTS_OK) return st;
    if (index < 0 || index >= (int64_t)s.ops.size()) {
        set_error("plan_op_bytes: index %lld outside [0, %zu)", (long long)index, s.ops.size());
        return FBLTS_E_ARG;
    }
    if (alg_bytes) *alg_bytes = s.ops[(size_t)index].alg_bytes;
    if (moved_bytes) *moved_bytes = s.ops[(size_t)index].moved_bytes;
    return FBLTS_OK;
}

extern "C" fblts_status fblts_state_profile_step(fblts_state *s, double *ms, int64_t *launches, double *bytes) {
    if (!s) { set_error("profile_step: NULL state"); return FBLTS_E_ARG; }
    const size_t n = s->sched.ops.size();
    std::vector<cudaEvent_t> ev(2 * n, nullptr);
    for (auto &e : ev) CK(cudaEventCreate(&e));
    fblts_status st = FBLTS_OK;
    for (size_t i = 0; i < n && st == FBLTS_OK; ++i) {
        const Op &op = s->sched.ops[i];
        cudaError_t e1 = cudaEventRecord(ev[2 * i], s->st);
        cudaError_t e2 = launch_op(op, s->dm, s->arr, s->fz, s->p.g, s->d_step, s->st);
        cudaError_t e3 = cudaEventRecord(ev[2 * i + 1], s->st);
        if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
            set_error("profile_step: launch failed: %s", cudaGetErrorString(e2 != cudaSuccess ? e2 : (e1 != cudaSuccess ? e1 : e3)));
            st = FBLTS_E_CUDA;
        }
    }
    if (st == FBLTS_OK && cudaStreamSynchronize(s->st) != cudaSuccess) {
        set_error("profile_step: %s", cudaGetErrorString(cudaGetLastError()));
        st = FBLTS_E_CUDA;
    }
    double tms[FBLTS_PROFILE_KINDS] = {0}, tb[FBLTS_PROFILE_KINDS] = {0};
    int64_t tl[FBLTS_PROFILE_KINDS] = {0};
    for (size_t i = 0; i < n && st == FBLTS_OK; ++i) {
        const Op &op = s->sched.ops[i];
        if (!op_launches(s, op)) continue;
        float t = 0.f;
        cudaEventElapsedTime(&t, ev[2 * i], ev[2 * i + 1]);
        int k = op_kind_profile(op.kind);
        tms[k] += t;
        tl[k] += 1;
        tb[k] += op.alg_bytes;
    }
    for (auto &e : ev) cudaEventDestroy(e);
    if (st != FBLTS_OK) return st;
    s->steps += 1;
    for (int k = 0; k < FBLTS_PROFILE_KINDS; ++k) {
        if (ms) ms[k] = tms[k];
        if (launches) launches[k] = tl[k];
        if (bytes) bytes[k] = tb[k];
    }
    return FBLTS_OK;
}

extern "C" fblts_status fblts_state_step_bytes(const fblts_state *s, double *bytes, int64_t *cell_updates) {
    if (!s) { set_error("step_bytes: NULL state"); return FBLTS_E_ARG; }
    double b = 0.0;
    for (const Op &op : s->sched.ops) b += op.alg_bytes;
    if (bytes) *bytes = b;
    if (cell_updates) *cell_updates = s->mesh->hm.cell_updates_per_step;
    return FBLTS_OK;
}

extern "C" fblts_status fblts_state_bytes_by_kind(const fblts_state *s, double *alg, double *moved) {
    if (!s) { set_error("bytes_by_kind: NULL state"); return FBLTS_E_ARG; }
    double a[FBLTS_PROFILE_KINDS] = {0}, m[FBLTS_PROFILE_KINDS] = {0};
    for (const Op &op : s->sched.ops) {
        if (!op_launches(s, op)) continue;
        const int k = op_kind_profile(op.kind);
        a[k] += op.alg_bytes;
        m[k] += op.moved_bytes;
    }
    for (int k = 0; k < FBLTS_PROFILE_KINDS; ++k) {
        if (alg) alg[k] = a[k];
        if (moved) moved[k] = m[k];
    }
    return FBLTS_OK;
}
