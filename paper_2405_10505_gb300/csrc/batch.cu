// Batched ensemble (fblts_batch_*): several FB-LTS states, each on its own
// mesh, advance together.  One coarse step of every member is merged into one
// launch list: each launch runs one op of several members that share a kernel
// body (same pass, same template configuration) as a persistent grid over the
// members' tiles.  Each tile copies its member's mesh tables, forcing and
// launch arguments into shared memory and runs the same per-element bodies as
// the single-state kernels, so a member's result is the same alone and in a
// batch up to the float rounding of multiply-adds the compiler may contract
// differently in these kernels (bitwise in branch mode, which launches the
// members' own kernels).  The launch shape (threads per block, resident CTAs per SM)
// and the order of the members' tiles are chosen online: the first rounds of
// fblts_batch_advance each run one candidate shape under CUDA events, and the
// fastest is kept.
#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <numeric>
#include <utility>
#include <vector>

#include "handles.h"
#include "kernel_bodies32.cuh"

namespace fblts {

namespace {

// kernel body of a batched launch (pass x template configuration)
enum BodyKind : int {
    BK_CELL8, BK_CELL12, BK_VERT, BK_TRISK8, BK_TRISK8V, BK_TRISK12, BK_TRISK12V, BK_EDGE, BK_EDGEF,
    BK_SAVE, BK_PRED, BK_FINAL, BK_FORCING, BK_STEP_END, BK_COUNT
};

// one member's op in a batched launch
struct alignas(16) BatchItem {
    DevMesh m;
    DevForcing fz;
    union Args {
        CellArgs32 c;
        VertArgs32 v;
        TriskArgs32 t;
        EdgeArgs32 e;
        IfArgs32 f;
        Args() {}
    } a;
    long long *step;   // the member's device step counter
    int lo;            // first element (cells, vertices, edges) or 0 for the interface ops
    int n;             // threads of work
    int tile0;         // first tile of the item in its launch
};
static_assert(sizeof(BatchItem) % 16 == 0, "item copied as int4");

constexpr int MAX_TPB = 256;

__device__ __forceinline__ void wait_predecessor() {
#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 900)
    cudaGridDependencySynchronize();
#endif
}

template <int BK>
__device__ __forceinline__ void run_body(const BatchItem &it, int idx) {
    const int x = it.lo + idx;
    if constexpr (BK == BK_CELL8) cell32_body<8, true>(it.m, it.a.c, x);
    if constexpr (BK == BK_CELL12) cell32_body<12, true>(it.m, it.a.c, x);
    if constexpr (BK == BK_VERT) vert32_body(it.m, it.a.v, x);
    if constexpr (BK == BK_TRISK8) trisk32_body<8, false>(it.m, it.a.t, it.fz, x);
    if constexpr (BK == BK_TRISK8V) trisk32_body<8, true>(it.m, it.a.t, it.fz, x);
    if constexpr (BK == BK_TRISK12) trisk32_body<12, false>(it.m, it.a.t, it.fz, x);
    if constexpr (BK == BK_TRISK12V) trisk32_body<12, true>(it.m, it.a.t, it.fz, x);
    if constexpr (BK == BK_EDGE) edge32_body<true, false>(it.m, it.a.e, it.fz, x);
    if constexpr (BK == BK_EDGEF) edge32_body<true, true>(it.m, it.a.e, it.fz, x);
    if constexpr (BK == BK_SAVE) save32_body(it.a.f, idx);
    if constexpr (BK == BK_PRED) pred32_body(it.a.f, idx);
    if constexpr (BK == BK_FINAL) final32_body(it.a.f, it.m.ebnd, idx);
    if constexpr (BK == BK_FORCING) {
        const double time = it.fz.t0 + (double)(*it.fz.step) * it.fz.dt;
        forcing32_body(it.m, it.fz, time, idx);
    }
    if constexpr (BK == BK_STEP_END) {
        if (idx == 0) *it.step += 1;
    }
}

// Persistent grid over the tiles of all items of one batched launch; tile t
// belongs to the last item whose tile0 <= t.  The block stages that item in
// shared memory once per change of item.
template <int BK>
__global__ void __launch_bounds__(MAX_TPB) batch_pass(const BatchItem *items, int nitems, int ntiles) {
    __shared__ __align__(16) unsigned char buf[sizeof(BatchItem)];
    const BatchItem &it = *reinterpret_cast<const BatchItem *>(buf);
    wait_predecessor();
    int cur = -1;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        int lo = 0, hi = nitems - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (items[mid].tile0 <= t) lo = mid;
            else hi = mid - 1;
        }
        if (lo != cur) {
            __syncthreads();
            const int4 *src = reinterpret_cast<const int4 *>(items + lo);
            int4 *dst = reinterpret_cast<int4 *>(buf);
            for (int w = threadIdx.x; w < (int)(sizeof(BatchItem) / 16); w += blockDim.x) dst[w] = src[w];
            __syncthreads();
            cur = lo;
        }
        const int idx = (t - it.tile0) * blockDim.x + threadIdx.x;
        if (idx < it.n) run_body<BK>(it, idx);
    }
}

template <int BK>
cudaError_t launch_batch_pass(const BatchItem *items, int nitems, int ntiles, int grid, int tpb, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(tpb);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, batch_pass<BK>, items, nitems, ntiles);
}

cudaError_t launch_body(int bk, const BatchItem *items, int nitems, int ntiles, int grid, int tpb, cudaStream_t st) {
    switch (bk) {
        case BK_CELL8: return launch_batch_pass<BK_CELL8>(items, nitems, ntiles, grid, tpb, st);
        case BK_CELL12: return launch_batch_pass<BK_CELL12>(items, nitems, ntiles, grid, tpb, st);
        case BK_VERT: return launch_batch_pass<BK_VERT>(items, nitems, ntiles, grid, tpb, st);
        case BK_TRISK8: return launch_batch_pass<BK_TRISK8>(items, nitems, ntiles, grid, tpb, st);
        case BK_TRISK8V: return launch_batch_pass<BK_TRISK8V>(items, nitems, ntiles, grid, tpb, st);
        case BK_TRISK12: return launch_batch_pass<BK_TRISK12>(items, nitems, ntiles, grid, tpb, st);
        case BK_TRISK12V: return launch_batch_pass<BK_TRISK12V>(items, nitems, ntiles, grid, tpb, st);
        case BK_EDGE: return launch_batch_pass<BK_EDGE>(items, nitems, ntiles, grid, tpb, st);
        case BK_EDGEF: return launch_batch_pass<BK_EDGEF>(items, nitems, ntiles, grid, tpb, st);
        case BK_SAVE: return launch_batch_pass<BK_SAVE>(items, nitems, ntiles, grid, tpb, st);
        case BK_PRED: return launch_batch_pass<BK_PRED>(items, nitems, ntiles, grid, tpb, st);
        case BK_FINAL: return launch_batch_pass<BK_FINAL>(items, nitems, ntiles, grid, tpb, st);
        case BK_FORCING: return launch_batch_pass<BK_FORCING>(items, nitems, ntiles, grid, tpb, st);
        case BK_STEP_END: return launch_batch_pass<BK_STEP_END>(items, nitems, ntiles, grid, tpb, st);
        default: return cudaErrorInvalidValue;
    }
}

// body kind of a member's op, or -1 when the op launches nothing
int body_kind(const fblts_state *s, const Op &op) {
    const DevMesh &m = s->dm;
    const bool vx = (s->fz.flags & FBLTS_FORCE_VORTEX) != 0;
    switch (op.kind) {
        case OP_CELL: return op.hi > op.lo ? (m.rowS == 8 ? BK_CELL8 : BK_CELL12) : -1;
        case OP_VERT: return op.hi > op.lo ? BK_VERT : -1;
        case OP_TRISK:
            if (op.hi <= op.lo) return -1;
            return m.rowS == 8 ? (vx ? BK_TRISK8V : BK_TRISK8) : (vx ? BK_TRISK12V : BK_TRISK12);
        case OP_EDGE: return op.hi > op.lo ? (s->fz.flags ? BK_EDGEF : BK_EDGE) : -1;
        case OP_SAVE: return BK_SAVE;
        case OP_PRED: return BK_PRED;
        case OP_FINAL: return BK_FINAL;
        case OP_FORCING: return s->fz.flags ? BK_FORCING : -1;
        case OP_STEP_END: return BK_STEP_END;
        default: return -2;
    }
}

BatchItem make_item(const fblts_state *s, const Op &op, int bk) {
    BatchItem it;
    std::memset(static_cast<void *>(&it), 0, sizeof(it));
    it.m = s->dm;
    it.fz = s->fz;
    it.step = s->d_step;
    const DevArrays &arr = s->arr;
    switch (bk) {
        case BK_CELL8: case BK_CELL12:
            it.a.c = cell_args32(op, arr, s->dm); it.lo = op.lo; it.n = op.hi - op.lo; break;
        case BK_VERT:
            it.a.v = vert_args32(op, arr); it.lo = op.lo; it.n = op.hi - op.lo; break;
        case BK_TRISK8: case BK_TRISK8V: case BK_TRISK12: case BK_TRISK12V:
            it.a.t = trisk_args32(op, arr, s->p.g, s->fz.rho0); it.lo = op.lo; it.n = op.hi - op.lo; break;
        case BK_EDGE: case BK_EDGEF:
            it.a.e = edge_args32(op, arr, s->p.g); it.lo = op.lo; it.n = op.hi - op.lo; break;
        case BK_SAVE: case BK_PRED: case BK_FINAL:
            it.a.f = if_args32(op, arr, s->dm); it.lo = 0; it.n = it.a.f.n; break;
        case BK_FORCING:
            it.lo = 0; it.n = s->dm.nE > s->dm.nC ? s->dm.nE : s->dm.nC; break;
        case BK_STEP_END:
            it.lo = 0; it.n = 1; break;
        default: break;
    }
    return it;
}

// launch shape.  mode 0: merged launches, each a grid over the members' tiles
// with tpb threads per block, ctas_per_sm x SM count CTAs looping over the
// tiles (0: one CTA per tile), tiles ordered largest member op first (order 0)
// or by member (1).  mode 1: no merging, the members' own launches as
// parallel branches of one graph (the GPU runs independent branches
// concurrently).  mode 2: members with the same op sequence (levels, M)
// merged, each such group a parallel branch; mode 3: as mode 2 with groups of
// at most 4 members.
struct Shape {
    int tpb, ctas_per_sm, order, mode;
    bool operator==(const Shape &o) const {
        return tpb == o.tpb && ctas_per_sm == o.ctas_per_sm && order == o.order && mode == o.mode;
    }
};

}  // namespace

}  // namespace fblts

using namespace fblts;

struct fblts_batch {
    std::vector<fblts_state *> members;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    int nsm = 0;
    // merged launch list: per launch, its body kind and (member, op) pairs
    struct Launch {
        int bk;
        std::vector<std::pair<int, int>> ops;
    };
    std::vector<Launch> launches;                 // mode 0: all members merged
    std::vector<std::vector<Launch>> glaunches;   // mode 2: per group of members with the same op sequence
    std::vector<std::vector<Launch>> slaunches;   // mode 3: those groups split into groups of at most 4
    // device items of the current shape, and the offsets of each launch's items
    BatchItem *d_items = nullptr;
    size_t d_items_cap = 0;
    std::vector<int> item_off, item_n, ntiles;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    Shape shape{256, 4, 0};
    // online tuning: candidate shapes, one timed round each
    std::vector<Shape> cands;
    std::vector<float> cand_ms;
    size_t next_cand = 0;
    bool tuned = false;
    cudaEvent_t e0 = nullptr, e1 = nullptr, done = nullptr;
    // branch mode: one capture stream and join event per member, and the fork event
    std::vector<cudaStream_t> bst;
    std::vector<cudaEvent_t> bjoin;
    cudaEvent_t fork = nullptr;
    int64_t rounds = 0;
    int64_t cell_updates_per_round = 0;
};

static void destroy_graph(fblts_batch *b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->gexec = nullptr;
    b->graph = nullptr;
}

// the members' own launch lists as parallel branches of one captured graph
static fblts_status build_branches(fblts_batch *b, const Shape &sh) {
    const int n = (int)b->members.size();
    CK(cudaStreamSynchronize(b->st));
    CK(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaEventRecord(b->fork, b->st);
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        const fblts_state *s = b->members[i];
        e = cudaStreamWaitEvent(b->bst[i], b->fork, 0);
        for (size_t k = 0; k < s->sched.ops.size() && e == cudaSuccess; ++k)
            e = launch_op(s->sched.ops[k], s->dm, s->arr, s->fz, s->p.g, s->d_step, b->bst[i]);
        if (e == cudaSuccess) e = cudaEventRecord(b->bjoin[i], b->bst[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->st, b->bjoin[i], 0);
    }
    if (e != cudaSuccess) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(b->st, &g);
        if (g) cudaGraphDestroy(g);
        set_error("batch: branch capture failed: %s", cudaGetErrorString(e));
        return FBLTS_E_CUDA;
    }
    CK(cudaStreamEndCapture(b->st, &b->graph));
    CK(cudaGraphInstantiate(&b->gexec, b->graph, 0));
    CK(cudaGraphUpload(b->gexec, b->st));
    b->shape = sh;
    return FBLTS_OK;
}

// items of every launch for a shape, uploaded, and the graph of one round:
// mode 0 the merged launches in one chain, mode 2 each group's merged
// launches as a parallel branch, mode 1 the members' own launches as branches
static fblts_status build_round(fblts_batch *b, const Shape &sh) {
    destroy_graph(b);
    if (sh.mode == 1) return build_branches(b, sh);
    std::vector<const std::vector<fblts_batch::Launch> *> lists;
    if (sh.mode == 0) lists.push_back(&b->launches);
    for (const auto &g : (sh.mode == 3 ? b->slaunches : b->glaunches))
        if (sh.mode >= 2) lists.push_back(&g);
    std::vector<BatchItem> items;
    b->item_off.clear();
    b->item_n.clear();
    b->ntiles.clear();
    for (const auto *list : lists)
        for (const auto &L : *list) {
            std::vector<BatchItem> its;
            for (const auto &mo : L.ops) {
                const fblts_state *s = b->members[mo.first];
                its.push_back(make_item(s, s->sched.ops[mo.second], L.bk));
            }
            if (sh.order == 0)
                std::stable_sort(its.begin(), its.end(),
                                 [](const BatchItem &x, const BatchItem &y) { return x.n > y.n; });
            int tiles = 0;
            for (auto &it : its) {
                it.tile0 = tiles;
                tiles += (it.n + sh.tpb - 1) / sh.tpb;
            }
            b->item_off.push_back((int)items.size());
            b->item_n.push_back((int)its.size());
            b->ntiles.push_back(tiles);
            items.insert(items.end(), its.begin(), its.end());
        }
    const size_t bytes = items.size() * sizeof(BatchItem);
    if (bytes > b->d_items_cap) {
        CK(cudaStreamSynchronize(b->st));
        if (b->d_items) cudaFree(b->d_items);
        b->d_items = nullptr;
        b->d_items_cap = 0;
        CK(cudaMalloc(&b->d_items, bytes));
        b->d_items_cap = bytes;
    }
    CK(cudaStreamSynchronize(b->st));
    CK(cudaMemcpy(b->d_items, items.data(), bytes, cudaMemcpyHostToDevice));
    CK(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
    const bool branches = sh.mode >= 2;
    cudaError_t e = branches ? cudaEventRecord(b->fork, b->st) : cudaSuccess;
    size_t k = 0;
    for (size_t li = 0; li < lists.size() && e == cudaSuccess; ++li) {
        cudaStream_t st = branches ? b->bst[li] : b->st;
        if (branches) e = cudaStreamWaitEvent(st, b->fork, 0);
        for (const auto &L : *lists[li]) {
            const int tiles = b->ntiles[k];
            if (tiles > 0 && e == cudaSuccess) {
                const int grid = sh.ctas_per_sm > 0 ? std::max(1, std::min(tiles, sh.ctas_per_sm * b->nsm)) : tiles;
                e = launch_body(L.bk, b->d_items + b->item_off[k], b->item_n[k], tiles, grid, sh.tpb, st);
            }
            ++k;
        }
        if (branches && e == cudaSuccess) e = cudaEventRecord(b->bjoin[li], st);
        if (branches && e == cudaSuccess) e = cudaStreamWaitEvent(b->st, b->bjoin[li], 0);
    }
    if (e != cudaSuccess) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(b->st, &g);
        if (g) cudaGraphDestroy(g);
        set_error("batch: launch capture failed: %s", cudaGetErrorString(e));
        return FBLTS_E_CUDA;
    }
    CK(cudaStreamEndCapture(b->st, &b->graph));
    CK(cudaGraphInstantiate(&b->gexec, b->graph, 0));
    CK(cudaGraphUpload(b->gexec, b->st));
    b->shape = sh;
    return FBLTS_OK;
}

extern "C" fblts_status fblts_batch_destroy(fblts_batch *b) {
    if (!b) return FBLTS_OK;
    if (b->st) cudaStreamSynchronize(b->st);
    destroy_graph(b);
    for (cudaStream_t x : b->bst) cudaStreamDestroy(x);
    for (cudaEvent_t x : b->bjoin) cudaEventDestroy(x);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->d_items) cudaFree(b->d_items);
    if (b->e0) cudaEventDestroy(b->e0);
    if (b->e1) cudaEventDestroy(b->e1);
    if (b->done) cudaEventDestroy(b->done);
    if (b->own_stream && b->st) cudaStreamDestroy(b->st);
    delete b;
    return FBLTS_OK;
}

extern "C" fblts_status fblts_batch_create(fblts_state *const *members, int32_t n, const fblts_batch_opts *opts,
                                           fblts_batch **out) {
    if (!out) { set_error("batch_create: out is NULL"); return FBLTS_E_ARG; }
    *out = nullptr;
    if (!members || n <= 0) { set_error("batch_create: no members"); return FBLTS_E_ARG; }
    int dev = 0;
    CK(cudaGetDevice(&dev));
    for (int i = 0; i < n; ++i) {
        const fblts_state *s = members[i];
        if (!s) { set_error("batch_create: member %d is NULL", i); return FBLTS_E_ARG; }
        for (int j = 0; j < i; ++j)
            if (members[j] == s) { set_error("batch_create: member %d repeats member %d", i, j); return FBLTS_E_ARG; }
        if (!s->arr.fp32 || !s->dm.rowS) {
            set_error("batch_create: member %d is not an FP32-tendency state on a mesh with cell rows", i);
            return FBLTS_E_ARG;
        }
        if (s->mesh->device != dev) { set_error("batch_create: member %d is on another device", i); return FBLTS_E_ARG; }
    }
    fblts_batch *b = new (std::nothrow) fblts_batch();
    if (!b) { set_error("batch_create: host allocation failed"); return FBLTS_E_OOM; }
    b->members.assign(members, members + n);
    CK(cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev));
    if (opts && opts->stream) {
        b->st = (cudaStream_t)opts->stream;
    } else {
        if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess) {
            set_error("batch_create: stream creation failed");
            delete b;
            return FBLTS_E_CUDA;
        }
        b->own_stream = true;
    }
    if (cudaEventCreate(&b->e0) != cudaSuccess || cudaEventCreate(&b->e1) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
        set_error("batch_create: event creation failed");
        fblts_batch_destroy(b);
        return FBLTS_E_CUDA;
    }
    for (int i = 0; i < n; ++i) {
        cudaStream_t x = nullptr;
        cudaEvent_t j = nullptr;
        if (cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&j, cudaEventDisableTiming) != cudaSuccess) {
            if (x) cudaStreamDestroy(x);
            set_error("batch_create: stream creation failed");
            fblts_batch_destroy(b);
            return FBLTS_E_CUDA;
        }
        b->bst.push_back(x);
        b->bjoin.push_back(j);
    }
    // each member's launching ops, in order
    std::vector<std::vector<std::pair<int, int>>> seq(n);   // (body kind, op index)
    for (int i = 0; i < n; ++i) {
        const fblts_state *s = members[i];
        for (size_t k = 0; k < s->sched.ops.size(); ++k) {
            const int bk = body_kind(s, s->sched.ops[k]);
            if (bk == -2) { set_error("batch_create: unknown op"); fblts_batch_destroy(b); return FBLTS_E_STATE; }
            if (bk >= 0) seq[i].push_back({bk, (int)k});
        }
        b->cell_updates_per_round += s->mesh->hm.cell_updates_per_step;
    }
    // merge: each launch takes the next op of every member whose next op has
    // the most common body kind (ties: lower kind); a member's ops stay in order
    auto merge = [&](const std::vector<int> &who) {
        std::vector<fblts_batch::Launch> out;
        std::vector<size_t> ptr(n, 0);
        for (;;) {
            int count[BK_COUNT] = {0};
            bool any = false;
            for (int i : who)
                if (ptr[i] < seq[i].size()) { count[seq[i][ptr[i]].first]++; any = true; }
            if (!any) break;
            const int bk = (int)(std::max_element(count, count + BK_COUNT) - count);
            fblts_batch::Launch L;
            L.bk = bk;
            for (int i : who)
                if (ptr[i] < seq[i].size() && seq[i][ptr[i]].first == bk) {
                    L.ops.push_back({i, seq[i][ptr[i]].second});
                    ptr[i]++;
                }
            out.push_back(std::move(L));
        }
        return out;
    };
    std::vector<int> everyone(n);
    std::iota(everyone.begin(), everyone.end(), 0);
    b->launches = merge(everyone);
    // groups: members with the same sequence of body kinds
    std::map<std::vector<int>, std::vector<int>> groups;
    for (int i = 0; i < n; ++i) {
        std::vector<int> sig;
        for (const auto &x : seq[i]) sig.push_back(x.first);
        groups[sig].push_back(i);
    }
    for (const auto &g : groups) {
        b->glaunches.push_back(merge(g.second));
        for (size_t k = 0; k < g.second.size(); k += 4) {
            std::vector<int> part(g.second.begin() + k, g.second.begin() + std::min(k + 4, g.second.size()));
            b->slaunches.push_back(merge(part));
        }
    }
    // launch shapes: fixed by the options, else tuned online over the candidates
    Shape fixed{opts && opts->threads_per_block ? opts->threads_per_block : 256, opts ? opts->ctas_per_sm : 0,
                opts ? opts->tile_order : 0, opts ? opts->mode : 0};
    if (fixed.tpb != 128 && fixed.tpb != 256) {
        set_error("batch_create: threads_per_block must be 128 or 256");
        fblts_batch_destroy(b);
        return FBLTS_E_ARG;
    }
    if (fixed.ctas_per_sm < 0 || fixed.ctas_per_sm > 32 || fixed.order < 0 || fixed.order > 1 || fixed.mode < 0 ||
        fixed.mode > 3) {
        set_error("batch_create: ctas_per_sm must be 0..32, tile_order 0 or 1, mode 0..3");
        fblts_batch_destroy(b);
        return FBLTS_E_ARG;
    }
    if (opts && opts->autotune) {
        for (int mode : {0, 2, 3})
            for (int tpb : {128, 256})
                for (int c : {0, 8}) b->cands.push_back(Shape{tpb, c, 0, mode});
        b->cands.push_back(Shape{256, 0, 0, 1});
    } else {
        b->tuned = true;
    }
    fblts_status st = build_round(b, b->tuned ? fixed : b->cands[0]);
    if (st != FBLTS_OK) { fblts_batch_destroy(b); return st; }
    *out = b;
    return FBLTS_OK;
}

extern "C" fblts_status fblts_batch_advance(fblts_batch *b, int64_t n) {
    if (!b || n < 0) { set_error("batch_advance: bad arguments"); return FBLTS_E_ARG; }
    if (n == 0) return FBLTS_OK;
    // the batch stream starts after the members' pending work
    for (fblts_state *s : b->members) {
        CK(cudaEventRecord(b->done, s->st));
        CK(cudaStreamWaitEvent(b->st, b->done, 0));
    }
    for (int64_t r = 0; r < n; ++r) {
        if (!b->tuned) {
            // one timed round per candidate shape (the results do not depend on it)
            const Shape &c = b->cands[b->next_cand];
            if (!(b->shape == c)) {
                fblts_status st = build_round(b, c);
                if (st != FBLTS_OK) return st;
            }
            CK(cudaEventRecord(b->e0, b->st));
            CK(cudaGraphLaunch(b->gexec, b->st));
            CK(cudaEventRecord(b->e1, b->st));
            CK(cudaEventSynchronize(b->e1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, b->e0, b->e1));
            b->cand_ms.push_back(ms);
            if (++b->next_cand == b->cands.size()) {
                const size_t best =
                    (size_t)(std::min_element(b->cand_ms.begin(), b->cand_ms.end()) - b->cand_ms.begin());
                b->tuned = true;
                fblts_status st = build_round(b, b->cands[best]);
                if (st != FBLTS_OK) return st;
            }
        } else {
            CK(cudaGraphLaunch(b->gexec, b->st));
        }
    }
    for (fblts_state *s : b->members) {
        CK(launch_check(s->arr.a[A_H], s->dm.bottom, s->mesh->hm.nC, s->arr.a[A_U], s->mesh->hm.nE, s->d_flag,
                        b->st));
        s->steps += n;
    }
    b->rounds += n;
    // the members' later calls (reads, diagnostics, advance) wait for the batch
    CK(cudaEventRecord(b->done, b->st));
    for (fblts_state *s : b->members) CK(cudaStreamWaitEvent(s->st, b->done, 0));
    return FBLTS_OK;
}

extern "C" fblts_status fblts_batch_synchronize(fblts_batch *b) {
    if (!b) { set_error("batch_synchronize: NULL batch"); return FBLTS_E_ARG; }
    CK(cudaStreamSynchronize(b->st));
    for (fblts_state *s : b->members) {
        fblts_status st = fblts_synchronize(s);
        if (st != FBLTS_OK) return st;
    }
    return FBLTS_OK;
}

extern "C" fblts_status fblts_batch_get_info(const fblts_batch *b, fblts_batch_info *info) {
    if (!b || !info) { set_error("batch_get_info: NULL argument"); return FBLTS_E_ARG; }
    std::memset(info, 0, sizeof(*info));
    info->members = (int32_t)b->members.size();
    int64_t single = 0;
    for (const fblts_state *s : b->members)
        for (const Op &op : s->sched.ops) single += body_kind(s, op) >= 0 ? 1 : 0;
    info->member_launches_per_round = single;
    int64_t grouped = 0, split = 0;
    for (const auto &g : b->glaunches) grouped += (int64_t)g.size();
    for (const auto &g : b->slaunches) split += (int64_t)g.size();
    const int64_t per_mode[4] = {(int64_t)b->launches.size(), single, grouped, split};
    info->launches_per_round = per_mode[b->shape.mode];
    info->groups = (int32_t)b->glaunches.size();
    info->cell_updates_per_round = b->cell_updates_per_round;
    info->threads_per_block = b->shape.tpb;
    info->ctas_per_sm = b->shape.ctas_per_sm;
    info->tile_order = b->shape.order;
    info->mode = b->shape.mode;
    info->tuned = b->tuned ? 1 : 0;
    info->rounds = b->rounds;
    info->n_candidates = (int32_t)std::min<size_t>(b->cands.size(), 16);
    for (size_t k = 0; k < b->cand_ms.size() && k < 16; ++k) info->candidate_ms[k] = b->cand_ms[k];
    return FBLTS_OK;
}
