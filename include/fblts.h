/*
 * fblts.h - C ABI of the GB300 FB-LTS shallow-water library.
 *
 * What it computes (Lilly et al., "Local Time-Stepping for the Shallow Water
 * Equations using CFL Optimized Forward-Backward Runge-Kutta Schemes"):
 *   - the TRiSK tendencies of the rotating shallow-water equations on an
 *     unstructured Voronoi C-grid [Sec. 2.2, Eq. nonlinear_swe, Eq.
 *     semi_discrete_sys]: thickness-flux divergence [Eq. trisk_thickness],
 *     vertex potential vorticity and the nonlinear Coriolis term q F_perp
 *     [Eq. trisk_vorticity], kinetic-energy and pressure gradients, and the
 *     wind-stress / bottom-drag / surface-pressure forcing of Eq.
 *     hurricane_model;
 *   - advanced by FB-RK(3,2) [Sec. 2.1, Eq. fbrk32] inside the FB-LTS scheme
 *     [Sec. 2.2]: coarse advancement, interface prediction [Eq. preds,
 *     Eq. hstar_preds], M fine subcycles [Eq. fine_fbrk32] and interface
 *     correction [Eq. if_correction].  More than two levels are handled by
 *     nesting: each fine subcycle of a level pair is an FB-LTS step of the
 *     next pair.
 *   - optionally with the fast/slow operator splitting [Sec. 3.2] or its
 *     per-fine-step variant [Sec. 4.2]; for comparison, global FB-RK(3,2) or
 *     classical RK4 [Sec. 4.2, Tab. 2] on a one-level mesh.
 *
 * Groups of calls: mesh (create, info, and the host-only region and launch
 * planning queries), state (init, advance, I/O, diagnostics, checkpoints,
 * measurement), allocation-free diagnostics, batched ensemble, serving loop.
 *
 * Conventions common to every call:
 *   - Every function returns an fblts_status; none aborts, traps or exits.
 *     On failure fblts_last_error() returns a message (thread-local).
 *   - Index arrays are 0-based int32, -1 = absent.  Real arrays are double.
 *   - Host arrays passed in are read during the call only; the library keeps
 *     its own copies (the caller keeps ownership).  Arrays handed out are
 *     always in the caller's original cell / edge order.
 *   - A handle may be used from one host thread at a time.
 *   - Device work is issued on the stream given in fblts_params (or the
 *     library's own stream) and is asynchronous unless a function says it
 *     synchronises.
 */
#ifndef FBLTS_H
#define FBLTS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum fblts_status {
    FBLTS_OK = 0,
    FBLTS_E_ARG = 1,      /* bad argument (NULL, size, range, inconsistent counts) */
    FBLTS_E_MESH = 2,     /* connectivity or metrics invalid */
    FBLTS_E_REGIONS = 3,  /* LTS levels cannot form the required interface bands */
    FBLTS_E_OOM = 4,      /* host or device allocation failed */
    FBLTS_E_CUDA = 5,     /* a CUDA call failed (message carries the CUDA error) */
    FBLTS_E_UNSTABLE = 6, /* the state became non-finite or a thickness <= 0 */
    FBLTS_E_TIMEOUT = 7,  /* a bounded device wait gave up */
    FBLTS_E_STATE = 8     /* handle in the wrong state (e.g. checkpoint mismatch) */
} fblts_status;

typedef struct fblts_mesh fblts_mesh;
typedef struct fblts_state fblts_state;

/* Thread-local text of the last error; never NULL. */
const char *fblts_last_error(void);

/* ---------------------------------------------------------------------- */
/* Mesh                                                                    */
/* ---------------------------------------------------------------------- */

/*
 * MPAS-style mesh description (Sec. 2.2, Fig. trisk).  Sizes: nC cells,
 * nE edges, nV vertices (dual triangles, vertexDegree = 3).
 *
 *  cellsOnEdge[nE*2]      (c0, c1); the edge normal n_e points from c0 to c1;
 *                         one entry -1 marks a no-flow boundary edge (u = 0).
 *  nEdgesOnCell[nC], edgesOnCell[nC*maxEdges]  edges of each cell (any order).
 *  verticesOnEdge[nE*2]   (v0, v1) ordered so that t_e = k x n_e points from
 *                         v0 to v1 (then t_{e,v0} = -1, t_{e,v1} = +1 in
 *                         Eq. trisk_vorticity).
 *  cellsOnVertex[nV*3]    cells around each vertex (-1 = absent/land).
 *  edgesOnVertex[nV*3]    edges around each vertex; may be NULL (derived).
 *  nEdgesOnEdge[nE], edgesOnEdge[nE*maxEdges2], weightsOnEdge[nE*maxEdges2]
 *                         TRiSK tangential reconstruction: the tangential
 *                         thickness flux is F_perp_e = sum_j w_j F_{e_j}
 *                         (the dv/dc metric factor is included in w).
 *  dcEdge[nE]             distance between the two cell centres (d_e).
 *  dvEdge[nE]             length of the primal edge (l_e).
 *  areaCell[nC]           A_i.
 *  kiteAreasOnVertex[nV*3] kite of cellsOnVertex[v][j] at v; A_v is the sum
 *                         of the kites of the present cells.
 *  fVertex[nV]            Coriolis parameter at vertices.
 *  angleEdge[nE]          direction of n_e (radians from +x); needed only for
 *                         wind forcing (may be NULL otherwise).
 *  xCell,yCell[nC]        optional; used for the space-filling-curve order
 *                         and the moving vortex forcing.
 *  xEdge,yEdge[nE]        optional; needed for the vortex forcing.
 *  ltsLevel[nC]           LTS level per cell, 0 = coarsest; NULL = all 0.
 *  nLevels                number of levels (>= 1); every level must be
 *                         populated.
 *  M[nLevels-1]           M[l] = dt_l / dt_{l+1} (positive integers).
 *  nIF1Layers, nIF2Layers cell layers of the IF-1 / IF-2 bands (0 = 2, the
 *                         stencil radius of TRiSK, Sec. 2.2).
 *
 *  flags                  FBLTS_MESH_* bits (0 = none).
 *
 * Layout rules checked by fblts_mesh_create (FBLTS_E_REGIONS otherwise):
 * level l cells adjacent only to levels l-1, l, l+1, and for three or more
 * levels every level l-1 cell at least 10 + nIF1 + nIF2 + 3 cell layers (17
 * with the default bands) from every level >= l+1 cell, so that the F^5 band
 * of one level pair and the interface bands of the next stay disjoint.  With
 * FBLTS_MESH_PROMOTE_LEVELS the library enforces the separation itself: a
 * level l-1 cell closer than that to a level >= l+1 cell is moved to level l
 * (a smaller time step, so stability is kept), repeated until nothing
 * changes; fblts_mesh_levels returns the levels in use.
 */
enum { FBLTS_MESH_PROMOTE_LEVELS = 1 };
typedef struct fblts_mesh_desc {
    int32_t nCells, nEdges, nVertices, maxEdges, maxEdges2;
    const int32_t *cellsOnEdge;
    const int32_t *nEdgesOnCell;
    const int32_t *edgesOnCell;
    const int32_t *verticesOnEdge;
    const int32_t *cellsOnVertex;
    const int32_t *edgesOnVertex;
    const int32_t *nEdgesOnEdge;
    const int32_t *edgesOnEdge;
    const double *weightsOnEdge;
    const double *dcEdge;
    const double *dvEdge;
    const double *areaCell;
    const double *kiteAreasOnVertex;
    const double *fVertex;
    const double *angleEdge;
    const double *xCell, *yCell;
    const double *xEdge, *yEdge;
    const int32_t *ltsLevel;
    int32_t nLevels;
    const int32_t *M;
    int32_t nIF1Layers, nIF2Layers;
    int32_t flags;
} fblts_mesh_desc;

/* Validates, classifies the LTS regions (Sec. 2.2: F, F^1..F^5, IF-1, IF-2,
 * interior, edge ownership "closest to the fine region"), renumbers cells,
 * edges and vertices so that every region is one contiguous range, and
 * uploads the metadata to the current CUDA device.  *out receives the handle. */
fblts_status fblts_mesh_create(const fblts_mesh_desc *desc, fblts_mesh **out);
/* Frees the mesh.  Refused with FBLTS_E_STATE (the mesh stays valid) while a
 * state created on it is not destroyed or a server request naming it is not
 * taken and its server not destroyed: all of them read the mesh's device
 * tables. */
fblts_status fblts_mesh_destroy(fblts_mesh *mesh);

/* The LTS level of every cell (caller order) as the mesh uses it: ltsLevel,
 * or after the promotion of FBLTS_MESH_PROMOTE_LEVELS.  level_out[nCells]
 * is caller-owned.  Host only. */
fblts_status fblts_mesh_levels(const fblts_mesh *mesh, int32_t *level_out);

/* Counts derived by fblts_mesh_create (host only, no device work). */
typedef struct fblts_mesh_info {
    int32_t nCells, nEdges, nVertices, nLevels;
    int64_t cells_per_level[8];
    /* cell-updates per coarse step: sum_l N_l * prod_{m<l} M_m */
    int64_t cell_updates_per_step;
    /* IF-1 u IF-2 cells of each level pair */
    int64_t band_cells[8];
    /* bit 0: cell rows.  Every edgesOnEdge list is the other edges of the
     * edge's two cells and weightsOnEdge is the kite-fraction TRiSK form
     * n_{e,i} n_{e',i} (1/2 - sum of R_{i,v} from e to e') dvEdge[e'] /
     * dcEdge[e] (R_{i,v} = kite / areaCell, matched to 1e-9), so the FP32
     * path forms the TRiSK sums per cell from the cells' edge rows and kite
     * fractions; otherwise it uses the edgesOnEdge / weightsOnEdge lists */
    int32_t flags;
} fblts_mesh_info;
fblts_status fblts_mesh_get_info(const fblts_mesh *mesh, fblts_mesh_info *info);

/* Region classes of one level pair (Sec. 2.2), host only: validates and
 * classifies the mesh exactly as fblts_mesh_create does, without touching a
 * device, and writes per cell and per edge (caller order) the class relative
 * to the pair (pair, pair + 1):
 *   FBLTS_REGION_FINE (levels > pair), FBLTS_REGION_IF1, FBLTS_REGION_IF2,
 *   FBLTS_REGION_INTERIOR (the other cells of level pair),
 *   FBLTS_REGION_OUTSIDE (levels < pair);
 * and for fine elements of level pair + 1 the band b of F^b (b = ceil(D/2),
 * D the cell-layer distance to level pair; 6 when D > 10), for deeper fine
 * levels 6, else 0.  An edge takes the level of its finest cells, their
 * smallest distance to the finer level and their smallest band (an edge is in
 * F_E^b when one of its cells is in F^b).  pair in [0, nLevels - 2], else
 * FBLTS_E_ARG.  Any output pointer may be NULL; arrays are caller-owned,
 * nCells resp. nEdges int32. */
enum { FBLTS_REGION_FINE = 0, FBLTS_REGION_IF1 = 1, FBLTS_REGION_IF2 = 2, FBLTS_REGION_INTERIOR = 3,
       FBLTS_REGION_OUTSIDE = 4 };
fblts_status fblts_mesh_regions(const fblts_mesh_desc *desc, int32_t pair, int32_t *cell_class,
                                int32_t *cell_band, int32_t *edge_class, int32_t *edge_band);

/* ---------------------------------------------------------------------- */
/* State                                                                   */
/* ---------------------------------------------------------------------- */

enum { FBLTS_FP64 = 0, FBLTS_FP32_TENDENCY = 1 };
enum { FBLTS_SCHEME_FBLTS = 0, FBLTS_SCHEME_RK4 = 1 };
enum {
    FBLTS_FORCE_WIND_STRESS = 1, /* C_W |u_W - u| (u_W - u) / h, Eq. hurricane_model */
    FBLTS_FORCE_BOTTOM_DRAG = 2, /* -C_D |u| u / h */
    FBLTS_FORCE_VORTEX = 4       /* moving Holland vortex: wind + surface pressure */
};

/*
 * Run parameters.
 *  g             gravitational acceleration (m s^-2).
 *  dt            coarse time step (s) of level 0.
 *  beta[3]       FB weights of Eq. fbrk32 (the paper uses 0.531, 0.531, 0.313).
 *  precision     FBLTS_FP64: all arithmetic in double.  FBLTS_FP32_TENDENCY:
 *                tendencies and stage intermediates in float; time levels,
 *                correction sums and diagnostics in double.
 *  forcing       FBLTS_FORCE_* bits.  Wind and pressure are evaluated at the
 *                start of each coarse step and held for its stages and
 *                subcycles; drag follows the state.
 *  wind_u,wind_v uniform wind (m s^-1) added to the vortex wind.
 *  cd            bottom-drag coefficient C_D.
 *  rho0,rho_air  water and air density (kg m^-3); the wind-stress
 *                coefficient is C_W = rho_air/rho0 (0.75 + 0.067 |u_W|) 1e-3.
 *  vortex[9]     pc, dp, rmax, B, x0, y0, vx, vy, f0: pressure
 *                p = pc + dp exp(-(rmax/r)^B) around the centre
 *                (x0 + vx t, y0 + vy t), gradient wind with Coriolis f0.
 *  t0            time of the initial state (s).
 *  stream        cudaStream_t to issue work on, or NULL for an own stream.
 *  use_graph     non-zero: capture one coarse step as a CUDA graph.
 *  split         1: the fast/slow operator splitting of Sec. 3.2
 *                (Eq. splitting): inside a coarse step Phi is replaced by the
 *                pressure gradient -g grad(h + b) at the stage state plus the
 *                remaining terms (Coriolis, kinetic-energy gradient, forcing)
 *                evaluated once at the coarse step's start time level; Psi is
 *                not split.  First order in time.  split = 2: as 1, and the
 *                slow terms of the edges of every finer level are evaluated
 *                again at the start of each of that level's steps (fine
 *                cells at their current state, IF-1 at the predictions of
 *                Eq. preds), so the fine region advances its slow part with
 *                its own step; coarse edges, the interface correction
 *                included, keep the values of the coarse step's start.  This
 *                is the variant proposed at the end of Sec. 4.2.
 *  scheme        FBLTS_SCHEME_FBLTS (0): FB-LTS (Sec. 2.2; on a one-level mesh
 *                global FB-RK(3,2), Eq. fbrk32).  FBLTS_SCHEME_RK4 (1): the
 *                classical four-stage Runge-Kutta scheme, the paper's
 *                comparison integrator (Sec. 4.2, Tab. 2), advancing the unsplit
 *                tendencies of all cells with dt; it needs a one-level mesh
 *                and split = 0 (else FBLTS_E_ARG).  Wind and pressure are
 *                evaluated at the start of each step and held for its stages.
 */
typedef struct fblts_params {
    double g;
    double dt;
    double beta[3];
    int32_t precision;
    int32_t forcing;
    double wind_u, wind_v;
    double cd;
    double rho0, rho_air;
    double vortex[9];
    double t0;
    void *stream;
    int32_t use_graph;
    int32_t split;
    int32_t scheme;
} fblts_params;

/* Allocates the device state (one arena), uploads h0[nC], u0[nE] and the
 * bottom b[nC] = -H (caller order).  u0 on no-flow edges is forced to 0. */
fblts_status fblts_state_init(const fblts_mesh *mesh, const fblts_params *params,
                              const double *h0, const double *u0, const double *bottom,
                              fblts_state **out);
fblts_status fblts_state_destroy(fblts_state *state);

/* Advances n coarse steps (asynchronous).  A non-finite value or h <= 0
 * found by the end-of-call check is reported as FBLTS_E_UNSTABLE by the next
 * synchronising call. */
fblts_status fblts_lts_advance(fblts_state *state, int64_t n_coarse_steps);

/* Blocks until the state's device work is done; reports FBLTS_E_UNSTABLE. */
fblts_status fblts_synchronize(fblts_state *state);

/* Copies the state to host arrays h_out[nC], u_out[nE] (caller order; either
 * may be NULL).  Synchronises. */
fblts_status fblts_state_read(const fblts_state *state, double *h_out, double *u_out);

/* Replaces the state from host arrays h[nC], u[nE] (caller order); either may
 * be NULL to keep that field.  Copies are issued on the state's stream. */
fblts_status fblts_state_write(fblts_state *state, const double *h, const double *u);

/* End-to-end call for host callers: uploads h_in/u_in, advances n coarse
 * steps and downloads the result to h_out/u_out (all caller order, host
 * memory; pinned memory makes the copies faster).  Synchronises. */
fblts_status fblts_run_host(fblts_state *state, const double *h_in, const double *u_in,
                            int64_t n_coarse_steps, double *h_out, double *u_out);

/* Total mass sum_i A_i h_i and total absolute vorticity sum_v A_v (zeta_v + f_v)
 * (Sec. 2.3), reduced on the device in a fixed order (deterministic).
 * Synchronises. */
fblts_status fblts_diagnostics(const fblts_state *state, double *total_mass,
                               double *total_abs_vorticity);

/* Coarse steps done and the current time. */
fblts_status fblts_state_time(const fblts_state *state, int64_t *steps, double *time);

/* Checkpoint: serialises (step, time, xi, u) to buf, with xi = h + b the
 * surface elevation the state stores (caller order), so that a run resumed
 * from it is bitwise the uninterrupted run.  With buf == NULL only *len is
 * set to the size needed.  Synchronises. */
fblts_status fblts_state_save(const fblts_state *state, void *buf, size_t *len);
/* Restores a checkpoint written by fblts_state_save for the same mesh. */
fblts_status fblts_state_load(fblts_state *state, const void *buf, size_t len);

/* Device bytes that fblts_state_init will allocate for one state on `mesh`
 * in `precision` (one arena per state; host only, no device work). */
fblts_status fblts_state_device_bytes(const fblts_mesh *mesh, int32_t precision, size_t *bytes);

/* The launch list of one coarse step as fblts_state_init would build it for
 * `desc` and `params`, host only (no device): the number of schedule ops
 * (kernel launches, counting any empty range), their algorithmic bytes (the
 * model of fblts_state_step_bytes) and the cell-updates per step.  Checks the
 * mesh and the scheme/splitting arguments as fblts_mesh_create and
 * fblts_state_init do.  Any output pointer may be NULL. */
fblts_status fblts_plan_step(const fblts_mesh_desc *desc, const fblts_params *params, int64_t *ops,
                             double *alg_bytes, int64_t *cell_updates);

/* Launch statistics of one coarse step: kernels launched per step. */
fblts_status fblts_state_launches_per_step(const fblts_state *state, int64_t *launches);

/* Per-kernel profile of one coarse step: the step is issued launch by launch
 * (no graph) with a CUDA event pair around each launch on the state's
 * stream; it advances the state by one step like fblts_lts_advance(state, 1).
 * For each kind k (FBLTS_PK_*), ms[k] is the summed device time, launches[k]
 * the launch count and alg_bytes[k] the algorithmic bytes: every array element
 * the launch's arithmetic must read or write, counted once at its storage
 * size (metadata included, at its real length; see
 * fblts_state_bytes_by_kind).  Arrays have FBLTS_PROFILE_KINDS entries; any may
 * be NULL.  Synchronises.  FBLTS_PK_TRISK is the FP32 path's cell-side TRiSK
 * pass, which replaces the edge prep on meshes whose neighbour lists and
 * weights are the cells' edge rows and kite-fraction weights (mesh_info flags
 * bit 0). */
enum {
    FBLTS_PK_CELL = 0, FBLTS_PK_VERTEX, FBLTS_PK_EDGE_PREP, FBLTS_PK_EDGE, FBLTS_PK_SAVE,
    FBLTS_PK_PREDICT, FBLTS_PK_CORRECT, FBLTS_PK_FORCING, FBLTS_PK_STEP_END, FBLTS_PK_TRISK,
    FBLTS_PROFILE_KINDS
};

/* One op of the launch list that fblts_plan_step describes, host only: its
 * kind (FBLTS_PK_*), its stage (1..3; 1..4 under RK4; 0 for kinds other than
 * the cell, vertex, edge-prep, TRiSK and edge passes) and, for those passes,
 * the segment mode of every element in caller order (cells for the cell and
 * TRiSK passes, vertices for the vertex pass, edges for the edge-prep and edge
 * passes): FBLTS_SEG_NONE where the launch does not touch the element, else
 * stage value, in-place update of the time level, correction sum set / add
 * (Eq. if_correction), kinetic energy only, the slow part of Phi (Sec. 3.2),
 * or the RK4 stage modes.  mode has nCells, nVertices or nEdges bytes (NULL
 * to skip).  index in [0, ops) of fblts_plan_step, else FBLTS_E_ARG. */
enum {
    FBLTS_SEG_NONE = 0, FBLTS_SEG_STAGE, FBLTS_SEG_IN_PLACE, FBLTS_SEG_SUM_SET, FBLTS_SEG_SUM_ADD,
    FBLTS_SEG_KE_ONLY, FBLTS_SEG_TENDENCY, FBLTS_SEG_RK4_SET, FBLTS_SEG_RK4_ADD2, FBLTS_SEG_RK4_FINAL
};
fblts_status fblts_plan_op(const fblts_mesh_desc *desc, const fblts_params *params, int64_t index,
                           int32_t *kind, int32_t *stage, uint8_t *mode);
/* The algorithmic and moved bytes (the models of fblts_state_bytes_by_kind)
 * of op `index` of that launch list, host only; either pointer may be NULL. */
fblts_status fblts_plan_op_bytes(const fblts_mesh_desc *desc, const fblts_params *params, int64_t index,
                                 double *alg_bytes, double *moved_bytes);
fblts_status fblts_state_profile_step(fblts_state *state, double *ms, int64_t *launches,
                                      double *alg_bytes);

/* Algorithmic bytes of one coarse step (sum over its launches, same model as
 * fblts_state_profile_step) and cell-updates per step. */
fblts_status fblts_state_step_bytes(const fblts_state *state, double *alg_bytes,
                                    int64_t *cell_updates);

/* Bytes of one coarse step per kind (FBLTS_PROFILE_KINDS entries each; either
 * pointer may be NULL), host only:
 *   alg[k]   - algorithmic: every array the stage's arithmetic needs (Eq.
 *              trisk_thickness, Eq. trisk_vorticity, Eq. fbrk32: state, stage
 *              values, the intermediates K, q, h*, F, and the mesh metadata),
 *              each element once per launch at its storage size, metadata at
 *              its real length (no row or record padding) with the metric
 *              factors per edge and per cell; the same model as
 *              fblts_state_step_bytes and fblts_state_profile_step;
 *   moved[k] - what this library's kernels read and write in their layout:
 *              padded rows and records, per-slot coefficients, and the
 *              shares that the FP32 path's TRiSK pass writes and its edge
 *              pass reads.
 * moved / alg is the layout's overhead; DRAM traffic above moved means
 * re-reads that the caches did not catch. */
fblts_status fblts_state_bytes_by_kind(const fblts_state *state, double *alg, double *moved);

/*
 * Allocation-free global diagnostics.  The paper has no counterpart: this is
 * a service for callers that must not allocate device memory during a run,
 * for instance code that owns all device memory through its own pool, or a
 * tight driver loop where cudaMalloc / cudaFree would synchronise the device
 * and stall other work.
 *
 * Computes the total mass and total absolute vorticity of
 * fblts_diagnostics, from state arrays the caller already holds on the
 * device: d_h[nCells] and d_u[nEdges] in the caller's cell / edge order.  The
 * two results are written to the device array d_out[2] (mass, absolute
 * vorticity) on `stream` (a cudaStream_t, NULL = legacy default stream);
 * the call does not wait for them.
 *
 * The call allocates nothing.  Its scratch (one pair of partial sums per
 * block of 8192 cells) is a static device array of 64 KiB, reserved on
 * every GPU that loads the library until the process exits; it bounds the
 * mesh to at most 33,554,432 cells and vertices (FBLTS_E_ARG beyond).  The
 * first call on a device looks up the array's device address with that
 * device current; make that first call before any stream capture.  All
 * calls share the one array, and every call overwrites all the partial sums
 * it reads (nothing carries over from an earlier call), so calls that
 * overlap on the GPU race: order them on one stream or synchronise between
 * them.  The mesh's device must be current.
 *
 * The result is deterministic, but it sums in another order than
 * fblts_diagnostics (contiguous blocks of 8192 elements against a
 * grid-stride tree), so the two agree to rounding, not bit for bit: compare
 * a mass drift between calls of the same entry point.  The looked-up address
 * belongs to the device's context of that moment; after a cudaDeviceReset
 * (which also frees every mesh and state of this library) do not use the
 * library again in the same process.
 */
fblts_status fblts_diagnostics_static(const fblts_mesh *mesh, const double *d_h, const double *d_u,
                                      double *d_out, void *stream);

/*
 * Batched ensemble.  The paper advances one scenario at a time; a batch
 * advances many independent states (members, each on its own mesh, with its
 * own levels, M, forcing and dt) together.  fblts_batch_advance(b, n) leaves
 * every member as fblts_lts_advance(member, n) would: the same per-element
 * arithmetic runs, only the launches are shared (bitwise in mode 1, which
 * runs the members' own kernels; in the merged modes, whose kernels are
 * compiled separately, float multiply-adds may be contracted differently, so
 * results agree to the FP32 path's rounding).  One round
 * (one coarse FB-LTS step, Sec. 2.2, of every member) is one CUDA graph in
 * which each launch runs the next op of several members that share a kernel
 * body, as a persistent grid over their tiles.
 *
 * Members: FP32-tendency states on meshes with cell rows (mesh_info flags
 * bit 0), on the current device, each at most once; otherwise FBLTS_E_ARG.
 * The batch borrows them: do not advance a member through
 * fblts_lts_advance while the batch is in use, and destroy the batch before
 * its members.  fblts_batch_advance orders itself after the members' pending
 * work and their later calls after itself, so fblts_state_read and
 * fblts_diagnostics on a member see the batch's result.
 */
typedef struct fblts_batch fblts_batch;

typedef struct fblts_batch_opts {
    /* 1: the first 13 rounds of fblts_batch_advance each run one candidate
     * launch shape under CUDA events, then the fastest is kept: modes 0, 2, 3
     * with threads per block 128 / 256 x CTAs per SM 0 / 8 (tiles largest
     * first), then mode 1.  Those rounds advance the members like any
     * other; they synchronise the host once each. */
    int32_t autotune;
    /* without autotune: */
    int32_t threads_per_block; /* 128 or 256 (0 = 256) */
    int32_t ctas_per_sm;       /* persistent grid = this x SM count CTAs looping over the tiles,
                                * 1..32; 0 = one CTA per tile */
    int32_t tile_order;        /* 0 largest member op first, 1 member order */
    /* 0: all members merged into one chain of launches; 1: no merging, the
     * members' own launches as parallel graph branches; 2: members with the
     * same op sequence (levels and M) merged, each group a parallel branch;
     * 3: as 2 with groups of at most 4 members */
    int32_t mode;
    void *stream;              /* cudaStream_t for the batch's work; NULL = a stream of its own */
} fblts_batch_opts;

typedef struct fblts_batch_info {
    int32_t members, groups;                                   /* groups: distinct op sequences */
    int32_t threads_per_block, ctas_per_sm, tile_order, mode; /* the shape in use */
    int32_t tuned;                                             /* 1 once the shape is final */
    int64_t launches_per_round;         /* batched launches per round */
    int64_t member_launches_per_round;  /* what the members launch alone per coarse step */
    int64_t cell_updates_per_round;     /* sum over the members */
    int64_t rounds;                     /* rounds advanced so far */
    /* tuning: the candidates in the order listed under autotune and each
     * one's round time in ms (0 = not run) */
    int32_t n_candidates;
    float candidate_ms[16];
} fblts_batch_info;

fblts_status fblts_batch_create(fblts_state *const *members, int32_t n, const fblts_batch_opts *opts,
                                fblts_batch **out);
/* Advances every member by n coarse steps (asynchronous on the batch's stream,
 * except for the tuning rounds). */
fblts_status fblts_batch_advance(fblts_batch *batch, int64_t n);
/* Waits for the batch and checks every member (FBLTS_E_UNSTABLE as for
 * fblts_synchronize). */
fblts_status fblts_batch_synchronize(fblts_batch *batch);
fblts_status fblts_batch_get_info(const fblts_batch *batch, fblts_batch_info *info);
fblts_status fblts_batch_destroy(fblts_batch *batch);

/*
 * Serving loop.  The paper runs one scenario; a server runs a stream of
 * scenario requests.  Each request is an FB-LTS run (Sec. 2.2) of n_steps
 * coarse steps on a resident mesh, and its result is bitwise what
 * fblts_state_init + fblts_lts_advance(n_steps) + fblts_state_read give alone.
 *
 * Requests are admitted first come, first served while the device bytes of
 * the running and finished-but-untaken states stay within hbm_budget (and
 * at most max_active run).  Each admitted request gets its own state and
 * captured coarse step; the server issues steps_per_issue steps at a time,
 * so the running requests' work overlaps on the GPU, and a request admitted
 * while others run starts without waiting for them.  Oldest first: the k-th
 * oldest running request's steps go to a stream of the k-th highest stream
 * priority the device offers, so the GPU favours older requests and younger
 * ones take the capacity left (a request's steps stay in order).
 * fblts_server_progress does not block: call it in a loop.  The server
 * borrows the request's h0, u0, bottom until the request is admitted
 * (request_info status leaves 0), and its mesh until the request is taken
 * (fblts_server_take) or the server destroyed; fblts_mesh_destroy refuses a
 * mesh that a request still names.
 */
typedef struct fblts_server fblts_server;

typedef struct fblts_server_opts {
    uint64_t hbm_budget;     /* bytes of request states on the device at once; 0 = no limit */
    int32_t max_active;      /* running requests at once; 0 = no limit */
    int32_t steps_per_issue; /* coarse steps issued per request per progress call; 0 = 1 */
} fblts_server_opts;

typedef struct fblts_request_desc {
    const fblts_mesh *mesh;
    fblts_params params;     /* as for fblts_state_init; stream must be NULL, use_graph is forced */
    const double *h0, *u0, *bottom;   /* caller order, read at admission */
    int64_t n_steps;         /* coarse steps to run */
} fblts_request_desc;

typedef struct fblts_request_info {
    int32_t status;          /* 0 queued, 1 running, 2 done, 3 failed, 4 taken */
    int32_t error;           /* fblts_status of a failed request */
    int64_t steps_done, n_steps;
    uint64_t device_bytes;   /* of its state */
    double t_submit, t_admit, t_done;  /* seconds on the server's monotonic clock */
} fblts_request_info;

typedef struct fblts_server_stats {
    int64_t queued, running, finished, max_running;
    uint64_t device_bytes_in_use, device_bytes_peak;
    int64_t cell_updates;    /* completed, over all requests */
    double t_now;            /* seconds since fblts_server_create */
} fblts_server_stats;

fblts_status fblts_server_create(const fblts_server_opts *opts, fblts_server **out);
/* Queues a request (FBLTS_E_OOM if it alone exceeds the budget); *id names it. */
fblts_status fblts_server_submit(fblts_server *server, const fblts_request_desc *request, int64_t *id);
/* Retires finished work, issues the next steps of the running requests and
 * admits queued ones; *n_finished (may be NULL) = requests finished in this call. */
fblts_status fblts_server_progress(fblts_server *server, int32_t *n_finished);
fblts_status fblts_server_request_info(const fblts_server *server, int64_t id, fblts_request_info *info);
/* Copies a finished request's h, u (caller order; either may be NULL) and
 * frees its state; a failed request returns its error. */
fblts_status fblts_server_take(fblts_server *server, int64_t id, double *h_out, double *u_out);
fblts_status fblts_server_get_stats(const fblts_server *server, fblts_server_stats *stats);
fblts_status fblts_server_destroy(fblts_server *server);

#ifdef __cplusplus
}
#endif
#endif /* FBLTS_H */
