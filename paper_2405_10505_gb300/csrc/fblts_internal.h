// Internal declarations of the FB-LTS library (host mesh builder, schedule,
// kernels, C ABI).  Not installed; include/fblts.h is the public surface.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "fblts.h"

namespace fblts {

// ---------------------------------------------------------------- errors
void set_error(const char *fmt, ...);

// ---------------------------------------------------------------- regions
// Every cell, edge and vertex carries a band key.  Blocks run from the finest
// level to the coarsest; inside a level block the order is
//   inner distance to the next finer level (1, 2, ... capped at kin_cap),
//   then the outer band 6 - b, b = ceil(D/2) the F^b band of the distance D
//   to the next coarser level (deep cells b = 6 first, F^1 last),
//   then a locality key (space-filling curve of the owning cell).
// With this order every set used by one launch of the scheme is a contiguous
// index range (Sec. 2.2: F, F^1..F^5, IF-1, IF-2, interior).
struct BandKey {
    static uint32_t make(int L, int level, int kin, int kout) {
        return (uint32_t)((L - 1 - level) << 16) | (uint32_t)(kin << 8) | (uint32_t)kout;
    }
};

struct HostMesh {
    int nC = 0, nE = 0, nV = 0, maxE = 0, maxE2 = 0;
    int L = 1, nIF1 = 2, nIF2 = 2, kin_cap = 7;
    std::vector<int> M;

    // permutations (new index -> caller index) and inverses
    std::vector<int> cell_n2o, edge_n2o, vert_n2o;
    std::vector<int> cell_o2n, edge_o2n, vert_o2n;

    // sorted band keys in new order
    std::vector<uint32_t> ckey, ekey, vkey;
    std::vector<int> level;  // per new cell

    // connectivity in new order (row-major per element; SoA on the device)
    std::vector<int> nEoC, eoc, coc;       // [nC], [nC*maxE], [nC*maxE]
    std::vector<int> eocS;                 // eoc with the sign n_{e,i}: e (first cell) or ~e (second)
    std::vector<double> dvE, keE, invA;    // l_e, d_e l_e / 4 per edge (0 on no-flow edges); 1/A_i
    std::vector<int> coe, voe;             // [nE*2]
    std::vector<int> cov, eov;             // [nV*3]
    std::vector<int> nEoE, eoe;            // [nE], [nE*maxE2]
    std::vector<uint8_t> ebnd;             // 1 = no-flow edge
    // metrics / coefficients
    std::vector<double> cDiv, cKE;         // [nC*maxE]
    std::vector<double> cVort, cKite;      // [nV*3]
    std::vector<double> woe;               // [nE*maxE2]
    // Neighbour edges read from the two cells' edge rows (FP32 edge pass).
    // Valid when every edge's neighbours are exactly the other edges of its two
    // cells and the weights are the kite-fraction TRiSK weights: then rowE holds
    // each cell's signed edge row and rowP the prefix sums of its kite
    // fractions, padded to rowS (8 or 12) slots, and eslot packs, in 4-bit
    // fields, the edge's slot in the row of c0 and of c1 and the two row lengths.
    // rowN holds the neighbour cell across each slot's edge (the cell itself on
    // a no-flow edge) and rowV the vertex at the counter-clockwise end of the
    // slot's edge, for the cell-side TRiSK pass.
    bool rows_canonical = false;
    int rowS = 8;
    std::vector<int> rowE;                 // [nC*rowS]
    std::vector<double> rowP;              // [nC*rowS]
    std::vector<int> rowN, rowV;           // [nC*rowS]
    std::vector<uint16_t> eslot;           // [nE]
    std::vector<double> invDc, area, fV, Av;
    std::vector<double> cosE, sinE, xC, yC, xE, yE;
    bool has_angle = false, has_xy_cell = false, has_xy_edge = false;

    // counts per level and cell-updates per coarse step
    std::vector<int64_t> cells_per_level;
    int64_t cell_updates_per_step = 0;

    // range helpers: [first index with key >= k)
    int cell_lb(uint32_t k) const;
    int edge_lb(uint32_t k) const;
    int vert_lb(uint32_t k) const;
};

// builds a HostMesh from a caller description (validates, classifies, orders)
fblts_status build_host_mesh(const fblts_mesh_desc *d, HostMesh &hm);

// ---------------------------------------------------------------- arrays
// Device arrays of a state, addressed by id in the schedule.
enum Arr : int {
    A_H = 0, A_U, A_HS1, A_HS2, A_HS3, A_HST1, A_HST2, A_HST3, A_US1, A_US2, A_US3,
    A_K, A_Q, A_FE, A_QE, A_FQ, A_FQU, A_ACCH, A_ACCU,
    A_SH0, A_SH1, A_SH2, A_SH3, A_SU0, A_SU1, A_SU2, A_SU3,
    A_SLOW,   // per edge: the slow part of Phi at the coarse step's start (splitting)
    A_COUNT
};
bool arr_is_cell(int a);
bool arr_is_vert(int a);

// ---------------------------------------------------------------- schedule
enum SegMode : int {
    SEG_NONE = 0,
    SEG_UPD = 1,      // write the stage array (hs_out / us_out) and, for cells, the FB average
    SEG_INPLACE = 2,  // overwrite the state array h / u (and FB average for cells)
    SEG_ACC_SET = 3,  // correction sum: acc = tendency
    SEG_ACC_ADD = 4,  // correction sum: acc += tendency
    SEG_KONLY = 5,    // cells: kinetic energy only
    SEG_PHI = 6,      // edges: write the tendency itself (us_out = Phi)
    // classical RK4: the stage array as SEG_UPD and the weighted sum of the
    // stage tendencies in the correction-sum array (set with weight 1, add
    // with weight 2), then the step X = X + (tau/6)(sum + tendency) in place
    SEG_RK_SET = 7,
    SEG_RK_ADD2 = 8,
    SEG_RK_FIN = 9
};

struct Seg {
    int begin = 0, end = 0, mode = SEG_NONE;
};

constexpr int MAX_SEG = 6;

enum OpKind : int {
    OP_CELL = 0, OP_VERT, OP_EPREP, OP_EDGE, OP_SAVE, OP_PRED, OP_FINAL, OP_FORCING, OP_STEP_END, OP_TRISK
};

struct Op {
    int kind = OP_CELL;
    int nseg = 0;
    Seg seg[MAX_SEG];
    int lo = 0, hi = 0;               // launch covers [lo, hi)
    int stage = 1;                    // 1..3 (RK4: 1..4)
    int in_u = A_U, in_h = A_H;       // tendency arguments (u, h) of the stage
    int h0 = A_H, u0 = A_U;           // time level the stage starts from
    int hprev = A_HS2;                // stage-3 FB average uses the stage-2 h
    int out_h = A_HS1, out_u = A_US1; // stage outputs (SEG_UPD)
    int hst = A_HST1;                 // FB-averaged thickness of the stage
    double cdt = 0.0;                 // c_s * tau
    double fb_a = 0, fb_b = 0, fb_c = 0;
    // SAVE / PRED / FINAL: cell and edge ranges of IF-1 and IF-1 u IF-2
    int c_if1_lo = 0, c_if1_hi = 0, c_if12_hi = 0;
    int e_if1_lo = 0, e_if1_hi = 0, e_if12_hi = 0;
    int k = 0, Mk = 1;
    int level = 0;
    // operator splitting (Sec. 3.2): 1 = this op evaluates the slow terms at
    // the time level (no gravity term), 2 = edge stage with Phi = fast + slow
    int split = 0;
    double alg_bytes = 0.0;           // algorithmic bytes of the launch (see op_bytes)
    double moved_bytes = 0.0;         // bytes its kernel moves in this layout (see op_bytes)
};

struct Schedule {
    std::vector<Op> ops;
    int64_t launches = 0;
};

// trisk_cells: the Coriolis / tangential sums are formed per cell (OP_TRISK
// over the cells of the edge pass) instead of per edge from edge records
// (OP_EPREP over the edges and their neighbours)
// split: the operator splitting of Sec. 3.2 (a slow-term evaluation at the
// start of every coarse step, stages without the vertex / TRiSK passes);
// split = 2 also re-evaluates the slow terms of each finer level's edges at
// the start of each of its steps (the variant proposed in Sec. 4.2)
// rk4: one step of the classical four-stage RK4 on a one-level mesh instead
// of an FB-LTS coarse step (beta and split unused)
void build_schedule(const HostMesh &hm, double dt, const double beta[3], bool trisk_cells, int split, bool rk4,
                    Schedule &s);
// fills Op::alg_bytes and Op::moved_bytes of every op (forcing: the edge
// passes read the forcing fields)
void schedule_bytes(const HostMesh &hm, int forcing_flags, bool fp32, Schedule &s);

}  // namespace fblts
