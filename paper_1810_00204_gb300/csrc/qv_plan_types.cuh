// qv_plan_types.cuh -- the plan's data structures, shared by the search
// kernel (qv_tree_device.cuh), its host side (qv_tree.cu) and the adjoint
// (qv_adjoint.cu): per-episode descriptors, the device view of a plan's
// workspace, and the host handle.
#pragma once

#include <vector>

#include "qv_common.cuh"

namespace qv {

constexpr int kMaxD = QV_MAX_DEPTH;
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kLeafGroup = 4;
constexpr float kBoundaryEps = 1e-6f;
constexpr int kStamps = 4 * kMaxD + 8;
// Offset of the encoded support-window words (PlanDev::win): a bound that
// exceeds every grid coordinate, so that 0 encodes "no cell yet".
constexpr int kWinBig = 1 << 24;

struct __align__(16) EpDev {
    int H, W, P, N;          // N = H * P
    int B, goal;
    float slip, acc, eta, gamma;
    const uint16_t *cell;
    const float *cost;
    const float *Q;          // [5][N]
    const float *b0;         // [N]
    const int *beacons;      // [B] beacon cells (row * P + col)
    int range;               // Manhattan sensing range
    int band_rows, bands;
    uint32_t episode;
    int cap[kMaxD + 1];         // node capacity of each level
    int node_base[kMaxD + 1];   // gid of local node 0 of level l
    int inode_base[kMaxD + 1];  // iid of local node 0 of internal level l < d
    int pad2;
    long long belief_off[kMaxD + 1];  // float offset of stored level-l beliefs, -1 when not stored
};
static_assert(sizeof(EpDev) % 16 == 0, "EpDev is copied to smem in 16-byte words");

// The scalars the band loops read, held in registers for the duration of a
// work item (reading them from the shared-memory descriptor inside the loops
// would reload them after every shared-memory store).
struct EpReg {
    int H, W, P, N, B, goal, range;
    float slip;
    const uint16_t *cell;
    const float *cost, *Q;
};
__device__ __forceinline__ EpReg ep_reg(const EpDev &e) {
    EpReg r;
    r.H = e.H;
    r.W = e.W;
    r.P = e.P;
    r.N = e.N;
    r.B = e.B;
    r.goal = e.goal;
    r.range = e.range;
    r.slip = e.slip;
    r.cell = e.cell;
    r.cost = e.cost;
    r.Q = e.Q;
    return r;
}

struct ResultDev {
    int action;
    float value;
    float q[5];
    int pad;
};

struct GridBar {
    unsigned count;
    unsigned gen;
};

struct PlanDev {
    int E, depth, K, weight_mode, leaf_mode, Bmax, rec_len, target, n_part;
    int sb_floats, sp_floats, q_floats;  // shared-memory band buffers
    int cmax;          // children of one V-node at most: 5 min(K, Bmax + 1)
    int kslots;        // per-warp child slots of the expand phase (expand_slots)
    int n_xrec;        // per-(item, child) total records of multi-item groups
    int n_frec;        // floats of the finalize chunk records
    // the deepest fused level's contraction form (ctr_item): allowed by the
    // host (ctr), chosen per run by the work lists (c_mode[0]); work items
    // per episode as a prefix (c_items [E+1]) and each episode's first
    // total record in xrec (c_rbase [E])
    int ctr;
    int *c_items;
    int *c_rbase;
    int *c_mode;
    uint64_t seed;
    const EpDev *eps;
    float *beliefs;
    int *count;        // [(d+1)][E] nodes per level
    int *uitems;       // [(d+1)][E] update work items per node
    int *wb_upd;       // [(d+1)][E+1]
    // expand work lists of level l: one group per V-node of level l - 1 with
    // its children (at l = 0, the root of each episode), split into band
    // ranges; group j of level l sits at gbase[l] + j
    int *ngrp;         // [d] groups of level l
    int *grp_off;      // [gbase[l] + l + j]: item prefix over the level's groups (G + 1 entries)
    int *grp_rec;      // first record of a group with several items (-1: one item, totals in ntot)
    int gbase[kMaxD + 1];
    int *npre;         // [(d+1)][E+1] exclusive prefix of the level sizes over the episodes
    int *fchunks;      // [d+1] beacon chunks per node of the finalize phase
    int *wb_fin;       // [(d+1)][E+1] finalize work-list prefixes
    float *ntot;       // [NI][kTot] per internal node totals
    float *xrec;       // [n_xrec][kTot] per (item, child rank) totals
    float *frec;       // [n_frec] label-histogram records of beacon chunks
    int *wb_leaf;      // [E+1]
    // [E][4] support window of b0: the largest kWinBig - row, row + 1,
    // kWinBig - col, col + 1 over its nonzero free cells (0 = none), found by
    // the root's expand pass and cleared at the end of every run
    unsigned *win;
    // [(d+1)][E][4] per stored level: a box holding every value an earlier
    // run left in the level's belief slots, rows [w0 - 1, w1) x float4
    // groups [w2, w3); w0 = 0: the slots are zero (the stored beliefs are
    // zeroed with the counters at creation and after a failed run)
    int *dirty;
    unsigned *work;    // [2 (d+1)] items taken so far of expand(l) and finalize(l) (cleared at the end of a run)
    unsigned *grp_done;  // per group (gbase[l] + j): expand items done, deepest fused level (cleared at the end)
    int *leaf_split;   // chunks per group of leaves in the leaf phase
    unsigned *leaf_cnt;  // [n_part] chunk arrivals per group of leaves
    // per node (gid over every level)
    int *parent, *action, *obs;
    float *weight, *pz, *value;
    unsigned long long *code;
    long long *src_slot;  // slot of the node in its parent's sample arrays
    // per internal node (iid over levels < d)
    unsigned *node_cnt;
    float *R, *UQ;     // [iid][5]
    int *nchild, *choff;
    int *samples;      // [iid][5][K]
    int *slot_z, *slot_cnt;
    float *slot_P, *slot_w, *slot_val;
    int *slot_arg;     // [iid][5][K] argmax action of a fused leaf's value (Eq. 4)
    int *leaf_arg;     // per node: argmax action of a leaf's value (ties to the lowest index)
    // arrival counters and scratch
    unsigned *ep_cnt;  // [(d+1)][E]
    unsigned *lvl_cnt; // [d+1]
    float *partials;   // [n_part][rec_len]
    unsigned *status;
    unsigned long long *boundary;
    GridBar *bar;
    unsigned long long *stamps;  // [kStamps] globaltimer at phase boundaries
    ResultDev *result; // [E]
    const int *replay;
    const uint32_t *episode_word;  // nullable: episode e draws with *episode_word + e (read at each run)
    uint32_t episode0;             // params.episode: episode e's own word is episode0 + e
    unsigned long long deadline_ns;  // anytime stop, 0 = none (status[1] set when it has run out)
    unsigned spin_limit;  // polls before a wait on other CTAs gives up
    // capacities of the workspace arrays, for the bounds-checked debug build
    long long n_nodes, n_inodes, n_belief;  // node ids, internal node ids, floats of stored beliefs
    int ngrp_cap;                           // expand group entries over every level
    EpDev ep0;            // the descriptor of a one-episode plan, in parameter space
};

}  // namespace qv

// Host handle of a plan (qv_plan_t in the C ABI).
struct qv_plan;
// Writes the fused mode's leaf records after a run (no-op otherwise);
// sync_device: wait for the whole device before and after (inspection).
qv_status qv_plan_leaf_records(qv_plan *pl, cudaStream_t st, bool sync_device);
struct qv_plan {
    int E = 0;
    qv_plan_params_t params{};
    std::vector<qv::EpDev> eps;
    qv::PlanDev dev{};
    char *ws = nullptr;
    size_t bytes = 0;
    int grid = 0;
    size_t smem = 0;
    size_t reset_off = 0, reset_bytes = 0;  // counters zeroed when a run failed
    size_t read_off = 0, read_bytes = 0;    // counts, results, status, boundary: one copy back
    bool dirty = false;
    bool records_fresh = false;  // the fused mode's leaf records match the last run
    cudaGraphExec_t graph = nullptr;
};
