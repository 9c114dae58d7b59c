// qv_tree.cu -- host side of the QV-tree search: workspace layout, plan
// creation, launch (eager or as a CUDA graph), profiling and result read-back.
// The device side (the persistent plan kernel) is in qv_tree_device.cuh.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "qv_tree_device.cuh"

// ======================================================================== host side
namespace {

struct Layout {
    size_t total = 0;
    size_t off_eps, off_count, off_uitems, off_wbu, off_wbl, off_ngrp, off_grp_off, off_grp_rec, off_npre, off_fchunks,
        off_wb_fin, off_ntot, off_xrec, off_frec, off_parent, off_action, off_obs,
        off_weight, off_pz, off_value, off_code, off_src_slot, off_node_cnt, off_R, off_UQ, off_nchild, off_choff, off_samples,
        off_slot_z, off_slot_cnt, off_slot_P, off_slot_w, off_slot_val, off_slot_arg, off_leaf_arg, off_ep_cnt, off_lvl_cnt, off_partials,
        off_leaf_split, off_leaf_cnt,
        off_status, off_boundary, off_bar, off_win, off_dirty, off_work, off_grp_done, off_stamps, off_result, off_c_items, off_c_rbase, off_c_mode,
        off_beliefs;
    long long NT = 0, NI = 0, n_belief = 0;
    int Bmax = 1, rec_len = 0, grid = 0, target = 0, n_part = 0, cmax = 0;
    long long n_xrec = 0, n_frec = 0;
    int gbase[QV_MAX_DEPTH + 1] = {};
    long long ngrp_cap = 0;  // group slots over every level
    int band_cells = 0, items_per_cta = 0;  // the launch-shape knobs in effect
    int sb_floats = 0, sp_floats = 0, q_floats = 0;
    int ctr = 0;  // the deepest fused level may take the contraction form
    size_t smem = 0;
    std::vector<qv::EpDev> eps;
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Upper bound on co-resident k_plan CTAs (8 per SM on 152 SMs).
constexpr int kMaxGridSizing = 8 * 152;
// SMs assumed when a workspace is sized without a device (GB300: 152).
constexpr int kSizingSMs = 160;

// ---- autotuner cache: shape class -> (band_cells, items_per_cta)
constexpr int kDefaultBandCells = 2048;
constexpr int kDefaultItemsPerCta = 2;
constexpr int kMaxItemsPerCta = 8;

using TuneKey = std::tuple<int, int, int, int, int, int, int, int, int>;
std::mutex g_tune_mu;
std::map<TuneKey, qv_tune_t> g_tune;

int log2_class(double v) { return v <= 1.0 ? 0 : static_cast<int>(std::ceil(std::log2(v))); }

TuneKey tune_key(int E, const qv_model_t *models, const qv_plan_params_t *p) {
    int Bmax = 1, Pmax = 1;
    double cells = 0.0;
    for (int e = 0; e < E; ++e) {
        Bmax = std::max(Bmax, models[e].num_beacons);
        Pmax = std::max(Pmax, models[e].pitch);
        cells += static_cast<double>(models[e].H) * models[e].pitch;
    }
    return TuneKey(E, p->depth, p->K, p->leaf_mode, p->weight_mode, Bmax, log2_class(Pmax), log2_class(cells / E),
                   p->grid_ctas);
}

// The knobs a plan uses: explicit values, else the cached choice for its
// shape class, else the defaults.
void resolve_tuning(int E, const qv_model_t *models, const qv_plan_params_t *p, int &bc, int &ipc) {
    bc = p->band_cells;
    ipc = p->items_per_cta;
    if (bc <= 0 || ipc <= 0) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(tune_key(E, models, p));
        if (it != g_tune.end()) {
            if (bc <= 0) bc = it->second.band_cells;
            if (ipc <= 0) ipc = it->second.items_per_cta;
        }
    }
    if (bc <= 0) bc = kDefaultBandCells;
    if (ipc <= 0) ipc = kDefaultItemsPerCta;
}

qv_status validate(int E, const qv_model_t *models, const qv_plan_params_t *p) {
    if (E < 1) return qv_set_error(QV_ERR_INVALID, "plan: E=%d", E);
    if (!models || !p) return qv_set_error(QV_ERR_INVALID, "plan: null pointer");
    if (p->depth < 0 || p->depth > QV_MAX_DEPTH) return qv_set_error(QV_ERR_INVALID, "plan: depth %d", p->depth);
    if (p->K < 1 || p->K > QV_MAX_K) return qv_set_error(QV_ERR_INVALID, "plan: K %d", p->K);
    if (p->weight_mode != QV_WEIGHT_FREQ && p->weight_mode != QV_WEIGHT_MARGINAL)
        return qv_set_error(QV_ERR_INVALID, "plan: weight_mode %d", p->weight_mode);
    if (p->leaf_mode != QV_LEAF_FUSED && p->leaf_mode != QV_LEAF_MATERIALISE)
        return qv_set_error(QV_ERR_INVALID, "plan: leaf_mode %d", p->leaf_mode);
    if (p->d_replay && E != 1) return qv_set_error(QV_ERR_INVALID, "plan: replay needs E = 1");
    if (!(p->deadline_ms >= 0.0) || p->deadline_ms > 1e12)
        return qv_set_error(QV_ERR_INVALID, "plan: deadline_ms %g", p->deadline_ms);
    if (p->deadline_ms > 0.0 && p->leaf_mode != QV_LEAF_FUSED)
        return qv_set_error(QV_ERR_INVALID, "plan: a deadline needs QV_LEAF_FUSED");
    if (p->deepest_form != QV_DEEPEST_AUTO && p->deepest_form != QV_DEEPEST_STENCIL)
        return qv_set_error(QV_ERR_INVALID, "plan: deepest_form %d", p->deepest_form);
    if (p->band_cells < 0 || p->band_cells > (1 << 16))
        return qv_set_error(QV_ERR_INVALID, "plan: band_cells %d", p->band_cells);
    if (p->items_per_cta < 0 || p->items_per_cta > kMaxItemsPerCta)
        return qv_set_error(QV_ERR_INVALID, "plan: items_per_cta %d", p->items_per_cta);
    for (int e = 0; e < E; ++e) {
        const qv_model_t &m = models[e];
        if (!m.d_cell) return qv_set_error(QV_ERR_INVALID, "plan: episode %d has no cell words", e);
        if (!m.d_beacons || m.sense_range < 0)
            return qv_set_error(QV_ERR_INVALID, "plan: episode %d needs its beacon cells and range", e);
        if (m.H < 1 || m.W < 1 || m.W > QV_MAX_WIDTH || m.pitch != QV_PITCH(m.W))
            return qv_set_error(QV_ERR_INVALID, "plan: episode %d grid %dx%d pitch %d", e, m.H, m.W, m.pitch);
        if (m.num_beacons < 1 || m.num_beacons > QV_MAX_BEACONS)
            return qv_set_error(QV_ERR_INVALID, "plan: episode %d B=%d", e, m.num_beacons);
        if (m.goal < 0 || m.goal >= m.H * m.pitch || m.goal % m.pitch >= m.W)
            return qv_set_error(QV_ERR_INVALID, "plan: episode %d goal %d", e, m.goal);
        if (!(m.slip >= 0.f && m.slip <= 0.5f) || !(m.accuracy > 0.f && m.accuracy <= 1.f) ||
            !(m.discount > 0.f && m.discount < 1.f))
            return qv_set_error(QV_ERR_INVALID, "plan: episode %d slip/accuracy/discount out of range", e);
        // path code: (5 (B+1))^d * 5 must stay below 2^56 for the Philox counter
        double code = 5.0;
        for (int l = 0; l < p->depth; ++l) code *= 5.0 * (m.num_beacons + 1);
        if (code >= 72057594037927936.0)
            return qv_set_error(QV_ERR_INVALID, "plan: depth %d with B=%d overflows the path code", p->depth,
                                m.num_beacons);
    }
    return QV_OK;
}

// The largest dynamic shared memory k_plan has been allowed on each device.
// The attribute belongs to the kernel, not to a plan, so it only ever grows:
// lowering it for a plan with small bands would make an earlier plan's
// launch (or graph) with larger bands fail.
std::mutex g_smem_mu;
constexpr int kMaxDevices = 64;
size_t g_smem_attr[kMaxDevices] = {};

bool allow_smem(size_t smem) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return false;
    std::lock_guard<std::mutex> lk(g_smem_mu);
    if (smem <= g_smem_attr[dev]) return true;
    if (cudaFuncSetAttribute(qv::k_plan, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) !=
        cudaSuccess)
        return false;
    g_smem_attr[dev] = smem;
    return true;
}

// Co-resident CTAs of k_plan for a given dynamic smem size (0 when it does
// not fit or there is no device).
int plan_grid(size_t smem) {
    int per_sm = 0;
    if (!allow_smem(smem) ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, qv::k_plan, qv::kThreads, smem) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        return 0;
    }
    return per_sm * qv_num_sms();
}

qv_status make_layout(int E, const qv_model_t *models, const qv_plan_params_t *p, Layout &L, bool need_grid) {
    qv_status st = validate(E, models, p);
    if (st != QV_OK) return st;
    const int D = p->depth, K = p->K;
    L.eps.assign(E, qv::EpDev{});
    resolve_tuning(E, models, p, L.band_cells, L.items_per_cta);
    L.Bmax = 1;
    for (int e = 0; e < E; ++e) L.Bmax = std::max(L.Bmax, models[e].num_beacons);
    long long NB[QV_MAX_DEPTH + 1] = {};
    for (int e = 0; e < E; ++e) {
        const qv_model_t &m = models[e];
        qv::EpDev &ep = L.eps[e];
        ep.H = m.H;
        ep.W = m.W;
        ep.P = m.pitch;
        ep.N = m.H * m.pitch;
        ep.B = m.num_beacons;
        ep.goal = m.goal;
        ep.slip = m.slip;
        ep.acc = m.accuracy;
        ep.eta = (1.0f - m.accuracy) / static_cast<float>(m.num_beacons);
        ep.gamma = m.discount;
        ep.cell = m.d_cell;
        ep.cost = m.d_cost;
        ep.beacons = m.d_beacons;
        ep.range = m.sense_range;
        ep.episode = p->episode + static_cast<uint32_t>(e);
        ep.band_rows = std::max(1, std::min(m.H, L.band_cells / m.pitch));
        ep.bands = (m.H + ep.band_rows - 1) / ep.band_rows;
        const long long br = std::min<long long>(K, m.num_beacons + 1) * 5;
        long long c = 1;
        for (int l = 0; l <= D; ++l) {
            if (c > (1LL << 30)) return qv_set_error(QV_ERR_INVALID, "plan: level %d capacity overflow", l);
            ep.cap[l] = static_cast<int>(c);
            NB[l] += c;
            c *= br;
        }
        if (p->leaf_mode == QV_LEAF_MATERIALISE && D > 0)  // the update phase's node band
            L.sb_floats = std::max(L.sb_floats, (ep.band_rows + 2) * ep.P);
        L.sp_floats = std::max(L.sp_floats, (ep.band_rows + 4) * ep.P);
        if (p->leaf_mode == QV_LEAF_FUSED && D > 0) L.q_floats = std::max(L.q_floats, 5 * ep.band_rows * ep.P);
    }
    L.cmax = 5 * std::min(K, L.Bmax + 1);
    // the contraction form of the deepest fused level works in the band
    // buffers: grow the Q buffer until they hold its arrays
    L.ctr = (p->leaf_mode == QV_LEAF_FUSED && D >= 2 && p->deepest_form == QV_DEEPEST_AUTO) ? 1 : 0;
    if (L.ctr) {
        const qv::SmemLayout s0 =
            qv::SmemLayout::make(L.sb_floats, L.sp_floats, L.q_floats, L.Bmax, K, L.cmax, qv::expand_slots(L.cmax));
        const size_t need = sizeof(float) * static_cast<size_t>(qv::ctr_layout().total) + 64;
        if (s0.band_end - s0.sb < need) L.q_floats += static_cast<int>((need - (s0.band_end - s0.sb)) / sizeof(float)) + 16;
    }
    L.smem = qv::SmemLayout::make(L.sb_floats, L.sp_floats, L.q_floats, L.Bmax, K, L.cmax, qv::expand_slots(L.cmax))
                 .total;
    if (L.smem > 200 * 1024) return qv_set_error(QV_ERR_INVALID, "plan: %zu bytes of shared memory", L.smem);
    L.grid = need_grid ? plan_grid(L.smem) : 0;
    if (need_grid && L.grid < 1) return qv_set_error(QV_ERR_CUDA, "plan: k_plan does not fit an SM");
    if (p->grid_ctas < 0) return qv_set_error(QV_ERR_INVALID, "plan: grid_ctas %d", p->grid_ctas);
    if (need_grid && p->grid_ctas > 0) L.grid = std::min(L.grid, p->grid_ctas);
    // work items per phase aimed at: two per co-resident CTA.  Band splits
    // keep every phase below 2 * target items, and the partial records are
    // sized for the largest possible grid so that sizing needs no device.
    L.target = L.items_per_cta * std::max(L.grid, 1);
    L.n_part = 2 * L.items_per_cta * kMaxGridSizing;
    // per-(item, child) totals of groups with several items (those items
    // number at most twice the target) and the beacon-chunk records of the
    // finalize phase (several chunks per node only when a level's nodes
    // times its chunks stay within the target, two or more chunks each);
    // sized for the largest grid so that sizing needs no device
    const long long per_sm = std::max<long long>(1, std::min<long long>(8, (228 * 1024) / std::max<size_t>(L.smem, 1)));
    const long long tmax = static_cast<long long>(L.items_per_cta) * kSizingSMs * per_sm;
    L.n_xrec = 2 * tmax * L.cmax;
    // the contraction form's records: its items are cut at two per CTA
    // whatever items_per_cta is, each with a record per child of its episode
    if (L.ctr) L.n_xrec = std::max<long long>(L.n_xrec, 12LL * kSizingSMs * per_sm * L.cmax);
    L.n_frec = tmax * 30 * ((L.Bmax + 1) / 2) + 30LL * L.Bmax;
    long long gbase = 0, ibase = 0;
    long long run_g[QV_MAX_DEPTH + 1], run_i[QV_MAX_DEPTH + 1];
    for (int l = 0; l <= D; ++l) {
        run_g[l] = gbase;
        gbase += NB[l];
        run_i[l] = ibase;
        if (l < D) ibase += NB[l];
    }
    L.NT = gbase;
    L.NI = std::max<long long>(ibase, 1);
    // expand groups of level l: the roots at l = 0, else the V-nodes of level l - 1
    L.ngrp_cap = 0;
    for (int l = 0; l <= D; ++l) {
        L.gbase[l] = static_cast<int>(L.ngrp_cap);
        L.ngrp_cap += l == 0 ? E : NB[l - 1];
    }
    if (L.ngrp_cap > (1LL << 30)) return qv_set_error(QV_ERR_INVALID, "plan: tree too large");
    if (L.NT > (1LL << 31) - 1 || L.NI * 5 * K > (1LL << 40))
        return qv_set_error(QV_ERR_INVALID, "plan: tree too large");
    const bool mat = p->leaf_mode == QV_LEAF_MATERIALISE || D == 0;
    L.n_belief = 0;
    for (int l = 0; l <= D; ++l)
        for (int e = 0; e < E; ++e) {
            qv::EpDev &ep = L.eps[e];
            ep.node_base[l] = static_cast<int>(run_g[l]);
            run_g[l] += ep.cap[l];
            if (l < D) {
                ep.inode_base[l] = static_cast<int>(run_i[l]);
                run_i[l] += ep.cap[l];
            } else {
                ep.inode_base[l] = -1;
            }
            // stored when a later phase reads them back
            const bool store = (l >= 1) && (l < D - 1 || (mat && l <= D));
            if (store) {
                ep.belief_off[l] = L.n_belief;
                L.n_belief += static_cast<long long>(ep.cap[l]) * ep.N;
            } else {
                ep.belief_off[l] = -1;
            }
        }
    L.rec_len = qv::kLeafGroup * 5;  // the leaf phase's chunk records
    size_t o = 0;
    auto take = [&](size_t bytes) {
        o = align_up(o, 256);
        const size_t r = o;
        o += bytes;
        return r;
    };
    const long long E1 = E + 1, D1 = D + 1;
    L.off_eps = take(sizeof(qv::EpDev) * E);
    L.off_uitems = take(sizeof(int) * D1 * E);
    L.off_wbu = take(sizeof(int) * D1 * E1);
    L.off_ngrp = take(sizeof(int) * D1);
    L.off_grp_off = take(sizeof(int) * (L.ngrp_cap + D1));
    L.off_grp_rec = take(sizeof(int) * L.ngrp_cap);
    L.off_npre = take(sizeof(int) * D1 * E1);
    L.off_fchunks = take(sizeof(int) * D1);
    L.off_wb_fin = take(sizeof(int) * D1 * E1);
    L.off_c_items = take(sizeof(int) * E1);
    L.off_c_rbase = take(sizeof(int) * E1);
    L.off_c_mode = take(sizeof(int));
    L.off_ntot = take(sizeof(float) * L.NI * qv::kTot);
    L.off_xrec = take(sizeof(float) * L.n_xrec * qv::kTot);
    L.off_frec = take(sizeof(float) * L.n_frec);
    L.off_wbl = take(sizeof(int) * E1);
    L.off_leaf_split = take(sizeof(int));
    L.off_parent = take(sizeof(int) * L.NT);
    L.off_action = take(sizeof(int) * L.NT);
    L.off_obs = take(sizeof(int) * L.NT);
    L.off_weight = take(sizeof(float) * L.NT);
    L.off_pz = take(sizeof(float) * L.NT);
    L.off_value = take(sizeof(float) * L.NT);
    L.off_code = take(sizeof(unsigned long long) * L.NT);
    L.off_src_slot = take(sizeof(long long) * L.NT);
    L.off_R = take(sizeof(float) * L.NI * 5);
    L.off_UQ = take(sizeof(float) * L.NI * 5);
    L.off_nchild = take(sizeof(int) * L.NI * 5);
    L.off_choff = take(sizeof(int) * L.NI * 5);
    L.off_samples = take(sizeof(int) * L.NI * 5 * K);
    L.off_slot_z = take(sizeof(int) * L.NI * 5 * K);
    L.off_slot_cnt = take(sizeof(int) * L.NI * 5 * K);
    L.off_slot_P = take(sizeof(float) * L.NI * 5 * K);
    L.off_slot_w = take(sizeof(float) * L.NI * 5 * K);
    L.off_slot_val = take(sizeof(float) * L.NI * 5 * K);
    L.off_slot_arg = take(sizeof(int) * L.NI * 5 * K);
    L.off_leaf_arg = take(sizeof(int) * L.NT);
    L.off_partials = take(sizeof(float) * static_cast<size_t>(L.n_part) * L.rec_len);
    L.off_stamps = take(sizeof(unsigned long long) * qv::kStamps);
    // what qv_plan_read copies back, contiguous: level sizes, root results,
    // then (first in the zeroed region) the status word and boundary count
    L.off_count = take(sizeof(int) * D1 * E);
    L.off_result = take(sizeof(qv::ResultDev) * E);
    // counters and status words: one contiguous region, zeroed at create
    L.off_status = take(sizeof(unsigned) * 8);
    L.off_boundary = take(sizeof(unsigned long long));
    L.off_node_cnt = take(sizeof(unsigned) * L.NI);
    L.off_ep_cnt = take(sizeof(unsigned) * D1 * E);
    L.off_lvl_cnt = take(sizeof(unsigned) * D1);
    L.off_leaf_cnt = take(sizeof(unsigned) * static_cast<size_t>(L.n_part));
    L.off_bar = take(sizeof(qv::GridBar));
    L.off_win = take(sizeof(unsigned) * 4 * E);
    L.off_dirty = take(sizeof(int) * 4 * E * D1);
    L.off_work = take(sizeof(unsigned) * 2 * D1);
    L.off_grp_done = take(sizeof(unsigned) * std::max<long long>(L.ngrp_cap, 1));
    L.off_beliefs = take(sizeof(float) * std::max<long long>(L.n_belief, 4));
    L.total = align_up(o, 256);
    return QV_OK;
}

template <typename T>
T *at(char *ws, size_t off) {
    return reinterpret_cast<T *>(ws + off);
}

qv_status launch_plan(qv_plan_t *pl, cudaStream_t st) {
    pl->dev.spin_limit = qv_cross_spin_limit();
    pl->records_fresh = false;
    if (pl->dirty) {
        if (qv_check_cuda(cudaMemsetAsync(pl->ws + pl->reset_off, 0, pl->reset_bytes, st), "counter reset") != QV_OK)
            return QV_ERR_CUDA;
        pl->dirty = false;
    }
    // per-run status word and boundary count (adjacent: one memset)
    const size_t sb_bytes = reinterpret_cast<char *>(pl->dev.boundary + 1) - reinterpret_cast<char *>(pl->dev.status);
    if (qv_check_cuda(cudaMemsetAsync(pl->dev.status, 0, sb_bytes, st), "status reset") != QV_OK) return QV_ERR_CUDA;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(pl->grid);
    cfg.blockDim = dim3(qv::kThreads);
    cfg.dynamicSmemBytes = pl->smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
#ifdef QV_BOUNDS_CHECK
    const unsigned inject = qv_bounds_injected_site();
    if (qv_check_cuda(cudaMemcpyToSymbolAsync(qv::g_bounds_inject, &inject, sizeof(inject), 0,
                                              cudaMemcpyHostToDevice, st),
                      "bounds injection") != QV_OK)
        return QV_ERR_CUDA;
    if (qv_check_cuda(cudaLaunchKernelEx(&cfg, qv::k_plan, pl->dev), "k_plan launch") != QV_OK) return QV_ERR_CUDA;
    qv::k_bounds_collect<<<1, 1, 0, st>>>(pl->dev.status);
    return qv_check_cuda(cudaGetLastError(), "k_bounds_collect launch");
#else
    return qv_check_cuda(cudaLaunchKernelEx(&cfg, qv::k_plan, pl->dev), "k_plan launch");
#endif
}

}  // namespace

extern "C" size_t qv_plan_workspace_bytes(int32_t E, const qv_model_t *models, const qv_plan_params_t *params) {
    Layout L;
    if (make_layout(E, models, params, L, false) != QV_OK) return 0;
    return L.total;
}

extern "C" qv_status qv_plan_create(int32_t E, const qv_model_t *models, const float *const *d_Q,
                                    const float *const *d_b0, const qv_plan_params_t *params, void *d_ws,
                                    size_t ws_bytes, qv_plan_t **plan_out, qv_stream_t stream) {
    QV_RANGE("qv_plan_create");
    if (const qv_status inj = qv_injected_fault("qv_plan_create", true)) return inj;
    if (!plan_out || !d_Q || !d_b0 || !d_ws) return qv_set_error(QV_ERR_INVALID, "qv_plan_create: null pointer");
    *plan_out = nullptr;
    Layout L;
    qv_status st = make_layout(E, models, params, L, true);
    if (st != QV_OK) return st;
    if (ws_bytes < L.total)
        return qv_set_error(QV_ERR_WORKSPACE, "qv_plan_create: workspace %zu < %zu bytes", ws_bytes, L.total);
    if (reinterpret_cast<uintptr_t>(d_ws) & 255)
        return qv_set_error(QV_ERR_INVALID, "qv_plan_create: workspace must be 256-byte aligned");
    for (int e = 0; e < E; ++e) {
        if (!d_Q[e] || !d_b0[e]) return qv_set_error(QV_ERR_INVALID, "qv_plan_create: episode %d null Q/b0", e);
        if ((reinterpret_cast<uintptr_t>(d_Q[e]) | reinterpret_cast<uintptr_t>(d_b0[e])) & 15)
            return qv_set_error(QV_ERR_INVALID, "qv_plan_create: episode %d Q/b0 not 16-byte aligned", e);
        if (models[e].d_cost && (reinterpret_cast<uintptr_t>(models[e].d_cost) & 15))
            return qv_set_error(QV_ERR_INVALID, "qv_plan_create: episode %d cost not 16-byte aligned", e);
        if (reinterpret_cast<uintptr_t>(models[e].d_cell) & 15)
            return qv_set_error(QV_ERR_INVALID, "qv_plan_create: episode %d cell words not 16-byte aligned", e);
        L.eps[e].Q = d_Q[e];
        L.eps[e].b0 = d_b0[e];
    }
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    qv_plan_t *pl = new qv_plan_t;
    pl->E = E;
    pl->params = *params;
    pl->eps = L.eps;
    pl->ws = static_cast<char *>(d_ws);
    pl->bytes = L.total;
    pl->grid = L.grid;
    pl->smem = L.smem;
    pl->params.band_cells = L.band_cells;
    pl->params.items_per_cta = L.items_per_cta;
    pl->dev.sb_floats = L.sb_floats;
    pl->dev.sp_floats = L.sp_floats;
    pl->dev.q_floats = L.q_floats;
    char *ws = pl->ws;
    qv::PlanDev &d = pl->dev;
    d.E = E;
    d.depth = params->depth;
    d.K = params->K;
    d.weight_mode = params->weight_mode;
    d.leaf_mode = params->leaf_mode;
    d.Bmax = L.Bmax;
    d.rec_len = L.rec_len;
    d.target = L.target;
    d.n_part = L.n_part;
    d.seed = params->seed;
    d.eps = at<qv::EpDev>(ws, L.off_eps);
    d.beliefs = at<float>(ws, L.off_beliefs);
    d.count = at<int>(ws, L.off_count);
    d.uitems = at<int>(ws, L.off_uitems);
    d.wb_upd = at<int>(ws, L.off_wbu);
    d.cmax = L.cmax;
    d.kslots = qv::expand_slots(L.cmax);
    d.n_xrec = static_cast<int>(std::min<long long>(L.n_xrec, (1LL << 31) - 1));
    d.n_frec = static_cast<int>(std::min<long long>(L.n_frec, (1LL << 31) - 1));
    d.ngrp = at<int>(ws, L.off_ngrp);
    d.grp_off = at<int>(ws, L.off_grp_off);
    d.grp_rec = at<int>(ws, L.off_grp_rec);
    for (int l = 0; l <= params->depth; ++l) d.gbase[l] = L.gbase[l];
    d.npre = at<int>(ws, L.off_npre);
    d.fchunks = at<int>(ws, L.off_fchunks);
    d.wb_fin = at<int>(ws, L.off_wb_fin);
    d.ctr = L.ctr;
    d.c_items = at<int>(ws, L.off_c_items);
    d.c_rbase = at<int>(ws, L.off_c_rbase);
    d.c_mode = at<int>(ws, L.off_c_mode);
    d.ntot = at<float>(ws, L.off_ntot);
    d.xrec = at<float>(ws, L.off_xrec);
    d.frec = at<float>(ws, L.off_frec);
    d.wb_leaf = at<int>(ws, L.off_wbl);
    d.leaf_split = at<int>(ws, L.off_leaf_split);
    d.leaf_cnt = at<unsigned>(ws, L.off_leaf_cnt);
    d.parent = at<int>(ws, L.off_parent);
    d.action = at<int>(ws, L.off_action);
    d.obs = at<int>(ws, L.off_obs);
    d.weight = at<float>(ws, L.off_weight);
    d.pz = at<float>(ws, L.off_pz);
    d.value = at<float>(ws, L.off_value);
    d.code = at<unsigned long long>(ws, L.off_code);
    d.src_slot = at<long long>(ws, L.off_src_slot);
    d.node_cnt = at<unsigned>(ws, L.off_node_cnt);
    d.R = at<float>(ws, L.off_R);
    d.UQ = at<float>(ws, L.off_UQ);
    d.nchild = at<int>(ws, L.off_nchild);
    d.choff = at<int>(ws, L.off_choff);
    d.samples = at<int>(ws, L.off_samples);
    d.slot_z = at<int>(ws, L.off_slot_z);
    d.slot_cnt = at<int>(ws, L.off_slot_cnt);
    d.slot_P = at<float>(ws, L.off_slot_P);
    d.slot_w = at<float>(ws, L.off_slot_w);
    d.slot_val = at<float>(ws, L.off_slot_val);
    d.slot_arg = at<int>(ws, L.off_slot_arg);
    d.leaf_arg = at<int>(ws, L.off_leaf_arg);
    d.ep_cnt = at<unsigned>(ws, L.off_ep_cnt);
    d.lvl_cnt = at<unsigned>(ws, L.off_lvl_cnt);
    d.partials = at<float>(ws, L.off_partials);
    d.status = at<unsigned>(ws, L.off_status);
    d.boundary = at<unsigned long long>(ws, L.off_boundary);
    d.bar = at<qv::GridBar>(ws, L.off_bar);
    d.win = at<unsigned>(ws, L.off_win);
    d.dirty = at<int>(ws, L.off_dirty);
    d.work = at<unsigned>(ws, L.off_work);
    d.grp_done = at<unsigned>(ws, L.off_grp_done);
    d.stamps = at<unsigned long long>(ws, L.off_stamps);
    d.result = at<qv::ResultDev>(ws, L.off_result);
    d.replay = params->d_replay;
    d.episode_word = nullptr;
    d.episode0 = params->episode;
    d.deadline_ns = params->deadline_ms > 0.0
                        ? std::max<unsigned long long>(1ull, static_cast<unsigned long long>(params->deadline_ms * 1e6))
                        : 0ull;
    d.n_nodes = L.NT;
    d.n_inodes = L.NI;
    d.n_belief = L.n_belief;
    d.ngrp_cap = static_cast<int>(L.ngrp_cap);
    d.ep0 = L.eps[0];
    pl->reset_off = L.off_status;
    // the stored beliefs too: the kernel writes zeros only where an earlier
    // run may have left values (PlanDev::dirty), so the region starts zeroed
    // and is zeroed again after a failed run
    pl->reset_bytes = L.off_beliefs + sizeof(float) * static_cast<size_t>(std::max<long long>(L.n_belief, 4)) -
                      L.off_status;
    pl->read_off = L.off_count;
    pl->read_bytes = L.off_boundary + sizeof(unsigned long long) - L.off_count;
    // static state: descriptors, the root of every episode, level-0 work lists
    const int D = params->depth;
    std::vector<int> cnt0(E, 1), it0(E), wbu(E + 1), wbl(E + 1), neg(E, -1), goff(E + 1), grec(E), npre(E + 1),
        wbf(E + 1);
    std::vector<float> one(E, 1.0f);
    std::vector<unsigned long long> zero64(E, 0ull);
    int s0 = 0, l0 = 0, g0 = 0, r0 = 0;
    // a depth-0 plan streams each root as one leaf, split into leaf0_split chunks
    const int leaf0_split = static_cast<int>(std::min<long long>(std::max<long long>(L.target / E, 1), 64));
    const int fch0 = qv::finalize_chunks(E, L.target, L.Bmax);
    for (int e = 0; e < E; ++e) {
        const long long want = std::max<long long>(L.target / E, 1);
        it0[e] = static_cast<int>(std::min<long long>(std::max<long long>(want, 1), L.eps[e].bands));
        wbu[e] = s0;
        s0 += D > 0 ? it0[e] : 0;
        wbl[e] = l0;
        l0 += leaf0_split;
        // level 0's expand group of episode e: its root alone
        const int gi = D > 0 ? qv::group_items(1, E, L.target, L.eps[e].bands) : 0;
        goff[e] = g0;
        g0 += gi;
        grec[e] = gi >= 2 ? r0 : -1;
        r0 += gi >= 2 ? gi : 0;
        npre[e] = e;
        wbf[e] = e * fch0;
    }
    wbu[E] = s0;
    wbl[E] = l0;
    goff[E] = g0;
    npre[E] = E;
    wbf[E] = E * fch0;
    const int ngrp0 = E;
    auto up = [&](void *dst, const void *src, size_t bytes) {
        return qv_check_cuda(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, cs), "plan upload");
    };
    // root gids are 0..E-1 (level 0 is first in the node id space)
    if (up(const_cast<qv::EpDev *>(d.eps), L.eps.data(), sizeof(qv::EpDev) * E) != QV_OK ||
        up(d.count, cnt0.data(), sizeof(int) * E) != QV_OK || up(d.uitems, it0.data(), sizeof(int) * E) != QV_OK ||
        up(d.wb_upd, wbu.data(), sizeof(int) * (E + 1)) != QV_OK ||
        up(d.ngrp, &ngrp0, sizeof(int)) != QV_OK ||
        up(d.grp_off + d.gbase[0], goff.data(), sizeof(int) * (E + 1)) != QV_OK ||
        up(d.grp_rec + d.gbase[0], grec.data(), sizeof(int) * E) != QV_OK ||
        up(d.npre, npre.data(), sizeof(int) * (E + 1)) != QV_OK || up(d.fchunks, &fch0, sizeof(int)) != QV_OK ||
        up(d.wb_fin, wbf.data(), sizeof(int) * (E + 1)) != QV_OK ||
        up(d.wb_leaf, wbl.data(), sizeof(int) * (E + 1)) != QV_OK ||
        up(d.leaf_split, &leaf0_split, sizeof(int)) != QV_OK ||
        up(d.parent, neg.data(), sizeof(int) * E) != QV_OK || up(d.action, neg.data(), sizeof(int) * E) != QV_OK ||
        up(d.obs, neg.data(), sizeof(int) * E) != QV_OK || up(d.weight, one.data(), sizeof(float) * E) != QV_OK ||
        up(d.pz, one.data(), sizeof(float) * E) != QV_OK ||
        up(d.code, zero64.data(), sizeof(unsigned long long) * E) != QV_OK ||
        qv_check_cuda(cudaMemsetAsync(ws + pl->reset_off, 0, pl->reset_bytes, cs), "counter reset") != QV_OK ||
        qv_check_cuda(cudaStreamSynchronize(cs), "plan upload") != QV_OK) {
        delete pl;
        return QV_ERR_CUDA;
    }
    *plan_out = pl;
    return QV_OK;
}

extern "C" qv_status qv_plan_set_episode_word(qv_plan_t *pl, const uint32_t *d_word) {
    if (!pl) return qv_set_error(QV_ERR_INVALID, "qv_plan_set_episode_word: null plan");
    if (reinterpret_cast<uintptr_t>(d_word) & 3)
        return qv_set_error(QV_ERR_INVALID, "qv_plan_set_episode_word: word not 4-byte aligned");
    pl->dev.episode_word = d_word;
    if (pl->graph) {  // the captured launch holds the old parameters
        cudaGraphExecDestroy(pl->graph);
        pl->graph = nullptr;
    }
    return QV_OK;
}

extern "C" qv_status qv_plan_run(qv_plan_t *pl, qv_stream_t stream) {
    QV_RANGE("qv_plan_run");
    if (const qv_status inj = qv_injected_fault("qv_plan_run", false)) return inj;
    if (!pl) return qv_set_error(QV_ERR_INVALID, "qv_plan_run: null plan");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    pl->records_fresh = false;
    if (pl->graph && !pl->dirty) return qv_check_cuda(cudaGraphLaunch(pl->graph, st), "qv_plan_run graph launch");
    return launch_plan(pl, st);
}

extern "C" qv_status qv_plan_profile(qv_plan_t *pl, qv_launch_time_t *out, int32_t max_launches, int32_t *n_out,
                                     qv_stream_t stream) {
    QV_RANGE("qv_plan_profile");
    if (!pl || !out || !n_out || max_launches < 0)
        return qv_set_error(QV_ERR_INVALID, "qv_plan_profile: bad argument");
    *n_out = 0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (qv_check_cuda(cudaEventCreate(&e0), "event") != QV_OK) return QV_ERR_CUDA;
    if (qv_check_cuda(cudaEventCreate(&e1), "event") != QV_OK) {
        cudaEventDestroy(e0);
        return QV_ERR_CUDA;
    }
    qv_status s = qv_check_cuda(cudaMemsetAsync(pl->dev.stamps, 0, sizeof(unsigned long long) * qv::kStamps, st),
                                "stamp reset");
    if (s == QV_OK) s = qv_check_cuda(cudaEventRecord(e0, st), "event");
    if (s == QV_OK) s = launch_plan(pl, st);
    if (s == QV_OK) s = qv_check_cuda(cudaEventRecord(e1, st), "event");
    unsigned long long stamps[qv::kStamps] = {};
    if (s == QV_OK)
        s = qv_check_cuda(cudaMemcpyAsync(stamps, pl->dev.stamps, sizeof(stamps), cudaMemcpyDeviceToHost, st),
                          "stamps");
    if (s == QV_OK) s = qv_check_cuda(cudaStreamSynchronize(st), "qv_plan_profile");
    int n = 0;
    if (s == QV_OK && max_launches > 0) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        std::memset(&out[0], 0, sizeof(out[0]));
        std::snprintf(out[0].name, sizeof(out[0].name), "k_plan");
        out[0].level = -1;
        out[0].ms = ms;
        n = 1;
        // phase durations from the device clock, in execution order
        const int D = pl->params.depth;
        const bool mat = pl->params.leaf_mode == QV_LEAF_MATERIALISE;
        struct Ph {
            const char *name;
            int level;
        };
        std::vector<Ph> ph;
        // one phase per level: its expand and finalize items
        for (int l = 0; l < D; ++l) ph.push_back({(l == D - 1 && !mat) ? "fused" : "level", l});
        if (D > 0 && mat) ph.push_back({"update", D - 1});
        if (D == 0 || mat) ph.push_back({"leaf", D});
        if (D > 0) ph.push_back({"backup", 0});
        for (size_t i = 0; i < ph.size() && n < max_launches && i + 1 < static_cast<size_t>(qv::kStamps); ++i) {
            std::memset(&out[n], 0, sizeof(out[n]));
            std::snprintf(out[n].name, sizeof(out[n].name), "phase:%s", ph[i].name);
            out[n].level = ph[i].level;
            out[n].ms = stamps[i + 1] > stamps[i] ? static_cast<float>((stamps[i + 1] - stamps[i]) * 1e-6) : 0.0f;
            ++n;
        }
    }
    *n_out = n;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return s;
}

extern "C" qv_status qv_plan_capture_graph(qv_plan_t *pl, qv_stream_t stream) {
    QV_RANGE("qv_plan_capture_graph");
    if (!pl) return qv_set_error(QV_ERR_INVALID, "qv_plan_capture_graph: null plan");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (st == nullptr) return qv_set_error(QV_ERR_INVALID, "qv_plan_capture_graph: needs a non-default stream");
    if (pl->graph) {
        cudaGraphExecDestroy(pl->graph);
        pl->graph = nullptr;
    }
    const bool was_dirty = pl->dirty;
    pl->dirty = false;
    cudaGraph_t g = nullptr;
    if (qv_check_cuda(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture") != QV_OK)
        return QV_ERR_CUDA;
    const qv_status ls = launch_plan(pl, st);
    const cudaError_t ce = cudaStreamEndCapture(st, &g);
    pl->dirty = was_dirty;
    if (ls != QV_OK) {
        if (g) cudaGraphDestroy(g);
        return ls;
    }
    if (qv_check_cuda(ce, "end capture") != QV_OK) return QV_ERR_CUDA;
    const cudaError_t ie = cudaGraphInstantiate(&pl->graph, g, 0);
    cudaGraphDestroy(g);
    return qv_check_cuda(ie, "graph instantiate");
}

extern "C" size_t qv_plan_readback_bytes(const qv_plan_t *pl) { return pl ? pl->read_bytes : 0; }

extern "C" qv_status qv_plan_read_async(const qv_plan_t *pl, void *h_buf, qv_stream_t stream) {
    if (!pl || !h_buf) return qv_set_error(QV_ERR_INVALID, "qv_plan_read_async: null pointer");
    return qv_check_cuda(cudaMemcpyAsync(h_buf, pl->ws + pl->read_off, pl->read_bytes, cudaMemcpyDeviceToHost,
                                         static_cast<cudaStream_t>(stream)),
                         "qv_plan_read_async");
}

extern "C" qv_status qv_plan_decode(qv_plan_t *pl, const void *h_buf, qv_plan_result_t *h) {
    if (!pl || !h_buf || !h) return qv_set_error(QV_ERR_INVALID, "qv_plan_decode: null pointer");
    const int E = pl->E, D = pl->params.depth;
    const char *buf = static_cast<const char *>(h_buf);
    auto at_host = [&](const void *dev_ptr) {
        return buf + (static_cast<const char *>(dev_ptr) - (pl->ws + pl->read_off));
    };
    const qv::ResultDev *r = reinterpret_cast<const qv::ResultDev *>(at_host(pl->dev.result));
    const int *cnt = reinterpret_cast<const int *>(at_host(pl->dev.count));
    unsigned status;
    unsigned long long bnd;
    std::memcpy(&status, at_host(pl->dev.status), sizeof(status));
    std::memcpy(&bnd, at_host(pl->dev.boundary), sizeof(bnd));
    for (int e = 0; e < E; ++e) {
        qv_plan_result_t &o = h[e];
        std::memset(&o, 0, sizeof(o));
        o.action = r[e].action;
        o.value = r[e].value;
        for (int a = 0; a < 5; ++a) o.q[a] = r[e].q[a];
        for (int l = 0; l <= D; ++l) o.nodes_per_level[l] = cnt[l * E + e];
        o.boundary_samples = static_cast<int64_t>(bnd);
        o.depth_reached = r[e].pad;
    }
    if (status) pl->dirty = true;  // counters may be mid-way: the next run re-zeroes them
    if (status & qv::kErrBounds) {
        unsigned site = 0;
        unsigned long long idx[2] = {0ull, 0ull};
        std::memcpy(&site, at_host(pl->dev.status + 2), sizeof(site));
        std::memcpy(idx, at_host(pl->dev.status + 4), sizeof(idx));
        return qv_set_error(QV_ERR_BOUNDS, "qv_plan: device bounds check failed at site %u (%s): index %lld, limit %lld",
                            site, qv::bounds_site_name(site), static_cast<long long>(idx[0]),
                            static_cast<long long>(idx[1]));
    }
    if (status & qv::kErrTimeout) return qv_set_error(QV_ERR_TIMEOUT, "qv_plan: a bounded device wait timed out");
    if (status & qv::kErrCapacity) return qv_set_error(QV_ERR_CAPACITY, "qv_plan: a level outgrew its capacity");
    return QV_OK;
}

extern "C" qv_status qv_plan_read(qv_plan_t *pl, qv_plan_result_t *h, qv_stream_t stream) {
    QV_RANGE("qv_plan_read");
    if (!pl || !h) return qv_set_error(QV_ERR_INVALID, "qv_plan_read: null pointer");
    std::vector<char> buf(pl->read_bytes);
    if (qv_plan_read_async(pl, buf.data(), stream) != QV_OK ||
        qv_check_cuda(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)), "qv_plan_read") != QV_OK)
        return QV_ERR_CUDA;
    return qv_plan_decode(pl, buf.data(), h);
}

extern "C" void qv_plan_destroy(qv_plan_t *pl) {
    if (!pl) return;
    if (pl->graph) cudaGraphExecDestroy(pl->graph);
    delete pl;
}

// The fused mode writes its leaves' records on demand, after the run that
// `stream` (or, with a null stream, the whole device) has finished or holds.
qv_status qv_plan_leaf_records(qv_plan_t *pl, cudaStream_t st, bool sync_device) {
    if (pl->params.leaf_mode == QV_LEAF_MATERIALISE || pl->params.depth == 0 || pl->records_fresh) return QV_OK;
    if (sync_device && qv_check_cuda(cudaDeviceSynchronize(), "leaf records") != QV_OK) return QV_ERR_CUDA;
    const int blocks = std::max(1, std::min(4 * qv_num_sms(), 1 << 16));
    qv::k_leaf_records<<<blocks, 256, 0, st>>>(pl->dev);
    if (qv_check_cuda(cudaGetLastError(), "leaf records launch") != QV_OK) return QV_ERR_CUDA;
    if (sync_device && qv_check_cuda(cudaDeviceSynchronize(), "leaf records") != QV_OK) return QV_ERR_CUDA;
    pl->records_fresh = true;
    return QV_OK;
}

extern "C" qv_status qv_plan_level(const qv_plan_t *cpl, int32_t e, int32_t l, qv_level_view_t *v) {
    if (!cpl || !v) return qv_set_error(QV_ERR_INVALID, "qv_plan_level: null pointer");
    if (e < 0 || e >= cpl->E || l < 0 || l > cpl->params.depth)
        return qv_set_error(QV_ERR_INVALID, "qv_plan_level: episode %d level %d out of range", e, l);
    qv_plan_t *pl = const_cast<qv_plan_t *>(cpl);
    if (l == pl->params.depth) {
        const qv_status rs = qv_plan_leaf_records(pl, nullptr, true);
        if (rs != QV_OK) return rs;
    }
    const qv::EpDev &ep = pl->eps[e];
    const qv::PlanDev &d = pl->dev;
    const int K = pl->params.K;
    std::memset(v, 0, sizeof(*v));
    v->cap = ep.cap[l];
    v->d_count = d.count + l * pl->E + e;
    const int g = ep.node_base[l];
    v->d_parent = d.parent + g;
    v->d_action = d.action + g;
    v->d_obs = d.obs + g;
    v->d_weight = d.weight + g;
    v->d_pz = d.pz + g;
    v->d_value = d.value + g;
    if (l < pl->params.depth) {
        const long long i = ep.inode_base[l];
        v->d_R = d.R + i * 5;
        v->d_UQ = d.UQ + i * 5;
        v->d_nchild = d.nchild + i * 5;
        v->d_samples = d.samples + i * 5 * K;
    }
    if (l == pl->params.depth) v->d_leaf_arg = d.leaf_arg + g;
    if (l == 0) v->d_belief = ep.b0;
    else if (ep.belief_off[l] >= 0) v->d_belief = d.beliefs + ep.belief_off[l];
    return QV_OK;
}

extern "C" qv_status qv_tree_plan_batched(int32_t E, const qv_model_t *models, const float *const *d_Q,
                                          const float *const *d_b0, const qv_plan_params_t *params, void *d_ws,
                                          size_t ws_bytes, qv_plan_result_t *h_results, qv_stream_t stream) {
    QV_RANGE("qv_tree_plan_batched");
    qv_plan_t *pl = nullptr;
    qv_status st = qv_plan_create(E, models, d_Q, d_b0, params, d_ws, ws_bytes, &pl, stream);
    if (st != QV_OK) return st;
    st = qv_plan_run(pl, stream);
    if (st == QV_OK) st = qv_plan_read(pl, h_results, stream);
    qv_plan_destroy(pl);
    return st;
}

extern "C" qv_status qv_tree_plan(const qv_model_t *model, const float *d_Q, const float *d_b0,
                                  const qv_plan_params_t *params, void *d_ws, size_t ws_bytes,
                                  qv_plan_result_t *h_result, qv_stream_t stream) {
    QV_RANGE("qv_tree_plan");
    return qv_tree_plan_batched(1, model, &d_Q, &d_b0, params, d_ws, ws_bytes, h_result, stream);
}

extern "C" int32_t qv_plan_grid(const qv_plan_t *pl) { return pl ? pl->grid : 0; }

extern "C" qv_status qv_plan_tuning(const qv_plan_t *pl, qv_tune_t *out) {
    if (!pl || !out) return qv_set_error(QV_ERR_INVALID, "qv_plan_tuning: null pointer");
    out->band_cells = pl->params.band_cells;
    out->items_per_cta = pl->params.items_per_cta;
    out->ms = 0.0f;
    return QV_OK;
}

extern "C" void qv_tune_clear(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.clear();
}

namespace {
const int kTuneBand[] = {1024, 2048, 4096, 8192};
const int kTuneItems[] = {1, 2, 4, 8};
}  // namespace

extern "C" size_t qv_plan_autotune_workspace_bytes(int32_t E, const qv_model_t *models,
                                                   const qv_plan_params_t *params) {
    if (!params) return 0;
    size_t best = 0;
    for (int bc : kTuneBand)
        for (int ipc : kTuneItems) {
            qv_plan_params_t p = *params;
            p.band_cells = bc;
            p.items_per_cta = ipc;
            Layout L;
            if (make_layout(E, models, &p, L, false) == QV_OK) best = std::max(best, L.total);
        }
    return best;
}

extern "C" qv_status qv_plan_autotune(int32_t E, const qv_model_t *models, const float *const *d_Q,
                                      const float *const *d_b0, const qv_plan_params_t *params, void *d_ws,
                                      size_t ws_bytes, int32_t reps, qv_tune_t *best, qv_tune_t *all, int32_t max_all,
                                      int32_t *n_all, qv_stream_t stream) {
    QV_RANGE("qv_plan_autotune");
    if (!params || !best) return qv_set_error(QV_ERR_INVALID, "qv_plan_autotune: null pointer");
    if (reps < 1) return qv_set_error(QV_ERR_INVALID, "qv_plan_autotune: reps %d", reps);
    qv_status st = validate(E, models, params);
    if (st != QV_OK) return st;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (qv_check_cuda(cudaEventCreate(&e0), "event") != QV_OK) return QV_ERR_CUDA;
    if (qv_check_cuda(cudaEventCreate(&e1), "event") != QV_OK) {
        cudaEventDestroy(e0);
        return QV_ERR_CUDA;
    }
    qv_tune_t win{0, 0, 0.0f};
    int n = 0;
    st = QV_OK;
    for (int bc : kTuneBand) {
        for (int ipc : kTuneItems) {
            qv_plan_params_t p = *params;
            p.band_cells = bc;
            p.items_per_cta = ipc;
            Layout L;
            if (make_layout(E, models, &p, L, true) != QV_OK || L.total > ws_bytes) continue;  // does not fit
            qv_plan_t *pl = nullptr;
            st = qv_plan_create(E, models, d_Q, d_b0, &p, d_ws, ws_bytes, &pl, stream);
            if (st != QV_OK) break;
            for (int w = 0; w < 2 && st == QV_OK; ++w) st = launch_plan(pl, cs);
            if (st == QV_OK) st = qv_check_cuda(cudaEventRecord(e0, cs), "event");
            for (int r = 0; r < reps && st == QV_OK; ++r) st = launch_plan(pl, cs);
            if (st == QV_OK) st = qv_check_cuda(cudaEventRecord(e1, cs), "event");
            if (st == QV_OK) st = qv_check_cuda(cudaEventSynchronize(e1), "autotune");
            unsigned status = 0;
            if (st == QV_OK)
                st = qv_check_cuda(cudaMemcpy(&status, pl->dev.status, sizeof(unsigned), cudaMemcpyDeviceToHost),
                                   "status");
            qv_plan_destroy(pl);
            if (st != QV_OK) break;
            if (status) continue;  // a candidate that ran out of capacity or timed out is not a choice
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            const qv_tune_t t{bc, ipc, ms / reps};
            if (all && n < max_all) all[n] = t;
            ++n;
            if (win.band_cells == 0 || t.ms < win.ms) win = t;
        }
        if (st != QV_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (n_all) *n_all = std::min(n, std::max(max_all, 0));
    if (st != QV_OK) return st;
    if (win.band_cells == 0) return qv_set_error(QV_ERR_INVALID, "qv_plan_autotune: no candidate fits");
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[tune_key(E, models, params)] = win;
    }
    *best = win;
    return QV_OK;
}

#ifdef QV_TRACE
// Trace builds only: copy out (and clear) the expand-phase timestamps.
extern "C" int qv_trace_read(unsigned long long *out, int max_records) {
    unsigned n = 0;
    if (cudaMemcpyFromSymbol(&n, qv::g_trace_n, sizeof(n)) != cudaSuccess) return -1;
    n = std::min<unsigned>(n, std::min<unsigned>(static_cast<unsigned>(max_records), qv::kTraceRecords));
    if (n && cudaMemcpyFromSymbol(out, qv::g_trace, sizeof(unsigned long long) * qv::kTraceWords * n) != cudaSuccess)
        return -1;
    const unsigned z = 0;
    cudaMemcpyToSymbol(qv::g_trace_n, &z, sizeof(z));
    return static_cast<int>(n);
}
#endif
