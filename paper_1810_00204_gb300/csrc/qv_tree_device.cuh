// qv_tree_device.cuh -- device side of the QV-tree search: one persistent
// cooperative kernel (k_plan) per plan or per batch of episodes.
//
// Phases of k_plan, separated by a bounded grid barrier: the support windows
// of every b0, then one phase per level l whose expand items run first and
// whose finalize items wait only for their own group's expand items, then:
//   expand(l)  for every V-node of level l (Alg. 2: every action) and a range
//              of row bands: the node's belief band.  At the root that is b0;
//              below it the band is recomputed from the parent's band (staged
//              with a two-row halo) as Phi(parent, a, z) of Eq. 3, and
//              written out when a later phase needs it.  On that band: the
//              motion stencil for all five actions (Eq. 3 numerator, Eq. 10),
//              the label histograms that give P(z | b, a) (Eq. 3
//              denominator) and R(b, a) (Sec. III).  Cells of the null label
//              are summed in registers; each beacon's sensing diamond is
//              summed by one warp (the finalize items), so no histogram
//              needs atomics.  The last work item of a node finalises it:
//              K Philox draws per action
//              inverted through the CDF (Alg. 3-4), the unique draws with
//              their frequencies.  The last node of an episode numbers its
//              children (prefix sum in (parent, action, z) order); the last
//              episode publishes the next level's work list.  At the deepest
//              internal level of the fused leaf mode the pass also sums
//              Q-weighted histograms, so every leaf value
//              max_a' sum_y b'(y) Q(a', y) (Eq. 4, Alg. 5) and the node's own
//              Q-node values (Alg. 6) follow without forming the leaves.
//   update     (materialised leaves) Phi(b, a, z) for every leaf: one read of
//              the parent band, one coalesced write per leaf.
//   leaf       (materialised leaves) streams leaf beliefs against Q.
//   backup     Alg. 6 / 7 bottom-up and the root argmax.
//
// Every band a work item touches arrives in shared memory by bulk (TMA)
// copies completing on one mbarrier: the belief rows with their halo, the
// cell words and, at the fused level, the band's rows of Q.
//
// Work items are (episode, node, band range) entries of per-level lists whose
// prefix sums and band splits are written on the device from the actual level
// sizes, so one launch covers episodes of uneven size and the host never
// waits for a level.
#pragma once

#include "qv_plan_types.cuh"

namespace qv {

// Per-warp buffers of the label histograms (finalize items): a tile of
// kTileH x kTileW cells of the node's belief is formed from the parent's
// belief with a two-cell rim, its cell words with a one-cell rim.
constexpr int kTileH = 17, kTileW = 18;  // one tile holds a range-8 diamond's 17 x 17 box
constexpr int kTileP = (kTileH + 4) * (kTileW + 4);   // parent values
constexpr int kTileC = (kTileH + 2) * (kTileW + 2);   // node values, cell words
constexpr int kTileFloats = kTileP + kTileC + (kTileC + 1) / 2 + kTileH * kTileW;  // + the cell list
// Totals of one V-node per work item: [0, 5) null-label masses, [5, 10)
// R(b, a) sums, [10, 35) Q-weighted null masses (fused level), [35] unused.
constexpr int kTot = 36;

// Bounds-checked debug build (compiled in with -DQV_BOUNDS_CHECK, the
// library libqvts_debug.so): QV_IN_BOUNDS(site, i, n) is false when i lies
// outside [0, n), and the access it guards is then skipped instead of
// faulting.  A failure is counted in g_bounds[0] and the first one is kept
// (site, index, limit); after the kernel, k_bounds_collect moves them into
// the plan's status words, so the call returns QV_ERR_BOUNDS with the site's
// name.  A site equal to g_bounds_inject (host-side fault injection,
// QVTS_FAULT=bounds) reports a failure while its index is in range, and its
// access still runs.  In release builds the checks compile to `true`.
enum BoundsSite : unsigned {
    kSiteNode = 1,     // per-node records at a node id (parent, action, obs, weight, pz, code, value)
    kSiteInode,        // per-internal-node arrays (R, UQ, samples, sample slots, child counts)
    kSiteSlot,         // a unique draw's slot within its (node, action) run of K
    kSiteChild,        // child numbering: child offsets and source slots
    kSiteBelief,       // a stored belief (read or written) within the level's slots
    kSiteCopy,         // the rows and columns of a band's bulk copies within the grid
    kSiteRecord,       // beacon-chunk and item records
    kSiteEpisode,      // per-episode results and level counts
    kSiteGroup,        // expand group lists
    kSiteCount
};
inline const char *bounds_site_name(unsigned site) {
    switch (site) {
        case kSiteNode: return "node record";
        case kSiteInode: return "internal node arrays";
        case kSiteSlot: return "sample slot";
        case kSiteChild: return "child numbering";
        case kSiteBelief: return "stored belief";
        case kSiteCopy: return "band copy";
        case kSiteRecord: return "chunk or item record";
        case kSiteEpisode: return "episode result or level count";
        case kSiteGroup: return "expand group list";
        default: return "unknown";
    }
}
#ifdef QV_BOUNDS_CHECK
__device__ unsigned long long g_bounds[4];  // failures, first site, its index, its limit
__device__ unsigned g_bounds_inject;
__device__ __noinline__ void bounds_record(unsigned site, long long i, long long n) {
    if (atomicAdd(&g_bounds[0], 1ull) == 0ull) {
        g_bounds[1] = site;
        g_bounds[2] = static_cast<unsigned long long>(i);
        g_bounds[3] = static_cast<unsigned long long>(n);
    }
}
__device__ __forceinline__ bool bounds_ok(unsigned site, long long i, long long n) {
    const bool in = i >= 0 && i < n;
    if (!in || site == *((volatile unsigned *)&g_bounds_inject)) bounds_record(site, i, n);
    return in;
}
#define QV_IN_BOUNDS(site, i, n) qv::bounds_ok((site), static_cast<long long>(i), static_cast<long long>(n))
// After k_plan on the same stream: the failure words into the plan's status
// (status[0] |= kErrBounds, status[2] = site, status[4..5] = index,
// status[6..7] = limit, as 64-bit words), then cleared for the next run.
__global__ void k_bounds_collect(unsigned *status) {
    if (g_bounds[0]) {
        status[0] |= kErrBounds;
        status[2] = static_cast<unsigned>(g_bounds[1]);
        reinterpret_cast<unsigned long long *>(status + 4)[0] = g_bounds[2];
        reinterpret_cast<unsigned long long *>(status + 4)[1] = g_bounds[3];
    }
    g_bounds[0] = g_bounds[1] = g_bounds[2] = g_bounds[3] = 0ull;
}
#else
#define QV_IN_BOUNDS(site, i, n) true
#endif

// The contraction form of the deepest fused level (ctr_item): a row
// segment of kCSC cells at a time, children in blocks of at most kCMB (of
// at most kCPar parents: every V-node has at least five children), 36
// planes per cell (the kTot totals).  Its arrays live in the band buffers.
constexpr int kCSC = 64;
constexpr int kCMB = 96;
constexpr int kCPar = kCMB / 5 + 3;
// staged columns: the segment with a one-cell rim, rounded out to 8-column
// chunks so that every copy is 16 bytes on a 16-byte boundary
constexpr int kCSW = kCSC + 16;
static_assert(kCSC == 64, "the contraction's task loops index cells with 6-bit shifts");
constexpr int kCBP = kCSC + 1;  // row stride of the predicted beliefs (rows of different children fall in different banks)
struct CtrLayout {
    int par, q, cost, cw, bp, W, cpi, ca, cz, csa, cse, total;  // float offsets from the band buffers
};
__host__ __device__ inline CtrLayout ctr_layout() {
    CtrLayout c;
    int o = 0;
    auto take = [&](int n) {
        o = (o + 3) & ~3;  // 16-byte aligned
        const int r = o;
        o += n;
        return r;
    };
    // two stages of the staged rows y - 1 .. y + 1 (double-buffered copies)
    c.par = take(2 * kCPar * 3 * kCSW);  // [stage][parent][row][column] the parents' values
    c.q = take(2 * 5 * 3 * kCSW);        // [stage][a'][row][column] Q
    c.cost = take(2 * 3 * kCSW);         // [stage][row][column] the cost map
    c.cw = take(2 * 3 * kCSW / 2);       // [stage][row][column] cell words (uint16)
    c.bp = take(kCPar * 5 * kCBP);       // [parent][a][cell] the parents' predicted beliefs T_a b_p
    c.W = take(kCSC * kTot);             // [cell][plane] T_a^T of the null, reward and null-Q weights
    c.cpi = take(kCMB);                  // per child of the block: parent slot, action, observation, alpha / P, eta / P
    c.ca = take(kCMB);
    c.cz = take(kCMB);
    c.csa = take(kCMB);
    c.cse = take(kCMB);
    c.total = o;
    return c;
}

// Shared-memory carve-up of k_plan (same arithmetic on host and device).
struct SmemLayout {
    size_t sb, sp, cw, q, tile, ep, bco, hist, histq, tot, red, P, C, cnt, T, uq, lut, lut4, u_n, u_off, u_z, u_sa, u_se,
        scan, flags, acc, c_pa, c_z, c_sa, c_se, wpart, wchild, band_end, total;
    __host__ __device__ static SmemLayout make(int sb_floats, int sp_floats, int q_floats, int Bm, int K, int cmax,
                                               int kslots) {
        SmemLayout s;
        size_t o = 0;
        auto take = [&](size_t bytes) {
            o = (o + 15) & ~size_t(15);
            const size_t r = o;
            o += bytes;
            return r;
        };
        s.sb = take(sizeof(float) * sb_floats);      // node band, one halo row (materialised leaves only)
        s.sp = take(sizeof(float) * sp_floats);      // parent band, two halo rows
        s.cw = take(sizeof(uint16_t) * (sp_floats > sb_floats ? sp_floats : sb_floats));  // cell words, two halo rows
        s.q = take(sizeof(float) * q_floats);        // the band's rows of Q
        // what only a finalize item uses -- the label tiles, the histograms,
        // P(z), the CDF and the draw counts -- shares the band buffers, which
        // only expand and update items use (a CTA runs one item at a time,
        // with a CTA barrier between items), as far as they are large enough
        const size_t band_end = o;
        s.band_end = band_end;
        size_t in = s.sb;
        auto place = [&](size_t bytes) {
            const size_t r = (in + 15) & ~size_t(15);
            if (r + bytes <= band_end) {
                in = r + bytes;
                return r;
            }
            return take(bytes);
        };
        s.tile = place(sizeof(float) * kTileFloats * kWarps);
        s.hist = place(sizeof(float) * 5 * Bm);
        s.histq = place(sizeof(float) * 25 * Bm);
        s.P = place(sizeof(float) * 5 * (Bm + 1));
        s.C = place(sizeof(float) * 5 * (Bm + 1));
        s.cnt = place(sizeof(int) * 5 * (Bm + 1));
        s.ep = take(sizeof(EpDev));
        s.bco = take(sizeof(int) * 2 * Bm);          // beacon (row, col)
        s.tot = take(sizeof(float) * kTot);
        s.red = take(sizeof(float) * kWarps * kTot);
        s.T = take(sizeof(float) * 28);
        s.uq = take(sizeof(float) * 8);
        s.lut = take(sizeof(float) * 64);
        s.lut4 = take(sizeof(float) * 64);           // the same weights as float4 [blocked nibble][action]
        s.u_n = take(sizeof(int) * 8);
        s.u_off = take(sizeof(int) * 8);
        s.u_z = take(sizeof(int) * 5 * K);
        s.u_sa = take(sizeof(float) * 5 * K);
        s.u_se = take(sizeof(float) * 5 * K);
        s.scan = take(sizeof(int) * (kWarps + 4));
        s.flags = take(sizeof(int) * 12);
        s.acc = take(sizeof(float) * kTot * cmax);   // per-child totals of a work item
        s.c_pa = take(sizeof(int) * cmax);           // per child: action, observation, alpha / P, eta / P
        s.c_z = take(sizeof(int) * cmax);
        s.c_sa = take(sizeof(float) * cmax);
        s.c_se = take(sizeof(float) * cmax);
        s.wpart = take(sizeof(float) * kTot * kWarps * kslots);  // per-warp sums of a band
        s.wchild = take(sizeof(int) * kWarps * kslots);          // the child of each slot, -1 unused
        s.total = (o + 127) & ~size_t(127);
        return s;
    }
};

struct Smem {
    float *sb, *sp, *q, *tile;
    uint16_t *cw;
    EpDev *ep;
    int *bco;
    float *hist, *histq, *tot, *red, *P, *C, *T, *uq, *lut;
    float4 *lut4;
    int *cnt;
    int *u_n, *u_off, *u_z;
    float *u_sa, *u_se;
    int *scan, *flags;
    float *acc;
    int *c_pa, *c_z;
    float *c_sa, *c_se;
    float *wpart;
    int *wchild;
    int nband;  // 4-byte words of the band buffers (from sb), free for scratch outside expand and update items
};

// Slots per warp for the per-child sums of one band: a warp's contiguous
// range of (child, strip, row) tasks spans at most cmax / kWarps + 3 children.
__host__ __device__ __forceinline__ int expand_slots(int cmax) { return cmax / kWarps + 3; }

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ int find_episode(const int *wb, int E, int w) {
    int lo = 0, hi = E - 1;  // last e with wb[e] <= w
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldcg(wb + mid) <= w) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The same search by one warp, 32 probes per step (log32 of n dependent
// loads instead of log2 of n): last j in [0, n) with wb[j] <= w, for a
// nondecreasing wb with wb[0] <= w.
__device__ __forceinline__ int warp_find(const int *wb, int n, int w) {
    const int lane = threadIdx.x & 31;
    int lo = 0, hi = n - 1;
    while (hi > lo) {
        const long long span = hi - lo;
        const int base = lo;
        auto probe = [&](int i) { return base + static_cast<int>((span * (i + 1) + 31) / 32); };
        const unsigned bal = __ballot_sync(0xffffffffu, __ldcg(wb + probe(lane)) <= w);
        const int m = __popc(bal);
        if (m == 0) {
            hi = probe(0) - 1;
        } else {
            if (m < 32) hi = probe(m) - 1;
            lo = probe(m - 1);
        }
    }
    return lo;
}
// warp_find by warp 0 for the whole CTA (one CTA barrier); `slot` is a
// shared word not read again before the CTA's next barrier.
__device__ __forceinline__ int block_find(const int *wb, int n, int w, int *slot) {
    if (threadIdx.x < 32) {
        const int r = warp_find(wb, n, w);
        if (threadIdx.x == 0) *slot = r;
    }
    __syncthreads();
    return *slot;
}

// Dynamic work distribution: the CTA's next item of a phase, taken from
// the phase's counter (one atomic per item; every item writes its own
// records, so the results do not depend on which CTA takes which item).
__device__ __forceinline__ int next_item(unsigned *ctr, int *slot) {
    __syncthreads();  // every thread has read the previous item's index
    if (threadIdx.x == 0) *slot = static_cast<int>(atomicAdd(ctr, 1u));
    __syncthreads();
    return *slot;
}

__device__ __forceinline__ const float *node_belief(const PlanDev &pl, const EpDev &ep, int l, int local) {
    if (l == 0) return ep.b0;
    const long long off = ep.belief_off[l] + static_cast<long long>(local) * ep.N;
    if (!QV_IN_BOUNDS(kSiteBelief, off + ep.N - 1, pl.n_belief)) return ep.b0;  // debug build: a readable stand-in
    return pl.beliefs + off;
}

// ---------------------------------------------------------------- support windows
// The motion stencil (Eq. 3 numerator, Eq. 10) moves mass by at most one
// cell and the observation weights (Eq. 3) only rescale it, so a node d
// levels below the root is zero outside the bounding box of b0's nonzero
// cells dilated by d cells.  The expand and finalize phases restrict their
// sums to that window; every cell outside it contributes exactly zero.
struct Win {
    int r0, r1, c0, c1;  // rows [r0, r1), columns [c0, c1); empty when r1 <= r0
};
__device__ __forceinline__ Win support_window(const PlanDev &pl, int e, int H, int W, int d) {
    const unsigned *w = pl.win + 4 * e;
    const int rmin = kWinBig - static_cast<int>(__ldcg(w)), rmax = static_cast<int>(__ldcg(w + 1)) - 1;
    const int cmin = kWinBig - static_cast<int>(__ldcg(w + 2)), cmax = static_cast<int>(__ldcg(w + 3)) - 1;
    Win v;
    if (rmax < rmin || cmax < cmin) {
        v.r0 = v.r1 = v.c0 = v.c1 = 0;
        return v;
    }
    v.r0 = max(0, rmin - d);
    v.r1 = min(H, rmax + d + 1);
    v.c0 = max(0, cmin - d);
    v.c1 = min(W, cmax + d + 1);
    return v;
}

// Band geometry of the expand phase at level l: task rows [r0, r1) and
// float4 column groups [g0, g1) (where the level's predicted masses can be
// nonzero: the support window of level l + 1), the staged columns
// [sc0, sc0 + sw) (the task columns with the two-cell reach of a child's
// stencil, rounded out to multiples of 8 so that every staged row starts and
// ends on a 16-byte boundary), `rows` task rows per band and `nb` bands.
// rows * sw never exceeds band_rows * P, so a windowed band fits the buffers
// sized for a full-width one.
struct BandGeo {
    int r0, r1, g0, g1, sc0, sw, rows, nb;
};
__device__ __forceinline__ BandGeo band_geo(const PlanDev &pl, int e, int H, int W, int P, int band_rows, int l) {
    BandGeo g;
    const Win t = support_window(pl, e, H, W, l + 1);
    g.r0 = t.r0;
    g.r1 = t.r1;
    g.g0 = t.c0 >> 2;
    g.g1 = (t.c1 + 3) >> 2;
    if (t.r1 <= t.r0 || t.c1 <= t.c0) {
        g.g1 = g.g0;
        g.sc0 = 0;
        g.sw = 8;
        g.rows = 1;
        g.nb = 0;
        return g;
    }
    g.sc0 = max(0, 4 * g.g0 - 2) & ~7;
    g.sw = min(P, (4 * g.g1 + 2 + 7) & ~7) - g.sc0;
    g.rows = max(1, min(t.r1 - t.r0, (band_rows * P) / g.sw));
    g.nb = (t.r1 - t.r0 + g.rows - 1) / g.rows;
    return g;
}

__device__ __forceinline__ void fill_self_lut(float *lut, float slip) {
    for (int i = threadIdx.x; i < 64; i += blockDim.x) lut[i] = self_weight(i >> 4, i & 15, slip);
}
// lut4[blocked nibble] = the four move actions' self weights, one 16-byte load.
__device__ __forceinline__ void fill_self_lut4(float4 *lut4, float slip) {
    for (int i = threadIdx.x; i < 16; i += blockDim.x)
        lut4[i] = make_float4(self_weight(0, i, slip), self_weight(1, i, slip), self_weight(2, i, slip),
                              self_weight(3, i, slip));
}

// Copy the descriptor of episode e (and its beacon coordinates) into shared
// memory, once per change of episode.
__device__ __forceinline__ void load_ep(const PlanDev &pl, int e, Smem &S, int &cur_e) {
    if (e == cur_e) return;
    __syncthreads();
    int4 *dst = reinterpret_cast<int4 *>(S.ep);
    if (pl.E == 1) {  // from the kernel's parameters, no global round trip
        const int4 *src = reinterpret_cast<const int4 *>(&pl.ep0);
        for (int i = threadIdx.x; i < static_cast<int>(sizeof(EpDev) / 16); i += blockDim.x) dst[i] = src[i];
    } else {
        const int4 *src = reinterpret_cast<const int4 *>(pl.eps + e);
        for (int i = threadIdx.x; i < static_cast<int>(sizeof(EpDev) / 16); i += blockDim.x) dst[i] = __ldg(src + i);
    }
    __syncthreads();
    const EpDev &ep = *S.ep;
    for (int k = threadIdx.x; k < ep.B; k += blockDim.x) {
        const int b = __ldg(ep.beacons + k);
        S.bco[2 * k] = b / ep.P;
        S.bco[2 * k + 1] = b - (b / ep.P) * ep.P;
    }
    fill_self_lut(S.lut, ep.slip);
    fill_self_lut4(S.lut4, ep.slip);
    __syncthreads();
    cur_e = e;
}

__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Arrival on a last-arriver counter: an acquire-release add, so that (after
// a CTA barrier) it publishes the CTA's writes and, for the last arriver,
// makes the earlier arrivals' writes visible.
__device__ __forceinline__ unsigned arrive_acq_rel(unsigned *p) {
    unsigned prev;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(prev) : "l"(p) : "memory");
    return prev;
}

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded grid barrier; every CTA of the cooperative launch calls it the
// same number of times.  False (for every CTA) once any wait gave up.  The
// arrival is an acquire-release add on the counter (after the CTA barrier,
// so it publishes every thread's writes); the last arriver releases the
// generation word, which the others acquire.
// With `deadline`, the last arriver also decides, once for every CTA,
// whether the plan's time budget (from the kernel's first stamp) has run
// out, and sets status[1] before it releases the others.
__device__ bool grid_sync(const PlanDev &pl, bool deadline = false) {
    __shared__ int s_ok;
    fence_proxy_async_global();
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned g;
        asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(g) : "l"(&pl.bar->gen) : "memory");
        unsigned prev;
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(prev) : "l"(&pl.bar->count) : "memory");
        if (prev == gridDim.x - 1) {
            if (deadline && globaltimer() - pl.stamps[0] >= pl.deadline_ns)
                asm volatile("st.relaxed.gpu.global.u32 [%0], 1;" ::"l"(pl.status + 1) : "memory");
            asm volatile("st.relaxed.gpu.global.u32 [%0], 0;" ::"l"(&pl.bar->count) : "memory");
            asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(&pl.bar->gen), "r"(g + 1u) : "memory");
        } else {
            unsigned i = 0;
            for (;;) {
                unsigned cur;
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(&pl.bar->gen) : "memory");
                if (cur != g) break;
                if (++i > pl.spin_limit || (*((volatile unsigned *)pl.status) & kErrTimeout)) {
                    atomicOr(pl.status, kErrTimeout);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        if (*((volatile unsigned *)pl.status) & kErrTimeout) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ void stamp(const PlanDev &pl, int slot) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && slot < kStamps) pl.stamps[slot] = globaltimer();
}

// Optional tracing (compiled in with -DQV_TRACE): device-clock timestamps of
// the steps of every expand work item, for latency analysis.
constexpr int kTraceWords = 16;
constexpr int kTraceRecords = 1 << 16;
#ifdef QV_TRACE
__device__ unsigned long long g_trace[kTraceRecords][kTraceWords];
__device__ unsigned g_trace_n;
#define QV_TRACE_MARK(arr, k) \
    do {                      \
        if (threadIdx.x == 0) arr[k] = globaltimer(); \
    } while (0)
__device__ __forceinline__ void trace_commit(const unsigned long long *t, int n) {
    if (threadIdx.x != 0) return;
    const unsigned i = atomicAdd(&g_trace_n, 1u);
    if (i < kTraceRecords)
        for (int k = 0; k < n && k < kTraceWords; ++k) g_trace[i][k] = t[k];
}
#else
#define QV_TRACE_MARK(arr, k) \
    do {                      \
    } while (0)
#endif


// Stage one band on one mbarrier: belief rows [r0-h, r1+h) of `b` (zero
// outside the grid) into bbuf; the cell words of rows [r0-ch, r1+ch) into cw
// (cw row i = grid row r0-ch+i); and, when q is given, rows [r0, r1) of the
// five Q planes into q (plane stride (r1-r0)*P).  Bounded wait, one decision
// for the whole CTA.
__device__ bool stage_band(const EpReg &ep, const float *b, int r0, int r1, int h, float *bbuf, uint16_t *cw,
                           float *q, uint64_t *bar, unsigned &phase, unsigned *status, int ch = 1) {
    const int P = ep.P;
    __syncthreads();  // previous readers of the buffers are done
    for (int r = r0 - h; r < r0; ++r)
        if (r < 0)
            for (int i = threadIdx.x; i < P; i += blockDim.x) bbuf[(r - (r0 - h)) * P + i] = 0.0f;
    for (int r = r1; r < r1 + h; ++r)
        if (r >= ep.H)
            for (int i = threadIdx.x; i < P; i += blockDim.x) bbuf[(r - (r0 - h)) * P + i] = 0.0f;
    fence_proxy_async();
    __syncthreads();
    if (threadIdx.x == 0 && !(QV_IN_BOUNDS(kSiteCopy, r0, ep.H) && QV_IN_BOUNDS(kSiteCopy, r1 - 1, ep.H))) {
        mbar_arrive_expect_tx(bar, 0u);  // debug build: no copy leaves the grid
    } else if (threadIdx.x == 0) {
        fence_proxy_async_global();
        const int lo = max(0, r0 - h), hi = min(ep.H, r1 + h);
        const int clo = max(0, r0 - ch), chi = min(ep.H, r1 + ch);
        const unsigned bb = static_cast<unsigned>((hi - lo) * P * sizeof(float));
        const unsigned cb = static_cast<unsigned>((chi - clo) * P * sizeof(uint16_t));
        const unsigned qb = static_cast<unsigned>((r1 - r0) * P * sizeof(float));
        mbar_arrive_expect_tx(bar, bb + cb + (q ? 5u * qb : 0u));
        bulk_copy_g2s(bbuf + (lo - (r0 - h)) * P, b + static_cast<size_t>(lo) * P, bb, bar);
        bulk_copy_g2s(cw + (clo - (r0 - ch)) * P, ep.cell + static_cast<size_t>(clo) * P, cb, bar);
        if (q)
            for (int a = 0; a < 5; ++a)
                bulk_copy_g2s(q + a * (r1 - r0) * P, ep.Q + static_cast<size_t>(a) * ep.N + static_cast<size_t>(r0) * P,
                              qb, bar);
    }
    const bool ok = mbar_wait_bounded(bar, phase);
    const int failed = __syncthreads_or(ok ? 0 : 1);
    if (failed) {
        if (threadIdx.x == 0) atomicOr(status, kErrTimeout);
        if (!ok) mbar_wait_bounded(bar, phase);  // let the copies in flight land before leaving
    }
    phase ^= 1u;
    return failed == 0;
}

// The expand phase's staging of one band of a column window: belief rows
// [r0-2, r1+2) (zero outside the grid) and cell words of the same rows,
// columns [sc0, sc0 + sw), into rows of sw values; with q, rows [r0, r1) of
// the five Q planes (plane stride (r1-r0)*sw).  A full-width window is
// contiguous: one bulk copy per array (five for Q); a narrower one takes one
// bulk copy per row and array.  The lanes of warp 0 issue the copies;
// stage_wait then waits for them (bounded), so that other work can run in
// between.  The caller has passed a CTA barrier since the buffers' last
// readers.
__device__ void stage_issue(const EpReg &ep, const float *b, int r0, int r1, int sc0, int sw, float *bbuf,
                            uint16_t *cw, float *q, uint64_t *bar) {
    const int P = ep.P;
    for (int r = r0 - 2; r < r0; ++r)
        if (r < 0)
            for (int i = threadIdx.x; i < sw; i += blockDim.x) bbuf[(r - (r0 - 2)) * sw + i] = 0.0f;
    for (int r = r1; r < r1 + 2; ++r)
        if (r >= ep.H)
            for (int i = threadIdx.x; i < sw; i += blockDim.x) bbuf[(r - (r0 - 2)) * sw + i] = 0.0f;
    fence_proxy_async();
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const int lo = max(0, r0 - 2), hi = min(ep.H, r1 + 2), R = r1 - r0;
        const int nbr = hi - lo;
        const unsigned rb = static_cast<unsigned>(sw * sizeof(float)), cb = static_cast<unsigned>(sw * sizeof(uint16_t));
        if (!(QV_IN_BOUNDS(kSiteCopy, sc0, P - sw + 1) && QV_IN_BOUNDS(kSiteCopy, r0, ep.H) &&
              QV_IN_BOUNDS(kSiteCopy, r1 - 1, ep.H))) {
            // debug build: no copy leaves the grid; the barrier completes empty
            if (lane == 0) mbar_arrive_expect_tx(bar, 0u);
            return;
        }
        if (lane == 0)
            mbar_arrive_expect_tx(bar, static_cast<unsigned>(nbr) * (rb + cb) + (q ? 5u * R * rb : 0u));
        __syncwarp();
        fence_proxy_async_global();
        if (sw == P) {
            if (lane == 0) bulk_copy_g2s(bbuf + (lo - (r0 - 2)) * P, b + static_cast<size_t>(lo) * P, nbr * rb, bar);
            if (lane == 1)
                bulk_copy_g2s(cw + (lo - (r0 - 2)) * P, ep.cell + static_cast<size_t>(lo) * P, nbr * cb, bar);
            if (q && lane >= 2 && lane < 7) {
                const int a = lane - 2;
                bulk_copy_g2s(q + a * R * P, ep.Q + static_cast<size_t>(a) * ep.N + static_cast<size_t>(r0) * P,
                              R * rb, bar);
            }
        } else {
            const int nq = q ? 5 * R : 0;
            for (int i = lane; i < 2 * nbr + nq; i += 32) {
                if (i < nbr) {
                    const int r = lo + i;
                    bulk_copy_g2s(bbuf + (r - (r0 - 2)) * sw, b + static_cast<size_t>(r) * P + sc0, rb, bar);
                } else if (i < 2 * nbr) {
                    const int r = lo + i - nbr;
                    bulk_copy_g2s(cw + (r - (r0 - 2)) * sw, ep.cell + static_cast<size_t>(r) * P + sc0, cb, bar);
                } else {
                    const int a = (i - 2 * nbr) / R, y = (i - 2 * nbr) - a * R;
                    bulk_copy_g2s(q + (a * R + y) * sw,
                                  ep.Q + static_cast<size_t>(a) * ep.N + static_cast<size_t>(r0 + y) * P + sc0, rb,
                                  bar);
                }
            }
        }
    }
}
__device__ bool stage_wait(uint64_t *bar, unsigned &phase, unsigned *status) {
    const bool ok = mbar_wait_bounded(bar, phase);
    const int failed = __syncthreads_or(ok ? 0 : 1);
    if (failed) {
        if (threadIdx.x == 0) atomicOr(status, kErrTimeout);
        if (!ok) mbar_wait_bounded(bar, phase);  // let the copies in flight land before leaving
    }
    phase ^= 1u;
    return failed == 0;
}

// Neighbourhood of the 4 cells (row, col..col+3): `mid` points at the
// cell's row inside a staged belief buffer (rows P floats apart), `cwr` at
// the same row of the staged cell words.
struct Nbr4 {
    float u[4], m[6], d[4];
    unsigned cw[4];
};
__device__ __forceinline__ void load_nbr(const EpReg &ep, const float *mid, const uint16_t *cwr, int col, Nbr4 &n) {
    const int P = ep.P;
    const float4 up = *reinterpret_cast<const float4 *>(mid - P + col);
    const float4 md = *reinterpret_cast<const float4 *>(mid + col);
    const float4 dn = *reinterpret_cast<const float4 *>(mid + P + col);
    n.u[0] = up.x; n.u[1] = up.y; n.u[2] = up.z; n.u[3] = up.w;
    n.m[0] = col > 0 ? mid[col - 1] : 0.0f;
    n.m[1] = md.x; n.m[2] = md.y; n.m[3] = md.z; n.m[4] = md.w;
    n.m[5] = col + 4 < P ? mid[col + 4] : 0.0f;
    n.d[0] = dn.x; n.d[1] = dn.y; n.d[2] = dn.z; n.d[3] = dn.w;
    const ushort4 cw4 = *reinterpret_cast<const ushort4 *>(cwr + col);
    n.cw[0] = cw4.x; n.cw[1] = cw4.y; n.cw[2] = cw4.z; n.cw[3] = cw4.w;
}

__device__ __forceinline__ void inflow_nb(const Nbr4 &n, int j, float nb[4]) {
    const unsigned in = QV_CELL_INFLOW(n.cw[j]);
    nb[kDirN] = (in & 1u) ? n.u[j] : 0.0f;
    nb[kDirE] = (in & 2u) ? n.m[j + 2] : 0.0f;
    nb[kDirS] = (in & 4u) ? n.d[j] : 0.0f;
    nb[kDirW] = (in & 8u) ? n.m[j] : 0.0f;
}

// Predicted mass of one cell (column c of the staged row `mid`) for all
// five actions.
__device__ __forceinline__ void predict_at(const EpReg &ep, const float *mid, int c, unsigned cw, bool is_goal,
                                           const float *lut, float out[5]) {
    const unsigned in = QV_CELL_INFLOW(cw);
    float nb[4];
    nb[kDirN] = (in & 1u) ? mid[c - ep.P] : 0.0f;
    nb[kDirE] = (in & 2u) ? mid[c + 1] : 0.0f;
    nb[kDirS] = (in & 4u) ? mid[c + ep.P] : 0.0f;
    nb[kDirW] = (in & 8u) ? mid[c - 1] : 0.0f;
    predict_cell(nb, mid[c], cw, is_goal, ep.slip, lut, out);
}

__device__ int block_exclusive_scan(int v, int *s_warp, int &total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int k = 0; k < kWarps; ++k) {
            const int t = s_warp[k];
            s_warp[k] = run;
            run += t;
        }
        s_warp[kWarps] = run;
    }
    __syncthreads();
    const int ex = x - v + s_warp[wid];
    total = s_warp[kWarps];
    __syncthreads();
    return ex;
}

// ---------------------------------------------------------------- node finalisation
// P(z | b, a) from the label histograms, R(b, a), K Philox draws per action
// inverted through the FP32 CDF, the unique draws with their frequencies.
// At the fused leaf level also each child's leaf value and then the node's
// U_Q (Alg. 6, discounted as in Eq. 2) and U_V (Alg. 7).  One warp per action.
__device__ void finalize_node(const PlanDev &pl, const EpDev &ep, int l, int local, bool fused, float bgoal,
                              unsigned long long code, Smem &S) {
    const int B = ep.B, nz = B + 1, K = pl.K, Bm = pl.Bmax;
    const int iid = ep.inode_base[l] + local;
    if (!QV_IN_BOUNDS(kSiteInode, iid, pl.n_inodes)) return;  // uniform over the CTA
    const float eta = ep.eta, acc = ep.acc;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < 5 * nz; i += blockDim.x) S.cnt[i] = 0;
    if (fused) {
        // T[a][a'] = the Q-weighted masses over every label: eight threads
        // per entry, each over every eighth beacon
        for (int t0 = 0; t0 < 25; t0 += kThreads / 8) {
            const int t = t0 + (threadIdx.x >> 3), sub = threadIdx.x & 7;
            float s = 0.0f;
            if (t < 25) {
                const int a = t / 5, ap = t % 5;
                for (int z = sub; z < B; z += 8) s += S.histq[(a * Bm + z) * 5 + ap];
            }
            s += __shfl_xor_sync(0xffffffffu, s, 1);
            s += __shfl_xor_sync(0xffffffffu, s, 2);
            s += __shfl_xor_sync(0xffffffffu, s, 4);
            if (t < 25 && sub == 0) S.T[t] = s + S.tot[10 + t];
        }
    }
    for (int a = wid; a < 5; a += kWarps) {
        // one warp per action: P(z | b, a) for every z, and its cumulative
        // sum in ascending z (FP32, a warp scan per 32 values)
        float m = 0.0f;
        for (int z = lane; z < B; z += 32) m += S.hist[a * Bm + z];
        const float Ssum = warp_sum(m) + S.tot[a];
        float carry = 0.0f;
        for (int zc = 0; zc < nz; zc += 32) {
            const int z = zc + lane;
            const float M = z < B ? S.hist[a * Bm + z] : (z == B ? S.tot[a] : 0.0f);
            const float p = z < nz ? fmaf(acc - eta, M, eta * Ssum) : 0.0f;
            float x = p;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const float y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            x += carry;
            if (z < nz) {
                S.P[a * nz + z] = p;
                S.C[a * nz + z] = x;
            }
            carry = __shfl_sync(0xffffffffu, x, 31);
        }
        if (lane == 0) pl.R[iid * 5 + a] = S.tot[5 + a] - 100.0f * bgoal;
    }
    __syncthreads();
    const uint32_t epw = pl.episode_word ? __ldcg(pl.episode_word) + (ep.episode - pl.episode0) : ep.episode;
    for (int t = threadIdx.x; t < 5 * K; t += blockDim.x) {
        const int a = t / K, k = t - a * K;
        const float *C = S.C + a * nz;
        const float u = sample_uniform(pl.seed, epw, l, code * 5ull + a, k);
        int z;
        if (pl.replay) {
            z = __ldg(pl.replay + (static_cast<long long>(iid) * 5 + a) * K + k);
            z = min(max(z, 0), B);
        } else {
            const float t_u = u * C[B];
            int lo = 0, hi = B;  // first z with t_u < C[z]
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (t_u < C[mid]) hi = mid;
                else lo = mid + 1;
            }
            z = lo;
        }
        const float inv = 1.0f / C[B];
        const bool near = (z < B && fabsf(u - C[z] * inv) < kBoundaryEps) ||
                          (z > 0 && fabsf(u - C[z - 1] * inv) < kBoundaryEps);
        if (near) atomicAdd(pl.boundary, 1ull);
        pl.samples[(static_cast<long long>(iid) * 5 + a) * K + k] = z;
        atomicAdd(&S.cnt[a * nz + z], 1);
    }
    __syncthreads();
    for (int a = wid; a < 5; a += kWarps) {
        const long long sb = (static_cast<long long>(iid) * 5 + a) * K;
        int base = 0;
        float psum = 0.0f;
        for (int zc = 0; zc < nz; zc += 32) {
            const int z = zc + lane;
            const int c = z < nz ? S.cnt[a * nz + z] : 0;
            const float p = z < nz ? S.P[a * nz + z] : 0.0f;
            const unsigned bal = __ballot_sync(0xffffffffu, c > 0);
            const int pos = base + __popc(bal & ((1u << lane) - 1u));
            if (c > 0 && QV_IN_BOUNDS(kSiteSlot, pos, K)) {
                pl.slot_z[sb + pos] = z;
                pl.slot_cnt[sb + pos] = c;
                pl.slot_P[sb + pos] = p;
                if (fused) {
                    float best = -3.402823466e38f;
                    int barg = 0;
                    for (int ap = 0; ap < 5; ++ap) {
                        const float mq = z < B ? S.histq[(a * Bm + z) * 5 + ap] : S.tot[10 + a * 5 + ap];
                        const float v = fmaf(acc - eta, mq, eta * S.T[a * 5 + ap]) / p;
                        if (v > best) {
                            best = v;
                            barg = ap;
                        }
                    }
                    pl.slot_val[sb + pos] = best;
                    pl.slot_arg[sb + pos] = barg;
                    S.C[a * nz + z] = best;  // the CDF is no longer read: it holds the leaf values now
                }
            }
            psum += warp_sum(c > 0 ? p : 0.0f);
            base += __popc(bal);
        }
        base = 0;
        float sv = 0.0f;  // sum of weight * leaf value over this action's children
        for (int zc = 0; zc < nz; zc += 32) {
            const int z = zc + lane;
            const int c = z < nz ? S.cnt[a * nz + z] : 0;
            const unsigned bal = __ballot_sync(0xffffffffu, c > 0);
            const int pos = base + __popc(bal & ((1u << lane) - 1u));
            if (c > 0 && QV_IN_BOUNDS(kSiteSlot, pos, K)) {
                const float wgt = pl.weight_mode == QV_WEIGHT_MARGINAL ? S.P[a * nz + z] / psum
                                                                        : static_cast<float>(c) / K;
                pl.slot_w[sb + pos] = wgt;
                if (fused) sv += wgt * S.C[a * nz + z];
            }
            base += __popc(bal);
        }
        if (lane == 0) pl.nchild[iid * 5 + a] = base;
        if (fused) {
            // children in ascending z, as the backup sums them
            const float total = warp_sum(sv);
            if (lane == 0) {
                const float uq = fmaf(ep.gamma, total, S.tot[5 + a] - 100.0f * bgoal);
                pl.UQ[iid * 5 + a] = uq;
                S.uq[a] = uq;
            }
        }
    }
    __syncthreads();
    if (fused && threadIdx.x == 0 && QV_IN_BOUNDS(kSiteNode, ep.node_base[l] + local, pl.n_nodes)) {
        float best = S.uq[0];
        for (int a = 1; a < 5; ++a) best = fmaxf(best, S.uq[a]);
        pl.value[ep.node_base[l] + local] = best;
    }
    __syncthreads();
}

// Number the children of every node of episode e at level l in (parent,
// action, z) order: prefix sum of the unique-sample counts, and for every
// child the slot of its sample record.  The child's own records are written
// by whoever first reads the child (the next expand phase, or the backup).
__device__ void compact_episode(const PlanDev &pl, int l, const EpDev &ep, int e, Smem &S) {
    const int n = __ldcg(pl.count + l * pl.E + e);
    const int M = n * 5;
    const long long ia = static_cast<long long>(ep.inode_base[l]) * 5;
    const int K = pl.K;
    const int cap = ep.cap[l + 1];
    int running = 0;
    for (int base = 0; base < M; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const int v = i < M ? __ldcg(pl.nchild + ia + i) : 0;
        int total;
        const int ex = block_exclusive_scan(v, S.scan, total);
        if (i < M && QV_IN_BOUNDS(kSiteChild, ia + i, 5 * pl.n_inodes)) {
            const int off = running + ex;
            pl.choff[ia + i] = off;
            for (int j = 0; j < v; ++j)
                if (off + j < cap && QV_IN_BOUNDS(kSiteChild, ep.node_base[l + 1] + off + j, pl.n_nodes))
                    pl.src_slot[ep.node_base[l + 1] + off + j] = (ia + i) * K + j;
        }
        running += total;
    }
    int nn = running;
    if (nn > cap) {
        if (threadIdx.x == 0) atomicOr(pl.status, kErrCapacity);
        nn = cap;
    }
    if (threadIdx.x == 0 && QV_IN_BOUNDS(kSiteEpisode, (l + 1) * pl.E + e, (pl.depth + 1) * pl.E))
        pl.count[(l + 1) * pl.E + e] = nn;
    __syncthreads();
}

// Finalize chunks per node of a level of n nodes: several beacon chunks
// (at least one beacon per warp each) when the level holds fewer nodes than
// the grid has work items, so that small levels spread their label
// histograms over the grid.
__host__ __device__ __forceinline__ int finalize_chunks(long long n, int target, int Bmax) {
    if (n <= 0 || n * 2 > target) return 1;
    const long long c = static_cast<long long>(target) / n;
    const int cap = (Bmax + kWarps - 1) / kWarps;
    return static_cast<int>(c < cap ? c : cap);
}

// Work items of one expand group: in proportion to its children, at least
// one; an item takes a range of the window's bands and a part of the
// group's children (at least two), so at most bands x children / 2.
__host__ __device__ __forceinline__ int group_items(int children, long long all_children, int target, int bands) {
    if (children <= 0) return 0;
    const long long want = (static_cast<long long>(target) * children + all_children - 1) / all_children;
    const long long cap = static_cast<long long>(bands) * (children / 2 > 1 ? children / 2 : 1);
    return static_cast<int>(want < 1 ? 1 : (want > cap ? cap : want));
}
// The requested items of a group over nb bands: bi band ranges times
// `parts` parts of the children (an empty window: one item).
__host__ __device__ __forceinline__ void group_split(int requested, int nb, int &bi, int &parts) {
    if (nb <= 0 || requested <= 1) {
        bi = 1;
        parts = 1;
        return;
    }
    bi = requested < nb ? requested : nb;
    parts = requested / bi;
}

// The work lists of level l1 once every node of level l1 - 1 is final and
// its children are numbered (one CTA):
//  - npre[l1]: exclusive prefix of the level sizes over the episodes;
//  - finalize (l1 < depth): fchunks[l1] beacon chunks per node, wb_fin[l1];
//  - expand (l1 < depth): one group per V-node of level l1 - 1, its band
//    ranges in proportion to its children (group_items), the item prefix
//    and, for groups of several items, their first total record;
//  - update (materialised leaves): about `target` items per level;
//  - leaf (l1 = depth): groups of kLeafGroup leaves split into chunks.
__device__ void level_prefix(const PlanDev &pl, int l1, Smem &S) {
    const int E = pl.E;
    // level sizes: totals, prefix over the episodes, leaf groups
    int T = 0, Gl = 0;
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        const int c = __ldcg(pl.count + l1 * E + e);
        T += c;
        Gl += (c + kLeafGroup - 1) / kLeafGroup;
    }
    int Tt, Gt;
    block_exclusive_scan(T, S.scan, Tt);
    block_exclusive_scan(Gl, S.scan, Gt);
    const long long want = Tt > 0 ? max(static_cast<long long>(pl.target) / Tt, 1LL) : 1;
    int C = 1;  // leaf chunks per group of leaves
    if (l1 == pl.depth) {
        C = static_cast<int>(min(max(Gt > 0 ? static_cast<long long>(pl.target) / Gt : 1LL, 1LL), 64LL));
        if (threadIdx.x == 0) *pl.leaf_split = C;
    }
    const int fch = l1 < pl.depth ? finalize_chunks(Tt, pl.target, pl.Bmax) : 1;
    // the fused mode's deepest level with one beacon chunk per node takes
    // finalize items per group (a V-node of level l1 - 1 and a piece of its
    // children, finalize_group_item), flagged by zero chunks
    const bool grp_mode = l1 >= 1 && l1 == pl.depth - 1 && pl.leaf_mode == QV_LEAF_FUSED && fch == 1;
    if (threadIdx.x == 0 && l1 < pl.depth) pl.fchunks[l1] = grp_mode ? 0 : fch;
    int wn = 0, wu = 0, wl = 0;
    for (int base = 0; base < E; base += blockDim.x) {
        const int e = base + threadIdx.x;
        int vn = 0, vu = 0, vl = 0, it = 0;
        if (e < E) {
            const int c = __ldcg(pl.count + l1 * E + e);
            const int bands = __ldg(&pl.eps[e].bands);
            it = static_cast<int>(min(max(want, 1LL), static_cast<long long>(bands)));
            vn = c;
            vu = c * it;
            vl = ((c + kLeafGroup - 1) / kLeafGroup) * C;
        }
        int tn, tu, tl;
        const int xn = block_exclusive_scan(vn, S.scan, tn);
        const int xu = block_exclusive_scan(vu, S.scan, tu);
        const int xl = block_exclusive_scan(vl, S.scan, tl);
        if (e < E) {
            pl.npre[l1 * (E + 1) + e] = wn + xn;
            if (l1 < pl.depth)
                pl.wb_fin[l1 * (E + 1) + e] = grp_mode ? __ldcg(pl.npre + (l1 - 1) * (E + 1) + e) : (wn + xn) * fch;
            pl.uitems[l1 * E + e] = it;
            pl.wb_upd[l1 * (E + 1) + e] = wu + xu;
            if (l1 == pl.depth) pl.wb_leaf[e] = wl + xl;
        }
        wn += tn;
        wu += tu;
        wl += tl;
    }
    if (threadIdx.x == 0) {
        pl.npre[l1 * (E + 1) + E] = wn;
        if (l1 < pl.depth)
            pl.wb_fin[l1 * (E + 1) + E] = grp_mode ? __ldcg(pl.npre + (l1 - 1) * (E + 1) + E) : wn * fch;
        pl.wb_upd[l1 * (E + 1) + E] = wu;
        if (l1 == pl.depth) pl.wb_leaf[E] = wl;
    }
    if (l1 >= pl.depth || l1 < 1) return;
    // expand groups of level l1: the V-nodes of level l1 - 1 with their children
    __syncthreads();
    const int *np = pl.npre + (l1 - 1) * (E + 1);
    const int G = __ldcg(np + E);
    int *goff = pl.grp_off + pl.gbase[l1] + l1;
    int *grec = pl.grp_rec + pl.gbase[l1];
    // the per-episode inputs of the lists, read once into the band buffers
    // (free in a finalize item once its node is final) when they fit: the
    // level sizes' prefix, internal-node bases, child counts, band counts
    // and the support window's rows and cells, so that no group search or
    // window needs a chain of global loads
    int *s_np = reinterpret_cast<int *>(S.sb), *s_ib = s_np + (E + 1), *s_cnt = s_ib + E, *s_nb = s_cnt + E;
    int *s_rows = s_nb + E, *s_cells = s_rows + E;
    const bool cache = 6 * (E + 1) <= S.nband;
    if (cache) {
        for (int e = threadIdx.x; e <= E; e += blockDim.x) {
            s_np[e] = __ldcg(np + e);
            if (e < E) {
                const EpDev *ep = pl.eps + e;
                const int H = __ldg(&ep->H), W = __ldg(&ep->W);
                s_ib[e] = __ldg(&ep->inode_base[l1 - 1]);
                s_cnt[e] = __ldcg(pl.count + l1 * E + e);
                s_nb[e] = band_geo(pl, e, H, W, __ldg(&ep->P), __ldg(&ep->band_rows), l1).nb;
                const Win v = support_window(pl, e, H, W, l1);
                s_rows[e] = max(0, v.r1 - v.r0);
                s_cells[e] = max(0, v.r1 - v.r0) * max(0, v.c1 - v.c0);
            }
        }
        __syncthreads();
    }
    auto children = [&](int j) {
        int e, lp, ib, cnt, nb;
        if (cache) {
            int lo = 0, hi = E - 1;  // last e with s_np[e] <= j
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_np[mid] <= j) lo = mid;
                else hi = mid - 1;
            }
            e = lo;
            lp = j - s_np[e];
            ib = s_ib[e];
            cnt = s_cnt[e];
            nb = s_nb[e];
        } else {
            e = find_episode(np, E, j);
            lp = j - __ldcg(np + e);
            const EpDev *ep = pl.eps + e;
            ib = __ldg(&ep->inode_base[l1 - 1]);
            cnt = __ldcg(pl.count + l1 * E + e);
            nb = band_geo(pl, e, __ldg(&ep->H), __ldg(&ep->W), __ldg(&ep->P), __ldg(&ep->band_rows), l1).nb;
        }
        const long long ia = static_cast<long long>(ib + lp) * 5;
        const int c0 = min(__ldcg(pl.choff + ia), cnt);
        const int c1 = min(__ldcg(pl.choff + ia + 4) + __ldcg(pl.nchild + ia + 4), cnt);
        return make_int2(max(0, c1 - c0), max(nb, 1));  // an empty window still writes its zero totals
    };
    // (the deepest fused level in its contraction form cuts its finalize
    // pieces by these items: two per CTA, whatever the items per CTA)
    const int gtarget = (pl.ctr && l1 == pl.depth - 1 && pl.leaf_mode == QV_LEAF_FUSED)
                            ? max(pl.target, 2 * static_cast<int>(gridDim.x))
                            : pl.target;
    int wi = 0, wr = 0;
    for (int base = 0; base < G; base += blockDim.x) {
        const int j = base + threadIdx.x;
        int vi = 0, vr = 0;
        if (j < G) {
            const int2 cb = children(j);
            vi = group_items(cb.x, Tt, gtarget, cb.y);
            vr = vi >= 2 ? vi : 0;
        }
        int ti, tr;
        const int xi = block_exclusive_scan(vi, S.scan, ti);
        const int xr = block_exclusive_scan(vr, S.scan, tr);
        if (j < G) {
            goff[j] = wi + xi;
            grec[j] = vr ? wr + xr : -1;
        }
        wi += ti;
        wr += tr;
    }
    if (threadIdx.x == 0) {
        goff[G] = wi;
        pl.ngrp[l1] = G;
        // group mode: one finalize item per expand item, a group's children
        // cut into as many pieces as it has expand items
        if (grp_mode) pl.wb_fin[l1 * (E + 1) + E] = wi;
    }
    // the contraction form of the deepest fused level (ctr_item) in place of
    // the group expand items: per episode, work items in proportion to its
    // children times its window's cells (at least one, at most one per
    // window row), all of them within the total records xrec holds; when
    // they cannot fit, the level keeps the group expand items
    bool groups = true;  // the level's expand runs as group items
    if (pl.ctr && l1 == pl.depth - 1 && pl.leaf_mode == QV_LEAF_FUSED) {
        unsigned long long *wsum = reinterpret_cast<unsigned long long *>(S.red);
        __syncthreads();
        if (threadIdx.x < 2) wsum[threadIdx.x] = 0ull;
        __syncthreads();
        auto geom = [&](int e, long long &n, long long &rows, long long &cells) {
            if (cache) {
                n = s_cnt[e];
                rows = s_rows[e];
                cells = s_cells[e];
                return;
            }
            const EpDev *ep = pl.eps + e;
            const Win v = support_window(pl, e, __ldg(&ep->H), __ldg(&ep->W), l1);
            n = __ldcg(pl.count + l1 * E + e);
            rows = max(0, v.r1 - v.r0);
            cells = rows * max(0, v.c1 - v.c0);
        };
        unsigned long long wl = 0;
        for (int e = threadIdx.x; e < E; e += blockDim.x) {
            long long n, rows, cells;
            geom(e, n, rows, cells);
            wl += static_cast<unsigned long long>(n * max(cells, 1LL));
        }
        atomicAdd(wsum, wl);  // integer sums: the same items whatever the order
        __syncthreads();
        const unsigned long long wt = max(wsum[0], 1ull);
        // items of episode e, scaled by num / den when den > 0: two per CTA
        // over the level (the items are alike, so two waves balance them),
        // whatever the launch shape's items per CTA
        const unsigned long long ctarget = 2ull * gridDim.x;
        auto items_of = [&](int e, unsigned long long num, unsigned long long den) -> long long {
            long long n, rows, cells;
            geom(e, n, rows, cells);
            if (n <= 0) return 0;
            const unsigned long long w = static_cast<unsigned long long>(n * max(cells, 1LL));
            long long it = static_cast<long long>((ctarget * w + wt - 1) / wt);
            it = min(max(it, 1LL), max(rows, 1LL));
            if (den > 0) it = max(1LL, static_cast<long long>(static_cast<unsigned long long>(it) * num / den));
            return it;
        };
        unsigned long long rl = 0;
        for (int e = threadIdx.x; e < E; e += blockDim.x) {
            long long n, rows, cells;
            geom(e, n, rows, cells);
            rl += static_cast<unsigned long long>(items_of(e, 0, 0) * n);
        }
        atomicAdd(wsum + 1, rl);
        __syncthreads();
        const unsigned long long r0 = wsum[1], cap = static_cast<unsigned long long>(max(pl.n_xrec, 0));
        const unsigned long long num = r0 > cap ? cap : 0ull, den = r0 > cap ? r0 : 0ull;
        __syncthreads();
        if (threadIdx.x == 0) wsum[1] = 0ull;
        __syncthreads();
        rl = 0;
        for (int e = threadIdx.x; e < E; e += blockDim.x) {
            long long n, rows, cells;
            geom(e, n, rows, cells);
            rl += static_cast<unsigned long long>(items_of(e, num, den) * n);
        }
        atomicAdd(wsum + 1, rl);
        __syncthreads();
        const bool fits = wsum[1] <= cap;
        groups = !fits;
        int ci = 0, cr = 0;
        for (int base = 0; base < E; base += blockDim.x) {
            const int e = base + threadIdx.x;
            int vi = 0, vr = 0;
            if (e < E && fits) {
                long long n, rows, cells;
                geom(e, n, rows, cells);
                vi = static_cast<int>(items_of(e, num, den));
                vr = static_cast<int>(vi * n);
            }
            int ti, tr;
            const int xi = block_exclusive_scan(vi, S.scan, ti);
            const int xr = block_exclusive_scan(vr, S.scan, tr);
            if (e < E) {
                pl.c_items[e] = ci + xi;
                pl.c_rbase[e] = cr + xr;
            }
            ci += ti;
            cr += tr;
        }
        if (threadIdx.x == 0) {
            pl.c_items[E] = ci;
            pl.c_mode[0] = fits ? 1 : 0;
        }
    }
    if (threadIdx.x == 0 && groups && static_cast<long long>(wr) * pl.cmax > pl.n_xrec) atomicOr(pl.status, kErrCapacity);
}

// A node of episode e at level l is final: the last one numbers the
// episode's children, the last episode publishes the next level.
__device__ void node_done(const PlanDev &pl, int l, int e, const EpDev &ep, Smem &S) {
    if (threadIdx.x == 0) {
        const int n = __ldcg(pl.count + l * pl.E + e);
        const unsigned prev = arrive_acq_rel(pl.ep_cnt + l * pl.E + e);
        const int last = prev == static_cast<unsigned>(n - 1);
        if (last) pl.ep_cnt[l * pl.E + e] = 0u;
        S.flags[1] = last;
    }
    __syncthreads();
    if (!S.flags[1]) return;
    compact_episode(pl, l, ep, e, S);
    if (pl.E > 1) {  // with one episode its last node is the level's last
        if (threadIdx.x == 0) {
            const unsigned prev = arrive_acq_rel(pl.lvl_cnt + l);
            const int last = prev == static_cast<unsigned>(pl.E - 1);
            if (last) pl.lvl_cnt[l] = 0u;
            S.flags[2] = last;
        }
        __syncthreads();
        if (!S.flags[2]) return;
    }
    level_prefix(pl, l + 1, S);
    __syncthreads();
}

// ---------------------------------------------------------------- window phase
// The support window of every episode's b0: the bounding box of its nonzero
// cells, one streaming read of b0 before the root's pass.  Each episode's
// float4 groups are split over gridDim / E CTAs (one CTA per episode when
// E >= gridDim); a CTA reduces its share and merges it with four atomicMax.
// (A float4 never straddles two rows: the pitch is a multiple of 8.)
__device__ void phase_window(const PlanDev &pl, Smem &S) {
    const int E = pl.E, G = gridDim.x;
    const int per = max(1, G / E);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned *red = reinterpret_cast<unsigned *>(S.red);
    for (int v = blockIdx.x; v < E * per; v += G) {
        const int e = v / per, part = v - e * per;
        const EpDev *ep = pl.eps + e;
        const int H = __ldg(&ep->H), P = __ldg(&ep->P);
        const float4 *b4 = reinterpret_cast<const float4 *>(ep->b0);
        const long long n4 = static_cast<long long>(H) * P / 4;
        const long long i0 = n4 * part / per, i1 = n4 * (part + 1) / per;
        unsigned wr0 = 0u, wr1 = 0u, wc0 = 0u, wc1 = 0u;
        for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
            const float4 x = __ldcs(b4 + i);
            const float xs[4] = {x.x, x.y, x.z, x.w};
            const int row = static_cast<int>((4 * i) / P), col = static_cast<int>(4 * i - static_cast<long long>(row) * P);
#pragma unroll
            for (int jj = 0; jj < 4; ++jj)
                if (xs[jj] != 0.0f) {
                    wr0 = max(wr0, static_cast<unsigned>(kWinBig - row));
                    wr1 = max(wr1, static_cast<unsigned>(row + 1));
                    wc0 = max(wc0, static_cast<unsigned>(kWinBig - (col + jj)));
                    wc1 = max(wc1, static_cast<unsigned>(col + jj + 1));
                }
        }
        wr0 = __reduce_max_sync(0xffffffffu, wr0);
        wr1 = __reduce_max_sync(0xffffffffu, wr1);
        wc0 = __reduce_max_sync(0xffffffffu, wc0);
        wc1 = __reduce_max_sync(0xffffffffu, wc1);
        __syncthreads();  // the previous episode's reader of red is done
        if (lane == 0) {
            red[wid * 4] = wr0;
            red[wid * 4 + 1] = wr1;
            red[wid * 4 + 2] = wc0;
            red[wid * 4 + 3] = wc1;
        }
        __syncthreads();
        if (threadIdx.x < 4) {
            unsigned m = 0u;
            for (int k = 0; k < kWarps; ++k) m = max(m, red[k * 4 + threadIdx.x]);
            if (m != 0u) atomicMax(pl.win + 4 * e + threadIdx.x, m);
        }
    }
}

// ---------------------------------------------------------------- expand phase
// A node's belief at four cells (grid row r, columns col..col+3) from its
// parent's staged band: Phi(parent, a, z) of Eq. 3, zero outside the grid.
// `m` points at the staged parent value of (r, col), `c` at its cell word;
// staged rows are SW values apart.
__device__ __forceinline__ float4 child4(const EpReg &ep, const float *m, const uint16_t *c, int SW, int r, int col,
                                         int a, int z, float sa, float se, const float *lut) {
    const int P = ep.P;
    if (r < 0 || r >= ep.H || col >= P) return make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 up = *reinterpret_cast<const float4 *>(m - SW);
    const float4 md = *reinterpret_cast<const float4 *>(m);
    const float4 dn = *reinterpret_cast<const float4 *>(m + SW);
    const float u[4] = {up.x, up.y, up.z, up.w}, d[4] = {dn.x, dn.y, dn.z, dn.w};
    const float mm[6] = {col > 0 ? m[-1] : 0.0f, md.x, md.y, md.z, md.w, col + 4 < P ? m[4] : 0.0f};
    const ushort4 c4 = *reinterpret_cast<const ushort4 *>(c);
    const unsigned cws[4] = {c4.x, c4.y, c4.z, c4.w};
    float v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const unsigned in = QV_CELL_INFLOW(cws[j]);
        float nb[4];
        nb[kDirN] = (in & 1u) ? u[j] : 0.0f;
        nb[kDirE] = (in & 2u) ? mm[j + 2] : 0.0f;
        nb[kDirS] = (in & 4u) ? d[j] : 0.0f;
        nb[kDirW] = (in & 8u) ? mm[j] : 0.0f;
        const float p = predict_one(nb, mm[j + 1], cws[j], r * P + col + j == ep.goal, ep.slip, lut, a);
        v[j] = p * (static_cast<int>(QV_CELL_LABEL(cws[j])) == z ? sa : se);
    }
    return make_float4(v[0], v[1], v[2], v[3]);
}

// child4 where no cell within two rows is the goal and the staged parent is
// zero on occupied cells (the expand items mask it once per band): every
// neighbour then moves its mass in without the inflow test, and the
// blocked moves' mass stays by the self weight of the action.
__device__ __forceinline__ float4 child4_open(const EpReg &ep, const float *m, const uint16_t *c, int SW, int col,
                                              int a, int z, float sa, float se, const float *lut) {
    const int P = ep.P;
    const float4 up = *reinterpret_cast<const float4 *>(m - SW);
    const float4 md = *reinterpret_cast<const float4 *>(m);
    const float4 dn = *reinterpret_cast<const float4 *>(m + SW);
    const float west = col > 0 ? m[-1] : 0.0f;
    const float east = col + 4 < P ? m[4] : 0.0f;
    const ushort4 c4 = *reinterpret_cast<const ushort4 *>(c);
    const float fwd = 1.0f - 2.0f * ep.slip, slip = ep.slip;
    const float u[4] = {up.x, up.y, up.z, up.w}, d[4] = {dn.x, dn.y, dn.z, dn.w};
    const float mm[6] = {west, md.x, md.y, md.z, md.w, east};
    const unsigned cws[4] = {c4.x, c4.y, c4.z, c4.w};
    float v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const unsigned w = cws[j];
        float p;
        if (a == 4) {
            p = mm[j + 1];
        } else {
            // intended move from the neighbour opposite a's step, slips from
            // the two perpendicular ones (a uniform over the warp)
            const float n_in = a == 0 ? d[j] : a == 1 ? mm[j] : a == 2 ? u[j] : mm[j + 2];
            const float n_pp = (a & 1) ? u[j] + d[j] : mm[j] + mm[j + 2];
            p = fmaf(lut[a * 16 + QV_CELL_BLOCKED(w)], mm[j + 1], fmaf(fwd, n_in, slip * n_pp));
        }
        const float o = static_cast<int>(QV_CELL_LABEL(w)) == z ? sa : se;
        v[j] = QV_CELL_FREE(w) ? p * o : 0.0f;
    }
    return make_float4(v[0], v[1], v[2], v[3]);
}

// The same at one cell (grid row r, column c; `m`, `cw` its staged value and
// word), for the edge of a column strip.
__device__ __forceinline__ float child1(const EpReg &ep, const float *m, const uint16_t *cwp, int SW, int r, int c,
                                        int a, int z, float sa, float se, const float *lut) {
    const int P = ep.P;
    if (r < 0 || r >= ep.H || c < 0 || c >= P) return 0.0f;
    const unsigned w = *cwp;
    const unsigned in = QV_CELL_INFLOW(w);
    float nb[4];
    nb[kDirN] = (in & 1u) ? m[-SW] : 0.0f;
    nb[kDirE] = (in & 2u) ? m[1] : 0.0f;
    nb[kDirS] = (in & 4u) ? m[SW] : 0.0f;
    nb[kDirW] = (in & 8u) ? m[-1] : 0.0f;
    const float p = predict_one(nb, m[0], w, r * P + c == ep.goal, ep.slip, lut, a);
    return p * (static_cast<int>(QV_CELL_LABEL(w)) == z ? sa : se);
}

// Work items are (group, band range).  A group is one V-node of level l - 1
// with all its children at level l (at l = 0, the root of one episode), so
// the parent's band, the cell words and (fused level) Q are staged once per
// band for every child.  Within a band the (child, column strip of 128
// cells, row) tasks are split into eight contiguous ranges, one per warp, so
// that each warp streams rows on its own: per row, each lane forms the
// child's belief at its four cells (Phi(parent, a, z), Eq. 3; written out
// when a later phase reads it) rolling three rows in registers, takes the
// row's east/west neighbours from the adjacent lanes, and applies the motion
// stencil for all five actions (Eq. 3 numerator, Eq. 10), summing the
// null-label masses, the rewards (Sec. III) and, at the fused level, the
// Q-weighted null masses in registers.  A warp's sums go to a per-warp slot
// when its task range moves to another child; at the end of the band the
// slots are added into each child's totals in warp order.  Cells with a
// beacon's label enter through the finalize items' tiles.
// One expand work item w of level l (false when a wait gave up).  With
// `signal` the item also counts itself done on its group's counter
// (grp_done), which the fused level's finalize items wait on.
template <bool FUSED>
__device__ bool expand_item(const PlanDev &pl, int l, bool store, Smem &S, uint64_t *mbar, unsigned &mphase,
                            int &cur_e, int w, bool signal) {
    const int E = pl.E, K = pl.K;
    const int G = __ldcg(pl.ngrp + l);
    const int *goff = pl.grp_off + pl.gbase[l] + l;
    const int *grec = pl.grp_rec + pl.gbase[l];
    const int *np = l > 0 ? pl.npre + (l - 1) * (E + 1) : nullptr;
    const int KS = pl.kslots;
    constexpr int NV = FUSED ? 35 : 10;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    {
#ifdef QV_TRACE
        unsigned long long tr[kTraceWords] = {};
#endif
        QV_TRACE_MARK(tr, 2);
        const int j = block_find(goff, G, w, S.flags + 6);
        if (!QV_IN_BOUNDS(kSiteGroup, pl.gbase[l] + j, pl.ngrp_cap)) return true;  // uniform over the CTA
        int e = j, lp = 0;
        if (l > 0) {
            e = block_find(np, E, j, S.flags + 7);
            lp = j - __ldcg(np + e);
        }
        const int g0 = __ldcg(goff + j);
        const int item = w - g0;
        // a group's items are bi band ranges times `parts` parts of its
        // children (at least one item, which writes the zero totals of an
        // empty window); surplus items of the list do nothing
        const EpDev *epg = pl.eps + e;
        const BandGeo geo =
            band_geo(pl, e, __ldg(&epg->H), __ldg(&epg->W), __ldg(&epg->P), __ldg(&epg->band_rows), l);
        int bi, parts;
        group_split(__ldcg(goff + j + 1) - g0, geo.nb, bi, parts);
        const int items = bi * parts;
        if (item >= items) return true;
        const int bslot = item % bi, part = item / bi;
        load_ep(pl, e, S, cur_e);
        const EpDev &ep = *S.ep;
        const int rec = __ldcg(grec + j);
        const int B = ep.B;
        int c0 = 0, nc = 1;
        const float *src = ep.b0;
        if (l > 0) {
            const long long ia = static_cast<long long>(ep.inode_base[l - 1] + lp) * 5;
            if (!QV_IN_BOUNDS(kSiteInode, ep.inode_base[l - 1] + lp, pl.n_inodes)) return true;
            const int cnt = __ldcg(pl.count + l * E + e);
            c0 = min(__ldcg(pl.choff + ia), cnt);
            const int c1 = min(__ldcg(pl.choff + ia + 4) + __ldcg(pl.nchild + ia + 4), cnt);
            nc = min(max(0, c1 - c0), pl.cmax);
            src = node_belief(pl, ep, l - 1, lp);
        }
        __syncthreads();  // the previous item's readers of the child table, totals and band buffers are done
        const int band0 = static_cast<int>((static_cast<long long>(bslot) * geo.nb) / bi);
        const int band1 = static_cast<int>((static_cast<long long>(bslot + 1) * geo.nb) / bi);
        // this item's part of the group's children
        const int cp0 = static_cast<int>((static_cast<long long>(part) * nc) / parts);
        const int ncp = static_cast<int>((static_cast<long long>(part + 1) * nc) / parts) - cp0;
        const EpReg er = ep_reg(ep);
        // the first band's copies fly while the child table is read
        if (band0 < band1) {
            const int r0 = geo.r0 + band0 * geo.rows, r1 = min(geo.r1, r0 + geo.rows);
            stage_issue(er, src, r0, r1, geo.sc0, geo.sw, S.sp, S.cw, FUSED ? S.q : nullptr, mbar);
        }
        if (l > 0) {
            for (int r = threadIdx.x; r < nc; r += blockDim.x) {
                const int gid = ep.node_base[l] + c0 + r;
                if (!QV_IN_BOUNDS(kSiteNode, gid, pl.n_nodes)) {
                    S.c_pa[r] = 0;
                    S.c_z[r] = 0;
                    S.c_sa[r] = S.c_se[r] = 0.0f;
                    continue;
                }
                // the child's sample record in its parent's arrays: (iid_p * 5 + a) * K + j
                const long long s = __ldcg(pl.src_slot + gid);
                if (!QV_IN_BOUNDS(kSiteSlot, s, 5 * K * pl.n_inodes)) {
                    S.c_pa[r] = 0;
                    S.c_z[r] = 0;
                    S.c_sa[r] = S.c_se[r] = 0.0f;
                    continue;
                }
                const int a = static_cast<int>((s / K) % 5);
                const int z = __ldcg(pl.slot_z + s);
                const float p = __ldcg(pl.slot_P + s);
                S.c_pa[r] = a;
                S.c_z[r] = z;
                S.c_sa[r] = ep.acc / p;
                S.c_se[r] = ep.eta / p;
                if (item == 0) {
                    const unsigned long long pcode = __ldcg(pl.code + ep.node_base[l - 1] + lp);
                    pl.parent[gid] = lp;
                    pl.action[gid] = a;
                    pl.obs[gid] = z;
                    pl.weight[gid] = __ldcg(pl.slot_w + s);
                    pl.pz[gid] = p;
                    pl.code[gid] = (pcode * 5ull + a) * static_cast<unsigned long long>(B + 1) + z;
                }
            }
        }
        for (int i = threadIdx.x; i < nc * kTot; i += blockDim.x) S.acc[i] = 0.0f;
        __syncthreads();
        QV_TRACE_MARK(tr, 3);
        const int P = er.P, goal = er.goal, SW = geo.sw;
        const int NS = (geo.g1 - geo.g0 + 31) >> 5;  // column strips of 32 float4 groups
        const float slip = er.slip;
        const float *cost = er.cost;
        float *dst0 = (l > 0 && store) ? pl.beliefs + ep.belief_off[l] : nullptr;
        if (dst0 && !QV_IN_BOUNDS(kSiteBelief, ep.belief_off[l] + static_cast<long long>(c0 + nc) * ep.N - 1,
                                  pl.n_belief))
            dst0 = nullptr;  // debug build: the children are not stored
        for (int band = band0; band < band1; ++band) {
            const int r0 = geo.r0 + band * geo.rows, r1 = min(geo.r1, r0 + geo.rows), R = r1 - r0;
            const int qstride = R * SW;
            if (band > band0) {
                __syncthreads();  // the previous band's readers are done
                stage_issue(er, src, r0, r1, geo.sc0, SW, S.sp, S.cw, FUSED ? S.q : nullptr, mbar);
            }
            if (!stage_wait(mbar, mphase, pl.status)) return false;
            // occupied cells of the staged parent (or root) carry no belief:
            // zero them once, so that rows away from the goal can move every
            // neighbour's mass without the per-cell inflow test
            {
                const int lo = max(0, r0 - 2) - (r0 - 2), hi = min(er.H, r1 + 2) - (r0 - 2);
                for (int i = lo * SW + threadIdx.x; i < hi * SW; i += blockDim.x)
                    if (!QV_CELL_FREE(static_cast<unsigned>(S.cw[i]))) S.sp[i] = 0.0f;
                __syncthreads();
            }
            if (band == band0) QV_TRACE_MARK(tr, 4);
            // this warp's contiguous range of (child, strip, row) tasks over the item's children
            const int T = ncp * NS * R;
            int t = static_cast<int>(static_cast<long long>(T) * wid / kWarps);
            const int tend = static_cast<int>(static_cast<long long>(T) * (wid + 1) / kWarps);
            int slot = 0, cur = -1;
            float acc_null[5], acc_r[5], acc_q[FUSED ? 25 : 1];
            auto zero_acc = [&]() {
#pragma unroll
                for (int a = 0; a < 5; ++a) acc_null[a] = acc_r[a] = 0.0f;
#pragma unroll
                for (int i = 0; i < (FUSED ? 25 : 1); ++i) acc_q[i] = 0.0f;
            };
            // the warp's sums of child `cur` into its next slot: values 0..31
            // by a reduce-scatter (lane i gets value i), 32..34 by warp sums
            auto flush = [&]() {
                float v[32];
#pragma unroll
                for (int a = 0; a < 5; ++a) {
                    v[a] = acc_null[a];
                    v[5 + a] = acc_r[a];
                }
#pragma unroll
                for (int i = 0; i < 22; ++i) {
                    if constexpr (FUSED) v[10 + i] = acc_q[i];
                    else v[10 + i] = 0.0f;
                }
                warp_reduce_scatter32(v);
                if (slot >= KS) {  // cannot happen (expand_slots); reported, never written past
                    if (lane == 0) atomicOr(pl.status, kErrCapacity);
                    return;
                }
                float *dstp = S.wpart + (wid * KS + slot) * kTot;
                dstp[lane] = v[0];
                if constexpr (FUSED) {
#pragma unroll
                    for (int i = 22; i < 25; ++i) {
                        const float tt = warp_sum(acc_q[i]);
                        if (lane == 0) dstp[10 + i] = tt;
                    }
                }
                if (lane == 0) S.wchild[wid * KS + slot] = cur;
                ++slot;
            };
            const int grow = goal / P;
            const float fwd = 1.0f - 2.0f * slip;
            zero_acc();
            while (t < tend) {
                const int r = cp0 + t / (NS * R);
                const int rem = t - (r - cp0) * NS * R;
                const int s = rem / R, ya = rem - s * R;
                const int yb = min(R, ya + (tend - t));
                if (r != cur) {
                    if (cur >= 0) flush();
                    zero_acc();
                    cur = r;
                }
                int pa = 0, pz = 0;
                float sa = 1.0f, se = 1.0f;
                if (l > 0) {
                    pa = S.c_pa[r];
                    pz = S.c_z[r];
                    sa = S.c_sa[r];
                    se = S.c_se[r];
                }
                const int gcol = geo.g0 + s * 32 + lane;
                const bool act = gcol < geo.g1;
                const int col = gcol << 2, sc = col - geo.sc0;
                float *dst = dst0 ? dst0 + static_cast<long long>(c0 + r) * er.N : nullptr;
                // the node's belief at this lane's four cells of band row y;
                // rows more than one row from the goal's take the open form
                auto row4 = [&](int y) -> float4 {
                    const int rr = r0 + y;
                    if (!act || rr < 0 || rr >= er.H) return make_float4(0.f, 0.f, 0.f, 0.f);
                    const int o = (y + 2) * SW + sc;
                    if (l == 0) return *reinterpret_cast<const float4 *>(S.sp + o);
                    if (abs(rr - grow) >= 2) return child4_open(er, S.sp + o, S.cw + o, SW, col, pa, pz, sa, se, S.lut);
                    return child4(er, S.sp + o, S.cw + o, SW, rr, col, pa, pz, sa, se, S.lut);
                };
                // (c is within the staged columns: the window keeps two
                // columns of reach on each side of its task columns)
                auto row1 = [&](int y, int c) -> float {
                    const int rr = r0 + y, o = (y + 2) * SW + (c - geo.sc0);
                    if (l == 0) return (rr >= 0 && rr < er.H && c >= 0 && c < P) ? S.sp[o] : 0.0f;
                    return child1(er, S.sp + o, S.cw + o, SW, rr, c, pa, pz, sa, se, S.lut);
                };
                float4 up = row4(ya - 1), md = row4(ya);
                // the strip's two edge cells (west of lane 0, east of lane 31),
                // formed for 16 rows at a time by the whole warp: lane k holds
                // row y0 + k / 2, the west edge for even k, the east for odd
                const int scol = (geo.g0 + s * 32) << 2;
                const bool east_in = geo.g0 + s * 32 + 31 < geo.g1;
                float edge = 0.0f;
                for (int y = ya; y < yb; ++y) {
                    const int k = (y - ya) & 15;
                    if (k == 0) {
                        const int ye = y + (lane >> 1);
                        const int c = (lane & 1) ? scol + 128 : scol - 1;
                        edge = (ye < yb && c >= 0 && c < P && ((lane & 1) == 0 || east_in)) ? row1(ye, c) : 0.0f;
                    }
                    const float4 dn = row4(y + 1);
                    // the row's west and east neighbours from the adjacent lanes
                    float hw = __shfl_up_sync(0xffffffffu, md.w, 1);
                    float he = __shfl_down_sync(0xffffffffu, md.x, 1);
                    const float e_w = __shfl_sync(0xffffffffu, edge, 2 * k);
                    const float e_e = __shfl_sync(0xffffffffu, edge, 2 * k + 1);
                    if (lane == 0) hw = e_w;
                    if (lane == 31) he = e_e;
                    if (act) {
                        const int yg = (r0 + y) * P + col;
                        if (dst) *reinterpret_cast<float4 *>(dst + yg) = md;
                        const ushort4 cw4 = *reinterpret_cast<const ushort4 *>(S.cw + (y + 2) * SW + sc);
                        const unsigned cws[4] = {cw4.x, cw4.y, cw4.z, cw4.w};
                        const float ups[4] = {up.x, up.y, up.z, up.w};
                        const float mds[6] = {hw, md.x, md.y, md.z, md.w, he};
                        const float dns[4] = {dn.x, dn.y, dn.z, dn.w};
                        if (abs(r0 + y - grow) >= 2) {
                            // open form: the node's belief is zero on occupied
                            // cells and no cell within a row is the goal, so
                            // every neighbour moves its mass in; occupied cells'
                            // outputs are masked by their reward and null weights
                            const float *qrow = S.q + y * SW + sc;
#pragma unroll
                            for (int jj = 0; jj < 4; ++jj) {
                                const unsigned cw = cws[jj];
                                const float nN = ups[jj], nS = dns[jj], nW = mds[jj], nE = mds[jj + 2];
                                const float sf = mds[jj + 1];
                                const float4 sw = S.lut4[QV_CELL_BLOCKED(cw)];
                                const float ew = slip * (nE + nW), ns = slip * (nN + nS);
                                float out[5];
                                out[0] = fmaf(sw.x, sf, fmaf(fwd, nS, ew));
                                out[1] = fmaf(sw.y, sf, fmaf(fwd, nW, ns));
                                out[2] = fmaf(sw.z, sf, fmaf(fwd, nN, ew));
                                out[3] = fmaf(sw.w, sf, fmaf(fwd, nE, ns));
                                out[4] = sf;
                                const bool fr = QV_CELL_FREE(cw) != 0u;
                                const float cst = cost ? __ldg(cost + yg + jj) : 0.0f;
                                const float rw = fr ? -1.0f - cst : 0.0f;
                                const float nf = (fr && static_cast<int>(QV_CELL_LABEL(cw)) >= B) ? 1.0f : 0.0f;
                                float vn[5];
#pragma unroll
                                for (int a = 0; a < 5; ++a) {
                                    acc_r[a] = fmaf(out[a], rw, acc_r[a]);
                                    vn[a] = out[a] * nf;
                                    acc_null[a] += vn[a];
                                }
                                if constexpr (FUSED) {
                                    // the cell's Q-weighted null masses (one cell at a
                                    // time, so that few values stay live)
#pragma unroll
                                    for (int ap = 0; ap < 5; ++ap) {
                                        const float q = qrow[ap * qstride + jj];
#pragma unroll
                                        for (int a = 0; a < 5; ++a) acc_q[a * 5 + ap] = fmaf(vn[a], q, acc_q[a * 5 + ap]);
                                    }
                                }
                            }
                        } else {
                            // the exact form near the goal: inflow masks and the
                            // goal's own mass staying put
                            const float *qrow = S.q + y * SW + sc;
#pragma unroll
                            for (int jj = 0; jj < 4; ++jj) {
                                const unsigned cw = cws[jj];
                                const unsigned in = QV_CELL_INFLOW(cw);
                                float nb[4], out[5];
                                nb[kDirN] = (in & 1u) ? ups[jj] : 0.0f;
                                nb[kDirE] = (in & 2u) ? mds[jj + 2] : 0.0f;
                                nb[kDirS] = (in & 4u) ? dns[jj] : 0.0f;
                                nb[kDirW] = (in & 8u) ? mds[jj] : 0.0f;
                                predict_cell(nb, mds[jj + 1], cw, (yg + jj) == goal, slip, S.lut, out);
                                const float cst = cost ? __ldg(cost + yg + jj) : 0.0f;
                                const float rw = stage_reward(QV_CELL_FREE(cw), (yg + jj) == goal, cst);
                                const float isnull = static_cast<int>(QV_CELL_LABEL(cw)) >= B ? 1.0f : 0.0f;
                                float qj[5];
                                if constexpr (FUSED) {
#pragma unroll
                                    for (int ap = 0; ap < 5; ++ap) qj[ap] = qrow[ap * qstride + jj];
                                }
#pragma unroll
                                for (int a = 0; a < 5; ++a) {
                                    const float v = out[a];
                                    acc_r[a] = fmaf(v, rw, acc_r[a]);
                                    const float vnn = v * isnull;
                                    acc_null[a] += vnn;
                                    if constexpr (FUSED) {
#pragma unroll
                                        for (int ap = 0; ap < 5; ++ap)
                                            acc_q[a * 5 + ap] = fmaf(vnn, qj[ap], acc_q[a * 5 + ap]);
                                    }
                                }
                            }
                        }
                    }
                    up = md;
                    md = dn;
                }
                t += yb - ya;
            }
            if (cur >= 0) flush();
            for (int sl = slot + lane; sl < KS; sl += 32) S.wchild[wid * KS + sl] = -1;
            __syncthreads();
            if (band == band0) QV_TRACE_MARK(tr, 5);
            // the warps' slots into each child's totals, in (warp, slot) order
            // (a warp's slots hold increasing children, -1 after the last)
            for (int i = threadIdx.x; i < nc * kTot; i += blockDim.x) {
                const int r = i / kTot, v = i - r * kTot;
                if (v >= NV) continue;
                float sum = 0.0f;
                for (int ww = 0; ww < kWarps; ++ww)
                    for (int sl = ww * KS; sl < (ww + 1) * KS; ++sl) {
                        const int c = S.wchild[sl];
                        if (c < 0 || c > r) break;
                        if (c == r) sum += S.wpart[sl * kTot + v];
                    }
                S.acc[i] += sum;
            }
        }
        if (dst0) {
            // the stored children are zero outside the task window: zeros go
            // where an earlier run may have left values (the level's dirty
            // box, nothing when it lies inside the window); this item's share
            // of the box's rows, one warp per (child, row)
            const int *dw = pl.dirty + 4 * (l * E + e);
            const int w0 = __ldcg(dw);
            if (w0 != 0) {
                const int dr0 = w0 - 1, dr1 = __ldcg(dw + 1), dg0 = __ldcg(dw + 2), dg1 = __ldcg(dw + 3);
                const bool inside = geo.nb > 0 && dr0 >= geo.r0 && dr1 <= geo.r1 && dg0 >= geo.g0 && dg1 <= geo.g1;
                if (!inside) {
                    const int zr0 = dr0 + static_cast<int>((static_cast<long long>(bslot) * (dr1 - dr0)) / bi);
                    const int zr1 = dr0 + static_cast<int>((static_cast<long long>(bslot + 1) * (dr1 - dr0)) / bi);
                    const int nr = zr1 - zr0;
                    for (int t2 = wid; t2 < ncp * nr; t2 += kWarps) {
                        const int r = cp0 + t2 / nr, row = zr0 + (t2 - (t2 / nr) * nr);
                        float4 *d4 = reinterpret_cast<float4 *>(dst0 + static_cast<long long>(c0 + r) * er.N +
                                                                static_cast<long long>(row) * P);
                        const bool in = row >= geo.r0 && row < geo.r1;
                        for (int g = dg0 + lane; g < dg1; g += 32)
                            if (!in || g < geo.g0 || g >= geo.g1) d4[g] = make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
            }
        }
        __syncthreads();
        // the item's totals of every child: final when the group has one item,
        // else one record per (item, child) that the finalize item adds in order
        for (int i = threadIdx.x; i < nc * kTot; i += blockDim.x) {
            const int r = i / kTot, k = i - r * kTot;
            const float v = S.acc[i];
            if (rec < 0) {
                pl.ntot[static_cast<long long>(ep.inode_base[l] + c0 + r) * kTot + k] = v;
            } else {
                const long long x = static_cast<long long>(rec + item) * pl.cmax + r;
                if (x < pl.n_xrec) pl.xrec[x * kTot + k] = v;
            }
        }
        QV_TRACE_MARK(tr, 6);
#ifdef QV_TRACE
        tr[0] = 2ull | (static_cast<unsigned long long>(l) << 8) | (static_cast<unsigned long long>(blockIdx.x) << 16) |
                (static_cast<unsigned long long>(nc) << 32) | (static_cast<unsigned long long>(band1 - band0) << 48);
        tr[1] = static_cast<unsigned long long>(w);
        trace_commit(tr, 7);
#endif
        if (signal) {
            __syncthreads();  // every thread's totals are written
            if (threadIdx.x == 0) arrive_acq_rel(pl.grp_done + pl.gbase[l] + j);
        }
    }
    return true;
}

// ---------------------------------------------------------------- label histograms
// For one V-node (belief Phi(parent, a, z), or b0 at the root) and beacon
// k: the five predicted masses sum_{y: label(y) = k} bbar_a(y) (Eq. 3
// denominator) and, fused, the 25 Q-weighted ones sum bbar_a(y) Q(a', y),
// into la / lq of the calling lane.  One warp: the beacon's sensing diamond
// is covered by tiles of kTileH x kTileW cells; per tile the parent's values
// with a two-cell rim and the cell words with a one-cell rim are read into
// the warp's shared buffers (tile_load), the diamond's cells of label k in
// the tile are listed (tile_list), the node's belief is formed on the tile
// with a one-cell rim (tile_form) and the listed cells predict from it
// (tile_predict).  Only the part of the diamond inside `win` (where the
// node's predicted masses can be nonzero) is visited.  The load and the
// list depend on the parent and the beacon only, so every child of one
// parent can reuse them.
struct TileBox {
    int rlo, rhi, clo, chi;  // the diamond's bounding box inside the grid and the window
};
__device__ __forceinline__ TileBox tile_box(const EpReg &ep, int br, int bc, const Win &win) {
    const int R = ep.range;
    TileBox b;
    b.rlo = max(max(0, br - R), win.r0);
    b.rhi = min(min(ep.H - 1, br + R), win.r1 - 1);
    b.clo = max(max(0, bc - R), win.c0);
    b.chi = min(min(ep.W - 1, bc + R), win.c1 - 1);
    return b;
}

// The tile at (y0, x0): at the root b0 itself (into tc) with the cell
// words; below it the parent's values with a two-cell rim (into tp) and the
// cell words with a one-cell rim; loads issued kLoadBatch at a time, before
// any of the batch is used, and only over the box and its rims.
__device__ void tile_load(const EpReg &ep, const float *par, bool root, int y0, int x0, const TileBox &bx, float *tp,
                          float *tc, uint16_t *tcw) {
    const int lane = threadIdx.x & 31;
    const int P = ep.P, H = ep.H, rhi = bx.rhi, chi = bx.chi;
    constexpr int PW = kTileW + 4, CW = kTileW + 2;
    constexpr int NP = (kTileP + 31) / 32, NC = (kTileC + 31) / 32;
    constexpr int kLoadBatch = 8;  // loads in flight per lane (the values wait in registers)
    __syncwarp();
    if (root) {
#pragma unroll 1
        for (int u0 = 0; u0 < NC; u0 += kLoadBatch) {
            uint16_t cv[kLoadBatch];
            float bv[kLoadBatch];
#pragma unroll
            for (int v = 0; v < kLoadBatch; ++v) {
                const int i = lane + 32 * (u0 + v), rr = i / CW, cc = i - rr * CW;
                const int r = y0 - 1 + rr, c = x0 - 1 + cc;
                const bool in = u0 + v < NC && i < kTileC && r >= 0 && r < H && c >= 0 && c < P && r <= rhi + 1 &&
                                c <= chi + 1;
                cv[v] = in ? __ldg(ep.cell + static_cast<size_t>(r) * P + c) : static_cast<uint16_t>(0);
                bv[v] = in ? __ldcg(par + static_cast<size_t>(r) * P + c) : 0.0f;
            }
#pragma unroll
            for (int v = 0; v < kLoadBatch; ++v) {
                const int i = lane + 32 * (u0 + v);
                if (u0 + v < NC && i < kTileC) {
                    tcw[i] = cv[v];
                    tc[i] = QV_CELL_FREE(static_cast<unsigned>(cv[v])) ? bv[v] : 0.0f;
                }
            }
        }
    } else {
#pragma unroll 1
        for (int u0 = 0; u0 < NP; u0 += kLoadBatch) {
            float pv[kLoadBatch];
#pragma unroll
            for (int v = 0; v < kLoadBatch; ++v) {
                const int i = lane + 32 * (u0 + v), rr = i / PW, cc = i - rr * PW;
                const int r = y0 - 2 + rr, c = x0 - 2 + cc;
                pv[v] = (u0 + v < NP && i < kTileP && r >= 0 && r < H && c >= 0 && c < P && r <= rhi + 2 &&
                         c <= chi + 2)
                            ? __ldcg(par + static_cast<size_t>(r) * P + c)
                            : 0.0f;
            }
#pragma unroll
            for (int v = 0; v < kLoadBatch; ++v)
                if (u0 + v < NP && lane + 32 * (u0 + v) < kTileP) tp[lane + 32 * (u0 + v)] = pv[v];
        }
#pragma unroll 1
        for (int u0 = 0; u0 < NC; u0 += kLoadBatch) {
            uint16_t cv[kLoadBatch];
#pragma unroll
            for (int v = 0; v < kLoadBatch; ++v) {
                const int i = lane + 32 * (u0 + v), rr = i / CW, cc = i - rr * CW;
                const int r = y0 - 1 + rr, c = x0 - 1 + cc;
                cv[v] = (u0 + v < NC && i < kTileC && r >= 0 && r < H && c >= 0 && c < P && r <= rhi + 1 &&
                         c <= chi + 1)
                            ? __ldg(ep.cell + static_cast<size_t>(r) * P + c)
                            : static_cast<uint16_t>(0);
            }
#pragma unroll
            for (int v = 0; v < kLoadBatch; ++v)
                if (u0 + v < NC && lane + 32 * (u0 + v) < kTileC) tcw[lane + 32 * (u0 + v)] = cv[v];
        }
    }
    __syncwarp();
}

// The diamond's cells of label k inside the tile at (y0, x0), as tile
// indices in `list` (ascending); returns their number.
__device__ int tile_list(const EpReg &ep, int k, int br, int bc, int y0, int x0, const TileBox &bx,
                         const uint16_t *tcw, int *list) {
    const int lane = threadIdx.x & 31;
    constexpr int CW = kTileW + 2, ND = (kTileH * kTileW + 31) / 32;
    int nh = 0;
#pragma unroll 1
    for (int u = 0; u < ND; ++u) {
        const int i = lane + 32 * u, rr = i / kTileW, cc = i - rr * kTileW;
        const int r = y0 + rr, c = x0 + cc;
        const bool hit = i < kTileH * kTileW && r <= bx.rhi && c <= bx.chi &&
                         abs(r - br) + abs(c - bc) <= ep.range &&
                         static_cast<int>(QV_CELL_LABEL(tcw[(rr + 1) * CW + cc + 1])) == k;
        const unsigned bal = __ballot_sync(0xffffffffu, hit);
        if (hit) list[nh + __popc(bal & ((1u << lane) - 1u))] = i;
        nh += __popc(bal);
    }
    __syncwarp();
    return nh;
}

// The node's belief Phi(parent, pa, zc) (Eq. 3) on the tile and its rim,
// from the parent's values in tp (not used at the root, where tc holds b0).
__device__ void tile_form(const EpReg &ep, int pa, int zc, float sa, float se, int y0, int x0, const TileBox &bx,
                          const float *tp, float *tc, const uint16_t *tcw, const float *lut) {
    const int lane = threadIdx.x & 31;
    const int P = ep.P, H = ep.H;
    constexpr int PW = kTileW + 4, CW = kTileW + 2;
    for (int i = lane; i < kTileC; i += 32) {
        const int rr = i / CW, cc = i - rr * CW;
        const int r = y0 - 1 + rr, c = x0 - 1 + cc;
        float v = 0.0f;
        if (r >= 0 && r < H && c >= 0 && c < P && r <= bx.rhi + 1 && c <= bx.chi + 1) {
            const unsigned cw = tcw[i];
            const float *m = tp + (rr + 1) * PW + (cc + 1);
            const unsigned in = QV_CELL_INFLOW(cw);
            float nb[4];
            nb[kDirN] = (in & 1u) ? m[-PW] : 0.0f;
            nb[kDirE] = (in & 2u) ? m[1] : 0.0f;
            nb[kDirS] = (in & 4u) ? m[PW] : 0.0f;
            nb[kDirW] = (in & 8u) ? m[-1] : 0.0f;
            const float p = predict_one(nb, m[0], cw, r * P + c == ep.goal, ep.slip, lut, pa);
            v = p * (static_cast<int>(QV_CELL_LABEL(cw)) == zc ? sa : se);
        }
        tc[i] = v;
    }
    __syncwarp();
}

// The listed cells' predicted masses for the five actions (from the node's
// belief in tc), added to la and, fused, their Q-weighted ones to lq.
template <bool FUSED>
__device__ void tile_predict(const EpReg &ep, int y0, int x0, const float *tc, const uint16_t *tcw, const int *list,
                             int nh, const float *lut, float la[5], float lq[FUSED ? 25 : 1]) {
    const int lane = threadIdx.x & 31;
    const int P = ep.P;
    constexpr int CW = kTileW + 2;
    for (int h = lane; h < nh; h += 32) {
        const int cell = list[h];
        const int rr = cell / kTileW, cc = cell - rr * kTileW;
        const int r = y0 + rr, c = x0 + cc;
        float qv[FUSED ? 5 : 1];
        if constexpr (FUSED) {
#pragma unroll
            for (int ap = 0; ap < 5; ++ap)
                qv[ap] = __ldg(ep.Q + static_cast<size_t>(ap) * ep.N + static_cast<size_t>(r) * P + c);
        }
        const unsigned cw = tcw[(rr + 1) * CW + cc + 1];
        const float *m = tc + (rr + 1) * CW + (cc + 1);
        const unsigned in = QV_CELL_INFLOW(cw);
        float nb[4], out[5];
        nb[kDirN] = (in & 1u) ? m[-CW] : 0.0f;
        nb[kDirE] = (in & 2u) ? m[1] : 0.0f;
        nb[kDirS] = (in & 4u) ? m[CW] : 0.0f;
        nb[kDirW] = (in & 8u) ? m[-1] : 0.0f;
        predict_cell(nb, m[0], cw, r * P + c == ep.goal, ep.slip, lut, out);
#pragma unroll
        for (int a = 0; a < 5; ++a) la[a] += out[a];
        if constexpr (FUSED) {
#pragma unroll
            for (int a = 0; a < 5; ++a)
#pragma unroll
                for (int ap = 0; ap < 5; ++ap) lq[a * 5 + ap] = fmaf(out[a], qv[ap], lq[a * 5 + ap]);
        }
    }
}

template <bool FUSED>
__device__ void label_tiles(const EpReg &ep, const float *par, bool root, int pa, int zc, float sa, float se, int k,
                            int br, int bc, const Win &win, float *tp, float *tc, uint16_t *tcw, int *list,
                            const float *lut, float la[5], float lq[FUSED ? 25 : 1]) {
    const TileBox bx = tile_box(ep, br, bc, win);
    for (int y0 = bx.rlo; y0 <= bx.rhi; y0 += kTileH) {
        for (int x0 = bx.clo; x0 <= bx.chi; x0 += kTileW) {
            tile_load(ep, par, root, y0, x0, bx, tp, tc, tcw);
            const int nh = tile_list(ep, k, br, bc, y0, x0, bx, tcw, list);
            if (!root) tile_form(ep, pa, zc, sa, se, y0, x0, bx, tp, tc, tcw, lut);
            tile_predict<FUSED>(ep, y0, x0, tc, tcw, list, nh, lut, la, lq);
        }
    }
}

// A node's totals -- final, or the records of its group's expand items in
// item order -- into S.tot, and its belief at the goal (whose arrivals
// R(b, a) must not pay) into S.flags[4].  With wait_group, first waits
// (bounded) until every expand item of its group has counted itself done.
// Totals of the deepest fused level's contraction form (ctr_item).
// A child's total v: its records of items 0 .. items - 1 added in item order.
__device__ __forceinline__ float ctr_total(const PlanDev &pl, int rb, int items, int n, int c, int v) {
    float sum = 0.0f;
    for (int i0 = 0; i0 < items; i0 += 8) {
        float t[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const long long x = static_cast<long long>(rb) + static_cast<long long>(i0 + u) * n + c;
            t[u] = (i0 + u < items && x < pl.n_xrec) ? __ldcg(pl.xrec + x * kTot + v) : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) sum += t[u];
    }
    return sum;
}

__device__ __forceinline__ bool ctr_level(const PlanDev &pl, int l) {
    return pl.ctr && l >= 1 && l == pl.depth - 1 && pl.leaf_mode == QV_LEAF_FUSED && __ldcg(pl.c_mode) != 0;
}

// Bounded wait until *gd >= need (thread 0; the caller's barrier follows).
__device__ __forceinline__ void wait_count(const PlanDev &pl, const unsigned *gd, unsigned need) {
    unsigned i = 0;
    for (;;) {
        unsigned v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(gd) : "memory");
        if (v >= need) break;
        if (++i > pl.spin_limit || (*((volatile unsigned *)pl.status) & kErrTimeout)) {
            atomicOr(pl.status, kErrTimeout);
            break;
        }
        __nanosleep(64);
    }
}

__device__ void node_totals(const PlanDev &pl, int l, const EpDev &ep, int e, int lp, int local, int iid,
                            const float *par, int pa, int zc, float sa, float se, bool wait_group, Smem &S) {
    const int E = pl.E;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int jg = e, r = 0;
    if (l > 0) {
        jg = __ldcg(pl.npre + (l - 1) * (E + 1) + e) + lp;
        const int cnt = __ldcg(pl.count + l * E + e);
        const int c0 = min(__ldcg(pl.choff + static_cast<long long>(ep.inode_base[l - 1] + lp) * 5), cnt);
        r = local - c0;
    }
    const int *goff = pl.grp_off + pl.gbase[l] + l;
    const int rec = __ldcg(pl.grp_rec + pl.gbase[l] + jg);
    constexpr int kGroups = kThreads / kTot;  // partial sums per value
    const BandGeo geo = band_geo(pl, e, ep.H, ep.W, ep.P, ep.band_rows, l);
    int gbi, gparts;
    group_split(__ldcg(goff + jg + 1) - __ldcg(goff + jg), geo.nb, gbi, gparts);
    const int nit = gbi * gparts;
    const bool cform = ctr_level(pl, l);
    const int cit0 = cform ? __ldcg(pl.c_items + e) : 0;
    const int citems = cform ? __ldcg(pl.c_items + e + 1) - cit0 : 0;
    if (wait_group) {
        if (threadIdx.x == 0)
            wait_count(pl, pl.grp_done + pl.gbase[l] + (cform ? e : jg), static_cast<unsigned>(cform ? citems : nit));
        __syncthreads();
    }
    if (cform) {
        if (threadIdx.x < kTot)
            S.tot[threadIdx.x] = ctr_total(pl, __ldcg(pl.c_rbase + e), citems, __ldcg(pl.count + l * E + e), local,
                                           threadIdx.x);
    } else if (rec < 0) {
        if (threadIdx.x < kTot) S.tot[threadIdx.x] = __ldcg(pl.ntot + static_cast<long long>(iid) * kTot + threadIdx.x);
    } else {
        const int t = threadIdx.x % kTot, g = threadIdx.x / kTot;
        if (g < kGroups) {
            // items g, g + 7, ... in order, eight loads in flight at a time
            float sum = 0.0f;
            for (int it0 = g; it0 < nit; it0 += 8 * kGroups) {
                float v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int it = it0 + u * kGroups;
                    const long long x = static_cast<long long>(rec + it) * pl.cmax + r;
                    v[u] = (it < nit && x < pl.n_xrec) ? __ldcg(pl.xrec + x * kTot + t) : 0.0f;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) sum += v[u];
            }
            S.red[g * kTot + t] = sum;
        }
        __syncthreads();
        if (threadIdx.x < kTot) {
            float sum = 0.0f;
            for (int g2 = 0; g2 < kGroups; ++g2) sum += S.red[g2 * kTot + threadIdx.x];
            S.tot[threadIdx.x] = sum;
        }
    }
    if (wid == 0) {
        // the node's belief at the goal, whose arrivals R(b, a) must not
        // pay: lanes 0-4 load the parent there and at its four
        // neighbours (inside the grid) at once
        const int y = ep.goal, P = ep.P, gr = y / P, gc = y - gr * P;
        const int dy[5] = {0, -P, 1, P, -1};
        const bool inside = lane < 5 && (lane != 1 || gr > 0) && (lane != 2 || gc + 1 < P) &&
                            (lane != 3 || gr + 1 < ep.H) && (lane != 4 || gc > 0);
        const float pv = inside ? __ldcg(par + y + dy[lane < 5 ? lane : 0]) : 0.0f;
        const unsigned cw = __ldg(ep.cell + y);
        const float m0 = __shfl_sync(0xffffffffu, pv, 0), mN = __shfl_sync(0xffffffffu, pv, 1);
        const float mE = __shfl_sync(0xffffffffu, pv, 2), mS = __shfl_sync(0xffffffffu, pv, 3);
        const float mW = __shfl_sync(0xffffffffu, pv, 4);
        if (lane == 0) {
            float bg;
            if (l == 0) {
                bg = m0;
            } else {
                const unsigned in = QV_CELL_INFLOW(cw);
                float nb[4];
                nb[kDirN] = (in & 1u) ? mN : 0.0f;
                nb[kDirE] = (in & 2u) ? mE : 0.0f;
                nb[kDirS] = (in & 4u) ? mS : 0.0f;
                nb[kDirW] = (in & 8u) ? mW : 0.0f;
                bg = predict_one(nb, m0, cw, true, ep.slip, S.lut, pa) *
                     (static_cast<int>(QV_CELL_LABEL(cw)) == zc ? sa : se);
            }
            S.flags[4] = __float_as_int(bg);
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------- finalize phase
// Work items are (node of level l, beacon chunk).  Each item forms the
// label histograms of its beacons (one warp per beacon, label_tiles); with
// several chunks per node the items write records and the last to arrive
// gathers them.  That item then adds the node's totals from its group's
// work items in item order, takes the node's belief at the goal (for
// R(b, a)), and finalises it: P(z | b, a), R(b, a), the K draws per action
// (Alg. 3-4), the unique draws; at the fused level the leaf values and the
// node's U_Q and U_V (Alg. 5-7).  At other levels the last node of an
// episode numbers its children and the last episode publishes the next
// level's work lists (NUMBER: every level but the fused deepest one).
// One finalize work item w of level l.  With `wait_group` the node first
// waits (bounded) until every expand item of its group has counted itself
// done on grp_done: the fused level runs its expand and finalize items as
// one phase, without a grid barrier between them.
template <bool FUSED, bool NUMBER>
__device__ void finalize_item(const PlanDev &pl, int l, Smem &S, int &cur_e, int w, bool wait_group) {
    const int E = pl.E, K = pl.K, Bm = pl.Bmax;
    const int *wb = pl.wb_fin + l * (E + 1);
    const int C = max(1, __ldcg(pl.fchunks + l));
    const int stride = 30 * ((Bm + C - 1) / C);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *tp = S.tile + wid * kTileFloats;
    float *tc = tp + kTileP;
    uint16_t *tcw = reinterpret_cast<uint16_t *>(tc + kTileC);
    int *tlist = reinterpret_cast<int *>(tc + kTileC + (kTileC + 1) / 2);
    {
#ifdef QV_TRACE
        unsigned long long tr[kTraceWords] = {};
#endif
        QV_TRACE_MARK(tr, 2);
        const int e = block_find(wb, E, w, S.flags + 6);
        load_ep(pl, e, S, cur_e);
        const EpDev &ep = *S.ep;
        const int rel = w - __ldcg(wb + e);
        const int local = rel / C, chunk = rel - local * C;
        const int B = ep.B;
        const int gid = ep.node_base[l] + local, iid = ep.inode_base[l] + local;
        int pa = 0, zc = 0, lp = 0;
        float sa = 1.0f, se = 1.0f;
        const float *par = ep.b0;
        if (l > 0) {
            const long long s = __ldcg(pl.src_slot + gid);
            const int iid_p = static_cast<int>(s / (5LL * K));
            pa = static_cast<int>((s / K) % 5);
            lp = iid_p - ep.inode_base[l - 1];
            zc = __ldcg(pl.slot_z + s);
            const float p = __ldcg(pl.slot_P + s);
            sa = ep.acc / p;
            se = ep.eta / p;
            par = node_belief(pl, ep, l - 1, lp);
        }
        const EpReg er = ep_reg(ep);
        const Win win = support_window(pl, e, ep.H, ep.W, l + 1);
        const int bpc = (B + C - 1) / C;
        const int k0 = min(B, chunk * bpc), k1 = min(B, k0 + bpc);
        __syncthreads();  // the previous item's readers of the histograms are done
        // the chunk's beacons whose diamond meets the window, listed by warp 0
        // (in the draw counts' buffer, unused until the node is finalised) and
        // dealt to the warps in turn; the others' masses are zero
        const int R = ep.range;
        auto meets = [&](int k) {
            const int br = S.bco[2 * k], bc = S.bco[2 * k + 1];
            return !(br + R < win.r0 || br - R >= win.r1 || bc + R < win.c0 || bc - R >= win.c1);
        };
        int *klist = S.cnt;
        if (wid == 0) {
            int n = 0;
            for (int kb = k0; kb < k1; kb += 32) {
                const int k = kb + lane;
                const bool hit = k < k1 && meets(k);
                const unsigned bal = __ballot_sync(0xffffffffu, hit);
                if (hit) klist[n + __popc(bal & ((1u << lane) - 1u))] = k;
                n += __popc(bal);
            }
            if (lane == 0) S.flags[9] = n;
        }
        for (int i = threadIdx.x; i < (k1 - k0) * 30; i += blockDim.x) {
            const int k = k0 + i / 30, t = i - (i / 30) * 30;
            if (meets(k)) continue;
            if (t < 5) S.hist[t * Bm + k] = 0.0f;
            else if (FUSED) S.histq[(((t - 5) / 5) * Bm + k) * 5 + (t - 5) % 5] = 0.0f;
        }
        __syncthreads();
        const int nlist = S.flags[9];
        for (int li = wid; li < nlist; li += kWarps) {
            const int k = klist[li];
            float la[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
            float lq[FUSED ? 25 : 1];
#pragma unroll
            for (int i = 0; i < (FUSED ? 25 : 1); ++i) lq[i] = 0.0f;
            label_tiles<FUSED>(er, par, l == 0, pa, zc, sa, se, k, S.bco[2 * k], S.bco[2 * k + 1], win, tp, tc, tcw,
                               tlist, S.lut, la, lq);
            // lane i ends with the warp total of value i: 0..4 the label
            // masses, 5..29 the Q-weighted ones
            float v[32];
#pragma unroll
            for (int a = 0; a < 5; ++a) v[a] = la[a];
#pragma unroll
            for (int i = 0; i < 25; ++i) {
                if constexpr (FUSED) v[5 + i] = lq[i];
                else v[5 + i] = 0.0f;
            }
            v[30] = v[31] = 0.0f;
            warp_reduce_scatter32(v);
            if (lane < 5) S.hist[lane * Bm + k] = v[0];
            else if (FUSED && lane < 30) S.histq[(((lane - 5) / 5) * Bm + k) * 5 + (lane - 5) % 5] = v[0];
        }
        __syncthreads();
        QV_TRACE_MARK(tr, 3);
        if (C > 1) {
            // a record of this chunk's beacons; the last chunk of the node gathers
            float *recp = pl.frec + static_cast<long long>(w) * stride;
            const bool room = static_cast<long long>(w + 1) * stride <= pl.n_frec;
            if (room)
                for (int i = threadIdx.x; i < (k1 - k0) * 30; i += blockDim.x) {
                    const int k = k0 + i / 30, t = i % 30;
                    recp[i] = t < 5 ? S.hist[t * Bm + k] : S.histq[(((t - 5) / 5) * Bm + k) * 5 + (t - 5) % 5];
                }
            __syncthreads();
            if (threadIdx.x == 0) {
                if (!room) atomicOr(pl.status, kErrCapacity);
                const unsigned prev = arrive_acq_rel(pl.node_cnt + iid);
                const int last = prev == static_cast<unsigned>(C - 1);
                if (last) pl.node_cnt[iid] = 0u;
                S.flags[0] = last;
            }
            __syncthreads();
            QV_TRACE_MARK(tr, 4);
            if (!S.flags[0]) {
#ifdef QV_TRACE
                tr[0] = 1ull | (static_cast<unsigned long long>(l) << 8) |
                        (static_cast<unsigned long long>(blockIdx.x) << 16);
                tr[1] = static_cast<unsigned long long>(w);
                trace_commit(tr, 5);
#endif
                return;
            }
            for (int i0 = threadIdx.x; i0 < B * 30; i0 += 4 * blockDim.x) {
                // four loads in flight per thread
                float v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int i = i0 + u * blockDim.x;
                    const int k = i / 30, t = i - k * 30, c = k / bpc;
                    const long long wi = static_cast<long long>(w - chunk + c);
                    v[u] = (i < B * 30 && c != chunk && (wi + 1) * stride <= pl.n_frec)
                               ? __ldcg(pl.frec + wi * stride + (k - c * bpc) * 30 + t)
                               : 0.0f;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int i = i0 + u * blockDim.x;
                    const int k = i / 30, t = i - k * 30, c = k / bpc;
                    if (i >= B * 30 || c == chunk) continue;
                    if (t < 5) S.hist[t * Bm + k] = v[u];
                    else if (FUSED) S.histq[(((t - 5) / 5) * Bm + k) * 5 + (t - 5) % 5] = v[u];
                }
            }
        }
        QV_TRACE_MARK(tr, 5);
        // the node's totals: final, or the records of its group's items in order
        node_totals(pl, l, ep, e, lp, local, iid, par, pa, zc, sa, se, wait_group, S);
        QV_TRACE_MARK(tr, 6);
        const unsigned long long code = __ldcg(pl.code + gid);
        finalize_node(pl, ep, l, local, FUSED, __int_as_float(S.flags[4]), code, S);
        QV_TRACE_MARK(tr, 7);
        if constexpr (NUMBER) node_done(pl, l, e, ep, S);
        QV_TRACE_MARK(tr, 8);
#ifdef QV_TRACE
        tr[0] = 1ull | (static_cast<unsigned long long>(l) << 8) | (static_cast<unsigned long long>(blockIdx.x) << 16) |
                (1ull << 56);
        tr[1] = static_cast<unsigned long long>(w);
        trace_commit(tr, 9);
#endif
    }
}

// A group's finalize item (the fused mode's deepest level when a node's
// beacons form one chunk): one V-node p of level l - 1 and a contiguous
// piece of its children (a group has as many pieces as expand items, which
// are in proportion to its children).  While the beacons whose diamond meets the window are at most one per
// warp and each diamond's box fits one tile, a warp loads its beacon's tile
// of p's values and cell words and lists its label cells once, and every
// child reuses them: per child the warps form the child's belief on their
// tiles (Eq. 3) and its label histograms, then the node is finalised as by
// a node item.  Otherwise each child walks its beacons' tiles afresh.
template <bool FUSED>
__device__ void finalize_group_item(const PlanDev &pl, int l, Smem &S, int &cur_e, int w) {
    const int E = pl.E, K = pl.K, Bm = pl.Bmax;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *tp = S.tile + wid * kTileFloats;
    float *tc = tp + kTileP;
    uint16_t *tcw = reinterpret_cast<uint16_t *>(tc + kTileC);
    int *tlist = reinterpret_cast<int *>(tc + kTileC + (kTileC + 1) / 2);
    const int G = __ldcg(pl.ngrp + l);
    const int *goff = pl.grp_off + pl.gbase[l] + l;
    const int *np = pl.npre + (l - 1) * (E + 1);
    const int j = block_find(goff, G, w, S.flags + 6);
    if (!QV_IN_BOUNDS(kSiteGroup, pl.gbase[l] + j, pl.ngrp_cap)) return;  // uniform over the CTA
    const int e = block_find(np, E, j, S.flags + 7);
    load_ep(pl, e, S, cur_e);
    const EpDev &ep = *S.ep;
    const int lp = j - __ldcg(np + e);  // the group's V-node p: node lp of level l - 1
    const int g0 = __ldcg(goff + j), pieces = max(1, __ldcg(goff + j + 1) - g0), piece = w - g0;
    const int B = ep.B;
    const long long ia = static_cast<long long>(ep.inode_base[l - 1] + lp) * 5;
    if (!QV_IN_BOUNDS(kSiteInode, ep.inode_base[l - 1] + lp, pl.n_inodes)) return;
    const int cnt = __ldcg(pl.count + l * E + e);
    const int cg0 = min(__ldcg(pl.choff + ia), cnt);
    const int cg1 = min(__ldcg(pl.choff + ia + 4) + __ldcg(pl.nchild + ia + 4), cnt);
    const int ncg = max(0, cg1 - cg0);
    // this item's piece of the children
    const int c0 = cg0 + static_cast<int>((static_cast<long long>(ncg) * piece) / pieces);
    const int nc = cg0 + static_cast<int>((static_cast<long long>(ncg) * (piece + 1)) / pieces) - c0;
    if (nc <= 0) return;
    const float *par = node_belief(pl, ep, l - 1, lp);
    const EpReg er = ep_reg(ep);
    const Win win = support_window(pl, e, ep.H, ep.W, l + 1);
    const int R = ep.range;
    auto meets = [&](int k) {
        const int br = S.bco[2 * k], bc = S.bco[2 * k + 1];
        return !(br + R < win.r0 || br - R >= win.r1 || bc + R < win.c0 || bc - R >= win.c1);
    };
    int *klist = S.cnt;  // free until a node is finalised
    auto list_beacons = [&]() {
        __syncthreads();  // the previous readers of the list and the histograms are done
        if (wid == 0) {
            int n = 0;
            for (int kb = 0; kb < B; kb += 32) {
                const int k = kb + lane;
                const bool hit = k < B && meets(k);
                const unsigned bal = __ballot_sync(0xffffffffu, hit);
                if (hit) klist[n + __popc(bal & ((1u << lane) - 1u))] = k;
                n += __popc(bal);
            }
            if (lane == 0) S.flags[9] = n;
        }
        __syncthreads();
    };
    // beacons whose diamond misses the window keep zero masses for every child
    __syncthreads();  // the previous item's readers of the histograms are done
    for (int i = threadIdx.x; i < B * 30; i += blockDim.x) {
        const int k = i / 30, t = i - (i / 30) * 30;
        if (meets(k)) continue;
        if (t < 5) S.hist[t * Bm + k] = 0.0f;
        else if (FUSED) S.histq[(((t - 5) / 5) * Bm + k) * 5 + (t - 5) % 5] = 0.0f;
    }
    list_beacons();
    const int nlist = S.flags[9];
    const bool resident = nlist <= kWarps && 2 * R + 1 <= kTileH && 2 * R + 1 <= kTileW;
    int myk = -1, nh = 0;
    TileBox bx{0, -1, 0, -1};
    if (resident && wid < nlist) {
        myk = klist[wid];
        bx = tile_box(er, S.bco[2 * myk], S.bco[2 * myk + 1], win);
        if (bx.rlo <= bx.rhi && bx.clo <= bx.chi) {
            tile_load(er, par, false, bx.rlo, bx.clo, bx, tp, tc, tcw);
            nh = tile_list(er, myk, S.bco[2 * myk], S.bco[2 * myk + 1], bx.rlo, bx.clo, bx, tcw, tlist);
        }
    }
    // the group's expand items all done (bounded wait), then the totals of
    // every child of the piece at once -- final, or the records of the
    // group's items in item order -- into S.acc (free in a finalize item),
    // and p's values at the goal and its four neighbours (every child's
    // belief there is formed from them)
    {
        const int rec = __ldcg(pl.grp_rec + pl.gbase[l] + j);
        const BandGeo geo = band_geo(pl, e, ep.H, ep.W, ep.P, ep.band_rows, l);
        int gbi, gparts;
        group_split(__ldcg(goff + j + 1) - g0, geo.nb, gbi, gparts);
        const int nit = gbi * gparts;
        // in the contraction form the episode's items instead (ctr_item)
        const bool cform = ctr_level(pl, l);
        const int cit0 = cform ? __ldcg(pl.c_items + e) : 0;
        const int citems = cform ? __ldcg(pl.c_items + e + 1) - cit0 : 0;
        const int crb = cform ? __ldcg(pl.c_rbase + e) : 0;
        if (threadIdx.x == 0)
            wait_count(pl, pl.grp_done + pl.gbase[l] + (cform ? e : j), static_cast<unsigned>(cform ? citems : nit));
        __syncthreads();
        for (int i = threadIdx.x; i < nc * kTot; i += blockDim.x) {
            const int rr = i / kTot, v = i - rr * kTot;
            float sum = 0.0f;
            if (cform) {
                sum = ctr_total(pl, crb, citems, cnt, c0 + rr, v);
            } else if (rec < 0) {
                sum = __ldcg(pl.ntot + static_cast<long long>(ep.inode_base[l] + c0 + rr) * kTot + v);
            } else {
                const int rk = c0 - cg0 + rr;  // the child's rank in the group
                for (int it = 0; it < nit; ++it) {
                    const long long x = static_cast<long long>(rec + it) * pl.cmax + rk;
                    sum += x < pl.n_xrec ? __ldcg(pl.xrec + x * kTot + v) : 0.0f;
                }
            }
            S.acc[i] = sum;
        }
        // every child's action, observation, Eq. 3 weights and path code
        // (S.c_* and S.red are free in a finalize item)
        unsigned long long *codes = reinterpret_cast<unsigned long long *>(S.red);
        for (int rr = threadIdx.x; rr < nc; rr += blockDim.x) {
            const int gid = ep.node_base[l] + c0 + rr;
            int a = 0, z = 0;
            float ca = 0.0f, ce = 0.0f;
            unsigned long long cd = 0ull;
            if (QV_IN_BOUNDS(kSiteNode, gid, pl.n_nodes)) {
                const long long sl = __ldcg(pl.src_slot + gid);
                cd = __ldcg(pl.code + gid);
                if (QV_IN_BOUNDS(kSiteSlot, sl, 5 * K * pl.n_inodes)) {
                    a = static_cast<int>((sl / K) % 5);
                    z = __ldcg(pl.slot_z + sl);
                    const float p = __ldcg(pl.slot_P + sl);
                    ca = ep.acc / p;
                    ce = ep.eta / p;
                }
            }
            S.c_pa[rr] = a;
            S.c_z[rr] = z;
            S.c_sa[rr] = ca;
            S.c_se[rr] = ce;
            codes[rr] = cd;
        }
        if (wid == 0) {
            const int y = ep.goal, P = ep.P, gr = y / P, gc = y - gr * P;
            const int dy[5] = {0, -P, 1, P, -1};
            const bool inside = lane < 5 && (lane != 1 || gr > 0) && (lane != 2 || gc + 1 < P) &&
                                (lane != 3 || gr + 1 < ep.H) && (lane != 4 || gc > 0);
            const float pv = inside ? __ldcg(par + y + dy[lane < 5 ? lane : 0]) : 0.0f;
            if (lane < 5) S.uq[lane] = pv;  // S.uq is written by finalize_node only at its end
        }
        __syncthreads();
    }
    const unsigned cwg = __ldg(ep.cell + ep.goal);
    const float pg0 = S.uq[0], pgN = S.uq[1], pgE = S.uq[2], pgS = S.uq[3], pgW = S.uq[4];
    for (int r = 0; r < nc; ++r) {
        const int local = c0 + r;
        const int gid = ep.node_base[l] + local, iid = ep.inode_base[l] + local;
        if (!QV_IN_BOUNDS(kSiteNode, gid, pl.n_nodes)) return;  // uniform over the CTA
        // the child's action, observation and Eq. 3 weights
        const int pa = S.c_pa[r], zc = S.c_z[r];
        const float sa = S.c_sa[r], se = S.c_se[r];
        if (!resident) list_beacons();
        float la[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        float lq[FUSED ? 25 : 1];
#pragma unroll
        for (int i = 0; i < (FUSED ? 25 : 1); ++i) lq[i] = 0.0f;
        auto store_hist = [&](int k) {
            // lane i ends with the warp total of value i: 0..4 the label
            // masses, 5..29 the Q-weighted ones
            float v[32];
#pragma unroll
            for (int a = 0; a < 5; ++a) v[a] = la[a];
#pragma unroll
            for (int i = 0; i < 25; ++i) {
                if constexpr (FUSED) v[5 + i] = lq[i];
                else v[5 + i] = 0.0f;
            }
            v[30] = v[31] = 0.0f;
            warp_reduce_scatter32(v);
            if (lane < 5) S.hist[lane * Bm + k] = v[0];
            else if (FUSED && lane < 30) S.histq[(((lane - 5) / 5) * Bm + k) * 5 + (lane - 5) % 5] = v[0];
        };
        if (resident) {
            if (myk >= 0) {
                if (nh > 0) {
                    tile_form(er, pa, zc, sa, se, bx.rlo, bx.clo, bx, tp, tc, tcw, S.lut);
                    tile_predict<FUSED>(er, bx.rlo, bx.clo, tc, tcw, tlist, nh, S.lut, la, lq);
                }
                store_hist(myk);
            }
        } else {
            for (int li = wid; li < nlist; li += kWarps) {
                const int k = klist[li];
#pragma unroll
                for (int a = 0; a < 5; ++a) la[a] = 0.0f;
#pragma unroll
                for (int i = 0; i < (FUSED ? 25 : 1); ++i) lq[i] = 0.0f;
                label_tiles<FUSED>(er, par, false, pa, zc, sa, se, k, S.bco[2 * k], S.bco[2 * k + 1], win, tp, tc,
                                   tcw, tlist, S.lut, la, lq);
                store_hist(k);
            }
        }
        // the child's totals and its belief at the goal (whose arrivals
        // R(b, a) must not pay)
        if (threadIdx.x < kTot) S.tot[threadIdx.x] = S.acc[r * kTot + threadIdx.x];
        if (threadIdx.x == 0) {
            const unsigned in = QV_CELL_INFLOW(cwg);
            float nb[4];
            nb[kDirN] = (in & 1u) ? pgN : 0.0f;
            nb[kDirE] = (in & 2u) ? pgE : 0.0f;
            nb[kDirS] = (in & 4u) ? pgS : 0.0f;
            nb[kDirW] = (in & 8u) ? pgW : 0.0f;
            const float bg = predict_one(nb, pg0, cwg, true, ep.slip, S.lut, pa) *
                             (static_cast<int>(QV_CELL_LABEL(cwg)) == zc ? sa : se);
            S.flags[4] = __float_as_int(bg);
        }
        __syncthreads();
        const unsigned long long code = reinterpret_cast<const unsigned long long *>(S.red)[r];
        finalize_node(pl, ep, l, local, FUSED, __int_as_float(S.flags[4]), code, S);
    }
}

// ---------------------------------------------------------------- contraction form (deepest fused level)
// At the fused mode's deepest level l every total of a child c is linear in
// its belief b_c = Phi(p, a_c, z_c) (Eq. 3): for each action a the
// null-label mass sum_y nf(y) bbar_a(y), the reward sum sum_y r(y) bbar_a(y)
// and the Q-weighted null masses sum_y nf(y) Q(a', y) bbar_a(y), with
// bbar_a = T_a b_c (Eq. 3 numerator, Eq. 10).  Moving T_a onto the weights
// gives sum_x b_c(x) W_j(x), W_j(x) = sum_y T(x, a, y) u_j(y), 35 planes
// that depend on the map and Q only.  A work item (episode, band of window
// rows) therefore multiplies the children's beliefs [children x cells] with
// the planes [cells x 36] for every child of the episode at once: per row
// segment of kCSC cells the parents' rows, Q, the cell words and the cost
// are staged, the planes and the children's beliefs formed in shared
// memory, and each thread accumulates a tile of 4 children x 12 planes over
// its share of the segment's cells (FP32 FMAs).  The tiles' partial sums
// are added in a fixed order and written as one record per (item, child);
// a child's finalize adds its records in item order.  The episode's first
// item also writes the children's records (parent, action, observation,
// weight, P(z), path code).  Items count themselves done on the episode's
// counter (grp_done at gbase[l] + e), which the finalize items wait on.

// 16-byte asynchronous copy global -> shared through L2 (zero-filled when
// !valid; src must still be a valid address).
__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src),
                 "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ void ctr_item(const PlanDev &pl, int l, Smem &S, int &cur_e, int w) {
    const int E = pl.E, K = pl.K, tid = threadIdx.x;
    const int wid = tid >> 5, lane = tid & 31;
    const int e = block_find(pl.c_items, E, w, S.flags + 6);
    if (!QV_IN_BOUNDS(kSiteEpisode, e, E)) return;  // uniform over the CTA
    const int i0 = __ldcg(pl.c_items + e);
    const int it = w - i0, items = __ldcg(pl.c_items + e + 1) - i0;
    load_ep(pl, e, S, cur_e);
    const EpDev &ep = *S.ep;
    const EpReg er = ep_reg(ep);
    const int n = __ldcg(pl.count + l * E + e);
    const int rb = __ldcg(pl.c_rbase + e);
    const int B = er.B, P = er.P, H = er.H, goal = er.goal;
    const long long N = er.N;
    const float slip = er.slip, fwd = 1.0f - 2.0f * slip;
    const Win win = support_window(pl, e, er.H, er.W, l);  // where the level's beliefs can be nonzero
    const int nr = max(0, win.r1 - win.r0), wc = max(0, win.c1 - win.c0);
    const int y0 = win.r0 + static_cast<int>((static_cast<long long>(it) * nr) / items);
    const int y1 = win.r0 + static_cast<int>((static_cast<long long>(it + 1) * nr) / items);
    const int nseg = (wc + kCSC - 1) / kCSC;
    const int segw = nseg > 0 ? (wc + nseg - 1) / nseg : 0;
    const CtrLayout CL = ctr_layout();
    float *spar = S.sb + CL.par, *sq = S.sb + CL.q, *scost = S.sb + CL.cost, *sbp = S.sb + CL.bp, *sW = S.sb + CL.W;
    uint16_t *scw = reinterpret_cast<uint16_t *>(S.sb + CL.cw);
    int *cpi = reinterpret_cast<int *>(S.sb + CL.cpi), *ca = reinterpret_cast<int *>(S.sb + CL.ca);
    int *cz = reinterpret_cast<int *>(S.sb + CL.cz);
    float *csa = S.sb + CL.csa, *cse = S.sb + CL.cse;
    const float *cost = er.cost;
    // the parents: level l - 1's stored beliefs, or the root's b0 (l = 1)
    const bool proot = l == 1;
    const float *pbase = proot ? ep.b0 : pl.beliefs + ep.belief_off[l - 1];
    if (it == 0)
        for (int r = tid; r < n; r += blockDim.x) {
            const int gid = ep.node_base[l] + r;
            if (!QV_IN_BOUNDS(kSiteNode, gid, pl.n_nodes)) continue;
            const long long sl = __ldcg(pl.src_slot + gid);
            if (!QV_IN_BOUNDS(kSiteSlot, sl, 5LL * K * pl.n_inodes)) continue;
            const int lp = static_cast<int>(sl / (5LL * K)) - ep.inode_base[l - 1];
            const int a = static_cast<int>((sl / K) % 5);
            const int z = __ldcg(pl.slot_z + sl);
            const unsigned long long pcode = __ldcg(pl.code + ep.node_base[l - 1] + lp);
            pl.parent[gid] = lp;
            pl.action[gid] = a;
            pl.obs[gid] = z;
            pl.weight[gid] = __ldcg(pl.slot_w + sl);
            pl.pz[gid] = __ldcg(pl.slot_P + sl);
            pl.code[gid] = (pcode * 5ull + a) * static_cast<unsigned long long>(B + 1) + z;
        }
    const int nblk = (n + kCMB - 1) / kCMB;
    for (int bk = 0; bk < nblk; ++bk) {
        const int cb0 = static_cast<int>((static_cast<long long>(bk) * n) / nblk);
        const int nb = static_cast<int>((static_cast<long long>(bk + 1) * n) / nblk) - cb0;
        __syncthreads();  // the previous block's readers of the child table and the sum buffer are done
        for (int r = tid; r < kCMB; r += blockDim.x) {
            int lp = -1, a = 0, z = -1;
            float sa = 0.0f, se = 0.0f;
            if (r < nb) {
                const int gid = ep.node_base[l] + cb0 + r;
                if (QV_IN_BOUNDS(kSiteNode, gid, pl.n_nodes)) {
                    const long long sl = __ldcg(pl.src_slot + gid);
                    if (QV_IN_BOUNDS(kSiteSlot, sl, 5LL * K * pl.n_inodes)) {
                        lp = static_cast<int>(sl / (5LL * K)) - ep.inode_base[l - 1];
                        a = static_cast<int>((sl / K) % 5);
                        z = __ldcg(pl.slot_z + sl);
                        const float pz = __ldcg(pl.slot_P + sl);
                        sa = ep.acc / pz;
                        se = ep.eta / pz;
                    }
                }
            }
            cpi[r] = lp;
            ca[r] = a;
            cz[r] = z;
            csa[r] = sa;
            cse[r] = se;
        }
        __syncthreads();
        // the block's parents [lp0, lp0 + npar) (children are numbered parent by parent)
        if (tid < 32) {
            int mn = 0x7fffffff, mx = -1;
            for (int r = tid; r < nb; r += 32) {
                const int v = cpi[r];
                if (v >= 0) {
                    mn = min(mn, v);
                    mx = max(mx, v);
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
                mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            }
            if (tid == 0) {
                S.scan[0] = mn;
                S.scan[1] = mx >= mn ? mx - mn + 1 : 0;
            }
        }
        __syncthreads();
        const int lp0 = S.scan[0], npar = S.scan[1];
        const bool fit = npar <= kCPar;  // always: a V-node has at least five children
        if (!fit && tid == 0) atomicOr(pl.status, kErrCapacity);
        // the GEMM tile of this thread: children c4 .. c4 + 3, planes j0 .. j0 + 11,
        // cells kg, kg + KG, ... of each segment
        const int cq = (nb + 3) >> 2, T = cq * 3;
        const int KG = T > 0 ? static_cast<int>(blockDim.x) / T : 1;
        const int tile = T > 0 ? tid % T : 0, kg = T > 0 ? tid / T : 0;
        const bool gt = T > 0 && kg < KG;
        const int c4 = (tile / 3) * 4, j0 = (tile - (tile / 3) * 3) * 12;
        int po[4], zz[4];
        float sa4[4], se4[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int c = c4 + i;
            const bool ok = gt && c < nb && cpi[c] >= 0 && fit;
            po[i] = ok ? ((cpi[c] - lp0) * 5 + ca[c]) * kCBP : 0;
            zz[i] = ok ? cz[c] : -1;
            sa4[i] = ok ? csa[c] : 0.0f;
            se4[i] = ok ? cse[c] : 0.0f;
        }
        float acc[4][12];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 12; ++j) acc[i][j] = 0.0f;
        // one step: window row y, columns [x0, x0 + xw); its rows y - 1 .. y + 1
        // are staged from column xa = x0 - 1 rounded down to 8, into stage bf
        // one warp per staged row (the parents', Q's, the cost's, the cell
        // words'), one 16-byte copy per lane and chunk
        const int nprow = npar * 3, ncrow = cost ? 3 : 0;
        const int nrows = nprow + 15 + ncrow + 3;
        auto issue = [&](int y, int x0, int xw, int bf) {
            const int xa = (x0 - 1) & ~7;
            const int width = ((x0 + xw + 1 - xa) + 7) & ~7;
            const int n4 = width >> 2, n8 = width >> 3;
            for (int rr = wid; rr < nrows; rr += kWarps) {
                int k = rr, r;
                const float *src;
                void *dst;
                bool fl = true;  // a float row (4-value chunks), else cell words (8 per chunk)
                if (k < nprow) {
                    const int pi = k / 3;
                    r = k - pi * 3;
                    src = pbase + static_cast<long long>(lp0 + pi) * N;
                    dst = spar + bf * (kCPar * 3 * kCSW) + k * kCSW;
                } else if ((k -= nprow) < 15) {
                    const int ap = k / 3;
                    r = k - ap * 3;
                    src = er.Q + ap * N;
                    dst = sq + bf * (15 * kCSW) + k * kCSW;
                } else if ((k -= 15) < ncrow) {
                    r = k;
                    src = cost;
                    dst = scost + bf * (3 * kCSW) + k * kCSW;
                } else {
                    r = k - ncrow;
                    src = nullptr;
                    dst = scw + bf * (3 * kCSW) + r * kCSW;
                    fl = false;
                }
                const int row = y - 1 + r;
                const bool rin = row >= 0 && row < H;
                const int nch = fl ? n4 : n8;
                for (int ch = lane; ch < nch; ch += 32) {
                    const int col = xa + (fl ? 4 : 8) * ch;
                    bool valid = rin && col >= 0 && col < P;
                    const long long o = static_cast<long long>(row) * P + col;
                    if (fl) {
                        if (valid && rr < nprow && !proot &&
                            !QV_IN_BOUNDS(kSiteBelief, ep.belief_off[l - 1] + (src - pbase) + o + 3, pl.n_belief))
                            valid = false;
                        cp_async16(static_cast<float *>(dst) + 4 * ch, valid ? src + o : src, valid);
                    } else {
                        cp_async16(static_cast<uint16_t *>(dst) + 8 * ch, valid ? er.cell + o : er.cell, valid);
                    }
                }
            }
            cp_async_commit();
        };
        const int nsteps = fit ? (y1 - y0) * nseg : 0;
        if (nsteps > 0) issue(y0, win.c0, min(segw, win.c1 - win.c0), 0);
        int y = y0, sg = 0;
        for (int st = 0; st < nsteps; ++st) {
            const int bf = st & 1;
            const int x0 = win.c0 + sg * segw, xw = min(segw, win.c1 - x0), off = x0 - ((x0 - 1) & ~7);
            cp_async_wait_all();
            __syncthreads();  // stage bf landed for every thread; the previous step's readers are done
            int ny = y, nsg = sg + 1;
            if (nsg == nseg) {
                nsg = 0;
                ++ny;
            }
            if (st + 1 < nsteps) {
                const int nx0 = win.c0 + nsg * segw;
                issue(ny, nx0, min(segw, win.c1 - nx0), bf ^ 1);
            }
            const float *pb = spar + bf * (kCPar * 3 * kCSW);
            const float *qb = sq + bf * (15 * kCSW);
            const float *cb = scost + bf * (3 * kCSW);
            const uint16_t *wb = scw + bf * (3 * kCSW);
            // one loop over the parents' predicted beliefs for the five actions
            // (Eq. 3 numerator, Eq. 10; task (parent, cell)) and the planes of
            // the segment's cells (W(x, a) = sum_y T(x, a, y) u(y); task
            // (action, cell)), dealt evenly to the threads
            const int nbp_t = npar * kCSC;
            for (int t = tid; t < nbp_t + 5 * kCSC; t += blockDim.x) {
                if (t < nbp_t) {
                    const int pi = t >> 6, xi = t & (kCSC - 1);
                    if (xi >= xw) continue;
                    const int c = off + xi;
                    const unsigned cwx = wb[kCSW + c];
                    const float *pp = pb + (pi * 3 + 1) * kCSW + c;
                    const unsigned in = QV_CELL_INFLOW(cwx);
                    float nbv[4], out[5];
                    nbv[kDirN] = (in & 1u) ? pp[-kCSW] : 0.0f;
                    nbv[kDirE] = (in & 2u) ? pp[1] : 0.0f;
                    nbv[kDirS] = (in & 4u) ? pp[kCSW] : 0.0f;
                    nbv[kDirW] = (in & 8u) ? pp[-1] : 0.0f;
                    predict_cell(nbv, pp[0], cwx, y * P + x0 + xi == goal, slip, S.lut, out);
#pragma unroll
                    for (int a = 0; a < 5; ++a) sbp[(pi * 5 + a) * kCBP + xi] = out[a];
                    continue;
                }
                // (action fastest: a warp's plane stores fall in different banks)
                const int xi = (t - nbp_t) / 5, a = (t - nbp_t) - xi * 5;
                if (xi >= xw) continue;
                const int c = off + xi;
                const unsigned cwx = wb[kCSW + c];
                float wn = 0.0f, wr = 0.0f, wq[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
                // weight g of the move from x to the staged cell (r, cc)
                auto add = [&](int r, int cc, float g) {
                    const unsigned cu = wb[r * kCSW + cc];
                    const bool fr = QV_CELL_FREE(cu) != 0u;
                    const bool gl = (y - 1 + r) * P + (x0 - off + cc) == goal;
                    wr = fmaf(g, stage_reward(fr, gl, cost ? cb[r * kCSW + cc] : 0.0f), wr);
                    const float gn = (fr && static_cast<int>(QV_CELL_LABEL(cu)) >= B) ? g : 0.0f;
                    wn += gn;
#pragma unroll
                    for (int ap = 0; ap < 5; ++ap) wq[ap] = fmaf(gn, qb[(ap * 3 + r) * kCSW + cc], wq[ap]);
                };
                if (QV_CELL_FREE(cwx)) {
                    if (y * P + x0 + xi == goal || a == 4) {
                        add(1, c, 1.0f);  // the goal keeps its mass; stay
                    } else {
                        // the intended move (1 - 2 slip) and the two
                        // perpendicular slips; a blocked one stays on x
                        const unsigned blk = QV_CELL_BLOCKED(cwx);
                        add(1, c, S.lut[a * 16 + blk]);
                        const int dirs[3] = {a, (a + 1) & 3, (a + 3) & 3};
#pragma unroll
                        for (int m = 0; m < 3; ++m) {
                            const int d = dirs[m];
                            if ((blk >> d) & 1u) continue;
                            const int dr = d == kDirN ? -1 : (d == kDirS ? 1 : 0);
                            const int dc = d == kDirE ? 1 : (d == kDirW ? -1 : 0);
                            add(1 + dr, c + dc, m == 0 ? fwd : slip);
                        }
                    }
                }
                float *wp = sW + xi * kTot;
                wp[a] = wn;
                wp[5 + a] = wr;
#pragma unroll
                for (int ap = 0; ap < 5; ++ap) wp[10 + a * 5 + ap] = wq[ap];
                if (a == 0) wp[35] = 0.0f;
            }
            __syncthreads();
            // the children's beliefs Phi(p, a_c, z_c) = T_a b_p O(., z_c) / P(z_c)
            // (Eq. 3) against the planes
            if (gt)
                for (int xi = kg; xi < xw; xi += KG) {
                    const int lab = static_cast<int>(QV_CELL_LABEL(static_cast<unsigned>(wb[kCSW + off + xi])));
                    float av[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) av[i] = sbp[po[i] + xi] * (lab == zz[i] ? sa4[i] : se4[i]);
                    const float4 *wp = reinterpret_cast<const float4 *>(sW + xi * kTot + j0);
                    const float4 w0 = wp[0], w1 = wp[1], w2 = wp[2];
                    const float wv[12] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w, w2.x, w2.y, w2.z, w2.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 12; ++j) acc[i][j] = fmaf(av[i], wv[j], acc[i][j]);
                }
            y = ny;
            sg = nsg;
        }
        // the tiles' sums in K-group order into the child records (the sum
        // buffer is the predicted beliefs' area)
        cp_async_wait_all();
        __syncthreads();  // every tile's last reads are done
        for (int g = 0; g < KG; ++g) {
            if (gt && kg == g)
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 12; ++j) {
                        const int x = (c4 + i) * kTot + j0 + j;
                        sbp[x] = (g == 0 ? 0.0f : sbp[x]) + acc[i][j];
                    }
            __syncthreads();
        }
        for (int i = tid; i < nb * kTot; i += blockDim.x) {
            const int r = i / kTot, v = i - r * kTot;
            const long long x = static_cast<long long>(rb) + static_cast<long long>(it) * n + cb0 + r;
            if (QV_IN_BOUNDS(kSiteRecord, x, pl.n_xrec)) pl.xrec[x * kTot + v] = sbp[i];
        }
    }
    __syncthreads();  // every record of the item is written
    if (tid == 0) arrive_acq_rel(pl.grp_done + pl.gbase[l] + e);
}

// One level as one phase: its expand items, then its finalize items, from
// one counter.  A finalize item forms its label histograms at once and waits
// only for its own group's expand records (grp_done), so CTAs that finish
// their last expand item start finalising instead of waiting at a grid
// barrier.  Every expand item is taken before any finalize item, and expand
// items wait on nothing but their own copies, so every wait ends.  NUMBER:
// the level's last nodes number their children and publish the next level's
// work lists (every level but the fused mode's deepest); the next level's
// expand reads this level's stored beliefs only after the grid barrier.
template <bool FUSED, bool NUMBER>
__device__ bool phase_level(const PlanDev &pl, int l, bool store, Smem &S, uint64_t *mbar, unsigned &mphase,
                            int &cur_e) {
    // the deepest fused level in its contraction form: ctr_item in place of
    // the group expand items
    const bool cform = !NUMBER && FUSED && ctr_level(pl, l);
    const int n_exp = cform ? __ldcg(pl.c_items + pl.E) : __ldcg(pl.grp_off + pl.gbase[l] + l + __ldcg(pl.ngrp + l));
    const int total = n_exp + __ldcg(pl.wb_fin + l * (pl.E + 1) + pl.E);
    unsigned *ctr = pl.work + 2 * l;
    for (int w = next_item(ctr, S.flags + 8); w < total; w = next_item(ctr, S.flags + 8)) {
        if (w < n_exp) {
            if (cform) ctr_item(pl, l, S, cur_e, w);
            else if (!expand_item<FUSED>(pl, l, store, S, mbar, mphase, cur_e, w, true)) return false;
        } else if (!NUMBER && __ldcg(pl.fchunks + l) == 0) {
            finalize_group_item<FUSED>(pl, l, S, cur_e, w - n_exp);
        } else {
            finalize_item<FUSED, NUMBER>(pl, l, S, cur_e, w - n_exp, true);
        }
    }
    return true;
}

// ---------------------------------------------------------------- update phase (Eq. 3)
__device__ bool phase_update(const PlanDev &pl, int l, Smem &S, uint64_t *mbar, unsigned &mphase, int &cur_e) {
    const int E = pl.E, K = pl.K;
    const int *wb = pl.wb_upd + l * (E + 1);
    const int total = __ldcg(wb + E);
    for (int w = blockIdx.x; w < total; w += gridDim.x) {
        const int e = find_episode(wb, E, w);
        load_ep(pl, e, S, cur_e);
        const EpDev &ep = *S.ep;
        const int items = __ldcg(pl.uitems + l * E + e);
        const int rel = w - __ldcg(wb + e);
        const int local = rel / items, item = rel - local * items;
        const long long ia = static_cast<long long>(ep.inode_base[l] + local) * 5;
        __syncthreads();
        if (threadIdx.x < 5) {
            S.u_n[threadIdx.x] = __ldcg(pl.nchild + ia + threadIdx.x);
            S.u_off[threadIdx.x] = __ldcg(pl.choff + ia + threadIdx.x);
        }
        for (int t = threadIdx.x; t < 5 * K; t += blockDim.x) {
            const int a = t / K, j = t - a * K;
            const long long sbi = (ia + a) * K + j;
            const float p = __ldcg(pl.slot_P + sbi);
            S.u_z[t] = __ldcg(pl.slot_z + sbi);
            S.u_sa[t] = ep.acc / p;
            S.u_se[t] = ep.eta / p;
        }
        const float *b = node_belief(pl, ep, l, local);
        float *child0 = pl.beliefs + ep.belief_off[l + 1];
        const int cap = ep.cap[l + 1];
        const int band0 = static_cast<int>((static_cast<long long>(item) * ep.bands) / items);
        const int band1 = static_cast<int>((static_cast<long long>(item + 1) * ep.bands) / items);
        const EpReg er = ep_reg(ep);
        const int P = er.P, P4 = P >> 2, goal = er.goal, band_rows = ep.band_rows, N = er.N;
        const float slip = er.slip;
        for (int band = band0; band < band1; ++band) {
            const int r0 = band * band_rows, r1 = min(er.H, r0 + band_rows);
            if (!stage_band(er, b, r0, r1, 1, S.sb, S.cw, nullptr, mbar, mphase, pl.status)) return false;
            const int ng = (r1 - r0) * P4;
            for (int gi = threadIdx.x; gi < ng; gi += blockDim.x) {
                const int rr = gi / P4, col = (gi - rr * P4) << 2;
                const int y = (r0 + rr) * P + col;
                Nbr4 n;
                load_nbr(er, S.sb + (rr + 1) * P, S.cw + (rr + 1) * P, col, n);
                float outs[4][5];
                int lab[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float nb[4];
                    inflow_nb(n, j, nb);
                    predict_cell(nb, n.m[j + 1], n.cw[j], (y + j) == goal, slip, S.lut, outs[j]);
                    lab[j] = QV_CELL_LABEL(n.cw[j]);
                }
#pragma unroll
                for (int a = 0; a < 5; ++a) {
                    const int cn = S.u_n[a], off = S.u_off[a];
                    for (int m = 0; m < cn; ++m) {
                        const int c = off + m;
                        if (c >= cap) break;
                        const int t = a * K + m;
                        const int z = S.u_z[t];
                        const float sa = S.u_sa[t], se = S.u_se[t];
                        float4 o;
                        o.x = outs[0][a] * (lab[0] == z ? sa : se);
                        o.y = outs[1][a] * (lab[1] == z ? sa : se);
                        o.z = outs[2][a] * (lab[2] == z ? sa : se);
                        o.w = outs[3][a] * (lab[3] == z ? sa : se);
                        if (!QV_IN_BOUNDS(kSiteBelief, ep.belief_off[l + 1] + static_cast<long long>(c) * N + y + 3,
                                          pl.n_belief))
                            continue;
                        __stcs(reinterpret_cast<float4 *>(child0 + static_cast<long long>(c) * N + y), o);
                    }
                }
            }
        }
    }
    return true;
}

// ---------------------------------------------------------------- leaf phase (Eq. 4)
// Work items are (group of kLeafGroup leaves, chunk of the grid); with more
// than one chunk the partial sums go to per-item records and the last chunk
// of a group adds them in chunk order.
__device__ void phase_leaf(const PlanDev &pl, int l, Smem &S, int &cur_e) {
    float(*s_red)[kLeafGroup * 5] = reinterpret_cast<float(*)[kLeafGroup * 5]>(S.red);
    const int *wb = pl.wb_leaf;
    const int total = __ldcg(wb + pl.E);
    const int C = max(1, __ldcg(pl.leaf_split));
    for (int w = blockIdx.x; w < total; w += gridDim.x) {
        const int e = find_episode(wb, pl.E, w);
        load_ep(pl, e, S, cur_e);
        const EpDev &ep = *S.ep;
        const int n = __ldcg(pl.count + l * pl.E + e);
        const int rel = w - __ldcg(wb + e);
        const int group = rel / C, chunk = rel - group * C;
        const int first = group * kLeafGroup;
        const int cnt = min(kLeafGroup, n - first);
        float acc[kLeafGroup][5];
#pragma unroll
        for (int i = 0; i < kLeafGroup; ++i)
#pragma unroll
            for (int a = 0; a < 5; ++a) acc[i][a] = 0.0f;
        const size_t plane = static_cast<size_t>(ep.N);
        const int n4 = ep.N >> 2;
        const int c0 = static_cast<int>((static_cast<long long>(chunk) * n4) / C);
        const int c1 = static_cast<int>((static_cast<long long>(chunk + 1) * n4) / C);
        // the group's leaf beliefs (streamed once from HBM) against Q (L2):
        // every load of kLeafUnroll consecutive float4 columns is issued
        // before the arithmetic that consumes them
        const float4 *bl[kLeafGroup];
#pragma unroll
        for (int i = 0; i < kLeafGroup; ++i)
            bl[i] = reinterpret_cast<const float4 *>(node_belief(pl, ep, l, first + min(i, cnt - 1)));
        const float4 *q4 = reinterpret_cast<const float4 *>(ep.Q);
        const int n4p = static_cast<int>(plane >> 2);
        constexpr int kLeafUnroll = 4;
        for (int i4 = c0 + threadIdx.x; i4 < c1; i4 += kLeafUnroll * blockDim.x) {
            float4 bv[kLeafUnroll][kLeafGroup];
#pragma unroll
            for (int u = 0; u < kLeafUnroll; ++u) {
                const int j4 = i4 + u * blockDim.x;
#pragma unroll
                for (int i = 0; i < kLeafGroup; ++i)
                    bv[u][i] = (j4 < c1 && i < cnt) ? __ldcs(bl[i] + j4) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < kLeafUnroll; ++u) {
                const int j4 = i4 + u * blockDim.x;
                if (j4 >= c1) break;
#pragma unroll
                for (int a = 0; a < 5; ++a) {
                    const float4 q = __ldg(q4 + a * n4p + j4);
#pragma unroll
                    for (int i = 0; i < kLeafGroup; ++i)
                        acc[i][a] = fmaf(bv[u][i].x, q.x,
                                         fmaf(bv[u][i].y, q.y, fmaf(bv[u][i].z, q.z, fmaf(bv[u][i].w, q.w, acc[i][a]))));
                }
            }
        }
        const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
        __syncthreads();
        {
            static_assert(kLeafGroup * 5 <= 32, "one reduce-scatter covers a leaf group");
            float v[32];
#pragma unroll
            for (int i = 0; i < kLeafGroup; ++i)
#pragma unroll
                for (int a = 0; a < 5; ++a) v[i * 5 + a] = acc[i][a];
#pragma unroll
            for (int i = kLeafGroup * 5; i < 32; ++i) v[i] = 0.0f;
            warp_reduce_scatter32(v);
            if (lane < kLeafGroup * 5) s_red[wid][lane] = v[0];
        }
        __syncthreads();
        if (threadIdx.x < kLeafGroup * 5) {
            float t = 0.0f;
            for (int k = 0; k < kWarps; ++k) t += s_red[k][threadIdx.x];
            S.tot[threadIdx.x] = t;
        }
        __syncthreads();
        if (C > 1) {
            float *rec = pl.partials + static_cast<long long>(w) * pl.rec_len;
            if (threadIdx.x < kLeafGroup * 5) rec[threadIdx.x] = S.tot[threadIdx.x];
            __syncthreads();
            if (threadIdx.x == 0) {
                const unsigned key = static_cast<unsigned>(w / C);
                const unsigned prev = arrive_acq_rel(pl.leaf_cnt + key);
                const int last = prev == static_cast<unsigned>(C - 1);
                if (last) pl.leaf_cnt[key] = 0u;
                S.flags[3] = last;
            }
            __syncthreads();
            if (!S.flags[3]) continue;
            if (threadIdx.x < kLeafGroup * 5) {
                const float *base = pl.partials + static_cast<long long>(w - chunk) * pl.rec_len;
                float t = 0.0f;
                for (int c = 0; c < C; ++c) t += __ldcg(base + static_cast<long long>(c) * pl.rec_len + threadIdx.x);
                S.tot[threadIdx.x] = t;
            }
            __syncthreads();
        }
        if (threadIdx.x < cnt) {
            const int i = threadIdx.x;
            float sums[5];
            float best = -3.402823466e38f;
            int ba = 0;
            for (int a = 0; a < 5; ++a) {
                const float t = S.tot[i * 5 + a];
                sums[a] = t;
                if (t > best) {
                    best = t;
                    ba = a;
                }
            }
            if (!QV_IN_BOUNDS(kSiteNode, ep.node_base[l] + first + i, pl.n_nodes)) return;
            pl.value[ep.node_base[l] + first + i] = best;
            pl.leaf_arg[ep.node_base[l] + first + i] = ba;
            if (l == 0) {  // depth-0 plan: the root is the leaf
                ResultDev r;
                r.action = ba;
                r.value = best;
                for (int a = 0; a < 5; ++a) r.q[a] = sums[a];
                r.pad = 0;
                if (QV_IN_BOUNDS(kSiteEpisode, e, pl.E)) pl.result[e] = r;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- backup phase (Alg. 6, 7)
// Records of the leaves, which nothing read before, from every (node,
// action) pair of the deepest internal level.  `write_value`: fused leaves,
// whose values live in the sample slots.
// One leaf record per call: t indexes the (node, action, sample slot)
// triples of level l, so every slot's loads are independent of the others.
__device__ __forceinline__ void leaf_records(const PlanDev &pl, const EpDev &ep, int l, int t, bool write_value) {
    const int K = pl.K, nz = ep.B + 1;
    const int node = t / (5 * K), a = (t / K) % 5, j = t % K;
    const long long ia = static_cast<long long>(ep.inode_base[l] + node) * 5 + a;
    if (!QV_IN_BOUNDS(kSiteInode, ep.inode_base[l] + node, pl.n_inodes)) return;
    const int m = __ldcg(pl.nchild + ia);
    if (j >= m) return;
    const int off = __ldcg(pl.choff + ia);
    if (off + j >= ep.cap[l + 1]) return;
    const long long sb = ia * K + j;
    const unsigned long long pcode = __ldcg(pl.code + ep.node_base[l] + node);
    const int z = __ldcg(pl.slot_z + sb);
    const float w = __ldcg(pl.slot_w + sb), p = __ldcg(pl.slot_P + sb);
    float v = 0.0f;
    int arg = 0;
    if (write_value) {
        v = __ldcg(pl.slot_val + sb);
        arg = __ldcg(pl.slot_arg + sb);
    }
    const int g = ep.node_base[l + 1] + off + j;
    if (!QV_IN_BOUNDS(kSiteNode, g, pl.n_nodes)) return;
    pl.parent[g] = node;
    pl.action[g] = a;
    pl.obs[g] = z;
    pl.weight[g] = w;
    pl.pz[g] = p;
    pl.code[g] = (pcode * 5ull + a) * static_cast<unsigned long long>(nz) + z;
    if (write_value) {
        pl.value[g] = v;
        pl.leaf_arg[g] = arg;
    }
}

// Fused leaves: the deepest internal level already holds U_Q and U_V (from
// its finalisation); every CTA writes leaf records, one CTA per episode backs
// up the levels above.  Materialised leaves: one CTA per episode backs up
// every level.  Each level handles its (node, action) pairs in parallel.
// D: the depth of the tree built (the plan's depth, or less when its
// deadline ran out; then the leaves' records are written here and the
// counts of the levels not built are cleared).
__device__ void phase_backup(const PlanDev &pl, Smem &S, int &cur_e, int D) {
    const int K = pl.K;
    const bool fused = pl.leaf_mode != QV_LEAF_MATERIALISE;
    const bool cut = D < pl.depth;
    if (fused) {
        // number the leaves of every episode (the children of the fused
        // level), on CTAs other than those that back the episode up when
        // there are enough; their records are written on demand
        // (k_leaf_records), or here when the search stopped early
        const int first = gridDim.x >= 2 * pl.E ? pl.E : 0;
        for (int e = static_cast<int>(blockIdx.x) - first; e >= 0 && e < pl.E;
             e += static_cast<int>(gridDim.x) - first) {
            load_ep(pl, e, S, cur_e);
            compact_episode(pl, D - 1, *S.ep, e, S);
            if (cut) {
                const int n = __ldcg(pl.count + (D - 1) * pl.E + e);
                for (int t = threadIdx.x; t < 5 * K * n; t += blockDim.x) leaf_records(pl, *S.ep, D - 1, t, true);
                for (int l = D + 1 + threadIdx.x; l <= pl.depth; l += blockDim.x) pl.count[l * pl.E + e] = 0;
            }
        }
    }
    for (int e = blockIdx.x; e < pl.E; e += gridDim.x) {
        load_ep(pl, e, S, cur_e);
        const EpDev &ep = *S.ep;
        for (int l = fused ? D - 2 : D - 1; l >= 0; --l) {
            const int n = __ldcg(pl.count + l * pl.E + e);
            for (int t = threadIdx.x; t < 5 * n; t += blockDim.x) {
                const int node = t / 5, a = t - node * 5;
                const long long ia = static_cast<long long>(ep.inode_base[l] + node) * 5 + a;
                const int m = __ldcg(pl.nchild + ia), off = __ldcg(pl.choff + ia);
                const long long sb = ia * K;
                const float *vals = pl.value + ep.node_base[l + 1] + off;
                float s = 0.0f;
                // loads of a batch of children issued together, summed in order
                for (int j0 = 0; j0 < m; j0 += 8) {
                    float wv[8], vv[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        wv[i] = j0 + i < m ? __ldcg(pl.slot_w + sb + j0 + i) : 0.0f;
                        vv[i] = j0 + i < m ? __ldcg(vals + j0 + i) : 0.0f;
                    }
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        if (j0 + i < m) s = fmaf(wv[i], vv[i], s);
                }
                pl.UQ[ia] = fmaf(ep.gamma, s, __ldcg(pl.R + ia));
                if (!fused && l == D - 1)
                    for (int j = 0; j < K; ++j) leaf_records(pl, ep, l, t * K + j, false);
            }
            __syncthreads();
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const long long ia = static_cast<long long>(ep.inode_base[l] + i) * 5;
                float best = pl.UQ[ia];
                for (int a = 1; a < 5; ++a) best = fmaxf(best, pl.UQ[ia + a]);
                pl.value[ep.node_base[l] + i] = best;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            const long long ia = static_cast<long long>(ep.inode_base[0]) * 5;
            ResultDev r;
            float q[5];
            int best = 0;
            for (int a = 0; a < 5; ++a) {
                q[a] = __ldcg(pl.UQ + ia + a);
                if (q[a] > q[best]) best = a;
            }
            r.action = best;
            for (int a = 0; a < 5; ++a) r.q[a] = q[a];
            r.value = __ldcg(pl.value + ep.node_base[0]);
            r.pad = D;  // the depth reached
            if (QV_IN_BOUNDS(kSiteEpisode, e, pl.E)) pl.result[e] = r;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- the plan kernel
__global__ void __launch_bounds__(kThreads, 2) k_plan(PlanDev pl) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t mbar;
    const SmemLayout L =
        SmemLayout::make(pl.sb_floats, pl.sp_floats, pl.q_floats, pl.Bmax, pl.K, pl.cmax, pl.kslots);
    Smem S;
    S.sb = reinterpret_cast<float *>(smem_raw + L.sb);
    S.tile = reinterpret_cast<float *>(smem_raw + L.tile);
    S.acc = reinterpret_cast<float *>(smem_raw + L.acc);
    S.c_pa = reinterpret_cast<int *>(smem_raw + L.c_pa);
    S.c_z = reinterpret_cast<int *>(smem_raw + L.c_z);
    S.c_sa = reinterpret_cast<float *>(smem_raw + L.c_sa);
    S.c_se = reinterpret_cast<float *>(smem_raw + L.c_se);
    S.wpart = reinterpret_cast<float *>(smem_raw + L.wpart);
    S.wchild = reinterpret_cast<int *>(smem_raw + L.wchild);
    S.sp = reinterpret_cast<float *>(smem_raw + L.sp);
    S.cw = reinterpret_cast<uint16_t *>(smem_raw + L.cw);
    S.q = reinterpret_cast<float *>(smem_raw + L.q);
    S.ep = reinterpret_cast<EpDev *>(smem_raw + L.ep);
    S.bco = reinterpret_cast<int *>(smem_raw + L.bco);
    S.hist = reinterpret_cast<float *>(smem_raw + L.hist);
    S.histq = reinterpret_cast<float *>(smem_raw + L.histq);
    S.tot = reinterpret_cast<float *>(smem_raw + L.tot);
    S.red = reinterpret_cast<float *>(smem_raw + L.red);
    S.P = reinterpret_cast<float *>(smem_raw + L.P);
    S.C = reinterpret_cast<float *>(smem_raw + L.C);
    S.cnt = reinterpret_cast<int *>(smem_raw + L.cnt);
    S.T = reinterpret_cast<float *>(smem_raw + L.T);
    S.uq = reinterpret_cast<float *>(smem_raw + L.uq);
    S.lut = reinterpret_cast<float *>(smem_raw + L.lut);
    S.lut4 = reinterpret_cast<float4 *>(smem_raw + L.lut4);
    S.u_n = reinterpret_cast<int *>(smem_raw + L.u_n);
    S.u_off = reinterpret_cast<int *>(smem_raw + L.u_off);
    S.u_z = reinterpret_cast<int *>(smem_raw + L.u_z);
    S.u_sa = reinterpret_cast<float *>(smem_raw + L.u_sa);
    S.u_se = reinterpret_cast<float *>(smem_raw + L.u_se);
    S.scan = reinterpret_cast<int *>(smem_raw + L.scan);
    S.flags = reinterpret_cast<int *>(smem_raw + L.flags);
    S.nband = static_cast<int>((L.band_end - L.sb) / 4);
    if (threadIdx.x == 0) {
        mbar_init(&mbar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    unsigned mphase = 0;
    int cur_e = -1;
    int slot = 0;
    stamp(pl, slot++);
    const int D = pl.depth;
    const bool mat = pl.leaf_mode == QV_LEAF_MATERIALISE;
    // with a deadline every level also forms its children's leaf values, so
    // that the search can stop after any level (anytime, Sec. IV-C)
    const bool dl = pl.deadline_ns != 0ull;
    int Deff = D;
    if (D > 0) {
        phase_window(pl, S);
        if (!grid_sync(pl)) return;
    }
    for (int l = 0; l < D; ++l) {
        const bool last = l == D - 1;
        const bool fused = (last && !mat) || dl;
        // a level's beliefs are stored when a later phase reads them
        const bool store = l > 0 && (l < D - 1 || mat);
        // expand and finalize of the level in one phase
        bool ok;
        if (last && !mat) ok = phase_level<true, false>(pl, l, false, S, &mbar, mphase, cur_e);
        else if (fused) ok = phase_level<true, true>(pl, l, store, S, &mbar, mphase, cur_e);
        else ok = phase_level<false, true>(pl, l, store, S, &mbar, mphase, cur_e);
        if (!ok && threadIdx.x == 0) atomicOr(pl.status, kErrTimeout);
        if (!grid_sync(pl, dl && !last)) return;
        stamp(pl, slot++);
        if (dl && !last) {
            if (threadIdx.x == 0) S.flags[5] = static_cast<int>(*((volatile unsigned *)(pl.status + 1)));
            __syncthreads();
            if (S.flags[5]) {
                Deff = l + 1;
                break;
            }
        }
    }
    if (D > 0 && mat) {
        if (!phase_update(pl, D - 1, S, &mbar, mphase, cur_e) && threadIdx.x == 0) atomicOr(pl.status, kErrTimeout);
        if (!grid_sync(pl)) return;
        stamp(pl, slot++);
    }
    if (D == 0 || mat) {
        phase_leaf(pl, D, S, cur_e);
        if (!grid_sync(pl)) return;
        stamp(pl, slot++);
    }
    // every reader of the support windows is past the last grid barrier:
    // each stored level's dirty box takes in the window this run wrote, then
    // the windows are cleared for the next run's root pass to find afresh
    if (blockIdx.x == 0) {
        for (int i = threadIdx.x; i < pl.E * D; i += blockDim.x) {
            const int e = i / D, l = i - e * D;
            if (l == 0 || l >= Deff || !(l < D - 1 || mat)) continue;
            const EpDev *ep = pl.eps + e;
            const BandGeo geo = band_geo(pl, e, __ldg(&ep->H), __ldg(&ep->W), __ldg(&ep->P), __ldg(&ep->band_rows), l);
            if (geo.nb == 0) continue;
            int *dw = pl.dirty + 4 * (l * pl.E + e);
            int r0 = geo.r0, r1 = geo.r1, g0 = geo.g0, g1 = geo.g1;
            if (dw[0] != 0) {
                r0 = min(r0, dw[0] - 1);
                r1 = max(r1, dw[1]);
                g0 = min(g0, dw[2]);
                g1 = max(g1, dw[3]);
            }
            dw[0] = r0 + 1;
            dw[1] = r1;
            dw[2] = g0;
            dw[3] = g1;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < 4 * pl.E; i += blockDim.x) pl.win[i] = 0u;
        for (int i = threadIdx.x; i < 2 * (D + 1); i += blockDim.x) pl.work[i] = 0u;
        for (int l = 0; l < Deff; ++l) {  // the group counters of every level run
            const int ng = __ldcg(pl.ngrp + l);
            for (int i = threadIdx.x; i < ng; i += blockDim.x) pl.grp_done[pl.gbase[l] + i] = 0u;
        }
    }
    if (D > 0) {
        phase_backup(pl, S, cur_e, Deff);
        stamp(pl, slot++);
    }
}

// Records (parent, action, observation, weight, P(z), path code, value,
// argmax) of the fused mode's leaves, written on demand after a run: one
// thread per (episode, node, action, sample slot) of the deepest internal
// level.
__global__ void __launch_bounds__(256) k_leaf_records(PlanDev pl) {
    const int D = pl.depth, K = pl.K;
    for (int e = 0; e < pl.E; ++e) {
        if (pl.result[e].pad < D) continue;  // stopped early: its leaves' records are written
        const EpDev &ep = pl.eps[e];
        const int n = __ldcg(pl.count + (D - 1) * pl.E + e);
        for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 5 * K * n; t += gridDim.x * blockDim.x)
            leaf_records(pl, ep, D - 1, t, true);
    }
}

}  // namespace qv
