// qv_common.cuh -- device helpers shared by the QV-Tree Search kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <stdint.h>

#include "../../include/qvts.h"

// ---------------------------------------------------------------------------
// Cell word (uint16 per grid cell), written by qv_model_build.
//   bits 0..3   blocked[D]: neighbour in direction D (N, E, S, W) is occupied
//               or outside the grid, so a move that way stays put (Eq. 10)
//   bits 4..7   inflow[D]: this cell is free and its neighbour in direction D
//               is a free, non-goal cell, so that neighbour's moves can land here
//   bits 8..14  observation label (0..B, B = null)
//   bit  15     free
// ---------------------------------------------------------------------------
#define QV_CELL_BLOCKED(w) ((w) & 0xFu)
#define QV_CELL_INFLOW(w) (((w) >> 4) & 0xFu)
#define QV_CELL_LABEL(w) (((w) >> 8) & 0x7Fu)
#define QV_CELL_FREE(w) (((w) >> 15) & 1u)

namespace qv {

constexpr int kA = QV_NUM_ACTIONS;
constexpr int kDirN = 0, kDirE = 1, kDirS = 2, kDirW = 3;

// Device status word bits (written by kernels, read by the host after a run).
constexpr unsigned kErrTimeout = 1u;
constexpr unsigned kErrCapacity = 2u;
constexpr unsigned kErrInput = 4u;
constexpr unsigned kErrBounds = 8u;  // a device bounds check failed (bounds-checked debug build)

// Bounded spin: after this many polls a wait gives up and reports a timeout.
// Waits on the CTA's own bulk copies always use it; waits on other CTAs (grid
// barriers, progress flags) use the limit the host passes in, which is this
// one unless a timeout is injected (qv_cross_spin_limit).
constexpr unsigned kSpinLimit = 1u << 22;

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// ---- mbarrier + bulk (TMA, non-tensor) copy global -> shared --------------
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
// Contiguous copy of `bytes` (multiple of 16, both addresses 16-byte aligned)
// from global memory into this CTA's shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, unsigned bytes,
                                              uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for phase `parity` of `bar`; false when the limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity) {
    for (unsigned i = 0; i < kSpinLimit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// ---- reductions ----------------------------------------------------------
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
// Reduce-scatter over a warp: on entry every lane holds 32 values v[0..31];
// on exit v[0] of lane i is the sum over the 32 lanes of their v[i].  Each
// halving step swaps half of the live values with the partner lane, so the
// whole reduction takes 31 shuffles instead of 32 separate 5-shuffle sums.
__device__ __forceinline__ void warp_reduce_scatter32(float v[32]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < o; ++i) {
            const float send = upper ? v[i] : v[i + o];
            const float keep = upper ? v[i + o] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        T u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u > v ? u : v;
    }
    return v;
}

// ---- Philox4x32-10 (Salmon et al., SC'11) --------------------------------
struct U4 {
    uint32_t x, y, z, w;
};
__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        U4 n;
        n.x = hi1 ^ c.y ^ k0;
        n.y = lo1;
        n.z = hi0 ^ c.w ^ k1;
        n.w = lo0;
        c = n;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}
// k-th uniform of the stream of one (V-node at `level`, action) whose
// mixed-radix path code is `path`: exact in FP32, in (0, 1).
__device__ __forceinline__ float sample_uniform(uint64_t seed, uint32_t episode, int level,
                                                uint64_t path, int k) {
    U4 c;
    c.x = static_cast<uint32_t>(k >> 2);
    c.y = episode;
    c.z = static_cast<uint32_t>(path & 0xFFFFFFFFull);
    c.w = (static_cast<uint32_t>(level) << 24) | static_cast<uint32_t>(path >> 32);
    const U4 r = philox4x32_10(c, static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
    const int j = k & 3;
    const uint32_t w = j == 0 ? r.x : j == 1 ? r.y : j == 2 ? r.z : r.w;
    return static_cast<float>(2u * (w >> 9) + 1u) * (1.0f / 16777216.0f);
}

// ---- the motion stencil (Eq. 3 numerator with Eq. 10) --------------------
// Self-transition weight of a free, non-goal cell for action a < 4, given
// its blocked-neighbour nibble: the intended move and the two perpendicular
// slips that hit a blocked neighbour stay on the cell.
__host__ __device__ __forceinline__ float self_weight(int a, unsigned blocked, float slip) {
    const float fwd = 1.0f - 2.0f * slip;
    const unsigned p1 = (a + 1) & 3, p2 = (a + 3) & 3;
    return fwd * ((blocked >> a) & 1u) + slip * (((blocked >> p1) & 1u) + ((blocked >> p2) & 1u));
}

// Predicted mass at one cell for all five actions.  nb[D] = inflow-masked
// belief of the neighbour in direction D; self = belief of the cell itself.
// For action a the intended move comes from the neighbour opposite to a's
// step, the slips from the two neighbours perpendicular to it.
__device__ __forceinline__ void predict_cell(const float nb[4], float self, unsigned cw, bool is_goal,
                                             float slip, const float *self_lut, float out[5]) {
    const float fwd = 1.0f - 2.0f * slip;
    const unsigned blk = QV_CELL_BLOCKED(cw);
    const float s = QV_CELL_FREE(cw) ? self : 0.0f;
    // a = N: intended from S, slips from E and W
    out[0] = fmaf(fwd, nb[kDirS], slip * (nb[kDirE] + nb[kDirW]));
    out[1] = fmaf(fwd, nb[kDirW], slip * (nb[kDirN] + nb[kDirS]));
    out[2] = fmaf(fwd, nb[kDirN], slip * (nb[kDirE] + nb[kDirW]));
    out[3] = fmaf(fwd, nb[kDirE], slip * (nb[kDirN] + nb[kDirS]));
    if (is_goal) {
#pragma unroll
        for (int a = 0; a < 4; ++a) out[a] += s;
    } else {
#pragma unroll
        for (int a = 0; a < 4; ++a) out[a] = fmaf(self_lut[a * 16 + blk], s, out[a]);
    }
    out[4] = s;
}

// Predicted mass at one cell for one action a (uniform across the warp):
// the same arithmetic as predict_cell's out[a], without the other four.
__device__ __forceinline__ float predict_one(const float nb[4], float self, unsigned cw, bool is_goal, float slip,
                                             const float *self_lut, int a) {
    const float s = QV_CELL_FREE(cw) ? self : 0.0f;
    if (a == 4) return s;
    const float fwd = 1.0f - 2.0f * slip;
    // intended move from the neighbour opposite a's step, slips from the two
    // perpendicular ones (in predict_cell's order of summation)
    const float n_in = a == 0 ? nb[kDirS] : a == 1 ? nb[kDirW] : a == 2 ? nb[kDirN] : nb[kDirE];
    const float n_p1 = (a & 1) ? nb[kDirN] : nb[kDirE];
    const float n_p2 = (a & 1) ? nb[kDirS] : nb[kDirW];
    const float v = fmaf(fwd, n_in, slip * (n_p1 + n_p2));
    return is_goal ? v + s : fmaf(self_lut[a * 16 + QV_CELL_BLOCKED(cw)], s, v);
}

// Stage reward of arriving in a cell: +100 at the goal, -1 - c(y) otherwise.
__device__ __forceinline__ float stage_reward(bool free_cell, bool is_goal, float cost) {
    return !free_cell ? 0.0f : (is_goal ? 100.0f : -1.0f - cost);
}

}  // namespace qv

// Host-side error reporting shared by the entry points (defined in qv_api.cu).
qv_status qv_set_error(qv_status st, const char *fmt, ...);
qv_status qv_check_cuda(cudaError_t e, const char *what);
int qv_num_sms();
// Poll limit for waits on other CTAs: kSpinLimit, or 0 when the environment
// variable QVTS_FAULT is "timeout" (host-side fault injection: every such wait
// that is not already satisfied gives up at once and reports QV_ERR_TIMEOUT,
// so the timeout path runs without a real hang).
unsigned qv_cross_spin_limit();
// Host-side fault injection by the environment variable QVTS_FAULT, checked
// on entry before any device work: "oom" makes calls that take a workspace
// return QV_ERR_WORKSPACE (the library's out-of-memory: it allocates no
// device memory itself), "invalid" makes the instrumented calls return
// QV_ERR_INVALID; each leaves a message naming the injection.
qv_status qv_injected_fault(const char *where, bool takes_workspace);
// QVTS_FAULT=bounds: the device bounds check whose site number this returns
// (1, the node records) reports a failure on every run although its index is
// in range (bounds-checked debug build only; 0 = no injection).
unsigned qv_bounds_injected_site();

// NVTX range over a host-side call (NVTX v3, header only): a profiler that
// reads NVTX (nsys, ncu --nvtx) shows every launching entry point as
// "qvts:<name>" and, where the host issues a tree's levels one by one, each
// level as "qvts:<name> level <l>".  Without a tool attached a push or pop is
// a call through a null-checked function pointer.  The plan kernel runs all of
// a tree's levels inside one launch, so its per-level times come from the
// device clock stamps (qv_plan_profile), not from ranges.
struct QvRange {
    explicit QvRange(const char *name);
    QvRange(const char *name, int level);
    ~QvRange();
    QvRange(const QvRange &) = delete;
    QvRange &operator=(const QvRange &) = delete;
};
#define QV_RANGE(...) QvRange qv_nvtx_range_(__VA_ARGS__)
