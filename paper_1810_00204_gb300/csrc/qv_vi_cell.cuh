// qv_vi_cell.cuh -- the per-cell Bellman backup of the value iteration and
// the bounded cross-CTA waits of row-band sweeps, shared by the forward
// sweeps (qv_vi.cu), the sweeps the adjoint recomputes from checkpoints
// (qv_adjoint.cu) and the FIB iteration (qv_fib.cu), so all run the same
// arithmetic and the same synchronisation.  For the cell backup `Args`
// provides P (row pitch), cost, goal, slip and gamma (of type T).
#pragma once

#include "qv_common.cuh"

namespace qv {

struct VIWork {
    unsigned bar_count;
    unsigned bar_gen;
    unsigned status;
    unsigned pad;
};

// Progress flags of a row-band decomposition (one band per CTA, in CTA
// order): CTA i publishes how many steps it has completed; a step whose
// reads reach one row into the neighbouring bands waits only for CTAs i - 1
// and i + 1 to have completed the step before.  That also keeps every CTA
// within one step of its neighbours, so a step may overwrite a buffer its
// neighbours read two steps back.
__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
static __device__ void publish_step(unsigned *done, unsigned step) {
    __syncthreads();  // every thread's writes of the step precede thread 0's release
    if (threadIdx.x == 0) st_release(done + blockIdx.x, step);
}
// Bounded wait for CTAs blockIdx.x +- 1 to reach `step` (lanes 0 and 1 of
// warp 0 watch one each); false (status bit set, every CTA then leaves) when
// the limit ran out.
static __device__ bool wait_neighbours(const unsigned *done, unsigned step, unsigned *status, unsigned limit) {
    __shared__ int s_ok;
    if (threadIdx.x < 32) {
        int ok = 1;
        if (threadIdx.x < 2) {
            const int nb = static_cast<int>(blockIdx.x) + (threadIdx.x == 0 ? -1 : 1);
            if (nb >= 0 && nb < static_cast<int>(gridDim.x)) {
                unsigned i = 0;
                while (ld_acquire(done + nb) < step) {
                    if (++i > limit || (*((volatile unsigned *)status) & kErrTimeout)) {
                        atomicOr(status, kErrTimeout);
                        ok = 0;
                        break;
                    }
                    __nanosleep(32);
                }
            }
        }
        ok = __all_sync(0xffffffffu, ok);
        if (threadIdx.x == 0) s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Row-band sweeps (the value iteration, the FIB iteration) share the two
// pieces below.  `Args` provides H, work, truncated, res_slots, arrive and
// spin_limit.

// Residual slots are a ring of this many sweeps: a slot is rewritten four
// sweeps later, after every CTA has passed the test that read it.
constexpr int kResRing = 4;

// Stage grid rows [c0-1, c1+1) of `src` (clipped to the grid; `row_elems`
// elements a row) into smem rows 0.. of Vs with one bulk copy.  False when
// the wait ran out (after a second bounded wait for the copy still in
// flight).
template <typename T, typename Args>
__device__ bool stage_rows(const Args &a, T *Vs, const T *src, int c0, int c1, int row_elems, uint64_t *bar,
                           unsigned &phase) {
    const int lo = max(0, c0 - 1), hi = min(a.H, c1 + 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("fence.proxy.async.global;" ::: "memory");
        fence_proxy_async();
        const unsigned bytes = static_cast<unsigned>((hi - lo) * row_elems * sizeof(T));
        mbar_arrive_expect_tx(bar, bytes);
        bulk_copy_g2s(Vs + (lo - (c0 - 1)) * row_elems, src + static_cast<size_t>(lo) * row_elems, bytes, bar);
    }
    const bool ok = mbar_wait_bounded(bar, phase);
    // one decision for the whole CTA, so an early exit never splits it
    const int failed = __syncthreads_or(ok ? 0 : 1);
    if (failed) {
        if (threadIdx.x == 0) atomicOr(&a.work->status, kErrTimeout);
        if (!ok) mbar_wait_bounded(bar, phase);  // let the copy in flight land before leaving
    }
    phase ^= 1u;
    return failed == 0;
}

// Largest residual of sweep j over every CTA: wait until all CTAs have
// posted it (a cumulative arrival count per ring slot), then every thread
// reads the slots.  Same value in every CTA.
template <typename T, typename Args>
__device__ bool sweep_residual(const Args &a, int j, T &res) {
    __shared__ int s_ok;
    __shared__ T s_m[8];
    const unsigned nblocks = gridDim.x;
    if (threadIdx.x == 0) {
        // every sweep posts when there is a stopping test; a truncated run
        // posts its last sweep only
        const unsigned want = a.truncated > 0 ? nblocks : nblocks * static_cast<unsigned>(j / kResRing + 1);
        unsigned i = 0;
        int ok = 1;
        while (ld_acquire(a.arrive + j % kResRing) < want) {
            if (++i > a.spin_limit || (*((volatile unsigned *)&a.work->status) & kErrTimeout)) {
                atomicOr(&a.work->status, kErrTimeout);
                ok = 0;
                break;
            }
            __nanosleep(32);
        }
        s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) return false;
    T m = T(0);
    const T *slot = a.res_slots + static_cast<size_t>(j % kResRing) * nblocks;
    for (unsigned b = threadIdx.x; b < nblocks; b += blockDim.x) {
        const T v = __ldcg(slot + b);
        m = v > m ? v : m;
    }
    m = warp_max(m);
    if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = m;
    __syncthreads();
    m = T(0);
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) m = s_m[w] > m ? s_m[w] : m;
    __syncthreads();
    res = m;
    return true;
}

// Temporally blocked sweeps (k_vi_blocked, k_fib_blocked) run at most this
// many sweeps between two exchanges with the neighbouring CTAs; `Args`
// provides s, bres ([kResRing][kMaxBlock][gridDim.x] per-sweep residuals of
// a block), arrive, tol, work and spin_limit.
constexpr int kMaxBlock = 8;

// Bounded wait for the CTAs within nh of this one to have completed `step`
// blocks (lane c of warp 0 watches CTA blockIdx.x - nh + c).
static __device__ bool wait_range(const unsigned *done, unsigned step, int nh, unsigned *status, unsigned limit) {
    __shared__ int s_ok;
    if (threadIdx.x < 32) {
        int ok = 1;
        const int nb = static_cast<int>(blockIdx.x) - nh + static_cast<int>(threadIdx.x) +
                       (static_cast<int>(threadIdx.x) >= nh ? 1 : 0);  // skip this CTA
        if (static_cast<int>(threadIdx.x) < 2 * nh && nb >= 0 && nb < static_cast<int>(gridDim.x)) {
            unsigned i = 0;
            while (ld_acquire(done + nb) < step) {
                if (++i > limit || (*((volatile unsigned *)status) & kErrTimeout)) {
                    atomicOr(status, kErrTimeout);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        ok = __all_sync(0xffffffffu, ok);
        if (threadIdx.x == 0) s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// The stopping test of block bt: waits (bounded) until every CTA has posted
// it, then f = the first sweep k of the block whose largest residual is below
// tol (-1 if none) and r = that residual; with last_only, r = the residual of
// the block's last sweep (a truncated run).  Same result in every CTA.
template <typename T, typename Args>
__device__ bool block_test(const Args &a, int bt, int ns, bool last_only, int &f, T &r) {
    __shared__ int s_ok;
    __shared__ T s_m[kMaxBlock];
    const unsigned G = gridDim.x;
    if (threadIdx.x == 0) {
        const unsigned want = G * static_cast<unsigned>(bt / kResRing + 1);
        unsigned i = 0;
        int ok = 1;
        while (ld_acquire(a.arrive + bt % kResRing) < want) {
            if (++i > a.spin_limit || (*((volatile unsigned *)&a.work->status) & kErrTimeout)) {
                atomicOr(&a.work->status, kErrTimeout);
                ok = 0;
                break;
            }
            __nanosleep(32);
        }
        s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) return false;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const T *slot = a.bres + static_cast<size_t>(bt % kResRing) * kMaxBlock * G;
    for (int j = wid; j < ns; j += static_cast<int>(blockDim.x >> 5)) {
        T m = T(0);
        for (unsigned c = lane; c < G; c += 32) {
            const T v = __ldcg(slot + static_cast<size_t>(j) * G + c);
            m = v > m ? v : m;
        }
        m = warp_max(m);
        if (lane == 0) s_m[j] = m;
    }
    __syncthreads();
    f = -1;
    r = s_m[ns - 1];
    if (!last_only)
        for (int j = 0; j < ns; ++j)
            if (s_m[j] < a.tol) {
                f = bt * a.s + j;
                r = s_m[j];
                break;
            }
    __syncthreads();
    return true;
}

template <typename T, typename Args>
__device__ __forceinline__ T arrive_value(const Args &a, int y, const T *Vs_row, int col) {
    // r(y) + gamma V(y) for a free cell y
    const float c = a.cost ? __ldg(a.cost + y) : 0.0f;
    const T r = (y == a.goal) ? T(100) : T(-1) - T(c);
    return r + a.gamma * Vs_row[col];
}

// Q_a(x) for the 5 actions from the arrival values r(y) + gamma V(y) of x
// (wx) and of its four neighbours (wn, taken only where the move is not
// blocked; a blocked move stays at x).
template <typename T>
__device__ __forceinline__ void q_from_arrivals(unsigned blk, T wx, T wn[4], float slip, T q[5]) {
    if (blk & 1u) wn[kDirN] = wx;
    if (blk & 2u) wn[kDirE] = wx;
    if (blk & 4u) wn[kDirS] = wx;
    if (blk & 8u) wn[kDirW] = wx;
    const T fwd = T(1) - T(2) * T(slip), eps = T(slip);
#pragma unroll
    for (int d = 0; d < 4; ++d) q[d] = fwd * wn[d] + eps * (wn[(d + 1) & 3] + wn[(d + 3) & 3]);
    q[4] = wx;
}

// Q_a(x) for the 5 actions of a free, non-goal cell, V staged in smem rows
// (row stride P) where `rowp` points at x's row.
template <typename T, typename Args>
__device__ __forceinline__ void cell_q(const Args &a, int y, int col, unsigned cw, const T *rowp,
                                       T q[5]) {
    const unsigned blk = QV_CELL_BLOCKED(cw);
    const T wx = arrive_value(a, y, rowp, col);
    T wn[4];
    wn[kDirN] = (blk & 1u) ? wx : arrive_value(a, y - a.P, rowp - a.P, col);
    wn[kDirE] = (blk & 2u) ? wx : arrive_value(a, y + 1, rowp, col + 1);
    wn[kDirS] = (blk & 4u) ? wx : arrive_value(a, y + a.P, rowp + a.P, col);
    wn[kDirW] = (blk & 8u) ? wx : arrive_value(a, y - 1, rowp, col - 1);
    q_from_arrivals(blk, wx, wn, a.slip, q);
}

}  // namespace qv
