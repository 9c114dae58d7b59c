// qv_vi_cell.cuh -- the per-cell Bellman backup of the value iteration and
// its bounded grid barrier, shared by the forward sweeps (qv_vi.cu) and the
// sweeps the adjoint recomputes from checkpoints (qv_adjoint.cu), so both run
// the same arithmetic.  `Args` provides P (row pitch), cost, goal, slip and
// gamma (of type T).
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

template <typename T, typename Args>
__device__ __forceinline__ T arrive_value(const Args &a, int y, const T *Vs_row, int col) {
    // r(y) + gamma V(y) for a free cell y
    const float c = a.cost ? __ldg(a.cost + y) : 0.0f;
    const T r = (y == a.goal) ? T(100) : T(-1) - T(c);
    return r + a.gamma * Vs_row[col];
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
    const T fwd = T(1) - T(2) * T(a.slip), eps = T(a.slip);
#pragma unroll
    for (int d = 0; d < 4; ++d) q[d] = fwd * wn[d] + eps * (wn[(d + 1) & 3] + wn[(d + 3) & 3]);
    q[4] = wx;
}

}  // namespace qv
