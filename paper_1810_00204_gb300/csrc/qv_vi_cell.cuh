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

// Bounded grid barrier (all CTAs co-resident through a cooperative launch).
static __device__ bool grid_barrier(VIWork *w, unsigned nblocks) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned *gen = &w->bar_gen;
        const unsigned g = *gen;
        __threadfence();
        if (atomicAdd(&w->bar_count, 1u) == nblocks - 1) {
            atomicExch(&w->bar_count, 0u);
            __threadfence();
            atomicAdd(&w->bar_gen, 1u);
        } else {
            unsigned i = 0;
            while (*gen == g) {
                if (++i > kSpinLimit || (*((volatile unsigned *)&w->status) & kErrTimeout)) {
                    atomicOr(&w->status, kErrTimeout);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok;
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
