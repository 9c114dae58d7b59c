// qv_pbvi.cu -- point-based value iteration, the lower bound of Sec. IV-B.
//
// Belief set expansion: every point b_j of the set yields tau(b_j, a, z)
// with a drawn uniformly and z ~ P(z | b_j, a) (one CTA per point).
//
// The Eq. 8 backup at a point b needs, for every action a, observation z and
// alpha-vector alpha_i of Gamma,
//   s(b, a, z, i) = sum_x sum_x' O(x', z) T(x, a, x') alpha_i(x') b(x)
//                 = sum_x' O(x', z) bbar_{b,a}(x') alpha_i(x'),
// with bbar_{b,a} = T_a^T b the predicted belief.  O(x', z) is eta plus
// (accuracy - eta) on the cells labelled z, so with
//   D_z(m, i) = sum over the cells x' labelled z of bbar_m(x') alpha_i(x'),   m = (b, a),
// s = eta sum_z' D_z'(m, i) + (accuracy - eta) D_z(m, i).  D is one dense
// contraction over the cells, split by label: the cells are ordered label by
// label (each label's run padded to a multiple of 32 with zeros, the goal and
// occupied cells left out because every alpha-vector is 0 there), so D_z is
// a matrix product over one contiguous range of that order.  Long ranges are
// cut into pieces so the grid fills the GPU; a piece's partial product is one
// slab, and the selection kernel adds the slabs of a label in piece order.
// The products run on the tcgen05 tensor cores as TF32 head x head + head x
// tail + tail x head; both operands are stored split, in the tile image the
// tensor core reads (see tiled_off).
//
// The selection kernel takes, per point, every (a, z) argmax over Gamma, the
// action a* maximising Q_b(a) = R(b, a) + gamma sum_z max_i s, and the set of
// distinct winning vectors with their multiplicities; the update kernel then
// forms alpha_b(x) = sum_{x'} T(x, a*, x') [r(x') + gamma c_b(x')] with
//   c_b(x') = eta sum_z alpha_{i*(z)}(x') + (accuracy - eta) alpha_{i*(label(x'))}(x'),
// band by band with c_b staged in shared memory.
#include <algorithm>
#include <cstring>
#include <vector>

#include "qv_common.cuh"
#include "qv_plan_types.cuh"  // kBoundaryEps, the window of a boundary draw

struct qv_pbvi;

namespace qv {
namespace {

constexpr int kPbThreads = 256;
constexpr int kSK = 16;          // K depth of one contraction stage (one 64-byte row of FP32)
constexpr int kKC = 32;          // K granularity of the label runs and pieces (two stages);
                                 // label runs are padded to it
constexpr int kTM = 128, kTN = 256;  // rows of A and of B (Gamma) per contraction CTA
constexpr int kRowTile = 128;        // rows of one 16 KB block of the tiled operand layout
constexpr int kPiecesExtra = 64; // pieces beyond one per label

struct PbModel {
    int H, W, P, N, B, nz, goal;
    float slip, acc, eta, gamma;
    const uint16_t *cell;
    const float *cost;
};

PbModel pb_model(const qv_model_t *m) {
    PbModel a;
    a.H = m->H;
    a.W = m->W;
    a.P = m->pitch;
    a.N = m->H * m->pitch;
    a.B = m->num_beacons;
    a.nz = m->num_beacons + 1;
    a.goal = m->goal;
    a.slip = m->slip;
    a.acc = m->accuracy;
    a.eta = (1.0f - m->accuracy) / static_cast<float>(m->num_beacons);
    a.gamma = m->discount;
    a.cell = m->d_cell;
    a.cost = m->d_cost;
    return a;
}

__device__ __forceinline__ float pb_reward(const PbModel &m, int y) {
    const unsigned cw = __ldg(m.cell + y);
    return stage_reward(QV_CELL_FREE(cw) != 0, y == m.goal, m.cost ? __ldg(m.cost + y) : 0.0f);
}

// The (at most three) cells a free, non-goal cell x reaches under action a,
// with their probabilities (Sec. II, Eq. 10: a blocked move stays on x).
__device__ __forceinline__ int pb_successors(const PbModel &m, int x, unsigned cw, int a, int y[3], float p[3]) {
    if (a == 4) {
        y[0] = x;
        p[0] = 1.0f;
        return 1;
    }
    const unsigned blk = QV_CELL_BLOCKED(cw);
    const int step[4] = {-m.P, 1, m.P, -1};
    const int d[3] = {a, (a + 1) & 3, (a + 3) & 3};
    const float w[3] = {1.0f - 2.0f * m.slip, m.slip, m.slip};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        y[i] = ((blk >> d[i]) & 1u) ? x : x + step[d[i]];
        p[i] = w[i];
    }
    return 3;
}

// x = hi + lo with hi = x rounded to TF32 (round to nearest, ties away) and
// lo the FP32 remainder rounded to TF32 in turn, so both halves are exact
// TF32 values and hi + lo is x to about 2^-22 relative.
__device__ __forceinline__ void tf32_split(float x, float &hi, float &lo) {
    uint32_t h, l;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
    hi = __uint_as_float(h);
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(x - hi));
    lo = __uint_as_float(l);
}

// Tiled operand layout of the contraction.  An operand of R rows (R padded
// to a multiple of 128, RT = R / 128 row tiles) over Kp positions (S = Kp / 16
// stages) is two planes, the TF32 heads and then the tails, each S x RT
// blocks of 128 rows x 16 positions (8 KB), stage-major so that the row tiles
// of one stage are adjacent.  Inside a block, row r holds its 16 values in
// four 16-byte chunks, chunk c stored at slot c ^ ((r >> 1) & 3): the
// K-major, 64-byte-swizzled image the tensor core reads (8-row groups of
// 512 bytes), so one bulk copy moves a block (or adjacent row tiles) from
// HBM into shared memory unchanged.
__device__ __forceinline__ int tiled_slot(int r, int kin) { return (((kin >> 2) ^ ((r >> 1) & 3)) << 2) | (kin & 3); }
__device__ __forceinline__ size_t tiled_off(int row, int k, int S, int RT) {
    const int rt = row >> 7, r = row & 127, s = k >> 4, kin = k & 15;
    return (static_cast<size_t>(s) * RT + rt) * (kRowTile * kSK) + r * kSK + tiled_slot(r, kin);
}
__host__ __device__ __forceinline__ size_t tiled_plane(int S, int RT) {
    return static_cast<size_t>(S) * RT * (kRowTile * kSK);
}
// Writes x split into the head and tail planes at tiled position (row, k).
__device__ __forceinline__ void tiled_store(float *T, int row, int k, int S, int RT, float x) {
    float hi, lo;
    tf32_split(x, hi, lo);
    const size_t o = tiled_off(row, k, S, RT);
    T[o] = hi;
    T[o + tiled_plane(S, RT)] = lo;
}

// ---------------------------------------------------------------- expansion
// One CTA per point j: pass 1 writes the predicted belief of the drawn action
// into out_j and sums its mass per label (one shared-memory column per
// thread, added in a fixed order, so the sums are reproducible); thread 0
// draws z from P(z) by the FP32 inverse CDF of the tree search; pass 2
// rescales out_j in place by O(., z) / P(z).
__global__ void __launch_bounds__(kPbThreads) k_pbvi_expand(PbModel m, const float *__restrict__ B, int round,
                                                            uint64_t seed, float *__restrict__ out,
                                                            int *__restrict__ action, int *__restrict__ obs,
                                                            int *__restrict__ boundary) {
    extern __shared__ float hist[];  // [nz][kPbThreads]
    __shared__ float lut[64];
    __shared__ float s_P[QV_MAX_BEACONS + 1], s_C[QV_MAX_BEACONS + 1];
    __shared__ int s_z;
    const int j = blockIdx.x, tid = threadIdx.x;
    const float *b = B + static_cast<size_t>(j) * m.N;
    float *o = out + static_cast<size_t>(j) * m.N;
    for (int i = tid; i < 64; i += blockDim.x) lut[i] = self_weight(i >> 4, i & 15, m.slip);
    for (int z = 0; z < m.nz; ++z) hist[z * kPbThreads + tid] = 0.0f;
    // the action: word 0 of the point's stream, a = floor(5 u) in exact arithmetic
    const float ua = sample_uniform(seed, static_cast<uint32_t>(round), 255, static_cast<uint64_t>(j), 0);
    const int a = min(4, static_cast<int>(floor(static_cast<double>(ua) * 5.0)));
    __syncthreads();
    for (int y = tid; y < m.N; y += blockDim.x) {
        const unsigned cw = __ldg(m.cell + y);
        const unsigned in = QV_CELL_INFLOW(cw);
        float nb[4];
        nb[kDirN] = (in & 1u) ? __ldg(b + y - m.P) : 0.0f;
        nb[kDirE] = (in & 2u) ? __ldg(b + y + 1) : 0.0f;
        nb[kDirS] = (in & 4u) ? __ldg(b + y + m.P) : 0.0f;
        nb[kDirW] = (in & 8u) ? __ldg(b + y - 1) : 0.0f;
        const float v = predict_one(nb, __ldg(b + y), cw, y == m.goal, m.slip, lut, a);
        o[y] = v;
        if (QV_CELL_FREE(cw)) hist[QV_CELL_LABEL(cw) * kPbThreads + tid] += v;
    }
    __syncthreads();
    for (int z = tid; z < m.nz; z += blockDim.x) {
        float s = 0.0f;
        for (int t = 0; t < kPbThreads; ++t) s += hist[z * kPbThreads + t];
        s_P[z] = s;  // mass on label z, turned into P(z) below
    }
    __syncthreads();
    if (tid == 0) {
        // P(z) = eta * total + (accuracy - eta) * mass(z), the total summed as
        // the tree search sums it (null label first, then z ascending)
        float tot = s_P[m.B];
        for (int z = 0; z < m.B; ++z) tot += s_P[z];
        float run = 0.0f;
        for (int z = 0; z < m.nz; ++z) {
            const float p = fmaf(m.acc - m.eta, s_P[z], m.eta * tot);
            s_P[z] = p;
            run = run + p;
            s_C[z] = run;
        }
        const float uz = sample_uniform(seed, static_cast<uint32_t>(round), 255, static_cast<uint64_t>(j), 1);
        const float t_u = uz * s_C[m.B];
        int lo = 0, hi = m.B;  // first z with t_u < C[z]
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (t_u < s_C[mid]) hi = mid;
            else lo = mid + 1;
        }
        const float inv = 1.0f / s_C[m.B];
        const bool near = (lo < m.B && fabsf(uz - s_C[lo] * inv) < kBoundaryEps) ||
                          (lo > 0 && fabsf(uz - s_C[lo - 1] * inv) < kBoundaryEps);
        s_z = lo;
        action[j] = a;
        obs[j] = lo;
        boundary[j] = near ? 1 : 0;
    }
    __syncthreads();
    const int z = s_z;
    const float inv = 1.0f / s_P[z];
    for (int y = tid; y < m.N; y += blockDim.x) {
        const unsigned cw = __ldg(m.cell + y);
        const float w = QV_CELL_FREE(cw) ? (static_cast<int>(QV_CELL_LABEL(cw)) == z ? m.acc : m.eta) : 0.0f;
        o[y] = o[y] * w * inv;
    }
}

// ---------------------------------------------------------------- the pessimistic start
__global__ void __launch_bounds__(kPbThreads) k_pbvi_init(PbModel m, float *__restrict__ alpha0) {
    __shared__ float s_min[kPbThreads / 32];
    __shared__ float s_v;
    float mn = INFINITY;
    for (int x = threadIdx.x; x < m.N; x += blockDim.x) {
        const unsigned cw = __ldg(m.cell + x);
        if (!QV_CELL_FREE(cw) || x == m.goal) continue;
        for (int a = 0; a < 5; ++a) {
            int y[3];
            float p[3];
            const int n = pb_successors(m, x, cw, a, y, p);
            float R = 0.0f;
            for (int i = 0; i < n; ++i) R = fmaf(p[i], pb_reward(m, y[i]), R);
            mn = fminf(mn, R);
        }
    }
    for (int o = 16; o > 0; o >>= 1) mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    if ((threadIdx.x & 31) == 0) s_min[threadIdx.x >> 5] = mn;
    __syncthreads();
    if (threadIdx.x == 0) {
        float v = s_min[0];
        for (int w = 1; w < kPbThreads / 32; ++w) v = fminf(v, s_min[w]);
        s_v = v / (1.0f - m.gamma);
    }
    __syncthreads();
    for (int x = threadIdx.x; x < m.N; x += blockDim.x) {
        const unsigned cw = __ldg(m.cell + x);
        alpha0[x] = (QV_CELL_FREE(cw) && x != m.goal) ? s_v : 0.0f;
    }
}

// ---------------------------------------------------------------- predicted beliefs of the set
// Grid (bands, points): every action's predicted belief of point b on the
// band's cells, scattered into the label order (row b * 5 + a of the tiled
// operand Bp, S stages, RT row tiles), and the band's share of
// sum_y bbar_a(y) r(y).
__global__ void __launch_bounds__(kPbThreads) k_pbvi_predict(PbModel m, const float *__restrict__ Bset,
                                                             const int *__restrict__ pos, int S, int RT,
                                                             int band_cells, float *__restrict__ Bp,
                                                             float *__restrict__ rpart) {
    __shared__ float lut[64];
    __shared__ float s_r[kPbThreads / 32][5];
    const int b = blockIdx.y, band = blockIdx.x;
    const float *bel = Bset + static_cast<size_t>(b) * m.N;
    for (int i = threadIdx.x; i < 64; i += blockDim.x) lut[i] = self_weight(i >> 4, i & 15, m.slip);
    __syncthreads();
    float rs[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    const int y0 = band * band_cells, y1 = min(m.N, y0 + band_cells);
    for (int y = y0 + threadIdx.x; y < y1; y += blockDim.x) {
        const unsigned cw = __ldg(m.cell + y);
        const unsigned in = QV_CELL_INFLOW(cw);
        float nb[4], o[5];
        nb[kDirN] = (in & 1u) ? __ldg(bel + y - m.P) : 0.0f;
        nb[kDirE] = (in & 2u) ? __ldg(bel + y + 1) : 0.0f;
        nb[kDirS] = (in & 4u) ? __ldg(bel + y + m.P) : 0.0f;
        nb[kDirW] = (in & 8u) ? __ldg(bel + y - 1) : 0.0f;
        predict_cell(nb, __ldg(bel + y), cw, y == m.goal, m.slip, lut, o);
        const int k = __ldg(pos + y);
        if (k >= 0) {
#pragma unroll
            for (int a = 0; a < 5; ++a) tiled_store(Bp, b * 5 + a, k, S, RT, o[a]);
        }
        if (QV_CELL_FREE(cw)) {
            const float r = stage_reward(true, y == m.goal, m.cost ? __ldg(m.cost + y) : 0.0f);
#pragma unroll
            for (int a = 0; a < 5; ++a) rs[a] = fmaf(o[a], r, rs[a]);
        }
    }
#pragma unroll
    for (int a = 0; a < 5; ++a) {
        float v = rs[a];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) s_r[threadIdx.x >> 5][a] = v;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        float v = 0.0f;
        for (int w = 0; w < kPbThreads / 32; ++w) v += s_r[w][threadIdx.x];
        rpart[(static_cast<size_t>(b) * gridDim.x + band) * 5 + threadIdx.x] = v;
    }
}

// R(b, a) = sum_y bbar_a(y) r(y) - 100 b(goal): the mass already on the goal
// stays there and earns nothing (R(goal, a) = 0).  Bands added in order.
__global__ void k_pbvi_reward(PbModel m, const float *__restrict__ Bset, int nB, int nbands,
                              const float *__restrict__ rpart, float *__restrict__ RB) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nB * 5) return;
    const int b = t / 5, a = t - b * 5;
    float v = 0.0f;
    for (int k = 0; k < nbands; ++k) v += rpart[(static_cast<size_t>(b) * nbands + k) * 5 + a];
    RB[t] = v - 100.0f * Bset[static_cast<size_t>(b) * m.N + m.goal];
}

// ---------------------------------------------------------------- Gamma in the label order
// Rows of grid-ordered vectors in the label order, tiled and split: row
// i < R of the operand is G_i at the live cells (0 at padding positions).
// Rows R .. of the last row tile are left as they are: an MMA row (or
// column) only feeds its own output row (or column), which the contraction
// does not store.  One thread per head element, a row's 16 values of a stage
// by 16 consecutive threads (one 64-byte segment per plane).
__device__ __forceinline__ void tiled_gather(const float *__restrict__ G, int N, const int *__restrict__ perm, int S,
                                             int RT, int R, float *__restrict__ Gp) {
    const size_t plane = tiled_plane(S, RT);
    const size_t per_stage = static_cast<size_t>(R) * kSK;
    const size_t total = static_cast<size_t>(S) * per_stage;
    for (size_t t = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
         t += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const int s = static_cast<int>(t / per_stage);
        const int rem = static_cast<int>(t - static_cast<size_t>(s) * per_stage);
        const int i = rem >> 4, slot = rem & 15;
        const int k = s * kSK + tiled_slot(i & 127, slot);  // the swizzle is its own inverse
        const size_t u = (static_cast<size_t>(s) * RT + (i >> 7)) * (kRowTile * kSK) + (i & 127) * kSK + slot;
        const int y = __ldg(perm + k);
        const float x = y >= 0 ? __ldg(G + static_cast<size_t>(i) * N + y) : 0.0f;
        float hi, lo;
        tf32_split(x, hi, lo);
        Gp[u] = hi;
        Gp[u + plane] = lo;
    }
}

// Gamma as the B operand of the contraction.
__global__ void __launch_bounds__(kPbThreads) k_pbvi_gather(const float *__restrict__ G, int nG, int N,
                                                            const int *__restrict__ perm, int S, int RT,
                                                            float *__restrict__ Gp) {
    tiled_gather(G, N, perm, S, RT, nG, Gp);
}

// ---------------------------------------------------------------- the contraction
// slab[p][m][n] = sum_{k in piece p} A[m][k] Bm[n][k] on the 5th-generation
// tensor cores, one 128 x 256 output tile (m tile, n tile, piece) at a time.
// TF32 keeps 10 mantissa bits, too few for the argmax decisions of Eq. 8, so
// both operands come split into TF32 heads and tails (x = hi + lo) and each
// product is formed as hi.hi + hi.lo + lo.hi, which restores FP32-level
// accuracy (the dropped lo.lo term is below 2^-21 of the product).  The
// operands sit in HBM in the tiled layout (tiled_off), so a stage of 16
// positions is four bulk copies (A heads and tails, 8 KB each; B heads and
// tails, 16 KB each) into one of four 48 KB shared-memory buffers.
//
// The kernel is persistent: one CTA per SM walks the tiles t = blockIdx.x,
// blockIdx.x + gridDim.x, ... with three roles.  Warp 0 issues the copies,
// running up to four stages ahead across tile boundaries; warp 1 issues the
// six MMAs of each stage (K = 8 each) into one of two TMEM accumulators of
// 256 columns and commits them to the buffer's "empty" barrier, and each
// finished tile to its accumulator's "full" barrier; warps 2-5 read a
// finished accumulator back (warp w owns TMEM lanes 32 (w % 4) ..) and store
// it, while the MMAs of the next tile run in the other accumulator.  Every
// wait is bounded and also ends when another role has given up; a CTA that
// gave up sets *status, lets its copies and MMAs in flight land and still
// frees the tensor memory.
constexpr int kTcThreads = 192;
constexpr int kTcStages = 4;
constexpr int kTcAFloats = kTM * kSK, kTcBFloats = kTN * kSK;  // one plane of one stage
constexpr int kTcStageFloats = 2 * kTcAFloats + 2 * kTcBFloats;  // A hi, A lo, B hi, B lo: 48 KB
constexpr unsigned kTcStageBytes = kTcStageFloats * sizeof(float);
constexpr size_t kTcSmem = kTcStages * static_cast<size_t>(kTcStageBytes) + 1024;
constexpr int kTcAccCols = kTN;                // FP32 accumulator: one column per B row
constexpr int kTcTmemCols = 2 * kTcAccCols;    // two accumulators
constexpr int kTcSpin = 1 << 24;               // polls of one wait before it gives up

__device__ __forceinline__ uint32_t tc_smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory descriptor of a K-major tile with the 64-byte swizzle:
// start address, stride of 512 bytes between groups of 8 rows, descriptor
// version 1, layout code 4 (64-byte swizzle).
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
    return static_cast<uint64_t>((saddr >> 4) & 0x3FFF) | (static_cast<uint64_t>(512 >> 4) << 32) |
           (static_cast<uint64_t>(1) << 46) | (static_cast<uint64_t>(4) << 61);
}

__device__ __forceinline__ bool tc_try(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(tc_smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Bounded wait for phase `parity` of `bar`, polled by the whole warp (the
// answer is made warp-uniform, so the warp stays converged); gives up (and
// raises *fail) after kTcSpin polls, or as soon as *fail is raised.
__device__ __forceinline__ bool tc_wait(uint64_t *bar, uint32_t parity, volatile int *fail) {
    for (int it = 0; it < kTcSpin; ++it) {
        if (__any_sync(0xffffffffu, tc_try(bar, parity))) return true;
        if ((it & 63) == 63 && __shfl_sync(0xffffffffu, *fail, 0)) return false;
    }
    *fail = 1;
    return false;
}

// Bounded wait that ignores *fail: the clean-up after a role gave up.
__device__ __forceinline__ void tc_drain(uint64_t *bar, uint32_t parity) {
    for (int it = 0; it < (1 << 20); ++it)
        if (__any_sync(0xffffffffu, tc_try(bar, parity))) return;
}

struct TcTile {
    int m0, n0, p, s0, nst;
};
__device__ __forceinline__ TcTile tc_tile(int t, int Mt, int Nt, const int *piece) {
    TcTile r;
    const int mt = t % Mt, rest = t / Mt;
    r.n0 = (rest % Nt) * kTN;
    r.p = rest / Nt;
    r.m0 = mt * kTM;
    const int k0 = __ldg(piece + 3 * r.p), k1 = __ldg(piece + 3 * r.p + 1);
    r.s0 = k0 / kSK;
    r.nst = (k1 - k0) / kSK;
    return r;
}

__global__ void __launch_bounds__(kTcThreads, 1) k_pbvi_scores(const float *__restrict__ A, int RTa,
                                                               const float *__restrict__ Bm, int RTb, int M, int N,
                                                               int S, int Mt, int Nt, int ntiles,
                                                               const int *__restrict__ piece,
                                                               float *__restrict__ slab, int *__restrict__ status) {
    extern __shared__ unsigned char tc_raw[];
    __shared__ __align__(8) uint64_t full[kTcStages], empty[kTcStages], acc_full[2], acc_empty[2];
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    __shared__ int s_loaded, s_consumed;  // stages whose copies / MMAs were issued
    float *st = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(tc_raw) + 1023) & ~uintptr_t(1023));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    volatile int *fail = &s_fail;
    if (tid == 0) {
        for (int i = 0; i < kTcStages; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem_u32(&full[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem_u32(&empty[i])));
        }
        for (int i = 0; i < 2; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem_u32(&acc_full[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(tc_smem_u32(&acc_empty[i])));
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
        s_fail = 0;
        s_loaded = 0;
        s_consumed = 0;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         tc_smem_u32(&s_tmem)),
                     "n"(kTcTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = s_tmem;
    const size_t planeA = tiled_plane(S, RTa), planeB = tiled_plane(S, RTb);
    if (warp == 0) {
        // ---- copies
        int g = 0;
        for (int t = blockIdx.x; t < ntiles && !*fail; t += gridDim.x) {
            const TcTile tl = tc_tile(t, Mt, Nt, piece);
            const int rta = tl.m0 / kRowTile, rtb = tl.n0 / kRowTile;
            for (int s = 0; s < tl.nst; ++s, ++g) {
                const int buf = g % kTcStages;
                if (g >= kTcStages && !tc_wait(&empty[buf], ((g / kTcStages) - 1) & 1, fail)) break;
                if (lane == 0) {
                    float *b = st + buf * kTcStageFloats;
                    uint64_t *bar = &full[buf];
                    const size_t oa = (static_cast<size_t>(tl.s0 + s) * RTa + rta) * (kRowTile * kSK);
                    const size_t ob = (static_cast<size_t>(tl.s0 + s) * RTb + rtb) * (kRowTile * kSK);
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc_smem_u32(bar)),
                                 "r"(kTcStageBytes)
                                 : "memory");
                    const void *src[4] = {A + oa, A + oa + planeA, Bm + ob, Bm + ob + planeB};
                    float *dst[4] = {b, b + kTcAFloats, b + 2 * kTcAFloats, b + 2 * kTcAFloats + kTcBFloats};
                    const unsigned bytes[4] = {kTcAFloats * 4u, kTcAFloats * 4u, kTcBFloats * 4u, kTcBFloats * 4u};
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        asm volatile(
                            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
                            "[%3];" ::"r"(tc_smem_u32(dst[i])),
                            "l"(src[i]), "r"(bytes[i]), "r"(tc_smem_u32(bar))
                            : "memory");
                    s_loaded = g + 1;
                }
                __syncwarp();
            }
        }
    } else if (warp == 1) {
        // ---- MMAs: FP32 accumulator, TF32 A and B, both K-major, N = 256, M = 128
        const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((kTN >> 3) << 17) | ((kTM >> 4) << 24);
        int g = 0, j = 0;
        for (int t = blockIdx.x; t < ntiles && !*fail; t += gridDim.x, ++j) {
            const TcTile tl = tc_tile(t, Mt, Nt, piece);
            const int acc = j & 1;
            // the epilogue of tile j - 2 has drained this accumulator
            if (j >= 2 && !tc_wait(&acc_empty[acc], ((j >> 1) - 1) & 1, fail)) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t d = tmem + static_cast<uint32_t>(acc * kTcAccCols);
            bool ok = true;
            for (int s = 0; s < tl.nst; ++s, ++g) {
                const int buf = g % kTcStages;
                if (!tc_wait(&full[buf], (g / kTcStages) & 1, fail)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                if (lane == 0) {
                    const float *b = st + buf * kTcStageFloats;
                    const uint64_t ah = tc_desc(tc_smem_u32(b)), al = tc_desc(tc_smem_u32(b + kTcAFloats));
                    const uint64_t bh = tc_desc(tc_smem_u32(b + 2 * kTcAFloats));
                    const uint64_t bl = tc_desc(tc_smem_u32(b + 2 * kTcAFloats + kTcBFloats));
#pragma unroll
                    for (int kk = 0; kk < kSK / 8; ++kk) {  // K = 8 per MMA: 32 bytes further along the rows
                        const uint64_t o = 2ull * kk;
                        const uint32_t accum = (s == 0 && kk == 0) ? 0u : 1u;
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                            "l"(ah + o), "l"(bh + o), "r"(idesc), "r"(accum));
                        asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;" ::"r"(d),
                                     "l"(ah + o), "l"(bl + o), "r"(idesc));
                        asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;" ::"r"(d),
                                     "l"(al + o), "l"(bh + o), "r"(idesc));
                    }
                    asm volatile(
                        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                            tc_smem_u32(&empty[buf])));
                    s_consumed = g + 1;
                }
                __syncwarp();
            }
            if (!ok) break;
            // every MMA of the tile done: the accumulator is ready
            if (lane == 0)
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    tc_smem_u32(&acc_full[acc])));
            __syncwarp();
        }
    } else {
        // ---- epilogue: warps 2..5, TMEM lanes 32 (warp % 4) ..
        const int q = warp & 3;
        int j = 0;
        for (int t = blockIdx.x; t < ntiles && !*fail; t += gridDim.x, ++j) {
            const TcTile tl = tc_tile(t, Mt, Nt, piece);
            const int acc = j & 1;
            if (!tc_wait(&acc_full[acc], (j >> 1) & 1, fail)) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            float *out = slab + static_cast<size_t>(tl.p) * M * N;
            const int row = tl.m0 + q * 32 + lane;
            for (int c0 = 0; c0 < kTN && tl.n0 + c0 < N; c0 += 16) {
                uint32_t r[16];
                if (tl.nst > 0) {
                    const uint32_t taddr = tmem + (static_cast<uint32_t>(q * 32) << 16) +
                                           static_cast<uint32_t>(acc * kTcAccCols + c0);
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
                        "%15}, [%16];"
                        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                          "=r"(r[14]), "=r"(r[15])
                        : "r"(taddr));
                    asm volatile("tcgen05.wait::ld.sync.aligned;");
                } else {
#pragma unroll
                    for (int i = 0; i < 16; ++i) r[i] = 0u;
                }
                if (row < M) {
                    float *dst = out + static_cast<size_t>(row) * N + tl.n0 + c0;
                    if (tl.n0 + c0 + 16 <= N && (N & 3) == 0) {
#pragma unroll
                        for (int i = 0; i < 16; i += 4)
                            *reinterpret_cast<float4 *>(dst + i) =
                                make_float4(__uint_as_float(r[i]), __uint_as_float(r[i + 1]),
                                            __uint_as_float(r[i + 2]), __uint_as_float(r[i + 3]));
                    } else {
#pragma unroll
                        for (int i = 0; i < 16; ++i)
                            if (tl.n0 + c0 + i < N) dst[i] = __uint_as_float(r[i]);
                    }
                }
            }
            // the accumulator may be overwritten once every epilogue warp has read it
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0)
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc_smem_u32(&acc_empty[acc]))
                             : "memory");
        }
    }
    __syncthreads();
    if (s_fail) {
        // let the copies and MMAs in flight land before the memory is freed
        if (warp == 0) {
            const int ld = s_loaded, cs = s_consumed;
            for (int g = cs; g < ld; ++g) tc_drain(&full[g % kTcStages], (g / kTcStages) & 1);
            if (cs > 0) tc_drain(&empty[(cs - 1) % kTcStages], ((cs - 1) / kTcStages) & 1);
            if (lane == 0) atomicOr(status, 1);
        }
        __syncthreads();
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(kTcTmemCols));
}

// ---------------------------------------------------------------- selection
// One CTA per point b.  For each action a the slab rows of (b, a) are read
// once, a chunk of vectors at a time: D_z(i) (the label's pieces in order)
// and D(i) (every piece in order) go to shared memory.  One warp per
// observation z then takes Eq. 8's argmax_i eta D(i) + (accuracy - eta)
// D_z(i): the best score over every chunk first, then the lowest index that
// attains it (a second read of the slabs only when nG spans more than one
// chunk).  Then a* = argmax_a Q_b(a) (ties to the lowest action) and the
// distinct winners of a* with their multiplicities.
// fix_astar / fix_best (nullable): decisions fixed by the caller, a* of
// point b when fix_astar[b] >= 0 and the winner of observation z for that
// a* when fix_best[b * nz + z] >= 0 (its own score then enters Q_b(a*)), so
// that another implementation's choices at near-ties can be replayed.
constexpr int kSelThreads = 512;
constexpr size_t kSelSmemBudget = 96 * 1024;  // D_z and D of one chunk, and the piece labels

int select_chunk(int nz, int nG, int npieces) {
    const size_t room = (kSelSmemBudget - (npieces + 1) * sizeof(int)) / sizeof(float) / (nz + 1);
    int c = static_cast<int>(std::min<size_t>(room, static_cast<size_t>(nG)));
    if (c < nG) c = std::max(32, c & ~31);
    return c;
}
// Piece groups of the selection: when a chunk has fewer vectors than the
// CTA has threads, groups of threads share the pieces (at most four, and as
// many as the shared-memory budget holds: each group keeps its own D_z and
// D).
__host__ __device__ inline int select_groups(int nz, int chunk) {
    const int cols = (chunk + 31) & ~31;
    int g = kSelThreads / cols;
    const int fit = static_cast<int>(kSelSmemBudget / (static_cast<size_t>(nz + 1) * chunk * sizeof(float)));
    g = g < fit ? g : fit;
    return cols >= kSelThreads ? 1 : (g < 1 ? 1 : (g > 4 ? 4 : g));
}
size_t select_smem(int nz, int chunk, int npieces) {
    return static_cast<size_t>(select_groups(nz, chunk)) * (nz + 1) * chunk * sizeof(float) +
           (npieces + 1) * sizeof(int);
}

__global__ void __launch_bounds__(kSelThreads, 2) k_pbvi_select(PbModel m, int nB, int nG, int chunk, int npieces,
                                                                const int *__restrict__ piece,
                                                                const float *__restrict__ slab,
                                                                const float *__restrict__ RB, float *__restrict__ value,
                                                                int *__restrict__ astar, int *__restrict__ best,
                                                                float *__restrict__ q, int *__restrict__ uniq,
                                                                int *__restrict__ mult, int *__restrict__ nuniq,
                                                                const int *__restrict__ fix_astar,
                                                                const int *__restrict__ fix_best) {
    extern __shared__ float sel_sm[];
    const int groups = select_groups(m.nz, chunk);
    float *Dz = sel_sm;                       // [nz][chunk] (group 0's, and the sums over the groups)
    float *D = sel_sm + m.nz * chunk;         // [chunk]
    int *plabel = reinterpret_cast<int *>(sel_sm + static_cast<size_t>(groups) * (m.nz + 1) * chunk);
                                              // [npieces + 1], -1 after the last
    __shared__ float s_bv[QV_MAX_BEACONS + 1], s_bs[QV_MAX_BEACONS + 1];
    __shared__ int s_bi[QV_MAX_BEACONS + 1];
    __shared__ int s_arg[5][QV_MAX_BEACONS + 1];
    __shared__ float s_val[QV_MAX_BEACONS + 1];
    __shared__ float s_q[5];
    __shared__ int s_empty[QV_MAX_BEACONS + 1];  // labels with no piece (D_z = 0)
    const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    constexpr int kWarps = kSelThreads / 32;
    const size_t slab_elems = static_cast<size_t>(nB) * 5 * nG;
    for (int p = tid; p <= npieces; p += kSelThreads) plabel[p] = p < npieces ? __ldg(piece + 3 * p + 2) : -1;
    for (int z = tid; z < m.nz; z += kSelThreads) s_empty[z] = 1;
    __syncthreads();
    for (int p = tid; p < npieces; p += kSelThreads) s_empty[plabel[p]] = 0;
    const int nchunks = (nG + chunk - 1) / chunk;
    // D_z and D of vectors i0 .. i0 + n - 1 of row (b, a).  One group: each
    // thread takes two vectors at a time, pieces in batches of eight, sixteen
    // loads in flight.  Several groups: group g adds its share of the pieces
    // (in order) for one vector a thread, and the group sums are then added
    // in group order.
    auto fill_groups = [&](size_t row, int i0, int n) {
        const int cols = (chunk + 31) & ~31, g = tid / cols, c = tid - g * cols;
        const int per = (npieces + groups - 1) / groups;
        const int p_lo = min(npieces, g * per), p_hi = min(npieces, p_lo + per);
        if (g < groups && c < n) {
            float *dzg = sel_sm + static_cast<size_t>(g) * (m.nz + 1) * chunk, *dg = dzg + m.nz * chunk;
            for (int z = 0; z < m.nz; ++z) dzg[z * chunk + c] = 0.0f;
            const float *col = slab + row + i0 + c;
            float d = 0.0f, dz = 0.0f;
            for (int p0 = p_lo; p0 < p_hi; p0 += 16) {
                float v[16];
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    v[j] = p0 + j < p_hi ? __ldg(col + static_cast<size_t>(p0 + j) * slab_elems) : 0.0f;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int p = p0 + j;
                    if (p < p_hi) {
                        d += v[j];
                        dz += v[j];
                        if (p + 1 == p_hi || plabel[p + 1] != plabel[p]) {
                            dzg[plabel[p] * chunk + c] = dz;
                            dz = 0.0f;
                        }
                    }
                }
            }
            dg[c] = d;
        }
        __syncthreads();
        for (int t = tid; t < (m.nz + 1) * n; t += kSelThreads) {
            const int z = t / n, i = t - z * n;
            float v = sel_sm[static_cast<size_t>(z) * chunk + i];
            for (int h = 1; h < groups; ++h) v += sel_sm[(static_cast<size_t>(h) * (m.nz + 1) + z) * chunk + i];
            sel_sm[static_cast<size_t>(z) * chunk + i] = v;
        }
    };
    auto fill = [&](size_t row, int i0, int n) {
        if (groups > 1) {
            fill_groups(row, i0, n);
            return;
        }
        for (int ia = tid; ia < n; ia += 2 * kSelThreads) {
            const int ib = ia + kSelThreads;
            const bool two = ib < n;
            const float *ca = slab + row + i0 + ia, *cb = slab + row + i0 + (two ? ib : ia);
            float d[2] = {0.0f, 0.0f}, dz[2] = {0.0f, 0.0f};
            for (int p0 = 0; p0 < npieces; p0 += 8) {
                float v[2][8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const bool in = p0 + j < npieces;
                    const size_t o = static_cast<size_t>(p0 + j) * slab_elems;
                    v[0][j] = in ? __ldg(ca + o) : 0.0f;
                    v[1][j] = in && two ? __ldg(cb + o) : 0.0f;
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int p = p0 + j;
                    if (p < npieces) {
                        d[0] += v[0][j];
                        d[1] += v[1][j];
                        dz[0] += v[0][j];
                        dz[1] += v[1][j];
                        if (plabel[p + 1] != plabel[p]) {
                            Dz[plabel[p] * chunk + ia] = dz[0];
                            if (two) Dz[plabel[p] * chunk + ib] = dz[1];
                            dz[0] = dz[1] = 0.0f;
                        }
                    }
                }
            }
            D[ia] = d[0];
            if (two) D[ib] = d[1];
            for (int z = 0; z < m.nz; ++z)
                if (s_empty[z]) {
                    Dz[z * chunk + ia] = 0.0f;
                    if (two) Dz[z * chunk + ib] = 0.0f;
                }
        }
    };
    const int fa = fix_astar ? __ldg(fix_astar + b) : -1;
    for (int a = 0; a < 5; ++a) {
        const size_t row = static_cast<size_t>(b * 5 + a) * nG;
        // pass 1: the best score of every z
        for (int c = 0; c < nchunks; ++c) {
            const int i0 = c * chunk, n = min(chunk, nG - i0);
            __syncthreads();
            fill(row, i0, n);
            __syncthreads();
            for (int z = wid; z < m.nz; z += kWarps) {
                const float *dz = Dz + z * chunk;
                float bv = -INFINITY;
                for (int i = lane; i < n; i += 32) bv = fmaxf(bv, fmaf(m.acc - m.eta, dz[i], m.eta * D[i]));
                for (int o = 16; o > 0; o >>= 1) bv = fmaxf(bv, __shfl_xor_sync(0xffffffffu, bv, o));
                if (lane == 0) {
                    s_bv[z] = c == 0 ? bv : fmaxf(s_bv[z], bv);
                    if (c == 0) s_bi[z] = 0x7fffffff;
                }
            }
        }
        // pass 2: the lowest index that attains the best (or the caller's
        // fixed winner, with its own score)
        for (int c = 0; c < nchunks; ++c) {
            const int i0 = c * chunk, n = min(chunk, nG - i0);
            __syncthreads();
            if (nchunks > 1) {
                fill(row, i0, n);
                __syncthreads();
            }
            for (int z = wid; z < m.nz; z += kWarps) {
                const int fz = (a == fa && fix_best) ? __ldg(fix_best + b * m.nz + z) : -1;
                if (fz >= 0) {  // warp-uniform
                    if (lane == 0 && fz >= i0 && fz < i0 + n) {
                        s_bi[z] = fz;
                        s_bs[z] = fmaf(m.acc - m.eta, Dz[z * chunk + (fz - i0)], m.eta * D[fz - i0]);
                    }
                    continue;
                }
                if (s_bi[z] != 0x7fffffff) continue;  // found in an earlier chunk (warp-uniform)
                const float *dz = Dz + z * chunk;
                const float floor_v = s_bv[z];
                int bi = 0x7fffffff;
                float bs = 0.0f;
                for (int i = lane; i < n; i += 32) {
                    const float sv = fmaf(m.acc - m.eta, dz[i], m.eta * D[i]);
                    if (sv >= floor_v) {
                        bi = i;
                        bs = sv;
                        break;
                    }
                }
                for (int o = 16; o > 0; o >>= 1) {
                    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                    const float os = __shfl_xor_sync(0xffffffffu, bs, o);
                    if (oi < bi) {
                        bi = oi;
                        bs = os;
                    }
                }
                if (lane == 0 && bi != 0x7fffffff) {
                    s_bi[z] = i0 + bi;
                    s_bs[z] = bs;
                }
            }
        }
        __syncthreads();
        if (tid == 0) {
            float sum = 0.0f;
            for (int z = 0; z < m.nz; ++z) {
                const bool found = s_bi[z] != 0x7fffffff;  // (none when every score is NaN)
                s_val[z] = found ? s_bs[z] : s_bv[z];
                s_arg[a][z] = found ? s_bi[z] : 0;
                sum += s_val[z];
            }
            s_q[a] = fmaf(m.gamma, sum, __ldg(RB + b * 5 + a));
        }
    }
    __syncthreads();
    if (tid == 0) {
        float qmax = s_q[0];
        for (int a = 1; a < 5; ++a) qmax = fmaxf(qmax, s_q[a]);
        int as = 0;
        while (as < 4 && !(s_q[as] >= qmax)) ++as;
        if (fa >= 0 && fa < 5) as = fa;
        astar[b] = as;
        value[b] = s_q[as];
        if (q)
            for (int a = 0; a < 5; ++a) q[b * 5 + a] = s_q[a];
        int n = 0;
        for (int z = 0; z < m.nz; ++z) {
            const int i = s_arg[as][z];
            best[b * m.nz + z] = i;
            int t = 0;
            while (t < n && uniq[b * m.nz + t] != i) ++t;
            if (t == n) {
                uniq[b * m.nz + n] = i;
                mult[b * m.nz + n] = 0;
                ++n;
            }
            ++mult[b * m.nz + t];
        }
        nuniq[b] = n;
    }
}

// ---------------------------------------------------------------- the new alpha-vectors
// Grid (bands of rows, points).  c_b on the band's rows and one halo row on
// each side goes to shared memory, then alpha_b(x) = sum over x's successors
// under a* of T [r(x') + gamma c_b(x')] on free, non-goal cells, 0 elsewhere.
__global__ void __launch_bounds__(kPbThreads) k_pbvi_alpha(PbModel m, int band_rows, const float *__restrict__ G,
                                                           const int *__restrict__ astar, const int *__restrict__ best,
                                                           const int *__restrict__ uniq, const int *__restrict__ mult,
                                                           const int *__restrict__ nuniq, float *__restrict__ Gout) {
    extern __shared__ float cs[];  // (band_rows + 2) rows of P
    const int b = blockIdx.y;
    const int r0 = blockIdx.x * band_rows, r1 = min(m.H, r0 + band_rows);
    const int lo = max(0, r0 - 1), hi = min(m.H, r1 + 1);
    const int nu = nuniq[b];
    const int *ub = uniq + b * m.nz;
    const int *mb = mult + b * m.nz;
    const int *bb = best + b * m.nz;
    const float dl = m.acc - m.eta;
    for (int t = threadIdx.x; t < (hi - lo) * m.P; t += blockDim.x) {
        const int y = lo * m.P + t;
        const unsigned cw = __ldg(m.cell + y);
        float c = 0.0f;
        if (QV_CELL_FREE(cw) && y != m.goal) {
            float s = 0.0f;
            for (int u = 0; u < nu; ++u) s = fmaf(static_cast<float>(__ldg(mb + u)), __ldg(G + static_cast<size_t>(__ldg(ub + u)) * m.N + y), s);
            const int own = __ldg(bb + QV_CELL_LABEL(cw));
            c = fmaf(dl, __ldg(G + static_cast<size_t>(own) * m.N + y), m.eta * s);
        }
        cs[(lo - (r0 - 1)) * m.P + t] = c;
    }
    __syncthreads();
    const int as = astar[b];
    float *out = Gout + static_cast<size_t>(b) * m.N;
    for (int t = threadIdx.x; t < (r1 - r0) * m.P; t += blockDim.x) {
        const int x = r0 * m.P + t;
        const unsigned cw = __ldg(m.cell + x);
        float v = 0.0f;
        if (QV_CELL_FREE(cw) && x != m.goal) {
            int y[3];
            float p[3];
            const int n = pb_successors(m, x, cw, as, y, p);
            for (int i = 0; i < n; ++i) {
                const float cy = cs[y[i] - (r0 - 1) * m.P];
                v = fmaf(p[i], fmaf(m.gamma, cy, pb_reward(m, y[i])), v);
            }
        }
        out[x] = v;
    }
}

// ---------------------------------------------------------------- V_PBVI(b) = max_i alpha_i . b
__global__ void __launch_bounds__(kPbThreads) k_pbvi_scatter_points(const float *__restrict__ Bset, int nb, int N,
                                                                    const int *__restrict__ perm, int S, int RT,
                                                                    float *__restrict__ Ap) {
    tiled_gather(Bset, N, perm, S, RT, nb, Ap);
}

// One CTA per belief j.  The threads form `groups` groups of cols =
// blockDim / groups columns; group g adds a contiguous run of the pieces
// (in order) for its columns, then the group sums are added in group order
// and the CTA takes the best column (ties to the lowest index).
constexpr int kRmThreads = 1024;
// Piece groups and threads of one CTA: several groups when the beliefs are
// too few to fill the GPU with one CTA each, one otherwise.
void rowmax_shape(int nb, int nG, int &groups, int &threads) {
    const int cols = std::max(32, (nG + 31) & ~31);
    groups = nb >= qv_num_sms() ? 1 : std::max(1, std::min(8, kRmThreads / cols));
    threads = std::min(kRmThreads, groups * cols);
}

__global__ void __launch_bounds__(kRmThreads) k_pbvi_rowmax(int nb, int nG, int npieces, int groups,
                                                            const float *__restrict__ slab, float *__restrict__ value,
                                                            int *__restrict__ arg) {
    __shared__ float part[kRmThreads];
    __shared__ float s_v[kRmThreads / 32];
    __shared__ int s_i[kRmThreads / 32];
    const int j = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int cols = blockDim.x / groups, g = tid / cols, c = tid - g * cols;
    const int per = (npieces + groups - 1) / groups;
    const int p_lo = min(npieces, g * per), p_hi = min(npieces, p_lo + per);
    const size_t slab_elems = static_cast<size_t>(nb) * nG;
    float bv = -INFINITY;
    int bi = 0x7fffffff;
    for (int i0 = 0; i0 < nG; i0 += cols) {
        const int i = i0 + c;
        float s = 0.0f;
        if (i < nG && g < groups) {
            // this group's pieces in order, sixteen loads in flight
            const float *col = slab + static_cast<size_t>(j) * nG + i;
            for (int p0 = p_lo; p0 < p_hi; p0 += 16) {
                float v[16];
#pragma unroll
                for (int t = 0; t < 16; ++t) v[t] = p0 + t < p_hi ? __ldg(col + (p0 + t) * slab_elems) : 0.0f;
#pragma unroll
                for (int t = 0; t < 16; ++t)
                    if (p0 + t < p_hi) s += v[t];
            }
        }
        __syncthreads();
        if (g < groups) part[tid] = s;
        __syncthreads();
        if (g == 0 && i < nG) {
            float t = part[c];
            for (int h = 1; h < groups; ++h) t += part[h * cols + c];
            if (t > bv) {
                bv = t;
                bi = i;
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) {
            bv = ov;
            bi = oi;
        }
    }
    if (lane == 0) {
        s_v[wid] = bv;
        s_i[wid] = bi;
    }
    __syncthreads();
    if (tid == 0) {
        float v = s_v[0];
        int ii = s_i[0];
        for (int w = 1; w < static_cast<int>(blockDim.x / 32); ++w)
            if (s_v[w] > v || (s_v[w] == v && s_i[w] < ii)) {
                v = s_v[w];
                ii = s_i[w];
            }
        value[j] = v;
        if (arg) arg[j] = ii < nG ? ii : 0;
    }
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// The contraction kernel's shared memory exceeds the 48 KB default.
qv_status tc_prepare() {
    return qv_check_cuda(cudaFuncSetAttribute(k_pbvi_scores, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              static_cast<int>(kTcSmem)),
                         "smem attr");
}

}  // namespace
}  // namespace qv

// ------------------------------------------------------------------ host side
struct qv_pbvi {
    qv_model_t model;
    int max_points, max_vectors;
    int Kp, nz, max_pieces;      // the slab region holds max_pieces x 5 max_points x max(vectors, points)
    int piece_table;             // entries of the piece table (at least max_pieces)
    std::vector<int> perm;       // Kp: grid index of each position, -1 for padding
    std::vector<int> pos;        // H * pitch: position of each cell, -1 off the live cells
    std::vector<int> seg;        // nz + 1: label z occupies [seg[z], seg[z + 1])
    std::vector<int> pieces;     // last uploaded piece table (k0, k1, label) triples
    size_t off_pos, off_perm, off_piece, off_Bp, off_RB, off_rpart, off_Gp, off_Ap, off_slab;
    size_t off_best, off_uniq, off_mult, off_nuniq, off_astar, off_val, off_status;
    size_t ws_bytes;
    void *ws;                    // workspace the tables live in (set by qv_pbvi_set_points)
    int nB;                      // points of the current set
    int gp_value_nG;             // vectors in Gp gathered by the last qv_pbvi_value call, 0 when a
                                 // backup has overwritten Gp since
    int nbands;                  // bands of k_pbvi_predict
    int band_cells;
    int S;                       // contraction stages, Kp / 16
    int RTa, RTb, RTp;           // row tiles of the tiled operands Bp (5 x max_points rows),
                                 // Gp (max_vectors rows, an even count) and Ap (max_points rows)
};

namespace {

using qv::align256;

// Pieces of the label runs: each run [seg[z], seg[z+1]) is cut into pieces of
// at most L positions (a multiple of kKC), L chosen so that tiles x pieces
// fills the GPU (a few times over for the backup's many tiles, about once
// for the few tiles of V_PBVI, with at least three stages a piece) and there
// are at most `cap` pieces.
void make_pieces(const qv_pbvi &h, int tiles, int total_len, bool by_label, int cap, std::vector<int> &out) {
    out.clear();
    const int target = (by_label ? 4 : 1) * qv_num_sms();
    const int want_pieces = std::max(1, (target + tiles - 1) / tiles);
    const int min_len = by_label ? qv::kKC : 3 * qv::kKC;
    int L = std::max(min_len, ((total_len / want_pieces + qv::kKC - 1) / qv::kKC) * qv::kKC);
    for (;;) {
        out.clear();
        if (by_label) {
            for (int z = 0; z < h.nz; ++z)
                for (int k = h.seg[z]; k < h.seg[z + 1]; k += L) out.insert(out.end(), {k, std::min(h.seg[z + 1], k + L), z});
        } else {
            for (int k = 0; k < total_len; k += L) out.insert(out.end(), {k, std::min(total_len, k + L), 0});
        }
        if (static_cast<int>(out.size() / 3) <= cap) break;
        L += qv::kKC * std::max(1, L / (8 * qv::kKC));  // about 12 % longer
    }
}

// Pieces the slab region and the piece table allow for an M x N product.
int piece_cap(const qv_pbvi &h, size_t M, size_t N) {
    const size_t slab = static_cast<size_t>(h.max_pieces) * 5 * h.max_points * std::max(h.max_vectors, h.max_points);
    return static_cast<int>(std::min<size_t>(h.piece_table, slab / std::max<size_t>(1, M * N)));
}

qv_status upload_pieces(qv_pbvi *h, const std::vector<int> &pc, cudaStream_t st) {
    if (pc == h->pieces) return QV_OK;
    h->pieces = pc;
    return qv_check_cuda(cudaMemcpyAsync(static_cast<char *>(h->ws) + h->off_piece, h->pieces.data(),
                                         h->pieces.size() * sizeof(int), cudaMemcpyHostToDevice, st),
                         "piece table");
}

}  // namespace

extern "C" qv_status qv_pbvi_create(const qv_model_t *m, int32_t max_points, qv_pbvi **out) {
    if (!m || !m->d_cell || !out) return qv_set_error(QV_ERR_INVALID, "qv_pbvi_create: null pointer");
    *out = nullptr;
    if (m->H < 1 || m->W < 1 || m->pitch != QV_PITCH(m->W) || m->W > QV_MAX_WIDTH || m->num_beacons < 1 ||
        m->num_beacons > QV_MAX_BEACONS || m->goal < 0 || m->goal >= m->H * m->pitch)
        return qv_set_error(QV_ERR_INVALID, "qv_pbvi_create: bad model");
    if (max_points < 1 || max_points > (1 << 16))
        return qv_set_error(QV_ERR_INVALID, "qv_pbvi_create: max_points %d outside 1..65536", max_points);
    const int N = m->H * m->pitch, nz = m->num_beacons + 1;
    std::vector<uint16_t> cell(N);
    if (qv_check_cuda(cudaMemcpy(cell.data(), m->d_cell, N * sizeof(uint16_t), cudaMemcpyDeviceToHost),
                      "cell words") != QV_OK)
        return QV_ERR_CUDA;
    qv_pbvi *h = new qv_pbvi();
    h->model = *m;
    h->max_points = max_points;
    h->max_vectors = max_points;
    h->nz = nz;
    // live cells (free, not the goal) in label order, grid order within a label
    std::vector<int> count(nz, 0);
    for (int y = 0; y < N; ++y)
        if (QV_CELL_FREE(cell[y]) && y != m->goal) ++count[QV_CELL_LABEL(cell[y])];
    h->seg.assign(nz + 1, 0);
    for (int z = 0; z < nz; ++z) h->seg[z + 1] = h->seg[z] + ((count[z] + qv::kKC - 1) / qv::kKC) * qv::kKC;
    h->Kp = std::max(h->seg[nz], qv::kKC);
    h->perm.assign(h->Kp, -1);
    h->pos.assign(N, -1);
    std::vector<int> fill(h->seg.begin(), h->seg.end() - 1);
    for (int y = 0; y < N; ++y)
        if (QV_CELL_FREE(cell[y]) && y != m->goal) {
            const int k = fill[QV_CELL_LABEL(cell[y])]++;
            h->perm[k] = y;
            h->pos[y] = k;
        }
    h->max_pieces = nz + qv::kPiecesExtra;
    h->piece_table = std::max(h->max_pieces, 512);
    h->band_cells = 4096;
    h->nbands = (N + h->band_cells - 1) / h->band_cells;
    const size_t P = max_points, G = h->max_vectors, Kp = h->Kp;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    h->off_pos = take(N * sizeof(int));
    h->off_perm = take(Kp * sizeof(int));
    h->off_piece = take(3 * h->piece_table * sizeof(int));
    h->S = h->Kp / qv::kSK;
    h->RTa = static_cast<int>((5 * P + qv::kRowTile - 1) / qv::kRowTile);
    h->RTb = static_cast<int>(2 * ((G + qv::kTN - 1) / qv::kTN));
    h->RTp = static_cast<int>((P + qv::kRowTile - 1) / qv::kRowTile);
    h->off_Bp = take(2 * qv::tiled_plane(h->S, h->RTa) * sizeof(float));
    h->off_RB = take(5 * P * sizeof(float));
    h->off_rpart = take(5 * P * h->nbands * sizeof(float));
    h->off_Gp = take(2 * qv::tiled_plane(h->S, h->RTb) * sizeof(float));
    h->off_Ap = take(2 * qv::tiled_plane(h->S, h->RTp) * sizeof(float));
    h->off_slab = take(static_cast<size_t>(h->max_pieces) * 5 * P * std::max(G, P) * sizeof(float));
    h->off_best = take(P * nz * sizeof(int));
    h->off_uniq = take(P * nz * sizeof(int));
    h->off_mult = take(P * nz * sizeof(int));
    h->off_nuniq = take(P * sizeof(int));
    h->off_astar = take(P * sizeof(int));
    h->off_val = take(P * sizeof(float));
    h->off_status = take(sizeof(int));
    h->ws_bytes = off;
    h->ws = nullptr;
    h->nB = 0;
    h->gp_value_nG = 0;
    *out = h;
    return QV_OK;
}

extern "C" void qv_pbvi_destroy(qv_pbvi *h) { delete h; }

extern "C" qv_status qv_pbvi_check(qv_pbvi *h, qv_stream_t stream) {
    if (!h) return qv_set_error(QV_ERR_INVALID, "qv_pbvi_check: null pointer");
    if (!h->ws) return QV_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int flag = 0;
    char *ws = static_cast<char *>(h->ws);
    if (qv_check_cuda(cudaMemcpyAsync(&flag, ws + h->off_status, sizeof(int), cudaMemcpyDeviceToHost, st), "copy") !=
            QV_OK ||
        qv_check_cuda(cudaStreamSynchronize(st), "qv_pbvi_check") != QV_OK)
        return QV_ERR_CUDA;
    if (!flag) return QV_OK;
    if (qv_check_cuda(cudaMemsetAsync(ws + h->off_status, 0, sizeof(int), st), "status reset") != QV_OK)
        return QV_ERR_CUDA;
    return qv_set_error(QV_ERR_TIMEOUT, "qv_pbvi: a tensor-core wait gave up");
}

extern "C" size_t qv_pbvi_workspace_bytes(const qv_pbvi *h) { return h ? h->ws_bytes : 0; }

extern "C" int32_t qv_pbvi_layout(const qv_pbvi *h, int32_t *seg_out) {
    if (!h) return 0;
    if (seg_out)
        for (int z = 0; z <= h->nz; ++z) seg_out[z] = h->seg[z];
    return h->Kp;
}

extern "C" qv_status qv_pbvi_init(const qv_model_t *m, float *d_alpha0, qv_stream_t stream) {
    QV_RANGE("qv_pbvi_init");
    if (!m || !m->d_cell || !d_alpha0) return qv_set_error(QV_ERR_INVALID, "qv_pbvi_init: null pointer");
    if (!(m->discount > 0.0f && m->discount < 1.0f) || m->num_beacons < 1)
        return qv_set_error(QV_ERR_INVALID, "qv_pbvi_init: bad model");
    qv::k_pbvi_init<<<1, qv::kPbThreads, 0, static_cast<cudaStream_t>(stream)>>>(qv::pb_model(m), d_alpha0);
    return qv_check_cuda(cudaGetLastError(), "qv_pbvi_init launch");
}

extern "C" qv_status qv_pbvi_expand(const qv_model_t *m, const float *d_B, int32_t nB, int32_t round, uint64_t seed,
                                    float *d_out, int32_t *d_action, int32_t *d_obs, int32_t *d_boundary,
                                    qv_stream_t stream) {
    QV_RANGE("qv_pbvi_expand");
    if (!m || !m->d_cell || !d_B || !d_out || !d_action || !d_obs || !d_boundary)
        return qv_set_error(QV_ERR_INVALID, "qv_pbvi_expand: null pointer");
    if (nB < 0 || round < 0 || m->num_beacons < 1 || m->num_beacons > QV_MAX_BEACONS)
        return qv_set_error(QV_ERR_INVALID, "qv_pbvi_expand: bad arguments");
    if (nB == 0) return QV_OK;
    const size_t smem = static_cast<size_t>(m->num_beacons + 1) * qv::kPbThreads * sizeof(float);
    if (smem > 48 * 1024 &&
        qv_check_cuda(cudaFuncSetAttribute(qv::k_pbvi_expand, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(smem)),
                      "smem attr") != QV_OK)
        return QV_ERR_CUDA;
    qv::k_pbvi_expand<<<nB, qv::kPbThreads, smem, static_cast<cudaStream_t>(stream)>>>(
        qv::pb_model(m), d_B, round, seed, d_out, d_action, d_obs, d_boundary);
    return qv_check_cuda(cudaGetLastError(), "qv_pbvi_expand launch");
}

extern "C" qv_status qv_pbvi_set_points(qv_pbvi *h, const float *d_B, int32_t nB, void *d_ws, size_t ws_bytes,
                                        qv_stream_t stream) {
    QV_RANGE("qv_pbvi_set_points");
    if (!h || !d_B || !d_ws) return qv_set_error(QV_ERR_INVALID, "qv_pbvi_set_points: null pointer");
    if (nB < 1 || nB > h->max_points)
        return qv_set_error(QV_ERR_INVALID, "qv_pbvi_set_points: %d points outside 1..%d", nB, h->max_points);
    if (ws_bytes < h->ws_bytes)
        return qv_set_error(QV_ERR_WORKSPACE, "qv_pbvi_set_points: workspace %zu < %zu bytes", ws_bytes, h->ws_bytes);
    if (reinterpret_cast<uintptr_t>(d_ws) & 255)
        return qv_set_error(QV_ERR_INVALID, "qv_pbvi_set_points: workspace must be 256-byte aligned");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(d_ws);
    if (h->ws != d_ws) {
        h->ws = d_ws;
        h->pieces.clear();
        if (qv_check_cuda(cudaMemsetAsync(ws + h->off_status, 0, sizeof(int), st), "status reset") != QV_OK)
            return QV_ERR_CUDA;
        if (qv_check_cuda(cudaMemcpyAsync(ws + h->off_pos, h->pos.data(), h->pos.size() * sizeof(int),
                                          cudaMemcpyHostToDevice, st), "pos table") != QV_OK ||
            qv_check_cuda(cudaMemcpyAsync(ws + h->off_perm, h->perm.data(), h->perm.size() * sizeof(int),
                                          cudaMemcpyHostToDevice, st), "perm table") != QV_OK)
            return QV_ERR_CUDA;
    }
    h->nB = nB;
    float *Bp = reinterpret_cast<float *>(ws + h->off_Bp);
    // zero the row tiles the contraction reads (both planes: 2 S stage rows
    // of RTa blocks, the first Mt of each), then scatter the live cells
    const size_t blk = static_cast<size_t>(qv::kRowTile) * qv::kSK * sizeof(float);
    const int Mt = (5 * nB + qv::kRowTile - 1) / qv::kRowTile;
    if (qv_check_cuda(cudaMemset2DAsync(Bp, h->RTa * blk, 0, Mt * blk, 2 * static_cast<size_t>(h->S), st),
                      "memset") != QV_OK)
        return QV_ERR_CUDA;
    const qv::PbModel pm = qv::pb_model(&h->model);
    qv::k_pbvi_predict<<<dim3(h->nbands, nB), qv::kPbThreads, 0, st>>>(
        pm, d_B, reinterpret_cast<const int *>(ws + h->off_pos), h->S, h->RTa, h->band_cells, Bp,
        reinterpret_cast<float *>(ws + h->off_rpart));
    qv::k_pbvi_reward<<<(nB * 5 + 127) / 128, 128, 0, st>>>(pm, d_B, nB, h->nbands,
                                                             reinterpret_cast<const float *>(ws + h->off_rpart),
                                                             reinterpret_cast<float *>(ws + h->off_RB));
    return qv_check_cuda(cudaGetLastError(), "qv_pbvi_set_points launch");
}

extern "C" qv_status qv_pbvi_backup(qv_pbvi *h, const float *d_G, int32_t nG, float *d_Gout, float *d_value,
                                    int32_t *d_astar, int32_t *d_best, float *d_q, qv_stream_t stream) {
    QV_RANGE("qv_pbvi_backup");
    return qv_pbvi_backup_fixed(h, d_G, nG, d_Gout, d_value, d_astar, d_best, d_q, nullptr, nullptr, stream);
}

extern "C" qv_status qv_pbvi_backup_fixed(qv_pbvi *h, const float *d_G, int32_t nG, float *d_Gout, float *d_value,
                                          int32_t *d_astar, int32_t *d_best, float *d_q, const int32_t *d_fix_astar,
                                          const int32_t *d_fix_best, qv_stream_t stream) {
    QV_RANGE("qv_pbvi_backup_fixed");
    if (!h || !d_G || !d_Gout) return qv_set_error(QV_ERR_INVALID, "qv_pbvi_backup: null pointer");
    if (d_fix_best && !d_fix_astar)
        return qv_set_error(QV_ERR_INVALID, "qv_pbvi_backup_fixed: fixed winners need the fixed actions");
    if (!h->ws || h->nB < 1) return qv_set_error(QV_ERR_INVALID, "qv_pbvi_backup: no point set (qv_pbvi_set_points)");
    if (nG < 1 || nG > h->max_vectors)
        return qv_set_error(QV_ERR_INVALID, "qv_pbvi_backup: %d vectors outside 1..%d", nG, h->max_vectors);
    const size_t N = static_cast<size_t>(h->model.H) * h->model.pitch;
    if (d_G < d_Gout + N * h->nB && d_Gout < d_G + N * nG)
        return qv_set_error(QV_ERR_INVALID, "qv_pbvi_backup: d_G and d_Gout overlap");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(h->ws);
    const int nB = h->nB, M = 5 * nB, Kp = h->Kp;
    const int Mt = (M + qv::kTM - 1) / qv::kTM, Nt = (nG + qv::kTN - 1) / qv::kTN;
    std::vector<int> pc;
    make_pieces(*h, Mt * Nt, Kp, true, std::min(h->max_pieces, piece_cap(*h, M, nG)), pc);
    if (upload_pieces(h, pc, st) != QV_OK) return QV_ERR_CUDA;
    const int npieces = static_cast<int>(pc.size() / 3);
    const int *piece = reinterpret_cast<const int *>(ws + h->off_piece);
    float *Gp = reinterpret_cast<float *>(ws + h->off_Gp);
    float *slab = reinterpret_cast<float *>(ws + h->off_slab);
    const int gthreads = 256, gblocks = 8 * qv_num_sms();
    h->gp_value_nG = 0;
    qv::k_pbvi_gather<<<gblocks, gthreads, 0, st>>>(d_G, nG, static_cast<int>(N),
                                                    reinterpret_cast<const int *>(ws + h->off_perm), h->S, h->RTb, Gp);
    if (qv::tc_prepare() != QV_OK) return QV_ERR_CUDA;
    const int ntiles = Mt * Nt * npieces;
    qv::k_pbvi_scores<<<std::min(ntiles, qv_num_sms()), qv::kTcThreads, qv::kTcSmem, st>>>(
        reinterpret_cast<const float *>(ws + h->off_Bp), h->RTa, Gp, h->RTb, M, nG, h->S, Mt, Nt, ntiles, piece,
        slab, reinterpret_cast<int *>(ws + h->off_status));
    const qv::PbModel pm = qv::pb_model(&h->model);
    int *best = d_best ? d_best : reinterpret_cast<int *>(ws + h->off_best);
    int *astar = d_astar ? d_astar : reinterpret_cast<int *>(ws + h->off_astar);
    float *value = d_value ? d_value : reinterpret_cast<float *>(ws + h->off_val);
    int *uniq = reinterpret_cast<int *>(ws + h->off_uniq), *mult = reinterpret_cast<int *>(ws + h->off_mult);
    int *nuniq = reinterpret_cast<int *>(ws + h->off_nuniq);
    const int chunk = qv::select_chunk(h->nz, nG, npieces);
    const size_t sel_smem = qv::select_smem(h->nz, chunk, npieces);
    if (sel_smem > 48 * 1024 &&
        qv_check_cuda(cudaFuncSetAttribute(qv::k_pbvi_select, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(sel_smem)),
                      "smem attr") != QV_OK)
        return QV_ERR_CUDA;
    qv::k_pbvi_select<<<nB, qv::kSelThreads, sel_smem, st>>>(pm, nB, nG, chunk, npieces, piece, slab,
                                                             reinterpret_cast<const float *>(ws + h->off_RB), value,
                                                             astar, best, d_q, uniq, mult, nuniq, d_fix_astar,
                                                             d_fix_best);
    const int band_rows = std::max(1, 4096 / h->model.pitch);
    const int nbands = (h->model.H + band_rows - 1) / band_rows;
    const size_t a_smem = static_cast<size_t>(band_rows + 2) * h->model.pitch * sizeof(float);
    if (a_smem > 48 * 1024 &&
        qv_check_cuda(cudaFuncSetAttribute(qv::k_pbvi_alpha, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(a_smem)),
                      "smem attr") != QV_OK)
        return QV_ERR_CUDA;
    qv::k_pbvi_alpha<<<dim3(nbands, nB), qv::kPbThreads, a_smem, st>>>(pm, band_rows, d_G, astar, best, uniq, mult,
                                                                        nuniq, d_Gout);
    return qv_check_cuda(cudaGetLastError(), "qv_pbvi_backup launch");
}

extern "C" qv_status qv_pbvi_value(qv_pbvi *h, const float *d_G, int32_t nG, const float *d_b, int32_t nb,
                                   float *d_value, int32_t *d_arg, qv_stream_t stream) {
    QV_RANGE("qv_pbvi_value");
    if (!h || !d_b || !d_value) return qv_set_error(QV_ERR_INVALID, "qv_pbvi_value: null pointer");
    if (!h->ws) return qv_set_error(QV_ERR_INVALID, "qv_pbvi_value: no workspace yet (qv_pbvi_set_points)");
    if (nG < 1 || nG > h->max_vectors || nb < 0)
        return qv_set_error(QV_ERR_INVALID, "qv_pbvi_value: %d vectors, %d beliefs", nG, nb);
    if (!d_G && h->gp_value_nG != nG)
        return qv_set_error(QV_ERR_INVALID, "qv_pbvi_value: no vectors of this count kept from the last call");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(h->ws);
    const int Kp = h->Kp, N = h->model.H * h->model.pitch;
    float *Ap = reinterpret_cast<float *>(ws + h->off_Ap);
    float *Gp = reinterpret_cast<float *>(ws + h->off_Gp);
    float *slab = reinterpret_cast<float *>(ws + h->off_slab);
    const int *perm = reinterpret_cast<const int *>(ws + h->off_perm);
    const int gb = 8 * qv_num_sms();
    const int Nt = (nG + qv::kTN - 1) / qv::kTN;
    if (d_G) {
        qv::k_pbvi_gather<<<gb, 256, 0, st>>>(d_G, nG, N, perm, h->S, h->RTb, Gp);
        h->gp_value_nG = nG;
    }
    // beliefs in chunks of up to max_points (the size of the Ap region)
    for (int c0 = 0; c0 < nb; c0 += h->max_points) {
        const int nc = std::min(h->max_points, nb - c0);
        const int Mt = (nc + qv::kTM - 1) / qv::kTM;
        std::vector<int> pc;
        make_pieces(*h, Mt * Nt, Kp, false, piece_cap(*h, nc, nG), pc);
        if (upload_pieces(h, pc, st) != QV_OK) return QV_ERR_CUDA;
        const int npieces = static_cast<int>(pc.size() / 3);
        qv::k_pbvi_scatter_points<<<gb, 256, 0, st>>>(d_b + static_cast<size_t>(c0) * N, nc, N, perm, h->S, h->RTp,
                                                       Ap);
        if (qv::tc_prepare() != QV_OK) return QV_ERR_CUDA;
        const int ntiles = Mt * Nt * npieces;
        qv::k_pbvi_scores<<<std::min(ntiles, qv_num_sms()), qv::kTcThreads, qv::kTcSmem, st>>>(
            Ap, h->RTp, Gp, h->RTb, nc, nG, h->S, Mt, Nt, ntiles, reinterpret_cast<const int *>(ws + h->off_piece),
            slab, reinterpret_cast<int *>(ws + h->off_status));
        int groups, threads;
        qv::rowmax_shape(nc, nG, groups, threads);
        qv::k_pbvi_rowmax<<<nc, threads, 0, st>>>(nc, nG, npieces, groups, slab, d_value + c0,
                                                  d_arg ? d_arg + c0 : nullptr);
    }
    return qv_check_cuda(cudaGetLastError(), "qv_pbvi_value launch");
}
