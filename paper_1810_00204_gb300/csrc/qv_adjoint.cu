// qv_adjoint.cu -- reverse mode of the plan's root value.
//
// The root value U_V(b0) depends on the slip eps (through T in every
// prediction, Eq. 3 with Eq. 10, and through R), the sensor accuracy alpha
// (through O in every correction, Eq. 3), the cost map c (through the stage
// reward, hence R(b, a) and the alpha-vectors Q) and b0.  Held fixed: the
// sampled measurements, the FREQ weights f/K and every max (Alg. 7 over
// actions, Eq. 4 over a leaf's alpha-vectors, the Bellman max of every value
// iteration sweep), ties to the lowest index as the forward takes them.
//
// Tree part (qv_tree_backward).  Only V-nodes on chosen actions carry an
// adjoint: u(root) = dL, and Alg. 6 / 7 pass u(child) = gamma * (f/K) * u(node)
// to the children of the node's argmax action.  Going up from the deepest
// internal level, the adjoint of a node's belief b (action a*, children z with
// beliefs b'_z = O_z bbar / P_z, bbar = T_{a*}^T b) is
//   g(y)    = sum_z O_z(y) (beta_z(y) - <beta_z, b'_z>) / P_z
//   h(y)    = u r(y) + g(y)
//   beta(x) = sum_y T(x, a*, y) h(y)          (x free, not the goal)
//   beta(g) = g(goal)                          (the goal is absorbing)
// with beta_z = u_z Q(a'_z, .) for a leaf (a'_z its argmax, Eq. 4).  Along the
// way: d/d eps += sum_x b(x) sum_y dT(x, a*, y)/d eps h(y); d/d alpha +=
// sum_z sum_y bbar(y) (beta_z - <beta_z, b'_z>)/P_z dO_z(y)/d alpha;
// d/dc(y) -= u bbar(y) (R(b, a*) = sum_y bbar(y) r(y) - 100 b(goal)); and
// dL/dQ(a'_z, y) += u_z b'_z(y) for leaf children.
//
// Value-iteration part (mdp_value_backward).  Q = sum_y T (r + gamma V_S) and
// V_{k+1}(x) = sum_y T(x, a*_k(x), y) (r(y) + gamma V_k(y)): the adjoint
// lambda_S = gamma T^T Qbar, lambda_k = gamma T_{a*_k}^T lambda_{k+1}, with
// d/dc(y) -= (T^T lambda)(y) and d/d eps += lambda(x) dT/d eps (r + gamma V)
// at every step.  Sweeps are recomputed from checkpoints, `every` at a time.
#include <algorithm>
#include <cstring>

#include "qv_plan_types.cuh"
#include "qv_vi_cell.cuh"

namespace qv {
namespace {

constexpr int kAdjThreads = 256;

// Active V-nodes of one level, ascending node index (children of one node
// are contiguous and follow their parent's order).
struct AdjLevel {
    int *node;       // local node index in the level
    int *astar;      // chosen action (argmax of U_Q)
    int *cbeg;       // index of the first child in the next level's list
    int *cnum;       // children of the chosen action
    double *u;       // adjoint of U_V
    double *beta;    // [cap][N] adjoint of the belief (levels 1..d-1)
    double *s_part;  // [cap][bands] partial <beta, b>
    double *red;     // [cap][bands][2] partial d/d eps, d/d alpha
    float *bsc;      // [cap][N] beliefs recomputed for a level the plan did not store
    int cap;
};

struct AdjArgs {
    PlanDev pl;
    EpDev ep;
    int e, depth, bands, band_rows;
    double dL;
    int *n_act;  // [d+1]
    AdjLevel lv[kMaxD + 1];
    double *Qbar, *dslip, *dacc, *dcost, *db0;
};

__device__ int block_scan_excl(int v, int *sh, int &total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int w = 0; w < nw; ++w) {
            const int t = sh[w];
            sh[w] = run;
            run += t;
        }
        sh[nw] = run;
    }
    __syncthreads();
    const int ex = sh[wid] + x - v;
    total = sh[nw];
    __syncthreads();
    return ex;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum of up to three values over the CTA; thread 0 gets the totals.
__device__ void block_sum3(double &a, double &b, double &c) {
    __shared__ double s[3][kAdjThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    a = warp_sum_d(a);
    b = warp_sum_d(b);
    c = warp_sum_d(c);
    if (lane == 0) {
        s[0][wid] = a;
        s[1][wid] = b;
        s[2][wid] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        a = b = c = 0.0;
        for (int w = 0; w < nw; ++w) {
            a += s[0][w];
            b += s[1][w];
            c += s[2][w];
        }
    }
    __syncthreads();
}

__device__ __forceinline__ void fill_lut(float *lut, float slip) {
    if (threadIdx.x < 64) lut[threadIdx.x] = self_weight(threadIdx.x >> 4, threadIdx.x & 15u, slip);
}

// Predicted mass bbar_a(y) = sum_x T(x, a, y) b(x) (Eq. 3 numerator), from
// global memory, with the same arithmetic as the search kernel.
__device__ __forceinline__ float predicted(const float *b, int y, int P, unsigned cw, bool is_goal, float slip,
                                           const float *lut, int a) {
    const unsigned inf = QV_CELL_INFLOW(cw);
    float nb[4];
    nb[kDirN] = (inf & 1u) ? __ldg(b + y - P) : 0.0f;
    nb[kDirE] = (inf & 2u) ? __ldg(b + y + 1) : 0.0f;
    nb[kDirS] = (inf & 4u) ? __ldg(b + y + P) : 0.0f;
    nb[kDirW] = (inf & 8u) ? __ldg(b + y - 1) : 0.0f;
    return predict_one(nb, __ldg(b + y), cw, is_goal, slip, lut, a);
}

// ---------------------------------------------------------------- tree adjoint kernels
// Active nodes of every level and their adjoints, top down (one CTA).
__global__ void __launch_bounds__(kAdjThreads) k_adj_setup(AdjArgs a) {
    __shared__ int sh[kAdjThreads / 32 + 1];
    __shared__ int s_n;
    const PlanDev &pl = a.pl;
    const EpDev &ep = a.ep;
    if (threadIdx.x == 0) {
        a.lv[0].node[0] = 0;
        a.lv[0].u[0] = a.dL;
        a.n_act[0] = 1;
        s_n = 1;
    }
    __syncthreads();
    for (int l = 0; l < a.depth; ++l) {
        const AdjLevel &L = a.lv[l];
        const AdjLevel &Lc = a.lv[l + 1];
        const int n = s_n;
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const long long ia = static_cast<long long>(ep.inode_base[l] + L.node[k]) * 5;
            int best = 0;
            float qb = __ldcg(pl.UQ + ia);
            for (int b = 1; b < 5; ++b) {
                const float q = __ldcg(pl.UQ + ia + b);
                if (q > qb) {
                    qb = q;
                    best = b;
                }
            }
            L.astar[k] = best;
            L.cnum[k] = __ldcg(pl.nchild + ia + best);
        }
        __syncthreads();
        int running = 0;
        for (int base = 0; base < n; base += blockDim.x) {
            const int k = base + threadIdx.x;
            const int v = k < n ? L.cnum[k] : 0;
            int total;
            const int ex = block_scan_excl(v, sh, total);
            if (k < n) L.cbeg[k] = running + ex;
            running += total;
        }
        __syncthreads();
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const long long ia = static_cast<long long>(ep.inode_base[l] + L.node[k]) * 5 + L.astar[k];
            const int off = __ldcg(pl.choff + ia);
            const int m = L.cnum[k], cb = L.cbeg[k];
            for (int j = 0; j < m && cb + j < Lc.cap; ++j) {
                Lc.node[cb + j] = off + j;
                Lc.u[cb + j] = static_cast<double>(ep.gamma) *
                               static_cast<double>(__ldcg(pl.weight + ep.node_base[l + 1] + off + j)) * L.u[k];
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            s_n = min(running, Lc.cap);
            a.n_act[l + 1] = s_n;
        }
        __syncthreads();
    }
}

// Beliefs of the active nodes of level l that the plan did not store (the
// deepest internal level of the fused mode): Phi(parent, a, z) of Eq. 3.
__global__ void __launch_bounds__(kAdjThreads) k_adj_recompute(AdjArgs a, int l) {
    __shared__ float lut[64];
    const EpDev &ep = a.ep;
    const PlanDev &pl = a.pl;
    fill_lut(lut, ep.slip);
    __syncthreads();
    const AdjLevel &L = a.lv[l];
    const int n = a.n_act[l];
    const int r0 = blockIdx.x * a.band_rows, r1 = min(ep.H, r0 + a.band_rows);
    for (int j = blockIdx.y; j < n; j += gridDim.y) {
        const int g = ep.node_base[l] + L.node[j];
        const int p = __ldcg(pl.parent + g), an = __ldcg(pl.action + g), z = __ldcg(pl.obs + g);
        const float P = __ldcg(pl.pz + g);
        const float sa = ep.acc / P, se = ep.eta / P;
        const float *bp = (l - 1 == 0) ? ep.b0 : pl.beliefs + ep.belief_off[l - 1] + static_cast<long long>(p) * ep.N;
        float *out = L.bsc + static_cast<long long>(j) * ep.N;
        for (int t = threadIdx.x; t < (r1 - r0) * ep.P; t += blockDim.x) {
            const int y = r0 * ep.P + t;
            const unsigned cw = __ldg(ep.cell + y);
            float v = 0.0f;
            if (QV_CELL_FREE(cw)) {
                const float pa = predicted(bp, y, ep.P, cw, y == ep.goal, ep.slip, lut, an);
                v = pa * (static_cast<int>(QV_CELL_LABEL(cw)) == z ? sa : se);
            }
            out[y] = v;
        }
    }
}

// One level of the bottom-up pass: per active node, per band of rows.
__global__ void __launch_bounds__(kAdjThreads) k_adj_level(AdjArgs a, int l) {
    extern __shared__ __align__(16) double sh_h[];  // h on the band's rows and one halo row each side
    __shared__ float lut[64];
    __shared__ int c_z[QV_MAX_K], c_arg[QV_MAX_K];
    __shared__ double c_invP[QV_MAX_K], c_u[QV_MAX_K], c_s[QV_MAX_K];
    __shared__ const double *c_beta[QV_MAX_K];
    const EpDev &ep = a.ep;
    const PlanDev &pl = a.pl;
    fill_lut(lut, ep.slip);
    const AdjLevel &L = a.lv[l];
    const AdjLevel &Lc = a.lv[l + 1];
    const int n = a.n_act[l];
    const int H = ep.H, P = ep.P, N = ep.N;
    const int r0 = blockIdx.x * a.band_rows, r1 = min(H, r0 + a.band_rows);
    const bool leafc = (l + 1 == a.depth);
    const double alpha = ep.acc, eta = ep.eta, dO_off = -1.0 / ep.B;
    const double slip = ep.slip, fwd = 1.0 - 2.0 * slip;
    for (int j = blockIdx.y; j < n; j += gridDim.y) {
        const int i = L.node[j], as = L.astar[j];
        const double u = L.u[j];
        const float *b = l == 0 ? ep.b0
                         : ep.belief_off[l] >= 0 ? pl.beliefs + ep.belief_off[l] + static_cast<long long>(i) * N
                                                 : L.bsc + static_cast<long long>(j) * N;
        const int cb = L.cbeg[j];
        const int nc = max(0, min(min(L.cnum[j], QV_MAX_K), Lc.cap - cb));
        __syncthreads();  // the previous node's use of the child tables is over
        for (int c = threadIdx.x; c < nc; c += blockDim.x) {
            const int idx = cb + c;
            const int g = ep.node_base[l + 1] + Lc.node[idx];
            c_z[c] = __ldcg(pl.obs + g);
            c_invP[c] = 1.0 / static_cast<double>(__ldcg(pl.pz + g));
            c_u[c] = Lc.u[idx];
            if (leafc) {
                c_arg[c] = __ldcg(pl.leaf_arg + g);
                c_s[c] = Lc.u[idx] * static_cast<double>(__ldcg(pl.value + g));
                c_beta[c] = nullptr;
            } else {
                double s = 0.0;
                for (int bb = 0; bb < a.bands; ++bb) s += Lc.s_part[static_cast<long long>(idx) * a.bands + bb];
                c_arg[c] = 0;
                c_s[c] = s;
                c_beta[c] = Lc.beta + static_cast<long long>(idx) * N;
            }
        }
        __syncthreads();
        double acc_part = 0.0, eps_part = 0.0, s_part = 0.0;
        // h(y) = u r(y) + g(y) on rows r0-1 .. r1 (clipped); the own rows also
        // take the alpha, cost and Q terms
        const int lo = max(0, r0 - 1), hi = min(H, r1 + 1);
        for (int t = threadIdx.x; t < (hi - lo) * P; t += blockDim.x) {
            const int row = lo + t / P;
            const int y = lo * P + t;
            const unsigned cw = __ldg(ep.cell + y);
            double hv = 0.0;
            if (QV_CELL_FREE(cw)) {
                const bool is_goal = (y == ep.goal);
                const double bbar = predicted(b, y, P, cw, is_goal, ep.slip, lut, as);
                const int lab = QV_CELL_LABEL(cw);
                const bool own = row >= r0 && row < r1;
                double gsum = 0.0;
                double qb[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
                for (int c = 0; c < nc; ++c) {
                    const bool hit = (lab == c_z[c]);
                    const double O = hit ? alpha : eta;
                    const double bc = leafc ? c_u[c] * static_cast<double>(__ldg(ep.Q + c_arg[c] * N + y))
                                            : __ldcg(c_beta[c] + y);
                    const double d = (bc - c_s[c]) * c_invP[c];
                    gsum += O * d;
                    if (own) {
                        acc_part += bbar * d * (hit ? 1.0 : dO_off);
                        if (leafc) qb[c_arg[c]] += c_u[c] * O * bbar * c_invP[c];
                    }
                }
                const double r = is_goal ? 100.0 : -1.0 - (ep.cost ? static_cast<double>(__ldg(ep.cost + y)) : 0.0);
                hv = u * r + gsum;
                if (own) {
                    if (a.dcost && !is_goal) atomicAdd(a.dcost + y, -u * bbar);
                    if (leafc)
                        for (int q = 0; q < 5; ++q)
                            if (qb[q] != 0.0) atomicAdd(a.Qbar + static_cast<long long>(q) * N + y, qb[q]);
                }
            }
            sh_h[(row - (r0 - 1)) * P + (y - row * P)] = hv;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < (r1 - r0) * P; t += blockDim.x) {
            const int rr = t / P, col = t - rr * P;
            const int x = r0 * P + t;
            const unsigned cw = __ldg(ep.cell + x);
            const double *hrow = sh_h + (rr + 1) * P;
            double beta = 0.0;
            if (QV_CELL_FREE(cw)) {
                const double hx = hrow[col];
                const double bx = __ldg(b + x);
                if (x == ep.goal) {
                    beta = hx - 100.0 * u;
                } else if (as == 4) {
                    beta = hx;
                } else {
                    const unsigned blk = QV_CELL_BLOCKED(cw);
                    double hn[4];
                    hn[kDirN] = (blk & 1u) ? hx : hrow[col - P];
                    hn[kDirE] = (blk & 2u) ? hx : hrow[col + 1];
                    hn[kDirS] = (blk & 4u) ? hx : hrow[col + P];
                    hn[kDirW] = (blk & 8u) ? hx : hrow[col - 1];
                    const double h0 = hn[as], h1 = hn[(as + 1) & 3], h2 = hn[(as + 3) & 3];
                    beta = fwd * h0 + slip * (h1 + h2);
                    eps_part += bx * (-2.0 * h0 + h1 + h2);
                }
                s_part += beta * bx;
            }
            if (l >= 1) L.beta[static_cast<long long>(j) * N + x] = beta;
            else if (a.db0) a.db0[x] += beta;
        }
        block_sum3(s_part, eps_part, acc_part);
        if (threadIdx.x == 0) {
            const long long rec = static_cast<long long>(j) * a.bands + blockIdx.x;
            L.s_part[rec] = s_part;
            L.red[2 * rec] = eps_part;
            L.red[2 * rec + 1] = acc_part;
        }
    }
}

// d/d eps and d/d alpha: the per-(node, band) records of every level, summed
// in a fixed order by one warp.
__global__ void k_adj_reduce(AdjArgs a) {
    double se = 0.0, sa = 0.0;
    for (int l = 0; l < a.depth; ++l) {
        const long long m = static_cast<long long>(a.n_act[l]) * a.bands;
        for (long long r = threadIdx.x; r < m; r += 32) {
            se += a.lv[l].red[2 * r];
            sa += a.lv[l].red[2 * r + 1];
        }
    }
    se = warp_sum_d(se);
    sa = warp_sum_d(sa);
    if (threadIdx.x == 0) {
        *a.dslip += se;
        *a.dacc += sa;
    }
}

// Depth 0: the root is the leaf, U_V(b0) = sum_x b0(x) Q(a', x) (Eq. 4).
__global__ void k_adj_depth0(AdjArgs a) {
    const EpDev &ep = a.ep;
    const int ap = a.pl.result[a.e].action;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < ep.N; x += gridDim.x * blockDim.x) {
        if (!QV_CELL_FREE(__ldg(ep.cell + x))) continue;
        a.Qbar[static_cast<long long>(ap) * ep.N + x] += a.dL * static_cast<double>(__ldg(ep.b0 + x));
        if (a.db0) a.db0[x] += a.dL * static_cast<double>(__ldg(ep.Q + static_cast<long long>(ap) * ep.N + x));
    }
}

// ---------------------------------------------------------------- value-iteration adjoint
struct VIBack {
    int H, W, P, N;
    const uint16_t *cell;
    const float *cost;
    int goal;
    float slip;
    double gamma;
    int sweeps, every;
    const double *ckpt;   // [ceil(sweeps / every)][N]
    const double *Qbar;   // [5][N]
    double *segV;         // [every + 1][N] V_k of the current segment
    unsigned char *segA;  // [every][N] argmax of sweep k
    double *lam0, *lam1;  // [N]
    double *dcost;        // [N] nullable
    double *dslip;        // scalar
    double *red;          // [gridDim.x]
    VIWork *work;
    unsigned *done;       // [gridDim.x] steps completed per CTA
    unsigned spin_limit;  // polls before a wait on other CTAs gives up
};

__device__ __forceinline__ double self_weight_d(int a, unsigned blk, double slip) {
    const double fwd = 1.0 - 2.0 * slip;
    const unsigned p1 = (a + 1) & 3, p2 = (a + 3) & 3;
    return fwd * static_cast<double>((blk >> a) & 1u) +
           slip * static_cast<double>(((blk >> p1) & 1u) + ((blk >> p2) & 1u));
}

// Weight with which a free, non-goal neighbour in direction D of y, taking
// action a, lands on y: the neighbour moves toward y along (D + 2) & 3.
__device__ __forceinline__ double inflow_weight(int a, int D, double fwd, double slip) {
    if (a == 4 || a == D) return 0.0;
    return a == ((D + 2) & 3) ? fwd : slip;
}

// r(t) + gamma V(t) on the four move targets of x (Eq. 10: a blocked move
// stays on x), and on x itself.
__device__ __forceinline__ void arrive4(const VIBack &a, int x, unsigned cw, const double *V, double wn[4],
                                        double &wx) {
    const int col = x % a.P;
    const double *row = V + (x - col);
    const unsigned blk = QV_CELL_BLOCKED(cw);
    wx = arrive_value(a, x, row, col);
    wn[kDirN] = (blk & 1u) ? wx : arrive_value(a, x - a.P, row - a.P, col);
    wn[kDirE] = (blk & 2u) ? wx : arrive_value(a, x + 1, row, col + 1);
    wn[kDirS] = (blk & 4u) ? wx : arrive_value(a, x + a.P, row + a.P, col);
    wn[kDirW] = (blk & 8u) ? wx : arrive_value(a, x - 1, row, col - 1);
}

// Each CTA owns a band of whole rows; every step reads one row into the
// neighbouring bands, so consecutive steps are ordered by the neighbours'
// progress flags only (publish_step / wait_neighbours).
__global__ void __launch_bounds__(kAdjThreads) k_vi_backward(VIBack a) {
    const unsigned nblocks = gridDim.x;
    const int rows_per_cta = (a.H + nblocks - 1) / nblocks;
    const int r_begin = min(a.H, static_cast<int>(blockIdx.x) * rows_per_cta);
    const int r_end = min(a.H, r_begin + rows_per_cta);
    const int y0 = r_begin * a.P, y1 = r_end * a.P;
    const int N = a.N, c = a.every, S = a.sweeps;
    const double slip = a.slip, fwd = 1.0 - 2.0 * slip;
    const int J = (S + c - 1) / c;
    double eps = 0.0;
    double *lam = a.lam0, *lam_next = a.lam1;
    unsigned step = 0;
    // V_{k0 + i} of the current segment: the checkpoint for i = 0
    auto slot = [&](int j, int i) -> const double * {
        return i == 0 ? a.ckpt + static_cast<size_t>(j) * N : a.segV + static_cast<size_t>(i) * N;
    };
    for (int j = J - 1; j >= 0; --j) {
        const int k0 = j * c, Lseg = min(S, k0 + c) - k0;
        // recompute sweeps k0 .. k0 + Lseg - 1 with the forward's arithmetic
        for (int i = 0; i < Lseg; ++i) {
            const double *Vk = slot(j, i);
            double *Vn = a.segV + static_cast<size_t>(i + 1) * N;
            unsigned char *Ak = a.segA + static_cast<size_t>(i) * N;
            for (int y = y0 + threadIdx.x; y < y1; y += blockDim.x) {
                const unsigned cw = __ldg(a.cell + y);
                double v = 0.0;
                int arg = 0;
                if (QV_CELL_FREE(cw) && y != a.goal) {
                    const int col = y % a.P;
                    double q[5];
                    cell_q(a, y, col, cw, Vk + (y - col), q);
                    v = q[0];
                    for (int d = 1; d < 5; ++d)
                        if (q[d] > v) {
                            v = q[d];
                            arg = d;
                        }
                }
                Vn[y] = v;
                Ak[y] = static_cast<unsigned char>(arg);
            }
            publish_step(a.done, ++step);
            if (!wait_neighbours(a.done, step, &a.work->status, a.spin_limit)) return;
        }
        if (j == J - 1) {
            // Q = sum_y T (r + gamma V_S): lambda_S = gamma T^T Qbar
            const double *VS = slot(j, Lseg);
            for (int y = y0 + threadIdx.x; y < y1; y += blockDim.x) {
                const unsigned cw = __ldg(a.cell + y);
                double rho = 0.0;
                if (QV_CELL_FREE(cw)) {
                    if (y != a.goal) {
                        const unsigned blk = QV_CELL_BLOCKED(cw);
                        double wn[4], wx;
                        arrive4(a, y, cw, VS, wn, wx);
                        for (int q = 0; q < 5; ++q) {
                            const double qb = __ldg(a.Qbar + static_cast<size_t>(q) * N + y);
                            rho += qb * (q == 4 ? 1.0 : self_weight_d(q, blk, slip));
                            if (q < 4) eps += qb * (-2.0 * wn[q] + wn[(q + 1) & 3] + wn[(q + 3) & 3]);
                        }
                    }
                    const unsigned inf = QV_CELL_INFLOW(cw);
                    for (int D = 0; D < 4; ++D) {
                        if (!((inf >> D) & 1u)) continue;
                        const int x = D == kDirN ? y - a.P : D == kDirE ? y + 1 : D == kDirS ? y + a.P : y - 1;
                        rho += fwd * __ldg(a.Qbar + static_cast<size_t>((D + 2) & 3) * N + x) +
                               slip * (__ldg(a.Qbar + static_cast<size_t>((D + 1) & 3) * N + x) +
                                       __ldg(a.Qbar + static_cast<size_t>((D + 3) & 3) * N + x));
                    }
                    if (a.dcost && y != a.goal) a.dcost[y] -= rho;
                }
                lam[y] = a.gamma * rho;
            }
            publish_step(a.done, ++step);
            if (!wait_neighbours(a.done, step, &a.work->status, a.spin_limit)) return;
        }
        // sweeps k = k0 + Lseg - 1 .. k0: lam holds lambda_{k+1}
        for (int i = Lseg - 1; i >= 0; --i) {
            const double *Vk = slot(j, i);
            const unsigned char *Ak = a.segA + static_cast<size_t>(i) * N;
            for (int y = y0 + threadIdx.x; y < y1; y += blockDim.x) {
                const unsigned cw = __ldg(a.cell + y);
                double rho = 0.0;
                if (QV_CELL_FREE(cw)) {
                    if (y != a.goal) {
                        const int act = __ldcg(Ak + y);
                        const double ly = __ldcg(lam + y);
                        rho += ly * (act == 4 ? 1.0 : self_weight_d(act, QV_CELL_BLOCKED(cw), slip));
                        if (act < 4 && ly != 0.0) {
                            double wn[4], wx;
                            arrive4(a, y, cw, Vk, wn, wx);
                            eps += ly * (-2.0 * wn[act] + wn[(act + 1) & 3] + wn[(act + 3) & 3]);
                        }
                    }
                    const unsigned inf = QV_CELL_INFLOW(cw);
                    for (int D = 0; D < 4; ++D) {
                        if (!((inf >> D) & 1u)) continue;
                        const int x = D == kDirN ? y - a.P : D == kDirE ? y + 1 : D == kDirS ? y + a.P : y - 1;
                        rho += __ldcg(lam + x) * inflow_weight(__ldcg(Ak + x), D, fwd, slip);
                    }
                    if (a.dcost && y != a.goal) a.dcost[y] -= rho;
                }
                lam_next[y] = a.gamma * rho;
            }
            publish_step(a.done, ++step);
            if (!wait_neighbours(a.done, step, &a.work->status, a.spin_limit)) return;
            double *t = lam;
            lam = lam_next;
            lam_next = t;
        }
    }
    double z1 = 0.0, z2 = 0.0;
    block_sum3(eps, z1, z2);
    if (threadIdx.x == 0) a.red[blockIdx.x] = eps;
    publish_step(a.done, ++step);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double s = 0.0;
        for (unsigned b = 0; b < nblocks; ++b) {
            unsigned it = 0;
            while (ld_acquire(a.done + b) < step) {
                if (++it > a.spin_limit || (*((volatile unsigned *)&a.work->status) & kErrTimeout)) {
                    atomicOr(&a.work->status, kErrTimeout);
                    return;
                }
                __nanosleep(32);
            }
            s += *((volatile double *)(a.red + b));
        }
        *a.dslip += s;
    }
}

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

// Worst-case active nodes per level: one action per node, at most
// min(K, B + 1) distinct children per action, and never above the level's
// capacity in the plan.
void level_caps(const qv_plan_t *pl, int e, int caps[kMaxD + 1]) {
    const qv::EpDev &ep = pl->eps[e];
    const long long m = std::min<long long>(pl->params.K, ep.B + 1);
    long long c = 1;
    for (int l = 0; l <= pl->params.depth; ++l) {
        caps[l] = static_cast<int>(std::min<long long>(c, ep.cap[l]));
        c = std::min<long long>(c * m, 1LL << 30);
    }
}

struct AdjLayout {
    size_t total = 0;
    size_t n_act = 0;
    size_t node[kMaxD + 1], astar[kMaxD + 1], cbeg[kMaxD + 1], cnum[kMaxD + 1], u[kMaxD + 1], beta[kMaxD + 1],
        s_part[kMaxD + 1], red[kMaxD + 1], bsc = 0;
    bool recompute = false;
    int caps[kMaxD + 1] = {};
    int bands = 0;
};

AdjLayout adj_layout(const qv_plan_t *pl, int e) {
    AdjLayout L;
    const qv::EpDev &ep = pl->eps[e];
    const int D = pl->params.depth;
    level_caps(pl, e, L.caps);
    L.bands = ep.bands;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        o = a256(o);
        const size_t r = o;
        o += std::max<size_t>(bytes, 16);
        return r;
    };
    L.n_act = take(sizeof(int) * (D + 1));
    for (int l = 0; l <= D; ++l) {
        const size_t c = L.caps[l];
        L.node[l] = take(sizeof(int) * c);
        L.astar[l] = take(sizeof(int) * c);
        L.cbeg[l] = take(sizeof(int) * c);
        L.cnum[l] = take(sizeof(int) * c);
        L.u[l] = take(sizeof(double) * c);
        L.beta[l] = (l >= 1 && l < D) ? take(sizeof(double) * c * ep.N) : 0;
        L.s_part[l] = l < D ? take(sizeof(double) * c * ep.bands) : 0;
        L.red[l] = l < D ? take(sizeof(double) * 2 * c * ep.bands) : 0;
    }
    L.recompute = D >= 2 && ep.belief_off[D - 1] < 0;
    if (L.recompute) L.bsc = take(sizeof(float) * static_cast<size_t>(L.caps[D - 1]) * ep.N);
    L.total = a256(o);
    return L;
}

}  // namespace
}  // namespace qv

extern "C" size_t qv_tree_backward_workspace_bytes(const qv_plan_t *pl, int32_t e) {
    if (!pl || e < 0 || e >= pl->E) return 0;
    return qv::adj_layout(pl, e).total;
}

extern "C" qv_status qv_tree_backward(const qv_plan_t *pl, int32_t e, double dL_dV, double *d_Qbar, double *d_dslip,
                                      double *d_dacc, double *d_dcost, double *d_db0, void *d_ws, size_t ws_bytes,
                                      qv_stream_t stream) {
    QV_RANGE("qv_tree_backward");
    using namespace qv;
    if (!pl || !d_Qbar || !d_dslip || !d_dacc || !d_ws)
        return qv_set_error(QV_ERR_INVALID, "qv_tree_backward: null pointer");
    if (e < 0 || e >= pl->E) return qv_set_error(QV_ERR_INVALID, "qv_tree_backward: episode %d", e);
    if (pl->params.weight_mode != QV_WEIGHT_FREQ)
        return qv_set_error(QV_ERR_INVALID, "qv_tree_backward: only FREQ weights are held fixed by the adjoint");
    const AdjLayout L = adj_layout(pl, e);
    if (ws_bytes < L.total)
        return qv_set_error(QV_ERR_WORKSPACE, "qv_tree_backward: workspace %zu < %zu bytes", ws_bytes, L.total);
    if (reinterpret_cast<uintptr_t>(d_ws) & 255)
        return qv_set_error(QV_ERR_INVALID, "qv_tree_backward: workspace must be 256-byte aligned");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int D = pl->params.depth;
    // the leaves' records (observations, P(z), values, argmax) in stream order
    if (qv_plan_leaf_records(const_cast<qv_plan_t *>(pl), st, false) != QV_OK) return QV_ERR_CUDA;
    char *ws = static_cast<char *>(d_ws);
    AdjArgs a;
    std::memset(&a, 0, sizeof(a));
    a.pl = pl->dev;
    a.ep = pl->eps[e];
    a.e = e;
    a.depth = D;
    a.bands = L.bands;
    a.band_rows = a.ep.band_rows;
    a.dL = dL_dV;
    a.n_act = reinterpret_cast<int *>(ws + L.n_act);
    for (int l = 0; l <= D; ++l) {
        AdjLevel &v = a.lv[l];
        v.cap = L.caps[l];
        v.node = reinterpret_cast<int *>(ws + L.node[l]);
        v.astar = reinterpret_cast<int *>(ws + L.astar[l]);
        v.cbeg = reinterpret_cast<int *>(ws + L.cbeg[l]);
        v.cnum = reinterpret_cast<int *>(ws + L.cnum[l]);
        v.u = reinterpret_cast<double *>(ws + L.u[l]);
        v.beta = (l >= 1 && l < D) ? reinterpret_cast<double *>(ws + L.beta[l]) : nullptr;
        v.s_part = l < D ? reinterpret_cast<double *>(ws + L.s_part[l]) : nullptr;
        v.red = l < D ? reinterpret_cast<double *>(ws + L.red[l]) : nullptr;
        v.bsc = (L.recompute && l == D - 1) ? reinterpret_cast<float *>(ws + L.bsc) : nullptr;
    }
    a.Qbar = d_Qbar;
    a.dslip = d_dslip;
    a.dacc = d_dacc;
    a.dcost = d_dcost;
    a.db0 = d_db0;
    if (D == 0) {
        const int blocks = std::max(1, std::min((a.ep.N + kAdjThreads - 1) / kAdjThreads, 4 * qv_num_sms()));
        k_adj_depth0<<<blocks, kAdjThreads, 0, st>>>(a);
        return qv_check_cuda(cudaGetLastError(), "qv_tree_backward launch");
    }
    k_adj_setup<<<1, kAdjThreads, 0, st>>>(a);
    if (qv_check_cuda(cudaGetLastError(), "qv_tree_backward setup") != QV_OK) return QV_ERR_CUDA;
    if (L.recompute) {
        const dim3 grid(L.bands, std::min(L.caps[D - 1], 65535));
        k_adj_recompute<<<grid, kAdjThreads, 0, st>>>(a, D - 1);
        if (qv_check_cuda(cudaGetLastError(), "qv_tree_backward recompute") != QV_OK) return QV_ERR_CUDA;
    }
    const size_t smem = sizeof(double) * static_cast<size_t>(a.band_rows + 2) * a.ep.P;
    if (smem > 48 * 1024 &&
        qv_check_cuda(cudaFuncSetAttribute(k_adj_level, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(smem)),
                      "qv_tree_backward smem") != QV_OK)
        return QV_ERR_CUDA;
    for (int l = D - 1; l >= 0; --l) {
        QV_RANGE("qv_tree_backward", l);
        const dim3 grid(L.bands, std::min(L.caps[l], 65535));
        k_adj_level<<<grid, kAdjThreads, smem, st>>>(a, l);
        if (qv_check_cuda(cudaGetLastError(), "qv_tree_backward level") != QV_OK) return QV_ERR_CUDA;
    }
    k_adj_reduce<<<1, 32, 0, st>>>(a);
    return qv_check_cuda(cudaGetLastError(), "qv_tree_backward reduce");
}

// ---------------------------------------------------------------- value-iteration adjoint host side
namespace {
size_t vib_bytes(int H, int P, int every, int nslots, size_t offs[7]) {
    const size_t N = static_cast<size_t>(H) * P;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        o = qv::a256(o);
        const size_t r = o;
        o += bytes;
        return r;
    };
    offs[0] = take(sizeof(qv::VIWork));
    offs[1] = take(sizeof(double) * N * (every + 1));
    offs[2] = take(N * every);
    offs[3] = take(sizeof(double) * N);
    offs[4] = take(sizeof(double) * N);
    offs[5] = take(sizeof(double) * nslots);
    offs[6] = take(sizeof(unsigned) * nslots);
    return qv::a256(o);
}
constexpr int kViBackMaxGrid = 4096;
}  // namespace

extern "C" size_t mdp_value_backward_workspace_bytes(const qv_model_t *m, int32_t every) {
    if (!m || every < 1 || m->H < 1 || m->pitch < 1) return 0;
    size_t offs[7];
    return vib_bytes(m->H, m->pitch, every, kViBackMaxGrid, offs);
}

extern "C" qv_status mdp_value_backward(const qv_model_t *m, int32_t sweeps, int32_t every, const double *d_Vckpt,
                                        const double *d_Qbar, double *d_dslip, double *d_dcost, void *d_ws,
                                        size_t ws_bytes, qv_stream_t stream) {
    QV_RANGE("mdp_value_backward");
    using namespace qv;
    if (!m || !m->d_cell || !d_Vckpt || !d_Qbar || !d_dslip || !d_ws)
        return qv_set_error(QV_ERR_INVALID, "mdp_value_backward: null pointer");
    if (m->H < 1 || m->W < 1 || m->pitch != QV_PITCH(m->W) || m->W > QV_MAX_WIDTH)
        return qv_set_error(QV_ERR_INVALID, "mdp_value_backward: bad grid");
    if (sweeps < 1 || every < 1)
        return qv_set_error(QV_ERR_INVALID, "mdp_value_backward: sweeps %d every %d", sweeps, every);
    if (reinterpret_cast<uintptr_t>(d_ws) & 255)
        return qv_set_error(QV_ERR_INVALID, "mdp_value_backward: workspace must be 256-byte aligned");
    size_t offs[7];
    const size_t need = vib_bytes(m->H, m->pitch, every, kViBackMaxGrid, offs);
    if (ws_bytes < need)
        return qv_set_error(QV_ERR_WORKSPACE, "mdp_value_backward: workspace %zu < %zu bytes", ws_bytes, need);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(d_ws);
    VIBack a;
    a.H = m->H;
    a.W = m->W;
    a.P = m->pitch;
    a.N = m->H * m->pitch;
    a.cell = m->d_cell;
    a.cost = m->d_cost;
    a.goal = m->goal;
    a.slip = m->slip;
    a.gamma = static_cast<double>(m->discount);
    a.sweeps = sweeps;
    a.every = every;
    a.ckpt = d_Vckpt;
    a.Qbar = d_Qbar;
    a.work = reinterpret_cast<VIWork *>(ws + offs[0]);
    a.segV = reinterpret_cast<double *>(ws + offs[1]);
    a.segA = reinterpret_cast<unsigned char *>(ws + offs[2]);
    a.lam0 = reinterpret_cast<double *>(ws + offs[3]);
    a.lam1 = reinterpret_cast<double *>(ws + offs[4]);
    a.red = reinterpret_cast<double *>(ws + offs[5]);
    a.done = reinterpret_cast<unsigned *>(ws + offs[6]);
    a.spin_limit = qv_cross_spin_limit();
    a.dcost = d_dcost;
    a.dslip = d_dslip;
    int per_sm = 0;
    if (qv_check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_vi_backward, kAdjThreads, 0),
                      "occupancy") != QV_OK)
        return QV_ERR_CUDA;
    if (per_sm < 1) return qv_set_error(QV_ERR_INVALID, "mdp_value_backward: kernel does not fit an SM");
    // bands of whole rows, at least one row and about one CTA's threads of cells each
    int grid = std::min(per_sm * qv_num_sms(), (a.N + kAdjThreads - 1) / kAdjThreads);
    grid = std::max(1, std::min(std::min(grid, kViBackMaxGrid), a.H));
    const int rows_per_cta = (a.H + grid - 1) / grid;
    grid = (a.H + rows_per_cta - 1) / rows_per_cta;
    if (qv_check_cuda(cudaMemsetAsync(a.work, 0, sizeof(VIWork), st), "memset") != QV_OK ||
        qv_check_cuda(cudaMemsetAsync(a.done, 0, sizeof(unsigned) * grid, st), "memset") != QV_OK)
        return QV_ERR_CUDA;
    void *args[] = {&a};
    if (qv_check_cuda(cudaLaunchCooperativeKernel(reinterpret_cast<void *>(k_vi_backward), grid, kAdjThreads, args,
                                                  0, st),
                      "mdp_value_backward launch") != QV_OK)
        return QV_ERR_CUDA;
    VIWork hw;
    if (qv_check_cuda(cudaMemcpyAsync(&hw, a.work, sizeof(hw), cudaMemcpyDeviceToHost, st), "copy") != QV_OK ||
        qv_check_cuda(cudaStreamSynchronize(st), "mdp_value_backward") != QV_OK)
        return QV_ERR_CUDA;
    if (hw.status & kErrTimeout)
        return qv_set_error(QV_ERR_TIMEOUT, "mdp_value_backward: grid barrier wait timed out");
    return QV_OK;
}
