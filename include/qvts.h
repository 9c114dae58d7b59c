/*
 * qvts.h -- C ABI of the GB300 (sm_103a) QV-Tree Search library.
 *
 * The operations follow "Stochastic 2-D Motion Planning with a POMDP
 * Framework" (Sun and Kumar): the model tuple (X, A, Z, T, O, R, b0, gamma) of
 * Sec. II, the Bayes update Phi of Eq. 3, the QMDP leaf bound of Eq. 4, MDP
 * value iteration for the offline Q (Sec. V-B), and the QV-tree expansion and
 * backup of Alg. 2-7.
 *
 * Conventions shared by every call:
 *   - Grids are row-major [H][pitch] with pitch = QV_PITCH(W) = round_up(W, 8)
 *     (rows of FP32 beliefs and of uint16 cell words are then whole 16-byte
 *     units, as the bulk copies need); cell y = row * pitch + col.  Columns
 *     W..pitch-1 are padding (occupied).
 *   - Actions: 0 = N (row - 1), 1 = E (col + 1), 2 = S (row + 1), 3 = W
 *     (col - 1), 4 = stay.  The intended move succeeds w.p. 1 - 2*slip, each
 *     perpendicular move happens w.p. slip; a move into an occupied or outside
 *     cell leaves the mass in place (Eq. 10).  The goal is absorbing.
 *   - Observations z = 0..B: the id of the nearest beacon within the sensing
 *     range (Manhattan distance, ties to the lower id) or B (null); observed
 *     w.p. accuracy, every other value w.p. (1 - accuracy)/B.
 *   - Rewards: arriving in the goal pays +100, any other arrival -1 - c(y)
 *     with c the optional cost map; the goal and occupied cells earn 0.
 *   - Pointers named d_* are device pointers owned by the caller and must stay
 *     valid until the stream work that uses them completes.  h_* / plain
 *     pointers are host memory.  Beliefs and Q are FP32, 16-byte aligned.
 *   - Every call is asynchronous on `stream` unless its comment says it
 *     synchronises.  Calls return a status and never abort; the message of the
 *     last failure on the calling thread is returned by qv_last_error().
 *   - Device scratch comes from a caller-provided workspace (d_ws, ws_bytes);
 *     the matching *_workspace_bytes call gives its size.  The library itself
 *     allocates no device memory in any call declared here.
 *   - Fault injection for tests of the caller's error handling, read from
 *     the environment variable QVTS_FAULT on every call, before any device
 *     work: "timeout" makes every wait on other CTAs give up at once (the
 *     call reports QV_ERR_TIMEOUT and the context stays usable), "oom" makes
 *     mdp_value_iterate, fib_value_iterate, belief_correct and
 *     qv_plan_create report QV_ERR_WORKSPACE (this library's out-of-memory),
 *     "invalid" makes those and belief_predict and qv_plan_run report
 *     QV_ERR_INVALID, and "bounds" (bounds-checked build only, below) makes
 *     the plan's node-record check report a failure on every run although its
 *     indices are in range.  Unset (or any other value): no injection.
 *   - Bounds-checked debug build: libqvts_debug.so, the same ABI compiled with
 *     -DQV_BOUNDS_CHECK.  The plan kernel then checks its workspace indices,
 *     the rows and columns of its bulk copies and its stored-belief offsets
 *     before each access; an index out of range skips the access (no fault)
 *     and the plan's read reports QV_ERR_BOUNDS with the site's name, the
 *     index and the limit.  Release builds compile the checks out.
 *   - Profiling: every call that launches device work opens an NVTX range
 *     "qvts:<call>" for its host-side duration (closed on every return);
 *     calls that issue a tree's levels one launch at a time (the adjoint,
 *     the nine-action plan, the bounds) also open "qvts:<call> level <l>"
 *     per level.  The plan kernel runs every level inside one launch: its
 *     per-level times come from qv_plan_profile's device clock stamps.
 *     Without an NVTX tool attached the ranges cost a pointer test.
 */
#ifndef QVTS_H
#define QVTS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef void *qv_stream_t; /* a cudaStream_t; NULL = the legacy default stream */

typedef enum {
    QV_OK = 0,
    QV_ERR_INVALID = 1,        /* bad argument (size, range, null pointer, alignment) */
    QV_ERR_CUDA = 2,           /* a CUDA runtime call failed                          */
    QV_ERR_WORKSPACE = 3,      /* ws_bytes smaller than the *_workspace_bytes figure  */
    QV_ERR_TIMEOUT = 4,        /* a bounded device-side wait gave up                  */
    QV_ERR_NOT_CONVERGED = 5,  /* value iteration hit max_sweeps before tol           */
    QV_ERR_CAPACITY = 6,       /* a tree level outgrew its preallocated capacity      */
    QV_ERR_BOUNDS = 7          /* a device bounds check failed (debug build only)     */
} qv_status;

#define QV_NUM_ACTIONS 5
#define QV_MAX_DEPTH 6
#define QV_MAX_BEACONS 126
#define QV_MAX_K 64
#define QV_MAX_WIDTH 2048
#define QV_PITCH(W) ((((W) + 7) / 8) * 8)

#define QV_F32 0
#define QV_F64 1
#define QV_WEIGHT_FREQ 0       /* child weight = sample frequency f/K (Alg. 3, Alg. 6)  */
#define QV_WEIGHT_MARGINAL 1   /* child weight = P(z|b,a) / sum over sampled z          */
#define QV_LEAF_FUSED 0        /* leaf values from the parent pass, no leaf beliefs     */
#define QV_LEAF_MATERIALISE 1  /* leaf beliefs written, then streamed against Q         */

/* A built model (Sec. II tuple on one grid).  d_cell comes from
 * qv_model_build; the struct itself is plain host memory. */
typedef struct {
    int32_t H, W, pitch;       /* grid size; pitch = QV_PITCH(W)                        */
    const uint16_t *d_cell;    /* [H][pitch] cell words written by qv_model_build       */
    int32_t num_beacons;       /* B in 1..QV_MAX_BEACONS; |Z| = B + 1                   */
    int32_t goal;              /* goal cell, row * pitch + col, must be free            */
    float slip;                /* epsilon in [0, 0.5]                                   */
    float accuracy;            /* alpha in (0, 1]                                       */
    float discount;            /* gamma in (0, 1)                                       */
    const float *d_cost;       /* nullable [H][pitch] per-cell cost c(y)                */
    const int32_t *d_beacons;  /* [B] beacon cells as given to qv_model_build; the tree
                                  search walks each beacon's sensing diamond           */
    int32_t sense_range;       /* Manhattan sensing range given to qv_model_build       */
} qv_model_t;

/* Tree-search parameters (Alg. 1-3 with the level-synchronous reading). */
typedef struct {
    int32_t depth;             /* d in 0..QV_MAX_DEPTH                                  */
    int32_t K;                 /* forward samples per (V-node, action), 1..QV_MAX_K     */
    uint64_t seed;             /* Philox4x32-10 key                                     */
    uint32_t episode;          /* Philox counter word 1                                 */
    int32_t weight_mode;       /* QV_WEIGHT_FREQ or QV_WEIGHT_MARGINAL                  */
    int32_t leaf_mode;         /* QV_LEAF_FUSED or QV_LEAF_MATERIALISE                  */
    const int32_t *d_replay;   /* nullable: observation samples to use instead of
                                  Philox draws, laid out like the samples array of
                                  qv_plan_level (per level, [node][action][K])         */
    int32_t band_cells;        /* cells per work item (a band of whole rows), 0 = the
                                  autotuner's choice for this shape, else 2048         */
    int32_t items_per_cta;     /* work items aimed at per co-resident CTA in a phase,
                                  0 = the autotuner's choice for this shape, else 2    */
    int32_t grid_ctas;         /* CTAs of the plan's launch, 0 = every CTA that can be
                                  co-resident; fewer leave room for plans launched
                                  concurrently on other streams (a latency-bound plan
                                  barely slows, the GPU runs several at once)         */
    double deadline_ms;        /* anytime stop (Sec. IV-C; Alg. 1 plans "while time
                                  permits"): 0 = none; > 0 = a budget from the start of
                                  the plan's kernel, checked each time a level is
                                  final: once it has run out, that level's children
                                  become the leaves (values by Eq. 4) and the backup
                                  returns the best root action of the levels built so
                                  far (depth_reached of the result; level 0 is always
                                  built).  Needs QV_LEAF_FUSED; every level then also
                                  sums its children's leaf values                     */
    int32_t deepest_form;      /* how the deepest level of a fused plan (depth >= 2)
                                  forms its children's sums: QV_DEEPEST_AUTO (0) the
                                  contraction of every child's belief with planes of
                                  the motion model applied to the weights, where its
                                  records fit the workspace; QV_DEEPEST_STENCIL (1)
                                  each child's five-action stencil.  Both compute the
                                  same sums of Eq. 3 and Alg. 5 (in another FP32
                                  order); other values return QV_ERR_INVALID          */
} qv_plan_params_t;
#define QV_DEEPEST_AUTO 0
#define QV_DEEPEST_STENCIL 1

typedef struct {
    int32_t action;            /* argmax_a U_Q(b0, a); ties to the lower index          */
    float value;               /* U_V(b0)                                               */
    float q[QV_NUM_ACTIONS];   /* U_Q(b0, a)                                            */
    int32_t nodes_per_level[QV_MAX_DEPTH + 1];
    int64_t boundary_samples;  /* draws whose uniform fell within 1e-6 of a CDF step    */
    int32_t depth_reached;     /* depth of the tree the result comes from: the plan's
                                  depth, or less when its deadline ran out            */
} qv_plan_result_t;

const char *qv_last_error(void);
const char *qv_version(void);

/* ---------------------------------------------------------------- model (Sec. II)
 * Builds the cell words of one grid: for every cell, which of its four
 * neighbours are blocked (occupied or outside; Eq. 10), which neighbours may
 * move mass into it, its observation label, and whether it is free.
 *   d_occ     [H][pitch] uint8, 1 = occupied (padding columns are ignored)
 *   d_beacons [B] int32 beacon cells (row * pitch + col), free and distinct
 *   d_cell    [H][pitch] uint16 output
 * Errors: QV_ERR_INVALID for sizes outside the QV_MAX_* limits. */
qv_status qv_model_build(int32_t H, int32_t W, int32_t pitch, const uint8_t *d_occ,
                         const int32_t *d_beacons, int32_t B, int32_t sense_range,
                         int32_t goal, uint16_t *d_cell, qv_stream_t stream);

/* ---------------------------------------------------------------- value iteration
 * MDP value iteration for the offline alpha-vectors Q (Sec. V-B baseline;
 * Bellman operator of Eq. 2 on a known state; contraction as in Sec. IV-A):
 *   V_{k+1}(x) = max_a [R(x, a) + gamma sum_y T(x, a, y) V_k(y)], V_0 = 0,
 * Jacobi sweeps, V(goal) = 0.  Stops at the first sweep with
 * max_x |V_{k+1} - V_k| < tol, or after exactly `truncated` sweeps when
 * truncated > 0.  Writes V (dtype QV_F32 or QV_F64, [H][pitch]) and
 * Q[a][y] = R(y, a) + gamma sum T V_final as FP32 [5][H][pitch].
 * Synchronises the stream (sweeps and residual are returned to the host).
 * Returns QV_ERR_NOT_CONVERGED when max_sweeps ran out first. */
size_t mdp_value_iterate_workspace_bytes(const qv_model_t *model, int32_t dtype);
qv_status mdp_value_iterate(const qv_model_t *model, int32_t dtype, double tol,
                            int32_t max_sweeps, int32_t truncated, void *d_V, float *d_Q,
                            void *d_ws, size_t ws_bytes, int32_t *sweeps_out,
                            double *residual_out, qv_stream_t stream);

/* mdp_value_iterate_checkpointed: exactly `sweeps` FP64 Jacobi sweeps of the
 * same operator from V_0 = 0 (d_V is zeroed first), for the adjoint below.
 * Also stores V_k for k = 0, every, 2*every, ... < sweeps into d_Vckpt
 * ([ceil(sweeps / every)][H][pitch] FP64).  Writes V_sweeps to d_V and Q
 * (FP32) as mdp_value_iterate does.  Workspace:
 * mdp_value_iterate_workspace_bytes(model, QV_F64).  Synchronises. */
qv_status mdp_value_iterate_checkpointed(const qv_model_t *model, int32_t sweeps, int32_t every,
                                         double *d_V, float *d_Q, double *d_Vckpt,
                                         void *d_ws, size_t ws_bytes, qv_stream_t stream);

/* mdp_value_backward: reverse mode of mdp_value_iterate_checkpointed (the
 * derivatives of Eq. 2's Bellman sweeps and of Eq. 10's transition model).
 * Given d_Qbar = dL/dQ[a][y] (FP64 [5][H][pitch]), accumulates (+=)
 *   *d_dslip       dL/d slip   (device FP64 scalar),
 *   d_dcost[y]     dL/d c(y)   (FP64 [H][pitch], nullable),
 * through Q = R + gamma T V_sweeps, every sweep V_{k+1} = max_a [R + gamma T
 * V_k] with its argmax held fixed (ties to the lowest action index, as the
 * forward takes them), and R(x, a) = sum_y T(x, a, y) r(y), r(y) = -1 - c(y)
 * off the goal.  The sweeps are recomputed segment by segment from the
 * checkpoints of the forward call (same model, sweeps and every), so memory
 * holds `every` sweeps at a time.  One persistent cooperative launch with a
 * bounded grid barrier; QV_ERR_TIMEOUT if a wait gives up.  Synchronises. */
size_t mdp_value_backward_workspace_bytes(const qv_model_t *model, int32_t every);
qv_status mdp_value_backward(const qv_model_t *model, int32_t sweeps, int32_t every,
                             const double *d_Vckpt, const double *d_Qbar, double *d_dslip,
                             double *d_dcost, void *d_ws, size_t ws_bytes, qv_stream_t stream);

/* ---------------------------------------------------------------- FIB bound (Sec. IV-A)
 * fib_value_iterate: the Fast Informed Bound alpha-vectors, one per action,
 * by Jacobi sweeps of Eq. 7 from alpha_0 = 0:
 *   alpha^a(x) = R(x, a) + gamma sum_z max_a' sum_x' O(x', z) T(x, a, x') alpha^a'(x'),
 * with the same T, O and R as the rest of the library and alpha = 0 on the
 * goal and on occupied cells.  Stops at the first sweep with
 * max_{a,x} |alpha_{k+1} - alpha_k| < tol, or after exactly `truncated`
 * sweeps when truncated > 0.  Outputs:
 *   d_alpha  [5][H][pitch] in `dtype` (QV_F32 or QV_F64), nullable, 16-byte aligned
 *   d_Q      [5][H][pitch] FP32 copy, the layout the tree search takes as its
 *            leaf alpha-vectors: with it the leaf value max_a sum_x b(x) Q is
 *            V_FIB(b) of Eq. 6, the upper bound U_V of Alg. 5.
 * Synchronises the stream.  Returns QV_ERR_NOT_CONVERGED when max_sweeps ran
 * out first, QV_ERR_INVALID for a pitch too wide to stage three rows of the
 * five planes in shared memory (FP64 above pitch 1928; FP32 fits every
 * width), QV_ERR_TIMEOUT when a wait on another CTA gave up. */
size_t fib_value_iterate_workspace_bytes(const qv_model_t *model, int32_t dtype);
qv_status fib_value_iterate(const qv_model_t *model, int32_t dtype, double tol,
                            int32_t max_sweeps, int32_t truncated, void *d_alpha, float *d_Q,
                            void *d_ws, size_t ws_bytes, int32_t *sweeps_out,
                            double *residual_out, qv_stream_t stream);

/* ---------------------------------------------------------------- PBVI bound (Sec. IV-B)
 * Point-based value iteration: alpha-vectors, one per point of a belief set,
 * backed up with Eq. 8 at the points; V_PBVI(b) = max_alpha alpha . b is a
 * lower bound of the optimal value (the L_V of Alg. 5) when the vectors start
 * from qv_pbvi_init.  Every belief and alpha-vector is FP32 [H][pitch] (sets
 * of them [count][H][pitch]); every alpha-vector is 0 on the goal and on
 * occupied cells.
 *
 * qv_pbvi_init: alpha_0 = R_min / (1 - gamma) on free, non-goal cells, with
 * R_min the least R(x, a) there (a lower bound on every policy's value).
 *
 * qv_pbvi_expand: one round of belief set expansion (Sec. IV-B): from point
 * j of d_B, an action a = floor(5 u_a) and an observation z drawn from
 * P(z | b_j, a) by the inverse CDF (FP32, ascending z, as the tree search
 * draws), giving d_out[j] = tau(b_j, a, z) (Eq. 3).  u_a and u_z are words 0
 * and 1 of the Philox4x32-10 stream with key `seed` and counter
 * {0, round, j, 255 << 24} (the tree's counter layout with level code 255).
 * d_action, d_obs, d_boundary [nB] record a, z and whether u_z lay within
 * 1e-6 of a CDF step.  One CTA per point.
 *
 * qv_pbvi_create builds a handle for one model (reads its cell words back,
 * so it synchronises): the live cells (free, not the goal) ordered label by
 * label for the contraction of Eq. 8.  The handle keeps host tables only;
 * device state lives in the caller's workspace of qv_pbvi_workspace_bytes,
 * which the later calls take from qv_pbvi_set_points.
 * qv_pbvi_set_points: the belief set (1..max_points points, d_B is read
 * during this call only): its five predicted beliefs per point and R(b, a).
 * The score contraction of Eq. 8 and of V_PBVI runs on the tensor cores
 * (tcgen05, TF32 operands split into head and tail, FP32 accumulation).
 * qv_pbvi_backup: one Eq. 8 backup of every point of the set given nG
 * vectors d_G (nG <= max_points); writes one new vector per point to d_Gout
 * (must not overlap d_G), and, where not NULL, the backed-up value at the
 * point d_value [nB] (= d_Gout[b] . b), the chosen action d_astar [nB]
 * (argmax of Q_b(a), exact ties to the lowest), the winning vector of each
 * observation for that action d_best [nB][B + 1] (exact ties to the lowest
 * index), d_q [nB][5] every Q_b(a).
 * qv_pbvi_value: V_PBVI(b) and its maximising vector (ties to the lowest
 * index) for nb beliefs d_b given nG <= max_points vectors d_G (the beliefs
 * go through in chunks of max_points).  d_G = NULL reuses the vectors of the
 * previous qv_pbvi_value call (same nG) unless a backup has run since
 * (QV_ERR_INVALID then): a caller asking about many beliefs against fixed
 * vectors skips their reordering.
 * The host may upload small tables (pageable copies) on the stream; none of
 * these calls synchronises except qv_pbvi_create. */
typedef struct qv_pbvi qv_pbvi_t;
qv_status qv_pbvi_init(const qv_model_t *model, float *d_alpha0, qv_stream_t stream);
qv_status qv_pbvi_expand(const qv_model_t *model, const float *d_B, int32_t nB, int32_t round,
                         uint64_t seed, float *d_out, int32_t *d_action, int32_t *d_obs,
                         int32_t *d_boundary, qv_stream_t stream);
qv_status qv_pbvi_create(const qv_model_t *model, int32_t max_points, qv_pbvi_t **out);
size_t qv_pbvi_workspace_bytes(const qv_pbvi_t *pbvi);
/* Length of the label-ordered cell axis (each label's run padded to a
 * multiple of 16); seg_out (nullable, B + 2 entries) gets the runs' starts. */
int32_t qv_pbvi_layout(const qv_pbvi_t *pbvi, int32_t *seg_out);
qv_status qv_pbvi_set_points(qv_pbvi_t *pbvi, const float *d_B, int32_t nB, void *d_ws,
                             size_t ws_bytes, qv_stream_t stream);
qv_status qv_pbvi_backup(qv_pbvi_t *pbvi, const float *d_G, int32_t nG, float *d_Gout,
                         float *d_value, int32_t *d_astar, int32_t *d_best, float *d_q,
                         qv_stream_t stream);
/* qv_pbvi_backup_fixed: qv_pbvi_backup with some of Eq. 8's decisions
 * fixed by the caller (device arrays, nullable): a* of point b is
 * d_fix_astar[b] when that is >= 0, and the winning vector of observation
 * z for that a* is d_fix_best[b][z] (B + 1 per point) when that is >= 0;
 * the fixed winner's own score enters Q_b(a*).  Entries < 0 leave the
 * decision to the argmax.  Used to replay another implementation's choices
 * at near-ties (d_fix_best needs d_fix_astar; QV_ERR_INVALID otherwise). */
qv_status qv_pbvi_backup_fixed(qv_pbvi_t *pbvi, const float *d_G, int32_t nG, float *d_Gout,
                               float *d_value, int32_t *d_astar, int32_t *d_best, float *d_q,
                               const int32_t *d_fix_astar, const int32_t *d_fix_best,
                               qv_stream_t stream);
qv_status qv_pbvi_value(qv_pbvi_t *pbvi, const float *d_G, int32_t nG, const float *d_b,
                        int32_t nb, float *d_value, int32_t *d_arg, qv_stream_t stream);
/* qv_pbvi_check: synchronises; QV_ERR_TIMEOUT (once) if a bounded wait of
 * the tensor-core contraction gave up since the last check, else QV_OK. */
qv_status qv_pbvi_check(qv_pbvi_t *pbvi, qv_stream_t stream);
void qv_pbvi_destroy(qv_pbvi_t *pbvi);

/* ---------------------------------------------------------------- belief update (Eq. 3)
 * belief_predict: bbar(y) = sum_x T(x, action, y) b(x), the numerator of
 * Eq. 3.  Values stored on occupied cells of b are read as 0. */
qv_status belief_predict(const qv_model_t *model, const float *d_b, int32_t action,
                         float *d_bbar, qv_stream_t stream);

/* belief_correct: b'(y) = O(y, z) bbar(y) / P(z), P(z) = sum_y O(y, z) bbar(y)
 * (Eq. 3); writes P(z) to the device scalar d_pz.  d_bbar and d_bout are
 * 16-byte aligned (QV_ERR_INVALID otherwise). */
size_t belief_correct_workspace_bytes(const qv_model_t *model);
qv_status belief_correct(const qv_model_t *model, const float *d_bbar, int32_t z,
                         float *d_bout, float *d_pz, void *d_ws, size_t ws_bytes,
                         qv_stream_t stream);

/* belief_correct_noalloc: the same result as belief_correct, for callers that
 * cannot allocate device memory -- for example a control loop that must not
 * call cudaMalloc after start-up (an allocation can synchronise the device
 * and stall the loop), or a host application that owns every device
 * allocation and forbids libraries to make their own.  The paper has no
 * counterpart.
 *   - Takes no workspace: the reduction's scratch is a fixed array compiled
 *     into the library (about 16 KB, resident on every device that loads
 *     the library until the process exits).  Nothing is allocated.
 *   - Grids are limited to QV_NOALLOC_MAX_CELLS cells (H * pitch); larger
 *     ones return QV_ERR_INVALID with a message.
 *   - The first call on a device looks up the array's device address (with
 *     that device current); make that first call before any stream capture.
 *     The address is kept for the life of the process and is valid only
 *     while the device's context lives: after cudaDeviceReset (or any loss
 *     of the primary context) the next call may use a stale address.  A
 *     call that fails with a CUDA error forgets the address, so the call
 *     after it looks it up again.
 *   - Every call on a device shares the one array: calls whose GPU work
 *     overlaps (other streams, other threads) race and must be serialised by
 *     the caller.  Each call clears the part that must start at zero. */
#define QV_NOALLOC_MAX_CELLS (4096 * 1024)
qv_status belief_correct_noalloc(const qv_model_t *model, const float *d_bbar, int32_t z,
                                 float *d_bout, float *d_pz, qv_stream_t stream);

/* leaf_value: v[i] = max_a sum_y b_i(y) Q[a][y] for n beliefs stored at
 * d_b + i * H * pitch (Eq. 4 with the QMDP alpha-vectors; Alg. 5). */
qv_status leaf_value(const qv_model_t *model, const float *d_Q, const float *d_b,
                     int32_t n, float *d_value, qv_stream_t stream);

/* ---------------------------------------------------------------- tree search (Alg. 1-7)
 * A plan holds the layout of one batch of E episodes (E = 1 for a single
 * tree) inside a caller workspace.  Every episode shares `params` except the
 * Philox episode word, which is params->episode + e.  qv_plan_create uploads
 * the episode descriptors (a synchronous host-to-device copy); qv_plan_run
 * launches the whole search (no host synchronisation, no allocation; it may be
 * captured in a CUDA graph); qv_plan_read copies the E results to the host and
 * synchronises.  The workspace stays the plan's until qv_plan_destroy.  */
typedef struct qv_plan qv_plan_t;

size_t qv_plan_workspace_bytes(int32_t E, const qv_model_t *models,
                               const qv_plan_params_t *params);
qv_status qv_plan_create(int32_t E, const qv_model_t *models, const float *const *d_Q,
                         const float *const *d_b0, const qv_plan_params_t *params,
                         void *d_ws, size_t ws_bytes, qv_plan_t **plan_out,
                         qv_stream_t stream);
qv_status qv_plan_run(qv_plan_t *plan, qv_stream_t stream);
/* qv_plan_set_episode_word: take the Philox episode word of the plan's
 * draws (counter word 1, Alg. 3) from a caller-owned device uint32 read at
 * every run: episode e of the batch draws with *d_word + e instead of
 * params.episode + e.  A closed loop (Alg. 1's outer loop) then re-runs one
 * plan step after step, writing the step's word on its stream, instead of
 * creating a plan per step.  NULL returns to params.episode.  Drops a
 * captured graph (capture again after this call). */
qv_status qv_plan_set_episode_word(qv_plan_t *plan, const uint32_t *d_word);
/* Capture the launches of qv_plan_run in a CUDA graph owned by the plan;
 * later qv_plan_run calls launch the graph. */
qv_status qv_plan_capture_graph(qv_plan_t *plan, qv_stream_t stream);
qv_status qv_plan_read(qv_plan_t *plan, qv_plan_result_t *h_results, qv_stream_t stream);
/* The same read in two steps, so that many plans' results come back with one
 * synchronisation: qv_plan_read_async enqueues the copy of the plan's
 * qv_plan_readback_bytes result bytes into h_buf (pinned host memory for the
 * copy to be asynchronous); once the stream has passed it, qv_plan_decode
 * turns them into the E results and the run's status, as qv_plan_read does. */
size_t qv_plan_readback_bytes(const qv_plan_t *plan);
qv_status qv_plan_read_async(const qv_plan_t *plan, void *h_buf, qv_stream_t stream);
qv_status qv_plan_decode(qv_plan_t *plan, const void *h_buf, qv_plan_result_t *h_results);

/* Run the plan once without the graph, with a CUDA event recorded on
 * `stream` before the first launch and after every launch; returns for each
 * launch its kernel name, tree level and duration (ms).  Synchronises. */
typedef struct {
    char name[32];
    int32_t level;
    float ms;
} qv_launch_time_t;
qv_status qv_plan_profile(qv_plan_t *plan, qv_launch_time_t *h_out, int32_t max_launches,
                          int32_t *n_out, qv_stream_t stream);
void qv_plan_destroy(qv_plan_t *plan);

/* ---------------------------------------------------------------- autotuner
 * The plan kernel's two launch-shape knobs: the band of rows one work item
 * covers (band_cells, the tile) and the work items a phase aims at per
 * co-resident CTA (items_per_cta, nodes per CTA).  qv_plan_autotune times
 * every candidate pair on the caller's inputs (each a full plan run,
 * `reps` timed runs after two warm-up runs, CUDA events on `stream`), keeps
 * the fastest in a process-wide cache under the inputs' shape class (E,
 * depth, K, leaf and weight modes, largest B, the power-of-two classes of
 * the widest pitch and the mean cell count, and grid_ctas) and returns it.  Plans created
 * later with band_cells = 0 / items_per_cta = 0 and the same shape class
 * take the cached pair.  Candidates whose shared memory does not fit are
 * skipped.  The workspace must hold qv_plan_autotune_workspace_bytes.
 * Synchronises; not capturable.  Results of a tuned plan equal the default
 * plan's up to FP32 summation order. */
typedef struct {
    int32_t band_cells;
    int32_t items_per_cta;
    float ms;                  /* mean time of one plan run                           */
} qv_tune_t;
size_t qv_plan_autotune_workspace_bytes(int32_t E, const qv_model_t *models,
                                        const qv_plan_params_t *params);
qv_status qv_plan_autotune(int32_t E, const qv_model_t *models, const float *const *d_Q,
                           const float *const *d_b0, const qv_plan_params_t *params,
                           void *d_ws, size_t ws_bytes, int32_t reps, qv_tune_t *h_best,
                           qv_tune_t *h_all, int32_t max_all, int32_t *n_all,
                           qv_stream_t stream);
/* The knobs a plan was created with. */
qv_status qv_plan_tuning(const qv_plan_t *plan, qv_tune_t *h_out);
/* CTAs of the plan's launch (grid_ctas, or every co-resident CTA). */
int32_t qv_plan_grid(const qv_plan_t *plan);
/* Forget every cached choice. */
void qv_tune_clear(void);

/* Device views of one level of episode e after a run (for inspection and
 * tests).  Level l nodes are ordered by (parent, action, z ascending).
 * Arrays with a NULL out-pointer are skipped.  Per-node arrays have
 * capacity cap; per-(node, action) arrays are [cap][5]; samples [cap][5][K].
 * belief is NULL for levels that hold no beliefs (fused leaves).  In the
 * fused mode the leaves' per-node records are written on demand: asking for
 * the leaf level synchronises the device, writes them (one small launch)
 * and synchronises again. */
typedef struct {
    int32_t cap;               /* capacity of the level (worst case)                   */
    const int32_t *d_count;    /* device scalar: nodes in the level                    */
    const int32_t *d_parent;   /* parent index in level l-1                            */
    const int32_t *d_action;   /* action from the parent                               */
    const int32_t *d_obs;      /* observation z from the parent                        */
    const float *d_weight;     /* child weight (FREQ or MARGINAL)                      */
    const float *d_pz;         /* P(z | parent belief, action)                         */
    const float *d_value;      /* U_V                                                  */
    const float *d_R;          /* [cap][5] R(b, a)                                     */
    const float *d_UQ;         /* [cap][5] U_Q(b, a)                                   */
    const int32_t *d_nchild;   /* [cap][5] unique children per action                  */
    const int32_t *d_samples;  /* [cap][5][K] raw sampled z                            */
    const float *d_belief;     /* [cap][H][pitch] or NULL                              */
    const int32_t *d_leaf_arg; /* leaves: argmax a' of sum_y b(y) Q(a', y), else NULL  */
} qv_level_view_t;
qv_status qv_plan_level(const qv_plan_t *plan, int32_t e, int32_t level, qv_level_view_t *view);

/* ---------------------------------------------------------------- AEMS fields (Alg. 5-7, Eq. 9)
 * qv_plan_bounds: the lower bound L, heuristic H and V-node to expand E of
 * every node of episode e of a plan that has run, bottom-up from the lower
 * bound of every leaf, d_leaf_L [leaves] (for example V_PBVI of the leaf
 * beliefs from qv_pbvi_value; the leaf level's order is qv_plan_level's):
 *   leaf     L_V = d_leaf_L, H_V = U_V - L_V, E_V = its own index
 *   Q-node   L_Q = R(b, a) + gamma sum_children w L_V; the child maximising
 *            gamma w H_V (ties: first in (parent, action, z) order) gives
 *            H_Q = gamma w H_V and E_Q = its E_V; no children: L_Q = R,
 *            H_Q = 0, E_Q = -1
 *   V-node   L_V = max_a L_Q; H_V, E_V = H_Q, E_Q of the action maximising
 *            U_Q (H(b, a) of Eq. 9; ties to the lowest)
 * E values index the leaf level.  The root's E is the V-node the paper's
 * search would expand next.  Results live in the caller's workspace of
 * qv_plan_bounds_workspace_bytes (256-byte aligned); qv_plan_bounds_view
 * gives level l's arrays ([cap] per node, [cap][5] per Q-node, Q arrays NULL
 * at the leaf level).  Asynchronous, except that a fused-mode plan's leaf
 * records are written first (qv_plan_level's synchronisation). */
typedef struct {
    float *d_LV;
    float *d_HV;
    int32_t *d_EV;
    float *d_LQ;
    float *d_HQ;
    int32_t *d_EQ;
} qv_bounds_view_t;
size_t qv_plan_bounds_workspace_bytes(const qv_plan_t *plan, int32_t e);
qv_status qv_plan_bounds(const qv_plan_t *plan, int32_t e, const float *d_leaf_L, void *d_ws,
                         size_t ws_bytes, qv_stream_t stream);
qv_status qv_plan_bounds_view(const qv_plan_t *plan, int32_t e, int32_t level, void *d_ws,
                              qv_bounds_view_t *view);

/* ---------------------------------------------------------------- best-first search (Alg. 1)
 * The planning loop of Alg. 1: each iteration expands the V-node the root's
 * E points at (Alg. 2-5: every action, K forward samples, the unique
 * observations with frequencies f, children tau(b, a, z) of weight f / K,
 * U = max_a sum b Qu (d_Qu: upper-bound alpha-vectors, FP32 [5][H][pitch],
 * e.g. fib_value_iterate's), L = V_PBVI (qv_pbvi_value with the nG vectors
 * d_G, whose handle must have a workspace), H = U - L, E = the child) and
 * updates it and its ancestors (Alg. 6-7 with H(b, a) of Eq. 9).  A node
 * created at max_depth is closed (H = 0).  The samples of (V-node, a) are
 * the level-synchronous tree's: level = the node's depth, path = its
 * mixed-radix code * 5 + a, so every node is the node of the same path in
 * that tree.  Node ids follow creation order (action, then z ascending).
 * Planning stops (later iterations do nothing) when the node to expand lies
 * at max_depth or the next expansion could overflow max_nodes.
 *   qv_bf_create   checks sizes (max_depth 0..8, (5 |Z|)^max_depth < 2^56)
 *   qv_bf_reset    the root from d_b0 in the caller's workspace (256-byte
 *                  aligned, qv_bf_workspace_bytes; one belief per node)
 *   qv_bf_run      `iters` iterations, launches only (no host waits)
 *   qv_bf_read     synchronises; root fields, iterations, nodes, stop flag
 *   qv_bf_view     device arrays of the tree (per node; per Q-node [n][5];
 *                  expanded [max_nodes]: the node of each iteration, -1 after) */
typedef struct qv_bf qv_bf_t;
typedef struct {
    int32_t iterations;        /* expansions done                                     */
    int32_t nodes;             /* V-nodes in the tree                                 */
    int32_t stopped;           /* 1 once planning stopped                             */
    int32_t root_action;       /* argmax_a U_Q(root, a), ties to the lowest; -1 unexpanded */
    float U, L, H;             /* the root's fields                                   */
    int32_t E;                 /* the V-node the next iteration expands               */
    float q[QV_NUM_ACTIONS];   /* U_Q(root, a)                                        */
    int64_t boundary_samples;  /* draws whose uniform fell within 1e-6 of a CDF step  */
} qv_bf_result_t;
typedef struct {
    int32_t max_nodes;
    const int32_t *d_parent, *d_action, *d_obs, *d_depth;
    const float *d_weight, *d_U, *d_L, *d_H;
    const int32_t *d_E;
    const float *d_R, *d_UQ, *d_LQ, *d_HQ;
    const int32_t *d_EQ, *d_first, *d_count;
    const float *d_belief;
    const int32_t *d_expanded;
} qv_bf_view_t;
qv_status qv_bf_create(const qv_model_t *model, const float *d_Qu, qv_pbvi_t *pbvi, const float *d_G,
                       int32_t nG, int32_t K, uint64_t seed, uint32_t episode, int32_t max_depth,
                       int32_t max_nodes, qv_bf_t **out);
size_t qv_bf_workspace_bytes(const qv_bf_t *bf);
qv_status qv_bf_reset(qv_bf_t *bf, const float *d_b0, void *d_ws, size_t ws_bytes, qv_stream_t stream);
qv_status qv_bf_run(qv_bf_t *bf, int32_t iters, qv_stream_t stream);
/* qv_bf_set_replay: fix the node expanded at some iterations: at iteration
 * t < n (counted from the last qv_bf_reset) with d_expand[t] >= 0 the loop
 * expands node d_expand[t] (an id below the node count, else the root's E)
 * instead of the root's E, to replay another implementation's choices
 * where Eq. 9's comparisons are near-ties.  d_expand is a device array the
 * caller keeps alive while runs use it; n = 0 clears the replay. */
qv_status qv_bf_set_replay(qv_bf_t *bf, const int32_t *d_expand, int32_t n);
qv_status qv_bf_read(qv_bf_t *bf, qv_bf_result_t *h_result, qv_stream_t stream);
qv_status qv_bf_view(const qv_bf_t *bf, qv_bf_view_t *view);
void qv_bf_destroy(qv_bf_t *bf);

/* ---------------------------------------------------------------- closed-loop episodes (Alg. 1)
 * The outer loop of Alg. 1 for E episodes on one map: plan (a batched plan
 * whose episode e plans from belief e), execute, measure, update.
 * qv_plan_actions_device: the device address of episode 0's root action in
 * a plan's results; episode e's is at e * *stride (int32 units).
 * qv_env_step: the true system's step of every episode not yet at the goal
 * (d_done[e] == 0): action a = d_action[e * action_stride] from state
 * d_state[e] (a cell, row * pitch + col), the motion outcome drawn with u_m
 * and the measurement at the new cell with u_o, words 0 and 1 of the Philox
 * stream {0, e, step, 254 << 24} (key seed): the intended move if
 * u_m < 1 - 2 eps, the first perpendicular (a + 1) if u_m < 1 - eps, else
 * the second (a + 3), FP32 comparisons, a blocked move staying (Eq. 10); z
 * by the FP32 inverse CDF of O(x', .) in ascending z.  Updates d_state,
 * d_obs (-1 for finished episodes), d_steps (+1), d_return (+= gamma^step
 * r(x'), Eq. 1), d_done (1 at the goal).
 * qv_belief_update_batched: b_e <- tau(b_e, a_e, z_e) (Eq. 3) in place for
 * every episode with d_obs[e] >= 0; d_B [E][H][pitch].  Workspace:
 * qv_belief_update_batched_workspace_bytes (256-byte aligned). */
const int32_t *qv_plan_actions_device(const qv_plan_t *plan, int32_t *stride);
qv_status qv_env_step(const qv_model_t *model, int32_t E, const int32_t *d_action,
                      int32_t action_stride, int32_t *d_state, uint64_t seed, int32_t step,
                      int32_t *d_obs, int32_t *d_steps, float *d_return, int32_t *d_done,
                      qv_stream_t stream);
size_t qv_belief_update_batched_workspace_bytes(const qv_model_t *model, int32_t E);
qv_status qv_belief_update_batched(const qv_model_t *model, int32_t E, float *d_B,
                                   const int32_t *d_action, int32_t action_stride,
                                   const int32_t *d_obs, void *d_ws, size_t ws_bytes,
                                   qv_stream_t stream);

/* ---------------------------------------------------------------- ancestral sampler (Alg. 4)
 * qv_forward_sample: K measurement samples for each of n (belief, action)
 * pairs by Alg. 4 as written, one thread per sample: x ~ b (the inverse CDF
 * of b over the cells in index order, FP32 prefix sums), x' ~ T(x, a, .)
 * and z ~ O(x', .) by qv_env_step's rules.  Sample k of pair j uses words
 * 3k, 3k + 1, 3k + 2 of the Philox stream {.., episode, d_path[j], level}.
 * The tree search draws z from the exact marginal P(z | b, a) instead (one
 * inverse CDF over z); both have the same law.  d_B [n][H][pitch],
 * d_action [n], d_path [n], d_z [n][K]; workspace
 * qv_forward_sample_workspace_bytes (the prefix sums); d_B and the
 * workspace 16-byte aligned (QV_ERR_INVALID otherwise). */
size_t qv_forward_sample_workspace_bytes(const qv_model_t *model, int32_t n);
qv_status qv_forward_sample(const qv_model_t *model, int32_t n, const float *d_B,
                            const int32_t *d_action, const uint64_t *d_path, int32_t level,
                            uint64_t seed, uint32_t episode, int32_t K, int32_t *d_z, void *d_ws,
                            size_t ws_bytes, qv_stream_t stream);

/* ---------------------------------------------------------------- adjoint of the plan
 * qv_tree_backward: reverse mode of the root value U_V(b0) of episode e of a
 * plan that has run (stream order), by the derivatives of Alg. 6 and 7
 * (backup), Eq. 4 (leaf values), Eq. 3 (prediction, correction and its
 * normalisation) and R(b, a).  Held fixed: the sampled measurements, the
 * FREQ weights f/K, and every max (Alg. 7 over actions, Eq. 4 over a leaf's
 * alpha-vectors; ties to the lowest index).  MARGINAL weights depend on the
 * parameters and are refused (QV_ERR_INVALID).  With seed adjoint dL_dV,
 * accumulates (+=) into FP64 device buffers:
 *   d_Qbar   [5][H][pitch]  dL/dQ (feed to mdp_value_backward)
 *   d_dslip  scalar         dL/d slip through every T_a in the tree
 *   d_dacc   scalar         dL/d accuracy through every O(., z)
 *   d_dcost  [H][pitch]     dL/d c(y) through every R(b, a)   (nullable)
 *   d_db0    [H][pitch]     dL/d b0(y)                        (nullable)
 * Only the V-nodes on the chosen actions carry a nonzero adjoint; their
 * beliefs come from the plan (the deepest internal level of the fused mode
 * is recomputed from its parents).  Asynchronous, allocation-free and
 * capturable; the workspace is the caller's (contents need no clearing).
 * Contributions to d_Qbar and d_dcost are summed with FP64 atomics. */
size_t qv_tree_backward_workspace_bytes(const qv_plan_t *plan, int32_t e);
qv_status qv_tree_backward(const qv_plan_t *plan, int32_t e, double dL_dV, double *d_Qbar,
                           double *d_dslip, double *d_dacc, double *d_dcost, double *d_db0,
                           void *d_ws, size_t ws_bytes, qv_stream_t stream);

/* One plan from b0 to the chosen action: create + run + read + destroy.
 * Synchronises the stream. */
qv_status qv_tree_plan(const qv_model_t *model, const float *d_Q, const float *d_b0,
                       const qv_plan_params_t *params, void *d_ws, size_t ws_bytes,
                       qv_plan_result_t *h_result, qv_stream_t stream);

/* E independent episodes on grids of uneven size, every level of every
 * episode in one launch per kernel.  Synchronises the stream. */
qv_status qv_tree_plan_batched(int32_t E, const qv_model_t *models, const float *const *d_Q,
                               const float *const *d_b0, const qv_plan_params_t *params,
                               void *d_ws, size_t ws_bytes, qv_plan_result_t *h_results,
                               qv_stream_t stream);

/* ------------------------------------------------------------------------
 * The paper's experimental model (Sec. V), a second model family beside the
 * beacon model above:
 *   - Grids are unpadded row-major [H][W], cell y = row * W + col.
 *   - Nine actions a = 0..8 move to the neighbour N_a(x) at (row + a/3 - 1,
 *     col + a%3 - 1); N_4(x) = x is stay.  T' (Fig. 2, not in the text) is
 *     read as: stay keeps the robot in place; any other action reaches N_a(x)
 *     w.p. 1 - 2*slip and each of the two cells 45 degrees to either side
 *     w.p. slip.  Mass that T' puts on an occupied or outside cell stays on x
 *     (the Sec. V transition equation).  The goal is absorbing.
 *   - Four sensors read the occupancy (outside = occupied) of N_1, N_3, N_5,
 *     N_7 (up, left, right, down) as bits 0..3 of z, |Z| = 16; each is right
 *     w.p. p_sensor, independently.
 *   - Stage reward r = -2 on occupied (or outside) cells, 0 at the goal, -1
 *     elsewhere; R(x, a) = -2 for stay off the goal, else sum_y r(y) T'(x, a,
 *     y); R = 0 at the goal and on occupied cells.
 * The tree is Alg. 2-7 as for the beacon model: full width to `depth`, K
 * samples of z per (V-node, action) from the same Philox streams (path code
 * = code * 9 + a, child code = path * 16 + z), FREQ weights f/K, leaves
 * valued by Eq. 4 against Q(., a') of qv9_value_iterate, the root action the
 * lowest index among the maxima. */
#define QV9_NUM_ACTIONS 9
#define QV9_NUM_OBS 16
#define QV9_MAX_DEPTH 3
#define QV9_MAX_K 16

typedef struct {
    int32_t H, W;             /* grid; W <= QV_MAX_WIDTH                               */
    const uint8_t *d_occ;     /* [H][W] device, caller-owned: 1 occupied, 0 free       */
    int32_t goal;             /* goal cell row * W + col, must be free                 */
    float slip;               /* each 45-degree slip, in [0, 1/3]                      */
    float p_sensor;           /* P(a sensor reads its cell right), in [0.5, 1]         */
    float discount;           /* gamma in (0, 1)                                       */
} qv9_model_t;

typedef struct qv9 qv9_t;

typedef struct {
    int32_t action;           /* root action, lowest index among the maxima            */
    float value;              /* U_V of the root                                       */
    float q[QV9_NUM_ACTIONS]; /* U_Q of the root's actions                             */
    int32_t nodes_per_level[QV9_MAX_DEPTH + 1];
    int64_t boundary_samples; /* draws within 1e-6 of a step of the FP32 CDF           */
} qv9_plan_result_t;

/* One level of the last plan, device pointers into the workspace (valid
 * until the next qv9_plan or qv9_value_iterate on the handle).  Nodes are in
 * (parent, action, z) order; belief is [count][H][W] for the internal levels
 * and NULL for the leaf level; R and UQ are [count][9] for the internal
 * levels and NULL for the leaf level. */
typedef struct {
    int32_t count;
    const int32_t *parent, *action, *obs;
    const float *weight, *pz, *value;
    const float *belief;
    const float *R, *UQ;
} qv9_level_view_t;

/* qv9_create: a handle for one model and tree shape (1 <= depth <= 3,
 * 1 <= K <= 16).  Reads the occupancy map back to the host to build the
 * cell words and the sensor-pattern order of the cells.  Synchronises.
 * qv9_workspace_bytes: device scratch the handle needs (the levels'
 * beliefs and node arrays at their worst-case sizes (9 min(K, 16))^l).
 * qv9_set_workspace: the caller's workspace (256-byte aligned, at least
 * qv9_workspace_bytes): uploads the handle's tables into it and builds the
 * R(x, a) table there.  Synchronises. */
qv_status qv9_create(const qv9_model_t *model, int32_t depth, int32_t K, qv9_t **out);
size_t qv9_workspace_bytes(const qv9_t *h);
qv_status qv9_set_workspace(qv9_t *h, void *d_ws, size_t ws_bytes, qv_stream_t stream);
void qv9_destroy(qv9_t *h);

/* MDP value iteration on the Sec. V model (Jacobi, from V = 0): stops at
 * the first sweep whose max-abs change is below tol, or runs exactly
 * `truncated` sweeps when truncated > 0; then Q = R + gamma T V.
 *   d_V  [H][W] in dtype (QV_F32 or QV_F64), caller-owned
 *   d_Q  [9][H][W] FP32, caller-owned
 * max_sweeps <= 131072.  QV_ERR_NOT_CONVERGED when max_sweeps ran out.
 * Synchronises (every 16 sweeps). */
qv_status qv9_value_iterate(qv9_t *h, int32_t dtype, double tol, int32_t max_sweeps, int32_t truncated,
                            void *d_V, float *d_Q, int32_t *sweeps_out, double *residual_out,
                            qv_stream_t stream);

/* One plan from d_b0 ([H][W] FP32, sums to 1; its occupied cells are
 * ignored) with leaves valued against d_Q ([9][H][W] FP32).  Synchronises
 * once per level (the next level's size is read back). */
qv_status qv9_plan(qv9_t *h, const float *d_Q, const float *d_b0, uint64_t seed, uint32_t episode,
                   qv9_plan_result_t *h_result, qv_stream_t stream);
qv_status qv9_level(const qv9_t *h, int32_t level, qv9_level_view_t *out);

#ifdef __cplusplus
}
#endif
#endif /* QVTS_H */
