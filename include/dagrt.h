/*
 * dagrt.h -- C ABI of libdagrt, a GB300 (sm_103a) library that evaluates the makespan
 * bound of "Exploiting Dependency and Parallelism: Real-Time Scheduling and Analysis for
 * GPU Tasks" (DAC '26) for batches of DAG-structured GPU tasks and candidate schedules.
 *
 * Problem statement (System Model, Sec. 2): a task is a DAG G = (V, E) whose nodes are
 * kernels v_i = {C^_i, C_i, m_i}: C^_i is the computation load (execution time on one SM,
 * integer ticks), m_i the SMs it is given and C_i its execution time (Eq.1); the GPU has M
 * SMs. The scheduler (Alg.1 Sub-graph_Division, Alg.2 Scheduling) chooses m_i, splits
 * nodes into segments and adds extra dependency edges; Lemma 1 and Theorem 1 bound the
 * makespan: R(G) <= sum_j max_{v_i in pi_j} C_i.
 *
 * Integer semantics (no floating point enters any bound; all times are int64 ticks):
 *   C(x, k, m) = max(1, ceil( ceil(m/M) * x * (64m - k(m-1)) / (64m) ))
 * is Eq.1 with t_min = 1, rounded up, and a per-kernel parallel fraction f = k/64 applied
 * as Amdahl's law; k = 64 gives Eq.1 exactly.
 *
 * Conventions shared by every call:
 *  - Every call returns DAGRT_OK (0) or a negative DAGRT_E_* code and never aborts; the
 *    message of the last failure is available from dagrt_last_error().
 *  - All device work is enqueued on the context's stream in order. Calls given host
 *    pointers copy through device staging buffers and synchronise that stream before they
 *    return. Calls given device pointers (DAGRT_PTR_DEVICE) only enqueue work; their
 *    outputs are valid once the caller synchronises the stream.
 *  - The caller owns every buffer it passes; the library owns the staging and scratch
 *    memory inside a context and a batch, and frees it in dagrt_destroy/dagrt_batch_free.
 *  - A context and its batches are used from one host thread at a time: the context's
 *    staging buffers (device and pinned host) are shared by its calls.
 */
#ifndef DAGRT_H
#define DAGRT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
#define DAGRT_OK 0
#define DAGRT_E_INVAL (-1)    /* null pointer, M outside [1, 4096], bad offsets or row_ptr,
                                 C^ outside [1, 2^32-1], k > 64, unknown variant/flag */
#define DAGRT_E_CYCLE (-2)    /* the graph of some DAG has a cycle */
#define DAGRT_E_RANGE (-3)    /* successor id outside [0, V), self loop, or a successor list
                                 that is not strictly increasing (duplicates included) */
#define DAGRT_E_OOM (-4)      /* device or pinned-host allocation failed */
#define DAGRT_E_DEVICE (-5)   /* a CUDA call failed */
#define DAGRT_E_TIMEOUT (-6)  /* a bounded device wait gave up (a tile copy never landed) */
#define DAGRT_E_CAP (-7)      /* an output buffer was smaller than the result (counts are
                                 still written) */
#define DAGRT_E_INTERNAL (-8) /* a device-side consistency check failed */

/* ---------------------------------------------------------------- flags */
#define DAGRT_PTR_DEVICE 1u   /* the call's array arguments are device pointers */

/* ---------------------------------------------------------------- structure variants
 * The schedule structure (groups, parallel launches, segments, extra edges) a bound is
 * evaluated on. DAGRT_VAR_PAPER is Alg.2 as the paper describes it, reading "S_j remaining
 * SMs" (Eq.6) as SMs still free after each launch. */
#define DAGRT_VAR_PAPER 0     /* Alg.1 groups; Alg.2 with parallel launches and segmentation */
#define DAGRT_VAR_NOPARA 1    /* Alg.1 groups; Eq.5 only, no parallel-node launches */
#define DAGRT_VAR_NOSEG 2     /* parallel launches of nodes that fit; never segments */
#define DAGRT_VAR_LITERAL 3   /* Alg.2 with S_j fixed per group and WS_j <- WS_j - C^_c */
#define DAGRT_VAR_NOREPAIR 4  /* as PAPER, but Eq.5's rounded SMs are not trimmed to M: the
                                 claim after Eq.5 that they fit is taken as it stands; a group
                                 whose SMs exceed M is bounded by the sum of its members'
                                 times (the sequential assumption) and launches nothing */
#define DAGRT_N_VARIANTS 5

/* ---------------------------------------------------------------- limits */
#define DAGRT_MAX_M 4096
#define DAGRT_MAX_V 65535     /* nodes per DAG */
#define DAGRT_MAX_E 16777216  /* edges per DAG */

typedef struct dagrt_ctx dagrt_ctx;
typedef struct dagrt_batch dagrt_batch;

/* Create a context on CUDA device `device`. `cuda_stream` is a cudaStream_t (for example a
 * torch stream's handle) or NULL for the legacy default stream. Returns DAGRT_E_DEVICE if
 * the device cannot be used. *out receives the context (NULL on failure). */
int dagrt_create(dagrt_ctx **out, int device, void *cuda_stream);

/* Change the stream later calls enqueue on. */
int dagrt_set_stream(dagrt_ctx *ctx, void *cuda_stream);

/* Synchronise the context's stream and report any CUDA error seen on it. */
int dagrt_sync(dagrt_ctx *ctx);

/* Free a context and every device buffer it owns. If batches, models or graphs of the
 * context are still alive, the context is freed when the last of them is (so they stay
 * usable until then). NULL is ignored. */
void dagrt_destroy(dagrt_ctx *ctx);

/* Text of the last error on this context ("" if none). Valid until the next call. */
const char *dagrt_last_error(const dagrt_ctx *ctx);

/* Number of kernels this context has launched so far (all calls), or -1 for NULL. */
int64_t dagrt_launch_count(const dagrt_ctx *ctx);

/* Load a batch of n_dags DAGs (System Model, Sec. 2.1: G = (V, E), C^_i; plus the
 * parallel fraction k_i/64 of each kernel) for an M-SM GPU (Sec. 2).
 *   node_off[n_dags+1] int64  DAG d owns nodes node_off[d] .. node_off[d+1]-1
 *                             (V_d <= DAGRT_MAX_V; V_d = 0 is an empty DAG)
 *   edge_off[n_dags+1] int64  DAG d owns edges edge_off[d] .. edge_off[d+1]-1
 *                             (E_d <= DAGRT_MAX_E)
 *   row_ptr[total_nodes + n_dags] int32  successor CSR of DAG d: its V_d+1 entries start
 *                             at node_off[d] + d, are local to edge_off[d], start at 0,
 *                             never decrease and end at E_d
 *   col[total_edges] int32    DAG-local successor ids, strictly increasing per row
 *   wcet[total_nodes] int64   C^_i in [1, 2^32-1] ticks
 *   k64[total_nodes] uint8    k_i in [0, 64]
 * With DAGRT_PTR_DEVICE the arrays are device pointers that the batch reads in place and
 * that must stay valid and unchanged until dagrt_batch_free; otherwise they are host
 * pointers that are copied. The offsets are checked here (E_INVAL); per-DAG graph checks
 * run on the device inside dagrt_schedule and are reported there, per DAG. */
int dagrt_load_csr(dagrt_ctx *ctx, int32_t n_dags, const int64_t *node_off,
                   const int64_t *edge_off, const int32_t *row_ptr, const int32_t *col,
                   const int64_t *wcet, const uint8_t *k64, int32_t M, uint32_t flags,
                   dagrt_batch **out);

/* Free a batch (NULL is ignored). Waits for the batch's work on the context stream. */
void dagrt_batch_free(dagrt_batch *batch);

int32_t dagrt_batch_n_dags(const dagrt_batch *batch);
int64_t dagrt_batch_total_nodes(const dagrt_batch *batch);

/* Outputs of dagrt_schedule. Every pointer may be NULL (not written). Per-node arrays are
 * indexed like wcet (node_off[d] + v); per-group and per-segment arrays of DAG d start at
 * node_off[d] (a DAG has at most V_d groups and V_d segments); plan rows of DAG d start at
 * 2*node_off[d]. Segment s of DAG d has the expanded-node id V_d + s. */
typedef struct {
    int64_t *bound;      /* [n_dags] R(G), Theorem 1; -1 where status != 0 */
    int32_t *status;     /* [n_dags] DAGRT_OK or the DAG's E_INVAL/E_RANGE/E_CYCLE/E_CAP */
    int32_t *n_groups;   /* [n_dags] |Pi| of Alg.1 (dropped groups included) */
    int32_t *n_seg;      /* [n_dags] segments made by Alg.2 */
    int32_t *n_rows;     /* [n_dags] plan rows (= V_d + n_seg) */
    int64_t *n_extra;    /* [n_dags] extra dependency edges of Alg.2 */
    int32_t *level;      /* [nodes] topological level: 0 for sources, 1 + max over preds */
    int64_t *wanc;       /* [nodes] W^anc, Eq.2 */
    int32_t *block_of;   /* [nodes] index k of B_k (Eq.3; k = index of theta_k in Theta),
                            or |Theta| for the residual block */
    int32_t *group_of;   /* [nodes] index of the node's balanced group in Pi (Alg.1) */
    int32_t *exec_group; /* [nodes] group during which the node's last part runs (Alg.2) */
    int32_t *m;          /* [nodes] SMs of the node's last part (Eq.5 or a parallel launch) */
    int64_t *group_R;    /* [groups] R(pi_j) per group (Lemma 1), 0 for a dropped group */
    int32_t *seg_parent; /* [segments] node split by the node-segmentation step */
    int64_t *seg_load;   /* [segments] load of the parallel segment */
    int32_t *seg_m;      /* [segments] its SMs */
    int32_t *seg_group;  /* [segments] group it runs in */
    int32_t *row_id;     /* [rows] node id (< V_d) or segment id (>= V_d) */
    int32_t *row_group;  /* [rows] group it runs in; rows are ordered by group, members by
                            id first, then parallel launches in launch order */
    int32_t *row_m0;     /* [rows] scheduled SMs */
    int64_t *row_load;   /* [rows] load executed by the row */
    int64_t *extra_off;  /* [n_dags+1] capacity layout of the extra-edge buffers (host or
                            device like the others); NULL = do not write edges */
    int32_t *extra_src;  /* [extra_off[n_dags]] (v_R, v_n) and (v_n, succ(v_R)) edges */
    int32_t *extra_dst;
    /* the baselines the Evaluation section compares Theorem 1 with (Sec. 5.2), per DAG,
     * -1 where status != 0 (the same for every structure variant):
     *   greedy          Greedy: m_i = min(C^_i, M), nodes assumed sequential: sum_i C_i
     *   greedy_unaware  Greedy + unaware (the normalisation reference): m_i = C^_i, so
     *                   Eq.1's wave factor ceil(C^_i / M) applies; sum_i C_i, exact,
     *                   saturated at 2^63 - 1
     *   graham_para     Graham_para: every node replaced by C^_i parallel unit loads on one
     *                   SM each, then Graham's bound L + ceil((sum C^ - L) / M) with L the
     *                   number of nodes on the longest path (parallel fractions ignored:
     *                   the units are fully parallel, as in the paper's model) */
    int64_t *greedy;
    int64_t *greedy_unaware;
    int64_t *graham_para;
    /* [n_dags] a lower bound of every execution of the schedule, -1 where status != 0: the
     * longest chain of its parts in G (a node's parts one after another, each edge of G
     * waiting for its tail's last part) weighted by the parts' times C (Eq.1), or the work
     * bound ceil(sum of m C over the parts / M) if larger (Sec. 2: path length). The
     * scheduler checks R(G) >= crit_path for every variant but LITERAL (whose launches can
     * outrun their group) and reports DAGRT_E_INTERNAL for the DAG if it fails. */
    int64_t *crit_path;
} dagrt_schedule_out;

/* Run Alg.1 and Alg.2 with structure variant `variant` on every DAG of the batch, evaluate
 * the bound of the resulting schedule (Lemma 1, Theorem 1) and keep the schedule in the
 * batch as the plan that dagrt_bound evaluates candidate allocations on.
 * flags: DAGRT_PTR_DEVICE if the `out` pointers are device pointers.
 * Returns the first failing DAG's status (E_INVAL, E_RANGE, E_CYCLE, E_CAP), or a device
 * error; with device outputs the per-DAG status array is the only report and the return
 * value covers launch errors only. */
int dagrt_schedule(dagrt_batch *batch, int32_t variant, const dagrt_schedule_out *out,
                   uint32_t flags);

/* Schedulability (System Model, Sec. 2: a periodic task tau = {G, T, D} with an implicit
 * deadline D = T is schedulable when its makespan bound R(G) <= D). For the bounds of the
 * batch's last dagrt_schedule(variant): ok[d] = 1 iff DAG d's schedule succeeded and its
 * bound is at most deadline[d] ticks, else 0; *n_ok = the number of such DAGs.
 *   deadline [n_dags] int64 (required), ok [n_dags] int32 (may be NULL), n_ok (may be NULL)
 * flags: DAGRT_PTR_DEVICE if all three are device pointers (then only enqueued); host
 * pointers are copied and the call synchronises. Returns DAGRT_E_INVAL if the variant was
 * not scheduled on the batch. */
int dagrt_schedulable(dagrt_batch *batch, int32_t variant, const int64_t *deadline, int32_t *ok,
                      int64_t *n_ok, uint32_t flags);

/* Bound of candidate allocations on fixed schedule structures (Lemma 1 / Theorem 1 on a
 * schedule whose SMs per node are given): per group, max C_i if the group's SMs fit in M,
 * else sum C_i (the sequential assumption of the Greedy analysis, Sec. 5.2); the bound is
 * the sum over groups (a max-plus sweep along the group chain).
 *   variant_ids[n_variants]  structure variant of each candidate block; each must have
 *                            been scheduled on this batch with dagrt_schedule
 *   n_alloc                  allocations per variant; candidate c = v*n_alloc + a
 *   m_alloc                  uint8 SMs per plan row and candidate, laid out
 *                            [(2*node_off[d] + row) * cand_stride + c]; 0 = keep the
 *                            scheduled m of the row
 *   cand_stride              >= n_variants*n_alloc, <= 65536 and a multiple of 16; a
 *                            device m_alloc must be 16-byte aligned and hold
 *                            2*total_nodes rows
 *   out_bound                [n_dags * n_cand] int64 (may be NULL)
 *   best_bound, best_cand    [n_dags] argmin over candidates (smallest bound, then
 *                            smallest candidate id); may be NULL
 * flags: DAGRT_PTR_DEVICE if all array arguments are device pointers. */
int dagrt_bound(dagrt_batch *batch, int32_t n_variants, const int32_t *variant_ids,
                int32_t n_alloc, const uint8_t *m_alloc, int64_t cand_stride,
                int64_t *out_bound, int64_t *best_bound, int32_t *best_cand, uint32_t flags);

/* Schedule search over generated candidate allocations (the problem formulation of Sec.
 * 2.2: choose m_i and the DAG structure to minimise the bound). Candidate c =
 * v * n_alloc + a of DAG d runs on the plan of structure variant variant_ids[v] (each must
 * have been scheduled on the batch); allocation a = 0 keeps the schedule's own m in every
 * mode. Every candidate's bound is exact (as dagrt_bound). Modes:
 *  DAGRT_SEARCH_RANDOM: for a > 0, plan row r gets levels[i] with i drawn by a
 *    counter-based generator: x = seed + (d << 40 | c << 20 | r), z = SplitMix64(x)
 *    (Steele, Lea and Flood, OOPSLA 2014), i = ((z >> 32) * n_levels) >> 32.
 *  DAGRT_SEARCH_EXHAUSTIVE: allocation a is a number in base B = n_levels + 1 whose digit
 *    u, (a / B^u) % B, sets the SMs of node u (on every plan row of u, its segments
 *    included): digit 0 keeps the schedule's m, digit i > 0 gives levels[i-1]. With
 *    n_alloc = B^V every allocation in ({schedule's m} + levels)^V of a V-node DAG is
 *    evaluated once; nodes with B^u > a keep the schedule's m. (seed is unused.)
 *  DAGRT_SEARCH_PERTURB: for a > 0, plan row r gets a change of its scheduled SMs m0,
 *    levels[i] (i drawn as in RANDOM) naming it: 0 keep, 1 halve (at least 1), 2 one fewer
 *    (at least 1), 3 one more, 4 double; changed counts are capped at 255. Repeating code 0
 *    in levels makes sparse perturbations of the schedule's own (Eq.5) allocation.
 * Limits: n_variants * n_alloc <= 2^20, n_levels in [1, 16] (at most 15 in EXHAUSTIVE),
 * levels in [1, 255] (codes in [0, 4] in PERTURB). */
#define DAGRT_SEARCH_RANDOM 0
#define DAGRT_SEARCH_EXHAUSTIVE 1
#define DAGRT_SEARCH_PERTURB 2
typedef struct {
    int32_t n_variants;
    const int32_t *variant_ids;  /* host array */
    int32_t n_alloc;
    int32_t n_levels;
    const uint8_t *levels;       /* host array */
    uint64_t seed;
    int32_t mode;                /* DAGRT_SEARCH_* */
} dagrt_search_cfg;

/* out_bound [n_dags * n_cand] (may be NULL); best_bound, best_cand [n_dags] as in
 * dagrt_bound (may be NULL); best_m [2*total_nodes] (may be NULL) receives the winning
 * allocation in rows [2*node_off[d], 2*node_off[d] + n_rows) of the winning variant's plan
 * (0 = keep the scheduled m). flags: DAGRT_PTR_DEVICE if the outputs are device pointers. */
int dagrt_search(dagrt_batch *batch, const dagrt_search_cfg *cfg, int64_t *out_bound,
                 int64_t *best_bound, int32_t *best_cand, uint8_t *best_m, uint32_t flags);

/* Scheduler entry point for callers that cannot allocate device memory at run time:
 * real-time executives that reserve every buffer before their task set starts (an
 * allocation may block for an unbounded time), work run under a memory budget owned by
 * someone else, and plug-ins whose host framework forbids cudaMalloc. The paper has no
 * counterpart; it is an operational variant of dagrt_load_csr + dagrt_schedule(variant)
 * that keeps only each DAG's bound and status.
 *
 * It allocates nothing: the scheduler's scratch (the per-team workspaces of the large-DAG
 * kernel and its work counter) lives in one fixed 4 MiB __device__ array inside the
 * library, which every GPU that loads the library holds until the process exits. All
 * array arguments are device pointers with dagrt_load_csr's layout; total_nodes and
 * total_edges are the lengths of wcet/k64 (row_ptr holds total_nodes + n_dags entries) and
 * of col. The offsets are not read on the host: the kernel checks each DAG against those
 * lengths and gives a DAG whose node or edge range reaches outside them (or has a negative
 * count) status DAGRT_E_INVAL and bound -1, as it does for DAGs of more than 512 nodes or
 * 8192 edges. bound[n_dags] and status[n_dags] receive dagrt_schedule's values otherwise.
 * The call only enqueues work on `cuda_stream` (a cudaStream_t, NULL = legacy default);
 * results are valid once the caller synchronises that stream.
 *
 * Every call looks up the array's device address (cudaGetSymbolAddress) with the caller's
 * current device, so a device reset between calls is harmless; the first call on a device
 * also loads the library's device code, so make it before capturing any stream. Every call
 * shares the array and resets its counter, so calls whose kernels overlap on the GPU (two
 * streams, two host threads) race and give wrong results: order them.
 * Returns DAGRT_OK, DAGRT_E_INVAL (a NULL pointer -- col may be NULL only when total_edges
 * is 0 --, n_dags or a length < 0, M or variant out of range) or DAGRT_E_DEVICE (a CUDA
 * call failed). */
int dagrt_schedule_noalloc(int32_t n_dags, const int64_t *node_off, const int64_t *edge_off,
                           const int32_t *row_ptr, const int32_t *col, const int64_t *wcet,
                           const uint8_t *k64, int64_t total_nodes, int64_t total_edges, int32_t M,
                           int32_t variant, int64_t *bound, int32_t *status, void *cuda_stream);

/* ---------------------------------------------------------------- conditional DAGs
 * The paper names conditional DAGs as future work; this is one reading of them. A node with
 * cond[v] = 1 takes exactly one of its out-edges per job (the branch its outcome selects).
 * A node runs when it is a source or one of its in-edges is active; an edge is active when
 * its tail runs and either is not conditional or chose that edge. A realisation (one choice
 * per conditional node) is then a plain DAG: the running nodes, renumbered in increasing
 * order, and the active edges. Choice tuples are enumerated in mixed radix (the lowest-id
 * conditional node varying fastest), a realisation equal to an earlier one is dropped, and
 * all realisations of all DAGs are scheduled and bounded (Alg.1, Alg.2 with `variant`,
 * Theorem 1) in one batched dagrt_schedule call; the worst one is taken on the device.
 * Inputs: host arrays in dagrt_load_csr's layout plus cond[total_nodes] (uint8 0/1); M;
 * max_real (1 .. 65536) realisations per DAG at most. Outputs per DAG (host arrays):
 *   adaptive[n_dags]   the largest bound over the realisations, each scheduled on its own
 *                      (the schedule chosen when a job's outcomes are known at release);
 *                      -1 if some realisation failed
 *   fixed[n_dags]      the bound of the whole DAG with every branch present: one schedule
 *                      for every job, a branch not taken running for no time (within its C,
 *                      so the bound holds by Theorem 1's sustainability); may be NULL
 *   worst_real[n_dags] index of the first realisation attaining `adaptive`; may be NULL
 *   n_real[n_dags]     number of distinct realisations; may be NULL
 * Synchronous; allocates its batch and scratch. Returns DAGRT_E_INVAL (bad arguments or
 * CSR shape), DAGRT_E_RANGE / DAGRT_E_CYCLE (a DAG's edges), DAGRT_E_CAP (more than 2^20
 * choice tuples or more than max_real realisations in some DAG), a scheduling error, or
 * DAGRT_E_DEVICE / DAGRT_E_OOM. */
int dagrt_cond_bound(dagrt_ctx *ctx, int32_t n_dags, const int64_t *node_off, const int64_t *edge_off,
                     const int32_t *row_ptr, const int32_t *col, const int64_t *wcet, const uint8_t *k64,
                     const uint8_t *cond, int32_t M, int32_t variant, int32_t max_real, int64_t *adaptive,
                     int64_t *fixed, int32_t *worst_real, int32_t *n_real);

/* ---------------------------------------------------------------- realisation on the GPU
 * A schedule of one DAG run on this GPU as a CUDA graph, as in the case study of the
 * Evaluation section (CUDA Graph API; m_i realised through the kernel's launch shape; loads
 * emulated by one kernel function run for different lengths). The GPU is narrowed to the
 * model's M SMs: before each replay, filler CTAs (one per SM, each running for a fixed time
 * longer than the replay) take the other SMs, and the graph is launched once every filler
 * has counted itself in (host-mapped memory). Every part of the schedule (a node's last
 * part, or a parallel segment) is one kernel node whose grid has m CTAs, each reserving
 * more than half of an SM's shared memory so that the kernel holds m SMs; every
 * CTA runs for C^ ((1 - f) + f / m) ticks of tick_us microseconds (Eq.1 with Amdahl's
 * parallel fraction f = k/64, not rounded). Edges: each DAG edge u -> v makes every part of
 * v wait for u's last part, and a node's segment runs before its residual part; then by
 * mode
 *   DAGRT_REALISE_BARRIER  plus a barrier after each group of Pi (the group-by-group
 *                          execution Theorem 1's proof assumes);
 *   DAGRT_REALISE_EDGES    plus the extra dependencies of Alg.2 only (the paper's claim
 *                          that they order the groups);
 *   DAGRT_REALISE_GREEDY   the Greedy baseline of the case study instead: every kernel on
 *                          min(C^, M) SMs, only the DAG's edges.
 * Inputs are one DAG in dagrt_load_csr's layout (host pointers, V >= 1), M <= the device's
 * SM count, the structure variant (ignored by GREEDY), reps >= 1 timed replays after one
 * warm-up; makespan_us[reps] receives each replay's time (CUDA events around the graph
 * launch) and *bound (may be NULL) the bound in ticks: Theorem 1's R(G), or the Greedy
 * baseline for GREEDY. Synchronous; allocates its own graph and streams. Returns
 * DAGRT_E_INVAL (bad argument, M above the SM count, a part above M SMs), the schedule's
 * per-DAG error, DAGRT_E_DEVICE, DAGRT_E_TIMEOUT (a kernel's wait hit its limit, or the
 * fillers did not all start within a quarter of their time) or DAGRT_E_INTERNAL (a replay
 * may have outlasted the fillers: it may have used more than M SMs). */
#define DAGRT_REALISE_BARRIER 0
#define DAGRT_REALISE_EDGES 1
#define DAGRT_REALISE_GREEDY 2
int dagrt_realise(dagrt_ctx *ctx, int32_t V, const int32_t *row_ptr, const int32_t *col,
                  const int64_t *wcet, const uint8_t *k64, int32_t M, int32_t variant, int32_t mode,
                  float tick_us, int32_t reps, float *makespan_us, int64_t *bound);

/* ---------------------------------------------------------------- batching controls
 * Launch-shape choices of the batched kernels. None of them changes a result: every
 * setting gives bit-identical outputs; they only move work between kernels.
 *   warp_max_v  scheduler: DAGs of at most this many nodes (and at most 12 edges per node
 *               of their class) are scheduled by warp teams in shared memory, larger ones by
 *               CTA teams with global workspaces; one of 0 (CTA teams only), 64, 128, 192,
 *               256. Default 256.
 *   chunk_rows  candidate bounds: the plan rows of a DAG are cut into work items of whole
 *               groups (Theorem 1's sum splits at group ends), as many as fit in this many
 *               rows (a longer group alone); 8 .. 256. Default 64.
 *   item_warps  candidate bounds: warps per CTA of the work-item kernel, 1 .. 8. Default 4.
 *   cta_smem    scheduler: k in 1 .. 4 = CTA teams keep their workspace in shared memory
 *               while it takes at most 1/k of a CTA's shared memory (smallest large DAGs
 *               first; k teams then fit per SM), 0 = always in global memory. Default 2. */
typedef struct {
    int32_t warp_max_v;
    int32_t chunk_rows;
    int32_t item_warps;
    int32_t cta_smem;
} dagrt_tuning;

int dagrt_get_tuning(const dagrt_batch *batch, dagrt_tuning *out);
/* Validates and applies t (DAGRT_E_INVAL on a value outside the ranges above). Host work
 * and one upload; synchronises the context's stream. */
int dagrt_set_tuning(dagrt_batch *batch, const dagrt_tuning *t);

/* Autotuner. Times dagrt_schedule(batch, variant) (device outputs) for every warp_max_v
 * in {64, 128, 192, 256} x cta_smem in {0, 1, 2, 3, 4}, `reps` times each after one warm-up (CUDA events on the
 * context's stream), keeps the fastest setting in the batch and returns it (*best_ms: its
 * median time). Synchronous. */
int dagrt_autotune_schedule(dagrt_batch *batch, int32_t variant, int32_t reps, dagrt_tuning *chosen,
                            float *best_ms);
/* Same for dagrt_bound with the given candidates (device m_alloc; every variant must have
 * been scheduled): chunk_rows in {24, 32, 48, 64} x item_warps in {2, 4, 8}. Only calls
 * that take the work-item kernel (n_alloc a multiple of 64) have anything to tune;
 * others return the current setting unchanged. */
int dagrt_autotune_bound(dagrt_batch *batch, int32_t n_variants, const int32_t *variant_ids,
                         int32_t n_alloc, const uint8_t *m_alloc, int64_t cand_stride, int32_t reps,
                         dagrt_tuning *chosen, float *best_ms);

/* ---------------------------------------------------------------- CUDA graphs
 * dagrt_graph_begin synchronises the context's stream and starts capturing (relaxed capture mode, on
 * a private stream of the context, so that the legacy default stream works too); every
 * library call made with DAGRT_PTR_DEVICE until dagrt_graph_end is recorded, not run, and
 * dagrt_graph_launch replays the recorded kernels and copies on the context's stream (the
 * same device buffers, whatever they hold at replay time). Calls that need the host
 * during capture (host outputs, dagrt_load_csr, schedule extra-edge buffers, a scratch
 * buffer that must grow) fail with DAGRT_E_INVAL and leave the capture open: make each
 * call once before capturing so that its buffers exist. */
typedef struct dagrt_graph dagrt_graph;
int dagrt_graph_begin(dagrt_ctx *ctx);
int dagrt_graph_end(dagrt_ctx *ctx, dagrt_graph **out);
int dagrt_graph_launch(dagrt_graph *graph);
void dagrt_graph_free(dagrt_graph *graph);

/* ---------------------------------------------------------------- failure detection
 * Every device-side wait of the library (mbarriers of TMA copies and tensor-core MMAs) has
 * an iteration limit; a wait that gives up makes the call return DAGRT_E_TIMEOUT and leaves
 * the context usable. dagrt_selftest_wait exercises that path: one CTA waits on a barrier
 * that nothing arrives on, gives up after `limit` polls and the call returns
 * DAGRT_E_TIMEOUT (DAGRT_OK would mean the wait did not give up). Synchronous. */
int dagrt_selftest_wait(dagrt_ctx *ctx, uint32_t limit);

/* ---------------------------------------------------------------- learned proposer
 * The paper gives the bound of one allocation (Eq.1, Lemma 1, Theorem 1) but no way to
 * choose among the many allocations of a DAG beyond the Eq.5 heuristic of Alg.2. The
 * proposer is an extension of the bound's evaluation, not a step of the paper: a
 * message-passing network scores, for every kernel, which SM level of a fixed level list
 * it should get; the k most likely joint assignments (and the paper's own allocation) are
 * then evaluated exactly on the paper schedule's structure (Alg.2 groups and segments,
 * Theorem 1) and the smallest bound wins. The exact check makes every returned bound a
 * true Theorem 1 bound of a valid allocation, whatever the network's quality.
 *
 * Network: x_i (8 features, zero-padded to 16): log2 C^_i / 32, k_i / 64,
 * log2(1 + indegree) / 8, log2(1 + outdegree) / 8, level_i / depth (Alg.1 levels),
 * W^anc_i / sum C^ (the ancestor weight Alg.1 orders by), log2 m_i / 12 (the paper
 * schedule's m_i, Eq.5), 1. Three layers h' = ReLU([h | mean_pred h | mean_succ h] W + b)
 * with hidden width 128 (W: [3*16 x 128] then [384 x 128]), then a head h3 Wh + bh to one
 * logit per level (Wh: [128 x 16], unused levels ignored). Activations and GEMM operands
 * are bf16 with fp32 accumulation; parameters are fp32 in the order W1, b1, W2, b2, W3,
 * b3, Wh, bh (row-major, input index first), dagrt_model_n_params() floats in all.
 * Training minimises the mean softmax cross-entropy over labelled kernels with Adam
 * (beta 0.9/0.999, eps 1e-8). Reductions over nodes run in a fixed order, so results
 * repeat bit for bit on one GPU. */
typedef struct dagrt_model dagrt_model;

/* Number of fp32 parameters. */
int64_t dagrt_model_n_params(void);

/* New model on ctx's device: levels[0..n_levels) are the SM counts a kernel may be given
 * (1 <= n_levels <= 16, each >= 1; levels above M are allowed and clamp like any m in
 * Eq.1's ceil(m/M) term). Weights are uniform in +-sqrt(6/fan_in) from the SplitMix64
 * stream starting at `seed`; biases are 0. Returns DAGRT_E_INVAL or DAGRT_E_DEVICE on
 * failure, with *out = NULL. */
int dagrt_model_create(dagrt_ctx *ctx, int32_t n_levels, const uint8_t *levels, uint64_t seed,
                       dagrt_model **out);
void dagrt_model_free(dagrt_model *model);

/* Host copy of the parameters out (get != NULL) and/or in (set != NULL; set is applied
 * first), dagrt_model_n_params() floats each. Synchronous. */
int dagrt_model_params(dagrt_model *model, float *get, const float *set);

/* The whole training state, for checkpoints: parameters, Adam's first and second moments
 * (3 * dagrt_model_n_params() floats, in that order) and the step count. set (may be NULL)
 * is applied first with set_step (>= 0); get and get_step (may be NULL) receive the state.
 * Training resumed from a state continues exactly as the uninterrupted run. Synchronous. */
int dagrt_model_state(dagrt_model *model, float *get, int32_t *get_step, const float *set,
                      int32_t set_step);

/* Logits of every kernel of the batch: logits[(node_off[d] + i) * n_levels + l]. The first
 * call on a batch also runs the paper schedule (variant 0) for the features. */
int dagrt_model_logits(dagrt_batch *batch, dagrt_model *model, float *logits, uint32_t flags);

/* Mean cross-entropy over the labelled kernels and its gradient. labels[total_nodes] (host)
 * holds each kernel's level index, or -1 for no label. grads (host, n_params floats, may be
 * NULL) receives dLoss/dparams; *loss (may be NULL) the loss. Synchronous. */
int dagrt_model_grad(dagrt_batch *batch, dagrt_model *model, const int8_t *labels, float *grads,
                     float *loss);

/* dagrt_model_grad followed by one Adam step with learning rate lr. Synchronous. */
int dagrt_train_step(dagrt_batch *batch, dagrt_model *model, const int8_t *labels, float lr,
                     float *loss);

/* Proposals and their exact check, per DAG: candidate 0 is the paper's allocation (Alg.2's
 * m_i), candidates 1..k (1 <= k <= 16) the k most likely level assignments under the
 * model, most likely first (kernel i's level applies to every plan row of i, its segments
 * included). Each is evaluated on the paper schedule's structure exactly as dagrt_bound
 * does. Outputs (any may be NULL):
 *   out_bound[d * (k+1) + c]    bound of candidate c of DAG d;
 *   cand_m[(2 * node_off[d] + r) * (k+1) + c]   candidate c's SMs for plan row r
 *                               (0 in column 0 = the schedule's own m; rows >= n_rows unset);
 *   best_bound[d], best_cand[d] the smallest bound and its candidate (lowest index on ties,
 *                               so the paper's allocation wins ties);
 *   best_m[2 * node_off[d] + r] the winning allocation of plan row r.
 * Host outputs are synchronous; with DAGRT_PTR_DEVICE the call only enqueues work. */
int dagrt_propose(dagrt_batch *batch, dagrt_model *model, int32_t k, int64_t *out_bound,
                  uint8_t *cand_m, int64_t *best_bound, int32_t *best_cand, uint8_t *best_m,
                  uint32_t flags);

#ifdef __cplusplus
}
#endif

#endif /* DAGRT_H */
