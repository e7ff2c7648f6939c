/*
 * oracle.c -- plain, slow CPU oracle (one thread per DAG) for the makespan bound of
 * "Exploiting Dependency and Parallelism: Real-Time Scheduling and Analysis for GPU
 * Tasks" (DAC '26).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the library's product path may link, load or
 * call this file: only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark do. It shares no source with the CUDA path.
 *
 * Style: every step follows the paper's order and notation, with explicit ancestor
 * sets, full scans instead of clever data structures, qsort for ordering and `/` for
 * every ceiling. All times are int64 ticks; no floating point is used anywhere.
 *
 * Readings of the paper applied here (the paper is silent or inconsistent on them):
 *  - Eq.1 is rounded up to whole ticks; a parallel fraction f = k/64 enters as
 *    Amdahl's law, time = ceil(m/M) * C^ * ((1-f) + f/m); f = 1 gives Eq.1 itself.
 *  - Theta is ordered by ASCENDING W^anc (ties: lower id); only that order keeps
 *    the topological order the Block Formulation section asks for and reproduces the
 *    Sub-graph Division example.
 *  - Top_M in Alg.1 takes the M heads with the LARGEST W^anc (ties: lower id).
 *  - Rule 2: if some head picked by Top_M has m^max = C^ >= M, the group is that
 *    head alone (largest C^, ties: first in Top_M order).
 *  - Eq.5 rounds half up on the exact rational, clamps to >= 1 and, if the group's
 *    SM sum exceeds M, decrements the largest m (ties: higher id) until it fits. Variant 4
 *    leaves the rounded SMs as they are; a group whose SMs then exceed M is bounded by the
 *    sum of its members' times (the sequential assumption) and launches no parallel node.
 *  - Launching parallel nodes (Alg.2) spends the REMAINING SMs: after each launch
 *    S <- S - m_c. The literal form (S fixed, WS <- WS - C^_c) is variant 3.
 *  - A parallel node is split iff it cannot finish within R(pi_j) on min(C^, S)
 *    SMs; its parallel segment is the largest load x that can (at min(x, S) SMs);
 *    after a split the launch loop ends (at most one segmentation per group).
 *  - Released nodes: every predecessor finished in an earlier group; para(pi_j) is
 *    every released, unfinished node outside pi_j, by descending W^anc (ties: id).
 *  - v_R = lowest id among the members with maximal C; succ(v_R) are its successors
 *    in G.
 *  - A group whose members were all launched earlier is dropped (R = 0).
 *  - The bound of an arbitrary allocation on a fixed schedule structure: per group,
 *    max C when the group's SM sum fits in M (Lemma 1), else the sum of C (the
 *    sequential assumption the paper's Greedy analysis makes).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_E_INVAL (-1)
#define OR_E_CYCLE (-2)
#define OR_E_RANGE (-3)
#define OR_E_OOM (-4)
#define OR_E_CAP (-7)

#define OR_MAX_M 4096
#define OR_MAX_WCET 4294967295LL

/* structure variants of the schedule */
#define OR_VAR_PAPER 0   /* Alg.2, remaining-SM accounting */
#define OR_VAR_NOPARA 1  /* Alg.1 groups only, no parallel-node launches */
#define OR_VAR_NOSEG 2   /* parallel launches that fit, never split */
#define OR_VAR_LITERAL 3 /* Alg.2 with S_j fixed and WS_j <- WS_j - C^_c */
#define OR_VAR_NOREPAIR 4 /* Alg.2 with Eq.5's rounded SMs left as they are */

typedef struct {
    /* per node, capacity V */
    int32_t *level;      /* Kahn level: 0 for sources, else 1 + max over predecessors */
    int64_t *wanc;       /* Eq.2 */
    int32_t *block_of;   /* index k of the block B_k (0-based); N = residual block */
    int32_t *group_of;   /* Alg.1: index of the node's balanced group in Pi */
    int32_t *exec_group; /* Alg.2: group during which the node (its last part) runs */
    int32_t *m;          /* Alg.2: SMs given to the node's last part */
    int32_t *theta;      /* join nodes in Theta order, n_join entries */
    int64_t *group_R;    /* R(pi_j) per group (0 for a dropped group), n_groups entries */
    int32_t *seg_parent; /* parallel segments, n_seg entries (segment id = V + s) */
    int64_t *seg_load;
    int32_t *seg_m;
    int32_t *seg_group;
    /* plan rows, capacity 2V, ordered by exec group; in a group: members by id,
       then launched nodes/segments in launch order */
    int32_t *row_id;
    int64_t *row_load;
    int32_t *row_k;
    int32_t *row_m0;
    int32_t *row_group;
    /* extra dependencies, capacity extra_cap (may be 0 with NULL arrays) */
    int32_t *extra_src;
    int32_t *extra_dst;
    int64_t extra_cap;
    /* scalars */
    int32_t n_join;
    int32_t n_groups;
    int32_t n_seg;
    int32_t n_rows;
    int64_t n_extra;
    int64_t bound;
} or_sched_out;

/* ------------------------------------------------------------------ Eq.1 */

/* Execution time of a kernel with load `load` (ticks at one SM), parallel fraction
 * k/64, on m SMs of an M-SM GPU: Eq.1 with t_min = 1 and Amdahl's law for the
 * parallel fraction, rounded up to a whole tick. */
int64_t or_exec_time(int64_t load, int64_t k, int64_t m, int64_t M)
{
    int64_t waves = (m + M - 1) / M;           /* ceil(m / M) */
    int64_t num = waves * load * (64 * m - k * (m - 1));
    int64_t den = 64 * m;
    int64_t c = (num + den - 1) / den;         /* ceil(num / den) */
    return c < 1 ? 1 : c;
}

/* --------------------------------------------------------- small helpers */

static int bit_get(const uint64_t *set, int64_t i) { return (int)((set[i >> 6] >> (i & 63)) & 1u); }
static void bit_set(uint64_t *set, int64_t i) { set[i >> 6] |= (uint64_t)1 << (i & 63); }

/* the sort key of the comparators below; one per thread, so that threads may schedule
 * different DAGs at once (the all-cores timing of the oracle) */
static _Thread_local const int64_t *g_key_w;
static int cmp_w_asc_id_asc(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    if (g_key_w[x] != g_key_w[y]) return g_key_w[x] < g_key_w[y] ? -1 : 1;
    return x < y ? -1 : (x > y);
}
static int cmp_w_desc_id_asc(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    if (g_key_w[x] != g_key_w[y]) return g_key_w[x] > g_key_w[y] ? -1 : 1;
    return x < y ? -1 : (x > y);
}

/* ------------------------------------------------------------ validation */

/* Checks in a fixed order; the first failing class decides the status:
 * row_ptr shape -> INVAL, load or fraction out of range -> INVAL,
 * successor id out of range, self loop, unsorted/duplicate successor -> RANGE. */
int or_validate(int32_t V, const int32_t *row_ptr, int64_t E, const int32_t *col,
                const int64_t *wcet, const uint8_t *k64, int32_t M)
{
    if (M < 1 || M > OR_MAX_M || V < 0 || E < 0) return OR_E_INVAL;
    if (row_ptr[0] != 0 || row_ptr[V] != E) return OR_E_INVAL;
    for (int32_t v = 0; v < V; v++)
        if (row_ptr[v + 1] < row_ptr[v]) return OR_E_INVAL;
    for (int32_t v = 0; v < V; v++) {
        if (wcet[v] < 1 || wcet[v] > OR_MAX_WCET) return OR_E_INVAL;
        if (k64[v] > 64) return OR_E_INVAL;
    }
    for (int32_t v = 0; v < V; v++)
        for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; e++) {
            if (col[e] < 0 || col[e] >= V || col[e] == v) return OR_E_RANGE;
            if (e > row_ptr[v] && col[e] <= col[e - 1]) return OR_E_RANGE;
        }
    return OR_OK;
}

/* ------------------------------------------------------- R8 segment size */

/* Largest load x in [1, load-1] that finishes within R ticks on min(x, S) SMs.
 * Exec time at min(x, S) SMs never decreases as x grows, so a binary search over x
 * finds the largest x that satisfies the test; x = 1 always does (time 1 <= R). */
static int64_t split_load(int64_t load, int64_t k, int64_t S, int64_t R, int64_t M)
{
    int64_t lo = 1, hi = load - 1;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo + 1) / 2;
        int64_t m = mid < S ? mid : S;
        if (or_exec_time(mid, k, m, M) <= R) lo = mid; else hi = mid - 1;
    }
    return lo;
}

/* ------------------------------------------------------------- schedule */

/* Schedule one DAG (Alg.1 then Alg.2) and evaluate its bound (Lemma 1, Theorem 1).
 * Returns OR_OK or an error code; the out arrays must hold V entries (rows: 2V). */
int or_schedule_dag(int32_t V, const int32_t *row_ptr, const int32_t *col,
                    const int64_t *wcet, const uint8_t *k64, int32_t M, int32_t variant,
                    or_sched_out *out)
{
    int64_t E = V > 0 ? row_ptr[V] : 0;
    out->n_join = out->n_groups = out->n_seg = out->n_rows = 0;
    out->n_extra = 0;
    out->bound = 0;
    if (variant < 0 || variant > 4) return OR_E_INVAL;
    int rc = or_validate(V, row_ptr, E, col, wcet, k64, M);
    if (rc != OR_OK) return rc;
    if (V == 0) return OR_OK;

    int64_t nw = (V + 63) / 64;
    int32_t *indeg = calloc(V, sizeof *indeg), *cnt = calloc(V, sizeof *cnt);
    int32_t *order = calloc(V, sizeof *order), *level = calloc(V, sizeof *level);
    uint64_t *anc = calloc((size_t)V * nw, sizeof *anc);
    int64_t *W = calloc(V, sizeof *W);
    if (!indeg || !cnt || !order || !level || !anc || !W) {
        free(indeg); free(cnt); free(order); free(level); free(anc); free(W);
        return OR_E_OOM;
    }

    /* --- topological levels (Kahn) and the cycle check --------------------- */
    for (int64_t e = 0; e < E; e++) indeg[col[e]]++;
    int32_t head = 0, tail = 0;
    for (int32_t v = 0; v < V; v++) {
        cnt[v] = indeg[v];
        if (cnt[v] == 0) { order[tail++] = v; level[v] = 0; }
    }
    while (head < tail) {
        int32_t u = order[head++];
        for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; e++) {
            int32_t s = col[e];
            if (level[u] + 1 > level[s]) level[s] = level[u] + 1;
            if (--cnt[s] == 0) order[tail++] = s;
        }
    }
    if (tail != V) {
        free(indeg); free(cnt); free(order); free(level); free(anc); free(W);
        return OR_E_CYCLE;
    }

    /* --- ancestor sets: every ancestor of u, and u itself, is an ancestor of each
     *     successor of u (u visited in topological order) ------------------- */
    for (int32_t i = 0; i < V; i++) {
        int32_t u = order[i];
        for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; e++) {
            int32_t s = col[e];
            for (int64_t w = 0; w < nw; w++) anc[(int64_t)s * nw + w] |= anc[(int64_t)u * nw + w];
            bit_set(&anc[(int64_t)s * nw], u);
        }
    }

    /* --- Eq.2: cumulative ancestor workload ---------------------------------- */
    for (int32_t v = 0; v < V; v++) {
        W[v] = wcet[v];
        for (int32_t u = 0; u < V; u++)
            if (bit_get(&anc[(int64_t)v * nw], u)) W[v] += wcet[u];
    }

    /* --- Alg.1, first step: join nodes (>= 2 predecessors) ordered by W^anc ------- */
    int32_t *theta = calloc(V, sizeof *theta);
    int32_t N = 0;
    for (int32_t v = 0; v < V; v++)
        if (indeg[v] >= 2) theta[N++] = v;
    g_key_w = W;
    qsort(theta, N, sizeof *theta, cmp_w_asc_id_asc);

    /* --- Alg.1, block step, Eq.3: B_k = ance(theta_k) minus earlier blocks; the
     *     remaining nodes form the residual block B_{N+1} (index N here) ------ */
    int32_t *block_of = malloc(V * sizeof *block_of);
    for (int32_t v = 0; v < V; v++) block_of[v] = -1;
    for (int32_t k = 0; k < N; k++) {
        const uint64_t *a = &anc[(int64_t)theta[k] * nw];
        for (int32_t u = 0; u < V; u++)
            if (bit_get(a, u) && block_of[u] < 0) block_of[u] = k;
    }
    for (int32_t u = 0; u < V; u++)
        if (block_of[u] < 0) block_of[u] = N;

    /* --- Alg.1, path step: per block, local complete paths (Eq.4) and balanced
     *     groups built from their heads ---------------------------------------- */
    int32_t *group_of = malloc(V * sizeof *group_of);
    for (int32_t v = 0; v < V; v++) group_of[v] = -1;
    int32_t G = 0;
    int32_t *in_pred = malloc(V * sizeof *in_pred);     /* in-block predecessor count */
    int32_t *in_succ = malloc(V * sizeof *in_succ);     /* in-block successor count */
    int32_t *stack = malloc((size_t)(V + 1) * sizeof *stack);
    int32_t *heads = malloc(V * sizeof *heads);
    int32_t *is_head = calloc(V, sizeof *is_head);
    int32_t *sel = calloc(V, sizeof *sel);
    for (int32_t v = 0; v < V; v++) { in_pred[v] = 0; in_succ[v] = 0; }
    for (int32_t u = 0; u < V; u++)
        for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; e++)
            if (block_of[col[e]] == block_of[u]) { in_succ[u]++; in_pred[col[e]]++; }

    /* path storage: all local complete paths of one block, concatenated */
    int64_t path_cap = 1024, npath = 0, pstore_cap = 4096, pstore_n = 0;
    int64_t *p_begin = malloc(path_cap * sizeof *p_begin);   /* current head position */
    int64_t *p_end = malloc(path_cap * sizeof *p_end);
    int32_t *pstore = malloc(pstore_cap * sizeof *pstore);
    int32_t *dfs_e = malloc(V * sizeof *dfs_e);

    for (int32_t k = 0; k <= N; k++) {
        npath = 0; pstore_n = 0;
        /* Eq.4: enumerate every path from a local source to a local sink by DFS along
         * in-block edges (a block is an out-forest: <= 1 in-block predecessor). */
        for (int32_t s = 0; s < V; s++) {
            if (block_of[s] != k || in_pred[s] != 0) continue;
            int32_t depth = 0;
            stack[depth] = s; dfs_e[s] = row_ptr[s];
            for (;;) {
                int32_t u = stack[depth];
                if (in_succ[u] == 0 && dfs_e[u] == row_ptr[u]) {
                    /* local sink reached: emit stack[0..depth] as a path */
                    if (npath == path_cap) {
                        path_cap *= 2;
                        p_begin = realloc(p_begin, path_cap * sizeof *p_begin);
                        p_end = realloc(p_end, path_cap * sizeof *p_end);
                    }
                    while (pstore_n + depth + 1 > pstore_cap) {
                        pstore_cap *= 2;
                        pstore = realloc(pstore, pstore_cap * sizeof *pstore);
                    }
                    p_begin[npath] = pstore_n;
                    for (int32_t i = 0; i <= depth; i++) pstore[pstore_n++] = stack[i];
                    p_end[npath] = pstore_n;
                    npath++;
                    dfs_e[u] = row_ptr[u + 1]; /* mark explored */
                }
                /* advance to the next unexplored in-block successor of u */
                int32_t next = -1;
                while (dfs_e[u] < row_ptr[u + 1]) {
                    int32_t c = col[dfs_e[u]++];
                    if (block_of[c] == k) { next = c; break; }
                }
                if (next >= 0) {
                    stack[++depth] = next;
                    dfs_e[next] = row_ptr[next];
                } else {
                    if (depth == 0) break;
                    depth--;
                }
            }
        }
        /* while Lambda_k is not empty: take the heads of its paths */
        for (;;) {
            int32_t nh = 0;
            for (int64_t p = 0; p < npath; p++) {
                if (p_begin[p] == p_end[p]) continue;
                int32_t h = pstore[p_begin[p]];
                if (!is_head[h]) { is_head[h] = 1; heads[nh++] = h; }
            }
            if (nh == 0) break;
            for (int32_t i = 0; i < nh; i++) is_head[heads[i]] = 0;
            /* Top_M by W^anc (largest first, ties: lower id) */
            qsort(heads, nh, sizeof *heads, cmp_w_desc_id_asc);
            int32_t t = nh < M ? nh : M;
            /* Rule 2: a head with m^max = C^ >= M runs alone */
            int32_t big = -1;
            for (int32_t i = 0; i < t; i++)
                if (wcet[heads[i]] >= M && (big < 0 || wcet[heads[i]] > wcet[big])) big = heads[i];
            if (big >= 0) { heads[0] = big; t = 1; }
            for (int32_t i = 0; i < t; i++) { group_of[heads[i]] = G; sel[heads[i]] = 1; }
            /* remove the group's nodes from the paths they head */
            for (int64_t p = 0; p < npath; p++)
                if (p_begin[p] < p_end[p] && sel[pstore[p_begin[p]]]) p_begin[p]++;
            for (int32_t i = 0; i < t; i++) sel[heads[i]] = 0;
            G++;
        }
    }
    free(p_begin); free(p_end); free(pstore); free(dfs_e);
    free(in_pred); free(in_succ); free(stack); free(is_head);

    /* --- Alg.2: scheduling over Pi, with Lemma 1 / Theorem 1 ----------------- */
    int64_t *rem = malloc(V * sizeof *rem);      /* load not yet executed */
    int32_t *done = calloc(V, sizeof *done);     /* node finished */
    int32_t *npl = malloc(V * sizeof *npl);      /* predecessors not yet finished */
    int32_t *mm = calloc(V, sizeof *mm);
    int64_t *C = calloc(V, sizeof *C);
    int32_t *exec_group = malloc(V * sizeof *exec_group);
    int32_t *P = malloc(V * sizeof *P), *Q = malloc(V * sizeof *Q);
    int32_t *launched = calloc(V, sizeof *launched);
    int32_t *fin = malloc(V * sizeof *fin);
    /* launch records of one group: node id (>= V for a segment) */
    int32_t *L_id = malloc(V * sizeof *L_id);
    for (int32_t v = 0; v < V; v++) { rem[v] = wcet[v]; npl[v] = indeg[v]; exec_group[v] = -1; }
    int64_t bound = 0;
    int rc_out = OR_OK;

    for (int32_t j = 0; j < G; j++) {
        int32_t np = 0;
        for (int32_t v = 0; v < V; v++)
            if (group_of[v] == j && !done[v]) P[np++] = v;
        if (out->group_R) out->group_R[j] = 0;
        if (np == 0) continue; /* every member already ran as a parallel node */

        /* Eq.5: parallelism scaling, round half up, clamp, repair sum <= M */
        int64_t Wg = 0;
        for (int32_t i = 0; i < np; i++) Wg += rem[P[i]];
        int64_t sum_m = 0;
        for (int32_t i = 0; i < np; i++) {
            int32_t v = P[i];
            int64_t r = (2 * rem[v] * M + Wg) / (2 * Wg);
            if (r < 1) r = 1;
            mm[v] = (int32_t)(rem[v] < r ? rem[v] : r);
            sum_m += mm[v];
        }
        while (variant != OR_VAR_NOREPAIR && sum_m > M) {
            int32_t best = -1;
            for (int32_t i = 0; i < np; i++)
                if (best < 0 || mm[P[i]] >= mm[best]) best = P[i]; /* ties: higher id */
            mm[best]--; sum_m--;
        }
        /* Eq.1 per member, Lemma 1: R(pi_j) = max C_i; v_R = lowest id with max C */
        int64_t R = 0, sum_c = 0; int32_t vR = -1;
        for (int32_t i = 0; i < np; i++) {
            int32_t v = P[i];
            C[v] = or_exec_time(rem[v], k64[v], mm[v], M);
            sum_c += C[v];
            if (C[v] > R) { R = C[v]; vR = v; }
        }
        /* a group whose SMs exceed M (possible only without the repair) runs its members
         * one after another: R is their summed time */
        if (sum_m > M) R = sum_c;
        /* Eq.6: remaining SMs and spare capacity */
        int64_t S = sum_m < M ? M - sum_m : 0;
        int64_t WS = R * S;

        /* Eq.7: released, unfinished nodes outside pi_j, by descending W^anc */
        int32_t nq = 0;
        for (int32_t u = 0; u < V; u++)
            if (npl[u] == 0 && !done[u] && group_of[u] != j) Q[nq++] = u;
        qsort(Q, nq, sizeof *Q, cmp_w_desc_id_asc);

        /* record the members as plan rows (by id) */
        for (int32_t i = 0; i < np; i++) {
            int32_t v = P[i], r = out->n_rows++;
            if (out->row_id) {
                out->row_id[r] = v; out->row_load[r] = rem[v]; out->row_k[r] = k64[v];
                out->row_m0[r] = mm[v]; out->row_group[r] = j;
            }
        }

        /* Alg.2, parallel step: launch parallel nodes, segment when one does not fit */
        int32_t nl = 0;
        for (int32_t q = 0; q < nq && variant != OR_VAR_NOPARA; q++) {
            int32_t u = Q[q];
            int64_t mu, load = rem[u];
            if (variant == OR_VAR_LITERAL) {
                if (WS <= 0) break;
                if (load > WS) {                      /* split: parallel part = WS_j */
                    int64_t p = WS;
                    mu = p < S ? p : S;
                    int32_t s = out->n_seg++;
                    if (out->seg_parent) {
                        out->seg_parent[s] = u; out->seg_load[s] = p;
                        out->seg_m[s] = (int32_t)mu; out->seg_group[s] = j;
                    }
                    int32_t r = out->n_rows++;
                    if (out->row_id) {
                        out->row_id[r] = V + s; out->row_load[r] = p; out->row_k[r] = k64[u];
                        out->row_m0[r] = (int32_t)mu; out->row_group[r] = j;
                    }
                    rem[u] -= p;
                    L_id[nl++] = V + s;
                    WS = 0;
                    break;
                }
                mu = load < S ? load : S;
                mm[u] = (int32_t)mu; exec_group[u] = j; launched[u] = 1;
                WS -= load;
            } else {
                if (S == 0) break;
                mu = load < S ? load : S;
                if (or_exec_time(load, k64[u], mu, M) > R) {
                    if (variant == OR_VAR_NOSEG) continue;
                    int64_t p = split_load(load, k64[u], S, R, M);
                    int64_t ms = p < S ? p : S;
                    int32_t s = out->n_seg++;
                    if (out->seg_parent) {
                        out->seg_parent[s] = u; out->seg_load[s] = p;
                        out->seg_m[s] = (int32_t)ms; out->seg_group[s] = j;
                    }
                    int32_t r = out->n_rows++;
                    if (out->row_id) {
                        out->row_id[r] = V + s; out->row_load[r] = p; out->row_k[r] = k64[u];
                        out->row_m0[r] = (int32_t)ms; out->row_group[r] = j;
                    }
                    rem[u] -= p;
                    L_id[nl++] = V + s;
                    break;
                }
                mm[u] = (int32_t)mu; exec_group[u] = j; launched[u] = 1;
                S -= mu;
            }
            int32_t r = out->n_rows++;
            if (out->row_id) {
                out->row_id[r] = u; out->row_load[r] = load; out->row_k[r] = k64[u];
                out->row_m0[r] = (int32_t)mu; out->row_group[r] = j;
            }
            L_id[nl++] = u;
        }

        /* extra dependencies: (launched, succ(v_R)) and (v_R, unlaunched para node) */
        for (int32_t i = 0; i < nl; i++)
            for (int32_t e = row_ptr[vR]; e < row_ptr[vR + 1]; e++) {
                if (out->n_extra < out->extra_cap) {
                    out->extra_src[out->n_extra] = L_id[i]; out->extra_dst[out->n_extra] = col[e];
                }
                out->n_extra++;
            }
        if (variant != OR_VAR_NOPARA)
            for (int32_t q = 0; q < nq; q++) {
                int32_t u = Q[q];
                if (launched[u]) continue;
                if (out->n_extra < out->extra_cap) {
                    out->extra_src[out->n_extra] = vR; out->extra_dst[out->n_extra] = u;
                }
                out->n_extra++;
            }

        /* members and whole launches finish with pi_j; release their successors */
        int32_t nf = 0;
        for (int32_t i = 0; i < np; i++) {
            int32_t v = P[i];
            done[v] = 1; rem[v] = 0; exec_group[v] = j; fin[nf++] = v;
        }
        for (int32_t q = 0; q < nq; q++) {
            int32_t u = Q[q];
            if (launched[u]) { done[u] = 1; rem[u] = 0; launched[u] = 0; fin[nf++] = u; }
        }
        for (int32_t i = 0; i < nf; i++)
            for (int32_t e = row_ptr[fin[i]]; e < row_ptr[fin[i] + 1]; e++) npl[col[e]]--;

        /* Theorem 1: the bound is the sum of the group response times */
        if (out->group_R) out->group_R[j] = R;
        bound += R;
    }
    if (out->extra_cap > 0 && out->n_extra > out->extra_cap) rc_out = OR_E_CAP;

    /* outputs */
    out->n_join = N; out->n_groups = G; out->bound = bound;
    for (int32_t v = 0; v < V; v++) {
        if (out->level) out->level[v] = level[v];
        if (out->wanc) out->wanc[v] = W[v];
        if (out->block_of) out->block_of[v] = block_of[v];
        if (out->group_of) out->group_of[v] = group_of[v];
        if (out->exec_group) out->exec_group[v] = exec_group[v];
        if (out->m) out->m[v] = mm[v];
    }
    if (out->theta) for (int32_t i = 0; i < N; i++) out->theta[i] = theta[i];

    free(rem); free(done); free(npl); free(mm); free(C); free(exec_group); free(P); free(Q);
    free(launched); free(fin); free(L_id); free(sel); free(heads);
    free(indeg); free(cnt); free(order); free(level); free(anc); free(W);
    free(theta); free(block_of); free(group_of);
    return rc_out;
}

/* ------------------------------------------- bound of a candidate allocation */

/* Bound of one allocation on a fixed schedule structure (plan rows ordered by group).
 * alloc[r * stride] is the SM count of row r; 0 keeps the scheduled row_m0[r].
 * Per group: Lemma 1 (max C) if the SM sum fits in M, else the sum of C. */
int64_t or_bound_plan(int32_t n_rows, const int64_t *row_load, const int32_t *row_k,
                      const int32_t *row_m0, const int32_t *row_group, int32_t M,
                      const uint8_t *alloc, int64_t stride)
{
    int64_t bound = 0;
    int32_t r = 0;
    while (r < n_rows) {
        int32_t g = row_group[r];
        int64_t sum_m = 0, max_c = 0, sum_c = 0;
        for (; r < n_rows && row_group[r] == g; r++) {
            int64_t m = alloc ? alloc[(int64_t)r * stride] : 0;
            if (m == 0) m = row_m0[r];
            int64_t c = or_exec_time(row_load[r], row_k[r], m, M);
            sum_m += m;
            sum_c += c;
            if (c > max_c) max_c = c;
        }
        bound += sum_m <= M ? max_c : sum_c;
    }
    return bound;
}

/* ------------------------------------------------------------ batch helpers */

/* Paper-schedule bound of every DAG of a batch (the CPU baseline's unit of work).
 * Writes bound[d] and status[d]; returns the number of DAGs that failed. */
int64_t or_schedule_batch(int32_t n_dags, const int64_t *node_off, const int64_t *edge_off,
                          const int32_t *row_ptr, const int32_t *col, const int64_t *wcet,
                          const uint8_t *k64, int32_t M, int32_t variant,
                          int64_t *bound, int32_t *status)
{
    int64_t fails = 0;
    for (int32_t d = 0; d < n_dags; d++) {
        or_sched_out o;
        memset(&o, 0, sizeof o);
        int32_t V = (int32_t)(node_off[d + 1] - node_off[d]);
        int rc = or_schedule_dag(V, row_ptr + node_off[d] + d, col + edge_off[d],
                                 wcet + node_off[d], k64 + node_off[d], M, variant, &o);
        bound[d] = rc == OR_OK ? o.bound : -1;
        status[d] = rc;
        fails += rc != OR_OK;
    }
    return fails;
}

/* ------------------------------------------------- generated candidate search */

/* SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
 * OOPSLA 2014): the output function applied to the counter x. */
uint64_t or_splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Level index of plan row r of candidate c of DAG d (candidates with allocation index 0
 * keep the schedule: the caller handles them). The counter packs (d, c, r) as
 * d << 40 | c << 20 | r added to the seed; the high 32 bits of the mixed value pick one of
 * n_levels levels by multiply-shift. */
int32_t or_gen_level(uint64_t seed, int64_t d, int64_t c, int64_t r, int32_t n_levels)
{
    uint64_t x = seed + (((uint64_t)d << 40) | ((uint64_t)c << 20) | (uint64_t)r);
    uint64_t hi = or_splitmix64(x) >> 32;
    return (int32_t)((hi * (uint64_t)n_levels) >> 32);
}

/* ------------------------------------------------- exhaustive allocation search */

/* Every allocation of a fixed schedule structure in which each node u gets either the
 * schedule's own SMs or one of n_levels levels, on all of its plan rows: allocation a is
 * read as a number in base B = n_levels + 1 whose digit u, (a / B^u) % B, is 0 (keep) or
 * i (levels[i-1]). row_owner[r] is the node plan row r belongs to (a segment's parent).
 * out[a] receives the bound of allocation a, for a in [0, n_alloc). */
void or_exhaustive_plan(int32_t n_rows, const int64_t *row_load, const int32_t *row_k,
                        const int32_t *row_m0, const int32_t *row_group, const int32_t *row_owner,
                        int32_t M, int32_t n_levels, const uint8_t *levels, int64_t n_alloc,
                        int64_t *out)
{
    int64_t B = n_levels + 1;
    uint8_t *alloc = malloc((size_t)(n_rows > 0 ? n_rows : 1));
    for (int64_t a = 0; a < n_alloc; a++) {
        for (int32_t r = 0; r < n_rows; r++) {
            int64_t q = a;
            for (int32_t u = 0; u < row_owner[r]; u++) q /= B;
            int64_t digit = q % B;
            alloc[r] = digit == 0 ? 0 : levels[digit - 1];
        }
        out[a] = or_bound_plan(n_rows, row_load, row_k, row_m0, row_group, M, alloc, 1);
    }
    free(alloc);
}

/* ------------------------------------------------------- baselines (Sec. 5.2) */

/* Eq.1 (with the parallel fraction) for any m, in 128-bit arithmetic, saturated at
 * 2^63 - 1: Greedy + unaware gives a kernel C^ SMs, far above M. */
static int64_t exec_time_wide(int64_t load, int64_t k, int64_t m, int64_t M)
{
    unsigned __int128 waves = (unsigned __int128)((m + M - 1) / M);
    unsigned __int128 num = waves * (unsigned __int128)load * (unsigned __int128)(64 * m - k * (m - 1));
    unsigned __int128 den = (unsigned __int128)(64 * m);
    unsigned __int128 c = (num + den - 1) / den;
    if (c < 1) c = 1;
    return c > (unsigned __int128)INT64_MAX ? INT64_MAX : (int64_t)c;
}

/* The three baselines the Evaluation section compares Theorem 1 with, for one DAG:
 *   out[0] Greedy: every kernel on m = min(C^, M) SMs, kernels one after another;
 *   out[1] Greedy + unaware: every kernel on m = C^ SMs (Eq.1's waves apply), one after
 *          another (saturated at 2^63 - 1);
 *   out[2] Graham_para: every kernel replaced by C^ unit loads on one SM each, Graham's
 *          bound L + (vol - L) / M rounded up, with L the number of nodes on the longest
 *          path and vol the sum of C^.
 * Returns OR_OK or the validation / cycle error (outputs untouched then). */
int or_baselines(int32_t V, const int32_t *row_ptr, const int32_t *col, const int64_t *wcet,
                 const uint8_t *k64, int32_t M, int64_t *out)
{
    int64_t E = V > 0 ? row_ptr[V] : 0;
    int rc = or_validate(V, row_ptr, E, col, wcet, k64, M);
    if (rc != OR_OK) return rc;
    /* longest path in nodes, by relaxing edges in a topological order (Kahn) */
    int32_t *indeg = calloc(V > 0 ? V : 1, sizeof *indeg), *order = calloc(V > 0 ? V : 1, sizeof *order);
    int64_t *len = calloc(V > 0 ? V : 1, sizeof *len);
    for (int64_t e = 0; e < E; e++) indeg[col[e]]++;
    int32_t head = 0, tail = 0;
    for (int32_t v = 0; v < V; v++) {
        len[v] = 1;
        if (indeg[v] == 0) order[tail++] = v;
    }
    while (head < tail) {
        int32_t u = order[head++];
        for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; e++) {
            int32_t s = col[e];
            if (len[u] + 1 > len[s]) len[s] = len[u] + 1;
            if (--indeg[s] == 0) order[tail++] = s;
        }
    }
    if (tail != V) {
        free(indeg); free(order); free(len);
        return OR_E_CYCLE;
    }
    int64_t greedy = 0, unaware = 0, vol = 0, L = 0;
    for (int32_t v = 0; v < V; v++) {
        int64_t m = wcet[v] < M ? wcet[v] : M;
        greedy += or_exec_time(wcet[v], k64[v], m, M);
        int64_t u = exec_time_wide(wcet[v], k64[v], wcet[v], M);
        unaware = (unaware > INT64_MAX - u) ? INT64_MAX : unaware + u;
        vol += wcet[v];
        if (len[v] > L) L = len[v];
    }
    out[0] = greedy;
    out[1] = unaware;
    out[2] = V > 0 ? L + (vol - L + M - 1) / M : 0;
    free(indeg); free(order); free(len);
    return OR_OK;
}
