// sched.cu -- per-DAG scheduling and bound kernels (Alg.1, Alg.2, Lemma 1, Theorem 1).
//
// One team (a warp for DAGs that fit a shared-memory workspace, a CTA otherwise) takes a
// whole DAG from a work-stealing counter and runs every step of the method on it without
// leaving its workspace: CSR validation, Kahn levels, the ancestor closure and W^anc
// (Eq.2), Theta and the blocks of Eq.3, the balanced groups of Alg.1, the scheduling loop
// of Alg.2 and the bound of Theorem 1. The schedule is written out as "plan rows" that the
// candidate-bound kernel evaluates other allocations on.
#include "dagrt_internal.cuh"
#include "sched.cuh"

namespace dagrt {

// node state bits
enum : uint8_t { ST_ACTIVE = 1, ST_INT = 2, ST_SEL = 4, ST_DONE = 8, ST_LAUNCH = 16 };

// ------------------------------------------------------------------ workspace layout
struct Ws {
    uint32_t *load, *rem;
    uint8_t *kk, *st;
    int32_t *indeg, *cnt, *lvl_off, *blk, *group_of, *gstart, *lst, *tmp;
    uint16_t *topo, *rank, *byrank, *rnd, *gmem, *mm;
    uint64_t *wanc, *relmask;
    int32_t *sc;
    // phase-local region (reused): closure / sort / peel / member lists
    uint64_t *anc, *planes;          // phase A
    uint64_t *skey, *bk;             // phase B
    int32_t *fcnt, *nround;          // phase C
    uint64_t *bigk;                  // phase C
    uint16_t *gtmp;                  // phase D
    int32_t *gfill;                  // phase D
};

__host__ __device__ inline int pow2_ceil(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

// Carve a workspace for DAGs of up to vc nodes out of `base`; returns the bytes used.
__host__ __device__ inline int64_t ws_carve(unsigned char *base, int vc, Ws *ws) {
    const int W = ceil_div(vc, 64) > 0 ? ceil_div(vc, 64) : 1;
    const int P = pow2_ceil(vc > 0 ? vc : 1);
    int64_t off = 0;
    auto take = [&](int64_t bytes) {
        unsigned char *p = base + off;
        off = align_up(off + bytes, 16);
        return p;
    };
    Ws w;
    w.load = (uint32_t *)take(4ll * vc);
    w.rem = (uint32_t *)take(4ll * vc);
    w.kk = (uint8_t *)take(vc);
    w.st = (uint8_t *)take(vc);
    w.indeg = (int32_t *)take(4ll * vc);
    w.cnt = (int32_t *)take(4ll * vc);
    w.lvl_off = (int32_t *)take(4ll * (vc + 1));
    w.blk = (int32_t *)take(4ll * vc);
    w.group_of = (int32_t *)take(4ll * vc);
    w.gstart = (int32_t *)take(4ll * (vc + 2));
    w.lst = (int32_t *)take(4ll * (vc + 1));
    w.tmp = (int32_t *)take(4ll * vc);
    w.topo = (uint16_t *)take(2ll * vc);
    w.rank = (uint16_t *)take(2ll * vc);
    w.byrank = (uint16_t *)take(2ll * vc);
    w.rnd = (uint16_t *)take(2ll * vc);
    w.gmem = (uint16_t *)take(2ll * vc);
    w.mm = (uint16_t *)take(2ll * vc);
    w.wanc = (uint64_t *)take(8ll * vc);
    w.relmask = (uint64_t *)take(8ll * W);
    w.sc = (int32_t *)take(4 * 16);
    const int64_t xbase = off;
    // phase A
    int64_t xa = 0, xb = 0, xc = 0, xd = 0;
    off = xbase;
    w.anc = (uint64_t *)take(8ll * vc * W);
    w.planes = (uint64_t *)take(8ll * 32 * W);
    xa = off;
    off = xbase;
    w.skey = (uint64_t *)take(8ll * P);
    w.bk = (uint64_t *)take(8ll * vc);
    xb = off;
    off = xbase;
    w.fcnt = (int32_t *)take(4ll * (vc + 1));
    w.nround = (int32_t *)take(4ll * (vc + 1));
    w.bigk = (uint64_t *)take(8ll * (vc + 1));
    xc = off;
    off = xbase;
    w.gtmp = (uint16_t *)take(2ll * vc);
    w.gfill = (int32_t *)take(4ll * (vc + 1));
    xd = off;
    int64_t end = xa;
    if (xb > end) end = xb;
    if (xc > end) end = xc;
    if (xd > end) end = xd;
    if (ws) *ws = w;
    return align_up(end, 128);
}

int64_t sched_ws_bytes(int vc) { return ws_carve(nullptr, vc, nullptr); }

// ------------------------------------------------------------------ per-DAG outputs
__device__ inline void write_failure(const SchedArgs &a, int d, int code) {
    a.status[d] = code;
    a.bound[d] = -1;
    a.nrows[d] = 0;
    if (a.o.status) a.o.status[d] = code;
    if (a.o.bound) a.o.bound[d] = -1;
    if (a.o.n_groups) a.o.n_groups[d] = 0;
    if (a.o.n_seg) a.o.n_seg[d] = 0;
    if (a.o.n_rows) a.o.n_rows[d] = 0;
    if (a.o.n_extra) a.o.n_extra[d] = 0;
}

__device__ inline void write_row(const SchedArgs &a, int64_t rbase, int r, int id, int group,
                                 uint32_t load, uint32_t k, uint32_t m, uint64_t c, bool last) {
    const int64_t i = rbase + r;
    a.plan_lc[i] = make_uint2(load, (uint32_t)c);
    a.plan_mkf[i] = m | (k << 16) | ((last ? 1u : 0u) << 24);
    if (a.o.row_id) a.o.row_id[i] = id;
    if (a.o.row_group) a.o.row_group[i] = group;
    if (a.o.row_m0) a.o.row_m0[i] = (int32_t)m;
    if (a.o.row_load) a.o.row_load[i] = load;
}

// ------------------------------------------------------------------ one DAG
template <int NT>
__device__ void schedule_one(const Team<NT> &tm, const Ws &ws, const SchedArgs &a, int d, int vc) {
    const int64_t n0 = a.node_off[d];
    const int V = (int)(a.node_off[d + 1] - n0);
    const int64_t e0 = a.edge_off[d];
    const int64_t E = a.edge_off[d + 1] - e0;
    const int32_t *__restrict__ rp = a.row_ptr + n0 + d;
    const int32_t *__restrict__ col = a.col + e0;
    const int64_t *__restrict__ wc = a.wcet + n0;
    const uint8_t *__restrict__ kp = a.k64 + n0;
    const uint32_t M = (uint32_t)a.M;
    const int variant = a.variant;
    volatile int32_t *sc = ws.sc;
    const bool lead = tm.t == 0;

    if (V > vc) {  // routed to the wrong size class: never expected
        if (lead) write_failure(a, d, DAGRT_E_INTERNAL);
        return;
    }

    // ---- validation: row_ptr shape, then loads and fractions, then successor ids
    bool bad = false;
    if (lead) bad = rp[0] != 0 || (int64_t)rp[V] != E;
    for (int v = tm.t; v < V; v += NT)
        if (rp[v + 1] < rp[v]) bad = true;
    if (tm.any(bad)) {
        if (lead) write_failure(a, d, DAGRT_E_INVAL);
        return;
    }
    bool badv = false, badc = false;
    for (int v = tm.t; v < V; v += NT) {
        const int64_t w = wc[v];
        const uint8_t k = kp[v];
        if (w < 1 || w > 0xffffffffll || k > 64) badv = true;
        ws.load[v] = (uint32_t)w;
        ws.kk[v] = k;
        ws.indeg[v] = 0;
        ws.st[v] = 0;
        int prev = -1;
        for (int e = rp[v]; e < rp[v + 1]; e++) {
            const int c = col[e];
            if (c < 0 || c >= V || c == v || c <= prev) badc = true;
            prev = c;
        }
    }
    if (tm.any(badv)) {
        if (lead) write_failure(a, d, DAGRT_E_INVAL);
        return;
    }
    if (tm.any(badc)) {
        if (lead) write_failure(a, d, DAGRT_E_RANGE);
        return;
    }
    if (V == 0) {
        if (lead) {
            a.status[d] = DAGRT_OK;
            a.bound[d] = 0;
            a.nrows[d] = 0;
            if (a.o.status) a.o.status[d] = DAGRT_OK;
            if (a.o.bound) a.o.bound[d] = 0;
            if (a.o.n_groups) a.o.n_groups[d] = 0;
            if (a.o.n_seg) a.o.n_seg[d] = 0;
            if (a.o.n_rows) a.o.n_rows[d] = 0;
            if (a.o.n_extra) a.o.n_extra[d] = 0;
        }
        return;
    }
    tm.sync();

    // ---- in-degrees; join = at least two predecessors
    for (int u = tm.t; u < V; u += NT)
        for (int e = rp[u]; e < rp[u + 1]; e++) atomicAdd(&ws.indeg[col[e]], 1);
    const int W = (V + 63) >> 6;
    for (int i = tm.t; i < V * W; i += NT) ws.anc[i] = 0;
    if (lead) sc[0] = 0;
    tm.sync();

    // ---- Kahn levels, and the ancestor closure pushed along each level's out-edges:
    //      everything that reaches u, and u itself, reaches each successor of u
    for (int v = tm.t; v < V; v += NT) {
        ws.cnt[v] = ws.indeg[v];
        if (ws.indeg[v] == 0) {
            const int p = atomicAdd((int *)&sc[0], 1);
            ws.topo[p] = (uint16_t)v;
            if (a.o.level) a.o.level[n0 + v] = 0;
        }
    }
    tm.sync();
    int ls = 0, le = sc[0], L = 0;
    if (lead) ws.lvl_off[0] = 0;
    while (ls < le) {
        for (int i = ls + tm.t; i < le; i += NT) {
            const int u = ws.topo[i];
            const uint64_t *au = ws.anc + (int64_t)u * W;
            for (int e = rp[u]; e < rp[u + 1]; e++) {
                const int s = col[e];
                unsigned long long *as = (unsigned long long *)(ws.anc + (int64_t)s * W);
                for (int w = 0; w < W; w++) {
                    const uint64_t x = au[w];
                    if (x) atomicOr(&as[w], (unsigned long long)x);
                }
                atomicOr(&as[u >> 6], 1ull << (u & 63));
                if (atomicSub(&ws.cnt[s], 1) == 1) {
                    const int p = atomicAdd((int *)&sc[0], 1);
                    ws.topo[p] = (uint16_t)s;
                    if (a.o.level) a.o.level[n0 + s] = L + 1;
                }
            }
        }
        tm.sync();
        const int ne = sc[0];
        tm.sync();
        L++;
        if (lead) ws.lvl_off[L] = le;
        ls = le;
        le = ne;
    }
    const int nlev = L;
    if (le != V) {
        if (lead) write_failure(a, d, DAGRT_E_CYCLE);
        return;
    }

    // ---- Eq.2: W^anc(v) = C^_v + sum of C^ over ancestors, by bit planes of C^
    uint64_t mx = 0;
    for (int v = tm.t; v < V; v += NT) mx = mx > ws.load[v] ? mx : ws.load[v];
    mx = tm.maxu(mx);
    const int nb = 64 - __clzll((long long)mx);
    for (int i = tm.t; i < nb * W; i += NT) {
        const int b = i / W, w = i - b * W;
        const int vb = w * 64, ve = min(V, vb + 64);
        uint64_t word = 0;
        for (int v = vb; v < ve; v++) word |= (uint64_t)((ws.load[v] >> b) & 1u) << (v - vb);
        ws.planes[i] = word;
    }
    tm.sync();
    for (int v = tm.t; v < V; v += NT) {
        const uint64_t *av = ws.anc + (int64_t)v * W;
        uint64_t acc = ws.load[v];
        for (int b = 0; b < nb; b++) {
            uint32_t c = 0;
            for (int w = 0; w < W; w++) c += __popcll(av[w] & ws.planes[b * W + w]);
            acc += (uint64_t)c << b;
        }
        ws.wanc[v] = acc;
    }
    tm.sync();

    // ---- order nodes by (W^anc, id): Theta uses it ascending, Top_M and para(pi_j)
    //      descending with ties broken by lower id
    const int P = pow2_ceil(V);
    for (int i = tm.t; i < P; i += NT)
        ws.skey[i] = i < V ? ((ws.wanc[i] << 16) | (uint64_t)i) : KEY_INF;
    tm.sync();
    team_bitonic_sort(tm, ws.skey, P);
    // per sorted position: join flag (-> Theta index), start and end of its W^anc run
    int32_t *jcnt = ws.lst, *rs = ws.cnt, *re = ws.gstart;
    for (int i = tm.t; i < V; i += NT) {
        const int v = (int)(ws.skey[i] & 0xffff);
        const uint64_t wv = ws.skey[i] >> 16;
        jcnt[i] = ws.indeg[v] >= 2 ? 1 : 0;
        rs[i] = (i == 0 || (ws.skey[i - 1] >> 16) != wv) ? i : 0;
        re[i] = (i == V - 1 || (ws.skey[i + 1] >> 16) != wv) ? i : 0x7fffffff;
    }
    tm.sync();
    team_scan_inplace(tm, jcnt, V, [](uint64_t x, uint64_t y) { return x + y; }, false);
    team_scan_inplace(tm, rs, V, [](uint64_t x, uint64_t y) { return x > y ? x : y; }, false);
    team_scan_inplace(tm, re, V, [](uint64_t x, uint64_t y) { return x < y ? x : y; }, true);
    const int N = jcnt[V - 1];  // number of join nodes
    uint16_t *jidx = ws.rnd;    // Theta index of each join node
    for (int i = tm.t; i < V; i += NT) {
        const int v = (int)(ws.skey[i] & 0xffff);
        const int r = (V - 1 - re[i]) + (i - rs[i]);
        ws.rank[v] = (uint16_t)r;
        ws.byrank[r] = (uint16_t)v;
        if (ws.indeg[v] >= 2) jidx[v] = (uint16_t)(jcnt[i] - 1);
    }
    tm.sync();

    // ---- Eq.3 blocks: a node belongs to the first join (in Theta order) it is an ancestor
    //      of, i.e. the smallest (W^anc, id) among the joins reachable from it; computed by
    //      a min over successors in reverse level order. No reachable join: residual.
    for (int v = tm.t; v < V; v += NT) ws.bk[v] = KEY_INF;
    tm.sync();
    for (int l = nlev - 1; l >= 0; l--) {
        const int lb = ws.lvl_off[l], lend = (l + 1 < nlev) ? ws.lvl_off[l + 1] : V;
        for (int i = lb + tm.t; i < lend; i += NT) {
            const int v = ws.topo[i];
            uint64_t b = KEY_INF;
            for (int e = rp[v]; e < rp[v + 1]; e++) {
                const int s = col[e];
                if (ws.indeg[s] >= 2) {
                    const uint64_t ks = (ws.wanc[s] << 16) | (uint64_t)s;
                    b = ks < b ? ks : b;
                }
                const uint64_t bs = ws.bk[s];
                b = bs < b ? bs : b;
            }
            ws.bk[v] = b;
        }
        tm.sync();
    }
    for (int v = tm.t; v < V; v += NT) {
        const uint64_t b = ws.bk[v];
        ws.blk[v] = b == KEY_INF ? N : (int)jidx[(int)(b & 0xffff)];
    }
    tm.sync();

    // ---- Alg.1: peel every block's out-forest (<= 1 in-block predecessor per node)
    //      round by round; a round of a block takes Top_M of its heads by W^anc (Rule 1),
    //      or a single head with C^ >= M (Rule 2). Blocks are independent, so all of them
    //      advance together; round r of block k becomes the group after block k's
    //      earlier rounds and after every group of blocks 0..k-1.
    for (int v = tm.t; v < V; v += NT) ws.cnt[v] = 0;
    for (int b = tm.t; b <= N; b += NT) {
        ws.fcnt[b] = 0;
        ws.nround[b] = 0;
        ws.bigk[b] = 0;
    }
    tm.sync();
    for (int u = tm.t; u < V; u += NT)
        for (int e = rp[u]; e < rp[u + 1]; e++)
            if (ws.blk[col[e]] == ws.blk[u]) atomicAdd(&ws.cnt[col[e]], 1);
    tm.sync();
    bad = false;
    for (int v = tm.t; v < V; v += NT) {
        if (ws.cnt[v] > 1) bad = true;
        ws.st[v] = ws.cnt[v] == 0 ? ST_ACTIVE : 0;
    }
    if (tm.any(bad)) {
        if (lead) write_failure(a, d, DAGRT_E_INTERNAL);
        return;
    }
    tm.sync();
    for (int round = 0;; round++) {
        if (round > V) {  // every round selects a node, so this cannot happen
            if (lead) write_failure(a, d, DAGRT_E_INTERNAL);
            return;
        }
        bool act = false;
        for (int v = tm.t; v < V; v += NT)
            if (ws.st[v] & ST_ACTIVE) {
                act = true;
                atomicAdd(&ws.fcnt[ws.blk[v]], 1);
            }
        if (!tm.any(act)) break;
        tm.sync();
        for (int v = tm.t; v < V; v += NT) {
            if (!(ws.st[v] & ST_ACTIVE)) continue;
            const int b = ws.blk[v];
            bool inT = true;
            if (ws.fcnt[b] > (int)M) {  // more heads than SMs: keep the M heaviest
                const int rv = ws.rank[v];
                int pos = 0;
                for (int u = 0; u < V; u++)
                    if ((ws.st[u] & ST_ACTIVE) && ws.blk[u] == b && ws.rank[u] < rv) pos++;
                inT = pos < (int)M;
            }
            if (inT) {
                ws.st[v] |= ST_INT;
                if (ws.load[v] >= M)
                    atomicMax((unsigned long long *)&ws.bigk[b],
                              ((unsigned long long)ws.load[v] << 16) | (0xffffu - ws.rank[v]));
            }
        }
        tm.sync();
        for (int v = tm.t; v < V; v += NT) {
            const uint8_t s0 = ws.st[v];
            if (!(s0 & ST_INT)) continue;
            const int b = ws.blk[v];
            const uint64_t bg = ws.bigk[b];
            const bool sel = bg == 0 || (int)(bg & 0xffff) == (int)(0xffffu - ws.rank[v]);
            if (sel) {
                ws.st[v] = (uint8_t)((s0 & ~(ST_INT | ST_ACTIVE)) | ST_SEL);
                ws.rnd[v] = (uint16_t)round;
                atomicMax(&ws.nround[b], round + 1);
            } else {
                ws.st[v] = (uint8_t)(s0 & ~ST_INT);
            }
        }
        tm.sync();
        for (int v = tm.t; v < V; v += NT) {
            const uint8_t s0 = ws.st[v];
            if (s0 & (ST_ACTIVE | ST_SEL)) {
                ws.fcnt[ws.blk[v]] = 0;
                ws.bigk[ws.blk[v]] = 0;
            }
            if (s0 & ST_SEL) {
                ws.st[v] = (uint8_t)(s0 & ~ST_SEL);
                for (int e = rp[v]; e < rp[v + 1]; e++) {
                    const int s = col[e];
                    if (ws.blk[s] == ws.blk[v]) ws.st[s] |= ST_ACTIVE;
                }
            }
        }
        tm.sync();
    }
    // group index = groups of earlier blocks + round within the block
    team_scan_inplace(tm, ws.nround, N + 1, [](uint64_t x, uint64_t y) { return x + y; }, false);
    const int G = ws.nround[N];
    for (int v = tm.t; v < V; v += NT) {
        const int b = ws.blk[v];
        ws.group_of[v] = (b ? ws.nround[b - 1] : 0) + ws.rnd[v];
    }
    tm.sync();

    // ---- member lists of each group, ordered by id
    for (int g = tm.t; g <= G; g += NT) {
        ws.gfill[g] = 0;
        ws.gstart[g + 1] = 0;
    }
    if (lead) ws.gstart[0] = 0;
    tm.sync();
    for (int v = tm.t; v < V; v += NT) atomicAdd(&ws.gstart[ws.group_of[v] + 1], 1);
    tm.sync();
    team_scan_inplace(tm, ws.gstart + 1, G, [](uint64_t x, uint64_t y) { return x + y; }, false);
    for (int v = tm.t; v < V; v += NT) {
        const int g = ws.group_of[v];
        const int p = atomicAdd(&ws.gfill[g], 1);
        ws.gtmp[ws.gstart[g] + p] = (uint16_t)v;
    }
    tm.sync();
    for (int i = tm.t; i < V; i += NT) {
        const int v = ws.gtmp[i];
        const int g = ws.group_of[v];
        int pos = 0;
        for (int j = ws.gstart[g]; j < ws.gstart[g + 1]; j++) pos += ws.gtmp[j] < v;
        ws.gmem[ws.gstart[g] + pos] = (uint16_t)v;
    }
    tm.sync();

    // ---- Alg.2 over the groups in order, with Lemma 1 and Theorem 1
    for (int v = tm.t; v < V; v += NT) {
        ws.rem[v] = ws.load[v];
        ws.cnt[v] = ws.indeg[v];  // predecessors not yet finished
        ws.st[v] = 0;
        ws.mm[v] = 0;
    }
    for (int w = tm.t; w < W; w += NT) ws.relmask[w] = 0;
    tm.sync();
    // released set as a bit mask over ranks (W^anc descending), so the next parallel
    // node to consider is always the lowest set bit
    for (int v = tm.t; v < V; v += NT)
        if (ws.indeg[v] == 0)
            atomicOr((unsigned long long *)&ws.relmask[ws.rank[v] >> 6], 1ull << (ws.rank[v] & 63));
    tm.sync();

    const int64_t rbase = 2 * n0;
    const bool want_edges = a.o.extra_off != nullptr;
    int64_t ecap = 0, ebase = 0;
    if (want_edges) {
        ebase = a.o.extra_off[d];
        ecap = a.o.extra_off[d + 1] - ebase;
    }
    uint64_t bound = 0;
    int64_t nextra = 0;
    int nrows = 0, nseg = 0;
    bool internal_err = false;

    for (int j = 0; j < G; j++) {
        const int gb = ws.gstart[j], ge = ws.gstart[j + 1];
        uint32_t cm = 0;
        uint64_t wl = 0;
        for (int i = gb + tm.t; i < ge; i += NT) {
            const int v = ws.gmem[i];
            if (!(ws.st[v] & ST_DONE)) {
                cm++;
                wl += ws.rem[v];
            }
        }
        const uint32_t np = (uint32_t)tm.sum(cm);
        if (np == 0) {  // every member already ran as a parallel node: the group is dropped
            if (lead && a.o.group_R) a.o.group_R[n0 + j] = 0;
            continue;
        }
        const uint64_t Wg = tm.sum(wl);
        // Eq.5: m_i = min(m_i^max, round(C^_i M / W(pi_j))), half up, >= 1
        uint64_t sml = 0;
        for (int i = gb + tm.t; i < ge; i += NT) {
            const int v = ws.gmem[i];
            if (ws.st[v] & ST_DONE) continue;
            uint64_t r = (2ull * ws.rem[v] * M + Wg) / (2ull * Wg);
            if (r < 1) r = 1;
            const uint32_t m = (uint32_t)(r < ws.rem[v] ? r : ws.rem[v]);
            ws.mm[v] = (uint16_t)m;
            sml += m;
        }
        uint64_t sum_m = tm.sum(sml);
        tm.sync();
        while (sum_m > M) {  // keep sum m_i <= M: trim the largest m (ties: higher id)
            uint64_t key = 0;
            for (int i = gb + tm.t; i < ge; i += NT) {
                const int v = ws.gmem[i];
                if (ws.st[v] & ST_DONE) continue;
                const uint64_t kv = ((uint64_t)ws.mm[v] << 16) | (uint64_t)v;
                key = kv > key ? kv : key;
            }
            key = tm.maxu(key);
            if (lead) ws.mm[key & 0xffff]--;
            sum_m--;
            tm.sync();
        }
        // Eq.1 per member; Lemma 1: R(pi_j) = max C_i; v_R = lowest id with C_i = R
        uint64_t cmax = 0;
        for (int i = gb + tm.t; i < ge; i += NT) {
            const int v = ws.gmem[i];
            if (ws.st[v] & ST_DONE) continue;
            const uint64_t c = exec_time(ws.rem[v], ws.kk[v], ws.mm[v], M);
            cmax = c > cmax ? c : cmax;
        }
        const uint64_t R = tm.maxu(cmax);
        uint64_t vr = KEY_INF;
        for (int i = gb + tm.t; i < ge; i += NT) {
            const int v = ws.gmem[i];
            if (ws.st[v] & ST_DONE) continue;
            if (exec_time(ws.rem[v], ws.kk[v], ws.mm[v], M) == R) vr = (uint64_t)v < vr ? (uint64_t)v : vr;
        }
        const int vR = (int)tm.minu(vr);
        const uint32_t S0 = M - (uint32_t)sum_m;  // Eq.6: remaining SMs
        // plan rows of the members, by id
        for (int base = gb; base < ge; base += NT) {
            const int i = base + tm.t;
            const bool mem = i < ge && !(ws.st[ws.gmem[i]] & ST_DONE);
            uint32_t tot;
            const uint32_t off = tm.excl_sum(mem ? 1u : 0u, &tot);
            if (mem) {
                const int v = ws.gmem[i];
                const int r = nrows + (int)off;
                if (r < 2 * V)
                    write_row(a, rbase, r, v, j, ws.rem[v], ws.kk[v], ws.mm[v],
                              exec_time(ws.rem[v], ws.kk[v], ws.mm[v], M), false);
            }
            nrows += (int)tot;
        }
        tm.sync();

        // Alg.2 lines 7-17: parallel nodes by descending W^anc (lowest rank first)
        if (lead) {
            int nl = 0, nwhole = 0, nr = nrows, ns = nseg;
            if (variant != DAGRT_VAR_NOPARA) {
                uint32_t S = S0;
                uint64_t WS = R * (uint64_t)S0;  // Eq.6
                bool stop = false;
                for (int w = 0; w < W && !stop; w++) {
                    uint64_t bits = ws.relmask[w];
                    while (bits) {
                        const int b = __ffsll((long long)bits) - 1;
                        bits &= bits - 1;
                        const int u = ws.byrank[w * 64 + b];
                        if (ws.group_of[u] == j) continue;  // a member of pi_j
                        const uint32_t load = ws.rem[u], k = ws.kk[u];
                        bool split = false;
                        uint32_t mu = 0;
                        uint64_t p = 0;
                        if (variant == DAGRT_VAR_LITERAL) {
                            if (WS == 0) { stop = true; break; }
                            if (load > WS) {
                                split = true;
                                p = WS;
                                mu = (uint32_t)(p < S ? p : S);
                            } else {
                                mu = load < S ? load : S;
                                WS -= load;
                            }
                        } else {
                            if (S == 0) { stop = true; break; }
                            mu = load < S ? load : S;
                            if (exec_time(load, k, mu, M) > R) {
                                if (variant == DAGRT_VAR_NOSEG) continue;
                                split = true;
                                p = split_size(load, k, S, R);
                                mu = (uint32_t)(p < S ? p : S);
                            } else {
                                S -= mu;
                            }
                        }
                        if (split) {  // node segmentation: the parallel part runs now
                            const int s = ns++;
                            if (a.o.seg_parent) {
                                a.o.seg_parent[n0 + s] = u;
                                a.o.seg_load[n0 + s] = (int64_t)p;
                                a.o.seg_m[n0 + s] = (int32_t)mu;
                                a.o.seg_group[n0 + s] = j;
                            }
                            if (nr < 2 * V)
                                write_row(a, rbase, nr, V + s, j, (uint32_t)p, k, mu,
                                          exec_time(p, k, mu, M), false);
                            nr++;
                            ws.rem[u] = load - (uint32_t)p;
                            ws.lst[nl++] = V + s;
                            stop = true;
                            break;
                        }
                        ws.st[u] |= ST_LAUNCH;
                        ws.mm[u] = (uint16_t)mu;
                        if (nr < 2 * V)
                            write_row(a, rbase, nr, u, j, load, k, mu, exec_time(load, k, mu, M), false);
                        nr++;
                        ws.lst[nl++] = u;
                        nwhole++;
                    }
                }
            }
            if (nr - 1 < 2 * V) a.plan_mkf[rbase + nr - 1] |= 1u << 24;  // last row of pi_j
            if (nr > 2 * V || ns > V) internal_err = true;
            sc[1] = nl;
            sc[2] = nwhole;
            sc[3] = nr;
            sc[4] = ns;
            sc[5] = internal_err;
        }
        tm.sync();
        const int nl = sc[1], nwhole = sc[2];
        nrows = sc[3];
        nseg = sc[4];

        // extra dependencies: (v_n, succ(v_R)) for launched parts, (v_R, v_n) for the
        // unlaunched parallel nodes (the split node's residual included)
        const int outdeg = rp[vR + 1] - rp[vR];
        uint32_t qp = 0;
        for (int w = tm.t; w < W; w += NT) qp += __popcll(ws.relmask[w]);
        const int64_t nq = (int64_t)tm.sum(qp) - np;  // |para(pi_j)|
        if (variant != DAGRT_VAR_NOPARA) {
            if (want_edges && lead) {
                int64_t idx = nextra;
                for (int i = 0; i < nl; i++)
                    for (int e = rp[vR]; e < rp[vR + 1]; e++, idx++)
                        if (idx < ecap) {
                            a.o.extra_src[ebase + idx] = ws.lst[i];
                            a.o.extra_dst[ebase + idx] = col[e];
                        }
                for (int w = 0; w < W; w++) {
                    uint64_t bits = ws.relmask[w];
                    while (bits) {
                        const int b = __ffsll((long long)bits) - 1;
                        bits &= bits - 1;
                        const int u = ws.byrank[w * 64 + b];
                        if (ws.group_of[u] == j || (ws.st[u] & ST_LAUNCH)) continue;
                        if (idx < ecap) {
                            a.o.extra_src[ebase + idx] = vR;
                            a.o.extra_dst[ebase + idx] = u;
                        }
                        idx++;
                    }
                }
            }
            nextra += (int64_t)nl * outdeg + (nq - nwhole);
        }
        tm.sync();

        // members and whole launches finish with pi_j: release their successors
        for (int i = gb + tm.t; i < ge + nl; i += NT) {
            int v;
            if (i < ge) {
                v = ws.gmem[i];
                if (ws.st[v] & ST_DONE) continue;
            } else {
                v = ws.lst[i - ge];
                if (v >= V) continue;  // a segment: its node is not finished
            }
            ws.st[v] = ST_DONE;
            ws.rem[v] = 0;
            if (a.o.exec_group) a.o.exec_group[n0 + v] = j;
            atomicAnd((unsigned long long *)&ws.relmask[ws.rank[v] >> 6], ~(1ull << (ws.rank[v] & 63)));
            for (int e = rp[v]; e < rp[v + 1]; e++) {
                const int s = col[e];
                if (atomicSub(&ws.cnt[s], 1) == 1)
                    atomicOr((unsigned long long *)&ws.relmask[ws.rank[s] >> 6], 1ull << (ws.rank[s] & 63));
            }
        }
        if (lead && a.o.group_R) a.o.group_R[n0 + j] = (int64_t)R;
        bound += R;
        tm.sync();
    }
    internal_err = sc[5] != 0 && G > 0;

    // ---- per-DAG and per-node outputs
    int code = DAGRT_OK;
    if (internal_err) code = DAGRT_E_INTERNAL;
    else if (want_edges && nextra > ecap) code = DAGRT_E_CAP;
    if (lead) {
        a.status[d] = code;
        a.bound[d] = code == DAGRT_E_INTERNAL ? -1 : (int64_t)bound;
        a.nrows[d] = nrows;
        if (a.o.status) a.o.status[d] = code;
        if (a.o.bound) a.o.bound[d] = code == DAGRT_E_INTERNAL ? -1 : (int64_t)bound;
        if (a.o.n_groups) a.o.n_groups[d] = G;
        if (a.o.n_seg) a.o.n_seg[d] = nseg;
        if (a.o.n_rows) a.o.n_rows[d] = nrows;
        if (a.o.n_extra) a.o.n_extra[d] = nextra;
    }
    for (int v = tm.t; v < V; v += NT) {
        if (a.o.wanc) a.o.wanc[n0 + v] = (int64_t)ws.wanc[v];
        if (a.o.block_of) a.o.block_of[n0 + v] = ws.blk[v];
        if (a.o.group_of) a.o.group_of[n0 + v] = ws.group_of[v];
        if (a.o.m) a.o.m[n0 + v] = ws.mm[v];
    }
    tm.sync();
}

// ------------------------------------------------------------------ kernels
template <int VC>
__global__ void __launch_bounds__(32 * kWarpsPerCta) k_sched_warp(SchedArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5;
    Ws ws;
    const int64_t bytes = ws_carve(nullptr, VC, nullptr);
    ws_carve(smem + warp * bytes, VC, &ws);
    Team<32> tm{(int)(threadIdx.x & 31), nullptr};
    for (;;) {
        int idx = 0;
        if (tm.t == 0) idx = atomicAdd(a.counter, 1);
        idx = __shfl_sync(FULL, idx, 0);
        if (idx >= a.n_list) break;
        schedule_one<32>(tm, ws, a, a.list[idx], VC);
        __syncwarp();
    }
}

template <int NT>
__global__ void __launch_bounds__(NT) k_sched_cta(SchedArgs a) {
    __shared__ uint64_t red[NT / 32];
    __shared__ int idx_s;
    Ws ws;
    ws_carve(a.gws + (int64_t)blockIdx.x * a.gws_stride, a.vcap, &ws);
    Team<NT> tm{(int)threadIdx.x, red};
    for (;;) {
        if (threadIdx.x == 0) idx_s = atomicAdd(a.counter, 1);
        __syncthreads();
        const int idx = idx_s;
        __syncthreads();
        if (idx >= a.n_list) break;
        schedule_one<NT>(tm, ws, a, a.list[idx], a.vcap);
        __syncthreads();
    }
}

// ------------------------------------------------------------------ launchers
template <int VC>
static cudaError_t launch_warp(const SchedArgs &a, int n_sm, cudaStream_t st) {
    const int64_t bytes = ws_carve(nullptr, VC, nullptr) * kWarpsPerCta;
    cudaError_t e = cudaFuncSetAttribute(k_sched_warp<VC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)bytes);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sched_warp<VC>, 32 * kWarpsPerCta, bytes);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int grid = n_sm * per_sm;
    const int need = ceil_div(a.n_list, kWarpsPerCta);
    if (grid > need) grid = need;
    if (grid < 1) return cudaSuccess;
    k_sched_warp<VC><<<grid, 32 * kWarpsPerCta, bytes, st>>>(a);
    return cudaGetLastError();
}

cudaError_t sched_launch_warp(int vc, const SchedArgs &a, int n_sm, cudaStream_t st) {
    switch (vc) {
        case 64: return launch_warp<64>(a, n_sm, st);
        case 128: return launch_warp<128>(a, n_sm, st);
        case 256: return launch_warp<256>(a, n_sm, st);
        default: return cudaErrorInvalidValue;
    }
}

int sched_cta_grid(int n_sm) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sched_cta<kCtaThreads>, kCtaThreads, 0) !=
            cudaSuccess || per_sm < 1)
        per_sm = 1;
    return n_sm * per_sm;
}

cudaError_t sched_launch_cta(const SchedArgs &a, int grid, cudaStream_t st) {
    if (grid < 1 || a.n_list < 1) return cudaSuccess;
    k_sched_cta<kCtaThreads><<<grid, kCtaThreads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace dagrt
