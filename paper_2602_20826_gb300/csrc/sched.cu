// sched.cu -- per-DAG scheduling and bound kernels (Alg.1, Alg.2, Lemma 1, Theorem 1).
//
// One team (a warp for DAGs that fit a shared-memory workspace, a CTA otherwise) takes a
// whole DAG from a work-stealing counter and runs every step of the method on it without
// leaving its workspace: CSR validation, Kahn levels, the ancestor closure and W^anc
// (Eq.2), Theta and the blocks of Eq.3, the balanced groups of Alg.1, the scheduling loop
// of Alg.2 and the bound of Theorem 1. The schedule is written out as "plan rows" that the
// candidate-bound kernel evaluates other allocations on.
//
// Alg.2 is sequential over the groups of a DAG. Groups with few members (the common case)
// are scheduled by one thread of the team with plain loads and stores and no team-wide
// barrier; large groups use the whole team.
#include <map>
#include <mutex>
#include <utility>

#include "dagrt_internal.cuh"
#include "sched.cuh"

namespace dagrt {

// node state bits
enum : uint8_t { ST_ACTIVE = 1, ST_INT = 2, ST_SEL = 4, ST_DONE = 8, ST_LAUNCH = 16, ST_JOIN = 32 };
constexpr uint16_t NONE16 = 0xffff;
constexpr int kSumWords = 8;  // released-set masks longer than this keep a summary of non-empty words

// ------------------------------------------------------------------ workspace layout
// Persistent arrays live for the whole DAG; the region after them is overlaid by the
// arrays of one phase at a time (A closure, B ordering, C peeling, D member lists, E Alg.2).
struct Ws {
    // persistent
    uint32_t *load;
    uint8_t *kk, *st;
    int32_t *cnt;  // atomic counters: in-degree, Kahn count, in-block parents, open preds
    uint32_t *srp;  // the DAG's successor CSR, staged: offsets ...
    uint16_t *scol; // ... and successor ids
    uint16_t *indeg, *lvl_off, *topo, *rank, *byrank, *blk, *group_of, *gstart, *gmem;
    uint64_t *relmask;
    uint64_t *relsum;  // bit w: relmask[w] may be non-zero (cleared lazily by the scan)
    int32_t *sc;
    // phase A (+ wanc, kept through phase B)
    uint64_t *wanc, *anc, *planes;
    int32_t *poff;  // CTA teams: predecessor lists by node (inclusive offsets) ...
    uint16_t *pid;  // ... and their entries
    // phase B
    uint64_t *skey;
    uint16_t *bk, *pos;
    int32_t *jcnt, *rs, *re;
    // phase C
    int32_t *fcnt, *nround;
    uint64_t *bigk;
    uint16_t *rnd;
    int32_t *thr, *ovl;  // per over-full block: rank of its M-th head; list of over-full blocks
    uint16_t *fr0, *fr1; // the heads of the current round and of the next one (Alg.1)
    uint64_t *hmask;     // CTA teams, Top_M of an over-full block: its heads by rank, one bit each
    int32_t *hcnt;       // ... and the heads in rank words 0..w
    // phase D
    uint16_t *gtmp;
    int32_t *gfill;
    // phase E
    uint32_t *rem, *cfull;
    uint16_t *mm;
    int32_t *lst, *tmp;
    // phase F (after Alg.2): the critical-path lower bound
    uint64_t *cpT, *cpM;
};

__host__ __device__ inline int pow2_ceil(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

// Carve a workspace for DAGs of up to vc nodes and ec edges out of `base`; returns the
// bytes used.
__host__ __device__ inline int64_t ws_carve(unsigned char *base, int vc, int ec, Ws *ws, bool cta = false) {
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
    w.kk = (uint8_t *)take(vc);
    w.st = (uint8_t *)take(vc);
    w.cnt = (int32_t *)take(4ll * vc);
    w.srp = (uint32_t *)take(4ll * (vc + 1));
    w.scol = (uint16_t *)take(2ll * (ec > 0 ? ec : 1));
    w.indeg = (uint16_t *)take(2ll * vc);
    w.lvl_off = (uint16_t *)take(2ll * (vc + 1));
    w.topo = (uint16_t *)take(2ll * vc);
    w.rank = (uint16_t *)take(2ll * vc);
    w.byrank = (uint16_t *)take(2ll * vc);
    w.blk = (uint16_t *)take(2ll * vc);
    w.group_of = (uint16_t *)take(2ll * vc);
    w.gstart = (uint16_t *)take(2ll * (vc + 2));
    w.gmem = (uint16_t *)take(2ll * vc);
    w.relmask = (uint64_t *)take(8ll * W);
    w.relsum = (uint64_t *)take(8ll * ((W + 63) / 64));
    w.sc = (int32_t *)take(4 * 16);
    const int64_t x0 = off;
    int64_t end = off;
    auto mark = [&]() { end = off > end ? off : end; };
    w.wanc = (uint64_t *)take(8ll * vc);
    const int64_t xa = off;  // phases A and B keep wanc
    w.anc = (uint64_t *)take(8ll * vc * W);
    w.planes = (uint64_t *)take(8ll * 32 * W);
    w.poff = cta ? (int32_t *)take(4ll * (vc + 1)) : nullptr;
    w.pid = cta ? (uint16_t *)take(2ll * (ec > 0 ? ec : 1)) : nullptr;
    mark();
    off = xa;
    w.skey = (uint64_t *)take(8ll * P);
    w.bk = (uint16_t *)take(2ll * vc);
    w.pos = (uint16_t *)take(2ll * vc);
    w.jcnt = (int32_t *)take(4ll * vc);
    w.rs = (int32_t *)take(4ll * vc);
    w.re = (int32_t *)take(4ll * vc);
    mark();
    off = x0;
    w.fcnt = (int32_t *)take(4ll * (vc + 1));
    w.nround = (int32_t *)take(4ll * (vc + 1));
    w.bigk = (uint64_t *)take(8ll * (vc + 1));
    w.rnd = (uint16_t *)take(2ll * vc);
    w.thr = (int32_t *)take(4ll * (vc + 1));
    w.ovl = (int32_t *)take(4ll * (vc + 1));
    w.fr0 = (uint16_t *)take(2ll * vc);
    w.fr1 = (uint16_t *)take(2ll * vc);
    w.hmask = (uint64_t *)take(8ll * W);
    w.hcnt = (int32_t *)take(4ll * W);
    mark();
    off = x0;
    w.gtmp = (uint16_t *)take(2ll * vc);
    w.gfill = (int32_t *)take(4ll * (vc + 1));
    mark();
    off = x0;
    w.rem = (uint32_t *)take(4ll * vc);
    w.cfull = (uint32_t *)take(4ll * vc);
    w.mm = (uint16_t *)take(2ll * vc);
    w.lst = (int32_t *)take(4ll * (vc + 1));
    w.tmp = (int32_t *)take(4ll * vc);
    mark();
    off = x0;
    w.cpT = (uint64_t *)take(8ll * vc);
    w.cpM = (uint64_t *)take(8ll * vc);
    mark();
    if (ws) *ws = w;
    return align_up(end, 128);
}

int64_t sched_ws_bytes(int vc, int ec) { return ws_carve(nullptr, vc, ec, nullptr, true); }

// ------------------------------------------------------------------ per-DAG context
struct Dag {
    int64_t n0, rbase, ebase, ecap;
    int V, W, variant;
    uint32_t M;
    bool want_edges;
    const uint32_t *rp;  // staged CSR
    const uint16_t *col;
};

// Alg.2 running totals, held by the team's first thread
struct Acc {
    uint64_t bound;
    int64_t nextra;
    int nrows, nseg, nrel;  // plan rows, segments, released-and-unfinished nodes
    bool err;
    int lastr;       // the last plan row written by this thread (-1: unknown) ...
    uint32_t lastz;  // ... and its packed m | k << 16, to mark it as the group's last row
};

__device__ inline void write_failure(const SchedArgs &a, int d, int code) {
    a.status[d] = code;
    a.bound[d] = -1;
    if (a.nrows) a.nrows[d] = 0;
    if (a.o.status) a.o.status[d] = code;
    if (a.o.bound) a.o.bound[d] = -1;
    if (a.o.n_groups) a.o.n_groups[d] = 0;
    if (a.o.n_seg) a.o.n_seg[d] = 0;
    if (a.o.n_rows) a.o.n_rows[d] = 0;
    if (a.o.n_extra) a.o.n_extra[d] = 0;
    if (a.o.greedy) a.o.greedy[d] = -1;
    if (a.o.greedy_unaware) a.o.greedy_unaware[d] = -1;
    if (a.o.graham_para) a.o.graham_para[d] = -1;
    if (a.o.crit_path) a.o.crit_path[d] = -1;
}

// Greedy + unaware kernel time (baseline of the Evaluation section): the kernel runs on
// m = x SMs whatever M is, so Eq.1's wave factor ceil(x / M) applies. Exact in 128-bit
// arithmetic, saturated at 2^63 - 1.
__device__ __forceinline__ uint64_t exec_time_unaware(uint64_t x, uint32_t k, uint32_t M) {
    const unsigned __int128 waves = (x + M - 1) / M;
    const unsigned __int128 num = waves * x * (64ull * x - (uint64_t)k * (x - 1));
    const unsigned __int128 den = 64ull * x;
    const unsigned __int128 c = (num + den - 1) / den;
    return c > (unsigned __int128)INT64_MAX ? (uint64_t)INT64_MAX : (c < 1 ? 1ull : (uint64_t)c);
}
__device__ __forceinline__ uint64_t sat_add(uint64_t a, uint64_t b) {
    const uint64_t s = a + b;
    return s > (uint64_t)INT64_MAX || s < a ? (uint64_t)INT64_MAX : s;
}

// plan row r: `id` is the node (< V) or segment (>= V) it runs, `owner` the node whose
// allocation it uses (the segment's parent for a segment)
__device__ inline uint32_t write_row(const SchedArgs &a, const Dag &g, int r, int id, int owner, int group,
                                     uint32_t load, uint32_t k, uint32_t m, uint64_t c) {
    const uint32_t z = m | (k << 16);
    if (r >= 2 * g.V) return z;
    const int64_t i = g.rbase + r;
    if (a.plan) a.plan[i] = make_uint4(load, (uint32_t)c, z, (uint32_t)owner);
    if (a.o.row_id) a.o.row_id[i] = id;
    if (a.o.row_group) a.o.row_group[i] = group;
    if (a.o.row_m0) a.o.row_m0[i] = (int32_t)m;
    if (a.o.row_load) a.o.row_load[i] = load;
    return z;
}

// ------------------------------------------------------------------ Alg.2 pieces
// Launch parallel nodes for group j (Alg.2's parallel-launch and segmentation step): released, unfinished nodes outside
// pi_j in descending W^anc order (lowest rank first). One thread. Returns the number of
// launched parts (ids in ws.lst; a segment id is >= V) and of whole-node launches.
template <bool SUM>
__device__ __forceinline__ void launch_parallel(const Ws &ws, const SchedArgs &a, const Dag &g, int j, uint64_t R, uint32_t S0,
                                Acc &acc, int *nl_out, int *nwhole_out) {
    int nl = 0, nwhole = 0;
    const uint32_t M = g.M;
    // no SMs left (S = 0, so also WS = 0): every variant stops at its first candidate
    if (g.variant != DAGRT_VAR_NOPARA && S0 > 0) {
        uint32_t S = S0;
        uint64_t WS = R * (uint64_t)S0;  // Eq.6
        bool stop = false;
        // the mask's words in order (lowest rank first); a long mask (SUM) is walked through
        // its summary of possibly non-empty words
        int w = -1, sw = -1;
        uint64_t sbits = 0;
        while (!stop) {
            if constexpr (SUM) {
                while (!sbits && ++sw < ((g.W + 63) >> 6)) sbits = ws.relsum[sw];
                if (!sbits) break;
                w = sw * 64 + __ffsll((long long)sbits) - 1;
                sbits &= sbits - 1;
            } else {
                if (++w >= g.W) break;
            }
            uint64_t bits = ws.relmask[w];
            if (SUM && !bits) {  // emptied since it was marked
                ws.relsum[sw] &= ~(1ull << (w & 63));
                continue;
            }
            while (bits) {
                const int b = __ffsll((long long)bits) - 1;
                bits &= bits - 1;
                const int u = ws.byrank[w * 64 + b];
                if (ws.group_of[u] == j) continue;  // a member of pi_j
                const uint32_t load = ws.rem[u], k = ws.kk[u];
                bool split = false;
                uint32_t mu = 0;
                uint64_t p = 0, c = 0;
                if (g.variant == DAGRT_VAR_LITERAL) {
                    if (WS == 0) { stop = true; break; }
                    if (load > WS) {
                        split = true;
                        p = WS;
                        mu = (uint32_t)(p < S ? p : S);
                    } else {
                        mu = load < S ? load : S;
                        WS -= load;
                        c = exec_time(load, k, mu, M);
                    }
                } else {
                    if (S == 0) { stop = true; break; }
                    mu = load < S ? load : S;
                    // fits within R on mu <= M SMs: ceil(load (64mu - k(mu-1)) / (64mu)) <= R
                    const uint64_t lhs = (uint64_t)load * (64ull * mu - (uint64_t)k * (mu - 1));
                    if (lhs > 64ull * mu * R) {
                        if (g.variant == DAGRT_VAR_NOSEG) continue;
                        split = true;
                        p = split_size(load, k, S, R);
                        mu = (uint32_t)(p < S ? p : S);
                    } else {
                        c = exec_time(load, k, mu, M);
                        S -= mu;
                    }
                }
                if (split) {  // node segmentation: the parallel part runs now
                    const int s = acc.nseg++;
                    if (a.o.seg_parent) {
                        a.o.seg_parent[g.n0 + s] = u;
                        a.o.seg_load[g.n0 + s] = (int64_t)p;
                        a.o.seg_m[g.n0 + s] = (int32_t)mu;
                        a.o.seg_group[g.n0 + s] = j;
                    }
                    acc.lastr = acc.nrows;
                    acc.lastz = write_row(a, g, acc.nrows++, g.V + s, u, j, (uint32_t)p, k, mu, exec_time(p, k, mu, M));
                    ws.rem[u] = load - (uint32_t)p;
                    ws.lst[nl++] = g.V + s;
                    stop = true;
                    break;
                }
                ws.st[u] |= ST_LAUNCH;
                ws.mm[u] = (uint16_t)mu;
                acc.lastr = acc.nrows;
                acc.lastz = write_row(a, g, acc.nrows++, u, u, j, load, k, mu, c);
                ws.lst[nl++] = u;
                nwhole++;
            }
        }
    }
    if (a.plan && acc.nrows - 1 < 2 * g.V) {  // mark the last row of pi_j
        if (acc.lastr == acc.nrows - 1)
            a.plan[g.rbase + acc.nrows - 1].z = acc.lastz | (1u << 24);  // a plain store: no read back
        else
            a.plan[g.rbase + acc.nrows - 1].z |= 1u << 24;
    }
    if (acc.nrows > 2 * g.V || acc.nseg > g.V) acc.err = true;
    *nl_out = nl;
    *nwhole_out = nwhole;
}

// Extra dependencies (Alg.2's segmentation step): (v_n, succ(v_R)) for every launched part and
// (v_R, v_n) for every unlaunched parallel node, the split node's residual included. The
// count is always kept; the edges are written when requested. One thread.
__device__ void extra_edges(const Ws &ws, const SchedArgs &a, const Dag &g, int j, int vR, int np, int nl,
                            int nwhole, Acc &acc) {
    if (g.variant == DAGRT_VAR_NOPARA) return;
    const int outdeg = g.rp[vR + 1] - g.rp[vR];
    if (g.want_edges) {
        int64_t idx = acc.nextra;
        for (int i = 0; i < nl; i++)
            for (int e = g.rp[vR]; e < g.rp[vR + 1]; e++, idx++)
                if (idx < g.ecap) {
                    a.o.extra_src[g.ebase + idx] = ws.lst[i];
                    a.o.extra_dst[g.ebase + idx] = g.col[e];
                }
        for (int w = 0; w < g.W; w++) {
            uint64_t bits = ws.relmask[w];
            while (bits) {
                const int b = __ffsll((long long)bits) - 1;
                bits &= bits - 1;
                const int u = ws.byrank[w * 64 + b];
                if (ws.group_of[u] == j || (ws.st[u] & ST_LAUNCH)) continue;
                if (idx < g.ecap) {
                    a.o.extra_src[g.ebase + idx] = vR;
                    a.o.extra_dst[g.ebase + idx] = u;
                }
                idx++;
            }
        }
    }
    acc.nextra += (int64_t)nl * outdeg + (int64_t)(acc.nrel - np - nwhole);
}

// Group j (any size in warp teams, at most 32 members in CTA teams): lane 0 of the team's
// first warp runs Eq.5, Lemma 1, the parallel launches and the extra edges serially; the 32
// lanes then release the finished nodes' successors together (the decrements commute).
// `acc` is valid in lane 0 only.
__device__ void group_serial(const Ws &ws, const SchedArgs &a, const Dag &g, int j, Acc &acc, int lane) {
    int nf = 0;
    uint64_t R = 0;
    if (lane == 0) {
        const uint32_t M = g.M;
        const int gb = ws.gstart[j], ge = ws.gstart[j + 1];
        int np = 0, vR = -1;
        uint32_t sum_m = 0;
        if (ge - gb == 1) {  // one member: Eq.5 gives m = min(C^, M)
            const int v = ws.gmem[gb];
            if (!(ws.st[v] & ST_DONE)) {
                np = 1;
                const uint32_t x = ws.rem[v], m = x < M ? x : M;
                ws.mm[v] = (uint16_t)m;
                sum_m = m;
                const uint64_t c = x == ws.load[v] ? ws.cfull[v] : exec_time(x, ws.kk[v], m, M);
                R = c;
                vR = v;
                acc.lastr = acc.nrows;
                acc.lastz = write_row(a, g, acc.nrows++, v, v, j, x, ws.kk[v], m, c);
            }
        } else {
            uint64_t Wg = 0;
            for (int i = gb; i < ge; i++) {
                const int v = ws.gmem[i];
                if (!(ws.st[v] & ST_DONE)) {
                    np++;
                    Wg += ws.rem[v];
                }
            }
            if (np > 0) {
                // Eq.5; a single member gets round(C^ M / C^) = M, i.e. m = min(C^, M)
                for (int i = gb; i < ge; i++) {
                    const int v = ws.gmem[i];
                    if (ws.st[v] & ST_DONE) continue;
                    const uint32_t x = ws.rem[v];
                    uint32_t m;
                    if (np == 1) {
                        m = x < M ? x : M;
                    } else {
                        const uint64_t num = 2ull * x * M + Wg, den = 2ull * Wg;
                        uint64_t r = (num >> 32) == 0 && (den >> 32) == 0 ? (uint64_t)((uint32_t)num / (uint32_t)den)
                                                                          : num / den;
                        if (r < 1) r = 1;
                        m = (uint32_t)(r < x ? r : x);
                    }
                    ws.mm[v] = (uint16_t)m;
                    sum_m += m;
                }
                // keep sum m_i <= M: trim the largest m (ties: higher id); the no-repair
                // variant leaves the rounded SMs as they are
                while (g.variant != DAGRT_VAR_NOREPAIR && sum_m > M) {
                    int best = -1;
                    for (int i = gb; i < ge; i++) {
                        const int v = ws.gmem[i];
                        if (ws.st[v] & ST_DONE) continue;
                        if (best < 0 || ws.mm[v] >= ws.mm[best]) best = v;
                    }
                    ws.mm[best]--;
                    sum_m--;
                }
                // Eq.1 per member and Lemma 1: R(pi_j) = max C_i, v_R = lowest id with C_i = R
                uint64_t csum = 0;
                for (int i = gb; i < ge; i++) {
                    const int v = ws.gmem[i];
                    if (ws.st[v] & ST_DONE) continue;
                    const uint32_t x = ws.rem[v], m = ws.mm[v];
                    const uint64_t c =
                        (x == ws.load[v] && m == (x < M ? x : M)) ? ws.cfull[v] : exec_time(x, ws.kk[v], m, M);
                    csum += c;
                    if (c > R) {
                        R = c;
                        vR = v;
                    }
                    acc.lastr = acc.nrows;
                    acc.lastz = write_row(a, g, acc.nrows++, v, v, j, x, ws.kk[v], m, c);
                }
                if (sum_m > M) R = csum;  // over-full (no repair): members one after another
            }
        }
        if (np == 0) {  // every member already ran as a parallel node: the group is dropped
            if (a.o.group_R) a.o.group_R[g.n0 + j] = 0;
        } else {
            int nl, nwhole;
            const uint32_t S0 = sum_m < M ? M - sum_m : 0u;
            if (g.W > kSumWords)
                launch_parallel<true>(ws, a, g, j, R, S0, acc, &nl, &nwhole);
            else
                launch_parallel<false>(ws, a, g, j, R, S0, acc, &nl, &nwhole);
            extra_edges(ws, a, g, j, vR, np, nl, nwhole, acc);
            nf = ge - gb + nl;  // candidates to finish: the members, then the launched parts
            if (a.o.group_R) a.o.group_R[g.n0 + j] = (int64_t)R;
            acc.bound += R;
        }
    }
    __syncwarp();  // lane 0's shared-memory writes (launch list, states) become visible
    // members (not finished before) and whole launches finish with pi_j: one lane each
    const int gb = __shfl_sync(FULL, lane == 0 ? (int)ws.gstart[j] : 0, 0);
    const int ncand = __shfl_sync(FULL, nf, 0);
    int nfin = 0;
    for (int base = 0; base < ncand; base += 32) {
        const int i = base + lane;
        int v = -1;
        if (i < ncand) {
            const int ge = ws.gstart[j + 1];
            if (gb + i < ge) {
                v = ws.gmem[gb + i];
                if (ws.st[v] & ST_DONE) v = -1;
            } else {
                v = ws.lst[gb + i - ge];
                if (v >= g.V) v = -1;  // a segment: its node is not finished
            }
        }
        const uint32_t fin = __ballot_sync(FULL, v >= 0);
        if (v >= 0) {
            ws.st[v] = ST_DONE;
            ws.rem[v] = 0;
            if (a.o.exec_group) a.o.exec_group[g.n0 + v] = j;
            atomicAnd((unsigned long long *)&ws.relmask[ws.rank[v] >> 6], ~(1ull << (ws.rank[v] & 63)));
            ws.tmp[nfin + __popc(fin & ((1u << lane) - 1))] = v;
        }
        nfin += __popc(fin);
    }
    if (lane == 0) acc.nrel -= nfin;
    nf = nfin;
    __syncwarp();
    // ... and release their successors
    int released = 0;
    for (int f = 0; f < nf; f++) {
        const int v = ws.tmp[f];
        for (int e = g.rp[v] + lane; e < g.rp[v + 1]; e += 32) {
            const int s = g.col[e];
            if (atomicSub(&ws.cnt[s], 1) == 1) {
                atomicOr((unsigned long long *)&ws.relmask[ws.rank[s] >> 6], 1ull << (ws.rank[s] & 63));
                if (g.W > kSumWords)
                    atomicOr((unsigned long long *)&ws.relsum[ws.rank[s] >> 12], 1ull << ((ws.rank[s] >> 6) & 63));
                released++;
            }
        }
    }
    released = __reduce_add_sync(FULL, released);
    if (lane == 0) acc.nrel += released;
    __syncwarp();
}

// Group j scheduled by the whole CTA team (groups of more than 32 members). `acc` is only valid in
// the team's first thread; sc[8] carries acc.nrows to the others.
template <int NT>
__device__ void group_team(const Team<NT> &tm, const Ws &ws, const SchedArgs &a, const Dag &g, int j, Acc &acc) {
    const uint32_t M = g.M;
    const bool lead = tm.t == 0;
    volatile int32_t *sc = ws.sc;
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
    if (np == 0) {
        if (lead && a.o.group_R) a.o.group_R[g.n0 + j] = 0;
        return;
    }
    const uint64_t Wg = tm.sum(wl);
    uint64_t sml = 0;
    for (int i = gb + tm.t; i < ge; i += NT) {
        const int v = ws.gmem[i];
        if (ws.st[v] & ST_DONE) continue;
        const uint64_t num = 2ull * ws.rem[v] * M + Wg, den = 2ull * Wg;
        uint64_t r = (num >> 32) == 0 && (den >> 32) == 0 ? (uint64_t)((uint32_t)num / (uint32_t)den) : num / den;
        if (r < 1) r = 1;
        const uint32_t m = (uint32_t)(r < ws.rem[v] ? r : ws.rem[v]);
        ws.mm[v] = (uint16_t)m;
        sml += m;
    }
    uint64_t sum_m = tm.sum(sml);
    tm.sync();
    while (g.variant != DAGRT_VAR_NOREPAIR && sum_m > M) {
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
    uint64_t ckey = 0, csum = 0;  // (C, 0xffff - id): the max is the largest C, then the lowest id
    for (int i = gb + tm.t; i < ge; i += NT) {
        const int v = ws.gmem[i];
        if (ws.st[v] & ST_DONE) continue;
        const uint64_t c = exec_time(ws.rem[v], ws.kk[v], ws.mm[v], M);
        const uint64_t kv = (c << 16) | (uint64_t)(0xffff - v);
        ckey = kv > ckey ? kv : ckey;
        csum += c;
    }
    ckey = tm.maxu(ckey);
    csum = tm.sum(csum);
    // over-full (no repair only): the members run one after another
    const uint64_t R = sum_m > M ? csum : ckey >> 16;
    const int vR = 0xffff - (int)(ckey & 0xffff);
    int nrows = sc[8];
    for (int base = gb; base < ge; base += NT) {
        const int i = base + tm.t;
        const bool mem = i < ge && !(ws.st[ws.gmem[i]] & ST_DONE);
        uint32_t tot;
        const uint32_t off = tm.excl_sum(mem ? 1u : 0u, &tot);
        if (mem) {
            const int v = ws.gmem[i];
            write_row(a, g, nrows + (int)off, v, v, j, ws.rem[v], ws.kk[v], ws.mm[v],
                      exec_time(ws.rem[v], ws.kk[v], ws.mm[v], M));
        }
        nrows += (int)tot;
    }
    tm.sync();
    if (lead) {
        acc.nrows = nrows;
        acc.lastr = -1;  // the members' rows were written by the team
        int nl, nwhole;
        const uint32_t S0 = sum_m < M ? M - (uint32_t)sum_m : 0u;
        if (g.W > kSumWords)
            launch_parallel<true>(ws, a, g, j, R, S0, acc, &nl, &nwhole);
        else
            launch_parallel<false>(ws, a, g, j, R, S0, acc, &nl, &nwhole);
        extra_edges(ws, a, g, j, vR, (int)np, nl, nwhole, acc);
        sc[1] = nl;
        sc[6] = 0;
        sc[7] = 0;
    }
    tm.sync();
    const int nl = sc[1];
    for (int i = gb + tm.t; i < ge + nl; i += NT) {
        int v;
        if (i < ge) {
            v = ws.gmem[i];
            if (ws.st[v] & ST_DONE) continue;
        } else {
            v = ws.lst[i - ge];
            if (v >= g.V) continue;
        }
        ws.st[v] = ST_DONE;
        ws.rem[v] = 0;
        if (a.o.exec_group) a.o.exec_group[g.n0 + v] = j;
        atomicAnd((unsigned long long *)&ws.relmask[ws.rank[v] >> 6], ~(1ull << (ws.rank[v] & 63)));
        ws.tmp[atomicAdd((int *)&sc[6], 1)] = v;
    }
    tm.sync();
    const int nf = sc[6];
    for (int f = 0; f < nf; f++) {
        const int v = ws.tmp[f];
        for (int e = g.rp[v] + tm.t; e < g.rp[v + 1]; e += NT) {
            const int s = g.col[e];
            if (atomicSub(&ws.cnt[s], 1) == 1) {
                atomicOr((unsigned long long *)&ws.relmask[ws.rank[s] >> 6], 1ull << (ws.rank[s] & 63));
                if (g.W > kSumWords)
                    atomicOr((unsigned long long *)&ws.relsum[ws.rank[s] >> 12], 1ull << ((ws.rank[s] >> 6) & 63));
                atomicAdd((int *)&sc[7], 1);
            }
        }
    }
    tm.sync();
    if (lead) {
        acc.nrel += sc[7] - nf;
        if (a.o.group_R) a.o.group_R[g.n0 + j] = (int64_t)R;
        acc.bound += R;
    }
}

// ------------------------------------------------------------------ one DAG
template <int NT>
__device__ void schedule_one(const Team<NT> &tm, const Ws &ws, const SchedArgs &a, int d, int vc, int ec) {
    const int64_t n0 = a.node_off[d];
    const int V = (int)(a.node_off[d + 1] - n0);
    const int64_t e0 = a.edge_off[d];
    const int64_t E = a.edge_off[d + 1] - e0;
    const int32_t *__restrict__ grp = a.row_ptr + n0 + d;
    const int32_t *__restrict__ gcol = a.col + e0;
    const int64_t *__restrict__ wc = a.wcet + n0;
    const uint8_t *__restrict__ kp = a.k64 + n0;
    const uint32_t M = (uint32_t)a.M;
    volatile int32_t *sc = ws.sc;
    const bool lead = tm.t == 0;

    // does not fit this workspace, or its offsets reach outside the arrays
    if (V < 0 || E < 0 || V > vc || E > ec ||
        (a.tot_nodes >= 0 && (n0 < 0 || n0 + V > a.tot_nodes || e0 < 0 || e0 + E > a.tot_edges))) {
        if (lead) write_failure(a, d, a.oversize_status);
        return;
    }

    // ---- validation: row_ptr shape, then loads and fractions, then successor ids; the
    //      CSR is staged into the workspace on the way (all later phases read the copy)
    bool bad = false;
    if (lead) bad = grp[0] != 0 || (int64_t)grp[V] != E;
    for (int v = tm.t; v <= V; v += NT) {
        const int x = grp[v];
        if (v < V && grp[v + 1] < x) bad = true;
        ws.srp[v] = (uint32_t)x;
    }
    if (tm.any(bad)) {
        if (lead) write_failure(a, d, DAGRT_E_INVAL);
        return;
    }
    bool badv = false, badc = false;
    for (int e = tm.t; e < (int)E; e += NT) {
        const int c = gcol[e];
        if (c < 0 || c >= V) badc = true;
        ws.scol[e] = (uint16_t)c;
    }
    for (int v = tm.t; v < V; v += NT) {
        const int64_t w = wc[v];
        const uint8_t k = kp[v];
        if (w < 1 || w > 0xffffffffll || k > 64) badv = true;
        ws.load[v] = (uint32_t)w;
        ws.kk[v] = k;
        ws.cnt[v] = 0;
    }
    tm.sync();
    const uint32_t *__restrict__ rp = ws.srp;
    const uint16_t *__restrict__ col = ws.scol;
    if (!badc) {  // self loops, unsorted or repeated successors (ids are in range here)
        for (int v = tm.t; v < V; v += NT) {
            int prev = -1;
            for (int e = rp[v]; e < (int)rp[v + 1]; e++) {
                const int c = col[e];
                if (c == v || c <= prev) badc = true;
                prev = c;
            }
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
            if (a.nrows) a.nrows[d] = 0;
            if (a.o.status) a.o.status[d] = DAGRT_OK;
            if (a.o.bound) a.o.bound[d] = 0;
            if (a.o.n_groups) a.o.n_groups[d] = 0;
            if (a.o.n_seg) a.o.n_seg[d] = 0;
            if (a.o.n_rows) a.o.n_rows[d] = 0;
            if (a.o.n_extra) a.o.n_extra[d] = 0;
            if (a.o.greedy) a.o.greedy[d] = 0;
            if (a.o.greedy_unaware) a.o.greedy_unaware[d] = 0;
            if (a.o.graham_para) a.o.graham_para[d] = 0;
            if (a.o.crit_path) a.o.crit_path[d] = 0;
        }
        return;
    }
    tm.sync();

    // ---- in-degrees (a join has at least two predecessors), one edge per thread
    for (int e = tm.t; e < (int)E; e += NT) atomicAdd(&ws.cnt[col[e]], 1);
    const int W = (V + 63) >> 6;
    if constexpr (NT == 32)  // CTA teams write every word of the closure (pulled below)
        for (int i = tm.t; i < V * W; i += NT) ws.anc[i] = 0;
    if (lead) sc[0] = 0;
    tm.sync();

    // ---- Kahn levels, and (warp teams) the ancestor closure pushed along each level's
    //      out-edges: everything that reaches u, and u itself, reaches each successor of u
    for (int v = tm.t; v < V; v += NT) {
        const int dg = ws.cnt[v];
        ws.indeg[v] = (uint16_t)dg;
        ws.st[v] = dg >= 2 ? ST_JOIN : 0;
        if (dg == 0) {
            const int p = atomicAdd((int *)&sc[0], 1);
            ws.topo[p] = (uint16_t)v;
            if (a.o.level) a.o.level[n0 + v] = 0;
        }
    }
    tm.sync();
    int ls = 0, le = sc[0], L = 0;
    if (lead) ws.lvl_off[0] = 0;
    while (ls < le) {
        // every warp spreads the out-edges of a slice of up to 32 of the level's nodes over
        // its lanes, each lane finding the owner of its edge by a binary search over the
        // slice's edge offsets (an exclusive scan of their out-degrees)
        const int ln = tm.lane();
        for (int base = ls + 32 * tm.warp(); base < le; base += NT) {
            const int i = base + ln;
            const int u = i < le ? ws.topo[i] : 0;
            const int eb = i < le ? (int)rp[u] : 0;
            const int deg = i < le ? (int)rp[u + 1] - eb : 0;
            int x = deg;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(FULL, x, o);
                if (ln >= o) x += y;
            }
            const int start = x - deg, total = __shfl_sync(FULL, x, 31);
            for (int f0 = 0; f0 < total; f0 += 32) {
                const int f = f0 + ln;
                int j = 0;  // the last node whose edges start at or before f
                for (int step = 16; step; step >>= 1) {
                    const int sj = __shfl_sync(FULL, start, j + step);
                    if (sj <= f) j += step;
                }
                const int uo = __shfl_sync(FULL, u, j), eo = __shfl_sync(FULL, eb, j);
                const int so = __shfl_sync(FULL, start, j);
                bool rel = false;
                int s = 0;
                if (f < total) {
                    s = col[eo + f - so];
                    if constexpr (NT == 32) {  // warp teams push the closure along the edge
                        const uint64_t *au = ws.anc + (int64_t)uo * W;
                        unsigned long long *as = (unsigned long long *)(ws.anc + (int64_t)s * W);
                        for (int w = 0; w < W; w++) {
                            const uint64_t y = au[w];
                            if (y) atomicOr(&as[w], (unsigned long long)y);
                        }
                        atomicOr(&as[uo >> 6], 1ull << (uo & 63));
                    }
                    rel = atomicSub(&ws.cnt[s], 1) == 1;
                }
                const uint32_t rm = __ballot_sync(FULL, rel);
                int p0 = 0;
                if (ln == 0 && rm) p0 = atomicAdd((int *)&sc[0], __popc(rm));
                p0 = __shfl_sync(FULL, p0, 0);
                if (rel) {
                    ws.topo[p0 + __popc(rm & ((1u << ln) - 1))] = (uint16_t)s;
                    if (a.o.level) a.o.level[n0 + s] = L + 1;
                }
            }
        }
        tm.sync();
        const int ne = sc[0];
        tm.sync();
        L++;
        if (lead) ws.lvl_off[L] = (uint16_t)le;
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
    if constexpr (NT == 32) {
        for (int v = tm.t; v < V; v += NT) {
            const uint64_t *av = ws.anc + (int64_t)v * W;
            uint64_t acc = ws.load[v];
            for (int b = 0; b < nb; b++) {
                uint32_t c = 0;
                for (int w = 0; w < W; w++) c += __popcll(av[w] & ws.planes[b * W + w]);
                acc += (uint64_t)c << b;
            }
            ws.wanc[v] = acc;
            if (a.o.wanc) a.o.wanc[n0 + v] = (int64_t)acc;
        }
    } else {
        // CTA teams: the closure pulled level by level with plain loads and stores, each
        // thread one (node, 64-bit word) pair -- everything that reaches a predecessor p,
        // and p itself, reaches v -- and the word's share of W^anc added right away
        for (int v = tm.t; v < V; v += NT) {
            ws.poff[v] = ws.indeg[v];
            ws.wanc[v] = ws.load[v];
        }
        tm.sync();
        team_scan_inplace(tm, ws.poff, V, [](uint64_t x, uint64_t y) { return x + y; }, false);
        for (int u = tm.t; u < V; u += NT)  // ws.cnt is zero again after Kahn's pass
            for (int e = rp[u]; e < (int)rp[u + 1]; e++) {
                const int s = col[e];
                ws.pid[ws.poff[s] - ws.indeg[s] + atomicAdd(&ws.cnt[s], 1)] = (uint16_t)u;
            }
        tm.sync();
        for (int l = 0; l < nlev; l++) {
            const int lb = ws.lvl_off[l], lend = (l + 1 < nlev) ? ws.lvl_off[l + 1] : V;
            const int n_items = (lend - lb) * W;
            for (int it = tm.t; it < n_items; it += NT) {
                const int q = it / W, w = it - q * W;
                const int v = ws.topo[lb + q];
                const int pe = ws.poff[v], pb = pe - ws.indeg[v];
                uint64_t word = 0;
                for (int k = pb; k < pe; k++) {
                    const int p = ws.pid[k];
                    word |= ws.anc[(int64_t)p * W + w];
                    if ((p >> 6) == w) word |= 1ull << (p & 63);
                }
                ws.anc[(int64_t)v * W + w] = word;
                if (word) {
                    uint64_t c = 0;
                    for (int b = 0; b < nb; b++) c += (uint64_t)__popcll(word & ws.planes[b * W + w]) << b;
                    atomicAdd((unsigned long long *)&ws.wanc[v], (unsigned long long)c);
                }
            }
            tm.sync();
        }
        if (a.o.wanc)
            for (int v = tm.t; v < V; v += NT) a.o.wanc[n0 + v] = (int64_t)ws.wanc[v];
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
    for (int i = tm.t; i < V; i += NT) {
        const int v = (int)(ws.skey[i] & 0xffff);
        const uint64_t wv = ws.skey[i] >> 16;
        ws.jcnt[i] = (ws.st[v] & ST_JOIN) ? 1 : 0;
        ws.rs[i] = (i == 0 || (ws.skey[i - 1] >> 16) != wv) ? i : 0;
        ws.re[i] = (i == V - 1 || (ws.skey[i + 1] >> 16) != wv) ? i : 0x7fffffff;
    }
    tm.sync();
    team_scan_inplace(tm, ws.jcnt, V, [](uint64_t x, uint64_t y) { return x + y; }, false);
    team_scan_inplace(tm, ws.rs, V, [](uint64_t x, uint64_t y) { return x > y ? x : y; }, false);
    team_scan_inplace(tm, ws.re, V, [](uint64_t x, uint64_t y) { return x < y ? x : y; }, true);
    const int N = ws.jcnt[V - 1];  // number of join nodes
    for (int i = tm.t; i < V; i += NT) {
        const int v = (int)(ws.skey[i] & 0xffff);
        const int r = (V - 1 - ws.re[i]) + (i - ws.rs[i]);
        ws.rank[v] = (uint16_t)r;
        ws.byrank[r] = (uint16_t)v;
        ws.pos[v] = (uint16_t)i;
        ws.bk[v] = NONE16;
    }
    tm.sync();

    // ---- Eq.3 blocks: a node belongs to the first join (in Theta order) it is an ancestor
    //      of, i.e. the smallest sorted position among the joins reachable from it; computed
    //      by a min over successors in reverse level order. No reachable join: residual.
    for (int l = nlev - 1; l >= 0; l--) {
        const int lb = ws.lvl_off[l], lend = (l + 1 < nlev) ? ws.lvl_off[l + 1] : V;
        for (int i = lb + tm.t; i < lend; i += NT) {
            const int v = ws.topo[i];
            int b = NONE16;
            for (int e = rp[v]; e < rp[v + 1]; e++) {
                const int s = col[e];
                if (ws.st[s] & ST_JOIN) b = min(b, (int)ws.pos[s]);
                b = min(b, (int)ws.bk[s]);
            }
            ws.bk[v] = (uint16_t)b;
        }
        tm.sync();
    }
    for (int v = tm.t; v < V; v += NT) {
        const int b = ws.bk[v];
        ws.blk[v] = (uint16_t)(b == NONE16 ? N : ws.jcnt[b] - 1);
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
    if (lead) {  // head counts of the current and the next round (sc[12 + (round & 1)])
        sc[12] = 0;
        sc[13] = 0;
    }
    tm.sync();
    // a block of more than M nodes may have more than M heads in a round (Top_M below)
    bool bigblk = false;
    if (V > (int)M) {
        for (int v = tm.t; v < V; v += NT) atomicAdd(&ws.fcnt[ws.blk[v]], 1);
        tm.sync();
        for (int b = tm.t; b <= N; b += NT) {
            bigblk |= ws.fcnt[b] > (int)M;
            ws.fcnt[b] = 0;
        }
        bigblk = tm.any(bigblk);
        tm.sync();
    }
    if constexpr (NT == 32) {
        // in-block parents, one edge per lane: the edges are in CSR order, so a lane finds its
        // source row a few rows after the row of the round's first edge
        for (int e0 = 0, u0 = 0; e0 < (int)E; e0 += 32) {
            const int e = e0 + tm.t;
            int u = u0;
            if (e < (int)E) {
                while ((int)rp[u + 1] <= e) u++;
                if (ws.blk[col[e]] == ws.blk[u]) atomicAdd(&ws.cnt[col[e]], 1);
            }
            u0 = __shfl_sync(FULL, u, 31);  // lane 31 holds the latest row (or u0 past the end)
        }
    } else {
        for (int u = tm.t; u < V; u += NT)
            for (int e = rp[u]; e < rp[u + 1]; e++)
                if (ws.blk[col[e]] == ws.blk[u]) atomicAdd(&ws.cnt[col[e]], 1);
    }
    tm.sync();
    bad = false;
    for (int v = tm.t; v < V; v += NT) {
        if (ws.cnt[v] > 1) bad = true;
        ws.st[v] = (uint8_t)((ws.st[v] & ST_JOIN) | (ws.cnt[v] == 0 ? ST_ACTIVE : 0));
        if (ws.cnt[v] == 0) ws.fr0[atomicAdd((int *)&sc[12], 1)] = (uint16_t)v;  // the first heads
    }
    if (tm.any(bad)) {
        if (lead) write_failure(a, d, DAGRT_E_INTERNAL);
        return;
    }
    tm.sync();
    // Each round works on the list of its heads only (the nodes marked ST_ACTIVE): the heads
    // that are not selected stay, and a selected node's in-block successor (it has no other
    // in-block predecessor) becomes a head of the next round.
    if (lead) sc[10] = 0;
    tm.sync();
    for (int round = 0;; round++) {
        const int cur = 12 + (round & 1), nxt = 12 + ((round + 1) & 1);
        const int nf = sc[cur];
        if (nf == 0) break;
        if (round > V) {  // every round selects a node, so this cannot happen
            if (lead) write_failure(a, d, DAGRT_E_INTERNAL);
            return;
        }
        const uint16_t *F = (round & 1) ? ws.fr1 : ws.fr0;
        uint16_t *Fn = (round & 1) ? ws.fr0 : ws.fr1;
        // heads per block; a block with more heads than SMs (only in a block of more than M
        // nodes) is listed once, by the head that takes its count past M
        for (int i = tm.t; i < nf; i += NT) {
            const int b = ws.blk[F[i]];
            if (atomicAdd(&ws.fcnt[b], 1) == (int)M && bigblk) ws.ovl[atomicAdd((int *)&sc[10], 1)] = b;
        }
        tm.sync();
        const int nov = sc[10];
        // blocks with more heads than SMs keep their M heaviest (Top_M): the heads up to the
        // rank of the block's M-th head (rank order = W^anc descending). A CTA team finds it
        // for a few such blocks from a bit mask of the block's heads over the ranks (a
        // popcount scan over V/64 words); otherwise one warp per block walks the nodes in rank
        // order with ballots until its M-th head.
        bool masked = false;
        if constexpr (NT > 32) {
            masked = nov > 0 && nov <= 2;
            for (int q = 0; masked && q < nov; q++) {
                const int b = ws.ovl[q];
                for (int w2 = tm.t; w2 < W; w2 += NT) ws.hmask[w2] = 0;
                tm.sync();
                for (int i = tm.t; i < nf; i += NT) {
                    const int v = F[i];
                    if (ws.blk[v] == b)
                        atomicOr((unsigned long long *)&ws.hmask[ws.rank[v] >> 6], 1ull << (ws.rank[v] & 63));
                }
                tm.sync();
                for (int w2 = tm.t; w2 < W; w2 += NT) ws.hcnt[w2] = __popcll(ws.hmask[w2]);
                tm.sync();
                team_scan_inplace(tm, ws.hcnt, W, [](uint64_t x, uint64_t y) { return x + y; }, false);
                for (int w2 = tm.t; w2 < W; w2 += NT) {
                    uint64_t mk = ws.hmask[w2];
                    const int upto = ws.hcnt[w2], before = upto - __popcll(mk);
                    if (before < (int)M && (int)M <= upto) {  // the M-th head is in this word
                        for (int i = 1; i < (int)M - before; i++) mk &= mk - 1;
                        ws.thr[b] = w2 * 64 + __ffsll((long long)mk) - 1;
                    }
                }
                tm.sync();
            }
        }
        for (int q = tm.warp(); !masked && q < nov; q += NT / 32) {
            const int b = ws.ovl[q];
            int cnt = 0, th = V;
            for (int base = 0; base < V; base += 32) {
                const int r = base + tm.lane();
                bool f = false;
                if (r < V) {
                    const int u = ws.byrank[r];
                    f = (ws.st[u] & ST_ACTIVE) && ws.blk[u] == b;
                }
                const uint32_t msk = __ballot_sync(FULL, f);
                const int c = __popc(msk);
                if (cnt + c >= (int)M) {  // the M-th head is in these 32 ranks
                    uint32_t mm = msk;
                    for (int i = 1; i < (int)M - cnt; i++) mm &= mm - 1;
                    th = base + __ffs(mm) - 1;
                    break;
                }
                cnt += c;
            }
            if (tm.lane() == 0) ws.thr[b] = th;
        }
        if (nov) tm.sync();
        if (lead) sc[cur] = 0;  // read by every thread above: it counts the round after next
        for (int i = tm.t; i < nf; i += NT) {
            const int v = F[i];
            const int b = ws.blk[v];
            const bool inT = ws.fcnt[b] <= (int)M || (int)ws.rank[v] <= ws.thr[b];
            if (inT) {
                ws.st[v] |= ST_INT;
                if (ws.load[v] >= M)
                    atomicMax((unsigned long long *)&ws.bigk[b],
                              ((unsigned long long)ws.load[v] << 16) | (0xffffu - ws.rank[v]));
            }
        }
        tm.sync();
        for (int i = tm.t; i < nf; i += NT) {
            const int v = F[i];
            const uint8_t s0 = ws.st[v];
            bool sel = false;
            if (s0 & ST_INT) {
                const uint64_t bg = ws.bigk[ws.blk[v]];
                sel = bg == 0 || (int)(bg & 0xffff) == (int)(0xffffu - ws.rank[v]);
            }
            if (sel) {
                ws.st[v] = (uint8_t)((s0 & ~(ST_INT | ST_ACTIVE)) | ST_SEL);
                ws.rnd[v] = (uint16_t)round;
                atomicMax(&ws.nround[ws.blk[v]], round + 1);
            } else {  // still a head next round
                ws.st[v] = (uint8_t)(s0 & ~ST_INT);
                Fn[atomicAdd((int *)&sc[nxt], 1)] = (uint16_t)v;
            }
        }
        tm.sync();
        for (int i = tm.t; i < nf; i += NT) {
            const int v = F[i];
            const uint8_t s0 = ws.st[v];
            ws.fcnt[ws.blk[v]] = 0;
            ws.bigk[ws.blk[v]] = 0;
            if (s0 & ST_SEL) {
                ws.st[v] = (uint8_t)(s0 & ~ST_SEL);
                for (int e = rp[v]; e < rp[v + 1]; e++) {
                    const int s2 = col[e];
                    if (ws.blk[s2] == ws.blk[v]) {
                        ws.st[s2] |= ST_ACTIVE;
                        Fn[atomicAdd((int *)&sc[nxt], 1)] = (uint16_t)s2;
                    }
                }
            }
        }
        if (lead) sc[10] = 0;
        tm.sync();
    }
    // group index = groups of earlier blocks + round within the block
    team_scan_inplace(tm, ws.nround, N + 1, [](uint64_t x, uint64_t y) { return x + y; }, false);
    const int G = ws.nround[N];
    for (int v = tm.t; v < V; v += NT) {
        const int b = ws.blk[v];
        ws.group_of[v] = (uint16_t)((b ? ws.nround[b - 1] : 0) + ws.rnd[v]);
    }
    tm.sync();

    // ---- member lists of each group, ordered by id
    for (int q = tm.t; q <= G; q += NT) ws.gfill[q] = 0;
    tm.sync();
    for (int v = tm.t; v < V; v += NT) atomicAdd(&ws.gfill[ws.group_of[v]], 1);
    tm.sync();
    team_scan_inplace(tm, ws.gfill, G, [](uint64_t x, uint64_t y) { return x + y; }, false);
    for (int q = tm.t; q <= G; q += NT) ws.gstart[q] = (uint16_t)(q ? ws.gfill[q - 1] : 0);
    tm.sync();
    for (int q = tm.t; q <= G; q += NT) ws.gfill[q] = 0;
    tm.sync();
    for (int v = tm.t; v < V; v += NT) {
        const int q = ws.group_of[v];
        const int p = atomicAdd(&ws.gfill[q], 1);
        ws.gtmp[ws.gstart[q] + p] = (uint16_t)v;
    }
    tm.sync();
    for (int i = tm.t; i < V; i += NT) {
        const int v = ws.gtmp[i];
        const int q = ws.group_of[v];
        int pos = 0;
        for (int x = ws.gstart[q]; x < ws.gstart[q + 1]; x++) pos += ws.gtmp[x] < v;
        ws.gmem[ws.gstart[q] + pos] = (uint16_t)v;
    }
    tm.sync();

    // ---- Alg.2 over the groups in order, with Lemma 1 and Theorem 1
    int nsrc = 0;
    const bool want_base = a.o.greedy || a.o.greedy_unaware || a.o.graham_para;
    uint64_t b_greedy = 0, b_unaware = 0, b_vol = 0;  // baseline sums (Evaluation section)
    for (int v = tm.t; v < V; v += NT) {
        const uint32_t x = ws.load[v];
        ws.rem[v] = x;
        ws.cfull[v] = (uint32_t)exec_time(x, ws.kk[v], x < M ? x : M, M);
        if (want_base) {
            b_greedy += ws.cfull[v];
            b_unaware = sat_add(b_unaware, exec_time_unaware(x, ws.kk[v], M));
            b_vol += x;
        }
        ws.cnt[v] = ws.indeg[v];  // predecessors not yet finished
        ws.st[v] = 0;
        ws.mm[v] = 0;
        nsrc += ws.indeg[v] == 0;
    }
    nsrc = (int)tm.sum(nsrc);
    if (want_base) {
        b_greedy = tm.sum(b_greedy);
        b_unaware = tm.reduce(b_unaware, [](uint64_t p, uint64_t q) { return sat_add(p, q); });
        b_vol = tm.sum(b_vol);
    }
    for (int w = tm.t; w < W; w += NT) ws.relmask[w] = 0;
    for (int w = tm.t; w < (W + 63) / 64; w += NT) ws.relsum[w] = 0;
    tm.sync();
    // released set as a bit mask over ranks (W^anc descending), so the next parallel
    // node to consider is always the lowest set bit; relsum marks its possibly non-empty
    // words
    for (int v = tm.t; v < V; v += NT)
        if (ws.indeg[v] == 0) {
            atomicOr((unsigned long long *)&ws.relmask[ws.rank[v] >> 6], 1ull << (ws.rank[v] & 63));
            if (W > kSumWords)
                atomicOr((unsigned long long *)&ws.relsum[ws.rank[v] >> 12], 1ull << ((ws.rank[v] >> 6) & 63));
        }
    tm.sync();

    Dag g;
    g.n0 = n0;
    g.rbase = 2 * n0;
    g.V = V;
    g.W = W;
    g.M = M;
    g.variant = a.variant;
    g.rp = rp;
    g.col = col;
    g.want_edges = a.o.extra_off != nullptr;
    g.ebase = g.want_edges ? a.o.extra_off[d] : 0;
    g.ecap = g.want_edges ? a.o.extra_off[d + 1] - g.ebase : 0;
    Acc acc;
    acc.bound = 0;
    acc.nextra = 0;
    acc.nrows = 0;
    acc.nseg = 0;
    acc.nrel = nsrc;
    acc.err = false;
    acc.lastr = -1;
    acc.lastz = 0;
    // Warp teams run every group on lane 0 (group_serial takes groups of any size; without
    // the team path the warp kernel needs 96 instead of 127 registers, and measured 2.6%
    // faster on the 10,000-DAG batch); CTA teams give groups of more than 32 members to the
    // whole team.
    constexpr int kSerialMax = NT == 32 ? 0x7fffffff : 32;
    for (int j = 0; j < G;) {
        int j1 = j;
        while (j1 < G && ws.gstart[j1 + 1] - ws.gstart[j1] <= kSerialMax) j1++;
        if (tm.t < 32)  // the team's first warp
            for (int q = j; q < j1; q++) group_serial(ws, a, g, q, acc, tm.t);
        if (j1 < G) {
            if (lead) sc[8] = acc.nrows;
            tm.sync();
            if constexpr (NT > 32) group_team(tm, ws, a, g, j1, acc);
        }
        tm.sync();
        j = j1 + 1;
    }

    // ---- per-DAG and per-node outputs
    if (lead) {
        // candidate bounds fit 32-bit arithmetic: loads < 2^17 and every group sum of
        // C <= ceil(255/M) * max C^ over at most 2V rows below 2^31
        const uint64_t waves = (255 + M - 1) / M;
        if (a.pflag) a.pflag[d] = (mx < (1ull << 17) && mx * waves * 2ull * (uint64_t)V < (1ull << 31)) ? 1 : 0;
        int code = DAGRT_OK;
        if (acc.err) code = DAGRT_E_INTERNAL;
        else if (g.want_edges && acc.nextra > g.ecap) code = DAGRT_E_CAP;
        const int64_t bnd = code == DAGRT_E_INTERNAL ? -1 : (int64_t)acc.bound;
        a.status[d] = code;
        a.bound[d] = bnd;
        if (a.nrows) a.nrows[d] = acc.nrows;
        if (a.o.status) a.o.status[d] = code;
        if (a.o.bound) a.o.bound[d] = bnd;
        if (a.o.n_groups) a.o.n_groups[d] = G;
        if (a.o.n_seg) a.o.n_seg[d] = acc.nseg;
        if (a.o.n_rows) a.o.n_rows[d] = acc.nrows;
        if (a.o.n_extra) a.o.n_extra[d] = acc.nextra;
        // baselines: Greedy (sequential, m = min(C^, M)), Greedy + unaware (sequential,
        // m = C^), Graham_para (unit-load nodes: L + ceil((vol - L) / M), L = nodes on the
        // longest path)
        if (a.o.greedy) a.o.greedy[d] = (int64_t)b_greedy;
        if (a.o.greedy_unaware) a.o.greedy_unaware[d] = (int64_t)b_unaware;
        if (a.o.graham_para) a.o.graham_para[d] = (int64_t)(nlev + (b_vol - nlev + M - 1) / M);
    }
    for (int v = tm.t; v < V; v += NT) {
        if (a.o.block_of) a.o.block_of[n0 + v] = ws.blk[v];
        if (a.o.group_of) a.o.group_of[n0 + v] = ws.group_of[v];
        if (a.o.m) a.o.m[n0 + v] = ws.mm[v];
    }
    tm.sync();

    // ---- critical-path lower bound of the schedule: the longest chain of its parts in G
    //      (a node's parts run one after another, and every edge waits for its tail's last
    //      part), weighted by the parts' times, and the work bound ceil(sum m C / M). Every
    //      execution of the schedule takes at least this long, so Theorem 1's bound must be
    //      at least it: a device-side consistency check (for the variants whose groups fit M
    //      or run in sequence). From the plan rows just written, level by level.
    uint64_t cp = 0;
    if (a.o.crit_path && a.plan) {  // uniform over the team
        if (lead) sc[11] = acc.nrows;  // (after the outputs that read ws.mm: phase F overlays it)
        for (int v = tm.t; v < V; v += NT) {
            ws.cpT[v] = 0;
            ws.cpM[v] = 0;
        }
        __threadfence_block();  // the plan rows written by other threads of the team
        tm.sync();
        const int nr = sc[11];
        uint64_t work = 0;
        for (int r = tm.t; r < nr; r += NT) {
            const uint4 x = a.plan[g.rbase + r];
            atomicAdd((unsigned long long *)&ws.cpT[x.w], (unsigned long long)x.y);
            work += (uint64_t)(x.z & 0xffffu) * x.y;
        }
        work = tm.sum(work);
        tm.sync();
        for (int l = 0; l < nlev; l++) {
            const int lb = ws.lvl_off[l], lend = (l + 1 < nlev) ? ws.lvl_off[l + 1] : V;
            for (int i = lb + tm.t; i < lend; i += NT) {
                const int v = ws.topo[i];
                const uint64_t dv = ws.cpT[v] + ws.cpM[v];
                ws.cpT[v] = dv;
                for (int e = rp[v]; e < (int)rp[v + 1]; e++)
                    atomicMax((unsigned long long *)&ws.cpM[col[e]], (unsigned long long)dv);
            }
            tm.sync();
        }
        uint64_t path = 0;
        for (int v = tm.t; v < V; v += NT) path = ws.cpT[v] > path ? ws.cpT[v] : path;
        path = tm.maxu(path);
        const uint64_t wb = (work + M - 1) / M;
        cp = path > wb ? path : wb;
    }

    if (lead && a.o.crit_path) {
        a.o.crit_path[d] = a.plan ? (int64_t)cp : -1;
        // Theorem 1's bound below a lower bound of every execution: an internal error
        if (a.plan && g.variant != DAGRT_VAR_LITERAL && acc.bound < cp && a.status[d] == DAGRT_OK) {
            write_failure(a, d, DAGRT_E_INTERNAL);
            a.o.crit_path[d] = (int64_t)cp;
        }
    }
    tm.sync();
}

// ------------------------------------------------------------------ kernels
// Warp teams for small DAGs: kWarpsPerCta teams per CTA, each with a shared-memory workspace
// sized for (a.vcap, a.ecap), the largest V and E of the launch's size class.
__global__ void __launch_bounds__(32 * kWarpsPerCta) k_sched_warp(SchedArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5;
    Ws ws;
    const int64_t bytes = ws_carve(nullptr, a.vcap, a.ecap, nullptr);
    ws_carve(smem + warp * bytes, a.vcap, a.ecap, &ws);
    Team<32> tm{(int)(threadIdx.x & 31), nullptr};
    for (;;) {
        int idx = 0;
        if (tm.t == 0) idx = atomicAdd(a.counter, 1);
        idx = __shfl_sync(FULL, idx, 0);
        if (idx >= a.n_list) break;
        schedule_one<32>(tm, ws, a, a.list[idx], a.vcap, a.ecap);
        __syncwarp();
    }
}

// CTA teams for large DAGs: the workspace sized for (a.vcap, a.ecap) lives in dynamic shared
// memory (SMEM) or in the global block a.gws + blockIdx.x * a.gws_stride.
template <int NT, bool SMEM>
__global__ void __launch_bounds__(NT) k_sched_cta(SchedArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint64_t red[NT / 32];
    __shared__ int idx_s;
    Ws ws;
    ws_carve(SMEM ? smem : a.gws + (int64_t)blockIdx.x * a.gws_stride, a.vcap, a.ecap, &ws, true);
    Team<NT> tm{(int)threadIdx.x, red};
    for (;;) {
        if (threadIdx.x == 0) idx_s = atomicAdd(a.counter, 1);
        __syncthreads();
        const int idx = idx_s;
        __syncthreads();
        if (idx >= a.n_list) break;
        schedule_one<NT>(tm, ws, a, a.list ? a.list[idx] : idx, a.vcap, a.ecap);
        __syncthreads();
    }
}

// ------------------------------------------------------------------ launchers
// Occupancy of the warp kernel per (device, dynamic shared memory), queried once per size
// (a schedule call launches up to 16 classes; these host queries were a visible part of
// its enqueue time).
namespace {
struct WarpLaunchCache {
    std::mutex mu;
    std::map<std::pair<int, int64_t>, int> occ;  // (device, bytes) -> CTAs per SM
    std::map<int, int> max_smem;                 // device -> max_dynamic_smem(k_sched_warp)
};
WarpLaunchCache &warp_cache() {
    static WarpLaunchCache c;
    return c;
}
}  // namespace

cudaError_t sched_launch_warp(const SchedArgs &a, int n_sm, cudaStream_t st) {
    const int64_t bytes = ws_carve(nullptr, a.vcap, a.ecap, nullptr) * kWarpsPerCta;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    {
        WarpLaunchCache &c = warp_cache();
        std::lock_guard<std::mutex> lock(c.mu);
        auto it = c.occ.find({dev, bytes});
        if (it == c.occ.end() && bytes > sched_smem_limit()) return cudaErrorInvalidValue;
        auto mx = c.max_smem.find(dev);
        if (mx == c.max_smem.end()) mx = c.max_smem.emplace(dev, max_dynamic_smem(k_sched_warp)).first;
        if (bytes > mx->second) return cudaErrorInvalidValue;
        // the classes differ in size: the attribute allows the largest, whatever launched last
        e = cudaFuncSetAttribute(k_sched_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, mx->second);
        if (e != cudaSuccess) return e;
        if (it != c.occ.end()) {
            per_sm = it->second;
        } else {
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sched_warp, 32 * kWarpsPerCta, bytes);
            if (e != cudaSuccess) return e;
            c.occ[{dev, bytes}] = per_sm;
        }
    }
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int grid = n_sm * per_sm;
    const int need = ceil_div(a.n_list, kWarpsPerCta);
    if (grid > need) grid = need;
    if (grid < 1) return cudaSuccess;
    k_sched_warp<<<grid, 32 * kWarpsPerCta, bytes, st>>>(a);
    return cudaGetLastError();
}

int sched_cta_grid(int n_sm) {
    int per_sm = 0;
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sched_cta<kCtaThreadsGlobal, false>,
                                                                        kCtaThreadsGlobal, 0);
    if (e != cudaSuccess || per_sm < 1) per_sm = 1;
    return n_sm * per_sm;
}

cudaError_t sched_launch_cta(const SchedArgs &a, int grid, cudaStream_t st) {
    if (grid < 1 || a.n_list < 1) return cudaSuccess;
    k_sched_cta<kCtaThreadsGlobal, false><<<grid, kCtaThreadsGlobal, 0, st>>>(a);
    return cudaGetLastError();
}

int64_t sched_smem_limit() {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return 0;
    return optin - (int64_t)sizeof(uint64_t) * (kCtaThreads / 32) - 64;  // the kernel's static shared memory
}

cudaError_t sched_launch_cta_smem(const SchedArgs &a, int n_sm, cudaStream_t st) {
    if (a.n_list < 1) return cudaSuccess;
    const int64_t bytes = sched_ws_bytes(a.vcap, a.ecap);
    const int mx = max_dynamic_smem(k_sched_cta<kCtaThreads, true>);
    if (bytes > mx) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_sched_cta<kCtaThreads, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sched_cta<kCtaThreads, true>, kCtaThreads, bytes);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int grid = n_sm * per_sm;
    if (grid > a.n_list) grid = a.n_list;
    k_sched_cta<kCtaThreads, true><<<grid, kCtaThreads, bytes, st>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ schedulability
__global__ void k_schedulable(int32_t n_dags, const int32_t *status, const int64_t *bound, const int64_t *deadline,
                              int32_t *ok, unsigned long long *n_ok) {
    __shared__ unsigned int s_cnt;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    unsigned int mine = 0;
    for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < n_dags; d += gridDim.x * blockDim.x) {
        const bool y = status[d] == DAGRT_OK && bound[d] <= deadline[d];
        if (ok) ok[d] = y ? 1 : 0;
        mine += y;
    }
    mine = __reduce_add_sync(FULL, mine);
    if ((threadIdx.x & 31) == 0 && mine) atomicAdd(&s_cnt, mine);
    __syncthreads();
    if (threadIdx.x == 0 && s_cnt && n_ok) atomicAdd(n_ok, (unsigned long long)s_cnt);
}

cudaError_t sched_schedulable(int32_t n_dags, const int32_t *status, const int64_t *bound, const int64_t *deadline,
                              int32_t *ok, unsigned long long *n_ok, int n_sm, cudaStream_t st) {
    if (n_dags < 1) return cudaSuccess;
    int grid = (n_dags + 255) / 256;
    if (grid > 4 * n_sm) grid = 4 * n_sm;
    k_schedulable<<<grid, 256, 0, st>>>(n_dags, status, bound, deadline, ok, n_ok);
    return cudaGetLastError();
}

}  // namespace dagrt
