// bound.cu -- bound of candidate allocations on fixed schedule structures, and the argmin
// over candidates per DAG.
//
// A plan is the schedule of one structure variant: rows ordered by the group they run in,
// each with its load, parallel fraction and scheduled SMs. For candidate allocation m^c
// the bound is a max-plus sweep along the group chain (Theorem 1): F_j = F_{j-1} + R_j,
// with R_j = max C_i over the group if its SMs fit in M (Lemma 1), else sum C_i.
//
// Two paths. Materialised candidates in blocks of 64 (n_alloc a multiple of 64) take the
// balanced work items (k_bound_items + k_bound_finish, below): chunks of whole groups of
// every plan, one warp per (chunk, 64-candidate block), its rows staged by 2-D TMA tensor
// copies, partial bounds added into per-candidate accumulators. Everything else (generated candidates, other n_alloc) takes
// the tile kernel k_bound_tma: one CTA per DAG; row tiles of the DAG -- the candidate bytes
// of T rows (one contiguous run of T * cand_stride bytes, or none when the candidates are
// generated in the kernel) and the T plan rows of every variant in the call -- stream from
// global to shared memory with TMA bulk copies into two stages that complete on mbarriers,
// so the loads of tile i+1 overlap the evaluation of tile i. Each thread owns 1, 2 or 4
// adjacent candidates of one variant and keeps their running group states; the argmin over
// the DAG's candidates is reduced with warp shuffles and shared memory in the same kernel.
#include <cuda.h>  // CUtensorMap and its encoding enums (header only)

#include <cstring>
#include <type_traits>

#include "bound.cuh"
#include "dagrt_internal.cuh"

namespace dagrt {

constexpr int kBoundMaxThreads = 256;
constexpr uint32_t kSpinLimit = 1u << 24;  // bounded mbarrier wait

// ------------------------------------------------------------------ TMA / mbarrier
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// bounded wait on a stage; false after `limit` polls
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit = kSpinLimit) {
    for (uint32_t i = 0; i < limit; i++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__global__ void k_selftest_wait(uint32_t limit, int32_t *word) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    // nothing arrives: the wait must give up and report, leaving the CTA free to exit
    const bool ok = mbar_wait(&bar, 0, limit);
    if (!ok && threadIdx.x == 0) atomicExch(word, DAGRT_E_TIMEOUT);
}

cudaError_t bound_selftest_wait(uint32_t limit, int32_t *word, cudaStream_t st) {
    k_selftest_wait<<<1, 32, 0, st>>>(limit, word);
    return cudaGetLastError();
}

// argmin helper: smaller bound wins, then the smaller candidate id
__device__ __forceinline__ void better(int64_t &bb, int32_t &bc, int64_t ob, int32_t oc) {
    if (oc < 0) return;
    if (bc < 0 || ob < bb || (ob == bb && oc < bc)) {
        bb = ob;
        bc = oc;
    }
}

// Shared-memory layout of one stage: T rows of candidate bytes, then T plan rows (16 B)
// of each variant.
struct TileLayout {
    int T;
    int64_t cand_bytes, stage_bytes;
};

__host__ __device__ inline TileLayout tile_layout(int T, int64_t stride, int nv) {
    TileLayout t;
    t.T = T;
    t.cand_bytes = (int64_t)T * stride;
    t.stage_bytes = t.cand_bytes + (int64_t)nv * T * 16;
    return t;
}

// SMs of plan row `row` (owner node `owner`, scheduled on m0 SMs) for generated candidate c
// of DAG d; 0 keeps the schedule's m.
__device__ __forceinline__ uint32_t gen_alloc(const BoundArgs &a, int d, int c, int row, uint32_t owner, uint32_t m0,
                                              const uint8_t *s_lev) {
    const int al = c % a.n_alloc;
    if (a.gen_mode == DAGRT_SEARCH_EXHAUSTIVE) {
        const uint32_t dg = exh_digit((uint32_t)al, owner, (uint32_t)a.n_levels + 1u);
        return dg ? s_lev[dg - 1] : 0u;
    }
    if (al == 0) return 0u;
    const uint32_t x = s_lev[gen_level(a.seed, d, c, row, a.n_levels)];
    if (a.gen_mode != DAGRT_SEARCH_PERTURB) return x;
    return x == 0 ? 0u : perturb_m(m0, x);  // code 0 keeps the row's own m (even above 255)
}

// Candidate bytes of one row for a thread's CPT adjacent candidates (one shared load), or
// the generated allocations of those candidates.
template <int CPT, bool GEN>
__device__ __forceinline__ uint32_t row_alloc(const BoundArgs &a, const unsigned char *cbuf, int64_t stride, int rr,
                                              int d, int c, int row, uint32_t owner, uint32_t m0,
                                              const uint8_t *s_lev) {
    if (GEN) {
        uint32_t m4 = 0;
#pragma unroll
        for (int q = 0; q < CPT; q++) m4 |= gen_alloc(a, d, c + q, row, owner, m0, s_lev) << (8 * q);
        return m4;
    }
    if (CPT == 4) return *(const uint32_t *)(cbuf + rr * stride);
    if (CPT == 2) return *(const uint16_t *)(cbuf + rr * stride);
    return cbuf[rr * stride];
}

// The tiles of DAG d for this thread's candidates c .. c+CPT-1 (variant vi, my_rows rows).
// FIT (uniform over the DAG): every variant's plan keeps all sums below 2^31, so the
// state is 32-bit and C for m = 2^l <= M takes the shift form
//   ceil(x (64m - k(m-1)) / 64m) = ((x(64-k) + 64) << l + x k - 1) >> (l + 6);
// other allocations (not a power of two, or above M) take exec_time. Group ends are
// applied without branches, so threads of different variants may share a warp.
// Returns false when a tile copy stalled (the CTA aborts).
template <int CPT, bool GEN, bool FIT>
__device__ __forceinline__ bool eval_tiles(const BoundArgs &a, int d, int c, int vi, int my_rows, int rows_max,
                                           const TileLayout &L, int64_t stride, unsigned char *const *stage,
                                           uint64_t *bar, uint32_t *uses, uint32_t *issued, uint32_t *landed,
                                           int *s_abort, const uint8_t *s_lev, uint64_t *bound_out) {
    using S = typename std::conditional<FIT, uint32_t, uint64_t>::type;
    const int T = L.T, nv = a.n_variants, tid = threadIdx.x;
    const uint32_t M = (uint32_t)a.M;
    const int64_t rbase = 2 * a.node_off[d];
    const int ntile = (rows_max + T - 1) / T;
    S bound[CPT], gmax[CPT], gsum[CPT];
    uint32_t gm[CPT];
#pragma unroll
    for (int q = 0; q < CPT; q++) bound[q] = gmax[q] = gsum[q] = 0, gm[q] = 0;

    auto issue = [&](int i) {  // tile i of the DAG into stage i & 1 (thread 0)
        const int s = i & 1;
        const int r0 = i * T;
        const int rn = min(T, rows_max - r0);
        const uint32_t cb = (uint32_t)(rn * stride);
        issued[s]++;
        mbar_expect_tx(&bar[s], cb + (uint32_t)(nv * rn * 16));
        if (!GEN) bulk_g2s(stage[s], a.m_alloc + (rbase + r0) * stride, cb, &bar[s]);
        for (int v = 0; v < nv; v++)
            bulk_g2s(stage[s] + L.cand_bytes + (int64_t)v * T * 16, a.plan[v] + rbase + r0, (uint32_t)(rn * 16),
                     &bar[s]);
    };
    if (tid == 0) {
        fence_proxy_async();
        for (int i = 0; i < 2 && i < ntile; i++) issue(i);
    }
    for (int i = 0; i < ntile; i++) {
        const int s = i & 1;
        const bool ok = mbar_wait(&bar[s], uses[s] & 1);
        uses[s]++;
        landed[s] += ok;
        if (!ok) atomicExch(s_abort, 1);
        __syncthreads();
        if (*s_abort) return false;
        const int r0 = i * T;
        const int rn = min(T, my_rows - r0);
        const unsigned char *cbuf = stage[s] + c;  // candidate column c of row r0
        const uint4 *pl = (const uint4 *)(stage[s] + L.cand_bytes) + (int64_t)vi * T;
        for (int rr = 0; rr < rn; rr++) {
            const uint4 x = pl[rr];
            const uint32_t k = (x.z >> 16) & 0xffu, m0 = x.z & 0xffffu;
            const bool last = (x.z >> 24) != 0;
            const uint32_t m4 = row_alloc<CPT, GEN>(a, cbuf, stride, rr, d, c, r0 + rr, x.w, m0, s_lev);
            S cc[CPT];
            if (FIT) {
                const uint32_t A1 = x.x * (64u - k) + 64u, B1 = x.x * k - 1u;
#pragma unroll
                for (int q = 0; q < CPT; q++) {
                    const uint32_t m = (m4 >> (8 * q)) & 0xffu;
                    const uint32_t ms = m ? m : 1u;
                    const int l = 31 - __clz(ms);
                    uint32_t v = ((A1 << l) + B1) >> (l + 6);
                    if ((ms != (1u << l)) | (ms > M)) v = (uint32_t)exec_time(x.x, k, ms, M);
                    cc[q] = m ? v : x.y;
                }
            } else {
#pragma unroll
                for (int q = 0; q < CPT; q++) {
                    const uint32_t m = (m4 >> (8 * q)) & 0xffu;
                    cc[q] = m ? exec_time(x.x, k, m, M) : (uint64_t)x.y;
                }
            }
#pragma unroll
            for (int q = 0; q < CPT; q++) {
                const uint32_t m = (m4 >> (8 * q)) & 0xffu;
                gmax[q] = cc[q] > gmax[q] ? cc[q] : gmax[q];
                gsum[q] += cc[q];
                gm[q] += m ? m : m0;
                const S r = gm[q] <= M ? gmax[q] : gsum[q];
                bound[q] += last ? r : (S)0;
                gmax[q] = last ? (S)0 : gmax[q];
                gsum[q] = last ? (S)0 : gsum[q];
                gm[q] = last ? 0u : gm[q];
            }
        }
        __syncthreads();  // every thread is done with stage s
        if (tid == 0 && i + 2 < ntile) {
            fence_proxy_async();
            issue(i + 2);
        }
    }
#pragma unroll
    for (int q = 0; q < CPT; q++) bound_out[q] = (uint64_t)bound[q];
    return true;
}

// FIT selects the DAGs this instance evaluates (the 32-bit form exact for every variant, or
// not); the host launches both instances over the batch, each skipping the other's DAGs,
// so each keeps only its own state in registers.
template <int CPT, bool GEN, bool FIT>
__global__ void __launch_bounds__(kBoundMaxThreads) k_bound_tma(BoundArgs a, int T) {
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int s_abort;
    __shared__ int64_t s_bb[kBoundMaxThreads / 32];
    __shared__ int32_t s_bc[kBoundMaxThreads / 32];
    __shared__ uint8_t s_lev[16];
    const int nv = a.n_variants;
    const int n_cand = nv * a.n_alloc;
    const int64_t stride = GEN ? 0 : a.stride;  // generated candidates stream plan rows only
    const TileLayout L = tile_layout(T, stride, nv);
    if (GEN && threadIdx.x < 16) s_lev[threadIdx.x] = a.levels[threadIdx.x];
    unsigned char *stage[2] = {sm, sm + L.stage_bytes};
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
        s_abort = 0;
    }
    __syncthreads();
    uint32_t uses[2] = {0, 0};    // waits per stage so far (identical in every thread)
    uint32_t issued[2] = {0, 0};  // copies issued per stage (thread 0)
    uint32_t landed[2] = {0, 0};  // waits that saw their copy land (thread 0)

    for (int d = blockIdx.x; d < a.n_dags; d += gridDim.x) {
        const int64_t rbase = 2 * a.node_off[d];
        int rows_max = 0;
        bool fit = true;  // the 32-bit form is exact for every variant
        for (int v = 0; v < nv; v++)
            if (a.status[v][d] == DAGRT_OK) {
                rows_max = max(rows_max, a.nrows[v][d]);
                fit = fit && (a.pflag[v][d] & 1);
            }
        if (fit != FIT) continue;  // uniform over the CTA
        int64_t best_b = 0;
        int32_t best_c = -1;

        for (int c0 = 0; c0 < n_cand; c0 += blockDim.x * CPT) {
            const int c = c0 + tid * CPT;
            const bool active = c < n_cand;
            const int vi = active ? c / a.n_alloc : 0;
            const bool valid = active && a.status[vi][d] == DAGRT_OK;
            const int my_rows = valid ? a.nrows[vi][d] : 0;
            uint64_t bound[CPT];
            const bool ok = eval_tiles<CPT, GEN, FIT>(a, d, c, vi, my_rows, rows_max, L, stride, stage, bar, uses,
                                                      issued, landed, &s_abort, s_lev, bound);
            if (!ok) break;
#pragma unroll
            for (int q = 0; q < CPT; q++) {
                const int cq = c + q;
                if (!active || cq >= n_cand) break;
                const int64_t b = valid ? (int64_t)bound[q] : -1;
                if (a.out) a.out[(int64_t)d * n_cand + cq] = b;
                if (valid) better(best_b, best_c, b, cq);
            }
        }
        if (s_abort) break;
        if (a.best_bound || a.best_cand) {
            for (int o = 16; o > 0; o >>= 1) {
                const int64_t ob = __shfl_xor_sync(FULL, best_b, o);
                const int32_t oc = __shfl_xor_sync(FULL, best_c, o);
                better(best_b, best_c, ob, oc);
            }
            if ((tid & 31) == 0) {
                s_bb[tid >> 5] = best_b;
                s_bc[tid >> 5] = best_c;
            }
            __syncthreads();
            if (tid == 0) {
                for (int w = 1; w < (int)(blockDim.x >> 5); w++) better(best_b, best_c, s_bb[w], s_bc[w]);
                if (a.best_bound) a.best_bound[d] = best_c < 0 ? -1 : best_b;
                if (a.best_cand) a.best_cand[d] = best_c;
                s_bc[0] = best_c;
            }
            __syncthreads();
            if (GEN && a.best_m && s_bc[0] >= 0) {  // the winning allocation, row by row
                const int wc = s_bc[0], wv = wc / a.n_alloc;
                const int rows = a.nrows[wv][d];
                for (int r = tid; r < rows; r += blockDim.x) {
                    const uint4 x = a.plan[wv][rbase + r];
                    a.best_m[rbase + r] = (uint8_t)gen_alloc(a, d, wc, r, x.w, x.z & 0xffffu, s_lev);
                }
            }
            __syncthreads();
        }
    }
    if (s_abort && tid == 0) {
        // a copy stalled: report it, and give the copies already issued a bounded chance to
        // land before the CTA's shared memory is released
        if (a.err) atomicExch(a.err, DAGRT_E_TIMEOUT);
        for (int s = 0; s < 2; s++)
            for (uint32_t k = landed[s]; k < issued[s]; k++) mbar_wait(&bar[s], k & 1);
    }
}

// ------------------------------------------------------------------ balanced work items
constexpr int kSubRows = 32;      // plan rows staged per load phase of a work item
// rows of one TMA box of candidate bytes (64 bytes wide): a whole phase, one copy (a short
// last phase copies rows it does not use; boxes of 8 or 16 rows measured slower)
constexpr int kBoxRows = kSubRows;
constexpr int kMaxItemWarps = 8;  // warps per CTA of the work-item kernel: ChunkArgs::warps <= this
// per warp: two staging buffers (the candidate bytes of a phase, then its plan rows) and the
// {C, m} table of the phase's rows; every piece 128-byte aligned
constexpr int kStageCand = kSubRows * 64;
constexpr int kStageBytes = kStageCand + kSubRows * 16;
constexpr int kWarpBytes = 2 * kStageBytes + kSubRows * 9 * 8;
static_assert(kStageCand % 128 == 0 && kStageBytes % 128 == 0 && kWarpBytes % 128 == 0, "TMA buffer alignment");

// Chunk starts of every DAG of one plan (one warp per DAG). Chunk 0 starts at row 0; each
// chunk takes whole groups, as many as fit in chunk_rows rows (at least one group), so a
// chunk ends at the last group end within chunk_rows rows of its start, or at the end of
// its first group if that group alone is longer. Any two neighbouring chunks hold more than
// chunk_rows rows together. The group-end bits of 32 rows at a time come from one ballot;
// every lane walks the same masks, lane 0 writes.
__global__ void k_plan_chunks(int32_t n_dags, const int64_t *node_off, const uint4 *plan, const int32_t *nrows,
                              const int32_t *status, int32_t *chunk, int32_t *nchunk, int chunk_rows) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int d = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; d < n_dags; d += warps) {
        const int rows = status[d] == DAGRT_OK ? nrows[d] : 0;
        const uint4 *pr = plan + 2 * node_off[d];
        int count = 0;
        for (int cur = 0; cur < rows;) {
            if (lane == 0) chunk[2 * node_off[d] + count] = cur;
            count++;
            const int limit = min(rows, cur + chunk_rows);
            int next = -1;  // one past the chunk's last row
            for (int base = cur; base < limit; base += 32) {
                const int r = base + lane;
                const uint32_t mask = __ballot_sync(FULL, r < limit && (pr[r].z >> 24) != 0);
                if (mask) next = base + 32 - __clz(mask);
            }
            for (int base = limit; next < 0 && base < rows; base += 32) {  // a group longer than chunk_rows
                const int r = base + lane;
                const uint32_t mask = __ballot_sync(FULL, r < rows && (pr[r].z >> 24) != 0);
                if (mask) next = base + __ffs(mask);
            }
            cur = next < 0 ? rows : next;
        }
        if (lane == 0) nchunk[d] = count;
    }
}

// exclusive prefix sum of n counts (one CTA of 1024 threads); out[n] = total
__global__ void __launch_bounds__(1024) k_scan_excl(int32_t n, const int32_t *in, int32_t *out) {
    __shared__ int32_t ws[32];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    int32_t carry = 0;
    for (int base = 0; base < n; base += 1024) {
        const int i = base + tid;
        const int32_t x = i < n ? in[i] : 0;
        int32_t incl = x;
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) ws[w] = incl;
        __syncthreads();
        if (w == 0) {
            int32_t v = ws[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(FULL, v, o);
                if (lane >= o) v += y;
            }
            ws[lane] = v;
        }
        __syncthreads();
        if (i < n) out[i] = carry + (w ? ws[w - 1] : 0) + incl - x;
        const int32_t tot = ws[31];
        __syncthreads();
        carry += tot;
    }
    if (tid == 0) out[n] = carry;
}

// item records {d, first row, end row, flags} in global plan-row numbering; flags bit 0:
// the DAG's sums fit 32-bit arithmetic
__global__ void k_fill_items(int32_t n_dags, const int64_t *node_off, const int32_t *nrows, const int32_t *pflag,
                             const int32_t *chunk, const int32_t *nchunk, const int32_t *cpre, int4 *item) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int d = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; d < n_dags; d += warps) {
        const int64_t rbase = 2 * node_off[d];
        const int nch = nchunk[d];
        const int flags = nch ? (pflag[d] & 1) : 0;
        for (int k = lane; k < nch; k += 32) {
            const int r0 = chunk[rbase + k], r1 = k + 1 < nch ? chunk[rbase + k + 1] : nrows[d];
            item[cpre[d] + k] = make_int4(d, (int)(rbase + r0), (int)(rbase + r1), flags);
        }
    }
}

cudaError_t bound_build_chunks(int32_t n_dags, const int64_t *node_off, const uint4 *plan, const int32_t *nrows,
                               const int32_t *status, const int32_t *pflag, const ChunkIndex &ci, int chunk_rows,
                               int n_sm, cudaStream_t st) {
    if (n_dags == 0) return cudaMemsetAsync(ci.cpre, 0, sizeof(int32_t), st);
    int grid = (n_dags + 7) / 8;
    if (grid > 16 * n_sm) grid = 16 * n_sm;
    k_plan_chunks<<<grid, 256, 0, st>>>(n_dags, node_off, plan, nrows, status, ci.chunk, ci.nchunk, chunk_rows);
    k_scan_excl<<<1, 1024, 0, st>>>(n_dags, ci.nchunk, ci.cpre);
    k_fill_items<<<grid, 256, 0, st>>>(n_dags, node_off, nrows, pflag, ci.chunk, ci.nchunk, ci.cpre, ci.item);
    return cudaGetLastError();
}

static int64_t chunk_items_call(int32_t n_dags, int64_t total_nodes, int32_t n_variants, int32_t n_alloc,
                                int chunk_rows) {
    return (int64_t)n_variants * chunk_items_bound(total_nodes, n_dags, chunk_rows) * (n_alloc / 64);
}

bool bound_chunk_eligible(const BoundArgs &a, int64_t total_nodes, int chunk_rows) {
    return !a.gen && a.n_alloc % 64 == 0 && a.n_dags > 0 &&
           chunk_items_call(a.n_dags, total_nodes, a.n_variants, a.n_alloc, chunk_rows) < (1ll << 30) &&
           2 * total_nodes < (1ll << 31);
}

size_t bound_chunk_scratch(int32_t n_dags, int64_t total_nodes, int32_t n_variants, int32_t n_alloc, int chunk_rows) {
    (void)total_nodes;
    (void)chunk_rows;
    return 256 + (size_t)n_dags * n_variants * n_alloc * 8;
}

// Programmatic dependent launch: the work-item kernel lets k_bound_finish start early;
// k_bound_finish reads what earlier kernels wrote, then waits for the work items to
// complete (and their stores to be visible) before it touches their partial sums.
__device__ __forceinline__ void griddep_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// After the work items, one warp per DAG: the items have added their partial bounds into
// the DAG's per-candidate accumulators; lane l reads candidates 2l and 2l + 1 of four
// 64-candidate blocks at a time, writes the bounds (-1 for a variant whose schedule
// failed), clears the accumulators for the next call and takes the argmin by shuffles. The
// statuses are read before the wait on the work items. Block 0 also resets the work-item
// counter.
__global__ void __launch_bounds__(32) k_bound_finish(BoundArgs a, ChunkArgs ch) {
    const int nv = a.n_variants, ncb = a.n_alloc / 64, n_cand = nv * a.n_alloc, nblk = nv * ncb;
    const int lane = threadIdx.x;
    int32_t st = 0;
    if (lane < nv && (int)blockIdx.x < a.n_dags) st = a.status[lane][blockIdx.x];
    griddep_wait();
    if (blockIdx.x == 0 && lane == 0) *ch.counter = 0u;
    for (int d = blockIdx.x; d < a.n_dags; d += gridDim.x) {
        if (d != (int)blockIdx.x && lane < nv) st = a.status[lane][d];
        unsigned long long *acc = ch.acc + (int64_t)d * n_cand;
        int64_t best_b = 0;
        int32_t best_c = -1;
        for (int k0 = 0; k0 < nblk; k0 += 4) {
            ulonglong2 x[4];
#pragma unroll
            for (int k = 0; k < 4; k++)
                x[k] = k0 + k < nblk ? __ldcg((const ulonglong2 *)(acc + (k0 + k) * 64 + 2 * lane))
                                     : make_ulonglong2(0, 0);
#pragma unroll
            for (int k = 0; k < 4; k++) {
                if (k0 + k >= nblk) break;
                const int c = (k0 + k) * 64 + 2 * lane;
                const bool ok = __shfl_sync(FULL, st, (k0 + k) / ncb) == DAGRT_OK;
                const int64_t s0 = ok ? (int64_t)x[k].x : -1, s1 = ok ? (int64_t)x[k].y : -1;
                if (ok) {
                    better(best_b, best_c, s0, c);
                    better(best_b, best_c, s1, c + 1);
                    *(ulonglong2 *)(acc + c) = make_ulonglong2(0, 0);
                }
                if (a.out) {  // the caller's buffer is only 8-byte aligned
                    a.out[(int64_t)d * n_cand + c] = s0;
                    a.out[(int64_t)d * n_cand + c + 1] = s1;
                }
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const int64_t ob = __shfl_xor_sync(FULL, best_b, o);
            const int32_t oc = __shfl_xor_sync(FULL, best_c, o);
            better(best_b, best_c, ob, oc);
        }
        if (lane == 0) {
            if (a.best_bound) a.best_bound[d] = best_c < 0 ? -1 : best_b;
            if (a.best_cand) a.best_cand[d] = best_c;
        }
    }
}

// nonzero iff some byte of w is neither 0 nor a power of two: per byte, (b | 0x80) - 1
// cannot borrow from the next byte, and its AND with b is 0 exactly for 0 and powers of two
__device__ __forceinline__ uint32_t bytes_not_pow2(uint32_t w) { return ((w | 0x80808080u) - 0x01010101u) & w; }

// index of the highest set bit, -1 for 0 (PTX bfind)
__device__ __forceinline__ int high_bit(uint32_t x) {
    int r;
    asm("bfind.u32 %0, %1;" : "=r"(r) : "r"(x));
    return r;
}

// One plan row of Lemma 1's group sweep for two candidates (C, m in ta, tb): a row that
// starts and ends its group adds C; a group's first row sets max / sum / SMs, later rows
// accumulate, its last row adds R_j = max C if the SMs fit in M, else sum C. `start` and
// `end` are the same in every lane, so the branches are uniform (bra.uni).
__device__ __forceinline__ void group_step(uint32_t start, uint32_t end, uint2 ta, uint2 tb, uint32_t M,
                                           uint32_t &gmax0, uint32_t &gmax1, uint32_t &gsum0, uint32_t &gsum1,
                                           uint32_t &gm0, uint32_t &gm1, uint32_t &b0, uint32_t &b1) {
    asm("{\n\t"
        ".reg .pred ps, pe, q0, q1;\n\t"
        ".reg .u32 t0, t1;\n\t"
        "setp.ne.u32 ps, %8, 0;\n\t"
        "setp.ne.u32 pe, %9, 0;\n\t"
        "@!ps bra.uni MID;\n\t"
        "@!pe bra.uni FIRST;\n\t"
        "add.u32 %6, %6, %10;\n\t"
        "add.u32 %7, %7, %12;\n\t"
        "bra.uni DONE;\n"
        "FIRST:\n\t"
        "mov.u32 %0, %10;\n\t"
        "mov.u32 %1, %12;\n\t"
        "mov.u32 %2, %10;\n\t"
        "mov.u32 %3, %12;\n\t"
        "mov.u32 %4, %11;\n\t"
        "mov.u32 %5, %13;\n\t"
        "bra.uni DONE;\n"
        "MID:\n\t"
        "max.u32 %0, %0, %10;\n\t"
        "max.u32 %1, %1, %12;\n\t"
        "add.u32 %2, %2, %10;\n\t"
        "add.u32 %3, %3, %12;\n\t"
        "add.u32 %4, %4, %11;\n\t"
        "add.u32 %5, %5, %13;\n\t"
        "@!pe bra.uni DONE;\n\t"
        "setp.le.u32 q0, %4, %14;\n\t"
        "setp.le.u32 q1, %5, %14;\n\t"
        "selp.u32 t0, %0, %2, q0;\n\t"
        "selp.u32 t1, %1, %3, q1;\n\t"
        "add.u32 %6, %6, t0;\n\t"
        "add.u32 %7, %7, t1;\n"
        "DONE:\n\t"
        "}"
        : "+r"(gmax0), "+r"(gmax1), "+r"(gsum0), "+r"(gsum1), "+r"(gm0), "+r"(gm1), "+r"(b0), "+r"(b1)
        : "r"(start), "r"(end), "r"(ta.x), "r"(ta.y), "r"(tb.x), "r"(tb.y), "r"(M));
}

// 2-D tensor copy (TMA) of one box of candidate bytes: x = first candidate column (a
// multiple of 64), y = first allocation row; rows past the end of the tensor read as zero
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void bulk_g2s_u32(uint32_t dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Persistent warps over the work items. Per item: its rows (64 candidate bytes and the plan
// row each, at most kSubRows per phase) are staged into one of the warp's two buffers by
// lane 0 -- a 2-D TMA tensor copy of the candidate bytes and a bulk copy of the plan rows,
// completing on the buffer's mbarrier -- and the next phase (of this item or the next one)
// is issued into the other buffer before the current one is evaluated.
//
// Items whose DAG's sums fit 32 bits: per phase, lane r handles plan row r -- it builds the
// row's {C, m} table (m = 0: the schedule's own C and m; m = 1, 2, 4, ..., 128: the 32-bit
// shift form, exec_time above M when CHECK_M) and checks whether all 64 candidate bytes of
// the row are 0 or powers of two; two ballots give the phase's group-end and exact-path row
// masks, and the group starts follow from the ends. Each lane then runs 2 candidates along
// the rows with table lookups; rows with other bytes take exec_time for those bytes. A
// group of one row adds its C directly; the first row of a longer group sets its running
// max / sum / SMs, its last row adds R_j (Lemma 1). Other items run their rows in 64-bit
// arithmetic with exec_time for every byte. Each item adds its 64 partial sums into the
// DAG's per-candidate 64-bit accumulators (the bound is their sum); k_bound_finish reads
// them once every item is done. At most 64 registers a thread, so that eight CTAs of four
// warps fit an SM by registers. A copy that does not land within the bounded wait sets
// DAGRT_E_TIMEOUT; the warp then waits (bounded) for its copies in flight and stops.
template <bool CHECK_M>
__global__ void __launch_bounds__(kMaxItemWarps * 32, 4)
    k_bound_items(const __grid_constant__ CUtensorMap tmap, BoundArgs a, ChunkArgs ch) {
    extern __shared__ unsigned char sm[];
    __shared__ int64_t s_cum[kMaxVariantsPerCall + 1];
    __shared__ __align__(8) uint64_t s_bar[kMaxItemWarps][2];
    griddep_launch_dependents();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // the warps' buffers from a 128-byte boundary (TMA destinations)
    unsigned char *wbase = sm + (((smem_addr(sm) + 127u) & ~127u) - smem_addr(sm)) + w * kWarpBytes;
    uint64_t *bar = s_bar[w];
    uint2 *tbuf = (uint2 *)(wbase + 2 * kStageBytes);
    const int nv = a.n_variants, ncb = a.n_alloc / 64, n_cand = nv * a.n_alloc;
    const uint32_t M = (uint32_t)a.M;
    if (threadIdx.x == 0) {
        s_cum[0] = 0;
        for (int v = 0; v < nv; v++) s_cum[v + 1] = s_cum[v] + (int64_t)ch.cpre[v][a.n_dags] * ncb;
    }
    if (lane == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    const uint32_t total = (uint32_t)s_cum[nv];

    auto grab = [&]() -> uint32_t {
        uint32_t v = 0;
        if (lane == 0) v = atomicAdd(ch.counter, 1u);
        return __shfl_sync(FULL, v, 0);
    };
    // variant slot, 64-candidate block and record of item j
    auto locate = [&](uint32_t j, int &vi, int &cb, int4 &rec) {
        vi = 0;
        while ((int64_t)j >= s_cum[vi + 1]) vi++;
        const uint32_t jj = j - (uint32_t)s_cum[vi];
        const uint32_t q = ncb == 1 ? jj : jj / (uint32_t)ncb;
        cb = (int)(jj - q * (uint32_t)ncb);
        rec = ch.item[vi][q];
    };
    uint32_t parity = 0u;    // bit b: parity of the next wait on buffer b
    uint32_t inflight = 0u;  // bit b: a copy issued into buffer b and not yet waited for
    // rows [g0, g1) of item (vi, cb) into staging buffer b (the warp is done reading it): one
    // 2-D TMA box per kBoxRows rows of the 64 candidate bytes, one bulk copy of the plan rows
    auto stage = [&](int b, int vi, int cb, int g0, int g1) {
        inflight |= 1u << b;
        if (lane == 0) {
            const int rn = g1 - g0, nb = (rn + kBoxRows - 1) / kBoxRows;
            const uint32_t dst = smem_addr(wbase + b * kStageBytes);
            fence_proxy_async();  // the warp's reads of the buffer come before the copy's writes
            mbar_expect_tx(&bar[b], (uint32_t)(nb * kBoxRows * 64 + rn * 16));
            const int x = vi * a.n_alloc + cb * 64;
            for (int i = 0; i < nb; i++) tma_load_2d(dst + i * kBoxRows * 64, &tmap, x, g0 + i * kBoxRows, &bar[b]);
            bulk_g2s_u32(dst + kSubRows * 64, a.plan[vi] + g0, (uint32_t)(rn * 16), &bar[b]);
        }
    };
    auto wait_buf = [&](int b) -> bool {
        const bool ok = __all_sync(FULL, mbar_wait(&bar[b], (parity >> b) & 1u));
        if (ok) {
            parity ^= 1u << b;
            inflight &= ~(1u << b);
        }
        return ok;
    };

    uint32_t j = grab();
    int vi = 0, cb = 0, buf = 0;
    int4 rec = make_int4(0, 0, 0, 0);
    if (j < total) {
        locate(j, vi, cb, rec);
        stage(0, vi, cb, rec.y, min(rec.z, rec.y + kSubRows));
    }
    bool failed = false;
    while (j < total && !failed) {
        const uint32_t jn = grab();
        int vn = 0, cbn = 0;
        int4 recn = make_int4(0, 0, 0, 0);
        if (jn < total) locate(jn, vn, cbn, recn);
        // the item's phases; FIT: 32-bit table path, else 64-bit sums with exec_time
        auto run_item = [&](auto fitc) {
            constexpr bool FIT = decltype(fitc)::value;
            using acc_t = typename std::conditional<FIT, uint32_t, uint64_t>::type;
            acc_t gmax0 = 0, gmax1 = 0, gsum0 = 0, gsum1 = 0, b0 = 0, b1 = 0;
            uint32_t gm0 = 0, gm1 = 0;
            uint32_t carry = 1u;  // chunks start at a group start
            for (int g0 = rec.y; g0 < rec.z; g0 += kSubRows) {
                const int rn = min(kSubRows, rec.z - g0);
                if (!wait_buf(buf)) {
                    failed = true;
                    return;
                }
                // the next phase into the other buffer, read completely by the last phase: the
                // item's next rows, or the first rows of the next item
                if (g0 + kSubRows < rec.z)
                    stage(buf ^ 1, vi, cb, g0 + kSubRows, min(rec.z, g0 + 2 * kSubRows));
                else if (jn < total)
                    stage(buf ^ 1, vn, cbn, recn.y, min(recn.z, recn.y + kSubRows));
                const unsigned char *cbuf = wbase + buf * kStageBytes;
                const uint4 *pbuf = (const uint4 *)(cbuf + kSubRows * 64);
                if constexpr (FIT) {
                    bool endg = false, odd = false;
                    if (lane < rn) {  // {C, m} table, group end and byte check of row `lane`
                        const uint4 x = pbuf[lane];
                        const uint32_t kk = (x.z >> 16) & 0xffu;
                        const uint32_t A1 = x.x * (64u - kk) + 64u, B1 = x.x * kk - 1u;
                        uint2 *t = tbuf + lane * 9;
                        t[0] = make_uint2(x.y, x.z & 0xffffu);
#pragma unroll
                        for (int l = 0; l < 8; l++) {
                            uint32_t v = ((A1 << l) + B1) >> (l + 6);
                            if (CHECK_M && (1u << l) > M) v = (uint32_t)exec_time(x.x, kk, 1u << l, M);
                            t[l + 1] = make_uint2(v, 1u << l);
                        }
                        endg = (x.z >> 24) != 0;
                        const uint4 *cw = (const uint4 *)(cbuf + lane * 64);
                        uint32_t acc = 0;
#pragma unroll
                        for (int q = 0; q < 4; q++) {  // rotated: 8 lanes hit 8 distinct 16-byte bank groups
                            const uint4 v = cw[(q + (lane >> 1)) & 3];
                            acc |= bytes_not_pow2(v.x) | bytes_not_pow2(v.y) | bytes_not_pow2(v.z) |
                                   bytes_not_pow2(v.w);
                        }
                        odd = acc != 0;
                    }
                    const uint32_t endm = __ballot_sync(FULL, endg);
                    const uint32_t oddm = __ballot_sync(FULL, odd);
                    const uint32_t startm = (endm << 1) | carry;
                    carry = (endm >> (rn - 1)) & 1u;
                    __syncwarp();
                    auto rows = [&](auto exact) {
#pragma unroll 4
                        for (int r = 0; r < rn; r++) {
                            const uint32_t w2 = *(const uint16_t *)(cbuf + r * 64 + 2 * lane);
                            const uint32_t ma = w2 & 0xffu, mb = w2 >> 8;
                            const uint2 *tr = tbuf + r * 9 + 1;
                            uint2 ta = tr[high_bit(ma)], tb = tr[high_bit(mb)];
                            const uint32_t bit = 1u << r;
                            if (decltype(exact)::value && (oddm & bit)) {
                                const uint4 x = pbuf[r];
                                const uint32_t kk = (x.z >> 16) & 0xffu;
                                if (ma & (ma - 1)) ta = make_uint2((uint32_t)exec_time(x.x, kk, ma, M), ma);
                                if (mb & (mb - 1)) tb = make_uint2((uint32_t)exec_time(x.x, kk, mb, M), mb);
                            }
                            group_step(startm & bit, endm & bit, ta, tb, M, gmax0, gmax1, gsum0, gsum1, gm0, gm1,
                                       b0, b1);
                        }
                    };
                    if (oddm)
                        rows(std::true_type());
                    else
                        rows(std::false_type());
                } else {  // 64-bit sums: exec_time for every byte
                    for (int r = 0; r < rn; r++) {
                        const uint4 x = pbuf[r];
                        const uint32_t kk = (x.z >> 16) & 0xffu, m0 = x.z & 0xffffu;
                        const uint32_t w2 = *(const uint16_t *)(cbuf + r * 64 + 2 * lane);
                        const uint32_t ma = w2 & 0xffu, mb = w2 >> 8;
                        const uint64_t ca = ma ? exec_time(x.x, kk, ma, M) : (uint64_t)x.y;
                        const uint64_t cv = mb ? exec_time(x.x, kk, mb, M) : (uint64_t)x.y;
                        gmax0 = ca > gmax0 ? ca : gmax0;
                        gmax1 = cv > gmax1 ? cv : gmax1;
                        gsum0 += ca;
                        gsum1 += cv;
                        gm0 += ma ? ma : m0;
                        gm1 += mb ? mb : m0;
                        if (x.z >> 24) {
                            b0 += gm0 <= M ? gmax0 : gsum0;
                            b1 += gm1 <= M ? gmax1 : gsum1;
                            gmax0 = gmax1 = gsum0 = gsum1 = 0;
                            gm0 = gm1 = 0;
                        }
                    }
                }
                __syncwarp();  // the buffer and the table are read
                buf ^= 1;
            }
            // add the item's partial bounds into its DAG's accumulators (reductions: no wait)
            unsigned long long *acc = ch.acc + (int64_t)rec.x * n_cand + vi * a.n_alloc + cb * 64 + 2 * lane;
            atomicAdd(acc, (unsigned long long)b0);
            atomicAdd(acc + 1, (unsigned long long)b1);
        };
        if (rec.w & 1)
            run_item(std::true_type());
        else
            run_item(std::false_type());
        j = jn;
        vi = vn;
        cb = cbn;
        rec = recn;
    }
    if (failed) {
        // a copy stalled: report it, and give the copies in flight a bounded chance to land
        // before the CTA's shared memory is released
        if (lane == 0) {
            if (a.err) atomicExch(a.err, DAGRT_E_TIMEOUT);
            for (int b = 0; b < 2; b++)
                if ((inflight >> b) & 1u) mbar_wait(&bar[b], (parity >> b) & 1u);
        }
        __syncwarp();
    }
}

// The candidate bytes as a 2-D tensor of bytes for TMA: `rows` allocation rows of `stride`
// bytes (a multiple of 16, the base 16-byte aligned: both checked by the API), boxes of 64
// bytes x kBoxRows rows, no swizzle, zero fill past the last row. cuTensorMapEncodeTiled
// (host-side encoding only) is taken from the driver through the runtime's entry-point query,
// so the library links no driver stub.
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled() {
    static const EncodeTiledFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return (EncodeTiledFn) nullptr;
        return (EncodeTiledFn)p;
    }();
    return fn;
}

static cudaError_t encode_alloc_map(const BoundArgs &a, int64_t rows, CUtensorMap *map) {
    std::memset(map, 0, sizeof *map);
    if (rows <= 0) return cudaSuccess;  // no candidate rows: no work item copies any
    const EncodeTiledFn fn = encode_tiled();
    if (!fn) return cudaErrorNotSupported;
    const cuuint64_t dim[2] = {(cuuint64_t)a.stride, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)a.stride};
    const cuuint32_t box[2] = {64u, (cuuint32_t)kBoxRows};
    const cuuint32_t estr[2] = {1u, 1u};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, (void *)a.m_alloc, dim, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t bound_launch(const BoundArgs &a, const ChunkArgs *ch, int n_sm, cudaStream_t st, int *launches) {
    *launches = 0;
    if (a.n_dags == 0) return cudaSuccess;
    const int n_cand = a.n_variants * a.n_alloc;
    const bool items = ch != nullptr;
    if (items) {
        // the item counter is zero here: set when the scratch was allocated, and reset by
        // k_bound_finish at the end of every call
        cudaError_t e;
        CUtensorMap tmap;
        if ((e = encode_alloc_map(a, ch->alloc_rows, &tmap)) != cudaSuccess) return e;
        const int warps = ch->warps < 1 ? 1 : (ch->warps > kMaxItemWarps ? kMaxItemWarps : ch->warps);
        const int smem = warps * kWarpBytes + 128;  // + alignment of the warps' buffers to 128 bytes
        auto kern = a.M < 128 ? k_bound_items<true> : k_bound_items<false>;
        int per_sm = 0;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxItemWarps * kWarpBytes + 128);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
        kern<<<per_sm * n_sm, warps * 32, smem, st>>>(tmap, a, *ch);
        const int g = a.n_dags < 32 * n_sm ? a.n_dags : 32 * n_sm;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(g);
        cfg.blockDim = dim3(32);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        if ((e = cudaLaunchKernelEx(&cfg, k_bound_finish, a, *ch)) != cudaSuccess) return e;
        *launches += 2;
        return cudaSuccess;  // k_bound_finish evaluated the DAGs that need 64-bit sums
    }
    // candidates per thread: a thread's candidates must never straddle two variants
    const int cpt = a.n_alloc % 4 == 0 ? 4 : (a.n_alloc % 2 == 0 ? 2 : 1);
    int threads = (n_cand + cpt - 1) / cpt;
    threads = (threads + 31) / 32 * 32;
    if (threads > kBoundMaxThreads) threads = kBoundMaxThreads;
    // rows per tile: about 8 KB of candidate bytes (plan rows when generating) per stage
    int T = (int)(8192 / ((a.gen ? 0 : a.stride) + 16ll * a.n_variants));
    if (T < 1) T = 1;
    if (T > 128) T = 128;
    const TileLayout L = tile_layout(T, a.gen ? 0 : a.stride, a.n_variants);
    const int64_t smem = 2 * L.stage_bytes;
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    using K = void (*)(BoundArgs, int);
    const K fast = a.gen ? (cpt == 4 ? k_bound_tma<4, true, true> : cpt == 2 ? k_bound_tma<2, true, true>
                                                                           : k_bound_tma<1, true, true>)
                         : (cpt == 4 ? k_bound_tma<4, false, true> : cpt == 2 ? k_bound_tma<2, false, true>
                                                                             : k_bound_tma<1, false, true>);
    const K wide = a.gen ? (cpt == 4 ? k_bound_tma<4, true, false> : cpt == 2 ? k_bound_tma<2, true, false>
                                                                            : k_bound_tma<1, true, false>)
                         : (cpt == 4 ? k_bound_tma<4, false, false> : cpt == 2 ? k_bound_tma<2, false, false>
                                                                              : k_bound_tma<1, false, false>);
    for (K kern : {fast, wide}) {
        int per_sm = 0;
        const int mx = max_dynamic_smem(kern);
        if (smem > mx) return cudaErrorInvalidValue;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
        int grid = a.n_dags;
        if (grid > per_sm * n_sm) grid = per_sm * n_sm;
        if (kern == wide && grid > 2 * n_sm) grid = 2 * n_sm;  // few DAGs need the 64-bit form
        kern<<<grid, threads, smem, st>>>(a, T);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        ++*launches;
    }
    return cudaSuccess;
}

}  // namespace dagrt
