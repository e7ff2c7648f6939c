// bound.cu -- bound of candidate allocations on fixed schedule structures, and the argmin
// over candidates per DAG.
//
// A plan is the schedule of one structure variant: rows ordered by the group they run in,
// each with its load, parallel fraction and scheduled SMs. For candidate allocation m^c
// the bound is a max-plus sweep along the group chain (Theorem 1): F_j = F_{j-1} + R_j,
// with R_j = max C_i over the group if its SMs fit in M (Lemma 1), else sum C_i.
//
// One CTA per DAG. Row tiles of the DAG -- the candidate bytes of T rows (one contiguous
// run of T * cand_stride bytes) and the T plan rows of every variant in the call -- stream
// from global to shared memory with TMA bulk copies into two stages that complete on
// mbarriers, so the loads of tile i+1 overlap the evaluation of tile i. Each thread owns
// 1, 2 or 4 adjacent candidates of one variant (one shared load per row), chosen so that a
// warp covers a single variant when possible, keeps their running group states, and the
// argmin over the DAG's candidates is reduced with warp shuffles and shared memory in the
// same kernel.
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

// bounded wait on a stage; false after kSpinLimit polls
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    for (uint32_t i = 0; i < kSpinLimit; i++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
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

template <int CPT, bool GEN>
__global__ void __launch_bounds__(kBoundMaxThreads) k_bound_tma(BoundArgs a, int T) {
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int s_abort;
    __shared__ int64_t s_bb[kBoundMaxThreads / 32];
    __shared__ int32_t s_bc[kBoundMaxThreads / 32];
    __shared__ uint8_t s_lev[16];
    const int nv = a.n_variants;
    const int n_cand = nv * a.n_alloc;
    const uint32_t M = (uint32_t)a.M;
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
        for (int v = 0; v < nv; v++)
            if (a.status[v][d] == DAGRT_OK) rows_max = max(rows_max, a.nrows[v][d]);
        const int ntile = (rows_max + T - 1) / T;
        int64_t best_b = 0;
        int32_t best_c = -1;

        for (int c0 = 0; c0 < n_cand; c0 += blockDim.x * CPT) {
            const int c = c0 + tid * CPT;
            const bool active = c < n_cand;
            const int vi = active ? c / a.n_alloc : 0;
            const bool valid = active && a.status[vi][d] == DAGRT_OK;
            const int my_rows = valid ? a.nrows[vi][d] : 0;
            const bool fit = valid && (a.pflag[vi][d] & 1);
            uint64_t bound[CPT];
            uint64_t gmax[CPT], gsum[CPT];              // group state, 64-bit path
            uint32_t gmax32[CPT], gsum32[CPT], gm[CPT];  // group state, 32-bit path; SM sum
#pragma unroll
            for (int i = 0; i < CPT; i++) bound[i] = gmax[i] = gsum[i] = gmax32[i] = gsum32[i] = gm[i] = 0;

            // tile i of the DAG into stage i & 1
            auto issue = [&](int i) {
                const int s = i & 1;
                const int r0 = i * T;
                const int rn = min(T, rows_max - r0);
                const uint32_t cb = (uint32_t)(rn * stride);
                issued[s]++;
                mbar_expect_tx(&bar[s], cb + (uint32_t)(nv * rn * 16));
                if (!GEN) bulk_g2s(stage[s], a.m_alloc + (rbase + r0) * stride, cb, &bar[s]);
                for (int v = 0; v < nv; v++)
                    bulk_g2s(stage[s] + L.cand_bytes + (int64_t)v * T * 16, a.plan[v] + rbase + r0,
                             (uint32_t)(rn * 16), &bar[s]);
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
                if (!ok) atomicExch(&s_abort, 1);
                __syncthreads();
                if (s_abort) break;
                const int r0 = i * T;
                const int rn = min(T, my_rows - r0);
                const unsigned char *cbuf = stage[s] + c;  // candidate column c of row r0
                const uint4 *pl = (const uint4 *)(stage[s] + L.cand_bytes) + (int64_t)vi * T;
                for (int rr = 0; rr < rn; rr++) {
                    const uint4 x = pl[rr];
                    const uint32_t k = (x.z >> 16) & 0xffu, m0 = x.z & 0xffffu;
                    const bool last = (x.z >> 24) != 0;
                    uint32_t m4;
                    if (GEN) {
                        m4 = 0;
#pragma unroll
                        for (int q = 0; q < CPT; q++) {
                            const int cq = c + q;
                            if (cq % a.n_alloc != 0)
                                m4 |= (uint32_t)s_lev[gen_level(a.seed, d, cq, r0 + rr, a.n_levels)] << (8 * q);
                        }
                    } else if (CPT == 4) {
                        m4 = *(const uint32_t *)(cbuf + rr * stride);
                    } else if (CPT == 2) {
                        m4 = *(const uint16_t *)(cbuf + rr * stride);
                    } else {
                        m4 = cbuf[rr * stride];
                    }
                    if (fit) {
                        // C for m = 2^l <= M, 32-bit exact for this DAG:
                        // ceil(x (64m - k(m-1)) / 64m) = ((x(64-k) + 64) << l + x k - 1) >> (l + 6)
                        const uint32_t A1 = x.x * (64u - k) + 64u, B1 = x.x * k - 1u;
                        uint32_t cc[CPT];
                        bool slow = false;
#pragma unroll
                        for (int q = 0; q < CPT; q++) {
                            const uint32_t m = (m4 >> (8 * q)) & 0xffu;
                            const int l = 31 - __clz(m | (m == 0));
                            cc[q] = m ? ((A1 << l) + B1) >> (l + 6) : x.y;
                            slow |= ((m & (m - 1)) != 0) | (m > M);
                        }
                        if (slow) {  // an allocation that is not a power of two, or above M
#pragma unroll
                            for (int q = 0; q < CPT; q++) {
                                const uint32_t m = (m4 >> (8 * q)) & 0xffu;
                                if (((m & (m - 1)) != 0) | (m > M)) cc[q] = (uint32_t)exec_time(x.x, k, m, M);
                            }
                        }
#pragma unroll
                        for (int q = 0; q < CPT; q++) {
                            const uint32_t m = (m4 >> (8 * q)) & 0xffu;
                            gmax32[q] = cc[q] > gmax32[q] ? cc[q] : gmax32[q];
                            gsum32[q] += cc[q];
                            gm[q] += m ? m : m0;
                        }
                        if (last) {
#pragma unroll
                            for (int q = 0; q < CPT; q++) {
                                bound[q] += gm[q] <= M ? gmax32[q] : gsum32[q];
                                gmax32[q] = gsum32[q] = gm[q] = 0;
                            }
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < CPT; q++) {
                            const uint32_t m = (m4 >> (8 * q)) & 0xffu;
                            const uint64_t ccw = m ? exec_time(x.x, k, m, M) : (uint64_t)x.y;
                            gmax[q] = ccw > gmax[q] ? ccw : gmax[q];
                            gsum[q] += ccw;
                            gm[q] += m ? m : m0;
                        }
                        if (last) {
#pragma unroll
                            for (int q = 0; q < CPT; q++) {
                                bound[q] += gm[q] <= M ? gmax[q] : gsum[q];
                                gmax[q] = gsum[q] = 0;
                                gm[q] = 0;
                            }
                        }
                    }
                }
                __syncthreads();  // every thread is done with stage s
                if (tid == 0 && i + 2 < ntile) {
                    fence_proxy_async();
                    issue(i + 2);
                }
            }
            if (s_abort) break;
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
                for (int r = tid; r < rows; r += blockDim.x)
                    a.best_m[rbase + r] = wc % a.n_alloc == 0 ? 0 : s_lev[gen_level(a.seed, d, wc, r, a.n_levels)];
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

cudaError_t bound_launch(const BoundArgs &a, int n_sm, cudaStream_t st) {
    if (a.n_dags == 0) return cudaSuccess;
    const int n_cand = a.n_variants * a.n_alloc;
    // candidates per thread: a warp should cover candidates of one variant only (uniform
    // group boundaries), and a thread's candidates must never straddle two variants
    int cpt = 1;
    for (int q : {4, 2})
        if (a.n_alloc % (32 * q) == 0) { cpt = q; break; }
    if (cpt == 1 && a.n_alloc % 32 != 0) cpt = a.n_alloc % 4 == 0 ? 4 : (a.n_alloc % 2 == 0 ? 2 : 1);
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
    void (*kern)(BoundArgs, int) =
        a.gen ? (cpt == 4 ? k_bound_tma<4, true> : cpt == 2 ? k_bound_tma<2, true> : k_bound_tma<1, true>)
              : (cpt == 4 ? k_bound_tma<4, false> : cpt == 2 ? k_bound_tma<2, false> : k_bound_tma<1, false>);
    int per_sm = 0;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int grid = a.n_dags;
    if (grid > per_sm * n_sm) grid = per_sm * n_sm;
    kern<<<grid, threads, smem, st>>>(a, T);
    return cudaGetLastError();
}

}  // namespace dagrt
