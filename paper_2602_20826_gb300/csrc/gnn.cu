// gnn.cu -- learned proposer: message-passing network forward/backward on the tensor
// cores (tcgen05 + TMEM), Adam, and top-k decoding of per-kernel SM-level distributions.
//
// GEMM tiles are 128 node rows. Operands are staged by the CTA's threads into shared memory
// in the K-major no-swizzle layout (umma.cuh): the forward A tile is built directly from
// neighbour gathers ([h | mean over predecessors | mean over successors]), so the
// concatenated layer input never goes to HBM. Reductions over nodes (weight gradients)
// run in a fixed order (per-CTA partials in TMEM, then a fixed-order sum), so training is
// deterministic for a given GPU.
#include <cuda_bf16.h>

#include "dagrt_internal.cuh"
#include "gnn.cuh"
#include "umma.cuh"

namespace dagrt {

constexpr uint32_t kWaitLimit = 1u << 24;

__device__ __forceinline__ float bf2f(uint16_t x) { return __uint_as_float((uint32_t)x << 16); }
__device__ __forceinline__ uint16_t f2bf(float f) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(f));
}

// ------------------------------------------------------------------ graph
constexpr int kGraphSmemV = 1024;  // DAGs up to this many nodes build in shared memory
constexpr int kGraphWarps = 8;     // warps per CTA of k_gnn_graph
constexpr int kGraphWarpInts = 2 * kGraphSmemV + 2;

// One warp per DAG: global successor CSR, in-degrees, then predecessor lists with every
// list in increasing predecessor id (deterministic). DAGs of at most kGraphSmemV nodes:
// in-degree counts by shared-memory atomics, their exclusive scan, then a stable fill --
// the edges in CSR order (increasing source), 32 at a time; lanes with the same target
// rank themselves with a match, so each list comes out sorted. Larger DAGs: counts and
// fill in global memory with atomics, then an insertion sort per list.
__global__ void __launch_bounds__(32 * kGraphWarps)
    k_gnn_graph(int32_t n_dags, const int64_t *node_off, const int64_t *edge_off, const int32_t *row_ptr,
                const int32_t *col, const int32_t *status, int32_t *pred_off, int32_t *pred_idx, int32_t *succ_off,
                int32_t *succ_idx, int32_t *cursor) {
    extern __shared__ int32_t s_graph[];
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    int32_t *off = s_graph + (threadIdx.x >> 5) * kGraphWarpInts;  // [V]: counts, then next free slot
    int32_t *rps = off + kGraphSmemV;                                // [V + 1]: the DAG's row pointers
    for (int d = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; d < n_dags; d += warps) {
        const int64_t n0 = node_off[d], e0 = edge_off[d];
        const int V = (int)(node_off[d + 1] - n0);
        if (status[d] != DAGRT_OK) {  // a DAG the scheduler rejected: its CSR is not trusted
            for (int v = lane; v < V; v += 32) {
                succ_off[n0 + v] = (int32_t)e0;
                pred_off[n0 + v] = (int32_t)e0;
            }
            if (lane == 0 && d == n_dags - 1) {
                pred_off[node_off[n_dags]] = (int32_t)edge_off[n_dags];
                succ_off[node_off[n_dags]] = (int32_t)edge_off[n_dags];
            }
            continue;
        }
        const int32_t *rp = row_ptr + n0 + d;
        const int32_t *cl = col + e0;
        if (V <= kGraphSmemV) {
            const int E = rp[V];
            for (int v = lane; v <= V; v += 32) rps[v] = rp[v];
            for (int v = lane; v < V; v += 32) {
                off[v] = 0;
                succ_off[n0 + v] = (int32_t)(e0 + rp[v]);
            }
            for (int e = lane; e < E; e += 32) succ_idx[e0 + e] = (int32_t)(n0 + cl[e]);
            __syncwarp();
            for (int e = lane; e < E; e += 32) atomicAdd(&off[cl[e]], 1);
            __syncwarp();
            int carry = 0;  // exclusive scan of the in-degrees, 32 nodes at a time
            for (int base = 0; base < V; base += 32) {
                const int v = base + lane;
                const int c = v < V ? off[v] : 0;
                int x = c;
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(FULL, x, o);
                    if (lane >= o) x += y;
                }
                if (v < V) {
                    pred_off[n0 + v] = (int32_t)(e0 + carry + x - c);
                    off[v] = carry + x - c;
                }
                carry += __shfl_sync(FULL, x, 31);
            }
            if (lane == 0 && d == n_dags - 1) {
                pred_off[node_off[n_dags]] = (int32_t)edge_off[n_dags];
                succ_off[node_off[n_dags]] = (int32_t)edge_off[n_dags];
            }
            __syncwarp();
            int u = 0;  // source row of the chunk's first edge
            for (int base = 0; base < E; base += 32) {
                const int e = base + lane;
                const bool act = e < E;
                const int t = act ? cl[e] : -1;
                int r = u;
                if (act)
                    while (rps[r + 1] <= e) r++;
                const uint32_t same = __match_any_sync(FULL, t);  // lanes of this chunk with target t
                const int rank = __popc(same & ((1u << lane) - 1));
                const int slot = act ? off[t] + rank : 0;
                __syncwarp();
                if (act) {
                    if (rank == __popc(same) - 1) off[t] = slot + 1;  // the set's last lane moves the cursor
                    pred_idx[e0 + slot] = (int32_t)(n0 + r);
                }
                u = __shfl_sync(FULL, r, 31);
                __syncwarp();
            }
            continue;
        }
        for (int v = lane; v < V; v += 32) {
            succ_off[n0 + v] = (int32_t)(e0 + rp[v]);
            cursor[n0 + v] = 0;
        }
        for (int e = lane; e < rp[V]; e += 32) succ_idx[e0 + e] = (int32_t)(n0 + cl[e]);
        __syncwarp();
        for (int v = lane; v < V; v += 32)
            for (int e = rp[v]; e < rp[v + 1]; e++) atomicAdd(&cursor[n0 + cl[e]], 1);
        __syncwarp();
        // exclusive scan of in-degrees -> pred_off (32 nodes at a time)
        int carry = (int)e0;
        for (int base = 0; base < V; base += 32) {
            const int v = base + lane;
            const int c = v < V ? cursor[n0 + v] : 0;
            int x = c;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(FULL, x, o);
                if (lane >= o) x += y;
            }
            if (v < V) pred_off[n0 + v] = carry + x - c;
            carry += __shfl_sync(FULL, x, 31);
        }
        __syncwarp();
        if (lane == 0 && d == n_dags - 1) {
            pred_off[node_off[n_dags]] = (int32_t)edge_off[n_dags];
            succ_off[node_off[n_dags]] = (int32_t)edge_off[n_dags];
        }
        for (int v = lane; v < V; v += 32) cursor[n0 + v] = 0;
        __syncwarp();
        for (int u = lane; u < V; u += 32)  // fill in any order ...
            for (int e = rp[u]; e < rp[u + 1]; e++) {
                const int s = cl[e];
                pred_idx[pred_off[n0 + s] + atomicAdd(&cursor[n0 + s], 1)] = (int32_t)(n0 + u);
            }
        __syncwarp();
        for (int v = lane; v < V; v += 32) {  // ... then sort each list (increasing predecessor id)
            int32_t *p = pred_idx + pred_off[n0 + v];
            const int n = cursor[n0 + v];
            for (int i = 1; i < n; i++) {
                const int32_t x = p[i];
                int j = i - 1;
                while (j >= 0 && p[j] > x) {
                    p[j + 1] = p[j];
                    j--;
                }
                p[j + 1] = x;
            }
        }
        __syncwarp();
    }
}

cudaError_t gnn_build_graph(int32_t n_dags, const int64_t *node_off, const int64_t *edge_off, const int32_t *row_ptr,
                            const int32_t *col, const int32_t *status, int32_t *pred_off, int32_t *pred_idx,
                            int32_t *succ_off, int32_t *succ_idx, int32_t *cursor, int n_sm, cudaStream_t st) {
    if (n_dags == 0) return cudaSuccess;
    int grid = (n_dags + kGraphWarps - 1) / kGraphWarps;
    if (grid > 16 * n_sm) grid = 16 * n_sm;
    const int smem = kGraphWarps * kGraphWarpInts * (int)sizeof(int32_t);
    cudaError_t e = cudaFuncSetAttribute(k_gnn_graph, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k_gnn_graph<<<grid, 32 * kGraphWarps, smem, st>>>(n_dags, node_off, edge_off, row_ptr, col, status, pred_off,
                                                      pred_idx, succ_off, succ_idx, cursor);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ features
// x = [log2 C^ / 32, k / 64, log2(1 + indeg) / 8, log2(1 + outdeg) / 8, level / depth,
//      W^anc / sum C^, log2 m / 12 (the paper schedule's SMs), 1, 0 ...] (16 bf16)
__global__ void k_gnn_features(int32_t n_dags, const int64_t *node_off, const int64_t *wcet, const uint8_t *k64,
                               const int32_t *level, const int64_t *wanc, const int32_t *m, const int32_t *status,
                               GnnGraph g, uint16_t *x) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int d = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; d < n_dags; d += warps) {
        const int64_t n0 = node_off[d];
        const int V = (int)(node_off[d + 1] - n0);
        if (status[d] != DAGRT_OK) {  // no schedule outputs: zero features
            for (int v = lane; v < V; v += 32) {
                uint4 *dst = (uint4 *)(x + (n0 + v) * kFeat);
                dst[0] = make_uint4(0, 0, 0, 0);
                dst[1] = make_uint4(0, 0, 0, 0);
            }
            continue;
        }
        double tot = 0;
        int depth = 0;
        for (int v = lane; v < V; v += 32) {
            tot += (double)wcet[n0 + v];
            depth = max(depth, level[n0 + v]);
        }
        for (int o = 16; o > 0; o >>= 1) {
            tot += __shfl_xor_sync(FULL, tot, o);
            depth = max(depth, __shfl_xor_sync(FULL, depth, o));
        }
        for (int v = lane; v < V; v += 32) {
            const int64_t i = n0 + v;
            float f[kFeat];
#pragma unroll
            for (int q = 0; q < kFeat; q++) f[q] = 0.f;
            f[0] = log2f((float)wcet[i]) / 32.f;
            f[1] = (float)k64[i] / 64.f;
            f[2] = log2f(1.f + (float)(g.pred_off[i + 1] - g.pred_off[i])) / 8.f;
            f[3] = log2f(1.f + (float)(g.succ_off[i + 1] - g.succ_off[i])) / 8.f;
            f[4] = depth > 0 ? (float)level[i] / (float)depth : 0.f;
            f[5] = tot > 0 ? (float)((double)wanc[i] / tot) : 0.f;
            f[6] = log2f((float)max(m[i], 1)) / 12.f;
            f[7] = 1.f;
            uint32_t w[kFeat / 2];
#pragma unroll
            for (int q = 0; q < kFeat / 2; q++) w[q] = (uint32_t)f2bf(f[2 * q]) | ((uint32_t)f2bf(f[2 * q + 1]) << 16);
            uint4 *dst = (uint4 *)(x + i * kFeat);
            dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
            dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
        }
    }
}

cudaError_t gnn_features(int32_t n_dags, const int64_t *node_off, const int64_t *wcet, const uint8_t *k64,
                         const int32_t *level, const int64_t *wanc, const int32_t *m, const int32_t *status, GnnGraph g,
                         uint16_t *x, int n_sm, cudaStream_t st) {
    if (n_dags == 0) return cudaSuccess;
    int grid = (n_dags + 7) / 8;
    if (grid > 16 * n_sm) grid = 16 * n_sm;
    k_gnn_features<<<grid, 256, 0, st>>>(n_dags, node_off, wcet, k64, level, wanc, m, status, g, x);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ aggregation
// Row v of the concatenated layer input, features [4*lane, 4*lane+4) of each third:
// self, mean over predecessors, mean over successors (fp32 sums, one rounding to bf16).
template <int KIN>
__device__ __forceinline__ void gather_row(const GnnGraph &g, const uint16_t *__restrict__ h, int64_t v, int lane,
                                           float *self, float *mp, float *ms) {
#pragma unroll
    for (int q = 0; q < 4; q++) self[q] = mp[q] = ms[q] = 0.f;
    if (lane * 4 >= KIN || v >= g.n_nodes) return;
    const uint2 sv = __ldg((const uint2 *)(h + v * KIN) + lane);
    self[0] = bf2f(sv.x & 0xffff);
    self[1] = bf2f(sv.x >> 16);
    self[2] = bf2f(sv.y & 0xffff);
    self[3] = bf2f(sv.y >> 16);
    const int pb = g.pred_off[v], pe = g.pred_off[v + 1];
    for (int e = pb; e < pe; e++) {
        const uint2 u = __ldg((const uint2 *)(h + (int64_t)g.pred_idx[e] * KIN) + lane);
        mp[0] += bf2f(u.x & 0xffff);
        mp[1] += bf2f(u.x >> 16);
        mp[2] += bf2f(u.y & 0xffff);
        mp[3] += bf2f(u.y >> 16);
    }
    const int sb = g.succ_off[v], se = g.succ_off[v + 1];
    for (int e = sb; e < se; e++) {
        const uint2 u = __ldg((const uint2 *)(h + (int64_t)g.succ_idx[e] * KIN) + lane);
        ms[0] += bf2f(u.x & 0xffff);
        ms[1] += bf2f(u.x >> 16);
        ms[2] += bf2f(u.y & 0xffff);
        ms[3] += bf2f(u.y >> 16);
    }
    const float ip = pe > pb ? 1.f / (float)(pe - pb) : 0.f, is = se > sb ? 1.f / (float)(se - sb) : 0.f;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        mp[q] *= ip;
        ms[q] *= is;
    }
}

__device__ __forceinline__ uint2 pack4(const float *f) {
    return make_uint2((uint32_t)f2bf(f[0]) | ((uint32_t)f2bf(f[1]) << 16),
                      (uint32_t)f2bf(f[2]) | ((uint32_t)f2bf(f[3]) << 16));
}

// ------------------------------------------------------------------ forward layer
// Persistent CTAs of kFwdWarps warps over 128-row tiles. The A tile (K = 3 KIN) is gathered
// straight into shared memory: a group of KIN/8 lanes owns one row (16 bytes = 8 features
// per lane), so a warp gathers 32 / (KIN/8) rows at once, and the neighbour loops are
// unrolled by 4 so that several neighbour rows are in flight per lane (the gather is
// latency-bound: neighbours are scattered over the DAG). One thread then issues the
// tcgen05 MMA chain against the resident W^T; the epilogue (bias, ReLU, bf16) reads TMEM with
// the first 16 warps: warp w takes TMEM lanes 32 (w % 4) .. + 31 and columns 32 (w / 4) .. + 31,
// while the other 16 warps already gather their rows of the next tile.
constexpr int kFwdWarps = 32;

__device__ __forceinline__ void acc8(float *a, uint4 u) {
    a[0] += bf2f(u.x & 0xffff);
    a[1] += bf2f(u.x >> 16);
    a[2] += bf2f(u.y & 0xffff);
    a[3] += bf2f(u.y >> 16);
    a[4] += bf2f(u.z & 0xffff);
    a[5] += bf2f(u.z >> 16);
    a[6] += bf2f(u.w & 0xffff);
    a[7] += bf2f(u.w >> 16);
}

// mean over the rows idx[b .. e) of h, features [8 sub, 8 sub + 8)
template <int KIN>
__device__ __forceinline__ void mean_rows(const uint16_t *__restrict__ h, const int32_t *__restrict__ idx, int b,
                                          int e, int sub, float *m) {
#pragma unroll
    for (int q = 0; q < 8; q++) m[q] = 0.f;
    int i = b;
    for (; i + 4 <= e; i += 4) {
        const int32_t j0 = __ldg(idx + i), j1 = __ldg(idx + i + 1), j2 = __ldg(idx + i + 2), j3 = __ldg(idx + i + 3);
        const uint4 u0 = __ldg((const uint4 *)(h + (int64_t)j0 * KIN) + sub);
        const uint4 u1 = __ldg((const uint4 *)(h + (int64_t)j1 * KIN) + sub);
        const uint4 u2 = __ldg((const uint4 *)(h + (int64_t)j2 * KIN) + sub);
        const uint4 u3 = __ldg((const uint4 *)(h + (int64_t)j3 * KIN) + sub);
        acc8(m, u0);
        acc8(m, u1);
        acc8(m, u2);
        acc8(m, u3);
    }
    for (; i < e; i++) acc8(m, __ldg((const uint4 *)(h + (int64_t)__ldg(idx + i) * KIN) + sub));
    const float inv = e > b ? 1.f / (float)(e - b) : 0.f;
#pragma unroll
    for (int q = 0; q < 8; q++) m[q] *= inv;
}

__device__ __forceinline__ uint4 pack8(const float *f) {
    return make_uint4((uint32_t)f2bf(f[0]) | ((uint32_t)f2bf(f[1]) << 16), (uint32_t)f2bf(f[2]) | ((uint32_t)f2bf(f[3]) << 16),
                      (uint32_t)f2bf(f[4]) | ((uint32_t)f2bf(f[5]) << 16), (uint32_t)f2bf(f[6]) | ((uint32_t)f2bf(f[7]) << 16));
}

// rows [32 w / ... ) of the tile: the A operand [h | mean_pred h | mean_succ h] in K-major order
template <int KIN>
__device__ __forceinline__ void gather_tile(const GnnGraph &g, const uint16_t *__restrict__ h_in, int64_t tile,
                                            unsigned char *sA, int w, int lane) {
    constexpr int K = 3 * KIN, LPR = KIN / 8, RPW = 32 / LPR;  // lanes per row, rows per warp pass
    constexpr int ROWS = 128 / kFwdWarps;                      // rows of the tile per warp
    const int sub = lane % LPR;
    for (int r0 = 0; r0 < ROWS; r0 += RPW) {
        const int rl = r0 + lane / LPR;
        if (rl >= ROWS) continue;
        const int r = w * ROWS + rl;
        const int64_t v = tile * 128 + r;
        uint4 s0 = make_uint4(0, 0, 0, 0), s1 = s0, s2 = s0;
        if (v < g.n_nodes) {
            s0 = __ldg((const uint4 *)(h_in + v * KIN) + sub);
            float m[8];
            mean_rows<KIN>(h_in, g.pred_idx, g.pred_off[v], g.pred_off[v + 1], sub, m);
            s1 = pack8(m);
            mean_rows<KIN>(h_in, g.succ_idx, g.succ_off[v], g.succ_off[v + 1], sub, m);
            s2 = pack8(m);
        }
        *(uint4 *)(sA + kmajor_off(r, 8 * sub, K)) = s0;
        *(uint4 *)(sA + kmajor_off(r, KIN + 8 * sub, K)) = s1;
        *(uint4 *)(sA + kmajor_off(r, 2 * KIN + 8 * sub, K)) = s2;
    }
}

template <int KIN>
__global__ void __launch_bounds__(32 * kFwdWarps) k_gnn_fwd(GnnGraph g, const uint16_t *__restrict__ h_in,
                                                            const uint16_t *__restrict__ wt,
                                                            const float *__restrict__ bias,
                                                            uint16_t *__restrict__ h_out, int32_t *err) {
    constexpr int K = 3 * KIN;
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tslot;
    __shared__ float sbias[kHidden];
    unsigned char *sA = sm, *sB = sm + 128 * K * 2;
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    for (int i = t; i < kHidden * (K / 8); i += blockDim.x) {  // W^T [H x K] -> K-major B operand
        const int r = i / (K / 8), kc = (i % (K / 8)) * 8;
        *(uint4 *)(sB + kmajor_off(r, kc, K)) = *(const uint4 *)(wt + (size_t)r * K + kc);
    }
    if (t < kHidden) sbias[t] = bias[t];
    if (w == 0) tmem_alloc(&tslot, 128);
    if (t == 0) mbar_init1(&bar);
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const uint32_t taddr = tslot;
    const int64_t n_tiles = (g.n_nodes + 127) / 128;
    const int lq = w & 3, cb = w >> 2;  // epilogue: TMEM lane quarter and 32-column block
    uint32_t phase = 0;
    bool ok = true;
    for (int64_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
        gather_tile<KIN>(g, h_in, tile, sA, w, lane);
        fence_async_smem();
        __syncthreads();
        if (t == 0) {
            tmem_fence_after();
            umma_gemm(taddr, sA, sB, K, kHidden, false);
            umma_commit(&bar);
        }
        ok = __syncthreads_and(mbar_wait_parity(&bar, phase, kWaitLimit)) != 0;  // uniform across the CTA
        phase ^= 1;
        tmem_fence_after();
        if (ok && w < 16) {
            const int64_t v = tile * 128 + 32 * lq + lane;  // this thread's TMEM lane = row 32 lq + lane
            const int c0 = 32 * cb;
            float acc[32];
            tmem_ld32(taddr + ((uint32_t)(32 * lq) << 16) + c0, acc);
            if (v < g.n_nodes) {
                uint32_t pk[16];
#pragma unroll
                for (int i = 0; i < 16; i++) {
                    const float a0 = fmaxf(acc[2 * i] + sbias[c0 + 2 * i], 0.f);
                    const float a1 = fmaxf(acc[2 * i + 1] + sbias[c0 + 2 * i + 1], 0.f);
                    pk[i] = (uint32_t)f2bf(a0) | ((uint32_t)f2bf(a1) << 16);
                }
                uint4 *dst = (uint4 *)(h_out + v * kHidden + c0);
#pragma unroll
                for (int i = 0; i < 4; i++) dst[i] = make_uint4(pk[4 * i], pk[4 * i + 1], pk[4 * i + 2], pk[4 * i + 3]);
            }
        } else if (!ok && t == 0 && err) {
            atomicExch(err, DAGRT_E_TIMEOUT);
        }
        // no barrier here: the warps without epilogue work start gathering the next tile
        // (the MMA that read the A tile has completed); the barrier after that gather orders
        // this epilogue's TMEM reads before the next MMA writes the accumulator
        tmem_fence_before();
    }
    __syncthreads();  // every epilogue has read TMEM before it is released
    if (w == 0) tmem_dealloc(taddr, 128);
}

template <int KIN>
static cudaError_t launch_fwd(GnnGraph g, const uint16_t *h_in, const uint16_t *wt, const float *bias,
                              uint16_t *h_out, int32_t *err, int n_sm, cudaStream_t st) {
    constexpr int K = 3 * KIN;
    const int smem = 2 * 128 * K * 2;
    cudaError_t e = cudaFuncSetAttribute(k_gnn_fwd<KIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gnn_fwd<KIN>, 32 * kFwdWarps, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (per_sm > 4) per_sm = 4;  // 4 x 128 TMEM columns per SM
    const int64_t n_tiles = (g.n_nodes + 127) / 128;
    int grid = (int)(n_tiles < (int64_t)n_sm * per_sm ? n_tiles : (int64_t)n_sm * per_sm);
    if (grid < 1) return cudaSuccess;
    k_gnn_fwd<KIN><<<grid, 32 * kFwdWarps, smem, st>>>(g, h_in, wt, bias, h_out, err);
    return cudaGetLastError();
}

cudaError_t gnn_layer_fwd(int kin, GnnGraph g, const uint16_t *h_in, const uint16_t *wt, const float *bias,
                          uint16_t *h_out, int32_t *err, int n_sm, cudaStream_t st) {
    if (kin == kFeat) return launch_fwd<kFeat>(g, h_in, wt, bias, h_out, err, n_sm, st);
    if (kin == kHidden) return launch_fwd<kHidden>(g, h_in, wt, bias, h_out, err, n_sm, st);
    return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------ head
// logits = h3 Wh + bh; with labels: softmax cross-entropy (mean over labelled nodes, via
// `scale` = 1 / count), dlogits and dh3 = dlogits Wh^T. One thread per node; the loss is
// reduced per CTA in a fixed order.
__global__ void __launch_bounds__(128) k_gnn_head(GnnGraph g, const uint16_t *__restrict__ h3,
                                                  const float *__restrict__ wh, const float *__restrict__ bh,
                                                  int L, const int8_t *__restrict__ labels, float scale,
                                                  float *logits, float *dlogits, float *dh3, float *loss_part) {
    __shared__ float swh[kHidden * kMaxLevels];
    __shared__ float sbh[kMaxLevels];
    __shared__ float sloss[128];
    for (int i = threadIdx.x; i < kHidden * kMaxLevels; i += blockDim.x) swh[i] = wh[i];
    if (threadIdx.x < kMaxLevels) sbh[threadIdx.x] = bh[threadIdx.x];
    __syncthreads();
    float my_loss = 0.f;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < g.n_nodes; v += (int64_t)gridDim.x * blockDim.x) {
        float z[kMaxLevels];
#pragma unroll
        for (int l = 0; l < kMaxLevels; l++) z[l] = l < L ? sbh[l] : 0.f;
        const uint4 *row = (const uint4 *)(h3 + v * kHidden);
        for (int c = 0; c < kHidden / 8; c++) {
            const uint4 q = row[c];
            const uint32_t wd[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int j = 0; j < 8; j++) {
                const float hv = bf2f((uint16_t)(wd[j >> 1] >> (16 * (j & 1))));
                const int o = 8 * c + j;
#pragma unroll
                for (int l = 0; l < kMaxLevels; l++)
                    if (l < L) z[l] = fmaf(hv, swh[o * kMaxLevels + l], z[l]);
            }
        }
        if (logits)
            for (int l = 0; l < L; l++) logits[v * L + l] = z[l];
        if (!labels) continue;
        const int y = labels[v];
        float gz[kMaxLevels];
#pragma unroll
        for (int l = 0; l < kMaxLevels; l++) gz[l] = 0.f;
        if (y >= 0 && y < L) {
            float mx = z[0];
            for (int l = 1; l < L; l++) mx = fmaxf(mx, z[l]);
            float se = 0.f;
            for (int l = 0; l < L; l++) se += __expf(z[l] - mx);
            const float lse = mx + __logf(se);
            my_loss += (lse - z[y]) * scale;
            for (int l = 0; l < L; l++) gz[l] = (__expf(z[l] - lse) - (l == y ? 1.f : 0.f)) * scale;
        }
        for (int l = 0; l < L; l++) dlogits[v * L + l] = gz[l];
        float *dr = dh3 + v * kHidden;
        for (int o = 0; o < kHidden; o++) {
            float s = 0.f;
            for (int l = 0; l < L; l++) s = fmaf(gz[l], swh[o * kMaxLevels + l], s);
            dr[o] = s;
        }
    }
    if (labels && loss_part) {
        sloss[threadIdx.x] = my_loss;
        __syncthreads();
        if (threadIdx.x == 0) {
            float s = 0.f;
            for (int i = 0; i < (int)blockDim.x; i++) s += sloss[i];
            loss_part[blockIdx.x] = s;
        }
    }
}

cudaError_t gnn_head(GnnGraph g, const uint16_t *h3, const float *wh, const float *bh, int n_levels,
                     const int8_t *labels, float scale, float *logits, float *dlogits, float *dh3,
                     float *loss_part, int n_sm, cudaStream_t st) {
    if (g.n_nodes == 0) return cudaSuccess;
    // the loss is reduced per CTA: a fixed grid keeps the summation order fixed
    k_gnn_head<<<n_sm, 128, 0, st>>>(g, h3, wh, bh, n_levels, labels, scale, logits, dlogits, dh3, loss_part);
    return cudaGetLastError();
}

// dWh = h3^T dlogits, dbh = sum dlogits: CTA c reduces a fixed node range; thread o owns
// row o of dWh (all levels), threads kHidden.. own dbh.
__global__ void __launch_bounds__(kHidden + kMaxLevels) k_gnn_head_grad(GnnGraph g, const uint16_t *__restrict__ h3,
                                                                       const float *__restrict__ dlogits, int L,
                                                                       float *part) {
    const int o = threadIdx.x;
    const int64_t per = (g.n_nodes + gridDim.x - 1) / gridDim.x;
    const int64_t v0 = blockIdx.x * per, v1 = min(g.n_nodes, v0 + per);
    float acc[kMaxLevels];
#pragma unroll
    for (int l = 0; l < kMaxLevels; l++) acc[l] = 0.f;
    for (int64_t v = v0; v < v1; v++) {
        const float hv = o < kHidden ? bf2f(h3[v * kHidden + o]) : 1.f;
#pragma unroll
        for (int l = 0; l < kMaxLevels; l++)
            if (l < L) acc[l] = fmaf(hv, dlogits[v * L + l], acc[l]);
    }
    float *pp = part + (int64_t)blockIdx.x * ParamLayout::total;
    if (o < kHidden) {
        for (int l = 0; l < kMaxLevels; l++) pp[ParamLayout::Wh + o * kMaxLevels + l] = l < L ? acc[l] : 0.f;
    } else {
        const int l = o - kHidden;
        float a = 0.f;
#pragma unroll
        for (int q = 0; q < kMaxLevels; q++)
            if (q == l) a = acc[q];
        pp[ParamLayout::bh + l] = l < L ? a : 0.f;
    }
}

cudaError_t gnn_head_grad(GnnGraph g, const uint16_t *h3, const float *dlogits, int n_levels, float *part,
                          int n_parts, cudaStream_t st) {
    k_gnn_head_grad<<<n_parts, kHidden + kMaxLevels, 0, st>>>(g, h3, dlogits, n_levels, part);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ backward: dW
// Per CTA over its tiles: dW_part += A^T dZ with A^T staged as the MMA A operand (feature
// rows x node columns) and dZ^T = (dh * [h_out > 0])^T as the B operand; db_part = column
// sums of dZ in a fixed order. Accumulators stay in TMEM across tiles (one 128-column block
// per 128 features).
template <int KIN>
__global__ void __launch_bounds__(128) k_gnn_bwd_dw(GnnGraph g, const uint16_t *__restrict__ h_in,
                                                    const uint16_t *__restrict__ h_out,
                                                    const float *__restrict__ dh_out, float *dw_part,
                                                    float *db_part, int64_t w_off, int64_t b_off, int32_t *err) {
    constexpr int K = 3 * KIN;
    constexpr int S = (K + 127) / 128;  // feature slices of 128
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tslot;
    unsigned char *sAT = sm;                    // S x [128 features x 128 rows] bf16
    unsigned char *sZT = sm + S * 128 * 128 * 2;  // [128 outputs x 128 rows] bf16
    float *sZ = (float *)(sZT + 128 * 128 * 2);   // [128 rows x 128 outputs] fp32
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    for (int i = t; i < S * 128 * 128 * 2 / 16; i += 128) ((uint4 *)sAT)[i] = make_uint4(0, 0, 0, 0);
    if (w == 0) tmem_alloc(&tslot, S * 128 <= 128 ? 128 : 512);
    if (t == 0) mbar_init1(&bar);
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const uint32_t taddr = tslot;
    const int64_t n_tiles = (g.n_nodes + 127) / 128;
    uint32_t phase = 0;
    bool ok = true, first = true;
    float db = 0.f;  // thread t owns output column t
    for (int64_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
        for (int rr = 0; rr < 32; rr++) {
            const int r = 32 * w + rr;
            float f[3][4];
            gather_row<KIN>(g, h_in, tile * 128 + r, lane, f[0], f[1], f[2]);
            if (lane * 4 < KIN)
                for (int part = 0; part < 3; part++)
                    for (int q = 0; q < 4; q++) {
                        const int feat = part * KIN + 4 * lane + q;
                        *(uint16_t *)(sAT + (feat >> 7) * (128 * 128 * 2) + kmajor_off(feat & 127, r, 128)) =
                            f2bf(f[part][q]);
                    }
        }
        {  // thread t: row t of dZ (fp32 to shared, for the bias gradient and the B operand)
            const int64_t v = tile * 128 + t;
            for (int o = 0; o < kHidden; o++) {
                float z = 0.f;
                if (v < g.n_nodes && h_out[v * kHidden + o] != 0) z = dh_out[v * kHidden + o];
                sZ[t * kHidden + o] = z;
            }
        }
        __syncthreads();
        {  // thread t: column t of dZ -> bias gradient (fixed row order) and the B operand
            float s = 0.f;
            for (int r = 0; r < 128; r++) {
                const float z = sZ[r * kHidden + t];
                s += z;
                *(uint16_t *)(sZT + kmajor_off(t, r, 128)) = f2bf(z);
            }
            db += s;
        }
        fence_async_smem();
        __syncthreads();
        if (t == 0) {
            tmem_fence_after();
            for (int s = 0; s < S; s++)
                umma_gemm(taddr + s * 128, sAT + s * (128 * 128 * 2), sZT, 128, kHidden, !first);
            umma_commit(&bar);
        }
        first = false;
        ok = __syncthreads_and(mbar_wait_parity(&bar, phase, kWaitLimit)) != 0;  // uniform across the CTA
        phase ^= 1;
        tmem_fence_after();
        __syncthreads();
    }
    if (!ok && t == 0 && err) atomicExch(err, DAGRT_E_TIMEOUT);
    float *pw = dw_part + (int64_t)blockIdx.x * ParamLayout::total;
    for (int s = 0; s < S; s++) {
        for (int c0 = 0; c0 < kHidden; c0 += 32) {
            float acc[32];
            if (!first && ok) tmem_ld32(taddr + ((uint32_t)(32 * w) << 16) + s * 128 + c0, acc);
            else
                for (int i = 0; i < 32; i++) acc[i] = 0.f;
            const int feat = s * 128 + t;  // TMEM lane t = feature row
            if (feat < K)
                for (int i = 0; i < 32; i++) pw[w_off + (int64_t)feat * kHidden + c0 + i] = acc[i];
        }
    }
    db_part[(int64_t)blockIdx.x * ParamLayout::total + b_off + t] = db;
    tmem_fence_before();
    __syncthreads();
    if (w == 0) tmem_dealloc(taddr, S * 128 <= 128 ? 128 : 512);
}

cudaError_t gnn_layer_bwd_dw(int kin, int layer, GnnGraph g, const uint16_t *h_in, const uint16_t *h_out,
                                const float *dh_out, float *part, int n_parts, int32_t *err, cudaStream_t st) {
    const int64_t woff[3] = {ParamLayout::W1, ParamLayout::W2, ParamLayout::W3};
    const int64_t boff[3] = {ParamLayout::b1, ParamLayout::b2, ParamLayout::b3};
    if (kin == kFeat) {
        constexpr int S = 1;
        const int smem = S * 128 * 128 * 2 + 128 * 128 * 2 + 128 * 128 * 4;
        cudaError_t e = cudaFuncSetAttribute(k_gnn_bwd_dw<kFeat>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        k_gnn_bwd_dw<kFeat><<<n_parts, 128, smem, st>>>(g, h_in, h_out, dh_out, part, part, woff[layer], boff[layer], err);
    } else {
        constexpr int S = 3;
        const int smem = S * 128 * 128 * 2 + 128 * 128 * 2 + 128 * 128 * 4;
        cudaError_t e = cudaFuncSetAttribute(k_gnn_bwd_dw<kHidden>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        k_gnn_bwd_dw<kHidden><<<n_parts, 128, smem, st>>>(g, h_in, h_out, dh_out, part, part, woff[layer], boff[layer],
                                                          err);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------ backward: dA
// dA = dZ W^T per 128-row tile: A operand dZ [rows x H], B operand W [K x H] (resident),
// three 128-column TMEM blocks for K = 384.
template <int KIN>
__global__ void __launch_bounds__(128) k_gnn_bwd_da(GnnGraph g, const uint16_t *__restrict__ h_out,
                                                    const float *__restrict__ dh_out,
                                                    const uint16_t *__restrict__ wb, float *da, int32_t *err) {
    constexpr int K = 3 * KIN;
    constexpr int S = (K + 127) / 128;
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tslot;
    unsigned char *sB = sm;                    // W [K x H] as B operand rows (zero-padded to S*128)
    unsigned char *sA = sm + S * 128 * kHidden * 2;  // dZ [128 x H]
    const int t = threadIdx.x, w = t >> 5;
    for (int i = t; i < S * 128 * (kHidden / 8); i += 128) {
        const int r = i / (kHidden / 8), kc = (i % (kHidden / 8)) * 8;
        uint4 val = make_uint4(0, 0, 0, 0);
        if (r < K) val = *(const uint4 *)(wb + (size_t)r * kHidden + kc);
        *(uint4 *)(sB + kmajor_off(r, kc, kHidden)) = val;
    }
    if (w == 0) tmem_alloc(&tslot, S * 128 <= 128 ? 128 : 512);
    if (t == 0) mbar_init1(&bar);
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const uint32_t taddr = tslot;
    const int64_t n_tiles = (g.n_nodes + 127) / 128;
    uint32_t phase = 0;
    bool ok = true;
    for (int64_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
        const int64_t v = tile * 128 + t;
        for (int o = 0; o < kHidden; o += 8) {
            uint32_t pk[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                float z0 = 0.f, z1 = 0.f;
                if (v < g.n_nodes) {
                    if (h_out[v * kHidden + o + 2 * q] != 0) z0 = dh_out[v * kHidden + o + 2 * q];
                    if (h_out[v * kHidden + o + 2 * q + 1] != 0) z1 = dh_out[v * kHidden + o + 2 * q + 1];
                }
                pk[q] = (uint32_t)f2bf(z0) | ((uint32_t)f2bf(z1) << 16);
            }
            *(uint4 *)(sA + kmajor_off(t, o, kHidden)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        }
        fence_async_smem();
        __syncthreads();
        if (t == 0) {
            tmem_fence_after();
            for (int s = 0; s < S; s++)
                umma_gemm(taddr + s * 128, sA, sB + s * 128 * kHidden * 2, kHidden, 128, false);
            umma_commit(&bar);
        }
        ok = __syncthreads_and(mbar_wait_parity(&bar, phase, kWaitLimit)) != 0;  // uniform across the CTA
        phase ^= 1;
        tmem_fence_after();
        if (ok) {
            for (int s = 0; s < S; s++)
                for (int c0 = 0; c0 < 128; c0 += 32) {
                    float acc[32];
                    tmem_ld32(taddr + ((uint32_t)(32 * w) << 16) + s * 128 + c0, acc);
                    if (v < g.n_nodes)
                        for (int i = 0; i < 32; i++) {
                            const int f = s * 128 + c0 + i;
                            if (f < K) da[v * K + f] = acc[i];
                        }
                }
        } else if (t == 0 && err) {
            atomicExch(err, DAGRT_E_TIMEOUT);
        }
        // no barrier here: each thread goes on to its row of the next dZ tile (the MMA that
        // read this one has completed); the barrier after that fill orders these TMEM reads
        // before the next MMA
        tmem_fence_before();
    }
    __syncthreads();  // every thread has read TMEM before it is released
    if (w == 0) tmem_dealloc(taddr, S * 128 <= 128 ? 128 : 512);
}

cudaError_t gnn_layer_bwd_da(int kin, GnnGraph g, const uint16_t *h_out, const float *dh_out, const uint16_t *wb,
                             float *da, int32_t *err, int n_sm, cudaStream_t st) {
    if (kin != kHidden) return cudaErrorInvalidValue;  // the first layer's input needs no gradient
    constexpr int S = 3;
    const int smem = S * 128 * kHidden * 2 + 128 * kHidden * 2;
    cudaError_t e = cudaFuncSetAttribute(k_gnn_bwd_da<kHidden>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int64_t n_tiles = (g.n_nodes + 127) / 128;
    int grid = (int)(n_tiles < n_sm ? n_tiles : n_sm);
    if (grid < 1) return cudaSuccess;
    k_gnn_bwd_da<kHidden><<<grid, 128, smem, st>>>(g, h_out, dh_out, wb, da, err);
    return cudaGetLastError();
}

// dh_in[u] = dA_self[u] + sum_{v in succ(u)} dA_pred[v] / indeg(v)
//                       + sum_{w in pred(u)} dA_succ[w] / outdeg(w)      (one warp per node)
template <int KIN>
__global__ void k_gnn_agg_bwd(GnnGraph g, const float *__restrict__ da, float *dh_in) {
    constexpr int K = 3 * KIN;
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < g.n_nodes; u += warps) {
        for (int f = lane; f < KIN; f += 32) {
            float s = da[u * K + f];
            for (int e = g.succ_off[u]; e < g.succ_off[u + 1]; e++) {
                const int64_t v = g.succ_idx[e];
                s += da[v * K + KIN + f] / (float)(g.pred_off[v + 1] - g.pred_off[v]);
            }
            for (int e = g.pred_off[u]; e < g.pred_off[u + 1]; e++) {
                const int64_t x = g.pred_idx[e];
                s += da[x * K + 2 * KIN + f] / (float)(g.succ_off[x + 1] - g.succ_off[x]);
            }
            dh_in[u * KIN + f] = s;
        }
    }
}

cudaError_t gnn_agg_bwd(int kin, GnnGraph g, const float *da, float *dh_in, int n_sm, cudaStream_t st) {
    if (kin != kHidden) return cudaErrorInvalidValue;
    int64_t grid = (g.n_nodes + 7) / 8;
    if (grid > 32 * n_sm) grid = 32 * n_sm;
    if (grid < 1) return cudaSuccess;
    k_gnn_agg_bwd<kHidden><<<(int)grid, 256, 0, st>>>(g, da, dh_in);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ Adam
__global__ void k_gnn_adam(float *p, float *m, float *v, const float *part, int n_parts, int64_t n, float lr,
                           float b1, float b2, float eps, float c1, float c2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float gsum = 0.f;
        for (int c = 0; c < n_parts; c++) gsum += part[(int64_t)c * n + i];
        const float mi = b1 * m[i] + (1.f - b1) * gsum;
        const float vi = b2 * v[i] + (1.f - b2) * gsum * gsum;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

cudaError_t gnn_adam(float *p, float *m, float *v, const float *part, int n_parts, int64_t n, float lr, float b1,
                     float b2, float eps, int step, cudaStream_t st) {
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    k_gnn_adam<<<(int)((n + 255) / 256), 256, 0, st>>>(p, m, v, part, n_parts, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

// bf16 copies: W^T [H x K] (forward B operand) and W [K x H] (backward B operand)
__global__ void k_gnn_refresh(const float *p, uint16_t *wt1, uint16_t *wt2, uint16_t *wt3, uint16_t *wb1,
                              uint16_t *wb2, uint16_t *wb3) {
    const int64_t woff[3] = {ParamLayout::W1, ParamLayout::W2, ParamLayout::W3};
    const int Ks[3] = {3 * kFeat, 3 * kHidden, 3 * kHidden};
    uint16_t *wt[3] = {wt1, wt2, wt3}, *wb[3] = {wb1, wb2, wb3};
    for (int l = 0; l < 3; l++) {
        const int K = Ks[l];
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)K * kHidden;
             i += (int64_t)gridDim.x * blockDim.x) {
            const int k = (int)(i / kHidden), o = (int)(i % kHidden);
            const uint16_t b = f2bf(p[woff[l] + i]);
            wb[l][i] = b;
            wt[l][(int64_t)o * K + k] = b;
        }
    }
}

cudaError_t gnn_refresh(const float *p, uint16_t *const *wt, uint16_t *const *wb, cudaStream_t st) {
    k_gnn_refresh<<<96, 256, 0, st>>>(p, wt[0], wt[1], wt[2], wb[0], wb[1], wb[2]);
    return cudaGetLastError();
}

}  // namespace dagrt

namespace dagrt {

// ------------------------------------------------------------------ top-k decode
// The network gives each node an independent distribution over levels. The k most likely
// joint assignments: start from every node's best level; any other assignment changes some
// nodes to other levels, costing delta = z_best - z_alt each (log-probability loss). Only
// the k-1 smallest deltas can appear among the k best (an assignment using a larger one is
// matched or beaten by the all-best assignment and the k-1 single changes), so the search
// runs over those items, grouped by node (at most one change per node). Groups are ordered
// by their smallest delta, options within a group ascending; a state (group g, option j,
// earlier groups fixed) has the successors: next option of g; keep g and take option 0 of
// g+1; and, from option 0 only, drop g and take option 0 of g+1. Every assignment has one
// parent and no successor is cheaper, so a best-first walk pops the k best in order.
// One warp per DAG; column 0 of every row keeps the paper's allocation (0), column 1 + j
// holds the j-th best assignment.
constexpr int kTopkMax = 16;

__global__ void __launch_bounds__(128) k_gnn_topk(int32_t n_dags, const int64_t *node_off, const float *logits,
                                                  int L, const uint8_t *levels, int k, const uint4 *plan,
                                                  const int32_t *nrows, uint8_t *best_level, uint8_t *m_alloc,
                                                  int64_t stride) {
    __shared__ float s_dv[4][32 * (kTopkMax - 1)];
    __shared__ int32_t s_dn[4][32 * (kTopkMax - 1)];
    __shared__ uint8_t s_dl[4][32 * (kTopkMax - 1)];
    __shared__ uint32_t s_mask[4][kTopkMax];
    __shared__ int s_nc[4];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int K1 = k - 1;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int d = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; d < n_dags; d += warps) {
        const int64_t n0 = node_off[d];
        const int V = (int)(node_off[d + 1] - n0);
        // per lane: the K1 smallest (delta, node, level) of its nodes, kept sorted
        float bv[kTopkMax - 1];
        int32_t bn[kTopkMax - 1];
        uint8_t bl[kTopkMax - 1];
        int cnt = 0;
        for (int v = lane; v < V; v += 32) {
            const float *z = logits + (n0 + v) * L;
            int b = 0;
            for (int l = 1; l < L; l++)
                if (z[l] > z[b]) b = l;
            best_level[n0 + v] = (uint8_t)b;
            for (int l = 0; l < L && K1 > 0; l++) {
                if (l == b) continue;
                const float dl = z[b] - z[l];
                if (cnt == K1 && !(dl < bv[K1 - 1])) continue;
                int pos = cnt < K1 ? cnt++ : K1 - 1;
                while (pos > 0 && bv[pos - 1] > dl) {
                    bv[pos] = bv[pos - 1];
                    bn[pos] = bn[pos - 1];
                    bl[pos] = bl[pos - 1];
                    pos--;
                }
                bv[pos] = dl;
                bn[pos] = v;
                bl[pos] = (uint8_t)l;
            }
        }
        for (int i = 0; i < K1; i++) {
            s_dv[wib][lane * K1 + i] = i < cnt ? bv[i] : __int_as_float(0x7f800000);
            s_dn[wib][lane * K1 + i] = i < cnt ? bn[i] : -1;
            s_dl[wib][lane * K1 + i] = i < cnt ? bl[i] : 0;
        }
        __syncwarp();
        // merge: the K1 smallest over all lanes (ties: lower node, then lower level), by a
        // warp argmin over the heads of the lanes' sorted lists
        float dv[kTopkMax - 1];
        int32_t dn[kTopkMax - 1];
        uint8_t dlv[kTopkMax - 1];
        int m = 0, hp = 0;
        for (int i = 0; i < K1; i++) {
            float hv = __int_as_float(0x7f800000);
            int32_t hn = 0x7fffffff;
            int hl = 0xff;
            if (hp < cnt) {
                hv = s_dv[wib][lane * K1 + hp];
                hn = s_dn[wib][lane * K1 + hp];
                hl = s_dl[wib][lane * K1 + hp];
            }
            float bvv = hv;
            int32_t bnn = hn;
            int bll = hl, bln = lane;
            for (int o = 16; o > 0; o >>= 1) {
                const float ov = __shfl_xor_sync(FULL, bvv, o);
                const int32_t on = __shfl_xor_sync(FULL, bnn, o);
                const int ol = __shfl_xor_sync(FULL, bll, o), oln = __shfl_xor_sync(FULL, bln, o);
                if (ov < bvv || (ov == bvv && (on < bnn || (on == bnn && (ol < bll || (ol == bll && oln < bln)))))) {
                    bvv = ov;
                    bnn = on;
                    bll = ol;
                    bln = oln;
                }
            }
            if (bnn == 0x7fffffff) break;  // every list is exhausted
            if (lane == bln) hp++;
            dv[m] = bvv;
            dn[m] = bnn;
            dlv[m] = (uint8_t)bll;
            m++;
        }
        __syncwarp();
        if (lane == 0) {
            // group-major order: groups in order of first appearance (= smallest delta)
            int gs[kTopkMax], gc[kTopkMax], G = 0, q = 0;
            bool used[kTopkMax - 1];
            for (int i = 0; i < m; i++) used[i] = false;
            for (int i = 0; i < m; i++) {
                if (used[i]) continue;
                gs[G] = q;
                gc[G] = 0;
                for (int j = i; j < m; j++)
                    if (!used[j] && dn[j] == dn[i]) {
                        used[j] = true;
                        s_dv[wib][q] = dv[j];
                        s_dn[wib][q] = dn[j];
                        s_dl[wib][q] = dlv[j];
                        q++;
                        gc[G]++;
                    }
                G++;
            }
            // best-first walk: heap entries (cost, mask of chosen items, group, option)
            constexpr int H = 3 * kTopkMax + 1;
            float hc[H];
            uint32_t hm[H];
            uint8_t hg[H], hj[H];
            int hn = 0, nc = 0;
            s_mask[wib][nc++] = 0;  // the all-best assignment
            if (G > 0) {
                hc[0] = s_dv[wib][0];
                hm[0] = 1u;
                hg[0] = 0;
                hj[0] = 0;
                hn = 1;
            }
            while (nc < k && hn > 0) {
                int bi = 0;
                for (int i = 1; i < hn; i++)
                    if (hc[i] < hc[bi] || (hc[i] == hc[bi] && hm[i] < hm[bi])) bi = i;
                const float c = hc[bi];
                const uint32_t msk = hm[bi];
                const int g = hg[bi], j = hj[bi];
                hn--;
                hc[bi] = hc[hn];
                hm[bi] = hm[hn];
                hg[bi] = hg[hn];
                hj[bi] = hj[hn];
                s_mask[wib][nc++] = msk;
                const int it = gs[g] + j;
                if (j + 1 < gc[g]) {  // next option of group g
                    hc[hn] = c - s_dv[wib][it] + s_dv[wib][it + 1];
                    hm[hn] = (msk & ~(1u << it)) | (1u << (it + 1));
                    hg[hn] = (uint8_t)g;
                    hj[hn] = (uint8_t)(j + 1);
                    hn++;
                }
                if (g + 1 < G) {
                    const int nx = gs[g + 1];
                    hc[hn] = c + s_dv[wib][nx];  // keep g, add group g+1
                    hm[hn] = msk | (1u << nx);
                    hg[hn] = (uint8_t)(g + 1);
                    hj[hn] = 0;
                    hn++;
                    if (j == 0) {  // swap g for g+1
                        hc[hn] = c - s_dv[wib][it] + s_dv[wib][nx];
                        hm[hn] = (msk & ~(1u << it)) | (1u << nx);
                        hg[hn] = (uint8_t)(g + 1);
                        hj[hn] = 0;
                        hn++;
                    }
                }
            }
            s_nc[wib] = nc;
        }
        __syncwarp();
        const int nc = s_nc[wib];  // m (the merged changes) is the same in every lane
        const int rows = nrows[d];
        const int64_t rbase = 2 * n0;
        for (int r = lane; r < rows; r += 32) {
            const int node = (int)plan[rbase + r].w;
            const int b = best_level[n0 + node];
            uint8_t *dst = m_alloc + (rbase + r) * stride;
            dst[0] = 0;
            for (int j = 0; j < k; j++) {
                const uint32_t msk = s_mask[wib][j < nc ? j : 0];
                int lv = b;
                for (int i = 0; i < m; i++)
                    if ((msk >> i & 1) && s_dn[wib][i] == node) lv = s_dl[wib][i];
                dst[1 + j] = levels[lv];
            }
        }
        __syncwarp();
    }
}

cudaError_t gnn_topk(int32_t n_dags, const int64_t *node_off, const float *logits, int n_levels,
                     const uint8_t *levels, int k, const uint4 *plan, const int32_t *nrows, uint8_t *best_level,
                     uint8_t *m_alloc, int64_t stride, int n_sm, cudaStream_t st) {
    if (n_dags == 0) return cudaSuccess;
    if (k < 1 || k > kTopkMax) return cudaErrorInvalidValue;
    int grid = (n_dags + 3) / 4;
    if (grid > 16 * n_sm) grid = 16 * n_sm;
    k_gnn_topk<<<grid, 128, 0, st>>>(n_dags, node_off, logits, n_levels, levels, k, plan, nrows, best_level, m_alloc,
                                     stride);
    return cudaGetLastError();
}

// the winning candidate's allocation, row by row (one warp per DAG)
__global__ void k_pick_column(int32_t n_dags, const int64_t *node_off, const int32_t *nrows, const int32_t *best,
                              const uint8_t *m_alloc, int64_t stride, uint8_t *out) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int d = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; d < n_dags; d += warps) {
        const int c = best[d];
        const int64_t rbase = 2 * node_off[d];
        for (int r = lane; r < nrows[d]; r += 32) out[rbase + r] = c >= 0 ? m_alloc[(rbase + r) * stride + c] : 0;
    }
}

cudaError_t gnn_pick_column(int32_t n_dags, const int64_t *node_off, const int32_t *nrows, const int32_t *best,
                            const uint8_t *m_alloc, int64_t stride, uint8_t *out, int n_sm, cudaStream_t st) {
    if (n_dags == 0) return cudaSuccess;
    int grid = (n_dags + 7) / 8;
    if (grid > 16 * n_sm) grid = 16 * n_sm;
    k_pick_column<<<grid, 256, 0, st>>>(n_dags, node_off, nrows, best, m_alloc, stride, out);
    return cudaGetLastError();
}

}  // namespace dagrt
