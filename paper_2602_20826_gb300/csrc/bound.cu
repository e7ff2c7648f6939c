// bound.cu -- bound of candidate allocations on fixed schedule structures, and the argmin
// over candidates per DAG.
//
// A plan is the schedule of one structure variant: rows ordered by the group they run in,
// each with its load, parallel fraction and scheduled SMs. For candidate allocation m^c
// the bound is a max-plus sweep along the group chain (Theorem 1): F_j = F_{j-1} + R_j,
// with R_j = max C_i over the group if its SMs fit in M (Lemma 1), else sum C_i.
#include "bound.cuh"
#include "dagrt_internal.cuh"

namespace dagrt {

__global__ void k_bound_simple(BoundArgs a) {
    const int64_t n_cand = (int64_t)a.n_variants * a.n_alloc;
    const int64_t total = (int64_t)a.n_dags * n_cand;
    const uint32_t M = (uint32_t)a.M;
    for (int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gid < total;
         gid += (int64_t)gridDim.x * blockDim.x) {
        const int d = (int)(gid / n_cand);
        const int c = (int)(gid - (int64_t)d * n_cand);
        const int vi = c / a.n_alloc;
        if (a.status[vi][d] != DAGRT_OK) {
            a.out[gid] = -1;
            continue;
        }
        const int rows = a.nrows[vi][d];
        const int64_t rbase = 2 * a.node_off[d];
        const uint2 *lc = a.lc[vi] + rbase;
        const uint32_t *mkf = a.mkf[vi] + rbase;
        const uint8_t *al = a.m_alloc + rbase * a.stride + c;
        uint64_t bound = 0, gmax = 0, gsum = 0;
        uint32_t gm = 0;
        for (int r = 0; r < rows; r++) {
            const uint2 x = lc[r];
            const uint32_t f = mkf[r];
            const uint32_t m = al[(int64_t)r * a.stride];
            const uint32_t mm = m ? m : (f & 0xffffu);
            const uint64_t C = m ? exec_time(x.x, (f >> 16) & 0xffu, mm, M) : (uint64_t)x.y;
            gmax = C > gmax ? C : gmax;
            gsum += C;
            gm += mm;
            if (f >> 24) {
                bound += gm <= M ? gmax : gsum;
                gmax = gsum = 0;
                gm = 0;
            }
        }
        a.out[gid] = (int64_t)bound;
    }
}

// argmin over the candidates of each DAG: smallest bound, then smallest candidate id
__global__ void k_argmin(BoundArgs a) {
    const int64_t n_cand = (int64_t)a.n_variants * a.n_alloc;
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int d = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; d < a.n_dags; d += warps) {
        const int64_t *row = a.out + (int64_t)d * n_cand;
        int64_t bb = INT64_MAX;
        int32_t bc = -1;
        for (int64_t c = lane; c < n_cand; c += 32) {
            const int64_t v = row[c];
            if (v >= 0 && v < bb) { bb = v; bc = (int32_t)c; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const int64_t ob = __shfl_xor_sync(FULL, bb, o);
            const int32_t oc = __shfl_xor_sync(FULL, bc, o);
            if (ob < bb || (ob == bb && oc >= 0 && (bc < 0 || oc < bc))) { bb = ob; bc = oc; }
        }
        if (lane == 0) {
            if (a.best_bound) a.best_bound[d] = bc < 0 ? -1 : bb;
            if (a.best_cand) a.best_cand[d] = bc;
        }
    }
}

cudaError_t bound_launch(const BoundArgs &a, int n_sm, cudaStream_t st) {
    const int64_t total = (int64_t)a.n_dags * a.n_variants * a.n_alloc;
    if (total == 0) return cudaSuccess;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 64ll * n_sm) blocks = 64ll * n_sm;
    k_bound_simple<<<(int)blocks, 256, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (a.best_bound || a.best_cand) {
        int64_t wb = ((int64_t)a.n_dags * 32 + 255) / 256;
        if (wb > 16ll * n_sm) wb = 16ll * n_sm;
        k_argmin<<<(int)wb, 256, 0, st>>>(a);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace dagrt
