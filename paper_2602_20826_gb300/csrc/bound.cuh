// bound.cuh -- host-visible interface of the candidate-bound kernels (bound.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "dagrt.h"

namespace dagrt {

constexpr int kMaxVariantsPerCall = 16;

// Bound of candidate allocations on fixed plans (Lemma 1 / Theorem 1 with the
// sequential fallback for over-subscribed groups), argmin per DAG.
struct BoundArgs {
    int32_t n_dags;
    const int64_t *node_off;
    int32_t M;
    int32_t n_variants;
    int32_t n_alloc;
    const uint4 *plan[kMaxVariantsPerCall];     // plan rows {load, scheduled C, m|k<<16|last<<24, 0}
    const int32_t *nrows[kMaxVariantsPerCall];
    const int32_t *pflag[kMaxVariantsPerCall];  // bit 0: 32-bit arithmetic is exact
    const int32_t *status[kMaxVariantsPerCall];
    const uint8_t *m_alloc;                     // [(2*node_off[d] + row) * stride + cand]
    int64_t stride;
    int64_t *out;                               // [n_dags * n_cand]
    int64_t *best_bound;                        // [n_dags] or NULL
    int32_t *best_cand;                         // [n_dags] or NULL
    int32_t *err;                               // device word: set to DAGRT_E_TIMEOUT on a stalled copy
    // generated candidates (dagrt_search): m of row r of candidate c = v*n_alloc + a is
    // levels[gen_level(seed, d, c, r)] for a > 0 and the scheduled m for a == 0
    int32_t gen;
    int32_t gen_mode;                           // DAGRT_SEARCH_RANDOM / _EXHAUSTIVE / _PERTURB
    uint64_t seed;
    int32_t n_levels;
    uint8_t levels[16];
    uint8_t *best_m;                            // [2*total_nodes] winning allocation or NULL
};

// SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014) on a counter
__host__ __device__ inline uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
// level index of plan row r of candidate c of DAG d: counter d<<40 | c<<20 | r (+ seed),
// high 32 bits of the mixed value scaled to [0, n_levels)
__host__ __device__ inline int gen_level(uint64_t seed, int64_t d, int64_t c, int64_t r, int n_levels) {
    const uint64_t x = seed + (((uint64_t)d << 40) | ((uint64_t)c << 20) | (uint64_t)r);
    return (int)(((splitmix64(x) >> 32) * (uint64_t)n_levels) >> 32);
}

// Digit of node u in allocation a written in base B (exhaustive search): (a / B^u) % B.
__host__ __device__ inline uint32_t exh_digit(uint32_t a, uint32_t u, uint32_t B) {
    for (; u > 0 && a; u--) a /= B;
    return a % B;
}
// SMs of a plan row scheduled on m0 SMs after perturbation `code` (perturbation search):
// 0 keep, 1 halve, 2 one fewer, 3 one more, 4 double; at least 1, at most 255.
__host__ __device__ inline uint32_t perturb_m(uint32_t m0, uint32_t code) {
    uint32_t m = code == 1 ? m0 / 2 : code == 2 ? m0 - 1 : code == 3 ? m0 + 1 : code == 4 ? 2 * m0 : m0;
    return m < 1 ? 1u : (m > 255 ? 255u : m);
}

// ---------------------------------------------------------------- balanced work items
// For materialised candidates (n_alloc a multiple of 64), the bound is evaluated per work
// item = (variant, DAG, chunk of whole groups of at most ~kChunkRows plan rows, block of 64
// candidates): the bound is a sum over groups (Theorem 1), so chunks evaluate independently
// and their partial sums add up. Chunks are a property of the plan and are built once per
// plan.
constexpr int kChunkRows = 64;     // default row limit of a work item (two staging phases)
constexpr int kMinChunkRows = 8;
// upper bound on the chunks of one plan (two neighbouring chunks hold more than chunk_rows
// rows together)
inline int64_t chunk_items_bound(int64_t total_nodes, int32_t n_dags, int chunk_rows) {
    return 2 * (2 * total_nodes / chunk_rows + 1) + n_dags + 1;
}
struct ChunkIndex {  // device arrays of one plan
    int32_t *chunk;   // [2*total_nodes]: chunk k of DAG d starts at row chunk[2*node_off[d] + k]
    int32_t *nchunk;  // [n_dags]: 0 where the DAG's schedule failed
    int32_t *cpre;    // [n_dags + 1]: exclusive prefix sum of nchunk
    int4 *item;       // [cpre[n_dags]]: {d, first global plan row, end global plan row, flags}, DAG-major;
                      // flags bit 0: the DAG's sums fit 32-bit arithmetic
};

cudaError_t bound_build_chunks(int32_t n_dags, const int64_t *node_off, const uint4 *plan, const int32_t *nrows,
                               const int32_t *status, const int32_t *pflag, const ChunkIndex &ci, int chunk_rows,
                               int n_sm, cudaStream_t st);

struct ChunkArgs {
    const int32_t *chunk[kMaxVariantsPerCall], *nchunk[kMaxVariantsPerCall], *cpre[kMaxVariantsPerCall];
    const int4 *item[kMaxVariantsPerCall];
    uint32_t *counter;            // work-item counter
    unsigned long long *acc;      // [n_dags * n_cand] bound accumulators; zero between calls
    int32_t warps;                // warps per CTA of the work-item kernel
    int64_t alloc_rows;           // rows of the candidate-byte array (2 * total nodes)
};

// scratch bytes the balanced path needs for a call (counter, accumulators); all of it must
// be zero before the first call, and every call leaves it zero
size_t bound_chunk_scratch(int32_t n_dags, int64_t total_nodes, int32_t n_variants, int32_t n_alloc, int chunk_rows);
// the call can take the balanced path (materialised candidates, n_alloc % 64 == 0, and few
// enough work items for 32-bit item ids)
bool bound_chunk_eligible(const BoundArgs &a, int64_t total_nodes, int chunk_rows);

// One CTA waits on an mbarrier that nothing arrives on, with the kernels' bounded wait,
// giving up after `limit` polls: *word = DAGRT_E_TIMEOUT (the failure path of every wait).
cudaError_t bound_selftest_wait(uint32_t limit, int32_t *word, cudaStream_t st);

// Enqueue the bound kernels; *launches receives the number of kernels enqueued. With ch
// (an eligible call), the balanced path: work items adding their partial bounds into
// per-candidate accumulators, then k_bound_finish (bounds, argmin); else the tile kernels.
cudaError_t bound_launch(const BoundArgs &a, const ChunkArgs *ch, int n_sm, cudaStream_t st, int *launches);

}  // namespace dagrt
