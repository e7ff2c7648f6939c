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

cudaError_t bound_launch(const BoundArgs &a, int n_sm, cudaStream_t st);

}  // namespace dagrt
