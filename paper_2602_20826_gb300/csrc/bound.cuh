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
};

cudaError_t bound_launch(const BoundArgs &a, int n_sm, cudaStream_t st);

}  // namespace dagrt
