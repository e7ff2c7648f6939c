// gnn.cuh -- host-visible interface of the learned proposer's kernels (gnn.cu).
//
// A 3-layer message-passing network over the nodes of every DAG of a batch scores the SM
// levels of each kernel: h' = ReLU([h | mean_pred h | mean_succ h] W + b), hidden width
// 128, then a linear head to one logit per level. Activations and GEMM operands are bf16,
// accumulation fp32 (tcgen05 MMAs with TMEM accumulators); the parameters are kept in fp32
// and trained with Adam.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace dagrt {

constexpr int kFeat = 16;      // input features per node (padded)
constexpr int kHidden = 128;
constexpr int kMaxLevels = 16;

// fp32 parameter layout (offsets in floats)
struct ParamLayout {
    static constexpr int64_t W1 = 0;                               // [3*kFeat x H]
    static constexpr int64_t b1 = W1 + 3 * kFeat * kHidden;        // [H]
    static constexpr int64_t W2 = b1 + kHidden;                    // [3H x H]
    static constexpr int64_t b2 = W2 + 3 * kHidden * kHidden;
    static constexpr int64_t W3 = b2 + kHidden;
    static constexpr int64_t b3 = W3 + 3 * kHidden * kHidden;
    static constexpr int64_t Wh = b3 + kHidden;                    // [H x kMaxLevels]
    static constexpr int64_t bh = Wh + kHidden * kMaxLevels;       // [kMaxLevels]
    static constexpr int64_t total = bh + kMaxLevels;
};

// the batch's graph for message passing (global node ids)
struct GnnGraph {
    int64_t n_nodes, n_edges;
    const int32_t *pred_off, *pred_idx;  // [N+1], [E]
    const int32_t *succ_off, *succ_idx;
};

struct GnnParams {
    const float *p;              // fp32 master parameters (ParamLayout)
    const uint16_t *wt[3];       // bf16 W^T per layer: [H x K]
    const uint16_t *wb[3];       // bf16 W per layer: [K x H]
    int32_t n_levels;
};

// graph build: per-DAG CSRs -> global pred/succ CSRs (deterministic order); DAGs whose
// paper schedule failed (status != DAGRT_OK) get no edges
cudaError_t gnn_build_graph(int32_t n_dags, const int64_t *node_off, const int64_t *edge_off, const int32_t *row_ptr,
                            const int32_t *col, const int32_t *status, int32_t *pred_off, int32_t *pred_idx,
                            int32_t *succ_off, int32_t *succ_idx, int32_t *cursor, int n_sm, cudaStream_t st);
// features from the batch and the paper schedule's outputs (zero for failed DAGs)
cudaError_t gnn_features(int32_t n_dags, const int64_t *node_off, const int64_t *wcet, const uint8_t *k64,
                         const int32_t *level, const int64_t *wanc, const int32_t *m, const int32_t *status,
                         GnnGraph g, uint16_t *x, int n_sm, cudaStream_t st);
// one layer: h_out = ReLU(agg(h_in) W + b); kin = 16 or 128
cudaError_t gnn_layer_fwd(int kin, GnnGraph g, const uint16_t *h_in, const uint16_t *wt, const float *bias,
                          uint16_t *h_out, int32_t *err, int n_sm, cudaStream_t st);
// head: logits (and, with labels, loss pieces and dlogits)
cudaError_t gnn_head(GnnGraph g, const uint16_t *h3, const float *wh, const float *bh, int n_levels,
                     const int8_t *labels, float scale, float *logits, float *dlogits, float *dh3,
                     float *loss_part, int n_sm, cudaStream_t st);
cudaError_t gnn_head_grad(GnnGraph g, const uint16_t *h3, const float *dlogits, int n_levels, float *part,
                          int n_parts, cudaStream_t st);
// backward of one layer
// weight and bias gradients of layer `layer` (0..2) into the per-CTA partial rows
cudaError_t gnn_layer_bwd_dw(int kin, int layer, GnnGraph g, const uint16_t *h_in, const uint16_t *h_out,
                             const float *dh_out, float *part, int n_parts, int32_t *err, cudaStream_t st);
cudaError_t gnn_layer_bwd_da(int kin, GnnGraph g, const uint16_t *h_out, const float *dh_out, const uint16_t *wb,
                             float *da, int32_t *err, int n_sm, cudaStream_t st);
cudaError_t gnn_agg_bwd(int kin, GnnGraph g, const float *da, float *dh_in, int n_sm, cudaStream_t st);
// reduce per-CTA partials (fixed order) and take one Adam step; refresh bf16 copies
cudaError_t gnn_adam(float *p, float *m, float *v, const float *part, int n_parts, int64_t n, float lr, float b1,
                     float b2, float eps, int step, cudaStream_t st);
cudaError_t gnn_refresh(const float *p, uint16_t *const *wt, uint16_t *const *wb, cudaStream_t st);
// top-k decode of the per-node level distributions into candidate allocations
cudaError_t gnn_topk(int32_t n_dags, const int64_t *node_off, const float *logits, int n_levels,
                     const uint8_t *levels, int k, const uint4 *plan, const int32_t *nrows, uint8_t *best_level,
                     uint8_t *m_alloc, int64_t stride, int n_sm, cudaStream_t st);
cudaError_t gnn_pick_column(int32_t n_dags, const int64_t *node_off, const int32_t *nrows, const int32_t *best,
                            const uint8_t *m_alloc, int64_t stride, uint8_t *out, int n_sm, cudaStream_t st);

}  // namespace dagrt
