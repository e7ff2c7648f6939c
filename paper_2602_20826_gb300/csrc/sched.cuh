// sched.cuh -- host-visible interface of the scheduling kernels (sched.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "dagrt.h"

namespace dagrt {

constexpr int kWarpsPerCta = 4;    // independent warp teams per CTA (small DAGs; 4 measured 3% faster than 2 on the 10,000-DAG batch)
constexpr int kCtaThreads = 256;   // threads of a CTA team with a shared-memory workspace
constexpr int kCtaThreadsGlobal = 384;  // threads of a CTA team with a global workspace (DAGs too large for shared
                                       // memory; 384 measured 13% faster than 256 on 200 DAGs of 2,000-20,000 nodes)
constexpr int kEdgesPerNode = 12;  // warp teams take DAGs of at most this many edges per node of warp_max_v
constexpr int kWarpClassStep = 16; // node capacities of the warp-team size classes: 16, 32, ..., 256

// Arguments of one scheduling launch. Every pointer is a device pointer.
struct SchedArgs {
    const int64_t *node_off;
    const int64_t *edge_off;
    const int32_t *row_ptr;
    const int32_t *col;
    const int64_t *wcet;
    const uint8_t *k64;
    int32_t M;
    int32_t variant;
    // DAGs of this size class (NULL: DAGs 0 .. n_list-1 in order) and the work-stealing
    // counter over them
    const int32_t *list;
    int32_t n_list;
    int32_t *counter;
    // always written: per-DAG status and bound
    int32_t *status;
    int64_t *bound;
    // status of a DAG larger than the workspace (or with negative offsets)
    int32_t oversize_status;
    // lengths of the node arrays (wcet, k64; row_ptr holds tot_nodes + n_dags entries) and
    // of col: a DAG whose offsets reach outside them gets oversize_status; -1 = not checked
    // (the offsets were checked on the host)
    int64_t tot_nodes, tot_edges;
    // plan of the schedule (NULL: not kept): row count, flags, rows at 2*node_off[d]
    int32_t *nrows;
    int32_t *pflag;      // per DAG: bit 0 = candidate bounds of this DAG fit 32-bit sums
    uint4 *plan;         // rows {load, scheduled C, m | k << 16 | last-row-of-group << 24, owner node}
    // optional caller outputs (device pointers, NULL = skip)
    dagrt_schedule_out o;
    // global workspace of the CTA-team kernel
    unsigned char *gws;
    int64_t gws_stride;
    int32_t vcap, ecap;
};

int64_t sched_ws_bytes(int vc, int ec);
// warp teams: the workspace (a.vcap, a.ecap) of kWarpsPerCta teams must fit sched_smem_limit()
cudaError_t sched_launch_warp(const SchedArgs &a, int n_sm, cudaStream_t st);
int sched_cta_grid(int n_sm);
cudaError_t sched_launch_cta(const SchedArgs &a, int grid, cudaStream_t st);
// CTA teams with the workspace (a.vcap, a.ecap) in shared memory: sched_ws_bytes of the
// class must not exceed sched_smem_limit()
int64_t sched_smem_limit();
cudaError_t sched_launch_cta_smem(const SchedArgs &a, int n_sm, cudaStream_t st);

// Schedulability of implicit-deadline tasks: ok[d] = status[d] == OK && bound[d] <=
// deadline[d]; *n_ok (zeroed by the caller) += the number of such DAGs.
cudaError_t sched_schedulable(int32_t n_dags, const int32_t *status, const int64_t *bound, const int64_t *deadline,
                              int32_t *ok, unsigned long long *n_ok, int n_sm, cudaStream_t st);

}  // namespace dagrt
