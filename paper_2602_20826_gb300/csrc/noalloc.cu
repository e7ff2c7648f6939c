// noalloc.cu -- dagrt_schedule_noalloc: the scheduler for callers that cannot allocate.
//
// Some callers must not allocate device memory at run time: real-time executives that
// reserve every buffer before the task set starts (an allocation can block for an
// unbounded time), code running under a memory budget enforced by another owner, and
// plug-ins whose host framework forbids cudaMalloc. For them this file keeps the
// scheduler's scratch memory -- the per-team workspace of the CTA-team kernel and its
// work-stealing counter -- in one file-scope __device__ array of fixed size, so the entry
// point below allocates nothing: the caller passes the batch and the output arrays, all in
// device memory.
//
// Limits: DAGs of at most kNoallocMaxV nodes and kNoallocMaxE edges (larger ones get
// status DAGRT_E_INVAL); kNoallocTeams CTA teams share the array. Every GPU that loads
// the library holds the array until the process exits.
//
// The offsets are device data the host never reads here, so the kernel checks every DAG's
// node and edge range against the array lengths the caller passes (DAGRT_E_INVAL for a DAG
// that reaches outside them) before it touches the DAG's arrays.
//
// Calls share the array: two calls whose kernels overlap on the GPU (different streams, or
// different host threads on one device) race on it and give wrong results. Issue them on
// one stream, or order them.
#include <cstring>

#include "dagrt.h"
#include "dagrt_internal.cuh"
#include "sched.cuh"

namespace dagrt {
namespace {

constexpr int kNoallocMaxV = 512;
constexpr int kNoallocMaxE = 8192;
constexpr int kNoallocTeams = 32;
constexpr int64_t kCounterBytes = 256;
constexpr int64_t kScratchBytes = 4ll << 20;  // 4 MiB

}  // namespace

// the scratch: work-stealing counter, then kNoallocTeams workspaces
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of the array on the current device. In host code `g_noalloc_scratch` is
// only a host-side stand-in, never a device address, so it is looked up here, on every call
// (a device reset or a new primary context between calls then cannot leave a stale address
// behind); the first lookup on a device loads the library's device code.
static int noalloc_scratch(unsigned char **out) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return DAGRT_E_DEVICE;
    *out = (unsigned char *)p;
    return DAGRT_OK;
}

}  // namespace dagrt

using namespace dagrt;

extern "C" int dagrt_schedule_noalloc(int32_t n_dags, const int64_t *node_off, const int64_t *edge_off,
                                      const int32_t *row_ptr, const int32_t *col, const int64_t *wcet,
                                      const uint8_t *k64, int64_t total_nodes, int64_t total_edges, int32_t M,
                                      int32_t variant, int64_t *bound, int32_t *status, void *cuda_stream) {
    if (n_dags < 0 || total_nodes < 0 || total_edges < 0 || M < 1 || M > DAGRT_MAX_M || variant < 0 ||
        variant >= DAGRT_N_VARIANTS)
        return DAGRT_E_INVAL;
    if (n_dags == 0) return DAGRT_OK;
    if (!node_off || !edge_off || !row_ptr || !wcet || !k64 || !bound || !status || (total_edges > 0 && !col))
        return DAGRT_E_INVAL;
    const int64_t ws = align_up(sched_ws_bytes(kNoallocMaxV, kNoallocMaxE), 256);
    if (kCounterBytes + ws * kNoallocTeams > kScratchBytes) return DAGRT_E_INTERNAL;
    unsigned char *scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc != DAGRT_OK) return rc;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // the counter must start at zero on every call
    if (cudaMemsetAsync(scratch, 0, sizeof(int32_t), st) != cudaSuccess) return DAGRT_E_DEVICE;
    SchedArgs a;
    memset(&a, 0, sizeof a);
    a.node_off = node_off;
    a.edge_off = edge_off;
    a.row_ptr = row_ptr;
    a.col = col;
    a.wcet = wcet;
    a.k64 = k64;
    a.M = M;
    a.variant = variant;
    a.list = nullptr;  // DAGs in batch order
    a.n_list = n_dags;
    a.counter = (int32_t *)scratch;
    a.status = status;
    a.bound = bound;
    a.oversize_status = DAGRT_E_INVAL;
    a.tot_nodes = total_nodes;
    a.tot_edges = total_edges;
    a.gws = scratch + kCounterBytes;
    a.gws_stride = ws;
    a.vcap = kNoallocMaxV;
    a.ecap = kNoallocMaxE;
    const int grid = n_dags < kNoallocTeams ? n_dags : kNoallocTeams;
    if (sched_launch_cta(a, grid, st) != cudaSuccess) return DAGRT_E_DEVICE;
    return DAGRT_OK;
}
