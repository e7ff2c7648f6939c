// api.cu -- the extern "C" entry points of libdagrt (declared in include/dagrt.h).
//
// Host code only: argument checks, device buffers owned by contexts and batches, size
// classes of DAGs for the scheduling kernels, and host<->device marshalling of outputs.
#include <algorithm>
#include <cstdarg>
#include <map>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "dagrt.h"
#include "bound.cuh"
#include "gnn.cuh"
#include "sched.cuh"

using namespace dagrt;

// NVTX range around a library call (visible in Nsight tools; free when none is attached)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

// Device buffers are recycled through a per-context pool (exact-size free lists), so a
// batch that is loaded and freed every step allocates nothing after the first step.
struct DevicePool {
    std::multimap<size_t, void *> free_list;
    std::vector<void *> all;
    cudaError_t get(void **p, size_t bytes) {
        bytes = (bytes + 255) / 256 * 256;
        auto it = free_list.find(bytes);
        if (it != free_list.end()) {
            *p = it->second;
            free_list.erase(it);
            return cudaSuccess;
        }
        cudaError_t e = cudaMalloc(p, bytes);
        if (e == cudaSuccess) all.push_back(*p);
        return e;
    }
    void put(void *p, size_t bytes) { free_list.emplace((bytes + 255) / 256 * 256, p); }
    void release_all() {
        for (void *p : all) cudaFree(p);
        all.clear();
        free_list.clear();
    }
};

struct dagrt_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int n_sm = 0;
    std::string err;
    int n_batches = 0;
    // batches, models and graphs alive: dagrt_destroy waits for the last of them
    int live = 0;
    bool destroy_pending = false;
    int64_t launches = 0;
    DevicePool pool;
    // side streams: the scheduler's size-class kernels run concurrently, forked from and
    // joined back into `stream` with events
    static constexpr int kSide = 18;  // one per scheduler size class
    cudaStream_t side[kSide] = {};
    cudaEvent_t fork = nullptr, join[kSide] = {};
    bool side_ready = false;
    // stream capture into a CUDA graph (dagrt_graph_begin .. dagrt_graph_end)
    bool capturing = false;
    int64_t capture_launch0 = 0;
    cudaStream_t cap_stream = nullptr;  // captures run here; `stream` is restored at the end
    cudaStream_t saved_stream = nullptr;
    // pinned host staging of dagrt_load_csr (offsets down, class lists up); pin_ev marks the
    // end of the last asynchronous copy out of it, waited for before the next reuse
    void *pin = nullptr;
    size_t pin_cap = 0;
    cudaEvent_t pin_ev = nullptr;
    bool pin_pending = false;
};

// The context's pinned staging buffer, at least `bytes` long, once its last asynchronous
// copy has completed.
static cudaError_t pinned(dagrt_ctx *c, size_t bytes, void **p) {
    cudaError_t e = cudaSuccess;
    if (c->pin_pending) {
        if ((e = cudaEventSynchronize(c->pin_ev)) != cudaSuccess) return e;
        c->pin_pending = false;
    }
    if (!c->pin_ev && (e = cudaEventCreateWithFlags(&c->pin_ev, cudaEventDisableTiming)) != cudaSuccess) return e;
    if (bytes > c->pin_cap) {
        if (c->pin) cudaFreeHost(c->pin);
        c->pin = nullptr;
        c->pin_cap = 0;
        const size_t cap = std::max<size_t>(bytes, 1 << 16);
        if ((e = cudaHostAlloc(&c->pin, cap, cudaHostAllocDefault)) != cudaSuccess) return e;
        c->pin_cap = cap;
    }
    *p = c->pin;
    return cudaSuccess;
}

// One side stream per size class, larger classes at higher priority: pending CTAs of the
// classes with the longest DAGs are dispatched first as SMs free up (measured 3% faster on
// the 10,000-DAG batch and 1.5% on config 3's schedule than streams of equal priority).
static cudaError_t ensure_side_streams(dagrt_ctx *c) {
    if (c->side_ready) return cudaSuccess;
    int lo = 0, hi = 0;  // least and greatest priority (greatest is the most negative)
    if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess) lo = hi = 0;
    cudaError_t e = cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming);
    for (int i = 0; i < dagrt_ctx::kSide && e == cudaSuccess; i++) {
        const int prio = lo - (i * (lo - hi + 1)) / dagrt_ctx::kSide;
        e = cudaStreamCreateWithPriority(&c->side[i], cudaStreamNonBlocking, prio);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->join[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) c->side_ready = true;
    return e;
}

namespace {

// warp-team size classes by node count: DAGs of 1-16, 17-32, ..., 241-256 nodes, each class
// with the edge capacity of its densest DAG (finer classes than powers of two keep the
// workspaces close to the DAGs' sizes, so more teams fit an SM)
constexpr int kNumWarpClasses = 256 / kWarpClassStep;
// classes after the warp classes: CTA teams with a shared-memory workspace, then CTA teams
// with global workspaces
constexpr int kClsCtaSmem = kNumWarpClasses, kClsCtaGlobal = kNumWarpClasses + 1, kNumClasses = kNumWarpClasses + 2;
static_assert(dagrt_ctx::kSide >= kNumClasses, "a side stream per size class");

struct Plan {
    bool valid = false;
    uint4 *rows = nullptr;
    int32_t *nrows = nullptr;
    int32_t *pflag = nullptr;
    int32_t *status = nullptr;
    int64_t *bound = nullptr;
    bool chunked = false;  // ci holds this plan's chunks, cut at chunk_rows
    int chunk_rows = 0;
    ChunkIndex ci = {};
};

}  // namespace

struct dagrt_batch {
    dagrt_ctx *ctx = nullptr;
    int32_t n_dags = 0;
    int32_t M = 0;
    int64_t total_nodes = 0, total_edges = 0;
    const int64_t *node_off = nullptr, *edge_off = nullptr, *wcet = nullptr;
    const int32_t *row_ptr = nullptr, *col = nullptr;
    const uint8_t *k64 = nullptr;
    std::vector<std::pair<void *, size_t>> owned;  // pooled device buffers of the batch
    std::vector<int64_t> h_node_off, h_edge_off;
    dagrt_tuning tune = {256, kChunkRows, 4, 2};
    // size classes: warp classes then the CTA class, lists concatenated
    int32_t *lists = nullptr;
    int32_t *counters = nullptr;  // [kNumClasses] work-stealing counters of the size classes
    int class_off[kNumClasses + 1] = {0};
    int max_v = 0, big_vcap = 0, big_ecap = 0, big_grid = 0;
    int smem_vcap = 0, smem_ecap = 0;  // capacity of the shared-memory CTA class
    int wcap_v[kNumWarpClasses] = {0}, wcap_e[kNumWarpClasses] = {0};  // capacities of the warp classes
    unsigned char *gws = nullptr;  // pooled, gws_cap bytes
    int64_t gws_stride = 0;
    size_t gws_cap = 0;
    Plan plan[DAGRT_N_VARIANTS];
    int32_t *err = nullptr;  // device error word (bounded waits that gave up)
    // scratch for candidate evaluation
    void *tmp = nullptr;
    size_t tmp_cap = 0;
    void *bscr = nullptr;  // work-item scratch of the bound kernels
    size_t bscr_cap = 0;
    bool bscr_dirty = false;  // a call failed part way: clear the counters and accumulators first
    // learned proposer: message-passing graph, features, activations (allocated on first use)
    struct Gnn {
        bool graph = false, train = false;
        int32_t *pred_off, *pred_idx, *succ_off, *succ_idx, *cursor, *level, *m;
        int64_t *wanc;
        uint16_t *x, *h[3];
        float *logits, *dlogits, *dh[3], *da, *loss_part;
        int8_t *labels;
        uint8_t *best_level, *cand;
        int32_t *cbest;
        int64_t *bbest;
    } gnn;
};

static int fail(dagrt_ctx *ctx, int code, const char *fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return code;
}

static int cuda_fail(dagrt_ctx *ctx, cudaError_t e, const char *what) {
    return fail(ctx, e == cudaErrorMemoryAllocation ? DAGRT_E_OOM : DAGRT_E_DEVICE, "%s: %s", what,
                cudaGetErrorString(e));
}

// calls that need the host (copies to or from host memory, synchronisation) cannot be
// recorded into a CUDA graph
static int refuse_in_capture(dagrt_ctx *ctx, bool needs_host, const char *fn) {
    if (ctx->capturing && needs_host)
        return fail(ctx, DAGRT_E_INVAL, "%s: needs the host; not allowed while capturing a graph (use DAGRT_PTR_DEVICE)", fn);
    return DAGRT_OK;
}

#define CK(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
    } while (0)

template <class T>
static cudaError_t batch_alloc(dagrt_batch *b, T **p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 1;
    void *q = nullptr;
    cudaError_t e = b->ctx->pool.get(&q, n * sizeof(T));
    if (e == cudaSuccess) {
        *p = (T *)q;
        b->owned.emplace_back(q, n * sizeof(T));
    }
    return e;
}

static void batch_release(dagrt_batch *b) {
    for (auto &pb : b->owned) b->ctx->pool.put(pb.first, pb.second);
    b->owned.clear();
    if (b->tmp) b->ctx->pool.put(b->tmp, b->tmp_cap);
    b->tmp = nullptr;
    b->tmp_cap = 0;
    if (b->bscr) b->ctx->pool.put(b->bscr, b->bscr_cap);
    b->bscr = nullptr;
    b->bscr_cap = 0;
    if (b->gws) b->ctx->pool.put(b->gws, b->gws_cap);
    b->gws = nullptr;
    b->gws_cap = 0;
}

extern "C" {

int dagrt_create(dagrt_ctx **out, int device, void *cuda_stream) {
    if (!out) return DAGRT_E_INVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return DAGRT_E_DEVICE;
    if (cudaSetDevice(device) != cudaSuccess) return DAGRT_E_DEVICE;
    dagrt_ctx *c = new dagrt_ctx();
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    if (cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        delete c;
        return DAGRT_E_DEVICE;
    }
    *out = c;
    return DAGRT_OK;
}

int dagrt_set_stream(dagrt_ctx *ctx, void *cuda_stream) {
    if (!ctx) return DAGRT_E_INVAL;
    if (ctx->capturing) return fail(ctx, DAGRT_E_INVAL, "dagrt_set_stream: not allowed while capturing a graph");
    ctx->stream = (cudaStream_t)cuda_stream;
    return DAGRT_OK;
}

int dagrt_sync(dagrt_ctx *ctx) {
    if (!ctx) return DAGRT_E_INVAL;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    CK(cudaStreamSynchronize(ctx->stream), "stream synchronize");
    return DAGRT_OK;
}

static void ctx_release(dagrt_ctx *ctx) {
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    ctx->pool.release_all();
    if (ctx->side_ready) {
        for (int i = 0; i < dagrt_ctx::kSide; i++) {
            cudaStreamDestroy(ctx->side[i]);
            cudaEventDestroy(ctx->join[i]);
        }
        cudaEventDestroy(ctx->fork);
    }
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->pin_ev) cudaEventDestroy(ctx->pin_ev);
    if (ctx->pin) cudaFreeHost(ctx->pin);
    delete ctx;
}

// an object of the context went away; the context follows if it was destroyed already
static void ctx_unref(dagrt_ctx *ctx) {
    if (--ctx->live == 0 && ctx->destroy_pending) ctx_release(ctx);
}

void dagrt_destroy(dagrt_ctx *ctx) {
    if (!ctx) return;
    if (ctx->live > 0) {  // batches, models or graphs still refer to it
        ctx->destroy_pending = true;
        return;
    }
    ctx_release(ctx);
}

const char *dagrt_last_error(const dagrt_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int64_t dagrt_launch_count(const dagrt_ctx *ctx) { return ctx ? ctx->launches : -1; }

int32_t dagrt_batch_n_dags(const dagrt_batch *b) { return b ? b->n_dags : -1; }
int64_t dagrt_batch_total_nodes(const dagrt_batch *b) { return b ? b->total_nodes : -1; }

void dagrt_batch_free(dagrt_batch *b) {
    if (!b) return;
    cudaSetDevice(b->ctx->device);
    cudaStreamSynchronize(b->ctx->stream);
    batch_release(b);
    dagrt_ctx *ctx = b->ctx;
    ctx->n_batches--;
    delete b;
    ctx_unref(ctx);
}

// Size classes for the scheduler: a DAG goes to the smallest warp class whose shared-memory
// workspace holds its V nodes and E edges, among the classes of at most tune.warp_max_v
// nodes; the rest go to CTA teams -- with a shared-memory workspace while the class's
// capacity (largest V and E so far, smallest DAGs first) still fits 1/tune.cta_smem of a
// CTA's shared memory (cta_smem = 0: never), else with global workspaces. Each class is ordered by
// descending node count (longest work first). Host work plus one list upload.
static int partition_classes(dagrt_batch *b) {
    dagrt_ctx *ctx = b->ctx;
    const int n_dags = b->n_dags, max_v = b->max_v;
    const std::vector<int64_t> &hn = b->h_node_off, &he = b->h_edge_off;
    const int wmax = b->tune.warp_max_v;  // warp teams: V <= wmax and E <= kEdgesPerNode * wmax
    int64_t wecap[kNumWarpClasses] = {0};
    int count[kNumClasses] = {0};
    // sequential passes over the offsets: warp-class DAGs are bucketed by V (their class is
    // a function of V), CTA-team DAGs listed apart and sorted by descending V
    std::vector<int32_t> cnt_v(max_v + 2, 0);
    std::vector<int32_t> big;  // CTA-team DAGs
    for (int d = 0; d < n_dags; d++) {
        const int v = (int)(hn[d + 1] - hn[d]);
        const int64_t ed = he[d + 1] - he[d];
        if (v <= wmax && ed <= (int64_t)kEdgesPerNode * wmax) {
            const int c = v > 0 ? (v - 1) / kWarpClassStep : 0;
            cnt_v[v]++;
            count[c]++;
            wecap[c] = std::max(wecap[c], ed);
        } else {
            big.push_back(d);
        }
    }
    std::stable_sort(big.begin(), big.end(),
                     [&](int x, int y) { return hn[x + 1] - hn[x] > hn[y + 1] - hn[y]; });  // descending V
    // cta_smem = k: a workspace takes at most 1/k of the shared memory, so k teams fit per SM
    const int64_t limit = b->tune.cta_smem > 0 ? sched_smem_limit() / b->tune.cta_smem : 0;
    int sv = 0, gv = 0;
    int64_t se = 0, ge = 0;
    std::vector<char> in_smem(big.size(), 0);
    for (int i = (int)big.size() - 1; i >= 0; i--) {  // smallest first
        const int d = big[i];
        const int v = (int)(hn[d + 1] - hn[d]);
        const int64_t ed = he[d + 1] - he[d];
        const int nv = std::max(sv, v);
        const int64_t ne = std::max(se, ed);
        if (ne < (1ll << 30) && sched_ws_bytes(nv, (int)ne) <= limit) {
            sv = nv;
            se = ne;
            in_smem[i] = 1;
        }
    }
    std::vector<int32_t> big_cls(big.size());
    for (size_t i = 0; i < big.size(); i++) {
        const int d = big[i];
        const int c = in_smem[i] ? kClsCtaSmem : kClsCtaGlobal;
        big_cls[i] = c;
        count[c]++;
        if (!in_smem[i]) {
            gv = std::max(gv, (int)(hn[d + 1] - hn[d]));
            ge = std::max(ge, he[d + 1] - he[d]);
        }
    }
    // the class lists, each in descending V (equal V: ascending DAG id), in pinned memory
    int off = 0, pos[kNumClasses];
    for (int c = 0; c < kNumClasses; c++) {
        b->class_off[c] = pos[c] = off;
        off += count[c];
    }
    b->class_off[kNumClasses] = off;
    std::vector<int32_t> start_v(max_v + 2, 0);  // next list slot of each node count
    for (int c = 0; c < kNumWarpClasses; c++) {
        int p = b->class_off[c];
        for (int v = std::min(max_v, (c + 1) * kWarpClassStep); v >= c * kWarpClassStep + (c == 0 ? 0 : 1); v--) {
            start_v[v] = p;
            p += cnt_v[v];
        }
    }
    int32_t *lists = nullptr;
    CK(pinned(ctx, 4 * (size_t)std::max(n_dags, 1), (void **)&lists), "pinned staging");
    for (int d = 0; d < n_dags; d++) {
        const int v = (int)(hn[d + 1] - hn[d]);
        if (v <= wmax && he[d + 1] - he[d] <= (int64_t)kEdgesPerNode * wmax) lists[start_v[v]++] = d;
    }
    for (size_t i = 0; i < big.size(); i++) lists[pos[big_cls[i]]++] = big[i];
    for (int c = 0; c < kNumWarpClasses; c++) {
        b->wcap_v[c] = (c + 1) * kWarpClassStep;
        b->wcap_e[c] = (int)std::max<int64_t>(wecap[c], 1);
    }
    b->smem_vcap = sv;
    b->smem_ecap = (int)se;
    b->big_vcap = gv;
    b->big_ecap = (int)ge;
    if (n_dags > 0) {
        CK(cudaMemcpyAsync(b->lists, lists, 4 * n_dags, cudaMemcpyHostToDevice, ctx->stream), "copy class lists");
        CK(cudaEventRecord(ctx->pin_ev, ctx->stream), "record staging event");
        ctx->pin_pending = true;
    }
    const int n_big = b->class_off[kClsCtaGlobal + 1] - b->class_off[kClsCtaGlobal];
    if (n_big > 0) {
        b->big_grid = std::min(sched_cta_grid(ctx->n_sm), n_big);
        b->gws_stride = sched_ws_bytes(b->big_vcap, b->big_ecap);
        const size_t need = (size_t)b->gws_stride * b->big_grid;
        if (need > b->gws_cap) {
            if (b->gws) ctx->pool.put(b->gws, b->gws_cap);
            b->gws = nullptr;
            b->gws_cap = 0;
            void *g = nullptr;
            CK(ctx->pool.get(&g, need), "allocate large-DAG workspace");
            b->gws = (unsigned char *)g;
            b->gws_cap = (need + 255) / 256 * 256;
        }
    }
    return DAGRT_OK;
}

int dagrt_load_csr(dagrt_ctx *ctx, int32_t n_dags, const int64_t *node_off, const int64_t *edge_off,
                   const int32_t *row_ptr, const int32_t *col, const int64_t *wcet, const uint8_t *k64,
                   int32_t M, uint32_t flags, dagrt_batch **out) {
    NvtxRange nvtx_range_("dagrt_load_csr");
    if (!ctx) return DAGRT_E_INVAL;
    if (!out) return fail(ctx, DAGRT_E_INVAL, "dagrt_load_csr: out is NULL");
    *out = nullptr;
    if (flags & ~DAGRT_PTR_DEVICE) return fail(ctx, DAGRT_E_INVAL, "dagrt_load_csr: unknown flags 0x%x", flags);
    if (int rc = refuse_in_capture(ctx, true, "dagrt_load_csr")) return rc;
    if (n_dags < 0) return fail(ctx, DAGRT_E_INVAL, "dagrt_load_csr: n_dags < 0");
    if (M < 1 || M > DAGRT_MAX_M) return fail(ctx, DAGRT_E_INVAL, "dagrt_load_csr: M=%d outside [1, %d]", M, DAGRT_MAX_M);
    if (!node_off || !edge_off) return fail(ctx, DAGRT_E_INVAL, "dagrt_load_csr: NULL offsets");
    const bool dev = (flags & DAGRT_PTR_DEVICE) != 0;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");

    std::vector<int64_t> hn(n_dags + 1), he(n_dags + 1);
    if (dev) {  // through the pinned staging buffer
        int64_t *pin = nullptr;
        const size_t nb = sizeof(int64_t) * (n_dags + 1);
        CK(pinned(ctx, 2 * nb, (void **)&pin), "pinned staging");
        CK(cudaMemcpyAsync(pin, node_off, nb, cudaMemcpyDeviceToHost, ctx->stream), "copy node_off");
        CK(cudaMemcpyAsync(pin + n_dags + 1, edge_off, nb, cudaMemcpyDeviceToHost, ctx->stream), "copy edge_off");
        CK(cudaStreamSynchronize(ctx->stream), "stream synchronize");
        std::memcpy(hn.data(), pin, nb);
        std::memcpy(he.data(), pin + n_dags + 1, nb);
    } else {
        std::memcpy(hn.data(), node_off, sizeof(int64_t) * (n_dags + 1));
        std::memcpy(he.data(), edge_off, sizeof(int64_t) * (n_dags + 1));
    }
    if (hn[0] != 0 || he[0] != 0) return fail(ctx, DAGRT_E_INVAL, "dagrt_load_csr: offsets must start at 0");
    int max_v = 0;
    for (int d = 0; d < n_dags; d++) {
        const int64_t v = hn[d + 1] - hn[d], e = he[d + 1] - he[d];
        if (v < 0 || e < 0) return fail(ctx, DAGRT_E_INVAL, "dagrt_load_csr: offsets decrease at DAG %d", d);
        if (v > DAGRT_MAX_V) return fail(ctx, DAGRT_E_INVAL, "dagrt_load_csr: DAG %d has %lld > %d nodes", d, (long long)v, DAGRT_MAX_V);
        if (e > DAGRT_MAX_E) return fail(ctx, DAGRT_E_INVAL, "dagrt_load_csr: DAG %d has %lld > %d edges", d, (long long)e, DAGRT_MAX_E);
        max_v = std::max<int>(max_v, (int)v);
    }
    const int64_t tn = hn[n_dags], te = he[n_dags];
    if (n_dags > 0 && (!row_ptr || !wcet || !k64 || (te > 0 && !col)))
        return fail(ctx, DAGRT_E_INVAL, "dagrt_load_csr: NULL array");

    dagrt_batch *b = new dagrt_batch();
    b->ctx = ctx;
    b->n_dags = n_dags;
    b->M = M;
    b->total_nodes = tn;
    b->total_edges = te;
    b->max_v = max_v;
    b->h_node_off = std::move(hn);
    auto bail = [&](int code) {
        batch_release(b);
        delete b;
        return code;
    };
    cudaError_t e;
    if (dev) {
        b->node_off = node_off;
        b->edge_off = edge_off;
        b->row_ptr = row_ptr;
        b->col = col;
        b->wcet = wcet;
        b->k64 = k64;
    } else {
        int64_t *dn, *de, *dw;
        int32_t *dr, *dc;
        uint8_t *dk;
        if ((e = batch_alloc(b, &dn, n_dags + 1)) != cudaSuccess || (e = batch_alloc(b, &de, n_dags + 1)) != cudaSuccess ||
            (e = batch_alloc(b, &dr, tn + n_dags)) != cudaSuccess || (e = batch_alloc(b, &dc, te)) != cudaSuccess ||
            (e = batch_alloc(b, &dw, tn)) != cudaSuccess || (e = batch_alloc(b, &dk, tn)) != cudaSuccess)
            return bail(cuda_fail(ctx, e, "allocate batch copy"));
        cudaStream_t st = ctx->stream;
        if ((e = cudaMemcpyAsync(dn, node_off, 8 * (n_dags + 1), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(de, edge_off, 8 * (n_dags + 1), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(dr, row_ptr, 4 * (tn + n_dags), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
            (te > 0 && (e = cudaMemcpyAsync(dc, col, 4 * te, cudaMemcpyHostToDevice, st)) != cudaSuccess) ||
            (e = cudaMemcpyAsync(dw, wcet, 8 * tn, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(dk, k64, tn, cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return bail(cuda_fail(ctx, e, "copy batch to device"));
        b->node_off = dn;
        b->edge_off = de;
        b->row_ptr = dr;
        b->col = dc;
        b->wcet = dw;
        b->k64 = dk;
    }

    b->h_edge_off = std::move(he);
    if ((e = batch_alloc(b, &b->lists, n_dags)) != cudaSuccess ||
        (e = batch_alloc(b, &b->counters, kNumClasses)) != cudaSuccess || (e = batch_alloc(b, &b->err, 1)) != cudaSuccess ||
        (e = cudaMemsetAsync(b->err, 0, sizeof(int32_t), ctx->stream)) != cudaSuccess)
        return bail(cuda_fail(ctx, e, "allocate class lists"));
    if (int rc = partition_classes(b)) return bail(rc);
    // host copies must be complete before the caller may reuse its buffers
    if (!dev && (e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) return bail(cuda_fail(ctx, e, "synchronize"));
    ctx->n_batches++;
    ctx->live++;
    *out = b;
    return DAGRT_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ schedule
namespace {

struct OutField {
    void *user;    // caller pointer
    void **slot;   // field in the device-side struct
    size_t bytes;  // size of the array
};

}  // namespace

static int ensure_plan(dagrt_batch *b, int variant) {
    dagrt_ctx *ctx = b->ctx;
    Plan &p = b->plan[variant];
    if (p.rows) return DAGRT_OK;
    cudaError_t e;
    const size_t rows = (size_t)(2 * b->total_nodes);
    if ((e = batch_alloc(b, &p.rows, rows)) != cudaSuccess ||
        (e = batch_alloc(b, &p.nrows, b->n_dags)) != cudaSuccess ||
        (e = batch_alloc(b, &p.pflag, b->n_dags)) != cudaSuccess ||
        (e = batch_alloc(b, &p.status, b->n_dags)) != cudaSuccess ||
        (e = batch_alloc(b, &p.bound, b->n_dags)) != cudaSuccess)
        return cuda_fail(ctx, e, "allocate plan");
    return DAGRT_OK;
}

// chunks of a plan for the balanced bound kernel (built once per plan)
static int ensure_chunks(dagrt_batch *b, int variant) {
    dagrt_ctx *ctx = b->ctx;
    Plan &p = b->plan[variant];
    if (p.chunked && p.chunk_rows == b->tune.chunk_rows) return DAGRT_OK;
    if (!p.ci.chunk) {  // sized for the smallest chunk_rows, so a retune never reallocates
        cudaError_t e;
        if ((e = batch_alloc(b, &p.ci.chunk, (size_t)(2 * b->total_nodes))) != cudaSuccess ||
            (e = batch_alloc(b, &p.ci.nchunk, (size_t)b->n_dags)) != cudaSuccess ||
            (e = batch_alloc(b, &p.ci.cpre, (size_t)b->n_dags + 1)) != cudaSuccess ||
            (e = batch_alloc(b, &p.ci.item, (size_t)chunk_items_bound(b->total_nodes, b->n_dags, kMinChunkRows))) !=
                cudaSuccess)
            return cuda_fail(ctx, e, "allocate plan chunks");
    }
    CK(bound_build_chunks(b->n_dags, b->node_off, p.rows, p.nrows, p.status, p.pflag, p.ci, b->tune.chunk_rows,
                          ctx->n_sm, ctx->stream),
       "build plan chunks");
    ctx->launches += 3;
    // a capture only records the build: an eager call after it must build again
    p.chunked = !ctx->capturing;
    p.chunk_rows = b->tune.chunk_rows;
    return DAGRT_OK;
}

static int ensure_bscr(dagrt_batch *b, size_t bytes) {
    dagrt_ctx *ctx = b->ctx;
    if (b->bscr_cap >= bytes && !b->bscr_dirty) return DAGRT_OK;
    if (b->bscr_cap >= bytes) {
        if (ctx->capturing) return fail(ctx, DAGRT_E_INVAL, "bound scratch must be cleared outside graph capture");
        CK(cudaMemsetAsync(b->bscr, 0, b->bscr_cap, ctx->stream), "clear bound scratch");
        b->bscr_dirty = false;
        return DAGRT_OK;
    }
    if (ctx->capturing) return fail(ctx, DAGRT_E_INVAL, "scratch must grow during graph capture: make the call once before capturing");
    CK(cudaStreamSynchronize(ctx->stream), "synchronize");
    if (b->bscr) ctx->pool.put(b->bscr, b->bscr_cap);
    b->bscr = nullptr;
    b->bscr_cap = 0;
    bytes = (bytes + 255) / 256 * 256;
    CK(ctx->pool.get(&b->bscr, bytes), "allocate bound scratch");
    b->bscr_cap = bytes;
    // the work-item counter and the bound accumulators start at zero; every call leaves
    // them zero
    CK(cudaMemsetAsync(b->bscr, 0, bytes, ctx->stream), "clear bound scratch");
    b->bscr_dirty = false;
    return DAGRT_OK;
}

static int ensure_tmp(dagrt_batch *b, size_t bytes) {
    dagrt_ctx *ctx = b->ctx;
    if (b->tmp_cap >= bytes) return DAGRT_OK;
    if (ctx->capturing) return fail(ctx, DAGRT_E_INVAL, "scratch must grow during graph capture: make the call once before capturing");
    CK(cudaStreamSynchronize(ctx->stream), "synchronize");
    if (b->tmp) ctx->pool.put(b->tmp, b->tmp_cap);
    b->tmp = nullptr;
    b->tmp_cap = 0;
    bytes = (bytes + 255) / 256 * 256;
    CK(ctx->pool.get(&b->tmp, bytes), "allocate scratch");
    b->tmp_cap = bytes;
    return DAGRT_OK;
}

extern "C" int dagrt_schedule(dagrt_batch *b, int32_t variant, const dagrt_schedule_out *out, uint32_t flags) {
    NvtxRange nvtx_range_("dagrt_schedule");
    if (!b) return DAGRT_E_INVAL;
    dagrt_ctx *ctx = b->ctx;
    if (variant < 0 || variant >= DAGRT_N_VARIANTS)
        return fail(ctx, DAGRT_E_INVAL, "dagrt_schedule: unknown variant %d", variant);
    if (flags & ~DAGRT_PTR_DEVICE) return fail(ctx, DAGRT_E_INVAL, "dagrt_schedule: unknown flags 0x%x", flags);
    if (int rc = refuse_in_capture(ctx, !(flags & DAGRT_PTR_DEVICE) || (out && out->extra_off), "dagrt_schedule"))
        return rc;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    int rc = ensure_plan(b, variant);
    if (rc) return rc;
    Plan &p = b->plan[variant];
    const bool dev = (flags & DAGRT_PTR_DEVICE) != 0;
    dagrt_schedule_out o;
    std::memset(&o, 0, sizeof o);
    if (out) o = *out;
    if ((o.extra_src == nullptr) != (o.extra_dst == nullptr) || (o.extra_src && !o.extra_off))
        return fail(ctx, DAGRT_E_INVAL, "dagrt_schedule: extra_src, extra_dst and extra_off go together");
    if (!o.extra_src) o.extra_off = nullptr;

    const size_t nd = b->n_dags, nn = b->total_nodes;
    int64_t n_extra_cap = 0;
    if (o.extra_off) {
        if (dev) {
            CK(cudaMemcpyAsync(&n_extra_cap, o.extra_off + nd, 8, cudaMemcpyDeviceToHost, ctx->stream), "copy extra_off");
            CK(cudaStreamSynchronize(ctx->stream), "synchronize");
        } else {
            n_extra_cap = o.extra_off[nd];
        }
        if (n_extra_cap < 0) return fail(ctx, DAGRT_E_INVAL, "dagrt_schedule: negative extra_off");
    }
    dagrt_schedule_out dv = o;  // device-side view
    std::vector<OutField> fields = {
        {o.bound, (void **)&dv.bound, 8 * nd},         {o.status, (void **)&dv.status, 4 * nd},
        {o.n_groups, (void **)&dv.n_groups, 4 * nd},   {o.n_seg, (void **)&dv.n_seg, 4 * nd},
        {o.n_rows, (void **)&dv.n_rows, 4 * nd},       {o.n_extra, (void **)&dv.n_extra, 8 * nd},
        {o.level, (void **)&dv.level, 4 * nn},         {o.wanc, (void **)&dv.wanc, 8 * nn},
        {o.block_of, (void **)&dv.block_of, 4 * nn},   {o.group_of, (void **)&dv.group_of, 4 * nn},
        {o.exec_group, (void **)&dv.exec_group, 4 * nn}, {o.m, (void **)&dv.m, 4 * nn},
        {o.group_R, (void **)&dv.group_R, 8 * nn},     {o.seg_parent, (void **)&dv.seg_parent, 4 * nn},
        {o.seg_load, (void **)&dv.seg_load, 8 * nn},   {o.seg_m, (void **)&dv.seg_m, 4 * nn},
        {o.seg_group, (void **)&dv.seg_group, 4 * nn}, {o.row_id, (void **)&dv.row_id, 8 * nn},
        {o.row_group, (void **)&dv.row_group, 8 * nn}, {o.row_m0, (void **)&dv.row_m0, 8 * nn},
        {o.row_load, (void **)&dv.row_load, 16 * nn},  {o.extra_off, (void **)&dv.extra_off, 8 * (nd + 1)},
        {o.extra_src, (void **)&dv.extra_src, 4 * (size_t)n_extra_cap},
        {o.extra_dst, (void **)&dv.extra_dst, 4 * (size_t)n_extra_cap},
        {o.greedy, (void **)&dv.greedy, 8 * nd},       {o.greedy_unaware, (void **)&dv.greedy_unaware, 8 * nd},
        {o.graham_para, (void **)&dv.graham_para, 8 * nd}, {o.crit_path, (void **)&dv.crit_path, 8 * nd},
    };
    if ((o.seg_parent || o.seg_load || o.seg_m || o.seg_group) &&
        !(o.seg_parent && o.seg_load && o.seg_m && o.seg_group))
        return fail(ctx, DAGRT_E_INVAL, "dagrt_schedule: segment outputs go together");
    if (!dev) {  // stage every requested host output through one device scratch block
        size_t total = 0;
        for (auto &f : fields)
            if (f.user) total += (f.bytes + 255) / 256 * 256;
        rc = ensure_tmp(b, total > 0 ? total : 256);
        if (rc) return rc;
        size_t off = 0;
        for (auto &f : fields) {
            if (!f.user) continue;
            *f.slot = (char *)b->tmp + off;
            off += (f.bytes + 255) / 256 * 256;
        }
        if (o.extra_off)
            CK(cudaMemcpyAsync(dv.extra_off, o.extra_off, 8 * (nd + 1), cudaMemcpyHostToDevice, ctx->stream),
               "copy extra_off");
    }

    SchedArgs a;
    std::memset(&a, 0, sizeof a);
    a.node_off = b->node_off;
    a.edge_off = b->edge_off;
    a.row_ptr = b->row_ptr;
    a.col = b->col;
    a.wcet = b->wcet;
    a.k64 = b->k64;
    a.M = b->M;
    a.variant = variant;
    a.status = p.status;
    a.bound = p.bound;
    a.oversize_status = DAGRT_E_INTERNAL;  // the size classes guarantee every DAG fits
    a.tot_nodes = -1;                       // offsets checked by dagrt_load_csr
    a.tot_edges = -1;
    a.nrows = p.nrows;
    a.pflag = p.pflag;
    a.plan = p.rows;
    a.o = dv;
    if (nd > 0) {
        CK(cudaMemsetAsync(b->counters, 0, kNumClasses * sizeof(int32_t), ctx->stream), "reset counters");
        CK(ensure_side_streams(ctx), "create side streams");
        // size classes run concurrently: fork from the context stream, join back into it.
        // Largest class first, so that the longest DAGs start at once and the short ones
        // fill in around them (with classes of 16 nodes and four teams per CTA this measured
        // 1-4% faster than smallest first on the 10,000-DAG batch)
        CK(cudaEventRecord(ctx->fork, ctx->stream), "record fork");
        int used[dagrt_ctx::kSide], nused = 0;
        for (int c = kNumClasses - 1; c >= 0; c--) {
            const int n = b->class_off[c + 1] - b->class_off[c];
            if (n == 0) continue;
            cudaStream_t st = ctx->side[c];
            CK(cudaStreamWaitEvent(st, ctx->fork, 0), "fork");
            a.list = b->lists + b->class_off[c];
            a.n_list = n;
            a.counter = b->counters + c;
            if (c < kNumWarpClasses) {
                a.vcap = b->wcap_v[c];
                a.ecap = b->wcap_e[c];
                CK(sched_launch_warp(a, ctx->n_sm, st), "launch scheduler (warp teams)");
            } else if (c == kClsCtaSmem) {
                a.vcap = b->smem_vcap;
                a.ecap = b->smem_ecap;
                CK(sched_launch_cta_smem(a, ctx->n_sm, st), "launch scheduler (CTA teams, shared memory)");
            } else {
                a.gws = b->gws;
                a.gws_stride = b->gws_stride;
                a.vcap = b->big_vcap;
                a.ecap = b->big_ecap;
                CK(sched_launch_cta(a, b->big_grid, st), "launch scheduler (CTA teams)");
            }
            ctx->launches++;
            CK(cudaEventRecord(ctx->join[c], st), "record join");
            used[nused++] = c;
        }
        for (int i = 0; i < nused; i++) CK(cudaStreamWaitEvent(ctx->stream, ctx->join[used[i]], 0), "join");
    }
    p.valid = true;
    p.chunked = false;
    if (dev) return DAGRT_OK;

    for (auto &f : fields) {
        if (!f.user || f.user == (void *)o.extra_off) continue;
        if (f.bytes) CK(cudaMemcpyAsync(f.user, *f.slot, f.bytes, cudaMemcpyDeviceToHost, ctx->stream), "copy output");
    }
    std::vector<int32_t> st(nd);
    if (nd) CK(cudaMemcpyAsync(st.data(), p.status, 4 * nd, cudaMemcpyDeviceToHost, ctx->stream), "copy status");
    CK(cudaStreamSynchronize(ctx->stream), "synchronize");
    for (size_t d = 0; d < nd; d++)
        if (st[d] != DAGRT_OK)
            return fail(ctx, st[d], "dagrt_schedule: DAG %zu failed with status %d", d, st[d]);
    return DAGRT_OK;
}

// ------------------------------------------------------------------ schedulability
extern "C" int dagrt_schedulable(dagrt_batch *b, int32_t variant, const int64_t *deadline, int32_t *ok,
                                 int64_t *n_ok, uint32_t flags) {
    NvtxRange nvtx_range_("dagrt_schedulable");
    if (!b) return DAGRT_E_INVAL;
    dagrt_ctx *ctx = b->ctx;
    if (flags & ~DAGRT_PTR_DEVICE) return fail(ctx, DAGRT_E_INVAL, "dagrt_schedulable: unknown flags 0x%x", flags);
    if (int rc = refuse_in_capture(ctx, !(flags & DAGRT_PTR_DEVICE), "dagrt_schedulable")) return rc;
    if (variant < 0 || variant >= DAGRT_N_VARIANTS || !b->plan[variant].valid)
        return fail(ctx, DAGRT_E_INVAL, "dagrt_schedulable: variant %d was not scheduled on this batch", variant);
    if (!deadline && b->n_dags > 0) return fail(ctx, DAGRT_E_INVAL, "dagrt_schedulable: deadline is NULL");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    const Plan &p = b->plan[variant];
    const bool dev = (flags & DAGRT_PTR_DEVICE) != 0;
    const size_t nd = b->n_dags;
    const int64_t *d_dl = deadline;
    int32_t *d_ok = ok;
    unsigned long long *d_n = (unsigned long long *)n_ok;
    if (!dev) {  // stage: [deadline | ok | count]
        const size_t a8 = (8 * nd + 255) / 256 * 256, a4 = (4 * nd + 255) / 256 * 256;
        int rc = ensure_tmp(b, a8 + a4 + 256);
        if (rc) return rc;
        char *t = (char *)b->tmp;
        d_dl = (const int64_t *)t;
        d_ok = ok ? (int32_t *)(t + a8) : nullptr;
        d_n = (unsigned long long *)(t + a8 + a4);
        if (nd) CK(cudaMemcpyAsync((void *)d_dl, deadline, 8 * nd, cudaMemcpyHostToDevice, ctx->stream), "copy deadlines");
    }
    if (d_n) CK(cudaMemsetAsync(d_n, 0, 8, ctx->stream), "clear count");
    CK(sched_schedulable(b->n_dags, p.status, p.bound, d_dl, d_ok, d_n, ctx->n_sm, ctx->stream), "schedulability");
    ctx->launches += nd > 0;
    if (dev) return DAGRT_OK;
    if (ok && nd) CK(cudaMemcpyAsync(ok, d_ok, 4 * nd, cudaMemcpyDeviceToHost, ctx->stream), "copy flags");
    int64_t cnt = 0;
    CK(cudaMemcpyAsync(&cnt, d_n, 8, cudaMemcpyDeviceToHost, ctx->stream), "copy count");
    CK(cudaStreamSynchronize(ctx->stream), "synchronize");
    if (n_ok) *n_ok = cnt;
    return DAGRT_OK;
}

// ------------------------------------------------------------------ candidate bounds
extern "C" int dagrt_bound(dagrt_batch *b, int32_t n_variants, const int32_t *variant_ids, int32_t n_alloc,
                           const uint8_t *m_alloc, int64_t cand_stride, int64_t *out_bound, int64_t *best_bound,
                           int32_t *best_cand, uint32_t flags) {
    NvtxRange nvtx_range_("dagrt_bound");
    if (!b) return DAGRT_E_INVAL;
    dagrt_ctx *ctx = b->ctx;
    if (flags & ~DAGRT_PTR_DEVICE) return fail(ctx, DAGRT_E_INVAL, "dagrt_bound: unknown flags 0x%x", flags);
    if (int rc = refuse_in_capture(ctx, !(flags & DAGRT_PTR_DEVICE), "dagrt_bound")) return rc;
    if (n_variants < 1 || n_variants > kMaxVariantsPerCall || !variant_ids)
        return fail(ctx, DAGRT_E_INVAL, "dagrt_bound: n_variants must be in [1, %d]", kMaxVariantsPerCall);
    if (n_alloc < 1) return fail(ctx, DAGRT_E_INVAL, "dagrt_bound: n_alloc < 1");
    const int64_t n_cand = (int64_t)n_variants * n_alloc;
    if (n_cand > (1ll << 30)) return fail(ctx, DAGRT_E_INVAL, "dagrt_bound: too many candidates");
    if (cand_stride < n_cand || cand_stride % 16 != 0 || cand_stride > 65536)
        return fail(ctx, DAGRT_E_INVAL, "dagrt_bound: cand_stride must be >= n_cand, <= 65536 and a multiple of 16");
    if (!m_alloc && b->total_nodes > 0) return fail(ctx, DAGRT_E_INVAL, "dagrt_bound: m_alloc is NULL");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    BoundArgs a;
    std::memset(&a, 0, sizeof a);
    a.n_dags = b->n_dags;
    a.node_off = b->node_off;
    a.M = b->M;
    a.n_variants = n_variants;
    a.n_alloc = n_alloc;
    a.stride = cand_stride;
    a.err = b->err;
    for (int i = 0; i < n_variants; i++) {
        const int v = variant_ids[i];  // variant_ids is always a host array
        if (v < 0 || v >= DAGRT_N_VARIANTS || !b->plan[v].valid)
            return fail(ctx, DAGRT_E_INVAL, "dagrt_bound: variant %d was not scheduled on this batch", v);
        a.plan[i] = b->plan[v].rows;
        a.nrows[i] = b->plan[v].nrows;
        a.pflag[i] = b->plan[v].pflag;
        a.status[i] = b->plan[v].status;
    }
    const bool dev = (flags & DAGRT_PTR_DEVICE) != 0;
    const size_t nd = b->n_dags;
    const size_t alloc_bytes = (size_t)(2 * b->total_nodes) * (size_t)cand_stride;
    const size_t out_bytes = nd * (size_t)n_cand * 8;
    if (dev) {
        if ((uintptr_t)m_alloc % 16 != 0)
            return fail(ctx, DAGRT_E_INVAL, "dagrt_bound: device m_alloc must be 16-byte aligned");
        a.m_alloc = m_alloc;
        a.out = out_bound;
        a.best_bound = best_bound;
        a.best_cand = best_cand;
    } else {  // stage through one device scratch block
        const size_t need = (alloc_bytes + 255) / 256 * 256 + (out_bound ? (out_bytes + 255) / 256 * 256 : 0) +
                            (8 * nd + 255) / 256 * 256 + (4 * nd + 255) / 256 * 256 + 256;
        int rc = ensure_tmp(b, need);
        if (rc) return rc;
        char *t = (char *)b->tmp;
        uint8_t *d_alloc = (uint8_t *)t;
        t += (alloc_bytes + 255) / 256 * 256;
        int64_t *d_out = nullptr;
        if (out_bound) {
            d_out = (int64_t *)t;
            t += (out_bytes + 255) / 256 * 256;
        }
        int64_t *d_bb = (int64_t *)t;
        t += (8 * nd + 255) / 256 * 256;
        int32_t *d_bc = (int32_t *)t;
        if (alloc_bytes)
            CK(cudaMemcpyAsync(d_alloc, m_alloc, alloc_bytes, cudaMemcpyHostToDevice, ctx->stream), "copy m_alloc");
        a.m_alloc = d_alloc;
        a.out = d_out;
        a.best_bound = best_bound ? d_bb : nullptr;
        a.best_cand = best_cand ? d_bc : nullptr;
    }
    ChunkArgs ch;
    std::memset(&ch, 0, sizeof ch);
    const bool items = bound_chunk_eligible(a, b->total_nodes, b->tune.chunk_rows);
    if (items) {
        for (int i = 0; i < n_variants; i++) {
            const int v = variant_ids[i];
            int rc = ensure_chunks(b, v);
            if (rc) return rc;
            ch.chunk[i] = b->plan[v].ci.chunk;
            ch.nchunk[i] = b->plan[v].ci.nchunk;
            ch.cpre[i] = b->plan[v].ci.cpre;
            ch.item[i] = b->plan[v].ci.item;
        }
        int rc = ensure_bscr(b, bound_chunk_scratch(b->n_dags, b->total_nodes, n_variants, n_alloc, b->tune.chunk_rows));
        if (rc) return rc;
        char *t = (char *)b->bscr;
        ch.counter = (uint32_t *)t;  // the first 256 bytes
        ch.acc = (unsigned long long *)(t + 256);
        ch.warps = b->tune.item_warps;
        ch.alloc_rows = 2 * b->total_nodes;
    }
    int nl = 0;
    {
        const cudaError_t e = bound_launch(a, items ? &ch : nullptr, ctx->n_sm, ctx->stream, &nl);
        if (e != cudaSuccess) {
            if (items) b->bscr_dirty = true;  // the work items may have run without the finish
            return cuda_fail(ctx, e, "launch bound kernel");
        }
    }
    ctx->launches += nl;
    if (dev) return DAGRT_OK;
    if (out_bound && out_bytes) CK(cudaMemcpyAsync(out_bound, a.out, out_bytes, cudaMemcpyDeviceToHost, ctx->stream), "copy bounds");
    if (best_bound && nd) CK(cudaMemcpyAsync(best_bound, a.best_bound, 8 * nd, cudaMemcpyDeviceToHost, ctx->stream), "copy best");
    if (best_cand && nd) CK(cudaMemcpyAsync(best_cand, a.best_cand, 4 * nd, cudaMemcpyDeviceToHost, ctx->stream), "copy best");
    int32_t err = 0;
    CK(cudaMemcpyAsync(&err, b->err, sizeof err, cudaMemcpyDeviceToHost, ctx->stream), "copy error word");
    CK(cudaStreamSynchronize(ctx->stream), "synchronize");
    if (err) return fail(ctx, err, "dagrt_bound: a tile copy did not complete in time");
    return DAGRT_OK;
}

// ------------------------------------------------------------------ search
extern "C" int dagrt_search(dagrt_batch *b, const dagrt_search_cfg *cfg, int64_t *out_bound, int64_t *best_bound,
                            int32_t *best_cand, uint8_t *best_m, uint32_t flags) {
    NvtxRange nvtx_range_("dagrt_search");
    if (!b) return DAGRT_E_INVAL;
    dagrt_ctx *ctx = b->ctx;
    if (!cfg) return fail(ctx, DAGRT_E_INVAL, "dagrt_search: cfg is NULL");
    if (flags & ~DAGRT_PTR_DEVICE) return fail(ctx, DAGRT_E_INVAL, "dagrt_search: unknown flags 0x%x", flags);
    if (int rc = refuse_in_capture(ctx, !(flags & DAGRT_PTR_DEVICE), "dagrt_search")) return rc;
    if (cfg->n_variants < 1 || cfg->n_variants > kMaxVariantsPerCall || !cfg->variant_ids)
        return fail(ctx, DAGRT_E_INVAL, "dagrt_search: n_variants must be in [1, %d]", kMaxVariantsPerCall);
    if (cfg->n_alloc < 1 || (int64_t)cfg->n_variants * cfg->n_alloc > (1 << 20))
        return fail(ctx, DAGRT_E_INVAL, "dagrt_search: need 1 <= n_alloc and n_variants * n_alloc <= 2^20");
    const int mode = cfg->mode;
    if (mode != DAGRT_SEARCH_RANDOM && mode != DAGRT_SEARCH_EXHAUSTIVE && mode != DAGRT_SEARCH_PERTURB)
        return fail(ctx, DAGRT_E_INVAL, "dagrt_search: unknown mode %d", mode);
    const int max_levels = mode == DAGRT_SEARCH_EXHAUSTIVE ? 15 : 16;
    if (cfg->n_levels < 1 || cfg->n_levels > max_levels || !cfg->levels)
        return fail(ctx, DAGRT_E_INVAL, "dagrt_search: n_levels must be in [1, %d]", max_levels);
    for (int i = 0; i < cfg->n_levels; i++) {
        if (mode != DAGRT_SEARCH_PERTURB && cfg->levels[i] < 1)
            return fail(ctx, DAGRT_E_INVAL, "dagrt_search: level %d is 0", i);
        if (mode == DAGRT_SEARCH_PERTURB && cfg->levels[i] > 4)
            return fail(ctx, DAGRT_E_INVAL, "dagrt_search: perturbation code %d is not in [0, 4]", i);
    }
    if (b->n_dags >= (1 << 24)) return fail(ctx, DAGRT_E_INVAL, "dagrt_search: too many DAGs");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    BoundArgs a;
    std::memset(&a, 0, sizeof a);
    a.n_dags = b->n_dags;
    a.node_off = b->node_off;
    a.M = b->M;
    a.n_variants = cfg->n_variants;
    a.n_alloc = cfg->n_alloc;
    a.stride = 16;
    a.err = b->err;
    a.gen = 1;
    a.gen_mode = mode;
    a.seed = cfg->seed;
    a.n_levels = cfg->n_levels;
    for (int i = 0; i < 16; i++) a.levels[i] = i < cfg->n_levels ? cfg->levels[i] : cfg->levels[0];
    for (int i = 0; i < cfg->n_variants; i++) {
        const int v = cfg->variant_ids[i];
        if (v < 0 || v >= DAGRT_N_VARIANTS || !b->plan[v].valid)
            return fail(ctx, DAGRT_E_INVAL, "dagrt_search: variant %d was not scheduled on this batch", v);
        a.plan[i] = b->plan[v].rows;
        a.nrows[i] = b->plan[v].nrows;
        a.pflag[i] = b->plan[v].pflag;
        a.status[i] = b->plan[v].status;
    }
    const bool dev = (flags & DAGRT_PTR_DEVICE) != 0;
    const size_t nd = b->n_dags;
    const int64_t n_cand = (int64_t)cfg->n_variants * cfg->n_alloc;
    const size_t out_bytes = nd * (size_t)n_cand * 8, m_bytes = (size_t)(2 * b->total_nodes);
    if (dev) {
        a.out = out_bound;
        a.best_bound = best_bound;
        a.best_cand = best_cand;
        a.best_m = best_m;
    } else {
        const size_t need = (out_bound ? (out_bytes + 255) / 256 * 256 : 0) + (8 * nd + 255) / 256 * 256 +
                            (4 * nd + 255) / 256 * 256 + (best_m ? (m_bytes + 255) / 256 * 256 : 0) + 256;
        int rc = ensure_tmp(b, need);
        if (rc) return rc;
        char *t = (char *)b->tmp;
        auto take = [&](size_t bytes) {
            char *p = t;
            t += (bytes + 255) / 256 * 256;
            return (void *)p;
        };
        a.out = out_bound ? (int64_t *)take(out_bytes) : nullptr;
        a.best_bound = (int64_t *)take(8 * nd);
        a.best_cand = (int32_t *)take(4 * nd);
        a.best_m = best_m ? (uint8_t *)take(m_bytes) : nullptr;
        if (best_m && m_bytes) CK(cudaMemsetAsync(a.best_m, 0, m_bytes, ctx->stream), "clear best_m");
    }
    int nl = 0;
    CK(bound_launch(a, nullptr, ctx->n_sm, ctx->stream, &nl), "launch search kernel");
    ctx->launches += nl;
    if (dev) return DAGRT_OK;
    if (out_bound && out_bytes) CK(cudaMemcpyAsync(out_bound, a.out, out_bytes, cudaMemcpyDeviceToHost, ctx->stream), "copy bounds");
    if (best_bound && nd) CK(cudaMemcpyAsync(best_bound, a.best_bound, 8 * nd, cudaMemcpyDeviceToHost, ctx->stream), "copy best");
    if (best_cand && nd) CK(cudaMemcpyAsync(best_cand, a.best_cand, 4 * nd, cudaMemcpyDeviceToHost, ctx->stream), "copy best");
    if (best_m && m_bytes) CK(cudaMemcpyAsync(best_m, a.best_m, m_bytes, cudaMemcpyDeviceToHost, ctx->stream), "copy best_m");
    int32_t err = 0;
    CK(cudaMemcpyAsync(&err, b->err, sizeof err, cudaMemcpyDeviceToHost, ctx->stream), "copy error word");
    CK(cudaStreamSynchronize(ctx->stream), "synchronize");
    if (err) return fail(ctx, err, "dagrt_search: a tile copy did not complete in time");
    return DAGRT_OK;
}

// ------------------------------------------------------------------ learned proposer
// proposal buffer: column 0 = the paper's allocation, columns 1..k = the k best assignments
constexpr int64_t kPropStride = 32;

struct dagrt_model {
    dagrt_ctx *ctx = nullptr;
    int32_t L = 0;
    uint8_t levels[kMaxLevels] = {0};
    uint8_t *d_levels = nullptr;
    float *p = nullptr, *m = nullptr, *v = nullptr, *part = nullptr;
    int n_parts = 0, step = 0;
    uint16_t *wt[3] = {}, *wb[3] = {};
    std::vector<std::pair<void *, size_t>> owned;
};

namespace {

template <class T>
cudaError_t model_alloc(dagrt_model *md, T **p, size_t n) {
    void *q = nullptr;
    cudaError_t e = md->ctx->pool.get(&q, (n ? n : 1) * sizeof(T));
    if (e == cudaSuccess) {
        *p = (T *)q;
        md->owned.emplace_back(q, (n ? n : 1) * sizeof(T));
    }
    return e;
}

GnnGraph graph_of(dagrt_batch *b) {
    GnnGraph g;
    g.n_nodes = b->total_nodes;
    g.n_edges = b->total_edges;
    g.pred_off = b->gnn.pred_off;
    g.pred_idx = b->gnn.pred_idx;
    g.succ_off = b->gnn.succ_off;
    g.succ_idx = b->gnn.succ_idx;
    return g;
}

}  // namespace

// variant-0 schedule (plan, levels, W^anc, m), message-passing graph and node features
static int gnn_prepare(dagrt_batch *b, bool train) {
    dagrt_ctx *ctx = b->ctx;
    auto &G = b->gnn;
    const size_t N = (size_t)b->total_nodes, E = (size_t)b->total_edges;
    cudaError_t e;
    if (!G.graph) {
        if ((e = batch_alloc(b, &G.pred_off, N + 1)) != cudaSuccess || (e = batch_alloc(b, &G.succ_off, N + 1)) != cudaSuccess ||
            (e = batch_alloc(b, &G.pred_idx, E)) != cudaSuccess || (e = batch_alloc(b, &G.succ_idx, E)) != cudaSuccess ||
            (e = batch_alloc(b, &G.cursor, N)) != cudaSuccess || (e = batch_alloc(b, &G.level, N)) != cudaSuccess ||
            (e = batch_alloc(b, &G.m, N)) != cudaSuccess || (e = batch_alloc(b, &G.wanc, N)) != cudaSuccess ||
            (e = batch_alloc(b, &G.x, N * kFeat)) != cudaSuccess || (e = batch_alloc(b, &G.h[0], N * kHidden)) != cudaSuccess ||
            (e = batch_alloc(b, &G.h[1], N * kHidden)) != cudaSuccess || (e = batch_alloc(b, &G.h[2], N * kHidden)) != cudaSuccess ||
            (e = batch_alloc(b, &G.logits, N * kMaxLevels)) != cudaSuccess ||
            (e = batch_alloc(b, &G.best_level, N)) != cudaSuccess || (e = batch_alloc(b, &G.cand, 2 * N * kPropStride)) != cudaSuccess ||
            (e = batch_alloc(b, &G.cbest, b->n_dags)) != cudaSuccess || (e = batch_alloc(b, &G.bbest, b->n_dags)) != cudaSuccess)
            return cuda_fail(ctx, e, "allocate proposer state");
        dagrt_schedule_out o;
        std::memset(&o, 0, sizeof o);
        o.level = G.level;
        o.wanc = G.wanc;
        o.m = G.m;
        int rc = dagrt_schedule(b, DAGRT_VAR_PAPER, &o, DAGRT_PTR_DEVICE);
        if (rc) return rc;
        const int32_t *st0 = b->plan[DAGRT_VAR_PAPER].status;
        CK(gnn_build_graph(b->n_dags, b->node_off, b->edge_off, b->row_ptr, b->col, st0, G.pred_off, G.pred_idx,
                           G.succ_off, G.succ_idx, G.cursor, ctx->n_sm, ctx->stream), "build message-passing graph");
        CK(gnn_features(b->n_dags, b->node_off, b->wcet, b->k64, G.level, G.wanc, G.m, st0, graph_of(b), G.x,
                        ctx->n_sm, ctx->stream), "node features");
        ctx->launches += 3;
        G.graph = !ctx->capturing;  // a capture only records the build
    }
    if (train && !G.train) {
        if ((e = batch_alloc(b, &G.dlogits, N * kMaxLevels)) != cudaSuccess ||
            (e = batch_alloc(b, &G.dh[0], N * kHidden)) != cudaSuccess || (e = batch_alloc(b, &G.dh[1], N * kHidden)) != cudaSuccess ||
            (e = batch_alloc(b, &G.dh[2], N * kHidden)) != cudaSuccess || (e = batch_alloc(b, &G.da, N * 3 * kHidden)) != cudaSuccess ||
            (e = batch_alloc(b, &G.labels, N)) != cudaSuccess || (e = batch_alloc(b, &G.loss_part, 1024)) != cudaSuccess)
            return cuda_fail(ctx, e, "allocate training state");
        G.train = true;
    }
    return DAGRT_OK;
}

static int gnn_forward(dagrt_batch *b, dagrt_model *md) {
    dagrt_ctx *ctx = b->ctx;
    auto &G = b->gnn;
    const GnnGraph g = graph_of(b);
    const int64_t boff[3] = {ParamLayout::b1, ParamLayout::b2, ParamLayout::b3};
    const uint16_t *in = G.x;
    for (int l = 0; l < 3; l++) {
        CK(gnn_layer_fwd(l == 0 ? kFeat : kHidden, g, in, md->wt[l], md->p + boff[l], G.h[l], b->err, ctx->n_sm,
                         ctx->stream), "layer forward");
        in = G.h[l];
    }
    ctx->launches += 3;
    return DAGRT_OK;
}

extern "C" int64_t dagrt_model_n_params(void) { return ParamLayout::total; }

extern "C" int dagrt_model_create(dagrt_ctx *ctx, int32_t n_levels, const uint8_t *levels, uint64_t seed,
                                  dagrt_model **out) {
    if (!ctx) return DAGRT_E_INVAL;
    if (!out) return fail(ctx, DAGRT_E_INVAL, "dagrt_model_create: out is NULL");
    *out = nullptr;
    if (n_levels < 1 || n_levels > kMaxLevels || !levels)
        return fail(ctx, DAGRT_E_INVAL, "dagrt_model_create: n_levels must be in [1, %d]", kMaxLevels);
    for (int i = 0; i < n_levels; i++)
        if (levels[i] < 1) return fail(ctx, DAGRT_E_INVAL, "dagrt_model_create: level %d is 0", i);
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    dagrt_model *md = new dagrt_model();
    md->ctx = ctx;
    md->L = n_levels;
    for (int i = 0; i < n_levels; i++) md->levels[i] = levels[i];
    md->n_parts = ctx->n_sm;
    const int64_t n = ParamLayout::total;
    cudaError_t e;
    auto bail = [&](int code) {
        for (auto &pb : md->owned) ctx->pool.put(pb.first, pb.second);
        delete md;
        return code;
    };
    if ((e = model_alloc(md, &md->p, n)) != cudaSuccess || (e = model_alloc(md, &md->m, n)) != cudaSuccess ||
        (e = model_alloc(md, &md->v, n)) != cudaSuccess || (e = model_alloc(md, &md->part, (size_t)n * md->n_parts)) != cudaSuccess ||
        (e = model_alloc(md, &md->d_levels, kMaxLevels)) != cudaSuccess)
        return bail(cuda_fail(ctx, e, "allocate model"));
    const int Ks[3] = {3 * kFeat, 3 * kHidden, 3 * kHidden};
    for (int l = 0; l < 3; l++)
        if ((e = model_alloc(md, &md->wt[l], (size_t)Ks[l] * kHidden)) != cudaSuccess ||
            (e = model_alloc(md, &md->wb[l], (size_t)Ks[l] * kHidden)) != cudaSuccess)
            return bail(cuda_fail(ctx, e, "allocate model"));
    // uniform(-a, a) weights with a = sqrt(6 / fan_in) from a SplitMix64 stream; zero biases
    std::vector<float> h(n, 0.f);
    uint64_t ctr = seed;
    auto unif = [&]() { return (float)((splitmix64(ctr++) >> 40) * (1.0 / (double)(1ull << 24))) * 2.f - 1.f; };
    const int64_t woff[4] = {ParamLayout::W1, ParamLayout::W2, ParamLayout::W3, ParamLayout::Wh};
    const int fan_in[4] = {3 * kFeat, 3 * kHidden, 3 * kHidden, kHidden};
    const int64_t wsz[4] = {3 * kFeat * kHidden, 3 * kHidden * kHidden, 3 * kHidden * kHidden, kHidden * kMaxLevels};
    for (int l = 0; l < 4; l++) {
        const float a = sqrtf(6.f / (float)fan_in[l]);
        for (int64_t i = 0; i < wsz[l]; i++) h[woff[l] + i] = a * unif();
    }
    cudaStream_t st = ctx->stream;
    if ((e = cudaMemcpyAsync(md->p, h.data(), n * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(md->m, 0, n * 4, st)) != cudaSuccess || (e = cudaMemsetAsync(md->v, 0, n * 4, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(md->d_levels, md->levels, kMaxLevels, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = gnn_refresh(md->p, md->wt, md->wb, st)) != cudaSuccess || (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return bail(cuda_fail(ctx, e, "initialise model"));
    *out = md;
    ctx->live++;
    return DAGRT_OK;
}

extern "C" void dagrt_model_free(dagrt_model *md) {
    if (!md) return;
    dagrt_ctx *ctx = md->ctx;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (auto &pb : md->owned) ctx->pool.put(pb.first, pb.second);
    delete md;
    ctx_unref(ctx);
}

extern "C" int dagrt_model_params(dagrt_model *md, float *get, const float *set) {
    if (!md) return DAGRT_E_INVAL;
    dagrt_ctx *ctx = md->ctx;
    if (int rc = refuse_in_capture(ctx, true, "dagrt_model_params")) return rc;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    const size_t bytes = ParamLayout::total * 4;
    if (set) {
        CK(cudaMemcpyAsync(md->p, set, bytes, cudaMemcpyHostToDevice, ctx->stream), "copy params");
        CK(gnn_refresh(md->p, md->wt, md->wb, ctx->stream), "refresh");
    }
    if (get) CK(cudaMemcpyAsync(get, md->p, bytes, cudaMemcpyDeviceToHost, ctx->stream), "copy params");
    CK(cudaStreamSynchronize(ctx->stream), "synchronize");
    return DAGRT_OK;
}

extern "C" int dagrt_model_state(dagrt_model *md, float *get, int32_t *get_step, const float *set,
                                 int32_t set_step) {
    if (!md) return DAGRT_E_INVAL;
    dagrt_ctx *ctx = md->ctx;
    if (int rc = refuse_in_capture(ctx, true, "dagrt_model_state")) return rc;
    if (set && set_step < 0) return fail(ctx, DAGRT_E_INVAL, "dagrt_model_state: negative step");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    const size_t n = ParamLayout::total, bytes = n * 4;
    float *dev[3] = {md->p, md->m, md->v};
    if (set) {
        for (int i = 0; i < 3; i++)
            CK(cudaMemcpyAsync(dev[i], set + i * n, bytes, cudaMemcpyHostToDevice, ctx->stream), "copy state");
        CK(gnn_refresh(md->p, md->wt, md->wb, ctx->stream), "refresh");
        md->step = set_step;
    }
    if (get)
        for (int i = 0; i < 3; i++)
            CK(cudaMemcpyAsync(get + i * n, dev[i], bytes, cudaMemcpyDeviceToHost, ctx->stream), "copy state");
    if (get_step) *get_step = md->step;
    CK(cudaStreamSynchronize(ctx->stream), "synchronize");
    return DAGRT_OK;
}

extern "C" int dagrt_model_logits(dagrt_batch *b, dagrt_model *md, float *logits, uint32_t flags) {
    NvtxRange nvtx_range_("dagrt_model_logits");
    if (!b || !md) return DAGRT_E_INVAL;
    dagrt_ctx *ctx = b->ctx;
    if (md->ctx != ctx) return fail(ctx, DAGRT_E_INVAL, "dagrt_model_logits: model of another context");
    if (int rc = refuse_in_capture(ctx, !(flags & DAGRT_PTR_DEVICE), "dagrt_model_logits")) return rc;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    int rc = gnn_prepare(b, false);
    if (rc) return rc;
    if ((rc = gnn_forward(b, md))) return rc;
    const GnnGraph g = graph_of(b);
    float *dst = (flags & DAGRT_PTR_DEVICE) ? logits : b->gnn.logits;
    CK(gnn_head(g, b->gnn.h[2], md->p + ParamLayout::Wh, md->p + ParamLayout::bh, md->L, nullptr, 0.f, dst, nullptr,
                nullptr, nullptr, ctx->n_sm, ctx->stream), "head");
    ctx->launches++;
    if (flags & DAGRT_PTR_DEVICE) return DAGRT_OK;
    if (logits && b->total_nodes)
        CK(cudaMemcpyAsync(logits, dst, (size_t)b->total_nodes * md->L * 4, cudaMemcpyDeviceToHost, ctx->stream), "copy logits");
    CK(cudaStreamSynchronize(ctx->stream), "synchronize");
    return DAGRT_OK;
}

// loss and gradients for the labelled nodes (host labels, -1 = unlabelled) into the model's
// per-CTA partial rows; *loss receives the mean cross-entropy
static int gnn_grad(dagrt_batch *b, dagrt_model *md, const int8_t *labels, float *loss) {
    dagrt_ctx *ctx = b->ctx;
    auto &G = b->gnn;
    int rc = gnn_prepare(b, true);
    if (rc) return rc;
    const size_t N = (size_t)b->total_nodes;
    int64_t nl = 0;
    for (size_t i = 0; i < N; i++) nl += labels[i] >= 0 && labels[i] < md->L;
    const float scale = nl ? 1.f / (float)nl : 0.f;
    cudaStream_t st = ctx->stream;
    if (N) CK(cudaMemcpyAsync(G.labels, labels, N, cudaMemcpyHostToDevice, st), "copy labels");
    if ((rc = gnn_forward(b, md))) return rc;
    const GnnGraph g = graph_of(b);
    CK(gnn_head(g, G.h[2], md->p + ParamLayout::Wh, md->p + ParamLayout::bh, md->L, G.labels, scale, G.logits, G.dlogits,
                G.dh[2], G.loss_part, ctx->n_sm, st), "head");
    CK(gnn_head_grad(g, G.h[2], G.dlogits, md->L, md->part, md->n_parts, st), "head gradient");
    // layer 3 and 2: weight gradients, then the gradient of the layer input
    for (int l = 2; l >= 1; l--) {
        CK(gnn_layer_bwd_dw(kHidden, l, g, G.h[l - 1], G.h[l], G.dh[l], md->part, md->n_parts, b->err, st), "dW");
        CK(gnn_layer_bwd_da(kHidden, g, G.h[l], G.dh[l], md->wb[l], G.da, b->err, ctx->n_sm, st), "dA");
        CK(gnn_agg_bwd(kHidden, g, G.da, G.dh[l - 1], ctx->n_sm, st), "aggregation backward");
    }
    CK(gnn_layer_bwd_dw(kFeat, 0, g, G.x, G.h[0], G.dh[0], md->part, md->n_parts, b->err, st), "dW");
    ctx->launches += 10;
    std::vector<float> lp(ctx->n_sm);
    CK(cudaMemcpyAsync(lp.data(), G.loss_part, 4 * ctx->n_sm, cudaMemcpyDeviceToHost, st), "copy loss");
    int32_t err = 0;
    CK(cudaMemcpyAsync(&err, b->err, sizeof err, cudaMemcpyDeviceToHost, st), "copy error word");
    CK(cudaStreamSynchronize(st), "synchronize");
    if (err) return fail(ctx, err, "a tensor-core wait did not complete in time");
    if (loss) {
        double s = 0;
        for (float x : lp) s += x;
        *loss = (float)s;
    }
    return DAGRT_OK;
}

extern "C" int dagrt_model_grad(dagrt_batch *b, dagrt_model *md, const int8_t *labels, float *grads, float *loss) {
    NvtxRange nvtx_range_("dagrt_model_grad");
    if (!b || !md || !labels) return b ? fail(b->ctx, DAGRT_E_INVAL, "dagrt_model_grad: NULL argument") : DAGRT_E_INVAL;
    dagrt_ctx *ctx = b->ctx;
    if (int rc = refuse_in_capture(ctx, true, "dagrt_model_grad")) return rc;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    int rc = gnn_grad(b, md, labels, loss);
    if (rc) return rc;
    if (grads) {  // fixed-order sum of the partial rows
        const int64_t n = ParamLayout::total;
        std::vector<float> part((size_t)n * md->n_parts);
        CK(cudaMemcpy(part.data(), md->part, part.size() * 4, cudaMemcpyDeviceToHost), "copy partials");
        for (int64_t i = 0; i < n; i++) {
            float s = 0.f;
            for (int c = 0; c < md->n_parts; c++) s += part[(size_t)c * n + i];
            grads[i] = s;
        }
    }
    return DAGRT_OK;
}

extern "C" int dagrt_train_step(dagrt_batch *b, dagrt_model *md, const int8_t *labels, float lr, float *loss) {
    NvtxRange nvtx_range_("dagrt_train_step");
    if (!b || !md || !labels) return b ? fail(b->ctx, DAGRT_E_INVAL, "dagrt_train_step: NULL argument") : DAGRT_E_INVAL;
    dagrt_ctx *ctx = b->ctx;
    if (int rc = refuse_in_capture(ctx, true, "dagrt_train_step")) return rc;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    int rc = gnn_grad(b, md, labels, loss);
    if (rc) return rc;
    md->step++;
    CK(gnn_adam(md->p, md->m, md->v, md->part, md->n_parts, ParamLayout::total, lr, 0.9f, 0.999f, 1e-8f, md->step,
                ctx->stream), "Adam");
    CK(gnn_refresh(md->p, md->wt, md->wb, ctx->stream), "refresh");
    ctx->launches += 2;
    return DAGRT_OK;
}

extern "C" int dagrt_propose(dagrt_batch *b, dagrt_model *md, int32_t k, int64_t *out_bound, uint8_t *cand_m,
                             int64_t *best_bound, int32_t *best_cand, uint8_t *best_m, uint32_t flags) {
    NvtxRange nvtx_range_("dagrt_propose");
    if (!b || !md) return b ? fail(b->ctx, DAGRT_E_INVAL, "dagrt_propose: model is NULL") : DAGRT_E_INVAL;
    dagrt_ctx *ctx = b->ctx;
    if (md->ctx != ctx) return fail(ctx, DAGRT_E_INVAL, "dagrt_propose: model of another context");
    if (k < 1 || k > 16) return fail(ctx, DAGRT_E_INVAL, "dagrt_propose: k must be in [1, 16]");
    if (flags & ~DAGRT_PTR_DEVICE) return fail(ctx, DAGRT_E_INVAL, "dagrt_propose: unknown flags 0x%x", flags);
    if (int rc = refuse_in_capture(ctx, !(flags & DAGRT_PTR_DEVICE), "dagrt_propose")) return rc;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    int rc = gnn_prepare(b, false);
    if (rc) return rc;
    if ((rc = gnn_forward(b, md))) return rc;
    auto &G = b->gnn;
    const GnnGraph g = graph_of(b);
    cudaStream_t st = ctx->stream;
    CK(gnn_head(g, G.h[2], md->p + ParamLayout::Wh, md->p + ParamLayout::bh, md->L, nullptr, 0.f, G.logits, nullptr,
                nullptr, nullptr, ctx->n_sm, st), "head");
    const Plan &pl = b->plan[DAGRT_VAR_PAPER];
    CK(gnn_topk(b->n_dags, b->node_off, G.logits, md->L, md->d_levels, k, pl.rows, pl.nrows, G.best_level, G.cand,
                kPropStride, ctx->n_sm, st), "top-k decode");
    const bool dev = (flags & DAGRT_PTR_DEVICE) != 0;
    const size_t nd = b->n_dags, nrow = (size_t)(2 * b->total_nodes), nc = (size_t)k + 1;
    // host outputs are staged in the scratch block: [out_bound | best_m]
    const size_t ob_bytes = (out_bound && !dev) ? (8 * nd * nc + 255) / 256 * 256 : 0;
    const size_t bm_bytes = (best_m && !dev) ? (nrow + 255) / 256 * 256 : 0;
    if (ob_bytes + bm_bytes) {
        int rc2 = ensure_tmp(b, ob_bytes + bm_bytes);
        if (rc2) return rc2;
    }
    // exact check of the candidates on the paper structure (Theorem 1, as dagrt_bound)
    BoundArgs a;
    std::memset(&a, 0, sizeof a);
    a.n_dags = b->n_dags;
    a.node_off = b->node_off;
    a.M = b->M;
    a.n_variants = 1;
    a.n_alloc = (int32_t)nc;
    a.stride = kPropStride;
    a.err = b->err;
    a.plan[0] = pl.rows;
    a.nrows[0] = pl.nrows;
    a.pflag[0] = pl.pflag;
    a.status[0] = pl.status;
    a.m_alloc = G.cand;
    a.out = out_bound ? (dev ? out_bound : (int64_t *)b->tmp) : nullptr;
    a.best_bound = dev && best_bound ? best_bound : G.bbest;
    a.best_cand = dev && best_cand ? best_cand : G.cbest;
    int nl = 0;
    CK(bound_launch(a, nullptr, ctx->n_sm, st, &nl), "exact check");
    ctx->launches += 2 + nl;  // head, top-k, exact check (forward counted apart)
    uint8_t *bm = best_m ? (dev ? best_m : (uint8_t *)b->tmp + ob_bytes) : nullptr;
    if (bm) {
        if (!dev && nrow) CK(cudaMemsetAsync(bm, 0, nrow, st), "clear best_m");
        CK(gnn_pick_column(b->n_dags, b->node_off, pl.nrows, a.best_cand, G.cand, kPropStride, bm, ctx->n_sm, st),
           "winning allocation");
        ctx->launches++;
    }
    if (cand_m && nrow)
        CK(cudaMemcpy2DAsync(cand_m, nc, G.cand, kPropStride, nc, nrow,
                             dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st), "copy candidates");
    if (dev) return DAGRT_OK;
    if (out_bound && nd) CK(cudaMemcpyAsync(out_bound, a.out, 8 * nd * nc, cudaMemcpyDeviceToHost, st), "copy bounds");
    if (best_bound && nd) CK(cudaMemcpyAsync(best_bound, a.best_bound, 8 * nd, cudaMemcpyDeviceToHost, st), "copy best");
    if (best_cand && nd) CK(cudaMemcpyAsync(best_cand, a.best_cand, 4 * nd, cudaMemcpyDeviceToHost, st), "copy best");
    if (best_m && nrow) CK(cudaMemcpyAsync(best_m, bm, nrow, cudaMemcpyDeviceToHost, st), "copy best_m");
    int32_t err = 0;
    CK(cudaMemcpyAsync(&err, b->err, sizeof err, cudaMemcpyDeviceToHost, st), "copy error word");
    CK(cudaStreamSynchronize(st), "synchronize");
    if (err) return fail(ctx, err, "a wait did not complete in time");
    return DAGRT_OK;
}

// ------------------------------------------------------------------ batching controls
extern "C" int dagrt_get_tuning(const dagrt_batch *b, dagrt_tuning *out) {
    if (!b || !out) return DAGRT_E_INVAL;
    *out = b->tune;
    return DAGRT_OK;
}

extern "C" int dagrt_set_tuning(dagrt_batch *b, const dagrt_tuning *t) {
    if (!b) return DAGRT_E_INVAL;
    dagrt_ctx *ctx = b->ctx;
    if (!t) return fail(ctx, DAGRT_E_INVAL, "dagrt_set_tuning: NULL");
    if (int rc = refuse_in_capture(ctx, true, "dagrt_set_tuning")) return rc;
    const int w = t->warp_max_v;
    if (w != 0 && w != 64 && w != 128 && w != 192 && w != 256)
        return fail(ctx, DAGRT_E_INVAL, "dagrt_set_tuning: warp_max_v must be 0, 64, 128, 192 or 256");
    if (t->chunk_rows < kMinChunkRows || t->chunk_rows > 256)
        return fail(ctx, DAGRT_E_INVAL, "dagrt_set_tuning: chunk_rows must be in [%d, 256]", kMinChunkRows);
    if (t->item_warps < 1 || t->item_warps > 8)
        return fail(ctx, DAGRT_E_INVAL, "dagrt_set_tuning: item_warps must be in [1, 8]");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    if (t->cta_smem < 0 || t->cta_smem > 4)
        return fail(ctx, DAGRT_E_INVAL, "dagrt_set_tuning: cta_smem must be in [0, 4]");
    const bool repart = t->warp_max_v != b->tune.warp_max_v || t->cta_smem != b->tune.cta_smem;
    b->tune = *t;
    if (repart) {
        CK(cudaStreamSynchronize(ctx->stream), "synchronize");  // the lists may be in use
        return partition_classes(b);
    }
    return DAGRT_OK;
}

namespace {
float median_of(std::vector<float> v) {
    std::sort(v.begin(), v.end());
    return v.empty() ? 0.f : v[v.size() / 2];
}
}  // namespace

// time `call` reps times after one warm-up (CUDA events on the context's stream)
template <class F>
static int time_call(dagrt_ctx *ctx, int reps, F call, float *ms) {
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0), "event");
    CK(cudaEventCreate(&e1), "event");
    std::vector<float> t;
    int rc = DAGRT_OK;
    for (int r = 0; r <= reps && rc == DAGRT_OK; r++) {
        cudaEventRecord(e0, ctx->stream);
        rc = call();
        cudaEventRecord(e1, ctx->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = cuda_fail(ctx, cudaGetLastError(), "time call");
        float x = 0.f;
        cudaEventElapsedTime(&x, e0, e1);
        if (r > 0) t.push_back(x);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = median_of(t);
    return rc;
}

extern "C" int dagrt_autotune_schedule(dagrt_batch *b, int32_t variant, int32_t reps, dagrt_tuning *chosen,
                                       float *best_ms) {
    NvtxRange nvtx_range_("dagrt_autotune_schedule");
    if (!b) return DAGRT_E_INVAL;
    dagrt_ctx *ctx = b->ctx;
    if (int rc = refuse_in_capture(ctx, true, "dagrt_autotune_schedule")) return rc;
    if (reps < 1) return fail(ctx, DAGRT_E_INVAL, "dagrt_autotune_schedule: reps < 1");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    dagrt_tuning best = b->tune;
    float bt = -1.f;
    for (int cfg = 0; cfg < 20; cfg++) {
        dagrt_tuning t = b->tune;
        t.warp_max_v = 64 * (1 + cfg % 4);
        t.cta_smem = cfg / 4;
        int rc = dagrt_set_tuning(b, &t);
        if (rc) return rc;
        dagrt_schedule_out o;
        std::memset(&o, 0, sizeof o);
        float ms = 0.f;
        rc = time_call(ctx, reps, [&]() { return dagrt_schedule(b, variant, &o, DAGRT_PTR_DEVICE); }, &ms);
        if (rc) return rc;
        if (bt < 0.f || ms < bt) {
            bt = ms;
            best = t;
        }
    }
    int rc = dagrt_set_tuning(b, &best);
    if (rc) return rc;
    if (chosen) *chosen = best;
    if (best_ms) *best_ms = bt;
    return DAGRT_OK;
}

extern "C" int dagrt_autotune_bound(dagrt_batch *b, int32_t n_variants, const int32_t *variant_ids, int32_t n_alloc,
                                    const uint8_t *m_alloc, int64_t cand_stride, int32_t reps, dagrt_tuning *chosen,
                                    float *best_ms) {
    NvtxRange nvtx_range_("dagrt_autotune_bound");
    if (!b) return DAGRT_E_INVAL;
    dagrt_ctx *ctx = b->ctx;
    if (int rc = refuse_in_capture(ctx, true, "dagrt_autotune_bound")) return rc;
    if (reps < 1) return fail(ctx, DAGRT_E_INVAL, "dagrt_autotune_bound: reps < 1");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    dagrt_tuning best = b->tune;
    float bt = -1.f;
    const bool tunable = n_alloc > 0 && n_alloc % 64 == 0;
    std::vector<std::pair<int, int>> grid;
    if (tunable) {
        for (int cr : {24, 32, 48, 64})
            for (int wp : {2, 4, 8}) grid.emplace_back(cr, wp);
    } else {
        grid.emplace_back(b->tune.chunk_rows, b->tune.item_warps);
    }
    for (auto &g : grid) {
        dagrt_tuning t = b->tune;
        t.chunk_rows = g.first;
        t.item_warps = g.second;
        int rc = dagrt_set_tuning(b, &t);
        if (rc) return rc;
        float ms = 0.f;
        rc = time_call(ctx, reps, [&]() {
            return dagrt_bound(b, n_variants, variant_ids, n_alloc, m_alloc, cand_stride, nullptr, nullptr, nullptr,
                               DAGRT_PTR_DEVICE);
        }, &ms);
        if (rc) return rc;
        if (bt < 0.f || ms < bt) {
            bt = ms;
            best = t;
        }
    }
    int rc = dagrt_set_tuning(b, &best);
    if (rc) return rc;
    if (chosen) *chosen = best;
    if (best_ms) *best_ms = bt;
    return DAGRT_OK;
}

// ------------------------------------------------------------------ CUDA graphs
struct dagrt_graph {
    dagrt_ctx *ctx = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t launches = 0;
};

extern "C" int dagrt_graph_begin(dagrt_ctx *ctx) {
    if (!ctx) return DAGRT_E_INVAL;
    if (ctx->capturing) return fail(ctx, DAGRT_E_INVAL, "dagrt_graph_begin: already capturing");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    CK(ensure_side_streams(ctx), "create side streams");  // not during capture
    // the legacy default stream cannot be captured: record on a private stream instead
    if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking), "create capture stream");
    CK(cudaStreamSynchronize(ctx->stream), "synchronize");
    CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeRelaxed), "begin capture");
    ctx->saved_stream = ctx->stream;
    ctx->stream = ctx->cap_stream;
    ctx->capturing = true;
    ctx->capture_launch0 = ctx->launches;
    return DAGRT_OK;
}

extern "C" int dagrt_graph_end(dagrt_ctx *ctx, dagrt_graph **out) {
    if (!ctx) return DAGRT_E_INVAL;
    if (!out) return fail(ctx, DAGRT_E_INVAL, "dagrt_graph_end: out is NULL");
    *out = nullptr;
    if (!ctx->capturing) return fail(ctx, DAGRT_E_INVAL, "dagrt_graph_end: not capturing");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &g);
    ctx->stream = ctx->saved_stream;
    ctx->capturing = false;
    const int64_t n = ctx->launches - ctx->capture_launch0;
    ctx->launches = ctx->capture_launch0;  // recorded, not run
    if (e != cudaSuccess) return cuda_fail(ctx, e, "end capture");
    cudaGraphExec_t x = nullptr;
    e = cudaGraphInstantiate(&x, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(ctx, e, "instantiate graph");
    }
    dagrt_graph *gr = new dagrt_graph();
    gr->ctx = ctx;
    gr->graph = g;
    gr->exec = x;
    gr->launches = n;
    *out = gr;
    ctx->live++;
    return DAGRT_OK;
}

extern "C" int dagrt_graph_launch(dagrt_graph *g) {
    NvtxRange nvtx_range_("dagrt_graph_launch");
    if (!g) return DAGRT_E_INVAL;
    dagrt_ctx *ctx = g->ctx;
    if (int rc = refuse_in_capture(ctx, true, "dagrt_graph_launch")) return rc;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    CK(cudaGraphLaunch(g->exec, ctx->stream), "launch graph");
    ctx->launches += g->launches;
    return DAGRT_OK;
}

extern "C" void dagrt_graph_free(dagrt_graph *g) {
    if (!g) return;
    cudaSetDevice(g->ctx->device);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    dagrt_ctx *ctx = g->ctx;
    delete g;
    ctx_unref(ctx);
}

// ------------------------------------------------------------------ failure detection
extern "C" int dagrt_selftest_wait(dagrt_ctx *ctx, uint32_t limit) {
    if (!ctx) return DAGRT_E_INVAL;
    if (int rc = refuse_in_capture(ctx, true, "dagrt_selftest_wait")) return rc;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    int32_t *word = nullptr;
    CK(ctx->pool.get((void **)&word, 256), "allocate error word");
    int32_t h = 0;
    cudaError_t e = cudaMemsetAsync(word, 0, sizeof(int32_t), ctx->stream);
    if (e == cudaSuccess) e = bound_selftest_wait(limit, word, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, word, sizeof h, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    ctx->pool.put(word, 256);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "self-test wait");
    ctx->launches++;
    if (h) return fail(ctx, h, "dagrt_selftest_wait: the wait gave up after %u polls (as it should)", limit);
    return DAGRT_OK;
}
