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

#include "dagrt.h"
#include "bound.cuh"
#include "sched.cuh"

using namespace dagrt;

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
    int64_t launches = 0;
    DevicePool pool;
};

namespace {

constexpr int kNumWarpClasses = 4;
constexpr int kWarpClassCap[kNumWarpClasses] = {64, 128, 192, 256};

struct Plan {
    bool valid = false;
    uint4 *rows = nullptr;
    int32_t *nrows = nullptr;
    int32_t *pflag = nullptr;
    int32_t *status = nullptr;
    int64_t *bound = nullptr;
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
    std::vector<int64_t> h_node_off;
    // size classes: warp classes then the CTA class, lists concatenated
    int32_t *lists = nullptr;
    int32_t *counters = nullptr;
    int class_off[kNumWarpClasses + 2] = {0};
    int max_v = 0, big_vcap = 0, big_ecap = 0, big_grid = 0;
    unsigned char *gws = nullptr;
    int64_t gws_stride = 0;
    Plan plan[DAGRT_N_VARIANTS];
    int32_t *err = nullptr;  // device error word (bounded waits that gave up)
    // scratch for candidate evaluation
    void *tmp = nullptr;
    size_t tmp_cap = 0;
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
    ctx->stream = (cudaStream_t)cuda_stream;
    return DAGRT_OK;
}

int dagrt_sync(dagrt_ctx *ctx) {
    if (!ctx) return DAGRT_E_INVAL;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    CK(cudaStreamSynchronize(ctx->stream), "stream synchronize");
    return DAGRT_OK;
}

void dagrt_destroy(dagrt_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    ctx->pool.release_all();
    delete ctx;
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
    b->ctx->n_batches--;
    delete b;
}

int dagrt_load_csr(dagrt_ctx *ctx, int32_t n_dags, const int64_t *node_off, const int64_t *edge_off,
                   const int32_t *row_ptr, const int32_t *col, const int64_t *wcet, const uint8_t *k64,
                   int32_t M, uint32_t flags, dagrt_batch **out) {
    if (!ctx) return DAGRT_E_INVAL;
    if (!out) return fail(ctx, DAGRT_E_INVAL, "dagrt_load_csr: out is NULL");
    *out = nullptr;
    if (flags & ~DAGRT_PTR_DEVICE) return fail(ctx, DAGRT_E_INVAL, "dagrt_load_csr: unknown flags 0x%x", flags);
    if (n_dags < 0) return fail(ctx, DAGRT_E_INVAL, "dagrt_load_csr: n_dags < 0");
    if (M < 1 || M > DAGRT_MAX_M) return fail(ctx, DAGRT_E_INVAL, "dagrt_load_csr: M=%d outside [1, %d]", M, DAGRT_MAX_M);
    if (!node_off || !edge_off) return fail(ctx, DAGRT_E_INVAL, "dagrt_load_csr: NULL offsets");
    const bool dev = (flags & DAGRT_PTR_DEVICE) != 0;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");

    std::vector<int64_t> hn(n_dags + 1), he(n_dags + 1);
    if (dev) {
        CK(cudaMemcpyAsync(hn.data(), node_off, sizeof(int64_t) * (n_dags + 1), cudaMemcpyDeviceToHost, ctx->stream),
           "copy node_off");
        CK(cudaMemcpyAsync(he.data(), edge_off, sizeof(int64_t) * (n_dags + 1), cudaMemcpyDeviceToHost, ctx->stream),
           "copy edge_off");
        CK(cudaStreamSynchronize(ctx->stream), "stream synchronize");
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
    b->h_node_off = hn;
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
        if ((e = cudaMemcpyAsync(dn, hn.data(), 8 * (n_dags + 1), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(de, he.data(), 8 * (n_dags + 1), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
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

    // size classes, each ordered by descending node count (longest work first)
    std::vector<int32_t> lists(n_dags);
    {
        std::vector<std::vector<int32_t>> cls(kNumWarpClasses + 1);
        std::vector<int32_t> order(n_dags);
        std::vector<int32_t> cnt(max_v + 2, 0);  // counting sort by descending V
        for (int d = 0; d < n_dags; d++) cnt[max_v - (int)(hn[d + 1] - hn[d])]++;
        for (int i = 1; i < (int)cnt.size(); i++) cnt[i] += cnt[i - 1];
        for (int d = n_dags - 1; d >= 0; d--) order[--cnt[max_v - (int)(hn[d + 1] - hn[d])]] = d;
        int big_v = 0;
        int64_t big_e = 0;
        for (int d : order) {
            const int v = (int)(hn[d + 1] - hn[d]);
            const int64_t ed = he[d + 1] - he[d];
            int c = 0;  // the smallest class whose workspace holds V nodes and E edges
            while (c < kNumWarpClasses && (v > kWarpClassCap[c] || ed > (int64_t)kEdgesPerNode * kWarpClassCap[c])) c++;
            cls[c].push_back(d);
            if (c == kNumWarpClasses) {
                big_v = std::max(big_v, v);
                big_e = std::max(big_e, ed);
            }
        }
        b->big_ecap = (int)big_e;
        int off = 0;
        for (int c = 0; c <= kNumWarpClasses; c++) {
            b->class_off[c] = off;
            std::copy(cls[c].begin(), cls[c].end(), lists.begin() + off);
            off += (int)cls[c].size();
        }
        b->class_off[kNumWarpClasses + 1] = off;
        b->big_vcap = big_v;
    }
    if ((e = batch_alloc(b, &b->lists, n_dags)) != cudaSuccess ||
        (e = batch_alloc(b, &b->counters, 8)) != cudaSuccess || (e = batch_alloc(b, &b->err, 1)) != cudaSuccess ||
        (e = cudaMemsetAsync(b->err, 0, sizeof(int32_t), ctx->stream)) != cudaSuccess)
        return bail(cuda_fail(ctx, e, "allocate class lists"));
    if (n_dags > 0 &&
        (e = cudaMemcpyAsync(b->lists, lists.data(), 4 * n_dags, cudaMemcpyHostToDevice, ctx->stream)) != cudaSuccess)
        return bail(cuda_fail(ctx, e, "copy class lists"));
    const int n_big = b->class_off[kNumWarpClasses + 1] - b->class_off[kNumWarpClasses];
    if (n_big > 0) {
        b->big_grid = std::min(sched_cta_grid(ctx->n_sm), n_big);
        b->gws_stride = sched_ws_bytes(b->big_vcap, b->big_ecap);
        unsigned char *g;
        if ((e = batch_alloc(b, &g, (size_t)b->gws_stride * b->big_grid)) != cudaSuccess)
            return bail(cuda_fail(ctx, e, "allocate large-DAG workspace"));
        b->gws = g;
    }
    // host copies must be complete before the caller may reuse its buffers
    if (!dev && (e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) return bail(cuda_fail(ctx, e, "synchronize"));
    ctx->n_batches++;
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

static int ensure_tmp(dagrt_batch *b, size_t bytes) {
    dagrt_ctx *ctx = b->ctx;
    if (b->tmp_cap >= bytes) return DAGRT_OK;
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
    if (!b) return DAGRT_E_INVAL;
    dagrt_ctx *ctx = b->ctx;
    if (variant < 0 || variant >= DAGRT_N_VARIANTS)
        return fail(ctx, DAGRT_E_INVAL, "dagrt_schedule: unknown variant %d", variant);
    if (flags & ~DAGRT_PTR_DEVICE) return fail(ctx, DAGRT_E_INVAL, "dagrt_schedule: unknown flags 0x%x", flags);
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
    a.nrows = p.nrows;
    a.pflag = p.pflag;
    a.plan = p.rows;
    a.o = dv;
    if (nd > 0) {
        CK(cudaMemsetAsync(b->counters, 0, 8 * sizeof(int32_t), ctx->stream), "reset counters");
        for (int c = 0; c < kNumWarpClasses; c++) {
            const int n = b->class_off[c + 1] - b->class_off[c];
            if (n == 0) continue;
            a.list = b->lists + b->class_off[c];
            a.n_list = n;
            a.counter = b->counters + c;
            CK(sched_launch_warp(kWarpClassCap[c], a, ctx->n_sm, ctx->stream), "launch scheduler (warp teams)");
            ctx->launches++;
        }
        const int nbig = b->class_off[kNumWarpClasses + 1] - b->class_off[kNumWarpClasses];
        if (nbig > 0) {
            a.list = b->lists + b->class_off[kNumWarpClasses];
            a.n_list = nbig;
            a.counter = b->counters + kNumWarpClasses;
            a.gws = b->gws;
            a.gws_stride = b->gws_stride;
            a.vcap = b->big_vcap;
            a.ecap = b->big_ecap;
            CK(sched_launch_cta(a, b->big_grid, ctx->stream), "launch scheduler (CTA teams)");
            ctx->launches++;
        }
    }
    p.valid = true;
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

// ------------------------------------------------------------------ candidate bounds
extern "C" int dagrt_bound(dagrt_batch *b, int32_t n_variants, const int32_t *variant_ids, int32_t n_alloc,
                           const uint8_t *m_alloc, int64_t cand_stride, int64_t *out_bound, int64_t *best_bound,
                           int32_t *best_cand, uint32_t flags) {
    if (!b) return DAGRT_E_INVAL;
    dagrt_ctx *ctx = b->ctx;
    if (flags & ~DAGRT_PTR_DEVICE) return fail(ctx, DAGRT_E_INVAL, "dagrt_bound: unknown flags 0x%x", flags);
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
    CK(bound_launch(a, ctx->n_sm, ctx->stream), "launch bound kernel");
    if (nd) ctx->launches++;
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
    if (!b) return DAGRT_E_INVAL;
    dagrt_ctx *ctx = b->ctx;
    if (!cfg) return fail(ctx, DAGRT_E_INVAL, "dagrt_search: cfg is NULL");
    if (flags & ~DAGRT_PTR_DEVICE) return fail(ctx, DAGRT_E_INVAL, "dagrt_search: unknown flags 0x%x", flags);
    if (cfg->n_variants < 1 || cfg->n_variants > kMaxVariantsPerCall || !cfg->variant_ids)
        return fail(ctx, DAGRT_E_INVAL, "dagrt_search: n_variants must be in [1, %d]", kMaxVariantsPerCall);
    if (cfg->n_alloc < 1 || (int64_t)cfg->n_variants * cfg->n_alloc > (1 << 20))
        return fail(ctx, DAGRT_E_INVAL, "dagrt_search: need 1 <= n_alloc and n_variants * n_alloc <= 2^20");
    if (cfg->n_levels < 1 || cfg->n_levels > 16 || !cfg->levels)
        return fail(ctx, DAGRT_E_INVAL, "dagrt_search: n_levels must be in [1, 16]");
    for (int i = 0; i < cfg->n_levels; i++)
        if (cfg->levels[i] < 1) return fail(ctx, DAGRT_E_INVAL, "dagrt_search: level %d is 0", i);
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
    CK(bound_launch(a, ctx->n_sm, ctx->stream), "launch search kernel");
    if (nd) ctx->launches++;
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
