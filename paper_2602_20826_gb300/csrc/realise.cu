// realise.cu -- a schedule run on this GPU as a CUDA graph, and its makespan measured.
//
// The case-study set-up of the Evaluation section, on the GB300: every part of the schedule
// (a node's last part or a parallel segment) becomes one kernel node of a CUDA graph whose
// grid is the part's SM count m, and whose CTAs each reserve more than half of an SM's
// shared memory, so that a CTA holds an SM to itself and a kernel of m CTAs holds m SMs.
// A load is emulated by time, as the paper emulates it by iteration counts: every CTA of a
// part with load C^ and parallel fraction f = k/64 on m SMs runs for C^ ((1 - f) + f / m)
// ticks (Amdahl's law; Eq.1 without rounding). The GPU is narrowed to the model's M SMs
// by filler CTAs that hold the other SMs for the length of a replay. The graph's edges are
// the DAG's edges (a node's parts wait for its predecessors' last parts; a node's segment
// runs before its residual part) plus, by mode, the schedule's extra edges of Alg.2 or a
// barrier between consecutive groups. The measured makespan can then be set against
// Theorem 1's bound in ticks.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <set>
#include <thread>
#include <vector>

#include "dagrt.h"
#include "dagrt_internal.cuh"

namespace dagrt {
namespace {

constexpr int kRealiseSmem = 120 * 1024;  // > half of an SM's shared memory: one CTA per SM

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// One emulated kernel: every CTA keeps its SM for `ns` nanoseconds. The wait ends when the
// timer has advanced by ns, or after an iteration limit well past that (a timer that
// stopped would otherwise hold the SM): then the error word is set. A filler CTA first
// counts itself in `started` (host-mapped memory), so that the host can launch the graph
// once every filler holds its SM.
__global__ void __launch_bounds__(32) k_emulate(uint64_t ns, int32_t *err, int32_t *started) {
    extern __shared__ unsigned char reserve[];  // reserved, not used: one CTA per SM
    if (threadIdx.x != 0) return;
    if (started) {
        atomicAdd_system(started, 1);
        __threadfence_system();
    }
    const uint64_t t0 = global_ns();
    const uint64_t limit = ns + (1ull << 20);  // each poll takes far more than a nanosecond
    for (uint64_t i = 0; i < limit; i++)
        if (global_ns() - t0 >= ns) return;
    atomicExch(err, DAGRT_E_TIMEOUT);
}

}  // namespace
}  // namespace dagrt

using namespace dagrt;

namespace {
struct GraphGuard {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t x = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int32_t *err = nullptr;
    int32_t *started = nullptr;  // host-mapped counter of filler CTAs that hold their SM
    dagrt_batch *b = nullptr;
    ~GraphGuard() {
        if (started) cudaFreeHost(started);
        if (x) cudaGraphExecDestroy(x);
        if (g) cudaGraphDestroy(g);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (err) cudaFree(err);
        if (b) dagrt_batch_free(b);
    }
};
}  // namespace

extern "C" int dagrt_realise(dagrt_ctx *ctx, int32_t V, const int32_t *row_ptr, const int32_t *col,
                             const int64_t *wcet, const uint8_t *k64, int32_t M, int32_t variant, int32_t mode,
                             float tick_us, int32_t reps, float *makespan_us, int64_t *bound) {
    if (!ctx) return DAGRT_E_INVAL;
    if (V < 1 || !row_ptr || !wcet || !k64 || !makespan_us || reps < 1 || !(tick_us > 0.f) || tick_us > 1e5f ||
        (mode != DAGRT_REALISE_BARRIER && mode != DAGRT_REALISE_EDGES && mode != DAGRT_REALISE_GREEDY))
        return DAGRT_E_INVAL;
    int dev = 0, n_sm = 0, optin = 0;
    if (dagrt_sync(ctx) != DAGRT_OK || cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return DAGRT_E_DEVICE;
    if (M < 1 || M > n_sm || optin < kRealiseSmem) return DAGRT_E_INVAL;  // m SMs must exist
    const int64_t E = row_ptr[V];
    if (E > 0 && !col) return DAGRT_E_INVAL;
    GraphGuard gg;
    const int64_t node_off[2] = {0, V}, edge_off[2] = {0, E};
    int rc = dagrt_load_csr(ctx, 1, node_off, edge_off, row_ptr, col, wcet, k64, M, 0, &gg.b);
    if (rc) return rc;

    // the parts to run: (owner node, load, k, m, group), and their order constraints
    std::vector<int32_t> owner, grp, m;
    std::vector<int64_t> load;
    std::vector<int32_t> kk;
    std::vector<int32_t> last(V, -1);      // part that finishes node v
    std::vector<std::vector<int32_t>> segs(V);
    std::vector<std::pair<int32_t, int32_t>> extra;
    int64_t the_bound = 0;
    dagrt_schedule_out o;
    std::memset(&o, 0, sizeof o);
    int32_t status = 0, n_rows = 0, n_seg = 0;
    int64_t n_extra = 0, base[3] = {0, 0, 0};
    std::vector<int32_t> row_id(2 * V), row_group(2 * V), row_m0(2 * V), seg_parent(V), seg_m(V), seg_group(V);
    std::vector<int64_t> row_load(2 * V), seg_load(V);
    o.bound = &the_bound;
    o.status = &status;
    o.n_rows = &n_rows;
    o.n_seg = &n_seg;
    o.n_extra = &n_extra;
    o.greedy = &base[0];
    o.row_id = row_id.data();
    o.row_group = row_group.data();
    o.row_m0 = row_m0.data();
    o.row_load = row_load.data();
    o.seg_parent = seg_parent.data();
    o.seg_load = seg_load.data();
    o.seg_m = seg_m.data();
    o.seg_group = seg_group.data();
    if ((rc = dagrt_schedule(gg.b, mode == DAGRT_REALISE_GREEDY ? DAGRT_VAR_PAPER : variant, &o, 0))) return rc;
    if (mode == DAGRT_REALISE_EDGES && n_extra > 0) {  // second pass for the extra edges
        std::vector<int64_t> eoff = {0, n_extra};
        std::vector<int32_t> es(n_extra), ed(n_extra);
        dagrt_schedule_out o2;
        std::memset(&o2, 0, sizeof o2);
        o2.extra_off = eoff.data();
        o2.extra_src = es.data();
        o2.extra_dst = ed.data();
        if ((rc = dagrt_schedule(gg.b, variant, &o2, 0))) return rc;
        for (int64_t i = 0; i < n_extra; i++) extra.emplace_back(es[i], ed[i]);
    }
    if (mode == DAGRT_REALISE_GREEDY) {  // every kernel on min(C^, M) SMs, DAG edges only
        for (int v = 0; v < V; v++) {
            owner.push_back(v);
            load.push_back(wcet[v]);
            kk.push_back(k64[v]);
            m.push_back((int32_t)(wcet[v] < M ? wcet[v] : M));
            grp.push_back(0);
            last[v] = v;
        }
        the_bound = base[0];
    } else {
        for (int r = 0; r < n_rows; r++) {
            const int id = row_id[r];
            const int ow = id < V ? id : seg_parent[id - V];
            owner.push_back(ow);
            load.push_back(row_load[r]);
            kk.push_back(k64[ow]);
            m.push_back(row_m0[r]);
            grp.push_back(row_group[r]);
            if (id < V)
                last[id] = r;
            else
                segs[ow].push_back(r);
        }
    }
    const int n_parts = (int)owner.size();
    for (int i = 0; i < n_parts; i++)
        if (m[i] < 1 || m[i] > n_sm) return DAGRT_E_INVAL;

    // the graph
    if (cudaFuncSetAttribute(k_emulate, cudaFuncAttributeMaxDynamicSharedMemorySize, kRealiseSmem) != cudaSuccess ||
        cudaMalloc(&gg.err, sizeof(int32_t)) != cudaSuccess || cudaMemset(gg.err, 0, sizeof(int32_t)) != cudaSuccess ||
        cudaGraphCreate(&gg.g, 0) != cudaSuccess)
        return DAGRT_E_DEVICE;
    std::vector<cudaGraphNode_t> node(n_parts);
    std::vector<uint64_t> ns(n_parts);
    std::vector<void *> args(3 * n_parts);
    int32_t *no_count = nullptr;
    for (int i = 0; i < n_parts; i++) {
        const double f = kk[i] / 64.0;
        ns[i] = (uint64_t)std::llround(1e3 * tick_us * (double)load[i] * ((1.0 - f) + f / m[i]));
        args[3 * i] = &ns[i];
        args[3 * i + 1] = &gg.err;
        args[3 * i + 2] = &no_count;
        cudaKernelNodeParams kp;
        std::memset(&kp, 0, sizeof kp);
        kp.func = (void *)k_emulate;
        kp.gridDim = dim3((unsigned)m[i]);
        kp.blockDim = dim3(32);
        kp.sharedMemBytes = kRealiseSmem;
        kp.kernelParams = &args[3 * i];
        if (cudaGraphAddKernelNode(&node[i], gg.g, nullptr, 0, &kp) != cudaSuccess) return DAGRT_E_DEVICE;
    }
    std::vector<cudaGraphNode_t> from, to;
    std::set<std::pair<int, int>> seen;  // a graph may hold each dependency only once
    auto dep = [&](int a, int b) {
        if (a >= 0 && b >= 0 && a != b && seen.emplace(a, b).second) {
            from.push_back(node[a]);
            to.push_back(node[b]);
        }
    };
    for (int u = 0; u < V; u++)
        for (int64_t q = row_ptr[u]; q < row_ptr[u + 1]; q++) {
            const int v = col[q];
            dep(last[u], last[v]);
            for (int s : segs[v]) dep(last[u], s);
        }
    for (int v = 0; v < V; v++)
        for (int s : segs[v]) dep(s, last[v]);
    for (auto &x : extra) {
        const int a = x.first < V ? last[x.first] : (int)(std::find(row_id.begin(), row_id.begin() + n_rows, x.first) - row_id.begin());
        const int b = x.second < V ? last[x.second] : (int)(std::find(row_id.begin(), row_id.begin() + n_rows, x.second) - row_id.begin());
        dep(a, b);
    }
    if (mode == DAGRT_REALISE_BARRIER) {  // every part of group j before every part of group j + 1
        int gmax = 0;
        for (int g : grp) gmax = g > gmax ? g : gmax;
        std::vector<cudaGraphNode_t> bar(gmax + 1);
        for (int j = 0; j <= gmax; j++)
            if (cudaGraphAddEmptyNode(&bar[j], gg.g, nullptr, 0) != cudaSuccess) return DAGRT_E_DEVICE;
        for (int i = 0; i < n_parts; i++) {
            from.push_back(node[i]);
            to.push_back(bar[grp[i]]);
            if (grp[i] > 0) {
                from.push_back(bar[grp[i] - 1]);
                to.push_back(node[i]);
            }
        }
        for (int j = 1; j <= gmax; j++) {  // a group of parts that all ran earlier still orders
            from.push_back(bar[j - 1]);
            to.push_back(bar[j]);
        }
    }
    if (!from.empty() && cudaGraphAddDependencies(gg.g, from.data(), to.data(), nullptr, from.size()) != cudaSuccess)
        return DAGRT_E_DEVICE;
    // an M-SM GPU on this n_sm-SM one: before each replay, n_sm - M filler CTAs (one per SM,
    // each holding its SM for a fixed time longer than the replay can take) take the other
    // SMs, so that the graph's kernels find M free SMs. The host launches the graph once
    // every filler has counted itself in (a bounded poll of host-mapped memory); nothing on
    // the device waits on anything: the fillers end by their own clock.
    cudaStream_t st = nullptr, fill = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return DAGRT_E_DEVICE;
    if (cudaStreamCreateWithFlags(&fill, cudaStreamNonBlocking) != cudaSuccess) {
        cudaStreamDestroy(st);
        return DAGRT_E_DEVICE;
    }
    const uint64_t fill_ns = (uint64_t)(2.0 * 1e3 * tick_us * (double)(the_bound > 0 ? the_bound : 1)) + 2000000ull;
    int out = DAGRT_OK;
    int32_t *d_started = nullptr;
    if (n_sm > M && (cudaHostAlloc(&gg.started, sizeof(int32_t), cudaHostAllocMapped) != cudaSuccess ||
                     cudaHostGetDevicePointer((void **)&d_started, gg.started, 0) != cudaSuccess))
        out = DAGRT_E_DEVICE;
    if (out == DAGRT_OK && (cudaGraphInstantiate(&gg.x, gg.g, 0) != cudaSuccess || cudaEventCreate(&gg.e0) != cudaSuccess ||
        cudaEventCreate(&gg.e1) != cudaSuccess || cudaGraphUpload(gg.x, st) != cudaSuccess))
        out = DAGRT_E_DEVICE;
    for (int r = -1; r < reps && out == DAGRT_OK; r++) {  // one warm-up replay
        if (n_sm > M) {
            *(volatile int32_t *)gg.started = 0;
            k_emulate<<<n_sm - M, 32, kRealiseSmem, fill>>>(fill_ns, gg.err, d_started);
            if (cudaGetLastError() != cudaSuccess) {
                out = DAGRT_E_DEVICE;
                break;
            }
            // wait until the fillers hold their SMs (at most a quarter of their time)
            const auto t0 = std::chrono::steady_clock::now();
            while (*(volatile int32_t *)gg.started < n_sm - M &&
                   std::chrono::steady_clock::now() - t0 < std::chrono::nanoseconds(fill_ns / 4))
                std::this_thread::yield();
            if (*(volatile int32_t *)gg.started < n_sm - M) {
                cudaStreamSynchronize(fill);
                out = DAGRT_E_TIMEOUT;
                break;
            }
        }
        if (cudaEventRecord(gg.e0, st) != cudaSuccess || cudaGraphLaunch(gg.x, st) != cudaSuccess ||
            cudaEventRecord(gg.e1, st) != cudaSuccess || cudaEventSynchronize(gg.e1) != cudaSuccess ||
            cudaStreamSynchronize(fill) != cudaSuccess) {
            out = DAGRT_E_DEVICE;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, gg.e0, gg.e1);
        if (r >= 0) makespan_us[r] = 1e3f * ms;
        if (n_sm > M && 1e3 * (double)ms + 1e-3 * (double)(fill_ns / 4) > 1e-3 * (double)fill_ns)
            out = DAGRT_E_INTERNAL;  // may have outlived the fillers
    }
    int32_t err = 0;
    if (out == DAGRT_OK && cudaMemcpy(&err, gg.err, sizeof err, cudaMemcpyDeviceToHost) != cudaSuccess) out = DAGRT_E_DEVICE;
    cudaStreamSynchronize(st);
    cudaStreamSynchronize(fill);
    cudaStreamDestroy(st);
    cudaStreamDestroy(fill);
    if (out == DAGRT_OK && err) out = err;
    if (bound) *bound = the_bound;
    return out;
}
