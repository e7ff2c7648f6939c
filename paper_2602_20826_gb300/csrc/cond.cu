// cond.cu -- conditional DAGs: the bound over every realisation, in one batched launch.
//
// The paper leaves conditional DAGs to future work. Here a conditional node takes exactly
// one of its out-edges per job (the branch its outcome selects). A node runs when it is a
// source, or when one of its in-edges is active; an edge is active when its tail runs and
// is either not conditional or took that edge. A realisation -- one choice per conditional
// node -- is then a plain DAG (the running nodes, renumbered in increasing order, with the
// active edges), and two bounds follow from Theorem 1:
//   adaptive: the largest bound over the realisations, each scheduled by Alg.1 + Alg.2 on
//             its own (the schedule picked when the job's outcomes are known at release);
//   fixed:    the bound of the whole DAG with every branch present (one schedule for every
//             job; a branch not taken runs for no time, within its C, so the bound holds by
//             the sustainability of Theorem 1).
// The host enumerates the realisations (choices in mixed radix, the first conditional node
// varying fastest; a realisation equal to an earlier one is dropped) into one batch, the
// scheduler bounds all of them in one dagrt_schedule call, and a segmented-max kernel takes
// the worst realisation of each conditional DAG on the device.
#include <cstring>
#include <set>
#include <string>
#include <vector>

#include "dagrt.h"
#include "dagrt_internal.cuh"

namespace dagrt {
namespace {

// per conditional DAG: the largest bound over its realisations [off[c], off[c+1]) and the
// first realisation that attains it; -1 where a realisation failed
__global__ void k_segmax(int32_t n, const int64_t *off, const int64_t *bound, const int32_t *status,
                         int64_t *out_bound, int32_t *out_arg) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < n; c += warps) {
        int64_t best = -1;
        int32_t arg = -1;
        bool bad = false;
        for (int64_t r = off[c] + lane; r < off[c + 1]; r += 32) {
            bad |= status[r] != DAGRT_OK;
            const int64_t b = bound[r];
            const int32_t i = (int32_t)(r - off[c]);
            if (b > best || (b == best && i < arg)) {
                best = b;
                arg = i;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const int64_t ob = __shfl_xor_sync(FULL, best, o);
            const int32_t oa = __shfl_xor_sync(FULL, arg, o);
            if (ob > best || (ob == best && oa >= 0 && (arg < 0 || oa < arg))) {
                best = ob;
                arg = oa;
            }
        }
        bad = __any_sync(FULL, bad);
        if (lane == 0) {
            out_bound[c] = bad ? -1 : best;
            out_arg[c] = bad ? -1 : arg;
        }
    }
}

}  // namespace
}  // namespace dagrt

using namespace dagrt;

extern "C" int dagrt_cond_bound(dagrt_ctx *ctx, int32_t n_dags, const int64_t *node_off, const int64_t *edge_off,
                                const int32_t *row_ptr, const int32_t *col, const int64_t *wcet, const uint8_t *k64,
                                const uint8_t *cond, int32_t M, int32_t variant, int32_t max_real,
                                int64_t *adaptive, int64_t *fixed, int32_t *worst_real, int32_t *n_real) {
    if (!ctx) return DAGRT_E_INVAL;
    if (n_dags < 0 || !node_off || !edge_off || max_real < 1 || max_real > (1 << 16)) return DAGRT_E_INVAL;
    if (n_dags == 0) return DAGRT_OK;
    if (!row_ptr || !wcet || !k64 || !cond || !adaptive) return DAGRT_E_INVAL;
    if (node_off[0] != 0 || edge_off[0] != 0) return DAGRT_E_INVAL;
    for (int d = 0; d < n_dags; d++) {
        const int64_t V = node_off[d + 1] - node_off[d], E = edge_off[d + 1] - edge_off[d];
        if (V < 0 || E < 0 || V > DAGRT_MAX_V || E > DAGRT_MAX_E) return DAGRT_E_INVAL;
        const int32_t *rp = row_ptr + node_off[d] + d;
        if (rp[0] != 0 || rp[V] != E) return DAGRT_E_INVAL;
        for (int64_t v = 0; v < V; v++)
            if (rp[v + 1] < rp[v]) return DAGRT_E_INVAL;
    }
    if (edge_off[n_dags] > 0 && !col) return DAGRT_E_INVAL;

    // the expanded batch: the realisations of each conditional DAG in turn (roff), then the
    // whole DAGs
    std::vector<int64_t> xn = {0}, xe = {0}, roff = {0};
    std::vector<int32_t> xrp, xcol;
    std::vector<int64_t> xw;
    std::vector<uint8_t> xk;
    std::vector<int32_t> counts(n_dags);
    auto append = [&](int d, const std::vector<char> &run, const std::vector<char> &act) {  // one DAG
        const int64_t n0 = node_off[d], V = node_off[d + 1] - n0;
        const int32_t *rp = row_ptr + n0 + d;
        const int32_t *cl = col + edge_off[d];
        std::vector<int32_t> id(V, -1);
        int32_t nv = 0;
        for (int64_t v = 0; v < V; v++)
            if (run[v]) id[v] = nv++;
        int64_t ne = 0;
        xrp.push_back(0);
        for (int64_t v = 0; v < V; v++) {
            if (!run[v]) continue;
            for (int32_t e = rp[v]; e < rp[v + 1]; e++)
                if (act[e]) {
                    xcol.push_back(id[cl[e]]);
                    ne++;
                }
            xrp.push_back((int32_t)ne);
            xw.push_back(wcet[n0 + v]);
            xk.push_back(k64[n0 + v]);
        }
        xn.push_back(xn.back() + nv);
        xe.push_back(xe.back() + ne);
    };
    for (int d = 0; d < n_dags; d++) {
        const int64_t n0 = node_off[d], V = node_off[d + 1] - n0;
        const int32_t *rp = row_ptr + n0 + d;
        const int32_t *cl = col ? col + edge_off[d] : nullptr;
        const int64_t E = rp[V];
        std::vector<int32_t> conds;
        for (int64_t v = 0; v < V; v++)
            if (cond[n0 + v] && rp[v + 1] > rp[v]) conds.push_back((int32_t)v);
        // topological order of the whole DAG (Kahn), to propagate "runs" forward
        std::vector<int32_t> indeg(V, 0), order;
        for (int64_t e = 0; e < E; e++) {
            if (cl[e] < 0 || cl[e] >= V) return DAGRT_E_RANGE;
            indeg[cl[e]]++;
        }
        std::vector<int32_t> cnt = indeg;
        for (int64_t v = 0; v < V; v++)
            if (!cnt[v]) order.push_back((int32_t)v);
        for (size_t i = 0; i < order.size(); i++)
            for (int32_t e = rp[order[i]]; e < rp[order[i] + 1]; e++)
                if (--cnt[cl[e]] == 0) order.push_back(cl[e]);
        if ((int64_t)order.size() != V) return DAGRT_E_CYCLE;
        int64_t combos = 1;  // choice tuples to enumerate (many may give the same realisation)
        for (int32_t c : conds) {
            combos *= rp[c + 1] - rp[c];
            if (combos > (1ll << 20)) return DAGRT_E_CAP;
        }
        std::set<std::string> seen;
        std::vector<int32_t> choice(conds.size(), 0);
        int32_t nr = 0;
        for (int64_t t = 0; t < combos; t++) {
            std::vector<char> run(V, 0), act(E, 0);
            for (int32_t u : order) {
                if (indeg[u] == 0) run[u] = 1;
                if (!run[u]) continue;
                int32_t pick = -1;
                for (size_t i = 0; i < conds.size(); i++)
                    if (conds[i] == u) pick = rp[u] + choice[i];
                for (int32_t e = rp[u]; e < rp[u + 1]; e++)
                    if (pick < 0 || e == pick) {
                        act[e] = 1;
                        run[cl[e]] = 1;
                    }
            }
            std::string key(act.begin(), act.end());
            key.append(run.begin(), run.end());
            if (seen.insert(key).second) {
                if (++nr > max_real) return DAGRT_E_CAP;
                append(d, run, act);
            }
            for (size_t i = 0; i < conds.size(); i++) {  // next choice, first node fastest
                if (++choice[i] < rp[conds[i] + 1] - rp[conds[i]]) break;
                choice[i] = 0;
            }
        }
        counts[d] = nr;
        roff.push_back(roff.back() + nr);
    }
    // the whole DAGs (every branch present) after all realisations: the fixed bounds
    const int64_t n_real_all = roff.back();
    for (int d = 0; d < n_dags; d++) {
        const int64_t V = node_off[d + 1] - node_off[d], E = edge_off[d + 1] - edge_off[d];
        append(d, std::vector<char>(V, 1), std::vector<char>(E, 1));
    }
    const int32_t nx = (int32_t)(xn.size() - 1);
    dagrt_batch *b = nullptr;
    int rc = dagrt_load_csr(ctx, nx, xn.data(), xe.data(), xrp.data(), xcol.empty() ? nullptr : xcol.data(), xw.data(),
                            xk.data(), M, 0, &b);
    if (rc) return rc;
    // bounds of every expanded DAG on the device, then the segmented max over realisations
    int64_t *d_bound = nullptr, *d_off = nullptr, *d_out = nullptr;
    int32_t *d_status = nullptr, *d_arg = nullptr;
    auto cleanup = [&](int code) {
        cudaFree(d_bound);
        cudaFree(d_off);
        cudaFree(d_out);
        cudaFree(d_status);
        cudaFree(d_arg);
        dagrt_batch_free(b);
        return code;
    };
    if (cudaMalloc(&d_bound, 8 * nx) != cudaSuccess || cudaMalloc(&d_status, 4 * nx) != cudaSuccess ||
        cudaMalloc(&d_off, 8 * (n_dags + 1)) != cudaSuccess || cudaMalloc(&d_out, 8 * n_dags) != cudaSuccess ||
        cudaMalloc(&d_arg, 4 * n_dags) != cudaSuccess ||
        cudaMemcpy(d_off, roff.data(), 8 * (n_dags + 1), cudaMemcpyHostToDevice) != cudaSuccess)
        return cleanup(DAGRT_E_OOM);
    dagrt_schedule_out o;
    std::memset(&o, 0, sizeof o);
    o.bound = d_bound;
    o.status = d_status;
    if ((rc = dagrt_schedule(b, variant, &o, DAGRT_PTR_DEVICE)) || (rc = dagrt_sync(ctx))) return cleanup(rc);
    int grid = (n_dags + 7) / 8;
    if (grid > 1024) grid = 1024;
    k_segmax<<<grid, 256>>>(n_dags, d_off, d_bound, d_status, d_out, d_arg);
    std::vector<int64_t> whole(n_dags);
    std::vector<int32_t> whole_st(n_dags), arg(n_dags);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(adaptive, d_out, 8 * n_dags, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(arg.data(), d_arg, 4 * n_dags, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(whole.data(), d_bound + n_real_all, 8 * n_dags, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(whole_st.data(), d_status + n_real_all, 4 * n_dags, cudaMemcpyDeviceToHost) != cudaSuccess)
        return cleanup(DAGRT_E_DEVICE);
    for (int d = 0; d < n_dags; d++) {
        if (fixed) fixed[d] = whole_st[d] == DAGRT_OK ? whole[d] : -1;
        if (worst_real) worst_real[d] = arg[d];
        if (n_real) n_real[d] = counts[d];
    }
    return cleanup(DAGRT_OK);
}
