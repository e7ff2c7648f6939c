// dagrt_internal.cuh -- device-side building blocks shared by the libdagrt kernels.
//
// A "team" is the set of threads that cooperates on one DAG: either one warp (NT == 32,
// several independent teams per CTA, workspace in shared memory) or a whole CTA
// (NT == blockDim.x, workspace in shared or global memory). Algorithms are written once
// against Team<NT> and run unchanged on both.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "dagrt.h"

namespace dagrt {

constexpr uint64_t KEY_INF = ~0ull;
constexpr unsigned FULL = 0xffffffffu;

__host__ __device__ constexpr int ceil_div(int a, int b) { return (a + b - 1) / b; }
__host__ __device__ constexpr int64_t align_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// ------------------------------------------------------------------ team
template <int NT>
struct Team {
    static constexpr int N = NT;
    static constexpr int NW = NT / 32;
    int t;              // rank in team
    uint64_t *red;      // NW words of shared scratch (NT > 32 only)

    __device__ __forceinline__ int lane() const { return t & 31; }
    __device__ __forceinline__ int warp() const { return t >> 5; }
    __device__ __forceinline__ void sync() const {
        if constexpr (NT == 32) __syncwarp(); else __syncthreads();
    }

    template <class Op>
    __device__ __forceinline__ uint64_t reduce(uint64_t v, Op op) const {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(FULL, v, o));
        if constexpr (NT == 32) {
            return v;
        } else {
            if (lane() == 0) red[warp()] = v;
            __syncthreads();
            uint64_t r = red[0];
#pragma unroll
            for (int i = 1; i < NW; i++) r = op(r, red[i]);
            __syncthreads();
            return r;
        }
    }
    __device__ __forceinline__ uint64_t sum(uint64_t v) const {
        return reduce(v, [](uint64_t a, uint64_t b) { return a + b; });
    }
    __device__ __forceinline__ uint64_t maxu(uint64_t v) const {
        return reduce(v, [](uint64_t a, uint64_t b) { return a > b ? a : b; });
    }
    __device__ __forceinline__ uint64_t minu(uint64_t v) const {
        return reduce(v, [](uint64_t a, uint64_t b) { return a < b ? a : b; });
    }
    __device__ __forceinline__ bool any(bool p) const {
        if constexpr (NT == 32) return __any_sync(FULL, p);
        else return __syncthreads_or(p) != 0;
    }

    // Inclusive scan of v across the team with an associative op; *total gets the
    // reduction of all values.
    template <class Op>
    __device__ __forceinline__ uint64_t incl_scan(uint64_t v, Op op, uint64_t *total) const {
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t x = __shfl_up_sync(FULL, v, o);
            if (lane() >= o) v = op(v, x);
        }
        if constexpr (NT == 32) {
            *total = __shfl_sync(FULL, v, 31);
            return v;
        } else {
            if (lane() == 31) red[warp()] = v;
            __syncthreads();
            uint64_t carry = 0, tot = 0;
            bool have = false;
            for (int i = 0; i < NW; i++) {
                if (i == warp()) { carry = tot; have = i > 0; }
                tot = i == 0 ? red[0] : op(tot, red[i]);
            }
            __syncthreads();
            *total = tot;
            return have ? op(carry, v) : v;
        }
    }
    // Exclusive prefix sum of non-negative counts.
    __device__ __forceinline__ uint32_t excl_sum(uint32_t v, uint32_t *total) const {
        uint64_t tot;
        uint64_t inc = incl_scan(v, [](uint64_t a, uint64_t b) { return a + b; }, &tot);
        *total = (uint32_t)tot;
        return (uint32_t)(inc - v);
    }
};

// In-place inclusive scan of arr[0..n) (team-wide, chunk by chunk with a carry); with
// `reverse` the scan runs from arr[n-1] down to arr[0]. Lanes past the end take part in
// the warp scan but sit after every real lane, so they never reach a real result.
template <int NT, class T, class Op>
__device__ void team_scan_inplace(const Team<NT> &tm, T *arr, int n, Op op, bool reverse) {
    uint64_t carry = 0;
    bool have = false;
    for (int base = 0; base < n; base += NT) {
        int i = base + tm.t;
        int idx = reverse ? n - 1 - i : i;
        uint64_t v = i < n ? (uint64_t)arr[idx] : 0;
        uint64_t tot;
        uint64_t s = tm.incl_scan(v, op, &tot);
        int last = min(n - base, NT) - 1;
        uint64_t chunk_tot;
        if constexpr (NT == 32) {
            chunk_tot = __shfl_sync(FULL, s, last);
        } else {
            if (tm.t == last) tm.red[0] = s;
            __syncthreads();
            chunk_tot = tm.red[0];
            __syncthreads();
        }
        if (i < n) arr[idx] = (T)(have ? op(carry, s) : s);
        carry = have ? op(carry, chunk_tot) : chunk_tot;
        have = true;
        tm.sync();
    }
}

// Bitonic sort of keys[0..P) ascending, P a power of two.
template <int NT>
__device__ void team_bitonic_sort(const Team<NT> &tm, uint64_t *keys, int P) {
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = tm.t; i < P; i += NT) {
                int l = i ^ j;
                if (l > i) {
                    uint64_t a = keys[i], b = keys[l];
                    bool up = (i & k) == 0;
                    if (up ? (a > b) : (a < b)) { keys[i] = b; keys[l] = a; }
                }
            }
            tm.sync();
        }
    }
}

// ------------------------------------------------------------------ Eq.1
// Execution time of a kernel with load x (ticks on one SM) and parallel fraction k/64 on m
// of M SMs: max(1, ceil(ceil(m/M) * x * (64m - k(m-1)) / (64m))). Products stay below
// 2^62 for x < 2^32, m <= 4096, M >= 1.
__device__ __forceinline__ uint64_t exec_time(uint64_t x, uint32_t k, uint32_t m, uint32_t M) {
    uint32_t waves = m <= M ? 1u : (m + M - 1) / M;
    uint64_t a = 64ull * m - (uint64_t)k * (m - 1);
    uint64_t num = (uint64_t)waves * x * a;
    uint64_t den = 64ull * m;
    uint64_t c;
    if ((m & (m - 1)) == 0) {
        int sh = 6 + (31 - __clz(m));
        c = (num + den - 1) >> sh;
    } else if (num < (1ull << 32)) {
        c = ((uint32_t)num - 1u) / (uint32_t)den + 1u;  // num >= 64 > 0
    } else {
        c = (num + den - 1) / den;
    }
    return c < 1 ? 1 : c;
}

// Largest load p in [1, L-1] that finishes within R ticks on min(p, S) SMs (S <= M):
// closed form of the node-segmentation size (see the scheduler for the derivation).
__device__ __forceinline__ uint64_t udiv(uint64_t n, uint64_t d) {  // 32-bit divide when both fit
    return (n >> 32) == 0 && (d >> 32) == 0 ? (uint64_t)((uint32_t)n / (uint32_t)d) : n / d;
}

__device__ __forceinline__ uint64_t split_size(uint64_t L, uint32_t k, uint32_t S, uint64_t R) {
    uint64_t a = 64ull * S - (uint64_t)k * (S - 1);
    uint64_t x2 = udiv(64ull * S * R, a);       // largest x >= S with x*a <= 64*S*R
    uint64_t p;
    if (x2 >= S) {
        p = x2;
    } else {                                    // k < 64 here; the answer is below S
        uint64_t x1 = udiv(64ull * R - k, 64ull - k);
        p = x1 < (uint64_t)S - 1 ? x1 : (uint64_t)S - 1;
    }
    if (p > L - 1) p = L - 1;
    if (p < 1) p = 1;
    return p;
}

// The largest dynamic shared memory a launch of `kern` may take on the current device: the
// opt-in maximum per block less the kernel's static shared memory (0 on error). Kernels
// whose launches use different sizes set their attribute to this, not to one launch's
// size: the attribute is per function, and a captured graph node launched on its own (as
// a profiler replays it) is checked against the attribute's current value.
template <class F>
inline int max_dynamic_smem(F *kern) {
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, kern) != cudaSuccess)
        return 0;
    return optin - (int)fa.sharedSizeBytes;
}

}  // namespace dagrt
