// Device-wide exclusive prefix sum (three passes: block totals, scan of the
// totals in one block, per-block scan with carry-in).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace aica {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

template <class T>
__device__ __forceinline__ T block_exclusive_scan(T v, T *sh, T &total) {
    // sh: kScanThreads / 32 entries
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T s = lane < kScanThreads / 32 ? sh[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < kScanThreads / 32) sh[lane] = s;
    }
    __syncthreads();
    T before = warp ? sh[warp - 1] : T(0);
    total = sh[kScanThreads / 32 - 1];
    __syncthreads();
    return before + x - v;
}

template <class T, class In>
__global__ void __launch_bounds__(kScanThreads) scan_tile_totals(const In *in, int64_t n, T *totals) {
    __shared__ T sh[kScanThreads / 32];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    T s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) s += (T)in[base + i];
    T total;
    block_exclusive_scan<T>(s, sh, total);
    if (threadIdx.x == 0) totals[blockIdx.x] = total;
}

template <class T>
__global__ void __launch_bounds__(kScanThreads) scan_totals(T *totals, int64_t nt) {
    __shared__ T sh[kScanThreads / 32];
    T carry = 0;
    for (int64_t b = 0; b < nt; b += kScanThreads) {
        int64_t i = b + threadIdx.x;
        T v = i < nt ? totals[i] : T(0);
        T total;
        T ex = block_exclusive_scan<T>(v, sh, total);
        if (i < nt) totals[i] = carry + ex;
        carry += total;
    }
}

// out[i] = sum_{k < i} in[k] for i in [0, n]; out has n + 1 entries.
template <class T, class In>
__global__ void __launch_bounds__(kScanThreads) scan_tiles(const In *in, int64_t n, const T *totals, T *out) {
    __shared__ T sh[kScanThreads / 32];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    T v[kScanItems];
    T s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = base + i < n ? (T)in[base + i] : T(0);
        s += v[i];
    }
    T total;
    T run = block_exclusive_scan<T>(s, sh, total) + totals[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i <= n) out[base + i] = run;
        run += v[i];
    }
}

// Exclusive scan of n values into out[0..n]; `work` must hold
// ceil((n + 1) / kScanTile) values of T.  Returns the launch count.
template <class T, class In>
inline int exclusive_scan(const In *in, int64_t n, T *out, T *work, cudaStream_t st) {
    int64_t tiles = (n + 1 + kScanTile - 1) / kScanTile;
    scan_tile_totals<T, In><<<(unsigned)tiles, kScanThreads, 0, st>>>(in, n, work);
    scan_totals<T><<<1, kScanThreads, 0, st>>>(work, tiles);
    scan_tiles<T, In><<<(unsigned)tiles, kScanThreads, 0, st>>>(in, n, work, out);
    return 3;
}

inline int64_t scan_work_items(int64_t n) { return (n + 1 + kScanTile - 1) / kScanTile; }

}  // namespace aica
