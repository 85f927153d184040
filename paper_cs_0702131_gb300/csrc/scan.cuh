// Device-wide exclusive prefix sums: three passes (block totals, scan of the
// totals in one block, per-block scan with carry-in), and a single pass with
// decoupled look-back for the per-step binning.
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

// Single pass (decoupled look-back).  Tiles are numbered by a ticket taken
// when a block starts, so a block only waits for tiles whose blocks already
// run.  Each tile publishes a status word: its own total (flag 1) as soon as
// it is known, its inclusive prefix (flag 2) once the tiles before it are
// summed; a block's first warp reads the statuses of the 32 tiles before it
// at once and sums back to the nearest prefix (further windows if none).
// Status words carry an epoch (bits 34-63, flag in 32-33, value in 0-31), so
// the words of earlier calls read as "not ready" without a reset.  state:
// [0] ticket counter (low 32 bits), [1] epoch, [2 + t] tile t's status; zero
// when first used.  The block of the last ticket rewinds the counter and
// advances the epoch: by then every block has taken its ticket and read the
// epoch (each tile's status was read by a later tile's look-back).  A wait
// gives up after kScanSpinMax polls and sets timeout_flag in *flags (the
// result is then wrong, but the kernel ends).
constexpr int kScanSpinMax = 1 << 20;

static __device__ __forceinline__ unsigned long long scan_word(unsigned epoch, unsigned flag, int v) {
    return ((unsigned long long)epoch << 34) | ((unsigned long long)flag << 32) | (unsigned long long)(unsigned)v;
}

static __global__ void __launch_bounds__(kScanThreads) scan_lookback(const int *in, int64_t n, int *out,
                                                              unsigned long long *state, unsigned *flags,
                                                              unsigned timeout_flag) {
    __shared__ int sh[kScanThreads / 32];
    __shared__ unsigned s_tile, s_epoch;
    __shared__ int s_prefix;
    if (threadIdx.x == 0) {
        s_tile = atomicAdd((unsigned *)state, 1u);
        s_epoch = (unsigned)(((volatile unsigned long long *)state)[1] & 0x3fffffffu);
    }
    __syncthreads();
    const unsigned tile = s_tile, epoch = s_epoch;
    const int64_t base = (int64_t)tile * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int v[kScanItems];
    int sum = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = base + i < n ? in[base + i] : 0;
        sum += v[i];
    }
    int total;
    int run = block_exclusive_scan<int>(sum, sh, total);
    if (threadIdx.x < 32) {
        // look-back by the first warp, 32 tiles per window (lane i: tile wend - 1 - i)
        const unsigned FULL = 0xffffffffu;
        const int lane = threadIdx.x;
        unsigned long long *st = state + 2;
        int prefix = 0;
        if (tile == 0) {
            if (lane == 0) atomicExch(st, scan_word(epoch, 2u, total));
        } else {
            if (lane == 0) atomicExch(st + tile, scan_word(epoch, 1u, total));
            int wend = (int)tile;            // window: tiles wend - 32 .. wend - 1
            for (;;) {
                const int j = wend - 1 - lane;
                unsigned long long w = 0;
                unsigned f = 2u;             // before tile 0: an inclusive prefix of 0
                int spins = 0;
                bool usable = false;
                for (;;) {
                    if (j >= 0) {
                        w = ((volatile unsigned long long *)st)[j];
                        f = (unsigned)(w >> 34) == epoch ? (unsigned)((w >> 32) & 3u) : 0u;
                    }
                    // usable: the nearest prefix and every tile nearer than it are published
                    const unsigned ready = __ballot_sync(FULL, f != 0u), pm = __ballot_sync(FULL, f == 2u);
                    const int p = pm ? __ffs(pm) - 1 : 31;
                    const unsigned need = p == 31 ? FULL : ((1u << (p + 1)) - 1u);
                    usable = (ready & need) == need;
                    if (usable || ++spins >= kScanSpinMax) break;
                }
                if (!usable) {
                    if (lane == 0) atomicOr(flags, timeout_flag);
                    break;
                }
                const unsigned pm = __ballot_sync(FULL, f == 2u);
                const int p = pm ? __ffs(pm) - 1 : 31;
                int part = (lane <= p && j >= 0) ? (int)(unsigned)(w & 0xffffffffu) : 0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(FULL, part, o);
                prefix += part;
                if (pm) break;
                wend -= 32;
            }
            if (lane == 0) {
                __threadfence();
                atomicExch(st + tile, scan_word(epoch, 2u, prefix + total));
            }
        }
        if (lane == 0) {
            s_prefix = prefix;
            if (tile == gridDim.x - 1) {
                ((volatile unsigned long long *)state)[0] = 0ull;
                ((volatile unsigned long long *)state)[1] = (unsigned long long)((epoch + 1u) & 0x3fffffffu);
            }
        }
    }
    __syncthreads();
    run += s_prefix;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i <= n) out[base + i] = run;
        run += v[i];
    }
}

// Words of state that scan_lookback needs for n values.
inline int64_t scan_lookback_words(int64_t n) { return 2 + (n + 1 + kScanTile - 1) / kScanTile; }

// Exclusive scan of n int values into out[0..n] in one launch.
inline int exclusive_scan_1pass(const int *in, int64_t n, int *out, unsigned long long *state, unsigned *flags,
                                unsigned timeout_flag, cudaStream_t st) {
    const int64_t tiles = (n + 1 + kScanTile - 1) / kScanTile;
    scan_lookback<<<(unsigned)tiles, kScanThreads, 0, st>>>(in, n, out, state, flags, timeout_flag);
    return 1;
}

}  // namespace aica
