// Molecule-to-cell binning (step a4; §2.2 requires each molecule's cell to be
// known at every step).
//
// Kernels
//   bin_locate   thread per molecule: wrap periodic coordinates, look up the
//                point-location bucket, test candidate cells until one holds
//                p + (e, e^2, e^3), and count the cell's molecules.  A cell
//                holds the point if it lies behind every face plane; a convex
//                cell (tetrahedra, and any cell checked convex at mesh
//                creation) does not if it lies in front of one; other
//                (star-shaped) cells take the cone from the vertex mean
//                through each face triangle.  FP32 filter on cell-local
//                coordinates (face planes precomputed at mesh creation,
//                n / |n|_1 and offset, 16 B per triangle), FP64 and exact
//                slow paths (predicates.cuh).
//   bin_locate_hint / bin_locate_miss   when the same molecules were binned
//                before: test each molecule's previous cell with the FP32
//                filter alone (and, when it left a convex cell, walk across
//                the faces it lies in front of, up to kWalk cells; the point
//                in a cell's frame formed in FP32 from an integer split of
//                the FP64 position), collect the ones still not
//                located (or that the filter could not decide), then search
//                those exactly in the previous cell, its face neighbours and
//                finally the grid.
//                The previous cell is only a search order: the test is exact.
//   scan_lookback  cell offsets from the counts (single pass, scan.cuh)
//   bin_scatter_down  warp-aggregated slot claims, counting the counts down;
//                each claimed slot also gets its cell (read in slot order
//                by bin_slots)
//   bin_slots / bin_cells   order each cell's slots by original index (the
//                stable counting sort by (cell, original index)), gather FP64
//                positions, float4 frame coordinates with the species in .w
//                and their FP32 remainders with the cell in .w (the pair
//                kernels' input layout), the inverse
//                permutation, and the cell's bounding sphere: per slot with
//                window-owned cells for cells of a few molecules, a warp per
//                cell otherwise
//   bin_count, bin_scatter, bin_fixup   the same sort for caller-given cells
//                (aica_sort_by_cell_noalloc)
#include <math.h>
#include <string.h>

#include <algorithm>

#include "aica_internal.cuh"
#include "predicates.cuh"
#include "scan.cuh"

namespace aica {
namespace {

struct BinArgs {
    int64_t n;
    const int *hint;       // previous cell of each molecule (or NULL)
    const int *nbr_off, *nbr;
    int *miss;             // [0] = count, then molecule indices
    float glo_f[3], inv_gh_f[3], gh_f[3];
    const double *pos;
    const int *species;
    double L[3];
    int per[3];
    int G[3];
    double glo[3], gh[3], ghi[3];
    const int *bkt_off, *bkt_cells;
    const int *tri_off, *ntri, *orgk;
    const int *tri_nbr;       // cell across each triangle (-1: boundary)
    const double *org;        // cell origins orgk * 2^-10 (FP64, exact): frame of the cell tests
    const double *orgm64;     // molecule-frame origins (FP64, exact): frame of the binned coordinates
    long long Lkey[3], glo_key[3], ghi_key[3];
    const float *tri32, *ctr32, *box32;
    const float4 *pl32;       // triangle planes n / |n|_1, offset (cell frame)
    const int2 *tric;         // per cell: first triangle, count | convex bit
    const float *orgf;        // cell origins in FP32 (exact when org32)
    const double *tri, *ctr;
    float max_local;
    int org32;                // cell origins exact in FP32 (the hint kernel's FP32 frame change)
    float4 *xlo;              // remainders x - o_m - xloc (binned order)
    int64_t n_owned;          // molecules >= n_owned are halo copies (n_owned = n: none)
    int *cell_of;
    int *cnt;              // molecules per cell (counted as they are located)
    int *inv;              // original -> binned index; -1 for molecules in no cell
    unsigned *flags;
};

// Add one molecule to cell c's count (c < 0: none), aggregated over the warp's
// lanes that located molecules in the same cell.  Every lane must call.
__device__ __forceinline__ void count_located(const BinArgs &a, int c) {
    const unsigned same = __match_any_sync(0xffffffffu, c);
    if (c >= 0 && (int)(threadIdx.x & 31) == __ffs(same) - 1) atomicAdd(a.cnt + c, __popc(same));
}

// Order-preserving integer key of a double: for non-NaN values a < b exactly
// when key(a) < key(b), and key(-0) = key(+0).  Range tests on keys run on the
// integer units instead of the (narrow) FP64 pipe; NaN and infinite
// coordinates still fail the mesh bounds test.
__host__ __device__ __forceinline__ long long dkey(double x) {
    long long b;
    memcpy(&b, &x, sizeof(b));
    return b >= 0 ? b : -(b & 0x7fffffffffffffffLL);
}

__device__ __forceinline__ double wrap_coord(double x, double L, long long Lkey) {
    const long long k = dkey(x);
    if (k >= 0 && k < Lkey) return x;
    x = __dsub_rn(x, __dmul_rn(L, floor(__ddiv_rn(x, L))));
    if (x >= L) x = __dsub_rn(x, L);
    return x;
}

__device__ __forceinline__ float3 ld3f(const float *p) { return make_float3(p[0], p[1], p[2]); }

// sign of O(a, b, c, p + (e, e^2, e^3)): FP32 filter, then (EXACT) the FP64 and
// exact stages; without EXACT an undecided filter returns 0
template <bool EXACT>
__device__ __forceinline__ int orient(float3 a, float3 b, float3 c, float3 q, float scale, const double *a64,
                                      const double *b64, const double *c64, const double *p64) {
    int s = orient_f32(a, b, c, q, scale);
    if (EXACT && !s) s = orient_sos_slow(a64, b64, c64, p64);
    return s;
}

// q (p local to cell c) inside cell c with the SoS tie-break: 1 inside, 0
// outside, -1 undecided (only without EXACT, when the FP32 filter cannot
// decide; the caller then defers to an exact pass).  Behind every face plane
// means inside for any closed cell star-shaped about its centre (the segment
// from the centre to an outside point leaves through a face it ends in front
// of); for a convex cell, in front of one face means outside.  Other cells
// take the cone test: find the triangle whose cone from the centre holds q,
// then q must lie behind that triangle.
// exit_t (optional): for a convex cell found outside, the triangle whose
// plane q lies in front of, else -1.
// boxcheck = false skips the bounding-box rejection, so that a convex cell
// the point lies outside of always reports an exit triangle (for walks).
template <bool EXACT>
__device__ int cell_test(const BinArgs &a, int c, float3 q, const double *p64, int *exit_t = nullptr,
                         bool boxcheck = true) {
    if (exit_t) *exit_t = -1;
    const float *B = a.box32 + 6 * c;
    const float scale = fmaxf(a.max_local, fmaxf(fabsf(q.x), fmaxf(fabsf(q.y), fabsf(q.z))));
    const float tol = 1e-5f * scale;
    if (boxcheck && (q.x < B[0] - tol || q.y < B[1] - tol || q.z < B[2] - tol || q.x > B[3] + tol ||
                     q.y > B[4] + tol || q.z > B[5] + tol))
        return 0;
    const int2 tc = a.tric[c];
    const int t0 = tc.x, code = tc.y, nt = code & 0xffff;
    // the face planes: e = n.q - d with |n|_1 = 1 carries at most about
    // 9 * 2^-24 * scale of rounding (plane, point, three FMAs), far below
    // the filter's bound; undecided faces go to the exact orientation
    const float pb = 1e-5f * scale;
    bool behind = true;
    for (int t = t0; t < t0 + nt; ++t) {
        const float4 P = a.pl32[t];
        const float e = fmaf(P.z, q.z, fmaf(P.y, q.y, fmaf(P.x, q.x, -P.w)));
        int s = e > pb ? 1 : (e < -pb ? -1 : 0);
        if (EXACT && s == 0) {
            const double *D = a.tri + 9 * t;
            s = orient_sos_slow(D, D + 3, D + 6, p64);
        }
        if (!EXACT && s == 0) return -1;
        if (s > 0) {
            behind = false;
            if (exit_t) *exit_t = t;
            break;
        }
    }
    if (behind) return 1;
    if (code >> 16) return 0;
    if (exit_t) *exit_t = -1;
    float3 C = ld3f(a.ctr32 + 3 * c);
    const double *C64 = a.ctr + 3 * c;
    for (int t = t0; t < t0 + nt; ++t) {
        const float *T = a.tri32 + 9 * t;
        const double *D = a.tri + 9 * t;
        float3 x0 = ld3f(T), x1 = ld3f(T + 3), x2 = ld3f(T + 6);
        // p in the cone from C through triangle (x0, x1, x2)?
        int s = orient<EXACT>(C, x0, x1, q, scale, C64, D, D + 3, p64);
        if (!EXACT && s == 0) return -1;
        if (s < 0) continue;
        s = orient<EXACT>(C, x1, x2, q, scale, C64, D + 3, D + 6, p64);
        if (!EXACT && s == 0) return -1;
        if (s < 0) continue;
        s = orient<EXACT>(C, x2, x0, q, scale, C64, D + 6, D, p64);
        if (!EXACT && s == 0) return -1;
        if (s < 0) continue;
        s = orient<EXACT>(x0, x1, x2, q, scale, D, D + 3, D + 6, p64);
        if (!EXACT && s == 0) return -1;
        return s < 0 ? 1 : 0;
    }
    return 0;
}

__device__ __forceinline__ bool cell_contains(const BinArgs &a, int c, float3 q, const double *p64) {
    return cell_test<true>(a, c, q, p64) == 1;
}

// FP64 -> FP32 without the conversion units (on GB300 those share the
// narrow FP64 pipe): hi = x with its 53-bit significand rounded (half up)
// to 24 bits, lo = x - hi rounded to 24 bits, both built from the IEEE bit
// pattern with integer operations.  |lo| <= ulp(hi) / 2 and hi + lo equals x
// to about 2^-48 |x|.  For |x| in [2^-100, 2^100] or x = 0 (positions in a
// molecule or cell frame); smaller values give 0.
__device__ __forceinline__ void split_f64(double x, float &hi, float &lo) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    int E = (int)((b >> 52) & 0x7ff);
    if (E < 1023 - 100) {
        hi = lo = 0.f;
        return;
    }
    const unsigned long long m = (b & 0xfffffffffffffULL) | (1ULL << 52);
    unsigned long long m24 = (m + (1ULL << 28)) >> 29;
    const long long rem = (long long)m - (long long)(m24 << 29);     // |rem| <= 2^28
    if (m24 >> 24) {
        m24 >>= 1;
        ++E;
    }
    hi = __int_as_float((int)(sign | ((unsigned)(E - 1023 + 127) << 23) | ((unsigned)m24 & 0x7fffffu)));
    if (rem == 0) {
        lo = 0.f;
        return;
    }
    // rem * 2^(E0 - 1075) with E0 the exponent before a carry (rem was taken against it)
    const int E0 = (int)((b >> 52) & 0x7ff);
    unsigned long long r = (unsigned long long)(rem < 0 ? -rem : rem);
    const int n = 63 - __clzll((long long)r);                           // bit length - 1, <= 28
    unsigned rm;
    int eb = E0 - 1075 + n;                                            // exponent of the leading bit
    if (n > 23) {
        const int sh = n - 23;
        unsigned long long q = (r + (1ULL << (sh - 1))) >> sh;
        if (q >> 24) {
            q >>= 1;
            ++eb;
        }
        rm = (unsigned)q;
    } else {
        rm = (unsigned)(r << (23 - n));
    }
    if (eb + 127 < 1) {          // below the normal FP32 range: negligible against hi
        lo = 0.f;
        return;
    }
    const unsigned lsign = sign ^ (rem < 0 ? 0x80000000u : 0u);
    lo = __int_as_float((int)(lsign | ((unsigned)(eb + 127) << 23) | (rm & 0x7fffffu)));
}

// p relative to the dyadic origin c_k * 2^-10 of cell c, in FP32 (one rounding)
__device__ __forceinline__ float3 local_to(const BinArgs &a, const double *p, int c) {
    const double *o = a.org + 3 * c;
    float3 q;
    float l;
    split_f64(p[0] - o[0], q.x, l);
    split_f64(p[1] - o[1], q.y, l);
    split_f64(p[2] - o[2], q.z, l);
    return q;
}

__device__ __forceinline__ void wrapped_position(const BinArgs &a, int64_t k, double *p, bool &ok) {
    ok = true;
    for (int d = 0; d < 3; ++d) {
        p[d] = a.pos[3 * k + d];
        if (a.per[d]) p[d] = wrap_coord(p[d], a.L[d], a.Lkey[d]);
        const long long key = dkey(p[d]);
        if (!(key >= a.glo_key[d] && key <= a.ghi_key[d])) ok = false;
    }
}

// Search the bucket grid for the cell holding p (skipping cell `skip`).
__device__ int grid_search(const BinArgs &a, const double *p, int skip) {
    int ib[3];
    for (int d = 0; d < 3; ++d)
        // bucket index in FP32; the buckets are registered with a tolerance
        ib[d] = min(max((int)floorf((float)(p[d] - a.glo[d]) * a.inv_gh_f[d]), 0), a.G[d] - 1);
    const int b = (ib[0] * a.G[1] + ib[1]) * a.G[2] + ib[2];
    // dyadic bucket origin: p relative to it is one rounding from exact
    int kb[3];
    for (int d = 0; d < 3; ++d) kb[d] = (int)rintf((a.glo_f[d] + ((float)ib[d] + 0.5f) * a.gh_f[d]) * 1024.0f);
    const float3 pb = make_float3((float)(p[0] - kb[0] * (1.0 / 1024.0)), (float)(p[1] - kb[1] * (1.0 / 1024.0)),
                                  (float)(p[2] - kb[2] * (1.0 / 1024.0)));
    for (int i = a.bkt_off[b]; i < a.bkt_off[b + 1]; ++i) {
        const int c = a.bkt_cells[i];
        if (c == skip) continue;
        const float3 q = make_float3(pb.x - (float)(a.orgk[3 * c] - kb[0]) * (1.0f / 1024.0f),
                                     pb.y - (float)(a.orgk[3 * c + 1] - kb[1]) * (1.0f / 1024.0f),
                                     pb.z - (float)(a.orgk[3 * c + 2] - kb[2]) * (1.0f / 1024.0f));
        if (cell_contains(a, c, q, p)) return c;
    }
    return -1;
}

// Full search for every molecule (no previous cells).
__global__ void __launch_bounds__(256) bin_locate(BinArgs a) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int found = -1;
    if (k < a.n) {
        double p[3];
        bool ok;
        wrapped_position(a, k, p, ok);
        found = ok ? grid_search(a, p, -1) : -1;
        a.cell_of[k] = found;
        if (found < 0) {
            a.inv[k] = -1;
            atomicOr(a.flags, kFlagOutside);
        }
    }
    count_located(a, found);
}

// Previous cell first.  A molecule that left a convex cell walks: into the
// cell across the face whose plane it lies in front of, up to kWalk cells
// (a visibility walk, as in point location in triangulations); the FP32
// filter alone decides each step.  Molecules not found so (the walk met a
// boundary, a non-convex cell, an undecided test, or ran out of steps) go
// to the miss list.
constexpr int kWalk = 8;
__global__ void __launch_bounds__(256) bin_locate_hint(BinArgs a) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool miss = false, undecided = false;
    int located = -1;
    if (k < a.n) {
        double p[3];
        bool ok;
        wrapped_position(a, k, p, ok);
        const int h = a.hint[k];
        if (ok && h >= 0) {
            // p in a cell's frame without the FP64 pipe: p = ph + pl (split on
            // the integer units), the cell origin exact in FP32, q = (ph - o) + pl
            // (at most about 2.2 * 2^-24 of the frame scale off the exact local
            // point, inside the filter's bound)
            float ph[3], pl[3];
            for (int d = 0; d < 3; ++d) split_f64(p[d], ph[d], pl[d]);
            auto loc = [&](int cc) {
                if (!a.org32) return local_to(a, p, cc);
                const float *o = a.orgf + 3 * cc;
                return make_float3((ph[0] - o[0]) + pl[0], (ph[1] - o[1]) + pl[1], (ph[2] - o[2]) + pl[2]);
            };
            int c = h, ex = -1;
            int r = cell_test<false>(a, c, loc(c), p, &ex, false);
            undecided = r < 0;
            for (int step = 0; step < kWalk && r == 0 && ex >= 0; ++step) {
                c = a.tri_nbr[ex];
                if (c < 0) break;
                r = cell_test<false>(a, c, loc(c), p, &ex, false);
            }
            if (r == 1) {
                a.cell_of[k] = c;
                located = c;
            } else {
                miss = true;
            }
        } else if (ok) {
            miss = true;
        } else {
            a.cell_of[k] = -1;
            a.inv[k] = -1;
            atomicOr(a.flags, kFlagOutside);
        }
    }
    count_located(a, located);
    const unsigned bal = __ballot_sync(0xffffffffu, miss);
    const int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == 0 && bal) base = atomicAdd(a.miss, __popc(bal));
    base = __shfl_sync(0xffffffffu, base, 0);
    // the top bit marks molecules whose previous cell the FP32 filter could not decide
    if (miss) a.miss[1 + base + __popc(bal & ((1u << lane) - 1u))] = (int)k | (undecided ? (int)0x80000000u : 0);
}

// Molecules that left their previous cell: one warp per molecule, lanes test
// the previous cell's face neighbours in parallel, then the cells of the
// molecule's bucket.  Exact predicates make at most one cell hold the point.
__global__ void __launch_bounds__(256) bin_locate_miss(BinArgs a) {
    const int lane = threadIdx.x & 31;
    const int nm = a.miss[0];
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nm; i += nw) {
        const int e = a.miss[1 + i];
        const int k = e & 0x7fffffff;
        double p[3];
        bool ok;
        wrapped_position(a, k, p, ok);
        const int h = a.hint[k];
        int found = -1;
        if (e < 0) {            // the previous cell, undecided by the FP32 filter: exactly, once
            bool in = false;
            if (lane == 0) in = cell_contains(a, h, local_to(a, p, h), p);
            if (__shfl_sync(0xffffffffu, in, 0)) found = h;
        }
        if (h >= 0 && found < 0) {
            const int j1 = a.nbr_off[h + 1];
            for (int j0 = a.nbr_off[h]; j0 < j1; j0 += 32) {
                const int j = j0 + lane;
                int c = -1;
                bool hit = false;
                if (j < j1) {
                    c = a.nbr[j];
                    hit = cell_contains(a, c, local_to(a, p, c), p);
                }
                const unsigned bal = __ballot_sync(0xffffffffu, hit);
                if (bal) {
                    found = __shfl_sync(0xffffffffu, c, __ffs(bal) - 1);
                    break;
                }
            }
        }
        if (found < 0) {
            int ib[3];
            for (int d = 0; d < 3; ++d)
                ib[d] = min(max((int)floorf((float)(p[d] - a.glo[d]) * a.inv_gh_f[d]), 0), a.G[d] - 1);
            const int b = (ib[0] * a.G[1] + ib[1]) * a.G[2] + ib[2];
            const int i1 = a.bkt_off[b + 1];
            for (int i0 = a.bkt_off[b]; i0 < i1; i0 += 32) {
                const int ii = i0 + lane;
                int c = -1;
                bool hit = false;
                if (ii < i1) {
                    c = a.bkt_cells[ii];
                    hit = c != h && cell_contains(a, c, local_to(a, p, c), p);
                }
                const unsigned bal = __ballot_sync(0xffffffffu, hit);
                if (bal) {
                    found = __shfl_sync(0xffffffffu, c, __ffs(bal) - 1);
                    break;
                }
            }
        }
        if (lane == 0) {
            a.cell_of[k] = found;
            if (found >= 0) {
                atomicAdd(a.cnt + found, 1);
            } else {
                a.inv[k] = -1;
                atomicOr(a.flags, kFlagOutside);
            }
        }
    }
}

// Counting sort of caller-given cells (aica_sort_by_cell_noalloc).  A cell
// id outside [0, C) is left out like -1; ids >= C are counted in *bad, so
// no access ever leaves cnt[0, C), cell_off[0, C] or order[0, n).
__global__ void __launch_bounds__(256) bin_count(const int *cell_of, int64_t n, int C, int *cnt, int *bad) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int c = k < n ? cell_of[k] : -1;
    if (c >= C) {
        atomicAdd(bad, 1);
        c = -1;
    }
    unsigned same = __match_any_sync(0xffffffffu, c);
    int lane = threadIdx.x & 31;
    if (c >= 0 && lane == __ffs(same) - 1) atomicAdd(cnt + c, __popc(same));
}

__global__ void __launch_bounds__(256) bin_scatter(const int *cell_of, int64_t n, int C, const int *cell_off,
                                                   int *fill, int *order) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int c = k < n ? cell_of[k] : -1;
    if (c >= C) c = -1;
    unsigned same = __match_any_sync(0xffffffffu, c);
    int lane = threadIdx.x & 31;
    int leader = __ffs(same) - 1;
    int base = 0;
    if (c >= 0 && lane == leader) base = atomicAdd(fill + c, __popc(same));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (c >= 0) order[cell_off[c] + base + __popc(same & ((1u << lane) - 1u))] = (int)k;
}

// Each cell's slots in ascending original index: a warp per cell, bitonic
// sort in shared memory for cells of up to kFixCap molecules (padded to a
// power of two with INT_MAX), a serial insertion sort beyond that.
constexpr int kFixWarps = 4, kFixCap = 2048;
__global__ void __launch_bounds__(kFixWarps * 32) bin_fixup(const int *cell_off, int C, int *order) {
    __shared__ int buf[kFixWarps][kFixCap];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int c = blockIdx.x * kFixWarps + w;
    if (c >= C) return;
    const int s = cell_off[c], m = cell_off[c + 1] - s;
    if (m < 2) return;
    if (m > kFixCap) {
        if (lane == 0)
            for (int i = s + 1; i < s + m; ++i) {
                int v = order[i], j = i - 1;
                while (j >= s && order[j] > v) {
                    order[j + 1] = order[j];
                    --j;
                }
                order[j + 1] = v;
            }
        return;
    }
    int P = 2;
    while (P < m) P <<= 1;
    int *b = buf[w];
    for (int i = lane; i < P; i += 32) b[i] = i < m ? order[s + i] : 0x7fffffff;
    __syncwarp();
    for (int size = 2; size <= P; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = lane; i < P / 2; i += 32) {
                const int lo = 2 * i - (i & (stride - 1)), hi = lo + stride;
                const bool up = (lo & size) == 0;
                const int x = b[lo], y = b[hi];
                if ((x > y) == up) {
                    b[lo] = y;
                    b[hi] = x;
                }
            }
            __syncwarp();
        }
    for (int i = lane; i < m; i += 32) order[s + i] = b[i];
}

// Slots of located molecules: cell c's count (from the locate kernels) is
// counted down, so the counts are zero again afterwards.  Order within a
// cell is fixed by bin_cells.
__global__ void __launch_bounds__(256) bin_scatter_down(const int *cell_of, int64_t n, const int *cell_off, int *cnt,
                                                        int *order, int *slot_cell) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int c = k < n ? cell_of[k] : -1;
    const unsigned same = __match_any_sync(0xffffffffu, c);
    const int lane = threadIdx.x & 31, leader = __ffs(same) - 1, m = __popc(same);
    int top = 0;
    if (c >= 0 && lane == leader) top = atomicSub(cnt + c, m);
    top = __shfl_sync(0xffffffffu, top, leader);
    if (c >= 0) {
        const int s = cell_off[c] + top - m + __popc(same & ((1u << lane) - 1u));
        order[s] = (int)k;
        if (slot_cell) slot_cell[s] = c;         // read in slot order by the in-cell sort
    }
}

// Coordinates of p in the molecule frame o: the nearest FP32 values and the
// FP32 remainders (hi + lo equals p - o to about 2^-48 |p - o|).  The FP32
// cluster pair kernel rebuilds exactly rounded separations from both.  The
// remainder's .w carries the molecule's cell (int bits): the cluster kernel
// tells cells of a cluster (at most 16 consecutive ones) apart by it.
__device__ __forceinline__ void frame_split(const BinArgs &a, const double *p, const double *o, int sp, int cell,
                                            float4 &hi, float4 &lo) {
    float h[3], l[3];
    for (int d = 0; d < 3; ++d) split_f64(p[d] - o[d], h[d], l[d]);   // p - o is exact (o dyadic, nearby)
    hi = make_float4(h[0], h[1], h[2], __int_as_float(sp));
    lo = make_float4(l[0], l[1], l[2], __int_as_float(cell));
}

// Per cell, by groups of G lanes: order the cell's molecules by original
// index (the stable counting sort), gather FP64 positions and FP32
// coordinates local to the cell's molecule-frame origin into binned order, record the
// inverse permutation, and the cell's bounding sphere (centre = mean, radius
// = largest distance, rounded up) that the pair kernels cull with.
template <int G>
__global__ void __launch_bounds__(256) bin_cells(BinArgs a, const int *cell_off, int C, int *order, double *xs64,
                                                 float4 *xloc, float4 *sph) {
    const int lane = threadIdx.x & 31, g = lane & (G - 1);
    const int groups = (gridDim.x * blockDim.x) / G;
    int spmax = 0;
    bool bad = false;
    // every lane runs the same number of rounds (shuffles below use the full warp)
    const int rounds = (C + groups - 1) / groups;
    for (int r = 0; r < rounds; ++r) {
        const int c = r * groups + (int)((blockIdx.x * blockDim.x + threadIdx.x) / G);
        const int s = c < C ? cell_off[c] : 0, m = c < C ? cell_off[c + 1] - s : 0;
        const bool small = m <= G;
        int k = (small && g < m) ? order[s + g] : 0x7fffffff;
        int rank = 0;
#pragma unroll
        for (int j = 0; j < G; ++j) rank += __shfl_sync(0xffffffffu, k, j, G) < k;
        __syncwarp();
        float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
        const bool mine = small && g < m;
        if (mine) {
            const int slot = s + rank;
            order[slot] = k;
            a.inv[k] = slot;
            const int sp = a.species[k];
            spmax = max(spmax, sp < 0 ? kMaxSpecies : sp);
            bad |= (unsigned)sp >= (unsigned)kMaxSpecies;
            double p[3];
            for (int d = 0; d < 3; ++d) {
                p[d] = a.pos[3 * (int64_t)k + d];
                if (a.per[d]) p[d] = wrap_coord(p[d], a.L[d], a.Lkey[d]);
                xs64[3 * (int64_t)slot + d] = p[d];
            }
            float4 lo;
            frame_split(a, p, a.orgm64 + 3 * c, (sp & (kMaxSpecies - 1)) | (k >= a.n_owned ? kGhostBit : 0), c, x, lo);
            xloc[slot] = x;
            a.xlo[slot] = lo;
        }
        float cx = mine ? x.x : 0.f, cy = mine ? x.y : 0.f, cz = mine ? x.z : 0.f;
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            cx += __shfl_xor_sync(0xffffffffu, cx, o, G);
            cy += __shfl_xor_sync(0xffffffffu, cy, o, G);
            cz += __shfl_xor_sync(0xffffffffu, cz, o, G);
        }
        const float inv_m = m > 0 ? 1.f / (float)m : 0.f;
        cx *= inv_m; cy *= inv_m; cz *= inv_m;
        float r2 = 0.f;
        if (mine) {
            const float dx = x.x - cx, dy = x.y - cy, dz = x.z - cz;
            r2 = dx * dx + dy * dy + dz * dz;
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) r2 = fmaxf(r2, __shfl_xor_sync(0xffffffffu, r2, o, G));
        if (small && c < C && g == 0) sph[c] = make_float4(cx, cy, cz, sqrtf(r2) * (1.f + 1e-5f) + 1e-5f);
        if (!small && g == 0) {
            // more molecules than lanes: one lane sorts, gathers and bounds the cell
            for (int i = s + 1; i < s + m; ++i) {
                const int v = order[i];
                int j = i - 1;
                while (j >= s && order[j] > v) {
                    order[j + 1] = order[j];
                    --j;
                }
                order[j + 1] = v;
            }
            float sx = 0.f, sy = 0.f, sz = 0.f;
            for (int slot = s; slot < s + m; ++slot) {
                const int kk = order[slot];
                a.inv[kk] = slot;
                const int sp = a.species[kk];
                spmax = max(spmax, sp < 0 ? kMaxSpecies : sp);
                bad |= (unsigned)sp >= (unsigned)kMaxSpecies;
                double p[3];
                for (int d = 0; d < 3; ++d) {
                    p[d] = a.pos[3 * (int64_t)kk + d];
                    if (a.per[d]) p[d] = wrap_coord(p[d], a.L[d], a.Lkey[d]);
                    xs64[3 * (int64_t)slot + d] = p[d];
                }
                float4 y, lo;
                frame_split(a, p, a.orgm64 + 3 * c, (sp & (kMaxSpecies - 1)) | (kk >= a.n_owned ? kGhostBit : 0), c, y, lo);
                xloc[slot] = y;
                a.xlo[slot] = lo;
                sx += y.x; sy += y.y; sz += y.z;
            }
            sx /= (float)m; sy /= (float)m; sz /= (float)m;
            float rr = 0.f;
            for (int slot = s; slot < s + m; ++slot) {
                const float4 y = xloc[slot];
                const float dx = y.x - sx, dy = y.y - sy, dz = y.z - sz;
                rr = fmaxf(rr, dx * dx + dy * dy + dz * dz);
            }
            sph[c] = make_float4(sx, sy, sz, sqrtf(rr) * (1.f + 1e-5f) + 1e-5f);
        }
    }
    // largest species index (flags[1]) and out-of-range species (flags[0])
    const int mx = __reduce_max_sync(0xffffffffu, spmax);
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.flags, kFlagSpecies);
    if (lane == 0 && mx > 0) atomicMax((int *)a.flags + 1, mx);
}

// The same per slot, for cells of a few molecules.  Warp w owns the cells
// whose first slot lies in its window of 32 slots [32 w, 32 w + 32); such a
// cell ends before the first cell start of the next window, so the warp
// stages the molecules of both windows (two slots per lane) in shared memory
// and orders, gathers and bounds its cells there: rank = number of the
// cell's original indices below the lane's, centre summed in rank order.  A
// cell that covers the whole next window is done by one lane in global
// memory.  `un` holds each cell's molecules in any order (bin_scatter_down);
// `order` gets them sorted.  nbp points at the binned count (cell_off[C]).
constexpr int kSlotWarps = 8;

__device__ __forceinline__ float4 local_xloc_from(const BinArgs &a, int k, int c, int slot, double *xs64, int &spmax,
                                                  bool &bad, int sp, const double (&raw)[3]) {
    spmax = max(spmax, sp < 0 ? kMaxSpecies : sp);
    bad |= (unsigned)sp >= (unsigned)kMaxSpecies;
    double p[3];
    for (int d = 0; d < 3; ++d) {
        p[d] = raw[d];
        if (a.per[d]) p[d] = wrap_coord(p[d], a.L[d], a.Lkey[d]);
        xs64[3 * (int64_t)slot + d] = p[d];
    }
    float4 hi, lo;
    frame_split(a, p, a.orgm64 + 3 * c, (sp & (kMaxSpecies - 1)) | (k >= a.n_owned ? kGhostBit : 0), c, hi, lo);
    a.xlo[slot] = lo;
    return hi;
}

__device__ __forceinline__ float4 local_xloc(const BinArgs &a, int k, int c, int slot, double *xs64, int &spmax,
                                             bool &bad) {
    const double raw[3] = {a.pos[3 * (int64_t)k], a.pos[3 * (int64_t)k + 1], a.pos[3 * (int64_t)k + 2]};
    return local_xloc_from(a, k, c, slot, xs64, spmax, bad, a.species[k], raw);
}

__device__ __forceinline__ float4 sphere_of(const float4 *x, int m) {
    float cx = 0.f, cy = 0.f, cz = 0.f;
    for (int j = 0; j < m; ++j) {
        cx += x[j].x;
        cy += x[j].y;
        cz += x[j].z;
    }
    const float im = 1.f / (float)m;
    cx *= im;
    cy *= im;
    cz *= im;
    float rr = 0.f;
    for (int j = 0; j < m; ++j) {
        const float dx = x[j].x - cx, dy = x[j].y - cy, dz = x[j].z - cz;
        rr = fmaxf(rr, dx * dx + dy * dy + dz * dz);
    }
    return make_float4(cx, cy, cz, sqrtf(rr) * (1.f + 1e-5f) + 1e-5f);
}

__global__ void __launch_bounds__(kSlotWarps * 32) bin_slots(BinArgs a, const int *cell_off, const int *nbp,
                                                             const int *un, const int *ucell, int *order,
                                                             double *xs64, float4 *xloc, float4 *sph) {
    __shared__ int sk[kSlotWarps][64];
    __shared__ float4 sx[kSlotWarps][64];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t w0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane;   // first slot of the window
    const int nb = *nbp;
    if (w0 >= nb) return;                 // whole warp
    int k[2], c[2], s0[2], m[2], sp[2] = {0, 0};
    double raw[2][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
    bool st[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int64_t S = w0 + 32 * h + lane;
        if (S < nb) {
            k[h] = un[S];
            c[h] = ucell[S];                  // the slot's cell, written with the slot claim
            // the molecule's data, loaded while the cell offsets arrive
            sp[h] = a.species[k[h]];
            for (int d = 0; d < 3; ++d) raw[h][d] = a.pos[3 * (int64_t)k[h] + d];
            s0[h] = cell_off[c[h]];
            m[h] = cell_off[c[h] + 1] - s0[h];
            st[h] = s0[h] == S;
        } else {                          // past the binned slots: every slot is a boundary
            k[h] = 0x7fffffff;
            c[h] = -1;
            s0[h] = (int)S;
            m[h] = 0;
            st[h] = true;
        }
    }
    const unsigned b0 = __ballot_sync(FULL, st[0]), b1 = __ballot_sync(FULL, st[1]);
    if (!b0) return;                      // the window lies inside a cell that starts earlier
    const int bw = __ffs(b0) - 1;         // first cell start (window-local index)
    const int last = 31 - __clz(b0);      // last cell start in the window
    const bool tail = b1 == 0;            // that cell covers the whole next window
    const int ew = tail ? last : 32 + __ffs(b1) - 1;
    sk[wib][lane] = k[0];
    sk[wib][32 + lane] = k[1];
    __syncwarp();
    int spmax = 0;
    bool bad = false;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int i = 32 * h + lane;
        if (i >= bw && i < ew && w0 + i < nb) {
            const int ls = (int)(s0[h] - w0);
            int rank = 0;
            for (int j = 0; j < m[h]; ++j) rank += sk[wib][ls + j] < k[h] ? 1 : 0;
            const int slot = s0[h] + rank;
            order[slot] = k[h];
            a.inv[k[h]] = slot;
            const float4 x = local_xloc_from(a, k[h], c[h], slot, xs64, spmax, bad, sp[h], raw[h]);
            xloc[slot] = x;
            sx[wib][ls + rank] = x;
        }
    }
    __syncwarp();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int i = 32 * h + lane;
        if (i >= bw && i < ew && w0 + i < nb && st[h]) sph[c[h]] = sphere_of(&sx[wib][i], m[h]);
    }
    if (tail && lane == last && w0 + last < nb) {
        // one lane: copy, sort by original index, gather and bound the cell
        const int cs = s0[0], cm = m[0], cc = c[0];
        for (int i = cs; i < cs + cm; ++i) {
            const int v = un[i];
            int j = i - 1;
            while (j >= cs && order[j] > v) {
                order[j + 1] = order[j];
                --j;
            }
            order[j + 1] = v;
        }
        float sxs = 0.f, sys = 0.f, szs = 0.f;
        for (int slot = cs; slot < cs + cm; ++slot) {
            const int kk = order[slot];
            a.inv[kk] = slot;
            const float4 y = local_xloc(a, kk, cc, slot, xs64, spmax, bad);
            xloc[slot] = y;
            sxs += y.x; sys += y.y; szs += y.z;
        }
        const float im = 1.f / (float)cm;
        sxs *= im; sys *= im; szs *= im;
        float rr = 0.f;
        for (int slot = cs; slot < cs + cm; ++slot) {
            const float4 y = xloc[slot];
            const float dx = y.x - sxs, dy = y.y - sys, dz = y.z - szs;
            rr = fmaxf(rr, dx * dx + dy * dy + dz * dz);
        }
        sph[cc] = make_float4(sxs, sys, szs, sqrtf(rr) * (1.f + 1e-5f) + 1e-5f);
    }
    const int mx = __reduce_max_sync(FULL, spmax);
    if (__any_sync(FULL, bad) && lane == 0) atomicOr(a.flags, kFlagSpecies);
    if (lane == 0 && mx > 0) atomicMax((int *)a.flags + 1, mx);
}

}  // namespace
}  // namespace aica

using namespace aica;

extern "C" aica_status aica_bin_molecules(aica_mesh *m, const double *pos, const int32_t *species, int64_t n,
                                          int32_t *cell_of, int32_t *order, int32_t *cell_off, void *stream) {
    AICA_RANGE("aica_bin_molecules");
    if (!m) { set_error("aica_bin_molecules: mesh is NULL"); return AICA_ERR_INVALID_ARG; }
    if (n < 0 || n > (int64_t)INT32_MAX / 2 || (n > 0 && (!pos || !species))) {
        set_error("aica_bin_molecules: bad molecule arrays (n = %lld)", (long long)n);
        return AICA_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int C = (int)m->n_cells;
    m->launches = 0;
    m->binned = false;
    if (n > m->cap_mol) {
        m->hint_valid = false;
        int64_t cap = std::max<int64_t>(n, 1024);
        AICA_CUDA(m->cell_of.reserve(sizeof(int) * cap));
        AICA_CUDA(m->order.reserve(sizeof(int) * cap));
        AICA_CUDA(m->unsorted.reserve(sizeof(int) * cap));
        AICA_CUDA(m->ucell.reserve(sizeof(int) * cap));
        AICA_CUDA(m->xloc.reserve(sizeof(float4) * cap));
        AICA_CUDA(m->xlo.reserve(sizeof(float4) * cap));
        AICA_CUDA(m->flag_list.reserve(sizeof(int) * (cap + 1)));
        AICA_CUDA(m->inv.reserve(sizeof(int) * cap));
        AICA_CUDA(m->xs64.reserve(sizeof(double) * 3 * cap));
        AICA_CUDA(m->facc.reserve(sizeof(double) * 4 * cap));
        AICA_CUDA(m->vsorted.reserve(sizeof(double) * 4 * cap));
        m->cap_mol = cap;
    }
    AICA_CUDA(m->cell_off.reserve(sizeof(int) * (C + 1)));
    AICA_CUDA(m->fill.reserve(sizeof(int) * (C + 1)));
    AICA_CUDA(m->sph.reserve(sizeof(float4) * C));
    AICA_CUDA(m->miss.reserve(sizeof(int) * (std::max<int64_t>(n, 1) + 1)));
    m->n_mol = n;
    BinArgs a{};
    a.n = n;
    a.pos = pos;
    a.species = species;
    for (int d = 0; d < 3; ++d) {
        a.L[d] = m->box.L[d];
        a.per[d] = m->box.periodic[d] ? 1 : 0;
        a.G[d] = m->G[d];
        a.glo[d] = m->glo[d];
        a.gh[d] = m->gh[d];
        a.ghi[d] = m->glo[d] + m->G[d] * m->gh[d];
    }
    a.bkt_off = m->bkt_off.as<int>();
    a.bkt_cells = m->bkt_cells.as<int>();
    a.tri_off = m->tri_off.as<int>();
    a.ntri = m->ntri.as<int>();
    a.orgk = m->orgk.as<int>();
    a.tri_nbr = m->tri_nbr.as<int>();
    a.org = m->org.as<double>();
    a.orgm64 = m->orgm64.as<double>();
    for (int d = 0; d < 3; ++d) {
        a.Lkey[d] = dkey(a.L[d]);
        a.glo_key[d] = dkey(a.glo[d]);
        a.ghi_key[d] = dkey(a.ghi[d]);
    }
    a.tri32 = m->tri32.as<float>();
    a.pl32 = m->pl32.as<float4>();
    a.tric = m->tric.as<int2>();
    a.orgf = m->orgf.as<float>();
    a.ctr32 = m->ctr32.as<float>();
    a.box32 = m->box32.as<float>();
    a.tri = m->tri.as<double>();
    a.ctr = m->ctr.as<double>();
    a.max_local = (float)(m->max_local * (1 + 1e-6));
    a.org32 = m->org32 ? 1 : 0;
    a.xlo = m->xlo.as<float4>();
    if (m->n_owned >= 0 && m->n_owned > n) {
        set_error("aica_bin_molecules: n_owned %lld exceeds the %lld molecules", (long long)m->n_owned, (long long)n);
        return AICA_ERR_INVALID_ARG;
    }
    a.n_owned = m->n_owned >= 0 ? m->n_owned : n;
    m->ghosts = m->n_owned >= 0 && m->n_owned < n;
    for (int d = 0; d < 3; ++d) {
        a.glo_f[d] = (float)m->glo[d];
        a.gh_f[d] = (float)m->gh[d];
        a.inv_gh_f[d] = (float)(1.0 / m->gh[d]);
    }
    // the previous binning of the same molecules is a search hint (exact result regardless)
    a.hint = (m->hint_valid && m->n_mol_prev == n) ? m->cell_of.as<int>() : nullptr;
    a.nbr_off = m->nbr_off.as<int>();
    a.nbr = m->nbr.as<int>();
    a.miss = m->miss.as<int>();
    a.cell_of = m->cell_of.as<int>();
    a.flags = m->flags.as<unsigned>();
    int *cnt = m->fill.as<int>();
    int *off = m->cell_off.as<int>();
    a.cnt = cnt;
    a.inv = m->inv.as<int>();
    // with deferred checks the error bits (flags[0]) accumulate until aica_check_status
    if (m->deferred) AICA_CUDA(cudaMemsetAsync(m->flags.as<unsigned>() + 1, 0, 12, st));
    else AICA_CUDA(cudaMemsetAsync(m->flags.p, 0, 16, st));
    AICA_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (C + 1), st));
    unsigned nb = (unsigned)((n + 255) / 256);
    if (n > 0) {
        // locate every molecule and count the cells' molecules
        if (a.hint) {
            AICA_CUDA(cudaMemsetAsync(m->miss.p, 0, sizeof(int), st));
            bin_locate_hint<<<nb, 256, 0, st>>>(a);
            bin_locate_miss<<<152 * 4, 256, 0, st>>>(a);
            m->launches += 2;
        } else {
            bin_locate<<<nb, 256, 0, st>>>(a);
            m->launches += 1;
        }
    }
    m->launches += exclusive_scan_1pass(cnt, C, off, m->scan_state.as<unsigned long long>(), m->flags.as<unsigned>(),
                                        kFlagTimeout, st);
    // wide cells are sorted in place in `order`; narrow ones go from `unsorted` to `order`
    const bool wide = (double)n > 6.0 * (double)C;
    int *slots_out = wide ? m->order.as<int>() : m->unsorted.as<int>();
    if (n > 0) {
        bin_scatter_down<<<nb, 256, 0, st>>>(a.cell_of, n, off, cnt, slots_out, wide ? nullptr : m->ucell.as<int>());
        m->launches += 1;
    }
    // order by original index, gather, bounding spheres: per slot for cells of
    // a few molecules, else per cell with a warp each
    if (C > 0 && n > 0) {
        if (wide) {
            const unsigned gc = (unsigned)std::min<int64_t>(((int64_t)C * 32 + 255) / 256, 152 * 16);
            bin_cells<32><<<gc, 256, 0, st>>>(a, off, C, m->order.as<int>(), m->xs64.as<double>(), m->xloc.as<float4>(), m->sph.as<float4>());
        } else {
            bin_slots<<<nb, kSlotWarps * 32, 0, st>>>(a, off, off + C, slots_out, m->ucell.as<int>(), m->order.as<int>(), m->xs64.as<double>(), m->xloc.as<float4>(), m->sph.as<float4>());
        }
        m->launches += 1;
    }
    m->n_mol_prev = n;
    m->hint_valid = true;
    AICA_CUDA(cudaGetLastError());
    if (cell_of && n) AICA_CUDA(cudaMemcpyAsync(cell_of, a.cell_of, sizeof(int) * n, cudaMemcpyDeviceToDevice, st));
    if (order && n) AICA_CUDA(cudaMemcpyAsync(order, m->order.p, sizeof(int) * n, cudaMemcpyDeviceToDevice, st));
    if (cell_off) AICA_CUDA(cudaMemcpyAsync(cell_off, off, sizeof(int) * (C + 1), cudaMemcpyDeviceToDevice, st));
    m->binned = true;
    m->max_species = -1;
    if (!m->deferred) {
        unsigned flags[2] = {0, 0};
        AICA_CUDA(cudaMemcpyAsync(flags, m->flags.p, 2 * sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        AICA_CUDA(cudaStreamSynchronize(st));
        m->max_species = (int)flags[1];
        if (flags[0] & kFlagSpecies) {
            set_error("aica_bin_molecules: species index outside [0, %d)", kMaxSpecies);
            return AICA_ERR_INVALID_ARG;
        }
        if (flags[0] & kFlagOutside) {
            set_error("aica_bin_molecules: some molecules lie in no cell (cell_of = -1)");
            return AICA_ERR_OUTSIDE_MESH;
        }
        if (flags[0] & kFlagTimeout) {
            set_error("aica_bin_molecules: a wait between blocks of the cell-offset scan timed out");
            return AICA_ERR_CUDA;
        }
    }
    return AICA_OK;
}

// ------------------------------------------------------------ no allocation
// Workspace of aica_sort_by_cell_noalloc: per-cell counters (reused as slot
// fill counters after the prefix sum) and the prefix-sum tile totals.  A
// file-scope device array: host code must not take its address directly (the
// host-side name is not a device address); each device's address is looked
// up once with cudaGetSymbolAddress.
namespace {
constexpr int64_t kNoAllocMaxCells = 1 << 20;
constexpr int64_t kNoAllocWords = (kNoAllocMaxCells + 1) + (kNoAllocMaxCells + 1 + aica::kScanTile - 1) / aica::kScanTile + 8;
constexpr int kNoAllocMaxDevices = 64;
int *g_noalloc_dev[kNoAllocMaxDevices];   // device address of the workspace, per device
}  // namespace

static __device__ __align__(256) int g_noalloc_scratch[kNoAllocWords];

extern "C" aica_status aica_sort_by_cell_noalloc(const int32_t *cell_of, int64_t n, int64_t n_cells, int32_t *order,
                                                 int32_t *cell_off, void *stream) {
    AICA_RANGE("aica_sort_by_cell_noalloc");
    if (n < 0 || n > (int64_t(1) << 30) || n_cells < 1 || !cell_off || (n > 0 && (!cell_of || !order))) {
        set_error("aica_sort_by_cell_noalloc: bad arguments (n = %lld, n_cells = %lld)", (long long)n,
                  (long long)n_cells);
        return AICA_ERR_INVALID_ARG;
    }
    if (n_cells > kNoAllocMaxCells) {
        set_error("aica_sort_by_cell_noalloc: %lld cells exceed the fixed workspace (at most %lld)",
                  (long long)n_cells, (long long)kNoAllocMaxCells);
        return AICA_ERR_CAPACITY;
    }
    int dev = 0;
    AICA_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        set_error("aica_sort_by_cell_noalloc: device %d beyond %d", dev, kNoAllocMaxDevices);
        return AICA_ERR_INVALID_ARG;
    }
    if (!g_noalloc_dev[dev]) {    // once per device, with that device current
        void *p = nullptr;
        AICA_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_dev[dev] = static_cast<int *>(p);
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int C = (int)n_cells;
    int *cnt = g_noalloc_dev[dev];
    int *work = cnt + (kNoAllocMaxCells + 1);
    int *bad = cnt + (kNoAllocWords - 1);      // ids >= n_cells seen by this call (left out)
    AICA_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (C + 1), st));
    AICA_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), st));
    const unsigned nb = (unsigned)((n + 255) / 256);
    if (n > 0) bin_count<<<nb, 256, 0, st>>>(cell_of, n, C, cnt, bad);
    exclusive_scan<int, int>(cnt, C, cell_off, work, st);
    AICA_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (C + 1), st));
    if (n > 0) {
        bin_scatter<<<nb, 256, 0, st>>>(cell_of, n, C, cell_off, cnt, order);
        bin_fixup<<<(C + kFixWarps - 1) / kFixWarps, kFixWarps * 32, 0, st>>>(cell_off, C, order);
    }
    AICA_CUDA(cudaGetLastError());
    return AICA_OK;
}
