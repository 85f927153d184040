// Interaction-list builder (steps a2, a3): direct interaction lists (§2.2,
// App. A.1) and periodic referred cells with their real-cell lists (§2.2.1,
// App. A.2), plus the per-cell pair schedule the force kernels walk.
//
// The paper builds DILs by a vertex-vertex search and notes it can miss
// slivers of twisted cells (§2.2); by default a cell pair is listed iff the
// exact minimum distance between the two closed triangulated polyhedra is
// below rc + skin.  The paper's vertex-vertex criterion is available as
// AICA_DIL_VERTEX (for the comparison of §2.2 and §2.4).  The paper's iterated referral across patch segments (App. A.2)
// reduces, for a translation-periodic box on one device, to enumerating
// image vectors n directly: the result does not depend on evaluation order.
//
// Kernels
//   lst_query<0/1>  warp per query cell A: candidates (B, n) from a centroid
//                   bucket grid, FP32 sphere / vertex / bounding-box filters,
//                   FP32 min distance with early exit, FP64 recomputation when
//                   the FP32 value is within 1e-3 (rc+skin)^2 of the cut;
//                   pass 0 counts, pass 1 writes keys (image, B)
//   lst_sort        per-segment bitonic sort of the keys
//   lst_classify    per-cell counts of DIL entries, referred cells, entries
//   lst_fill        CSR outputs and the pair schedule (each cell's DIL, then
//                   the periodic image pairs it owns: every image pair once)
#include <math.h>

#include <algorithm>
#include <vector>

#include "aica_internal.cuh"
#include "geom.cuh"
#include "scan.cuh"

namespace aica {
namespace {

constexpr int kQWarps = 4;
constexpr int kSortMax = 4096;

struct QArgs {
    int C;
    int vertex_only;      // the paper's vertex-vertex criterion instead of the minimum distance
    double thr2;
    float thr, thr2_lo, thr2_hi;
    double L[3];
    float Lf[3];
    int per[3];
    int G[3];
    double g0[3], gh[3];
    const int *bkt_off, *bkt_cells;
    float rad_max;
    const int *tri_off, *vtx_off, *edg_off, *orgk;
    const float *tri32, *vtx32, *edg32, *ctr32, *rad32;
    const double *tri, *vtx, *edg, *ctr;
    int *count;
    const long long *seg_off;
    unsigned long long *keys;
    unsigned long long *ties;
};

__device__ __forceinline__ V3<float> ldf(const float *p) { return {p[0], p[1], p[2]}; }
__device__ __forceinline__ V3<double> ldd(const double *p) { return {p[0], p[1], p[2]}; }

__device__ __forceinline__ int floordiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// FP64 minimum squared distance between cell A and cell B shifted by s.
__device__ __noinline__ double min_d2_f64(const QArgs &a, int A, int B, V3<double> s) {
    double m = INFINITY;
    for (int i = a.vtx_off[A]; i < a.vtx_off[A + 1]; ++i) {
        V3<double> p = ldd(a.vtx + 3 * i);
        for (int t = a.tri_off[B]; t < a.tri_off[B + 1]; ++t) {
            const double *T = a.tri + 9 * t;
            m = fmin(m, d2_point_triangle(p, ldd(T) + s, ldd(T + 3) + s, ldd(T + 6) + s));
        }
    }
    for (int i = a.vtx_off[B]; i < a.vtx_off[B + 1]; ++i) {
        V3<double> p = ldd(a.vtx + 3 * i) + s;
        for (int t = a.tri_off[A]; t < a.tri_off[A + 1]; ++t) {
            const double *T = a.tri + 9 * t;
            m = fmin(m, d2_point_triangle(p, ldd(T), ldd(T + 3), ldd(T + 6)));
        }
    }
    for (int i = a.edg_off[A]; i < a.edg_off[A + 1]; ++i) {
        V3<double> p0 = ldd(a.edg + 6 * i), p1 = ldd(a.edg + 6 * i + 3);
        for (int j = a.edg_off[B]; j < a.edg_off[B + 1]; ++j)
            m = fmin(m, d2_segment_segment(p0, p1, ldd(a.edg + 6 * j) + s, ldd(a.edg + 6 * j + 3) + s));
    }
    return m;
}

// FP64 smallest vertex-vertex squared distance between cell A and cell B shifted by s.
__device__ __noinline__ double min_vv_d2_f64(const QArgs &a, int A, int B, V3<double> s) {
    double m = INFINITY;
    for (int i = a.vtx_off[A]; i < a.vtx_off[A + 1]; ++i) {
        const V3<double> p = ldd(a.vtx + 3 * i);
        for (int j = a.vtx_off[B]; j < a.vtx_off[B + 1]; ++j) {
            const V3<double> q = ldd(a.vtx + 3 * j) + s;
            const double dx = __dsub_rn(p.x, q.x), dy = __dsub_rn(p.y, q.y), dz = __dsub_rn(p.z, q.z);
            m = fmin(m, __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
        }
    }
    return m;
}

struct WarpA {
    const float *T, *V, *E;   // shared: A's triangles, vertices, edges in A's frame
    int nt, nv, ne;
    V3<float> lo, hi, c;
    float rad;
    int ok[3];
};

// Decide whether cell B shifted by image n is within rc + skin of cell A:
// bit 0 = listed, bit 1 = an FP64 decision within 1e-9 (rc+skin)^2 of the cut.
// One out-of-line function serves both passes, so both make the same choices.
__device__ __noinline__ int decide(const QArgs &a, const WarpA &w, int A, int B, int nx, int ny, int nz) {
    // B's frame relative to A's: integer origin difference (exact) plus n.L
    V3<float> D = {(float)(a.orgk[3 * B] - a.orgk[3 * A]) * (1.0f / 1024.0f) + (float)nx * a.Lf[0],
                   (float)(a.orgk[3 * B + 1] - a.orgk[3 * A + 1]) * (1.0f / 1024.0f) + (float)ny * a.Lf[1],
                   (float)(a.orgk[3 * B + 2] - a.orgk[3 * A + 2]) * (1.0f / 1024.0f) + (float)nz * a.Lf[2]};
    V3<float> cB = ldf(a.ctr32 + 3 * B) + D - w.c;
    float R = a.thr + w.rad + a.rad32[B];
    float dc2 = dot3(cB, cB);
    if (dc2 > R * R * 1.0001f + 1e-4f) return 0;
    // vertex-vertex distances (an upper bound on the minimum) and B's box
    float m = INFINITY;
    V3<float> blo = {INFINITY, INFINITY, INFINITY}, bhi = {-INFINITY, -INFINITY, -INFINITY};
    int v0 = a.vtx_off[B], v1 = a.vtx_off[B + 1];
    for (int i = v0; i < v1; ++i) {
        V3<float> q = ldf(a.vtx32 + 3 * i) + D;
        blo = {fminf(blo.x, q.x), fminf(blo.y, q.y), fminf(blo.z, q.z)};
        bhi = {fmaxf(bhi.x, q.x), fmaxf(bhi.y, q.y), fmaxf(bhi.z, q.z)};
        for (int k = 0; k < w.nv; ++k) {
            V3<float> d = q - ldf(w.V + 3 * k);
            m = fminf(m, dot3(d, d));
        }
    }
    if (a.vertex_only) {
        if (m < a.thr2_lo) return 1;
        if (m > a.thr2_hi) return 0;
        V3<double> s = {nx * a.L[0], ny * a.L[1], nz * a.L[2]};
        const double d2 = min_vv_d2_f64(a, A, B, s);
        return (d2 < a.thr2 ? 1 : 0) | (fabs(d2 - a.thr2) <= 1e-9 * a.thr2 ? 2 : 0);
    }
    if (m < a.thr2_lo) return 1;
    float gx = fmaxf(0.f, fmaxf(blo.x - w.hi.x, w.lo.x - bhi.x));
    float gy = fmaxf(0.f, fmaxf(blo.y - w.hi.y, w.lo.y - bhi.y));
    float gz = fmaxf(0.f, fmaxf(blo.z - w.hi.z, w.lo.z - bhi.z));
    if (gx * gx + gy * gy + gz * gz > a.thr2_hi) return 0;
    // FP32 minimum distance with early acceptance
    for (int t = a.tri_off[B]; t < a.tri_off[B + 1]; ++t) {
        const float *T = a.tri32 + 9 * t;
        V3<float> p0 = ldf(T) + D, p1 = ldf(T + 3) + D, p2 = ldf(T + 6) + D;
        for (int k = 0; k < w.nv; ++k) m = fminf(m, d2_point_triangle(ldf(w.V + 3 * k), p0, p1, p2));
        if (m < a.thr2_lo) return 1;
    }
    for (int i = v0; i < v1; ++i) {
        V3<float> q = ldf(a.vtx32 + 3 * i) + D;
        for (int t = 0; t < w.nt; ++t)
            m = fminf(m, d2_point_triangle(q, ldf(w.T + 9 * t), ldf(w.T + 9 * t + 3), ldf(w.T + 9 * t + 6)));
        if (m < a.thr2_lo) return 1;
    }
    for (int j = a.edg_off[B]; j < a.edg_off[B + 1]; ++j) {
        V3<float> q0 = ldf(a.edg32 + 6 * j) + D, q1 = ldf(a.edg32 + 6 * j + 3) + D;
        for (int k = 0; k < w.ne; ++k)
            m = fminf(m, d2_segment_segment(ldf(w.E + 6 * k), ldf(w.E + 6 * k + 3), q0, q1));
        if (m < a.thr2_lo) return 1;
    }
    if (m > a.thr2_hi) return 0;
    // close to the cut: decide in FP64 on the original coordinates
    V3<double> s = {nx * a.L[0], ny * a.L[1], nz * a.L[2]};
    double d2 = min_d2_f64(a, A, B, s);
    return (d2 < a.thr2 ? 1 : 0) | (fabs(d2 - a.thr2) <= 1e-9 * a.thr2 ? 2 : 0);
}

__device__ __forceinline__ unsigned long long make_key(int B, int nx, int ny, int nz) {
    // sort key: image n' = -n lexicographic, then B
    unsigned nk = ((unsigned)(-nx + 128) << 16) | ((unsigned)(-ny + 128) << 8) | (unsigned)(-nz + 128);
    return ((unsigned long long)nk << 32) | (unsigned)B;
}

template <int PASS>
__global__ void __launch_bounds__(32 * kQWarps) lst_query(QArgs a) {
    __shared__ float sh[kQWarps][kMaxTri * 9 + kMaxVtx * 3 + kMaxEdg * 6];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpA w;
    w.T = sh[wid];
    w.V = w.T + kMaxTri * 9;
    w.E = w.V + kMaxVtx * 3;
    float *T = sh[wid], *V = T + kMaxTri * 9, *E = V + kMaxVtx * 3;
    for (int A = blockIdx.x * kQWarps + wid; A < a.C; A += gridDim.x * kQWarps) {
        int t0 = a.tri_off[A], v0 = a.vtx_off[A], e0 = a.edg_off[A];
        w.nt = a.tri_off[A + 1] - t0;
        w.nv = a.vtx_off[A + 1] - v0;
        w.ne = a.edg_off[A + 1] - e0;
        __syncwarp();
        for (int i = lane; i < 9 * w.nt; i += 32) T[i] = a.tri32[9 * t0 + i];
        for (int i = lane; i < 3 * w.nv; i += 32) V[i] = a.vtx32[3 * v0 + i];
        for (int i = lane; i < 6 * w.ne; i += 32) E[i] = a.edg32[6 * e0 + i];
        __syncwarp();
        w.lo = {INFINITY, INFINITY, INFINITY};
        w.hi = {-INFINITY, -INFINITY, -INFINITY};
        for (int k = 0; k < w.nv; ++k) {
            V3<float> q = ldf(V + 3 * k);
            w.lo = {fminf(w.lo.x, q.x), fminf(w.lo.y, q.y), fminf(w.lo.z, q.z)};
            w.hi = {fmaxf(w.hi.x, q.x), fmaxf(w.hi.y, q.y), fmaxf(w.hi.z, q.z)};
        }
        w.c = ldf(a.ctr32 + 3 * A);
        w.rad = a.rad32[A];
        // bucket range of the query sphere around A's vertex mean
        int b0[3], b1[3];
        double Rq = (double)a.thr + (double)w.rad + (double)a.rad_max;
        for (int d = 0; d < 3; ++d) {
            double cA = a.ctr[3 * A + d];
            b0[d] = (int)floor((cA - Rq - a.g0[d]) / a.gh[d]);
            b1[d] = (int)floor((cA + Rq - a.g0[d]) / a.gh[d]);
            if (!a.per[d]) {
                b0[d] = max(b0[d], 0);
                b1[d] = min(b1[d], a.G[d] - 1);
            }
        }
        int cnt = 0;
        long long wbase = PASS ? a.seg_off[A] : 0;
        for (int bx = b0[0]; bx <= b1[0]; ++bx) {
            int wx = bx - floordiv(bx, a.G[0]) * a.G[0], nx = a.per[0] ? floordiv(bx, a.G[0]) : 0;
            for (int by = b0[1]; by <= b1[1]; ++by) {
                int wy = by - floordiv(by, a.G[1]) * a.G[1], ny = a.per[1] ? floordiv(by, a.G[1]) : 0;
                for (int bz = b0[2]; bz <= b1[2]; ++bz) {
                    int wz = bz - floordiv(bz, a.G[2]) * a.G[2], nz = a.per[2] ? floordiv(bz, a.G[2]) : 0;
                    int b = (wx * a.G[1] + wy) * a.G[2] + wz;
                    int s = a.bkt_off[b], e = a.bkt_off[b + 1];
                    for (int base = s; base < e; base += 32) {
                        int i = base + lane;
                        int dec = 0;
                        int B = -1;
                        if (i < e) {
                            B = a.bkt_cells[i];
                            if (!(B == A && nx == 0 && ny == 0 && nz == 0)) dec = decide(a, w, A, B, nx, ny, nz);
                        }
                        bool acc = dec & 1;
                        unsigned bal = __ballot_sync(0xffffffffu, acc);
                        if (PASS == 0 && (dec & 2)) atomicAdd(a.ties, 1ull);
                        if (PASS == 1 && acc) {
                            long long slot = wbase + cnt + __popc(bal & ((1u << lane) - 1u));
                            if (slot < a.seg_off[A + 1]) a.keys[slot] = make_key(B, nx, ny, nz);
                        }
                        cnt += __popc(bal);
                    }
                }
            }
        }
        if (PASS == 0 && lane == 0) a.count[A] = cnt;
        __syncwarp();
    }
}

__global__ void __launch_bounds__(256) lst_sort(const long long *seg_off, unsigned long long *keys, int C,
                                                unsigned *flags) {
    __shared__ unsigned long long s[kSortMax];
    for (int A = blockIdx.x; A < C; A += gridDim.x) {
        long long s0 = seg_off[A];
        int len = (int)(seg_off[A + 1] - s0);
        if (len <= 1) continue;
        if (len > kSortMax) {
            if (threadIdx.x == 0) atomicOr(flags, kFlagCapacity);
            continue;
        }
        int P = 1;
        while (P < len) P <<= 1;
        for (int i = threadIdx.x; i < P; i += blockDim.x) s[i] = i < len ? keys[s0 + i] : ~0ull;
        __syncthreads();
        for (int k = 2; k <= P; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = threadIdx.x; i < P; i += blockDim.x) {
                    int l = i ^ j;
                    if (l > i) {
                        unsigned long long x = s[i], y = s[l];
                        bool up = (i & k) == 0;
                        if ((x > y) == up) {
                            s[i] = y;
                            s[l] = x;
                        }
                    }
                }
                __syncthreads();
            }
        for (int i = threadIdx.x; i < len; i += blockDim.x) keys[s0 + i] = s[i];
        __syncthreads();
    }
}

__device__ __forceinline__ void key_fields(unsigned long long k, int &B, int &npx, int &npy, int &npz) {
    B = (int)(k & 0xffffffffu);
    unsigned nk = (unsigned)(k >> 32);
    npx = (int)((nk >> 16) & 0xff) - 128;
    npy = (int)((nk >> 8) & 0xff) - 128;
    npz = (int)(nk & 0xff) - 128;
}

// The pair schedule evaluates every periodic image pair once, with Newton's
// third law: of the mirror entries (A sees B at +n) and (B sees A at -n) it
// keeps the one with B > A, or B == A and n lexicographically positive.
__device__ __forceinline__ bool canonical_image(int A, int B, int nx, int ny, int nz) {
    if (B != A) return B > A;
    return nx > 0 || (nx == 0 && (ny > 0 || (ny == 0 && nz > 0)));
}

__global__ void lst_classify(const long long *seg_off, const unsigned long long *keys, int C, int *c_dil, int *c_re,
                             int *c_rc, int *c_rw) {
    int A = blockIdx.x * blockDim.x + threadIdx.x;
    if (A >= C) return;
    int nd = 0, nr = 0, ng = 0, nw = 0;
    int px = 1000, py = 0, pz = 0;
    for (long long i = seg_off[A]; i < seg_off[A + 1]; ++i) {
        int B, x, y, z;
        key_fields(keys[i], B, x, y, z);
        if (x == 0 && y == 0 && z == 0) {
            nd += B > A;
        } else {
            nr++;
            nw += canonical_image(A, B, -x, -y, -z);
            if (x != px || y != py || z != pz) ng++;
            px = x; py = y; pz = z;
        }
    }
    c_dil[A] = nd;
    c_re[A] = nr;
    c_rc[A] = ng;
    c_rw[A] = nw;
}

struct FillArgs {
    int C;
    const long long *seg_off;
    const unsigned long long *keys;
    const int *o_dil, *o_re, *o_rc, *o_rw;
    const int *orgk;
    double L[3];
    int *dil_ids, *ref_src, *ref_n, *ref_off, *ref_ids;
    int *work_off, *work_split;
    WorkEntry *work;
};

__global__ void lst_fill(FillArgs f) {
    int A = blockIdx.x * blockDim.x + threadIdx.x;
    if (A > f.C) return;
    if (A == f.C) {
        f.work_off[f.C] = f.o_dil[f.C] + f.o_rw[f.C];
        f.ref_off[f.o_rc[f.C]] = f.o_re[f.C];
        return;
    }
    int wd = f.o_dil[A], wr = f.o_re[A], g = f.o_rc[A];
    int nd = f.o_dil[A + 1] - wd;
    int w0 = wd + f.o_rw[A];
    f.work_off[A] = w0;
    f.work_split[A] = w0 + nd;
    int id = 0, ir = 0, iw = 0;
    int px = 1000, py = 0, pz = 0;
    for (long long i = f.seg_off[A]; i < f.seg_off[A + 1]; ++i) {
        int B, x, y, z;
        key_fields(f.keys[i], B, x, y, z);
        int slot;
        if (x == 0 && y == 0 && z == 0) {
            if (B <= A) continue;
            f.dil_ids[wd + id] = B;
            slot = w0 + id;
            id++;
        } else {
            if (x != px || y != py || z != pz) {
                f.ref_src[g] = A;
                f.ref_n[3 * g] = x;
                f.ref_n[3 * g + 1] = y;
                f.ref_n[3 * g + 2] = z;
                f.ref_off[g] = wr + ir;
                g++;
                px = x; py = y; pz = z;
            }
            f.ref_ids[wr + ir] = B;
            ir++;
            if (!canonical_image(A, B, -x, -y, -z)) continue;
            slot = w0 + nd + iw;
            iw++;
        }
        // partner B seen from A: its molecules shifted by n = -n'
        int nx = -x, ny = -y, nz = -z;
        f.work[slot] = WorkEntry{B, pack_n(nx, ny, nz)};
    }
}

// Runs of the pair schedule: consecutive entries of one cell whose partner
// cells are consecutive, share the image vector and share the molecule-frame
// origin collapse into one run (first partner, count): their molecules are
// one contiguous range of the binned order under one shift.
__device__ __forceinline__ bool run_continues(const WorkEntry &p, const WorkEntry &e, const int *orgm, int len) {
    if (e.j != p.j + 1 || e.n != p.n || len >= 256) return false;
    const int *a = orgm + 3 * p.j, *b = orgm + 3 * e.j;
    return a[0] == b[0] && a[1] == b[1] && a[2] == b[2];
}

__global__ void lst_runs(const int *work_off, const WorkEntry *work, const int *orgm, int C, const int *run_off,
                         int *run_cnt, RunEntry *runs) {
    const int A = blockIdx.x * blockDim.x + threadIdx.x;
    if (A >= C) return;
    const int r = run_off ? run_off[A] : 0;
    int nr = 0, len = 0, j0 = 0;
    WorkEntry p{0, 0};
    auto flush = [&]() {
        if (runs) runs[r + nr] = RunEntry{j0, (p.n & 0xffffff) | ((len - 1) << 24)};
        ++nr;
    };
    for (int e = work_off[A]; e < work_off[A + 1]; ++e) {
        const WorkEntry w = work[e];
        if (len > 0 && run_continues(p, w, orgm, len)) {
            ++len;
        } else {
            if (len > 0) flush();
            j0 = w.j;
            len = 1;
        }
        p = w;
    }
    if (len > 0) flush();
    if (run_cnt) run_cnt[A] = nr;
}

// ------------------------------------------------------------ cluster schedule
// The FP32 box-periodic pair kernel works on clusters (runs of consecutive
// cells, mesh.cu).  Every cell-level schedule entry (I -> J, n) has J >= I
// (the DIL half rule and the canonical image rule), so with contiguous
// clusters the cluster pair (cl(I), cl(J), n) has cl(J) >= cl(I): each owner
// cluster A collects its own cells' entries only.  For B = A with n != 0 the
// pairs of (A, A, n) and (A, A, -n) are mirror images; the lexicographically
// positive image is kept.  B = A with n = 0 (pairs inside the cluster) is
// implicit.  Keys (n << 32 | B) are sorted and made unique per cluster; runs
// are consecutive partner clusters under one image and one molecule frame.
// The full list (for the FP64 refinement of single molecules) holds, for each
// cluster, every (partner cluster, image) whose molecules can lie within the
// cut-off of its molecules: its own keys and the mirrors of the keys that
// name it.
constexpr int kClKeys = 2048, kClWarps = 4;
constexpr unsigned long long kNoKey = ~0ull;

__device__ __forceinline__ int32_t neg_n(int32_t p) {
    return pack_n(-unpack_n(p, 0), -unpack_n(p, 1), -unpack_n(p, 2));
}
__device__ __forceinline__ unsigned long long cl_key(int B, int32_t n) {
    return ((unsigned long long)(n & 0xffffff) << 32) | (unsigned)B;
}

// Ascending bitonic sort of b[0, P), P a power of two, by one warp.
__device__ void warp_bitonic(unsigned long long *b, int P, int lane) {
    for (int size = 2; size <= P; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = lane; i < P / 2; i += 32) {
                const int lo = 2 * i - (i & (stride - 1)), hi = lo + stride;
                const bool up = (lo & size) == 0;
                const unsigned long long x = b[lo], y = b[hi];
                if ((x > y) == up) {
                    b[lo] = y;
                    b[hi] = x;
                }
            }
            __syncwarp();
        }
}

struct ClArgs {
    int ncl;
    const int *cl_first, *cl_of, *work_off, *orgm;
    const WorkEntry *work;
    int *run_cnt, *own_cnt, *rev_cnt;            // pass 0
    const int *run_off, *full_off;               // pass 1
    int *cursor;
    ClRun *runs;
    unsigned long long *full;
    unsigned *flags;
    const double *orgm64;
    double L[3];
    double qs, qsi, dmax;        // 2^q, 2^-q, largest |shift| with an exact FP32 hi part
};

// The run of clusters B0 .. B0 + len - 1 under image n, seen from cluster A.
__device__ ClRun make_clrun(const ClArgs &a, int A, int B0, int len, int32_t n) {
    const int c0 = a.cl_first[B0], c1 = a.cl_first[B0 + len], cA = a.cl_first[A];
    const double *oB = a.orgm64 + 3 * c0, *oA = a.orgm64 + 3 * cA;
    float h[3], l[3];
    int code = 0;
    for (int d = 0; d < 3; ++d) {
        const int nd = unpack_n(n, d);
        const double D = (oB[d] - oA[d]) + (double)nd * a.L[d];
        if (!(fabs(D) < a.dmax)) atomicOr(a.flags, kFlagCapacity);
        const double hi = rint(D * a.qs) * a.qsi;
        h[d] = (float)hi;
        l[d] = (float)(D - hi);
        if (nd < -8 || nd > 7) atomicOr(a.flags, kFlagCapacity);
        code |= (nd & 15) << (4 * d);
    }
    if (c1 - c0 > 4095) atomicOr(a.flags, kFlagCapacity);
    ClRun r;
    r.dh = make_float4(h[0], h[1], h[2], __int_as_float(c0));
    r.dl = make_float4(l[0], l[1], l[2], __int_as_float((c1 - c0) | (code << 12)));
    return r;
}

__device__ __forceinline__ bool same_frame(const int *orgm, const int *cl_first, int B0, int B1) {
    const int *a = orgm + 3 * cl_first[B0], *b = orgm + 3 * cl_first[B1];
    return a[0] == b[0] && a[1] == b[1] && a[2] == b[2];
}

template <int PASS>
__global__ void __launch_bounds__(kClWarps * 32) cl_sched(ClArgs a) {
    extern __shared__ unsigned long long cl_sh[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long *b = cl_sh + (size_t)w * kClKeys;
    for (int A = blockIdx.x * kClWarps + w; A < a.ncl; A += gridDim.x * kClWarps) {
        const int e0 = a.work_off[a.cl_first[A]], e1 = a.work_off[a.cl_first[A + 1]], m = e1 - e0;
        if (m > kClKeys) {
            if (lane == 0) atomicOr(a.flags, kFlagCapacity);
            continue;
        }
        int P = 2;
        while (P < m) P <<= 1;
        for (int i = lane; i < P; i += 32) {
            unsigned long long key = kNoKey;
            if (i < m) {
                const WorkEntry e = a.work[e0 + i];
                const int B = a.cl_of[e.j];
                int32_t n = e.n & 0xffffff;
                if (B != A) key = cl_key(B, n);
                else if (n != 0) {
                    const int x = unpack_n(n, 0), y = unpack_n(n, 1), z = unpack_n(n, 2);
                    const bool pos = x > 0 || (x == 0 && (y > 0 || (y == 0 && z > 0)));
                    key = cl_key(A, pos ? n : neg_n(n));
                }
            }
            b[i] = key;
        }
        __syncwarp();
        warp_bitonic(b, P, lane);
        if (lane == 0) {
            int nu = 0, nr = 0, len = 0, B0 = 0, Bp = 0;
            int32_t np = 0;
            const int r0 = PASS == 1 ? a.run_off[A] : 0, f0 = PASS == 1 ? a.full_off[A] : 0;
            for (int i = 0; i < m && b[i] != kNoKey; ++i) {
                if (i > 0 && b[i] == b[i - 1]) continue;
                const int B = (int)(b[i] & 0xffffffffu);
                const int32_t n = (int32_t)(b[i] >> 32);
                if (PASS == 0) {
                    atomicAdd(a.rev_cnt + B, 1);
                } else {
                    a.full[f0 + nu] = b[i];
                    a.full[atomicAdd(a.cursor + B, 1)] = cl_key(A, neg_n(n));
                }
                ++nu;
                const bool cont = len > 0 && n == np && B == Bp + 1 && len < 255 && same_frame(a.orgm, a.cl_first, B0, B);
                if (cont) {
                    ++len;
                } else {
                    if (len > 0) {
                        if (PASS == 1) a.runs[r0 + nr] = make_clrun(a, A, B0, len, np);
                        ++nr;
                    }
                    B0 = B;
                    len = 1;
                }
                Bp = B;
                np = n;
            }
            if (len > 0) {
                if (PASS == 1) a.runs[r0 + nr] = make_clrun(a, A, B0, len, np);
                ++nr;
            }
            if (PASS == 0) {
                a.run_cnt[A] = nr;
                a.own_cnt[A] = nu;
            }
        }
        __syncwarp();
    }
}

// rev_cnt[A] += own_cnt[A]: the full list of A holds its own keys and the mirrors naming it
__global__ void add_counts(int ncl, const int *own_cnt, int *rev_cnt) {
    const int A = blockIdx.x * blockDim.x + threadIdx.x;
    if (A < ncl) rev_cnt[A] += own_cnt[A];
}

__global__ void cl_cursor(int ncl, const int *full_off, const int *own_cnt, int *cursor) {
    const int A = blockIdx.x * blockDim.x + threadIdx.x;
    if (A < ncl) cursor[A] = full_off[A] + own_cnt[A];
}

// Sort each cluster's full list (its reverse entries arrive in any order).
__global__ void __launch_bounds__(kClWarps * 32) cl_sort_full(int ncl, const int *full_off, unsigned long long *full,
                                                               unsigned *flags) {
    extern __shared__ unsigned long long cl_sh[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long *b = cl_sh + (size_t)w * kClKeys;
    for (int A = blockIdx.x * kClWarps + w; A < ncl; A += gridDim.x * kClWarps) {
        const int f0 = full_off[A], m = full_off[A + 1] - f0;
        if (m > kClKeys) {
            if (lane == 0) atomicOr(flags, kFlagCapacity);
            continue;
        }
        int P = 2;
        while (P < m) P <<= 1;
        for (int i = lane; i < P; i += 32) b[i] = i < m ? full[f0 + i] : kNoKey;
        __syncwarp();
        warp_bitonic(b, P, lane);
        for (int i = lane; i < m; i += 32) full[f0 + i] = b[i];
        __syncwarp();
    }
}

}  // namespace
}  // namespace aica

namespace aica {
// Build the cluster schedule of the FP32 box-periodic kernel (see cl_sched)
// from the cell-level work entries.  Leaves n_cl_runs = -1 (the FP32 forces
// then use the cell kernel) under general referring transforms or the
// vertex criterion, when a cluster has more entries than a warp sorts in
// shared memory, or when the exact-separation bound of the binned
// coordinates does not cover the cut-off.
aica_status build_cluster_schedule(aica_mesh *m, cudaStream_t st) {
    m->n_cl_runs = -1;
    m->n_cl_full = 0;
    const int ncl = (int)m->n_cl;
    // the cluster kernel evaluates every pair within rc of two partner
    // clusters: that is the method's pair set only when the cell lists are
    // complete (minimum-distance criterion), not under the vertex criterion
    if (ncl < 1 || !m->xf_gen.empty() || m->criterion != AICA_DIL_MIN_DISTANCE) return AICA_OK;
    if (!(m->max_mlocal + m->rc + m->skin < ldexp(1.0, 24 - m->qexp) * 0.999)) return AICA_OK;
    DevBuf cnt, sw;
    AICA_CUDA(cnt.reserve(sizeof(int) * 4 * (size_t)(ncl + 1)));
    AICA_CUDA(sw.reserve(sizeof(int) * (scan_work_items(ncl) + 8)));
    int *run_cnt = cnt.as<int>(), *own_cnt = run_cnt + (ncl + 1), *rev_cnt = own_cnt + (ncl + 1),
        *cursor = rev_cnt + (ncl + 1);
    AICA_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int) * 4 * (size_t)(ncl + 1), st));
    AICA_CUDA(cudaMemsetAsync(m->flags.p, 0, sizeof(unsigned), st));
    const size_t shm = sizeof(unsigned long long) * kClWarps * kClKeys;
    AICA_CUDA(cudaFuncSetAttribute(cl_sched<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    AICA_CUDA(cudaFuncSetAttribute(cl_sched<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    AICA_CUDA(cudaFuncSetAttribute(cl_sort_full, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    const unsigned grid = (unsigned)std::min<int64_t>((ncl + kClWarps - 1) / kClWarps, 152 * 8);
    ClArgs a{};
    a.ncl = ncl;
    a.cl_first = m->cl_first.as<int>();
    a.cl_of = m->cl_of.as<int>();
    a.work_off = m->work_off.as<int>();
    a.orgm = m->orgm.as<int>();
    a.work = m->work.as<WorkEntry>();
    a.run_cnt = run_cnt;
    a.own_cnt = own_cnt;
    a.rev_cnt = rev_cnt;
    a.flags = m->flags.as<unsigned>();
    a.orgm64 = m->orgm64.as<double>();
    for (int d = 0; d < 3; ++d) a.L[d] = m->box.periodic[d] ? m->box.L[d] : 0.0;
    a.qs = ldexp(1.0, m->qexp);
    a.qsi = ldexp(1.0, -m->qexp);
    a.dmax = ldexp(1.0, 24 - m->qexp) * 0.999;
    cl_sched<0><<<grid, kClWarps * 32, shm, st>>>(a);
    // full list sizes: own keys + mirrors
    AICA_CUDA(m->cl_run_off.reserve(sizeof(int) * (ncl + 1)));
    AICA_CUDA(m->cl_full_off.reserve(sizeof(int) * (ncl + 1)));
    m->launches += 1 + exclusive_scan<int, int>(run_cnt, ncl, m->cl_run_off.as<int>(), sw.as<int>(), st);
    add_counts<<<(ncl + 255) / 256, 256, 0, st>>>(ncl, own_cnt, rev_cnt);
    m->launches += 1 + exclusive_scan<int, int>(rev_cnt, ncl, m->cl_full_off.as<int>(), sw.as<int>(), st);
    int tot[2] = {0, 0};
    unsigned flags = 0;
    AICA_CUDA(cudaMemcpyAsync(&tot[0], m->cl_run_off.as<int>() + ncl, sizeof(int), cudaMemcpyDeviceToHost, st));
    AICA_CUDA(cudaMemcpyAsync(&tot[1], m->cl_full_off.as<int>() + ncl, sizeof(int), cudaMemcpyDeviceToHost, st));
    AICA_CUDA(cudaMemcpyAsync(&flags, m->flags.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    AICA_CUDA(cudaStreamSynchronize(st));
    if (flags & kFlagCapacity) {
        AICA_CUDA(cudaMemsetAsync(m->flags.p, 0, sizeof(unsigned), st));
        return AICA_OK;
    }
    AICA_CUDA(m->cl_runs.reserve(sizeof(ClRun) * std::max(tot[0], 1)));
    AICA_CUDA(m->cl_full.reserve(sizeof(unsigned long long) * std::max(tot[1], 1)));
    AICA_CUDA(m->cl_box.reserve(sizeof(float4) * 2 * (size_t)ncl));
    cl_cursor<<<(ncl + 255) / 256, 256, 0, st>>>(ncl, m->cl_full_off.as<int>(), own_cnt, cursor);
    a.run_off = m->cl_run_off.as<int>();
    a.full_off = m->cl_full_off.as<int>();
    a.cursor = cursor;
    a.runs = m->cl_runs.as<ClRun>();
    a.full = m->cl_full.as<unsigned long long>();
    cl_sched<1><<<grid, kClWarps * 32, shm, st>>>(a);
    cl_sort_full<<<grid, kClWarps * 32, shm, st>>>(ncl, m->cl_full_off.as<int>(), m->cl_full.as<unsigned long long>(),
                                                   m->flags.as<unsigned>());
    m->launches += 3;
    AICA_CUDA(cudaMemcpyAsync(&flags, m->flags.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    AICA_CUDA(cudaStreamSynchronize(st));
    if (flags & kFlagCapacity) {
        AICA_CUDA(cudaMemsetAsync(m->flags.p, 0, sizeof(unsigned), st));
        return AICA_OK;
    }
    m->n_cl_runs = tot[0];
    m->n_cl_full = tot[1];
    return AICA_OK;
}
}  // namespace aica

using namespace aica;

extern "C" aica_status aica_build_interaction_list(aica_mesh *m, double rc, double skin, void *stream) {
    return aica_build_interaction_list_ex(m, rc, skin, AICA_DIL_MIN_DISTANCE, stream);
}

extern "C" aica_status aica_build_interaction_list_ex(aica_mesh *m, double rc, double skin,
                                                      aica_dil_criterion criterion, void *stream) {
    AICA_RANGE("aica_build_interaction_list_ex");
    if (criterion != AICA_DIL_MIN_DISTANCE && criterion != AICA_DIL_VERTEX) {
        set_error("aica_build_interaction_list_ex: unknown criterion %d", (int)criterion);
        return AICA_ERR_INVALID_ARG;
    }
    if (m && !m->xf_gen.empty() && criterion != AICA_DIL_MIN_DISTANCE) {
        set_error("aica_build_interaction_list_ex: general transforms take the minimum-distance criterion only");
        return AICA_ERR_INVALID_ARG;
    }
    if (!m) { set_error("aica_build_interaction_list: mesh is NULL"); return AICA_ERR_INVALID_ARG; }
    if (!(rc > 0) || !(skin >= 0) || !isfinite(rc + skin)) {
        set_error("aica_build_interaction_list: need rc > 0 and skin >= 0");
        return AICA_ERR_INVALID_ARG;
    }
    double thr = rc + skin;
    for (int d = 0; d < 3; ++d)
        if (m->box.periodic[d] && !(thr < 0.5 * m->box.L[d])) {
            set_error("aica_build_interaction_list: rc + skin must be below L/2 on periodic axis %d", d);
            return AICA_ERR_INVALID_ARG;
        }
    cudaStream_t st = (cudaStream_t)stream;
    const int C = (int)m->n_cells;
    m->launches = 0;
    m->built = false;
    m->n_cl_runs = -1;

    // ---- centroid bucket grid (host): about one cell per bucket
    QArgs a{};
    double lo[3], hi[3], vol = 1;
    for (int d = 0; d < 3; ++d) {
        if (m->box.periodic[d]) {
            lo[d] = 0;
            hi[d] = m->box.L[d];
        } else {
            lo[d] = INFINITY;
            hi[d] = -INFINITY;
            for (int c = 0; c < C; ++c) {
                lo[d] = std::min(lo[d], m->h_ctr[3 * c + d]);
                hi[d] = std::max(hi[d], m->h_ctr[3 * c + d]);
            }
            hi[d] = std::max(hi[d], lo[d] + 1e-9);
        }
        vol *= hi[d] - lo[d];
    }
    double h0 = cbrt(vol / C);
    int64_t nb = 1;
    for (int d = 0; d < 3; ++d) {
        a.G[d] = std::max(1, std::min(2048, (int)floor((hi[d] - lo[d]) / h0)));
        a.g0[d] = lo[d];
        a.gh[d] = (hi[d] - lo[d]) / a.G[d];
        nb *= a.G[d];
    }
    std::vector<int> boff(nb + 1, 0), bcell(C), bidx(C);
    for (int c = 0; c < C; ++c) {
        int ix[3];
        for (int d = 0; d < 3; ++d)
            ix[d] = std::min(a.G[d] - 1, std::max(0, (int)floor((m->h_ctr[3 * c + d] - a.g0[d]) / a.gh[d])));
        bidx[c] = (ix[0] * a.G[1] + ix[1]) * a.G[2] + ix[2];
        boff[bidx[c] + 1]++;
    }
    for (int64_t b = 0; b < nb; ++b) boff[b + 1] += boff[b];
    {
        std::vector<int> fl(boff.begin(), boff.end() - 1);
        for (int c = 0; c < C; ++c) bcell[fl[bidx[c]]++] = c;
    }
    float rad_max = 0;
    for (int c = 0; c < C; ++c) rad_max = std::max(rad_max, (float)m->h_rad[c]);

    DevBuf d_boff, d_bcell, d_cnt, d_seg, d_keys, d_scan, d_ties;
    auto fail = [&](cudaError_t e, const char *w) {
        d_boff.release(); d_bcell.release(); d_cnt.release(); d_seg.release(); d_keys.release();
        d_scan.release(); d_ties.release();
        return cuda_fail(e, w);
    };
#define CK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) return fail(e_, #x); } while (0)
    CK(d_boff.reserve(sizeof(int) * (nb + 1)));
    CK(d_bcell.reserve(sizeof(int) * C));
    CK(cudaMemcpyAsync(d_boff.p, boff.data(), sizeof(int) * (nb + 1), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_bcell.p, bcell.data(), sizeof(int) * C, cudaMemcpyHostToDevice, st));
    CK(d_cnt.reserve(sizeof(int) * 4 * (C + 1)));
    CK(d_seg.reserve(sizeof(long long) * (C + 1)));
    CK(d_scan.reserve(sizeof(long long) * (scan_work_items(C) + 8)));
    CK(d_ties.reserve(sizeof(unsigned long long)));
    CK(cudaMemsetAsync(d_ties.p, 0, sizeof(unsigned long long), st));
    CK(cudaMemsetAsync(m->flags.p, 0, 16, st));

    a.C = C;
    a.vertex_only = criterion == AICA_DIL_VERTEX ? 1 : 0;
    a.thr = (float)thr;
    a.thr2 = thr * thr;
    a.thr2_lo = (float)(a.thr2 * (1 - 1e-3));
    a.thr2_hi = (float)(a.thr2 * (1 + 1e-3));
    for (int d = 0; d < 3; ++d) {
        a.L[d] = m->box.periodic[d] ? m->box.L[d] : 0.0;
        a.Lf[d] = (float)a.L[d];
        a.per[d] = m->box.periodic[d] ? 1 : 0;
    }
    a.bkt_off = d_boff.as<int>();
    a.bkt_cells = d_bcell.as<int>();
    a.rad_max = rad_max;
    a.tri_off = m->tri_off.as<int>(); a.vtx_off = m->vtx_off.as<int>(); a.edg_off = m->edg_off.as<int>();
    a.orgk = m->orgk.as<int>();
    a.tri32 = m->tri32.as<float>(); a.vtx32 = m->vtx32.as<float>(); a.edg32 = m->edg32.as<float>();
    a.ctr32 = m->ctr32.as<float>(); a.rad32 = m->rad32.as<float>();
    a.tri = m->tri.as<double>(); a.vtx = m->vtx.as<double>(); a.edg = m->edg.as<double>(); a.ctr = m->ctr.as<double>();
    a.count = d_cnt.as<int>();
    a.ties = d_ties.as<unsigned long long>();

    int qblocks = (int)std::min<int64_t>((C + kQWarps - 1) / kQWarps, 152 * 64);
    lst_query<0><<<qblocks, 32 * kQWarps, 0, st>>>(a);
    m->launches += 1;
    m->launches += exclusive_scan<long long, int>(d_cnt.as<int>(), C, d_seg.as<long long>(), d_scan.as<long long>(), st);
    long long total = 0;
    CK(cudaMemcpyAsync(&total, d_seg.as<long long>() + C, sizeof(long long), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    CK(d_keys.reserve(sizeof(unsigned long long) * std::max<long long>(total, 1)));
    a.seg_off = d_seg.as<long long>();
    a.keys = d_keys.as<unsigned long long>();
    lst_query<1><<<qblocks, 32 * kQWarps, 0, st>>>(a);
    lst_sort<<<(unsigned)std::min<int64_t>(C, 152 * 32), 256, 0, st>>>(a.seg_off, a.keys, C, m->flags.as<unsigned>());
    int *c_dil = d_cnt.as<int>(), *c_re = c_dil + (C + 1), *c_rc = c_re + (C + 1), *c_rw = c_rc + (C + 1);
    lst_classify<<<(C + 255) / 256, 256, 0, st>>>(a.seg_off, a.keys, C, c_dil, c_re, c_rc, c_rw);
    m->launches += 3;
    CK(m->dil_off.reserve(sizeof(int) * (C + 1)));
    CK(m->tmp.reserve(sizeof(int) * 3 * (C + 1) + sizeof(int) * (scan_work_items(C) + 8)));
    int *o_re = m->tmp.as<int>(), *o_rc = o_re + (C + 1), *o_rw = o_rc + (C + 1), *sw = o_rw + (C + 1);
    m->launches += exclusive_scan<int, int>(c_dil, C, m->dil_off.as<int>(), sw, st);
    m->launches += exclusive_scan<int, int>(c_re, C, o_re, sw, st);
    m->launches += exclusive_scan<int, int>(c_rc, C, o_rc, sw, st);
    m->launches += exclusive_scan<int, int>(c_rw, C, o_rw, sw, st);
    int tot[4];
    unsigned flags = 0;
    unsigned long long ties = 0;
    CK(cudaMemcpyAsync(&tot[0], m->dil_off.as<int>() + C, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&tot[1], o_re + C, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&tot[2], o_rc + C, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&tot[3], o_rw + C, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&flags, m->flags.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&ties, d_ties.p, sizeof(ties), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (flags & kFlagCapacity) {
        fail(cudaSuccess, "");
        set_error("aica_build_interaction_list: a cell has more than %d neighbour cells", kSortMax);
        return AICA_ERR_CAPACITY;
    }
    int64_t n_work = (int64_t)tot[0] + tot[3];
    CK(m->dil_ids.reserve(sizeof(int) * std::max(tot[0], 1)));
    CK(m->ref_src.reserve(sizeof(int) * std::max(tot[2], 1)));
    CK(m->ref_n.reserve(sizeof(int) * 3 * std::max(tot[2], 1)));
    CK(m->ref_off.reserve(sizeof(int) * (tot[2] + 1)));
    CK(m->ref_ids.reserve(sizeof(int) * std::max(tot[1], 1)));
    CK(m->work_off.reserve(sizeof(int) * (C + 1)));
    CK(m->work_split.reserve(sizeof(int) * C));
    CK(m->work.reserve(sizeof(WorkEntry) * std::max<int64_t>(n_work, 1)));
    FillArgs f{};
    f.C = C;
    f.seg_off = a.seg_off;
    f.keys = a.keys;
    f.o_dil = m->dil_off.as<int>();
    f.o_re = o_re;
    f.o_rc = o_rc;
    f.o_rw = o_rw;
    f.orgk = a.orgk;
    for (int d = 0; d < 3; ++d) f.L[d] = a.L[d];
    f.dil_ids = m->dil_ids.as<int>();
    f.ref_src = m->ref_src.as<int>();
    f.ref_n = m->ref_n.as<int>();
    f.ref_off = m->ref_off.as<int>();
    f.ref_ids = m->ref_ids.as<int>();
    f.work_off = m->work_off.as<int>();
    f.work_split = m->work_split.as<int>();
    f.work = m->work.as<WorkEntry>();
    lst_fill<<<(C + 1 + 255) / 256, 256, 0, st>>>(f);
    m->launches += 1;
    // runs of the schedule (FP32 pair kernel): count, offsets, fill
    CK(m->run_off.reserve(sizeof(int) * (C + 1)));
    int *run_cnt = o_re;     // the referral scratch is free again
    lst_runs<<<(C + 255) / 256, 256, 0, st>>>(f.work_off, f.work, m->orgm.as<int>(), C, nullptr, run_cnt, nullptr);
    m->launches += 1 + exclusive_scan<int, int>(run_cnt, C, m->run_off.as<int>(), sw, st);
    int n_runs = 0;
    CK(cudaMemcpyAsync(&n_runs, m->run_off.as<int>() + C, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    CK(m->runs.reserve(sizeof(RunEntry) * std::max(n_runs, 1)));
    lst_runs<<<(C + 255) / 256, 256, 0, st>>>(f.work_off, f.work, m->orgm.as<int>(), C, m->run_off.as<int>(),
                                               nullptr, m->runs.as<RunEntry>());
    m->launches += 1;
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
#undef CK
    m->n_xf = 0;
    if (!m->xf_gen.empty()) {
        // general referring transforms: the referral and schedule are built on the host
        m->n_work = n_work;
        m->n_ties = (int64_t)ties;
        aica_status s2 = build_transform_referral(m, thr, st);
        d_boff.release(); d_bcell.release(); d_cnt.release(); d_seg.release(); d_keys.release(); d_scan.release();
        d_ties.release();
        if (s2 != AICA_OK) return s2;
        m->n_dil = tot[0];
        m->rc = rc;
        m->skin = skin;
        m->criterion = (int)criterion;
        m->built = true;
        return AICA_OK;
    }
    d_boff.release(); d_bcell.release(); d_cnt.release(); d_seg.release(); d_keys.release(); d_scan.release();
    d_ties.release();
    m->rc = rc;
    m->skin = skin;
    m->criterion = (int)criterion;
    {
        aica_status s3 = build_cluster_schedule(m, st);
        if (s3 != AICA_OK) return s3;
    }
    m->n_dil = tot[0];
    m->n_ref_ids = tot[1];
    m->n_ref = tot[2];
    m->n_work = n_work;
    m->n_runs = n_runs;
    m->n_ties = (int64_t)ties;
    m->rc = rc;
    m->skin = skin;
    m->criterion = (int)criterion;
    m->built = true;
    return AICA_OK;
}

extern "C" aica_status aica_get_list_info(const aica_mesh *m, aica_list_info *info) {
    if (!m || !info) { set_error("aica_get_list_info: NULL argument"); return AICA_ERR_INVALID_ARG; }
    if (!m->built) { set_error("aica_get_list_info: lists not built"); return AICA_ERR_NOT_BUILT; }
    info->n_cells = m->n_cells;
    info->n_dil = m->n_dil;
    info->n_ref = m->n_ref;
    info->n_ref_ids = m->n_ref_ids;
    info->n_ties = m->n_ties;
    info->rc = m->rc;
    info->skin = m->skin;
    info->criterion = (aica_dil_criterion)m->criterion;
    return AICA_OK;
}

extern "C" aica_status aica_get_lists(const aica_mesh *m, int64_t *dil_off, int32_t *dil_ids, int32_t *ref_src,
                                      int32_t *ref_n, int64_t *ref_off, int32_t *ref_ids) {
    if (!m) { set_error("aica_get_lists: mesh is NULL"); return AICA_ERR_INVALID_ARG; }
    if (!m->built) { set_error("aica_get_lists: lists not built"); return AICA_ERR_NOT_BUILT; }
    const int64_t C = m->n_cells;
    if (dil_off) {
        std::vector<int> t(C + 1);
        AICA_CUDA(cudaMemcpy(t.data(), m->dil_off.p, sizeof(int) * (C + 1), cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i <= C; ++i) dil_off[i] = t[i];
    }
    if (dil_ids && m->n_dil)
        AICA_CUDA(cudaMemcpy(dil_ids, m->dil_ids.p, sizeof(int) * m->n_dil, cudaMemcpyDeviceToHost));
    if (ref_src && m->n_ref)
        AICA_CUDA(cudaMemcpy(ref_src, m->ref_src.p, sizeof(int) * m->n_ref, cudaMemcpyDeviceToHost));
    if (ref_n && m->n_ref)
        AICA_CUDA(cudaMemcpy(ref_n, m->ref_n.p, sizeof(int) * 3 * m->n_ref, cudaMemcpyDeviceToHost));
    if (ref_off) {
        std::vector<int> t(m->n_ref + 1);
        AICA_CUDA(cudaMemcpy(t.data(), m->ref_off.p, sizeof(int) * (m->n_ref + 1), cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i <= m->n_ref; ++i) ref_off[i] = t[i];
    }
    if (ref_ids && m->n_ref_ids)
        AICA_CUDA(cudaMemcpy(ref_ids, m->ref_ids.p, sizeof(int) * m->n_ref_ids, cudaMemcpyDeviceToHost));
    return AICA_OK;
}
