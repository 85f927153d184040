// Pair-force kernels (steps a5-a10): the force loops of §2.3 on the binned
// molecules and the per-cell pair schedule built with the lists.
//
// Schedule.  For real cell I the schedule lists its DIL cells (J > I, App.
// A.1) and then the periodic image pairs (J, n) it owns.  §2.3 evaluates a
// real-referred pair from both sides, each time acting on the real molecule
// only, because the source molecule may live on another processor; on one
// device the source molecule is in memory, so each periodic image pair is
// evaluated once with Newton's third law (the reaction goes to the source
// molecule).  Forces are the same; the referred work halves.  Same-cell pairs
// (sorted index k' > k, §2.3) come first.  A referred molecule is never
// copied: it is read through the cell-pair shift Delta = o_J + n.L - o_I
// (step a5).
//
// Culling.  Per step every cell carries the bounding sphere of its molecules
// (computed at binning).  A partner cell whose sphere is farther than rc from
// I's, and a partner molecule farther than rc from I's sphere, cannot hold a
// pair within rc (triangle inequality; margins above the FP32 cut-off) and is
// skipped.  The counters still report every pair of every scheduled cell pair
// as "evaluated".
//
// Kernels.  With box periodicity and the minimum-distance lists the FP32
// forces come from the cluster kernel pair_fwd32c (further below: a warp
// per cluster of cells, candidates culled against the cluster's box), then
// flag_ill_conditioned and refine_ds recompute in double-single arithmetic
// the molecules whose FP32 force the error bound cannot certify.  The cell
// kernel pair_fwd32 described next serves general referring transforms, the
// vertex criterion and AICA_OPT_FP32_KERNEL = 1; pair_fwd64 is the FP64 path.
//
// FP32 cell kernel layout.  A persistent grid of 4-warp blocks; warps claim
// cells from a global counter.  The chunk (up to NI molecules of I: 4 for cells of a
// few molecules, 8 otherwise) sits in shared memory.  The FP32 schedule is
// kept in runs: consecutive partner cells under one image vector and one
// molecule-frame origin are one contiguous range of binned molecules under
// one shift.  32 runs at a time are culled, compacted (ballot), and their
// molecules indexed by a ballot/redux map from candidate position to run;
// candidates that survive the sphere test go to a per-warp ring in shared
// memory, and each 32 queued partners are evaluated one partner per lane
// against the chunk (branch-free pair body).  A lane sums its partner's
// reaction in registers and adds it with one vector atomic; the chunk's
// forces are summed over the warp by recursive halving.
//
// Precision (FP32 path).  Coordinates are local to dyadic origins shared by
// groups of consecutive cells of bounded extent (o_J - o_I exact in FP32).
// Pairs whose FP32 r^2 falls within 1e-5 rc^2 of the cut-off are re-decided
// in FP64 exactly as the all-pairs definition computes r^2, so the pair set
// within rc is the same as in FP64.  The virial sum over pairs of r (x) f is
// accumulated as sum_k x_k (x) F_k + sum_l x_l (x) F_l over the forces each
// warp adds (both in I's frame; every pair contributes f and -f, so the
// origin cancels).  Energy and virial are summed per lane in FP32 over at
// most four cells, then in FP64 per warp; warps add their totals to striped
// FP64 rows that a small kernel sums.
//
// Adjoint (step a10).  pair_bwd32 runs the FP32 kernel's schedule walk
// (walk_runs) with the adjoint pair body, so it recomputes exactly the
// forward's pair set; pair_bwd64 is its FP64 comparison path.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "aica_internal.cuh"

namespace aica {
namespace {

constexpr int kPairThreads = 256;
constexpr int kWarps = kPairThreads / 32;
constexpr int kParts = 16;           // accumulator row: U, W[6], counters[8]
constexpr int NI = 8;                // i-molecules per chunk in the FP64 kernel

struct SpeciesTab {
    float4 f[kMaxSpecies * kMaxSpecies];    // sigma^2, 24 eps, 4 eps, u(rc) for FP32
    double d[kMaxSpecies * kMaxSpecies][4]; // same in FP64
};

struct PairArgs {
    int C;
    const int *cell_off, *work_off;
    const WorkEntry *work;
    const int *run_off;
    const RunEntry *runs;
    const int *orgm;             // molecule-frame origins in units of 2^-10
    float Lhi[3], Llo[3];        // box lengths as float pairs (Lhi + Llo = L to ~1e-14)
    const float4 *xloc;
    const double *xs64;
    const float4 *sph;           // per-cell molecule bounding spheres (local frame)
    float rc2_lo, rc2_hi;
    float rc2_pre;               // cluster kernel: hi-part test threshold (margin above the remainders)
    double rc2_d;
    double L[3];
    int S;
    void *facc;                  // float4 (FP32) or double4 (FP64), binned order
    const void *vs;              // backward: grad_force in binned order (float4 / double4)
    double *acc;                 // [0..6] U, W; [8..15] counters (as unsigned long long); [16..] grads
    unsigned *next_cell;         // FP32 kernel: next unclaimed cell (zero at launch)
    int ghosts;                  // portion mode: xloc.w carries kGhostBit on halo molecules
    int xf;                      // general referring transforms: image field = transform index
    int n_xf;                    // transforms in xft
    const XfDev *xft;            // [n_xf] transforms (identity first)
    const float4 *run_d;         // general transforms: shift of each run in I's molecule frame
    SpeciesTab tab;
};

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

template <class R> struct R3 { R x, y, z; };

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// FP64 re-decision of r^2 < rc^2 with the all-pairs definition's operation order
// image y_t + R_t x of x under referring transform t, in the oracle's operation order
__device__ __forceinline__ void xf_image(const XfDev &t, const double *x, double *q) {
    for (int i = 0; i < 3; ++i)
        q[i] = __dadd_rn(t.y[i], __dadd_rn(__dadd_rn(__dmul_rn(t.R[3 * i], x[0]), __dmul_rn(t.R[3 * i + 1], x[1])),
                                           __dmul_rn(t.R[3 * i + 2], x[2])));
}

// the same decision under referring transform np (general transforms)
__device__ __noinline__ bool band_in_xf(const PairArgs &a, int k, int l, int np) {
    const double *xk = a.xs64 + 3 * (size_t)k, *xl = a.xs64 + 3 * (size_t)l;
    double q[3] = {xl[0], xl[1], xl[2]};
    if (np != 0) xf_image(a.xft[np], xl, q);
    const double dx = __dsub_rn(xk[0], q[0]), dy = __dsub_rn(xk[1], q[1]), dz = __dsub_rn(xk[2], q[2]);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)) < a.rc2_d;
}

__device__ __noinline__ bool band_in(const PairArgs &a, int k, int l, int np) {
    const double *xk = a.xs64 + 3 * (size_t)k, *xl = a.xs64 + 3 * (size_t)l;
    double dx = __dsub_rn(__dsub_rn(xk[0], xl[0]), __dmul_rn(a.L[0], (double)unpack_n(np, 0)));
    double dy = __dsub_rn(__dsub_rn(xk[1], xl[1]), __dmul_rn(a.L[1], (double)unpack_n(np, 1)));
    double dz = __dsub_rn(__dsub_rn(xk[2], xl[2]), __dmul_rn(a.L[2], (double)unpack_n(np, 2)));
    double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    return r2 < a.rc2_d;
}

// Sums of the pair kernels.  Every warp adds its totals (FP64 sums identical
// in all lanes; counters per lane) to one of kStripes rows of FP64
// accumulators (row = warp index mod kStripes, so few warps share an
// address); finish_sums adds the rows.  Row layout: [0..6] U and W,
// [7..14] the counters, exactly representable in FP64.
constexpr int kStripes = 64;
constexpr int kAccStripes = 64;        // offset of the rows in acc (doubles)

__device__ void warp_to_stripe(const PairArgs &a, int gwarp, const double (&dsum)[7], const unsigned (&cv)[8],
                               int lane) {
    double *row = a.acc + kAccStripes + (size_t)(gwarp % kStripes) * kParts;
    for (int i = 0; i < 8; ++i) {
        const unsigned s = __reduce_add_sync(0xffffffffu, cv[i]);
        if (lane == 0 && s) atomicAdd(row + 7 + i, (double)s);
    }
    if (lane < 7) atomicAdd(row + lane, dsum[lane < 7 ? lane : 0]);
}

// Totals of the stripe rows into acc ([0..6] FP64, [8..15] counters as
// unsigned 64-bit) and the caller's energy/virial [7] and pair counts [6].
// Value i of the sums (one warp): lanes over the stripe rows.
__device__ __forceinline__ void finish_value(double *acc, double *ev, long long *counts, int i, int lane) {
    double v = 0.0;
    for (int r = lane; r < kStripes; r += 32) v += acc[kAccStripes + r * kParts + i];
    v = warp_sum(v);
    if (lane != 0) return;
    if (i < 7) {
        acc[i] = v;
        if (ev) ev[i] = v;
    } else {
        const unsigned long long c = (unsigned long long)llrint(v);
        ((unsigned long long *)(acc + 8))[i - 7] = c;
        if (counts && i < 13) counts[i - 7] = (long long)c;
    }
}

// One warp per value (15 warps); used when no molecule was binned (otherwise
// the first block of unsort_forces does it).
__global__ void __launch_bounds__(15 * 32) finish_sums(double *acc, double *ev, long long *counts) {
    finish_value(acc, ev, counts, threadIdx.x >> 5, threadIdx.x & 31);
}

// ------------------------------------------------------------------ FP32 path
// Shift from cell I's frame to cell J's image n: (o_J - o_I) + n.L.  The
// origin difference is a multiple of 2^-10 (exact in FP32); n.Lhi cancels
// against it exactly for image pairs (Sterbenz), leaving one rounding for
// the n.Llo term.
__device__ __forceinline__ float3 cell_shift(const PairArgs &a, const int *oI, int J, int np) {
    const int *oJ = a.orgm + 3 * J;
    float3 d;
    const float nx = (float)unpack_n(np, 0), ny = (float)unpack_n(np, 1), nz = (float)unpack_n(np, 2);
    d.x = fmaf(nx, a.Lhi[0], (float)(oJ[0] - oI[0]) * (1.0f / 1024.0f)) + nx * a.Llo[0];
    d.y = fmaf(ny, a.Lhi[1], (float)(oJ[1] - oI[1]) * (1.0f / 1024.0f)) + ny * a.Llo[1];
    d.z = fmaf(nz, a.Lhi[2], (float)(oJ[2] - oI[2]) * (1.0f / 1024.0f)) + nz * a.Llo[2];
    return d;
}

// R x for a row-major FP32 rotation R
__device__ __forceinline__ float3 rot32(const float *R, float x, float y, float z) {
    return make_float3(fmaf(R[0], x, fmaf(R[1], y, R[2] * z)), fmaf(R[3], x, fmaf(R[4], y, R[5] * z)),
                       fmaf(R[6], x, fmaf(R[7], y, R[8] * z)));
}

// Per-warp queue of partner molecules that survived culling: position in I's
// frame (species bits in .w), binned index and image vector.
constexpr int kQ = 64;
struct WarpQueue {
    float4 x[kQ];
    int l[kQ];
    int np[kQ];
};

// Same-cell candidates carry this marker in their image field: they pair
// only with chunk molecules of lower binned index (k' > k, §2.3).
constexpr int kSameCell = 1 << 24;

// Lennard-Jones force factor and energy for r^2, branch-free.  t0 holds the
// single-species parameters (sigma^2, 24 eps, 4 eps, u(rc)).
template <bool MULTI, bool SHIFT>
__device__ __forceinline__ void lj32(const float4 *tab, float4 t0, int spi, int spj, float r2, float &fs, float &u) {
    float4 t = MULTI ? tab[spi * kMaxSpecies + spj] : t0;
    float inv = rcp_approx(r2);
    float s = t.x * inv;
    float s3 = s * s * s;
    fs = (t.y * inv) * s3 * fmaf(2.f, s3, -1.f);
    u = t.z * s3 * (s3 - 1.f);
    if (SHIFT) u -= t.w;
}

// FP32 kernel: persistent grid of 4-warp blocks; warps claim cells from a
// global counter.  Per warp, shared memory holds the partner ring, the live
// schedule entries of the current batch and the chunk's molecules.
constexpr int kThreads32 = 128;
constexpr int kWarps32 = kThreads32 / 32;
constexpr int kRing = 64;            // partner ring (power of two, >= 2 x 32)
constexpr int kGrab = 2;             // cells claimed per counter update

template <int NI_>
struct Warp32 {
    float4 qx[kRing];    // queued partners: position in I's frame (.w species bits)
    int2 ql[kRing];      // queued partners: binned index, image code (kSameCell: same cell)
    float4 ed[32];       // live entries of the batch, compacted: shift (xyz), image code (.w bits)
    int eb[32];          // ... and binned index minus candidate position
    float4 xi[NI_];      // molecules of the current chunk
    unsigned cnt[5];     // evaluated same / DIL / image, pair tests, sphere tests
};

// One pair's force and energy (FP32 body, branch-free): f is added to fi3
// and subtracted from fj when `in`, u to v[0].  Under general transforms
// (XF) the pair's energy and virial r (x) f are added here with weight w.
template <bool MULTI, bool SHIFT, bool XF>
__device__ __forceinline__ void pair32(const float4 *tab, float4 t0, int spi, int spj, float rx, float ry, float rz,
                                       float r2, bool in, float w, float *fi4, R3<float> &fj, float &gj,
                                       float &u_acc, float *v) {
    float fs, u;
    lj32<MULTI, SHIFT>(tab, t0, spi, spj, r2, fs, u);
    fs = in ? fs : 0.f;
    if (XF) u_acc += in ? w * u : 0.f;
    else u_acc += in ? u : 0.f;
    fi4[0] = fmaf(fs, rx, fi4[0]);
    fi4[1] = fmaf(fs, ry, fi4[1]);
    fi4[2] = fmaf(fs, rz, fi4[2]);
    fj.x = fmaf(-fs, rx, fj.x);
    fj.y = fmaf(-fs, ry, fj.y);
    fj.z = fmaf(-fs, rz, fj.z);
    // |f|^2 of the pair: the scale of the FP32 error of both molecules' forces
    const float g = fs * fs;
    fi4[3] = fmaf(g, r2, fi4[3]);
    gj = fmaf(g, r2, gj);
    if (XF) {
        const float g = w * fs, gx = g * rx, gy = g * ry;
        v[1] = fmaf(gx, rx, v[1]);
        v[2] = fmaf(gy, ry, v[2]);
        v[3] = fmaf(g * rz, rz, v[3]);
        v[4] = fmaf(gx, ry, v[4]);
        v[5] = fmaf(gx, rz, v[5]);
        v[6] = fmaf(gy, rz, v[6]);
    }
}

// One lane's partner xj against the chunk's ni molecules: every pair with
// r^2 < rc^2 adds f to the chunk molecule's sum and -f to the partner's.
// FP32 r^2 within 1e-5 rc^2 of the cut-off is re-decided in FP64 after the
// pass (one vote per batch).  With SAME, only chunk molecules of binned
// index below lmax_k take part.  Returns the pairs within rc.
template <int NI_, bool MULTI, bool SHIFT, bool SAME, bool XF>
__device__ __forceinline__ unsigned eval_partner(const PairArgs &a, const float4 *tab, const float4 *xi, int ni,
                                                 int k0, float4 xj, int l, int np, int lmax_k, float (&fi)[4 * NI_],
                                                 R3<float> &fj, float &gj, float &u_acc, float *v, float w) {
    unsigned nin = 0, bm = 0;
    const float4 t0 = tab[0];
#pragma unroll
    for (int t = 0; t < NI_; ++t) {
        if (t < ni) {
            const float4 x = xi[t];
            const float rx = x.x - xj.x, ry = x.y - xj.y, rz = x.z - xj.z;
            const float r2 = fmaf(rz, rz, fmaf(ry, ry, rx * rx));
            const bool ok = !SAME || k0 + t < lmax_k;
            const bool in = ok && r2 < a.rc2_lo;
            if (ok && !in && r2 < a.rc2_hi) bm |= 1u << t;
            pair32<MULTI, SHIFT, XF>(tab, t0, __float_as_int(x.w), __float_as_int(xj.w), rx, ry, rz, r2, in, w,
                                     &fi[4 * t], fj, gj, u_acc, v);
            nin += in;
        }
    }
    if (__any_sync(0xffffffffu, bm != 0)) {
#pragma unroll
        for (int t = 0; t < NI_; ++t) {
            if ((bm >> t) & 1u) {
                if (XF ? band_in_xf(a, k0 + t, l, np) : band_in(a, k0 + t, l, np)) {
                    const float4 x = xi[t];
                    const float rx = x.x - xj.x, ry = x.y - xj.y, rz = x.z - xj.z;
                    const float r2 = fmaf(rz, rz, fmaf(ry, ry, rx * rx));
                    pair32<MULTI, SHIFT, XF>(tab, t0, __float_as_int(x.w), __float_as_int(xj.w), rx, ry, rz, r2, true,
                                             w, &fi[4 * t], fj, gj, u_acc, v);
                    nin++;
                }
            }
        }
    }
    return nin;
}

// Sum v[0..3 NI_) over the warp by recursive halving: on return the lanes
// t * (32 / NI_) .. (t + 1) * (32 / NI_) - 1 hold the totals of v[3t..3t+3)
// in v[0..3).
template <int N>
__device__ __forceinline__ void halve(float *v, int lane, int o) {
    const bool up = lane & o;
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
        const float send = up ? v[i] : v[i + N / 2];
        const float keep = up ? v[i + N / 2] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
}
template <int NI_>
__device__ __forceinline__ void chunk_reduce(float (&v)[3 * NI_], int lane) {
    if (NI_ >= 2) halve<3 * NI_>(v, lane, 16);
    if (NI_ >= 4) halve<3 * NI_ / 2>(v, lane, 8);
    if (NI_ >= 8) halve<3 * NI_ / 4>(v, lane, 4);
#pragma unroll
    for (int o = 16 / NI_; o > 0; o >>= 1)
#pragma unroll
        for (int i = 0; i < 3; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
}

// The same for NI_ groups of 4 values (x, y, z, |f|^2): on return lanes
// t * (32 / NI_) .. hold the totals of v[4t..4t+4) in v[0..4).
template <int NI_>
__device__ __forceinline__ void chunk_reduce4(float (&v)[4 * NI_], int lane) {
    if (NI_ >= 2) halve<4 * NI_>(v, lane, 16);
    if (NI_ >= 4) halve<2 * NI_>(v, lane, 8);
    if (NI_ >= 8) halve<NI_>(v, lane, 4);
#pragma unroll
    for (int o = 16 / NI_; o > 0; o >>= 1)
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
}

__device__ __forceinline__ void outer7(float (&v)[7], float ax, float ay, float az, float bx, float by, float bz) {
    v[1] = fmaf(ax, bx, v[1]);
    v[2] = fmaf(ay, by, v[2]);
    v[3] = fmaf(az, bz, v[3]);
    v[4] = fmaf(ax, by, v[4]);
    v[5] = fmaf(ax, bz, v[5]);
    v[6] = fmaf(ay, bz, v[6]);
}

// Candidates of cell I's schedule runs e0 .. e1 for a chunk of ni molecules:
// a run's partner cells are consecutive, so their molecules are one binned
// range under one shift.  32 runs at a time are culled by their partner
// cell's sphere (single-cell runs), compacted (ballot) into ed / ebi, and
// their molecules indexed by a ballot/redux map from candidate position to
// run; every candidate (lane = candidate) goes to push(alive, position in I's
// frame, binned index, image field), alive = inside I's culling sphere.
// COUNT adds the evaluated-pair and sphere-test tallies to cnt[1], cnt[2], cnt[4].
template <bool XF, bool COUNT, class Push>
__device__ __forceinline__ void walk_runs(const PairArgs &a, float4 *ed, int *ebi, unsigned *cnt,
                                          const float (*xR)[9], int e0, int e1, int ni, const int *oI, float4 sI,
                                          float rcut, float cull_i, int lane, Push &push) {
    const unsigned FULL = 0xffffffffu, lt = (1u << lane) - 1u, le = FULL >> (31 - lane);
    const float4 far = make_float4(1e18f, 1e18f, 1e18f, 0.f);
    RunEntry we = e0 + lane < e1 ? a.runs[e0 + lane] : RunEntry{0, 0};
    for (int eb = e0; eb < e1; eb += 32) {
        const RunEntry cur = we;
        const bool has = eb + lane < e1;
        if (eb + 32 + lane < e1) we = a.runs[eb + 32 + lane];
        const int np = cur.n & 0xffffff, len = ((unsigned)cur.n >> 24) + 1;
        int js = 0, n = 0, nall = 0;
        bool tested = false;
        float3 d = make_float3(0.f, 0.f, 0.f);
        if (has) {
            js = a.cell_off[cur.j];
            nall = n = a.cell_off[cur.j + len] - js;
            if (n > 0) {
                if (XF) {
                    const float4 rd = a.run_d[eb + lane];
                    d = make_float3(rd.x, rd.y, rd.z);
                } else {
                    d = cell_shift(a, oI, cur.j, np);
                }
                if (len == 1) {      // one partner cell: its sphere may rule it out
                    float4 sJ = a.sph[cur.j];
                    if (XF) {
                        const float3 c = rot32(xR[np], sJ.x, sJ.y, sJ.z);
                        sJ.x = c.x; sJ.y = c.y; sJ.z = c.z;
                    }
                    const float dx = sJ.x + d.x - sI.x, dy = sJ.y + d.y - sI.y, dz = sJ.z + d.z - sI.z;
                    const float R = rcut + sI.w + sJ.w;
                    tested = true;
                    if (dx * dx + dy * dy + dz * dz > R * R * 1.00002f + 1e-5f) n = 0;
                }
            }
        }
        unsigned ev_d = 0, ev_r = 0, ncull = 0;
        if (COUNT) {
            ev_d = __reduce_add_sync(FULL, np == 0 ? (unsigned)(nall * ni) : 0u);
            ev_r = __reduce_add_sync(FULL, np != 0 ? (unsigned)(nall * ni) : 0u);
            ncull = __popc(__ballot_sync(FULL, tested));
        }
        int inc = n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += y;
        }
        const int total = __shfl_sync(FULL, inc, 31);
        const bool live = n > 0;
        const unsigned lbal = __ballot_sync(FULL, live);
        if (live) {
            const int s = __popc(lbal & lt);
            ed[s] = make_float4(d.x, d.y, d.z, __int_as_float(np));
            ebi[s] = js - (inc - n);
        }
        if (COUNT && lane == 0) {
            cnt[1] += ev_d;
            cnt[2] += ev_r;
            cnt[4] += ncull + (unsigned)total;
        }
        __syncwarp();
        for (int p0 = 0; p0 < total; p0 += 32) {
            // entry holding candidate p = p0 + lane: the live entries ending at or before p
            const int b = inc - p0;
            const int base = __popc(__ballot_sync(FULL, live && b <= 0));
            const unsigned M = __reduce_or_sync(FULL, (live && b > 0 && b < 32) ? (1u << b) : 0u);
            const int p = p0 + lane;
            bool alive = false;
            float4 xj = far;
            int l = 0, npl = 0;
            if (p < total) {
                const int o = base + __popc(M & le);
                const float4 e = ed[o];
                l = p + ebi[o];
                npl = __float_as_int(e.w);
                float4 xl = a.xloc[l];
                if (XF) {
                    const float3 c = rot32(xR[npl], xl.x, xl.y, xl.z);
                    xl.x = c.x; xl.y = c.y; xl.z = c.z;
                }
                xj = make_float4(xl.x + e.x, xl.y + e.y, xl.z + e.z, xl.w);
                const float cx = xj.x - sI.x, cy = xj.y - sI.y, cz = xj.z - sI.z;
                alive = cx * cx + cy * cy + cz * cz <= cull_i;
            }
            push(alive, xj, l, npl);
        }
        __syncwarp();
    }
}

// XF: general referring transforms (rotated referred cells, evaluated from
// the real side only, energy and virial per pair with weight 1/2).
template <int NI_, bool MULTI, bool SHIFT, int MINB, bool XF>
__global__ void __launch_bounds__(kThreads32, MINB) pair_fwd32(PairArgs a) {
    __shared__ float4 tab[kMaxSpecies * kMaxSpecies];
    __shared__ Warp32<NI_> wsh[kWarps32];
    __shared__ double dsums[kWarps32][8];
    __shared__ float xR[XF ? kMaxXf : 1][9];
    for (int i = threadIdx.x; i < kMaxSpecies * kMaxSpecies; i += blockDim.x) tab[i] = a.tab.f[i];
    if (XF)
        for (int i = threadIdx.x; i < 9 * kMaxXf; i += blockDim.x)
            xR[i / 9][i % 9] = (a.xft && i / 9 < a.n_xf) ? a.xft[i / 9].Rf[i % 9] : 0.f;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    Warp32<NI_> &w = wsh[wib];
    if (lane < 8) dsums[wib][lane] = 0.0;
    if (lane < 5) w.cnt[lane] = 0;
    __syncthreads();
    const unsigned FULL = 0xffffffffu, lt = (1u << lane) - 1u;
    const float4 far = make_float4(1e18f, 1e18f, 1e18f, 0.f);
    const float rcut = sqrtf(a.rc2_hi);
    double *dsum = dsums[wib];
    float v[7];
#pragma unroll
    for (int i = 0; i < 7; ++i) v[i] = 0.f;
    unsigned within[3] = {0, 0, 0};
    int ncell = 0;
    int I0 = lane == 0 ? (int)atomicAdd(a.next_cell, (unsigned)kGrab) : 0;
    I0 = __shfl_sync(FULL, I0, 0);
    while (I0 < a.C) {
        const int Inext = lane == 0 ? (int)atomicAdd(a.next_cell, (unsigned)kGrab) : 0;
        const int Iend = min(I0 + kGrab, a.C);
        for (int I = I0; I < Iend; ++I) {
            const int s0 = a.cell_off[I], nI = a.cell_off[I + 1] - s0;
            if (nI == 0) continue;
            const int e0 = a.run_off[I], e1 = a.run_off[I + 1];
            const float4 sI = a.sph[I];
            const int *oI = a.orgm + 3 * I;
            const float cull_i = (rcut + sI.w) * (rcut + sI.w) * 1.00002f + 1e-5f;
            for (int i0 = 0; i0 < nI; i0 += NI_) {
                const int ni = min(NI_, nI - i0), k0 = s0 + i0;
                __syncwarp();
                if (lane < ni) w.xi[lane] = a.xloc[k0 + lane];
                float fi[4 * NI_];
#pragma unroll
                for (int i = 0; i < 4 * NI_; ++i) fi[i] = 0.f;
                int head = 0, qn = 0;
                __syncwarp();
                // evaluate the `count` partners at the ring's head (lane = partner)
                auto run = [&](int count) {
                    const int s = (head + lane) & (kRing - 1);
                    const bool valid = lane < count;
                    const float4 xj = valid ? w.qx[s] : far;
                    const int2 q = valid ? w.ql[s] : make_int2(0, 0);
                    if (lane == 0) w.cnt[3] += (unsigned)(count * ni);
                    R3<float> fj = {0.f, 0.f, 0.f};
                    float gj = 0.f;
                    const bool same = q.y == kSameCell;
                    const bool one = XF && !same && q.y != 0;     // referred under a transform: one side
                    const float wgt = one ? 0.5f : 1.f;
                    const unsigned nin =
                        __any_sync(FULL, same)
                            ? eval_partner<NI_, MULTI, SHIFT, true, XF>(a, tab, w.xi, ni, k0, xj, q.x, same ? 0 : q.y,
                                                                        same ? q.x : 0x7fffffff, fi, fj, gj, v[0],
                                                                        XF ? v : nullptr, wgt)
                            : eval_partner<NI_, MULTI, SHIFT, false, XF>(a, tab, w.xi, ni, k0, xj, q.x, q.y, 0, fi, fj,
                                                                         gj, v[0], XF ? v : nullptr, wgt);
                    if (same) within[0] += nin;
                    else if (q.y != 0) within[2] += nin;
                    else within[1] += nin;
                    if (nin && !one) {
                        atomicAdd((float4 *)a.facc + q.x, make_float4(fj.x, fj.y, fj.z, gj));
                        if (!XF) outer7(v, xj.x, xj.y, xj.z, fj.x, fj.y, fj.z);
                    }
                    head = (head + count) & (kRing - 1);
                    __syncwarp();
                };
                // append the live lanes' partners to the ring; evaluate each full 32
                auto push = [&](bool alive, float4 xj, int l, int np) {
                    const unsigned bal = __ballot_sync(FULL, alive);
                    if (alive) {
                        const int s = (head + qn + __popc(bal & lt)) & (kRing - 1);
                        w.qx[s] = xj;
                        w.ql[s] = make_int2(l, np);
                    }
                    qn += __popc(bal);
                    __syncwarp();
                    if (qn >= 32) {
                        run(32);
                        qn -= 32;
                    }
                };
                // same-cell partners (k' > k, §2.3): I's molecules after the chunk's first
                for (int lb = i0 + 1; lb < nI; lb += 32) {
                    const int li = lb + lane;
                    const bool alive = li < nI;
                    push(alive, alive ? a.xloc[s0 + li] : far, s0 + li, kSameCell);
                }
                walk_runs<XF, true>(a, w.ed, w.eb, w.cnt, xR, e0, e1, ni, oI, sI, rcut, cull_i, lane, push);
                if (qn > 0) run(qn);
                // forces on the chunk's molecules: transposed warp sum, one vector atomic each, k-side virial
                chunk_reduce4<NI_>(fi, lane);
                const int t = lane / (32 / NI_);
                if ((lane & (32 / NI_ - 1)) == 0 && t < ni) {
                    atomicAdd((float4 *)a.facc + k0 + t, make_float4(fi[0], fi[1], fi[2], fi[3]));
                    if (!XF) {
                        const float4 x = w.xi[t];
                        outer7(v, x.x, x.y, x.z, fi[0], fi[1], fi[2]);
                    }
                }
            }
            if (lane == 0) w.cnt[0] += (unsigned)(nI * (nI - 1) / 2);
            if (++ncell == 4) {          // flush the FP32 running sums to FP64
                ncell = 0;
#pragma unroll
                for (int i = 0; i < 7; ++i) {
                    const float s = warp_sum(v[i]);
                    if (lane == 0) dsum[i] += (double)s;
                    v[i] = 0.f;
                }
            }
        }
        I0 = __shfl_sync(FULL, Inext, 0);
    }
    double fin[7];
#pragma unroll
    for (int i = 0; i < 7; ++i) {
        const float s = warp_sum(v[i]);
        fin[i] = dsum[i] + (double)s;
    }
    __syncwarp();
    unsigned cv[8] = {w.cnt[0], w.cnt[1], w.cnt[2], within[0], within[1], within[2], w.cnt[3], w.cnt[4]};
    for (int i = 0; i < 3; ++i) cv[i] = __shfl_sync(FULL, cv[i], 0);
    cv[6] = __shfl_sync(FULL, cv[6], 0);
    cv[7] = __shfl_sync(FULL, cv[7], 0);
    if (lane != 0) cv[0] = cv[1] = cv[2] = cv[6] = cv[7] = 0;
    warp_to_stripe(a, blockIdx.x * kWarps32 + wib, fin, cv, lane);
}

// ------------------------------------------------------------------ FP64 path
// w: weight of the pair's energy and virial (1/2 for a pair evaluated from
// each of its sides, under general referring transforms)
template <bool MULTI, bool SHIFT>
__device__ __forceinline__ void pair64(const double (*tab)[4], double rx, double ry, double rz, double r2, int spi,
                                       int spj, R3<double> &fi, R3<double> &fj, double (&acc)[7], double w = 1.0) {
    const double *t = MULTI ? tab[spi * kMaxSpecies + spj] : tab[0];
    double inv = 1.0 / r2;
    double s = t[0] * inv;
    double s3 = s * s * s;
    double fs = t[1] * inv * s3 * (2.0 * s3 - 1.0);
    double fx = fs * rx, fy = fs * ry, fz = fs * rz;
    fi.x += fx; fi.y += fy; fi.z += fz;
    fj.x -= fx; fj.y -= fy; fj.z -= fz;
    double u = t[2] * s3 * (s3 - 1.0);
    if (SHIFT) u -= t[3];
    acc[0] += w * u;
    acc[1] += w * (rx * fx); acc[2] += w * (ry * fy); acc[3] += w * (rz * fz);
    acc[4] += w * (rx * fy); acc[5] += w * (rx * fz); acc[6] += w * (ry * fz);
}

__device__ __forceinline__ void atomic_add3(double *p, double x, double y, double z) {
    atomicAdd(p, x);
    atomicAdd(p + 1, y);
    atomicAdd(p + 2, z);
}

// r = (x_k - x_l) - n.L with the all-pairs definition's rounding
__device__ __forceinline__ void sep64(const double *xk, const double *xl, const double *L, int np, double &rx,
                                      double &ry, double &rz, double &r2) {
    rx = __dsub_rn(__dsub_rn(xk[0], xl[0]), __dmul_rn(L[0], (double)unpack_n(np, 0)));
    ry = __dsub_rn(__dsub_rn(xk[1], xl[1]), __dmul_rn(L[1], (double)unpack_n(np, 1)));
    rz = __dsub_rn(__dsub_rn(xk[2], xl[2]), __dmul_rn(L[2], (double)unpack_n(np, 2)));
    r2 = __dadd_rn(__dadd_rn(__dmul_rn(rx, rx), __dmul_rn(ry, ry)), __dmul_rn(rz, rz));
}

// r = x_k - (y_t + R_t x_l) under referring transform t (general transforms), else sep64
template <bool XF>
__device__ __forceinline__ void sep64x(const PairArgs &a, const double *xk, const double *xl, int np, double &rx,
                                       double &ry, double &rz, double &r2) {
    if (XF && np != 0) {
        double q[3];
        xf_image(a.xft[np], xl, q);
        rx = __dsub_rn(xk[0], q[0]);
        ry = __dsub_rn(xk[1], q[1]);
        rz = __dsub_rn(xk[2], q[2]);
        r2 = __dadd_rn(__dadd_rn(__dmul_rn(rx, rx), __dmul_rn(ry, ry)), __dmul_rn(rz, rz));
    } else {
        sep64(xk, xl, a.L, np, rx, ry, rz, r2);
    }
}

// Shift of cell J's molecule frame (under transform t) into cell I's, FP64 then FP32
__device__ __forceinline__ float3 xf_shift(const PairArgs &a, int I, int J, int t) {
    const XfDev &T = a.xft[t];
    const int *oJ = a.orgm + 3 * J, *oI = a.orgm + 3 * I;
    const double o[3] = {oJ[0] * (1.0 / 1024.0), oJ[1] * (1.0 / 1024.0), oJ[2] * (1.0 / 1024.0)};
    double q[3];
    xf_image(T, o, q);
    return make_float3((float)(q[0] - oI[0] * (1.0 / 1024.0)), (float)(q[1] - oI[1] * (1.0 / 1024.0)),
                       (float)(q[2] - oI[2] * (1.0 / 1024.0)));
}

// FP64: one warp per cell, lanes over the culled partner molecules (queue
// batches of 32), up to NI molecules of I per chunk in registers.
template <bool MULTI, bool SHIFT, bool XF>
__global__ void __launch_bounds__(kPairThreads) pair_fwd64(PairArgs a) {
    __shared__ double tab[kMaxSpecies * kMaxSpecies][4];
    __shared__ WarpQueue queues[kWarps];
    for (int i = threadIdx.x; i < kMaxSpecies * kMaxSpecies; i += blockDim.x)
        for (int c = 0; c < 4; ++c) tab[i][c] = a.tab.d[i][c];
    __syncthreads();
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int gwarp = blockIdx.x * kWarps + wib;
    const int nwarps = gridDim.x * kWarps;
    double *facc = (double *)a.facc;
    WarpQueue &q = queues[wib];
    const float rcut = sqrtf(a.rc2_hi);
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    unsigned eval[3] = {0, 0, 0}, within[3] = {0, 0, 0}, tests = 0, culls = 0;
    for (int I = gwarp; I < a.C; I += nwarps) {
        const int sI = a.cell_off[I], nI = a.cell_off[I + 1] - sI;
        if (nI == 0) continue;
        const int e0 = a.work_off[I], e1 = a.work_off[I + 1];
        const float4 sI4 = a.sph[I];
        const float cull_i = (rcut + sI4.w) * (rcut + sI4.w) * 1.00002f + 1e-5f;
        for (int i0 = 0; i0 < nI; i0 += NI) {
            const int ni = min(NI, nI - i0);
            double xi[NI][3];
            int spi[NI];
            R3<double> fi[NI];
#pragma unroll
            for (int t = 0; t < NI; ++t) {
                int k = sI + i0 + min(t, ni - 1);
                for (int c = 0; c < 3; ++c) xi[t][c] = a.xs64[3 * (size_t)k + c];
                spi[t] = __float_as_int(a.xloc[k].w);      // species | kGhostBit on halo molecules
                fi[t] = {0, 0, 0};
            }
            // same-cell pairs k' > k
            for (int lb = i0 + 1; lb < nI; lb += 32) {
                int li = lb + lane;
                if (li < nI) {
                    int l = sI + li;
                    const double *xl = a.xs64 + 3 * (size_t)l;
                    int spj = __float_as_int(a.xloc[l].w);
                    R3<double> fj = {0, 0, 0};
                    bool any = false;
#pragma unroll
                    for (int t = 0; t < NI; ++t) {
                        if (t < ni && li > i0 + t) {
                            double rx, ry, rz, r2;
                            sep64(xi[t], xl, a.L, 0, rx, ry, rz, r2);
                            const int g = ((spi[t] & kGhostBit) ? 1 : 0) + ((spj & kGhostBit) ? 1 : 0);
                            if (r2 < a.rc2_d && g < 2) {
                                pair64<MULTI, SHIFT>(tab, rx, ry, rz, r2, spi[t] & (kMaxSpecies - 1),
                                                     spj & (kMaxSpecies - 1), fi[t], fj, acc, g ? 0.5 : 1.0);
                                within[0]++;
                                any = true;
                            }
                        }
                    }
                    if (any) atomic_add3(facc + 4 * (size_t)l, fj.x, fj.y, fj.z);
                }
            }
            if (lane == 0) tests += (unsigned)(ni * (2 * nI - 2 * i0 - ni - 1) / 2);
            // partners: cull, compact, evaluate in batches of 32
            int qn = 0;
            auto run = [&](int count) {
                if (lane == 0) tests += (unsigned)(count * ni);
                if (lane < count) {
                    int l = q.l[lane], npl = q.np[lane];
                    int spj = __float_as_int(q.x[lane].w);
                    const double *xl = a.xs64 + 3 * (size_t)l;
                    R3<double> fj = {0, 0, 0};
                    bool any = false;
                    unsigned nin = 0;
                    // general transforms: a referred pair acts on I's molecule only and is met
                    // again from the other side, so its energy and virial count half (so does
                    // a pair of an owned and a halo molecule in portion mode)
                    const bool one = XF && npl != 0;
#pragma unroll
                    for (int t = 0; t < NI; ++t) {
                        if (t < ni) {
                            double rx, ry, rz, r2;
                            sep64x<XF>(a, xi[t], xl, npl, rx, ry, rz, r2);
                            const int g = ((spi[t] & kGhostBit) ? 1 : 0) + ((spj & kGhostBit) ? 1 : 0);
                            const double w = (one || g) ? 0.5 : 1.0;
                            if (r2 < a.rc2_d && g < 2) {
                                pair64<MULTI, SHIFT>(tab, rx, ry, rz, r2, spi[t] & (kMaxSpecies - 1),
                                                     spj & (kMaxSpecies - 1), fi[t], fj, acc, w);
                                nin++;
                                any = true;
                            }
                        }
                    }
                    if (npl != 0) within[2] += nin;
                    else within[1] += nin;
                    if (any && !one) atomic_add3(facc + 4 * (size_t)l, fj.x, fj.y, fj.z);
                }
                __syncwarp();
            };
            for (int eb = e0; eb < e1; eb += 32) {
                int e = eb + lane;
                int js = 0, n = 0, np = 0;
                float4 d = make_float4(0.f, 0.f, 0.f, 0.f);
                if (e < e1) {
                    WorkEntry we = a.work[e];
                    js = a.cell_off[we.j];
                    n = a.cell_off[we.j + 1] - js;
                    np = we.n;
                    if (n > 0) {
                        if (np != 0) eval[2] += (unsigned)(n * ni);
                        else eval[1] += (unsigned)(n * ni);
                        const float3 s3 = XF ? xf_shift(a, I, we.j, np) : cell_shift(a, a.orgm + 3 * I, we.j, np);
                        d = make_float4(s3.x, s3.y, s3.z, 0.f);
                        float4 sJ = a.sph[we.j];
                        if (XF) {
                            const float3 c = rot32(a.xft[np].Rf, sJ.x, sJ.y, sJ.z);
                            sJ.x = c.x; sJ.y = c.y; sJ.z = c.z;
                        }
                        float dx = sJ.x + d.x - sI4.x, dy = sJ.y + d.y - sI4.y, dz = sJ.z + d.z - sI4.z;
                        float R = rcut + sI4.w + sJ.w;
                        culls++;
                        if (dx * dx + dy * dy + dz * dz > R * R * 1.00002f + 1e-5f) n = 0;
                    }
                }
                int inc = n;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    int y = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= o) inc += y;
                }
                const int total = __shfl_sync(0xffffffffu, inc, 31);
                const int exc = inc - n;
                for (int p0 = 0; p0 < total; p0 += 32) {
                    int p = p0 + lane;
                    int o = 0;
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1)
                        if (__shfl_sync(0xffffffffu, inc, o + step - 1) <= p) o += step;
                    int jsl = __shfl_sync(0xffffffffu, js, o);
                    int exl = __shfl_sync(0xffffffffu, exc, o);
                    float dx = __shfl_sync(0xffffffffu, d.x, o);
                    float dy = __shfl_sync(0xffffffffu, d.y, o);
                    float dz = __shfl_sync(0xffffffffu, d.z, o);
                    int npl = __shfl_sync(0xffffffffu, np, o);
                    bool alive = false;
                    int l = jsl + (p - exl);
                    float4 xj;
                    if (p < total) {
                        float4 xl = a.xloc[l];
                        if (XF) {
                            const float3 c = rot32(a.xft[npl].Rf, xl.x, xl.y, xl.z);
                            xl.x = c.x; xl.y = c.y; xl.z = c.z;
                        }
                        xj = make_float4(xl.x + dx, xl.y + dy, xl.z + dz, xl.w);
                        float cx = xj.x - sI4.x, cy = xj.y - sI4.y, cz = xj.z - sI4.z;
                        alive = cx * cx + cy * cy + cz * cz <= cull_i;
                        culls++;
                    }
                    unsigned bal = __ballot_sync(0xffffffffu, alive);
                    if (alive) {
                        int s = qn + __popc(bal & ((1u << lane) - 1u));
                        q.x[s] = xj;
                        q.l[s] = l;
                        q.np[s] = npl;
                    }
                    qn += __popc(bal);
                    __syncwarp();
                    if (qn >= 32) {
                        run(32);
                        qn -= 32;
                        if (lane < qn) {
                            q.x[lane] = q.x[32 + lane];
                            q.l[lane] = q.l[32 + lane];
                            q.np[lane] = q.np[32 + lane];
                        }
                        __syncwarp();
                    }
                }
            }
            if (qn > 0) run(qn);
#pragma unroll
            for (int t = 0; t < NI; ++t) {
                if (t < ni) {
                    double x = warp_sum(fi[t].x), y = warp_sum(fi[t].y), z = warp_sum(fi[t].z);
                    if (lane == t) atomic_add3(facc + 4 * (size_t)(sI + i0 + t), x, y, z);
                }
            }
        }
        if (lane == 0) eval[0] += (unsigned)(nI * (nI - 1) / 2);
    }
    double dsum[7];
    for (int i = 0; i < 7; ++i) dsum[i] = warp_sum(acc[i]);
    unsigned cv[8] = {eval[0], eval[1], eval[2], within[0], within[1], within[2], tests, culls};
    warp_to_stripe(a, gwarp, dsum, cv, lane);
}

// ---------------------------------------------------------------- unsort
// Forces back to the original order; with acc, the first block also adds
// up the pair kernel's striped sums (finish_value).
template <class T>
__global__ void __launch_bounds__(256) unsort_forces(const int *inv, int64_t n, const void *facc, T *out, int f64,
                                                     double *acc = nullptr, double *ev = nullptr,
                                                     long long *counts = nullptr, int *flag_list = nullptr,
                                                     float kflag2 = 0.f) {
    if (acc && blockIdx.x == 0)
        for (int i = threadIdx.x >> 5; i < 15; i += blockDim.x >> 5) finish_value(acc, ev, counts, i, threadIdx.x & 31);
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int s = inv[k];
    double x = 0, y = 0, z = 0;
    if (s >= 0) {
        if (f64) {
            const double *f = (const double *)facc + 4 * (size_t)s;
            x = f[0]; y = f[1]; z = f[2];
        } else {
            float4 f = ((const float4 *)facc)[s];
            x = f.x; y = f.y; z = f.z;
            (void)flag_list;
            (void)kflag2;
        }
    }
    out[3 * k] = (T)x;
    out[3 * k + 1] = (T)y;
    out[3 * k + 2] = (T)z;
}

// A binned molecule split at multiples of 2^-q: hi exact on the grid, lo the
// rest (xloc - hi is exact; adding the stored remainder rounds far below
// the separation's own rounding).  Valid for |x| < 2^(22 - q).
__device__ __forceinline__ void grid_split(float4 x, float4 r, float qr, float4 &hi, float4 &lo) {
    hi.x = __fsub_rn(__fadd_rn(x.x, qr), qr);
    hi.y = __fsub_rn(__fadd_rn(x.y, qr), qr);
    hi.z = __fsub_rn(__fadd_rn(x.z, qr), qr);
    hi.w = x.w;
    lo = make_float4(__fsub_rn(x.x, hi.x) + r.x, __fsub_rn(x.y, hi.y) + r.y, __fsub_rn(x.z, hi.z) + r.z, 0.f);
}

// The FP32 error of a molecule's force is about a fixed multiple of
// sqrt(sum |f|^2) (the .w of its accumulator); a molecule whose force is too
// small against it goes to the list for recomputation.  In binned order,
// one append per warp, so the list follows the molecules' positions.
__global__ void __launch_bounds__(256) flag_ill_conditioned(const float4 *facc, const float4 *xloc, int nb,
                                                              float kflag2, int *flag_list) {
    __shared__ int wcnt[8], wbase[8];
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    bool f = false;
    if (s < nb) {
        const float4 v = facc[s];
        f = v.x * v.x + v.y * v.y + v.z * v.z < kflag2 * v.w && !(__float_as_int(xloc[s].w) & kGhostBit);
    }
    const unsigned b = __ballot_sync(0xffffffffu, f);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) wcnt[w] = __popc(b);
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int i = 0; i < 8; ++i) {
            wbase[i] = t;
            t += wcnt[i];
        }
        const int base = t ? atomicAdd(flag_list, t) : 0;
        for (int i = 0; i < 8; ++i) wbase[i] += base;
    }
    __syncthreads();
    if (f) flag_list[1 + wbase[w] + __popc(b & ((1u << lane) - 1u))] = s;
}

// Double-single ("float-float") arithmetic: a value is an unevaluated sum
// hi + lo of two FP32 numbers (about 48 significant bits) built from
// error-free transformations: Knuth's TwoSum, the FMA form of Dekker's
// TwoProduct, and a Newton step for the reciprocal (x' = x + x (1 - a x)).
// GB300 runs FP32 about 75 times faster than FP64, so recomputing a
// molecule this way costs far less than in FP64.
struct ds {
    float h, l;
};
__device__ __forceinline__ ds ds_fast2sum(float a, float b) {   // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ds ds_twosum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ ds ds_add(ds a, ds b) {
    const ds s = ds_twosum(a.h, b.h);
    return ds_fast2sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ ds ds_mul(ds a, ds b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return ds_fast2sum(p, e);
}
__device__ __forceinline__ ds ds_rcp(ds a) {
    const float y = __frcp_rn(a.h);
    const float e = __fmaf_rn(-a.l, y, __fmaf_rn(-a.h, y, 1.f));   // 1 - a y
    return ds_fast2sum(y, __fmul_rn(y, e));
}

// Recomputation of the molecules flagged by unsort_forces: a warp per
// molecule k (binned) of cluster A, lanes over the molecules of A and of
// every (partner cluster, image) of A's full list.  Each separation is
// formed exactly before one rounding (hi parts on the 2^-q grid, as in the
// cluster kernel) and an FP32 test with a wide margin queues the nearby
// ones; the queue is evaluated one pair per lane in double-single
// arithmetic.  r^2 < rc^2 is decided on the double-single r^2 (relative
// error ~1e-14); within 1e-10 rc^2 of the cut-off the FP64 all-pairs
// operation order decides, so the pair set is exactly the pairs within rc.
// Writes the force (original order) over the FP32 one.
struct RefineArgs {
    const int *flag_list, *cl_first, *cl_of, *full_off, *order;
    const unsigned long long *full;
    const float4 *xlo;
    const float4 *cl_box;        // boxes of the clusters' molecules from the FP32 pass
    float *out;
    int C;
    const int *orgm;             // molecule-frame origins in units of 2^-10 (per cell)
    float Lh[3], Ll[3];          // box lengths: multiple of 2^-q plus FP32 remainder
    float qround;                // grid_split constant
    float sig2[kMaxSpecies * kMaxSpecies][2];   // sigma_ab^2 and 24 eps_ab, double-single
    float c24[kMaxSpecies * kMaxSpecies][2];
    float rc2h, rc2l;            // rc^2, double-single
    unsigned *next;              // next unclaimed entry of the flag list (zero at launch)
};

constexpr int kRefineGrab = 4;        // flagged molecules claimed per warp at a time
__global__ void __launch_bounds__(256) refine_ds(PairArgs a, RefineArgs r) {
    __shared__ float4 ed[8][32];       // per warp: live entries of the batch: shift hi (xyz), image (w)
    __shared__ float4 el[8][32];       //           shift remainder (xyz)
    __shared__ int eb[8][32];          //           first molecule minus candidate position
    __shared__ float4 rq[8][64][2];    //           queued pairs: separation hi, lo (+ molecule, image)
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u, le = FULL >> (31 - lane);
    const int nflag = r.flag_list[0];
    const float pre2 = a.rc2_hi * 1.001f + 1e-3f;
    const float reach = sqrtf(pre2) + 1e-3f;
    // warps claim consecutive entries of the (spatially ordered) list, up to
    // kRefineGrab at a time when the list is long enough to keep every warp
    // busy: neighbouring molecules share their candidates in the caches, and
    // the claims balance molecules of unequal cost
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int grab = max(1, min(kRefineGrab, nflag / (4 * nw)));      // c5: 4, c2 and c4: 1
    int prev = 0;                      // cell of the warp's previous molecule (the list ascends)
    for (;;) {
    int i0 = lane == 0 ? (int)atomicAdd(r.next, (unsigned)grab) : 0;
    i0 = __shfl_sync(FULL, i0, 0);
    if (i0 >= nflag) break;
    const int i_end = min(nflag, i0 + grab);
    for (int i = i0; i < i_end; ++i) {
        const int k = r.flag_list[1 + i];
        // cell of k (cell_off[c] <= k < cell_off[c + 1]): first the 32 cells
        // from the previous molecule's, then a 32-ary search, one probe per lane
        int lo = 0, hi = r.C;
        {
            const int probe = prev + lane;
            const bool le_k = probe < r.C && a.cell_off[probe] <= k;
            const unsigned bl = __ballot_sync(FULL, le_k);
            // cells prev .. prev + 31 start at or before k; the last of them holds k
            // when a later probe starts beyond k (or the mesh ends)
            if ((bl & 1u) && bl != FULL) {
                lo = prev + 31 - __clz(bl);
                hi = lo + 1;
            } else if ((bl & 1u) && prev + 32 >= r.C) {
                lo = r.C - 1;
                hi = r.C;
            }
        }
        while (hi - lo > 1) {
            const int step = (hi - lo + 31) / 32;
            const int probe = lo + lane * step;
            const bool le_k = probe < hi && a.cell_off[probe] <= k;
            const int last = 31 - __clz(__ballot_sync(FULL, le_k));
            lo += last * step;
            hi = min(lo + step, hi);
        }
        prev = lo;
        const int A = r.cl_of[lo];
        float4 kh, kl;
        grid_split(a.xloc[k], r.xlo[k], r.qround, kh, kl);
        const int spk = __float_as_int(kh.w) & (kMaxSpecies - 1);
        const int *oA = r.orgm + 3 * (size_t)r.cl_first[A];
        ds Fx = {0.f, 0.f}, Fy = {0.f, 0.f}, Fz = {0.f, 0.f};
        int nq = 0;
        // the queued pairs, one per lane
        auto drain = [&](int count) {
            if (lane < count) {
                const float4 q0 = rq[wib][lane][0], q1 = rq[wib][lane][1];
                const ds rx = ds_fast2sum(q0.x, q0.w), ry = ds_fast2sum(q0.y, q1.x), rz = ds_fast2sum(q0.z, q1.y);
                const int l = __float_as_int(q1.z);
                const int32_t nl = __float_as_int(q1.w);
                // r^2 = sum (h + l)^2 with the squares of the hi parts exact
                ds r2 = {0.f, 0.f};
                const ds cs[3] = {rx, ry, rz};
                for (int c = 0; c < 3; ++c) {
                    const float p = __fmul_rn(cs[c].h, cs[c].h);
                    const float e = __fmaf_rn(2.f * cs[c].h, cs[c].l, __fmaf_rn(cs[c].h, cs[c].h, -p));
                    r2 = ds_add(r2, ds_fast2sum(p, e));
                }
                const ds dr = ds_add(r2, ds{-r.rc2h, -r.rc2l});
                bool in = dr.h < 0.f;
                if (fabsf(dr.h) <= 1e-10f * r.rc2h) {
                    double x, y, z, rr;
                    sep64(a.xs64 + 3 * (size_t)k, a.xs64 + 3 * (size_t)l, a.L, nl, x, y, z, rr);
                    in = rr < a.rc2_d;
                }
                if (in) {
                    const int ab = a.S > 1 ? spk * kMaxSpecies + (__float_as_int(a.xloc[l].w) & (kMaxSpecies - 1)) : 0;
                    const ds inv = ds_rcp(r2);
                    const ds s = ds_mul(ds{r.sig2[ab][0], r.sig2[ab][1]}, inv);
                    const ds s3 = ds_mul(ds_mul(s, s), s);
                    const ds t = ds_add(ds{2.f * s3.h, 2.f * s3.l}, ds{-1.f, 0.f});
                    const ds fs = ds_mul(ds_mul(ds_mul(ds{r.c24[ab][0], r.c24[ab][1]}, inv), s3), t);
                    Fx = ds_add(Fx, ds_mul(fs, rx));
                    Fy = ds_add(Fy, ds_mul(fs, ry));
                    Fz = ds_add(Fz, ds_mul(fs, rz));
                }
            }
            __syncwarp();
        };
        const int f0 = r.full_off[A], f1 = r.full_off[A + 1];
        // entries: A itself (image 0), then A's full list; 32 at a time, one per lane
        for (int e0 = f0 - 1; e0 < f1; e0 += 32) {
            const int e = e0 + lane;
            int n = 0, js = 0;
            int32_t np = 0;
            float4 dh = make_float4(0.f, 0.f, 0.f, 0.f), dl = dh;
            if (e < f1) {
                int B = A;
                if (e >= f0) {
                    const unsigned long long key = r.full[e];
                    B = (int)(key & 0xffffffffu);
                    np = (int32_t)(key >> 32);
                }
                // shift into A's frame: origin difference (a multiple of 2^-10, exact)
                // plus n.L (a multiple of 2^-q plus a remainder), all in FP32
                const int *oB = r.orgm + 3 * (size_t)r.cl_first[B];
                float D[3], H[3], R[3];
                for (int d = 0; d < 3; ++d) {
                    const float nd = (float)unpack_n(np, d);
                    H[d] = __fmaf_rn(nd, r.Lh[d], (float)(oB[d] - oA[d]) * (1.f / 1024.f));
                    R[d] = nd * r.Ll[d];
                    D[d] = H[d] + R[d];
                }
                dh = make_float4(H[0], H[1], H[2], __int_as_float(np));
                dl = make_float4(R[0], R[1], R[2], 0.f);
                js = a.cell_off[r.cl_first[B]];
                n = a.cell_off[r.cl_first[B + 1]] - js;
                // a partner cluster whose molecules' box (moved into A's frame) lies beyond
                // reach of molecule k holds none of its pairs
                const float4 bl = r.cl_box[2 * B], bh = r.cl_box[2 * B + 1];
                const float qx = fmaxf(fmaxf(bl.x + D[0] - kh.x, kh.x - (bh.x + D[0])), 0.f);
                const float qy = fmaxf(fmaxf(bl.y + D[1] - kh.y, kh.y - (bh.y + D[1])), 0.f);
                const float qz = fmaxf(fmaxf(bl.z + D[2] - kh.z, kh.z - (bh.z + D[2])), 0.f);
                if (qx * qx + qy * qy + qz * qz > reach * reach) n = 0;
            }
            int inc = n;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(FULL, inc, o);
                if (lane >= o) inc += y;
            }
            const int total = __shfl_sync(FULL, inc, 31);
            const bool live = n > 0;
            const unsigned lbal = __ballot_sync(FULL, live);
            if (live) {
                const int sl = __popc(lbal & lt);
                ed[wib][sl] = dh;
                el[wib][sl] = dl;
                eb[wib][sl] = js - (inc - n);
            }
            __syncwarp();
            for (int p0 = 0; p0 < total; p0 += 32) {
                const int b = inc - p0;
                const int base = __popc(__ballot_sync(FULL, live && b <= 0));
                const unsigned M = __reduce_or_sync(FULL, (live && b > 0 && b < 32) ? (1u << b) : 0u);
                const int p = p0 + lane;
                bool near = false;
                float4 q0 = make_float4(0.f, 0.f, 0.f, 0.f), q1 = q0;
                if (p < total) {
                    const int o = base + __popc(M & le);
                    const int l = p + eb[wib][o];
                    const float4 d = ed[wib][o], dlo = el[wib][o];
                    const int32_t nl = __float_as_int(d.w);
                    if (!(l == k && nl == 0)) {
                        float4 lh, ll;
                        grid_split(a.xloc[l], r.xlo[l], r.qround, lh, ll);
                        // separation k - (l + shift): exact hi part, small remainder
                        const float hx = kh.x - (lh.x + d.x), hy = kh.y - (lh.y + d.y), hz = kh.z - (lh.z + d.z);
                        const float lx = kl.x - (ll.x + dlo.x), ly = kl.y - (ll.y + dlo.y), lz = kl.z - (ll.z + dlo.z);
                        const float x = hx + lx, y = hy + ly, z = hz + lz;
                        near = x * x + y * y + z * z <= pre2;
                        q0 = make_float4(hx, hy, hz, lx);
                        q1 = make_float4(ly, lz, __int_as_float(l), __int_as_float(nl));
                    }
                }
                const unsigned nb = __ballot_sync(FULL, near);
                if (near) {
                    const int slot = nq + __popc(nb & lt);
                    rq[wib][slot][0] = q0;
                    rq[wib][slot][1] = q1;
                }
                nq += __popc(nb);
                __syncwarp();
                if (nq >= 32) {
                    drain(32);
                    nq -= 32;
                    if (lane < nq) {
                        rq[wib][lane][0] = rq[wib][32 + lane][0];
                        rq[wib][lane][1] = rq[wib][32 + lane][1];
                    }
                    __syncwarp();
                }
            }
        }
        if (nq > 0) drain(nq);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            Fx = ds_add(Fx, ds{__shfl_xor_sync(FULL, Fx.h, o), __shfl_xor_sync(FULL, Fx.l, o)});
            Fy = ds_add(Fy, ds{__shfl_xor_sync(FULL, Fy.h, o), __shfl_xor_sync(FULL, Fy.l, o)});
            Fz = ds_add(Fz, ds{__shfl_xor_sync(FULL, Fz.h, o), __shfl_xor_sync(FULL, Fz.l, o)});
        }
        if (lane == 0) {
            const int o = r.order[k];
            r.out[3 * (size_t)o] = Fx.h + Fx.l;
            r.out[3 * (size_t)o + 1] = Fy.h + Fy.l;
            r.out[3 * (size_t)o + 2] = Fz.h + Fz.l;
        }
    }
    }
}

// ---------------------------------------------------------------- adjoint
// Per pair with r = x_k - x_l', f = g(r^2) r, g = 24 e inv s3 (2 s3 - 1):
//   J = df/dr = g I + 2 g' r r^T,  g' = dg/d(r^2) = 24 e inv^2 s3 (4 - 14 s3).
// For L = sum_k v_k . F_k (v = dL/dF), a pair evaluated with Newton's third
// law (every scheduled pair under box periodicity, image pairs included)
// adds (v_k - v_l) . f, so with w = v_k - v_l x_k gets +J w and the partner
// (for an image pair, its source molecule) gets -J w.  A pair whose partner
// is referred through a general transform t (x_l' = y_t + R_t x_l, §2.2.2)
// acts on x_k only and is met again from the other side: w = v_k, and the
// source molecule gets -R_t^T J w.  dL/d eps_ab = g (r.w) / eps_ab and
// dL/d sigma_ab = 24 e inv s3 (24 s3 - 6) (r.w) / sigma_ab, chained to the
// species parameters through the mixing rule (eps_ab = sqrt(eps_a eps_b),
// sigma_ab = (sigma_a + sigma_b) / 2).  Pair terms are recomputed over the
// forward call's pair set (same schedule, same cut-off decisions).
//
// Species sums: slots [0, 8) hold dL/d eps_s and [8, 16) dL/d sigma_s; each
// warp adds its totals to the striped FP64 rows of the forward kernels, and
// finish_bwd adds the rows.
constexpr int kGradSlots = 2 * kMaxSpecies;
static_assert(kGradSlots <= kParts, "gradient slots must fit a stripe row");

struct BwdTab {
    double eps, sig2, inv_eps, inv_sig, fa, fb;   // fa, fb: d eps_ab / d eps_a, d eps_ab / d eps_b
};

struct BwdArgs {
    PairArgs p;
    BwdTab t[kMaxSpecies * kMaxSpecies];
    float4 tb[kMaxSpecies * kMaxSpecies];   // FP32 chain factors {fa / eps_ab, fb / eps_ab, 1 / (2 sigma_ab), 0}
    double e1, s1;                          // one species: 1 / eps, 1 / sigma
    int S;
};

// A warp's species-gradient totals (lane q < kGradSlots holds slot q) into its stripe row.
__device__ __forceinline__ void grads_to_stripe(const PairArgs &a, int gwarp, double g, int lane) {
    double *row = a.acc + kAccStripes + (size_t)(gwarp % kStripes) * kParts;
    if (lane < kGradSlots && g != 0.0) atomicAdd(row + lane, g);
}

// R^T g for a row-major FP32 rotation R
__device__ __forceinline__ float3 rot32t(const float *R, float x, float y, float z) {
    return make_float3(fmaf(R[0], x, fmaf(R[3], y, R[6] * z)), fmaf(R[1], x, fmaf(R[4], y, R[7] * z)),
                       fmaf(R[2], x, fmaf(R[5], y, R[8] * z)));
}

// One pair's adjoint terms (FP32 body, branch-free but for the species
// slots): +J w to gi3, -J w to gj; (r.w) g and (r.w) dg/d sigma to the species
// sums (one species: ea, sa in registers; several: the lane's column of the
// warp's slots gsl).
template <bool MULTI>
__device__ __forceinline__ void bwd32(const float4 *tab, const float4 *tb, float4 t0, int spi, int spj, float rx,
                                      float ry, float rz, float r2, bool in, float wx, float wy, float wz,
                                      float *gi3, R3<float> &gj, float &ea, float &sa, float (*gsl)[32], int lane) {
    const float4 t = MULTI ? tab[spi * kMaxSpecies + spj] : t0;
    const float inv = rcp_approx(r2);
    const float s = t.x * inv, s3 = s * s * s;
    const float a24 = (t.y * inv) * s3;
    const float rw = fmaf(rz, wz, fmaf(ry, wy, rx * wx));
    const float fs = in ? a24 * fmaf(2.f, s3, -1.f) : 0.f;
    const float c = in ? (2.f * a24 * inv) * fmaf(-14.f, s3, 4.f) * rw : 0.f;
    const float jx = fmaf(fs, wx, c * rx), jy = fmaf(fs, wy, c * ry), jz = fmaf(fs, wz, c * rz);
    gi3[0] += jx;
    gi3[1] += jy;
    gi3[2] += jz;
    gj.x -= jx;
    gj.y -= jy;
    gj.z -= jz;
    const float A = fs * rw;
    const float B = in ? a24 * fmaf(24.f, s3, -6.f) * rw : 0.f;
    if (MULTI) {
        if (in) {
            const int p = spi & (kMaxSpecies - 1), q = spj & (kMaxSpecies - 1);
            const float4 f = tb[p * kMaxSpecies + q];
            gsl[p][lane] = fmaf(A, f.x, gsl[p][lane]);
            gsl[q][lane] = fmaf(A, f.y, gsl[q][lane]);
            gsl[kMaxSpecies + p][lane] = fmaf(B, f.z, gsl[kMaxSpecies + p][lane]);
            gsl[kMaxSpecies + q][lane] = fmaf(B, f.z, gsl[kMaxSpecies + q][lane]);
        }
    } else {
        ea += A;
        sa += B;
    }
}

// One lane's partner (xj, its v in vl; vl = 0 for a one-sided pair) against
// the chunk: the forward's pair set (FP32 test, FP64 re-decision in the
// 1e-5 rc^2 band, SAME: chunk molecules below lmax_k only).
template <int NI_, bool MULTI, bool SAME, bool XF>
__device__ __forceinline__ unsigned bwd_partner(const PairArgs &a, const float4 *tab, const float4 *tb,
                                                const float4 *xi, const float4 *vi, int ni, int k0, float4 xj,
                                                float4 vl, int l, int np, int lmax_k, float (&gi)[3 * NI_],
                                                R3<float> &gj, float &ea, float &sa, float (*gsl)[32], int lane) {
    unsigned nin = 0, bm = 0;
    const float4 t0 = tab[0];
#pragma unroll
    for (int t = 0; t < NI_; ++t) {
        if (t < ni) {
            const float4 x = xi[t], vk = vi[t];
            const float rx = x.x - xj.x, ry = x.y - xj.y, rz = x.z - xj.z;
            const float r2 = fmaf(rz, rz, fmaf(ry, ry, rx * rx));
            const bool ok = !SAME || k0 + t < lmax_k;
            const bool in = ok && r2 < a.rc2_lo;
            if (ok && !in && r2 < a.rc2_hi) bm |= 1u << t;
            bwd32<MULTI>(tab, tb, t0, __float_as_int(x.w), __float_as_int(xj.w), rx, ry, rz, r2, in, vk.x - vl.x,
                         vk.y - vl.y, vk.z - vl.z, &gi[3 * t], gj, ea, sa, gsl, lane);
            nin += in;
        }
    }
    if (__any_sync(0xffffffffu, bm != 0)) {
#pragma unroll
        for (int t = 0; t < NI_; ++t) {
            if ((bm >> t) & 1u) {
                if (XF ? band_in_xf(a, k0 + t, l, np) : band_in(a, k0 + t, l, np)) {
                    const float4 x = xi[t], vk = vi[t];
                    const float rx = x.x - xj.x, ry = x.y - xj.y, rz = x.z - xj.z;
                    const float r2 = fmaf(rz, rz, fmaf(ry, ry, rx * rx));
                    bwd32<MULTI>(tab, tb, t0, __float_as_int(x.w), __float_as_int(xj.w), rx, ry, rz, r2, true,
                                 vk.x - vl.x, vk.y - vl.y, vk.z - vl.z, &gi[3 * t], gj, ea, sa, gsl, lane);
                    nin++;
                }
            }
        }
    }
    return nin;
}

template <int NI_>
struct WarpB32 {
    float4 qx[kRing];    // queued partners: position in I's frame (.w species bits)
    int2 ql[kRing];      // queued partners: binned index, image code (kSameCell: same cell)
    float4 ed[32];       // live runs of the batch (walk_runs)
    int eb[32];
    float4 xi[NI_];      // molecules of the current chunk
    float4 vi[NI_];      // ... and their v = dL/dF
};

// FP32 adjoint: the forward kernel's schedule walk (persistent grid, cells
// claimed from a counter, runs culled and queued, one partner per lane
// against the chunk), with the adjoint pair body.
template <int NI_, bool MULTI, bool XF, int MINB>
__global__ void __launch_bounds__(kThreads32, MINB) pair_bwd32(BwdArgs b) {
    const PairArgs &a = b.p;
    __shared__ float4 tab[kMaxSpecies * kMaxSpecies];
    __shared__ float4 tbs[MULTI ? kMaxSpecies * kMaxSpecies : 1];
    __shared__ WarpB32<NI_> wsh[kWarps32];
    __shared__ float slots[kWarps32][MULTI ? kGradSlots : 1][32];
    __shared__ float xR[XF ? kMaxXf : 1][9];
    for (int i = threadIdx.x; i < kMaxSpecies * kMaxSpecies; i += blockDim.x) {
        tab[i] = a.tab.f[i];
        if (MULTI) tbs[i] = b.tb[i];
    }
    if (XF)
        for (int i = threadIdx.x; i < 9 * kMaxXf; i += blockDim.x)
            xR[i / 9][i % 9] = (a.xft && i / 9 < a.n_xf) ? a.xft[i / 9].Rf[i % 9] : 0.f;
    for (int i = threadIdx.x; i < kWarps32 * (MULTI ? kGradSlots : 1) * 32; i += blockDim.x)
        (&slots[0][0][0])[i] = 0.f;
    __syncthreads();
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    WarpB32<NI_> &w = wsh[wib];
    float(*gsl)[32] = slots[wib];
    const unsigned FULL = 0xffffffffu, lt = (1u << lane) - 1u;
    const float4 far = make_float4(1e18f, 1e18f, 1e18f, 0.f), zero = make_float4(0.f, 0.f, 0.f, 0.f);
    const float rcut = sqrtf(a.rc2_hi);
    const float4 *vs = (const float4 *)a.vs;
    float4 *gacc = (float4 *)a.facc;
    float ea = 0.f, sa = 0.f;
    double dg = 0.0;     // lane q < kGradSlots: slot q
    // FP32 species sums into the lane's FP64 slot (every few cells)
    auto flush = [&]() {
        if (MULTI) {
            __syncwarp();
            if (lane < kGradSlots) {
                double t = 0.0;
                for (int c = 0; c < 32; ++c) {
                    const int cc = (c + lane) & 31;
                    t += (double)gsl[lane][cc];
                    gsl[lane][cc] = 0.f;
                }
                dg += t;
            }
            __syncwarp();
        } else {
            const float e = warp_sum(ea), s = warp_sum(sa);
            if (lane == 0) dg += (double)e * b.e1;
            if (lane == kMaxSpecies) dg += (double)s * b.s1;
            ea = sa = 0.f;
        }
    };
    int ncell = 0;
    int I0 = lane == 0 ? (int)atomicAdd(a.next_cell, (unsigned)kGrab) : 0;
    I0 = __shfl_sync(FULL, I0, 0);
    while (I0 < a.C) {
        const int Inext = lane == 0 ? (int)atomicAdd(a.next_cell, (unsigned)kGrab) : 0;
        const int Iend = min(I0 + kGrab, a.C);
        for (int I = I0; I < Iend; ++I) {
            const int s0 = a.cell_off[I], nI = a.cell_off[I + 1] - s0;
            if (nI == 0) continue;
            const int e0 = a.run_off[I], e1 = a.run_off[I + 1];
            const float4 sI = a.sph[I];
            const int *oI = a.orgm + 3 * I;
            const float cull_i = (rcut + sI.w) * (rcut + sI.w) * 1.00002f + 1e-5f;
            for (int i0 = 0; i0 < nI; i0 += NI_) {
                const int ni = min(NI_, nI - i0), k0 = s0 + i0;
                __syncwarp();
                if (lane < ni) {
                    w.xi[lane] = a.xloc[k0 + lane];
                    w.vi[lane] = vs[k0 + lane];
                }
                float gi[3 * NI_];
#pragma unroll
                for (int i = 0; i < 3 * NI_; ++i) gi[i] = 0.f;
                int head = 0, qn = 0;
                __syncwarp();
                auto run = [&](int count) {
                    const int s = (head + lane) & (kRing - 1);
                    const bool valid = lane < count;
                    const float4 xj = valid ? w.qx[s] : far;
                    const int2 q = valid ? w.ql[s] : make_int2(0, 0);
                    const bool same = q.y == kSameCell;
                    const bool one = XF && !same && q.y != 0;
                    const float4 vl = valid && !one ? vs[q.x] : zero;
                    R3<float> gj = {0.f, 0.f, 0.f};
                    const unsigned nin =
                        __any_sync(FULL, same)
                            ? bwd_partner<NI_, MULTI, true, XF>(a, tab, tbs, w.xi, w.vi, ni, k0, xj, vl, q.x,
                                                                same ? 0 : q.y, same ? q.x : 0x7fffffff, gi, gj, ea,
                                                                sa, gsl, lane)
                            : bwd_partner<NI_, MULTI, false, XF>(a, tab, tbs, w.xi, w.vi, ni, k0, xj, vl, q.x, q.y, 0,
                                                                 gi, gj, ea, sa, gsl, lane);
                    if (nin) {
                        if (one) {
                            const float3 r = rot32t(xR[q.y], gj.x, gj.y, gj.z);
                            gj.x = r.x; gj.y = r.y; gj.z = r.z;
                        }
                        atomicAdd(gacc + q.x, make_float4(gj.x, gj.y, gj.z, 0.f));
                    }
                    head = (head + count) & (kRing - 1);
                    __syncwarp();
                };
                auto push = [&](bool alive, float4 xj, int l, int np) {
                    const unsigned bal = __ballot_sync(FULL, alive);
                    if (alive) {
                        const int s = (head + qn + __popc(bal & lt)) & (kRing - 1);
                        w.qx[s] = xj;
                        w.ql[s] = make_int2(l, np);
                    }
                    qn += __popc(bal);
                    __syncwarp();
                    if (qn >= 32) {
                        run(32);
                        qn -= 32;
                    }
                };
                for (int lb = i0 + 1; lb < nI; lb += 32) {
                    const int li = lb + lane;
                    const bool alive = li < nI;
                    push(alive, alive ? a.xloc[s0 + li] : far, s0 + li, kSameCell);
                }
                walk_runs<XF, false>(a, w.ed, w.eb, nullptr, xR, e0, e1, ni, oI, sI, rcut, cull_i, lane, push);
                if (qn > 0) run(qn);
                chunk_reduce<NI_>(gi, lane);
                const int t = lane / (32 / NI_);
                if ((lane & (32 / NI_ - 1)) == 0 && t < ni)
                    atomicAdd(gacc + k0 + t, make_float4(gi[0], gi[1], gi[2], 0.f));
            }
            if (++ncell == 4) {
                ncell = 0;
                flush();
            }
        }
        I0 = __shfl_sync(FULL, Inext, 0);
    }
    flush();
    grads_to_stripe(a, blockIdx.x * kWarps32 + wib, dg, lane);
}

// FP64 pair terms (same formulas)
template <bool MULTI>
__device__ __forceinline__ void bwd64(const BwdTab *tab, int spi, int spj, double rx, double ry, double rz, double r2,
                                      double wx, double wy, double wz, R3<double> &gi, R3<double> &gj, double &ea,
                                      double &sa, double (*gsl)[32], int lane) {
    spi &= kMaxSpecies - 1;
    spj &= kMaxSpecies - 1;
    const BwdTab &t = tab[MULTI ? spi * kMaxSpecies + spj : 0];
    const double inv = 1.0 / r2;
    const double s = t.sig2 * inv, s3 = s * s * s;
    const double a24 = 24.0 * t.eps * inv * s3;
    const double fs = a24 * (2.0 * s3 - 1.0);
    const double rw = rx * wx + ry * wy + rz * wz;
    const double c = 2.0 * a24 * inv * (4.0 - 14.0 * s3) * rw;
    const double jx = fs * wx + c * rx, jy = fs * wy + c * ry, jz = fs * wz + c * rz;
    gi.x += jx; gi.y += jy; gi.z += jz;
    gj.x -= jx; gj.y -= jy; gj.z -= jz;
    const double A = fs * rw * t.inv_eps;
    const double B = a24 * (24.0 * s3 - 6.0) * rw * t.inv_sig;
    if (MULTI) {
        gsl[spi][lane] += A * t.fa;
        gsl[spj][lane] += A * t.fb;
        gsl[kMaxSpecies + spi][lane] += 0.5 * B;
        gsl[kMaxSpecies + spj][lane] += 0.5 * B;
    } else {
        ea += A;
        sa += B;
    }
}

// FP64 adjoint: one warp per cell I, lanes over the (molecule of I, partner
// molecule) pairs of one schedule entry at a time; pairs within rc are
// decided in FP64 exactly as the forward FP64 kernel decides them.
template <bool MULTI, bool XF>
__global__ void __launch_bounds__(kPairThreads) pair_bwd64(BwdArgs b) {
    const PairArgs &a = b.p;
    __shared__ BwdTab tab[kMaxSpecies * kMaxSpecies];
    __shared__ double slots[kWarps][MULTI ? kGradSlots : 1][32];
    for (int i = threadIdx.x; i < kMaxSpecies * kMaxSpecies; i += blockDim.x) tab[i] = b.t[i];
    for (int i = threadIdx.x; i < kWarps * (MULTI ? kGradSlots : 1) * 32; i += blockDim.x)
        (&slots[0][0][0])[i] = 0.0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int gwarp = blockIdx.x * kWarps + wib, nwarps = gridDim.x * kWarps;
    double(*gsl)[32] = slots[wib];
    const double *vs = (const double *)a.vs;
    double *gacc = (double *)a.facc;
    double ea = 0.0, sa = 0.0;
    for (int I = gwarp; I < a.C; I += nwarps) {
        const int sI = a.cell_off[I], nI = a.cell_off[I + 1] - sI;
        if (nI == 0) continue;
        const int e0 = a.work_off[I], e1 = a.work_off[I + 1];
        // entry e0 - 1 stands for the cell itself (pairs k' > k)
        for (int e = e0 - 1; e < e1; ++e) {
            int J = I, np = 0;
            if (e >= e0) {
                const WorkEntry we = a.work[e];
                J = we.j;
                np = we.n;
            }
            const bool one = XF && np != 0;
            const int sJ = a.cell_off[J], nJ = a.cell_off[J + 1] - sJ;
            const int npairs = nI * nJ;
            for (int p = lane; p < npairs; p += 32) {
                const int ki = p / nJ, lj = p - ki * nJ;
                if (e < e0 && lj <= ki) continue;
                const int k = sI + ki, l = sJ + lj;
                double rx, ry, rz, r2;
                sep64x<XF>(a, a.xs64 + 3 * (size_t)k, a.xs64 + 3 * (size_t)l, np, rx, ry, rz, r2);
                if (!(r2 < a.rc2_d)) continue;
                const double *vk = vs + 4 * (size_t)k, *vl = vs + 4 * (size_t)l;
                const double wx = one ? vk[0] : vk[0] - vl[0];
                const double wy = one ? vk[1] : vk[1] - vl[1];
                const double wz = one ? vk[2] : vk[2] - vl[2];
                R3<double> gi = {0, 0, 0}, gj = {0, 0, 0};
                bwd64<MULTI>(tab, __float_as_int(a.xloc[k].w), __float_as_int(a.xloc[l].w), rx, ry, rz, r2, wx, wy,
                             wz, gi, gj, ea, sa, gsl, lane);
                atomic_add3(gacc + 4 * (size_t)k, gi.x, gi.y, gi.z);
                if (one) {
                    const double *R = a.xft[np].R;
                    atomic_add3(gacc + 4 * (size_t)l, R[0] * gj.x + R[3] * gj.y + R[6] * gj.z,
                                R[1] * gj.x + R[4] * gj.y + R[7] * gj.z, R[2] * gj.x + R[5] * gj.y + R[8] * gj.z);
                } else {
                    atomic_add3(gacc + 4 * (size_t)l, gj.x, gj.y, gj.z);
                }
            }
        }
    }
    double dg = 0.0;
    if (MULTI) {
        __syncwarp();
        if (lane < kGradSlots)
            for (int c = 0; c < 32; ++c) dg += gsl[lane][(c + lane) & 31];
    } else {
        const double e = warp_sum(ea), s = warp_sum(sa);
        dg = lane == 0 ? e : lane == kMaxSpecies ? s : 0.0;
    }
    grads_to_stripe(a, gwarp, dg, lane);
}

template <class T>
__global__ void __launch_bounds__(256) gather_grad(const int *order, int64_t nb, const T *g, void *vs, int f64) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nb) return;
    int k = order[s];
    if (f64) {
        double *v = (double *)vs + 4 * (size_t)s;
        v[0] = (double)g[3 * (size_t)k]; v[1] = (double)g[3 * (size_t)k + 1]; v[2] = (double)g[3 * (size_t)k + 2];
        v[3] = 0;
    } else {
        ((float4 *)vs)[s] = make_float4((float)g[3 * (size_t)k], (float)g[3 * (size_t)k + 1], (float)g[3 * (size_t)k + 2], 0.f);
    }
}

// Totals of the species-gradient slots over the stripe rows (one warp per slot).
__global__ void __launch_bounds__(kGradSlots * 32) finish_bwd(const double *acc, int S, double *ge, double *gs) {
    const int i = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double v = 0.0;
    for (int r = lane; r < kStripes; r += 32) v += acc[kAccStripes + r * kParts + i];
    v = warp_sum(v);
    const int q = i % kMaxSpecies;
    if (lane == 0 && q < S) {
        if (i < kMaxSpecies) {
            if (ge) ge[q] = v;
        } else if (gs) {
            gs[q] = v;
        }
    }
}

// ------------------------------------------------------ FP32 cluster kernel
// The box-periodic FP32 forces over clusters (runs of consecutive cells,
// mesh.cu) instead of single cells.  A warp takes one cluster A at a time:
//   1. the joint bounding box of A's molecules (this step's positions);
//   2. candidates: A's own molecules (pairs k < l, §2.3's same-cell rule
//      extended to the cluster) and the molecules of the partner runs of A's
//      cluster schedule, each moved into A's frame by the run's shift; a
//      candidate farther than rc from the box cannot pair with any molecule
//      of A (margins above the FP32 cut-off) and is dropped, the rest go to
//      a per-warp survivor buffer in shared memory;
//   3. whenever the buffer cannot take 32 more survivors, and at the end:
//      for every i-tile of kNI molecules of A, every batch of 32 survivors
//      is evaluated one survivor per lane against the tile (the tile's
//      molecules read from shared memory): forces by FMA, the survivor's
//      reaction summed in registers and added to its slot of the buffer, the
//      tile's forces summed per lane and over the warp at the end of the tile
//      (recursive halving), one vector atomic per molecule;
//   4. one vector atomic per survivor adds its reaction.
// Separations are formed exactly before one rounding: binned coordinates are
// multiples of 2^-q (xloc) plus a remainder (xlo), run shifts likewise, so
// (x_k,hi - x_l,hi - shift_hi) is exact and adding the remainders rounds once.
// Every force accumulator's .w sums |f|^2 over the molecule's pairs: the
// scale of the FP32 error of its force (see flag_ill_conditioned and
// refine_ds).
struct ClKArgs {
    const int *cl_first, *cl_run_off;
    const ClRun *runs;
    const float4 *xlo;
    float4 *cl_box;              // out: each cluster's box of molecules (lo, hi; hi parts, own frame)
    int ncl;
    float qround;                // 1.5 * 2^(23 - q): x + qround - qround rounds x to a multiple of 2^-q
};


constexpr int kCT = 128, kCW = kCT / 32;
// A molecule's FP32 force error is about a multiple of sqrt(sum_l |f_kl|^2)
// (rounding of each pair force, mostly; the separations are rounded once);
// kRefineScale bounds that multiple with a wide safety margin.  A molecule
// whose force is below kRefineScale / tol times that scale gets refined.
constexpr double kRefineScale = 1.25e-6;
constexpr int kCap = 176;                 // survivors buffered per warp (5 blocks of 4 warps per SM)
constexpr int kNI = 8;                    // molecules of A per i-tile
// packed survivor / tile word (.w of the hi position)
constexpr int kSpBits = 7, kSameBit = 1 << 3, kImgBit = 1 << 4, kGhostW = 1 << 21;
__device__ __forceinline__ int cellq_of(int w) { return (w >> 5) & 15; }
__device__ __forceinline__ int32_t n_of(int w) {   // 3 x 4-bit image -> pack_n
    const int c = w >> 9;
    return pack_n((c << 28) >> 28, (c << 24) >> 28, (c << 20) >> 28);
}

struct WarpC {
    float4 sh[kCap];      // survivor: position in A's frame, hi part (exact); .w packed word
    float4 sl[kCap];      // survivor: remainder (xyz); .w binned index (int bits)
    float4 sf[kCap];      // survivor: reaction (xyz) and sum of |f|^2 (w) over the tiles
    float4 ih[kNI];       // tile: hi part; .w packed word (species, cell within the cluster);
    float4 il[kNI];       //   unused slots hold a far-away dummy
    float4 ed[32], el[32];
    int eb[32];
    float box[6];         // joint box of A's molecules (lo, hi)
    float vl[6][32];      // per-lane virial sums (xx, yy, zz, xy, xz, yz) of the current cluster
    unsigned cnt[2];      // pair tests, culling tests
};

// One pair of the cluster kernel (FP32 body, branch-free): tile molecule t
// (h, lo) against a lane's survivor (xh, xl); the force goes to fi[4t..] and
// fj, |f|^2 to both .w/[4t+3], the energy to u_acc; a pair whose FP32 r^2
// falls within the 1e-5 rc^2 band sets bit t of bm for the FP64 re-decision
// after the tile (band_pair).  Pairs outside rc get 1/r^2 = 0, which zeroes
// their force and energy without further selects: u = 4 eps (s^6 - s^3).
template <bool MULTI, bool SHIFT, bool SAME, bool GHOST>
__device__ __forceinline__ void tile_pair(const PairArgs &a, const float4 *tab, float4 t0, float4 h, float4 lo,
                                          float4 xh, float4 xl, int t, int k0, float (&fi)[4 * kNI],
                                          float4 &fj, float &u_acc, unsigned &nin, unsigned &nsame, unsigned &bm,
                                          float (&vg)[6]) {
    const int wi = __float_as_int(h.w), wj = __float_as_int(xh.w), l = __float_as_int(xl.w);
    const bool sj = SAME && (wj & kSameBit) != 0;
    const float rx = (h.x - xh.x) + (lo.x - xl.x);
    const float ry = (h.y - xh.y) + (lo.y - xl.y);
    const float rz = (h.z - xh.z) + (lo.z - xl.z);
    const float r2 = fmaf(rz, rz, fmaf(ry, ry, rx * rx));
    // portion mode: a pair of two halo molecules is not evaluated here,
    // an owned-halo pair carries half its energy and virial
    const bool gi = GHOST && (wi & kGhostW), gj = GHOST && (wj & kGhostW);
    const bool ok = (!sj || k0 + t < l) && !(gi && gj);
    const bool in = ok && r2 < a.rc2_lo;
    if (ok && !in && r2 < a.rc2_hi) bm |= 1u << t;
    const float4 p = MULTI ? tab[(wi & kSpBits) * kMaxSpecies + (wj & kSpBits)] : t0;
    const float inv = in ? rcp_approx(r2) : 0.f;      // (r^2 = 0 for a molecule against itself)
    const float s = p.x * inv;
    const float s3 = s * s * s;
    const float fs = (p.y * inv) * s3 * fmaf(2.f, s3, -1.f);
    const float v = fmaf(s3, s3, -s3);
    const float wt = (GHOST && (gi || gj)) ? 0.5f : 1.f;
    u_acc = fmaf(GHOST ? wt * p.z : p.z, v, u_acc);
    if (SHIFT) u_acc -= in ? (GHOST ? wt * p.w : p.w) : 0.f;
    if (GHOST) {
        const float g = wt * fs, gx = g * rx, gy = g * ry;
        vg[0] = fmaf(gx, rx, vg[0]);
        vg[1] = fmaf(gy, ry, vg[1]);
        vg[2] = fmaf(g * rz, rz, vg[2]);
        vg[3] = fmaf(gx, ry, vg[3]);
        vg[4] = fmaf(gx, rz, vg[4]);
        vg[5] = fmaf(gy, rz, vg[5]);
    }
    fi[4 * t] = fmaf(fs, rx, fi[4 * t]);
    fi[4 * t + 1] = fmaf(fs, ry, fi[4 * t + 1]);
    fi[4 * t + 2] = fmaf(fs, rz, fi[4 * t + 2]);
    fj.x = fmaf(-fs, rx, fj.x);
    fj.y = fmaf(-fs, ry, fj.y);
    fj.z = fmaf(-fs, rz, fj.z);
    const float g = fs * fs;
    fi[4 * t + 3] = fmaf(g, r2, fi[4 * t + 3]);
    fj.w = fmaf(g, r2, fj.w);
    nin += in;
    if (SAME) nsame += (in && sj && cellq_of(wi) == cellq_of(wj)) ? 1u : 0u;
}

// x (x) f added to the virial sums v[0], v[S], .. v[5 S] (xx, yy, zz, xy, xz, yz)
template <int S = 1>
__device__ __forceinline__ void vir_add(float *v, float x, float y, float z, float fx, float fy, float fz) {
    v[0] = fmaf(x, fx, v[0]);
    v[S] = fmaf(y, fy, v[S]);
    v[2 * S] = fmaf(z, fz, v[2 * S]);
    v[3 * S] = fmaf(x, fy, v[3 * S]);
    v[4 * S] = fmaf(x, fz, v[4 * S]);
    v[5 * S] = fmaf(y, fz, v[5 * S]);
}

// A pair of the 1e-5 rc^2 band that the FP64 decision puts within rc: the
// body of tile_pair with the pair inside, the tile molecule's force added
// to its accumulator at once (rare; one copy of the body in the code).
template <bool MULTI, bool SHIFT, bool SAME, bool GHOST>
__device__ __forceinline__ void band_pair(const PairArgs &a, const float4 *tab, float4 t0, float4 h, float4 lo,
                                       float4 xh, float4 xl, float4 &fj, float &u_acc, unsigned &nin,
                                       unsigned &nsame, float (&vg)[6], float *vl, float4 *fdst) {
    const int wi = __float_as_int(h.w), wj = __float_as_int(xh.w);
    const bool sj = SAME && (wj & kSameBit) != 0;
    const float rx = (h.x - xh.x) + (lo.x - xl.x);
    const float ry = (h.y - xh.y) + (lo.y - xl.y);
    const float rz = (h.z - xh.z) + (lo.z - xl.z);
    const float r2 = fmaf(rz, rz, fmaf(ry, ry, rx * rx));
    const bool gi = GHOST && (wi & kGhostW), gj = GHOST && (wj & kGhostW);
    const float4 p = MULTI ? tab[(wi & kSpBits) * kMaxSpecies + (wj & kSpBits)] : t0;
    const float inv = rcp_approx(r2);
    const float s = p.x * inv;
    const float s3 = s * s * s;
    const float fs = (p.y * inv) * s3 * fmaf(2.f, s3, -1.f);
    const float wt = (GHOST && (gi || gj)) ? 0.5f : 1.f;
    u_acc = fmaf(GHOST ? wt * p.z : p.z, fmaf(s3, s3, -s3), u_acc);
    if (SHIFT) u_acc -= GHOST ? wt * p.w : p.w;
    const float fx = fs * rx, fy = fs * ry, fz = fs * rz, g = fs * fs * r2;
    fj.x -= fx;
    fj.y -= fy;
    fj.z -= fz;
    fj.w += g;
    atomicAdd(fdst, make_float4(fx, fy, fz, g));
    if (GHOST) {
        const float q = wt * fs, gx = q * rx, gy = q * ry;
        vg[0] = fmaf(gx, rx, vg[0]);
        vg[1] = fmaf(gy, ry, vg[1]);
        vg[2] = fmaf(q * rz, rz, vg[2]);
        vg[3] = fmaf(gx, ry, vg[3]);
        vg[4] = fmaf(gx, rz, vg[4]);
        vg[5] = fmaf(gy, rz, vg[5]);
    } else {
        vir_add<32>(vl, h.x, h.y, h.z, fx, fy, fz);     // the force issued on the tile molecule
    }
    nin += 1u;
    if (SAME) nsame += (sj && cellq_of(wi) == cellq_of(wj)) ? 1u : 0u;
}

// A lane's survivor (xh, xl) against the tile (broadcast from shared
// memory); afterwards the pairs whose FP32 r^2 fell in the 1e-5 rc^2 band
// are re-decided in FP64 with the all-pairs operation order.  SAME:
// own-cluster survivors pair only with tile molecules of lower binned index.
template <bool MULTI, bool SHIFT, bool SAME, bool GHOST>
__device__ __forceinline__ void eval_tile(const PairArgs &a, const float4 *tab, const float4 *th, const float4 *tl,
                                          int ni, int k0,
                                          float4 xh, float4 xl, float (&fi)[4 * kNI], float4 &fj, float &u_acc,
                                          unsigned &nin, unsigned &nsame, float (&vg)[6], float *vl,
                                          float4 *facc) {
    unsigned bm = 0;
    const float4 t0 = tab[0];
#pragma unroll
    for (int t = 0; t < kNI; ++t) {
        if (t >= ni) break;
        const float4 h = th[t], lo = tl[t];
        tile_pair<MULTI, SHIFT, SAME, GHOST>(a, tab, t0, h, lo, xh, xl, t, k0, fi, fj, u_acc, nin, nsame, bm, vg);
    }
    if (__any_sync(0xffffffffu, bm != 0)) {
        const int l = __float_as_int(xl.w);
        const int32_t np = n_of(__float_as_int(xh.w));
#pragma unroll 1
        for (int t = 0; t < ni; ++t)
            if (((bm >> t) & 1u) && band_in(a, k0 + t, l, np))
                band_pair<MULTI, SHIFT, SAME, GHOST>(a, tab, t0, th[t], tl[t], xh, xl, fj, u_acc, nin, nsame, vg,
                                                     vl, facc + k0 + t);
    }
}

// Sum v[0..4 kNI) (kNI groups of x, y, z, |f|^2) over the warp by recursive
// halving: on return lanes t * (32 / kNI) .. hold the totals of group t in v[0..4).
__device__ __forceinline__ void tile_reduce4(float (&v)[4 * kNI], int lane) {
    halve<4 * kNI>(v, lane, 16);
    halve<2 * kNI>(v, lane, 8);
    halve<kNI>(v, lane, 4);
#pragma unroll
    for (int o = 2; o > 0; o >>= 1)
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
}

template <bool MULTI, bool SHIFT, bool GHOST, int MINB>
__global__ void __launch_bounds__(kCT, MINB) pair_fwd32c(PairArgs a, ClKArgs c) {
    extern __shared__ float4 csh[];
    WarpC *wsh = reinterpret_cast<WarpC *>(csh);
    __shared__ float4 tab[kMaxSpecies * kMaxSpecies];
    __shared__ double dsums[kCW][8];
    for (int i = threadIdx.x; i < kMaxSpecies * kMaxSpecies; i += blockDim.x) tab[i] = a.tab.f[i];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    WarpC &w = wsh[wib];
    if (lane < 8) dsums[wib][lane] = 0.0;
    if (lane < 2) w.cnt[lane] = 0;
    __syncthreads();
    const unsigned FULL = 0xffffffffu, lt = (1u << lane) - 1u, le = FULL >> (31 - lane);
    const float4 far = make_float4(1e18f, 1e18f, 1e18f, 0.f), zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const float rcut = sqrtf(a.rc2_hi) * 1.00001f + 1e-5f;
    const float rcut2 = rcut * rcut;
    float4 *facc = (float4 *)a.facc;
    double *dsum = dsums[wib];
    float u_acc = 0.f;
    // virial: sum of x (x) F over the forces this lane issues (positions in
    // the cluster's frame; the forces of a cluster sum to zero, so this is
    // the sum of r (x) f over its pairs), in the lane's column vl of shared
    // memory; portion mode sums r (x) f per pair in registers (vg)
    float vg[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float *vl = &w.vl[0][lane];
#pragma unroll
    for (int i = 0; i < 6; ++i) vl[32 * i] = 0.f;
    unsigned wc0 = 0, wc1 = 0, wc2 = 0;     // this lane's pairs within rc: same cell, DIL, image
    for (;;) {
        int A = lane == 0 ? (int)atomicAdd(a.next_cell, 1u) : 0;
        A = __shfl_sync(FULL, A, 0);
        if (A >= c.ncl) break;
        const int c0 = c.cl_first[A], c1 = c.cl_first[A + 1];
        const int s0 = a.cell_off[c0], s1 = a.cell_off[c1], nA = s1 - s0;
        if (nA == 0) {
            if (lane == 0) {
                c.cl_box[2 * A] = make_float4(1e30f, 1e30f, 1e30f, 0.f);
                c.cl_box[2 * A + 1] = make_float4(-1e30f, -1e30f, -1e30f, 0.f);
            }
            continue;
        }
        // 1. joint box of A's molecules (hi parts; the remainders lie inside the margins)
        float bl[3] = {1e30f, 1e30f, 1e30f}, bh[3] = {-1e30f, -1e30f, -1e30f};
        for (int k = s0 + lane; k < s1; k += 32) {
            const float4 x = a.xloc[k];
            bl[0] = fminf(bl[0], x.x); bl[1] = fminf(bl[1], x.y); bl[2] = fminf(bl[2], x.z);
            bh[0] = fmaxf(bh[0], x.x); bh[1] = fmaxf(bh[1], x.y); bh[2] = fmaxf(bh[2], x.z);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                bl[d] = fminf(bl[d], __shfl_xor_sync(FULL, bl[d], o));
                bh[d] = fmaxf(bh[d], __shfl_xor_sync(FULL, bh[d], o));
            }
        if (lane < 3) {
            w.box[lane] = lane == 0 ? bl[0] : lane == 1 ? bl[1] : bl[2];
            w.box[3 + lane] = lane == 0 ? bh[0] : lane == 1 ? bh[1] : bh[2];
        }
        if (lane == 0) {
            c.cl_box[2 * A] = make_float4(bl[0], bl[1], bl[2], 0.f);
            c.cl_box[2 * A + 1] = make_float4(bh[0], bh[1], bh[2], 0.f);
        }
        __syncwarp();
        int nq = 0;
        // append the live lanes' candidates to the buffer
        auto push = [&](bool alive, float4 xh, float4 xl) {
            const unsigned bal = __ballot_sync(FULL, alive);
            if (alive) {
                const int sl = nq + __popc(bal & lt);
                w.sh[sl] = xh;
                w.sl[sl] = xl;
                w.sf[sl] = zero4;
            }
            nq += __popc(bal);
        };
        // 2. fill the buffer (A's own molecules, then the partner runs 32 at
        // a time) until it cannot take 32 more; 3./4. evaluate it; repeat
        int own = s0;                               // next own molecule to push
        bool own_first = true;                      // no flush of this cluster yet
        const int e1 = c.cl_run_off[A + 1];
        int eb = c.cl_run_off[A];                   // next batch of 32 runs
        int p0 = 0, total = 0, inc = 0;             // candidate cursor of the loaded batch
        bool live = false;
        for (;;) {
            bool more = true;
            while (nq <= kCap - 32) {
                if (own < s1) {
                    // 2a. A's own molecules: pairs k < l inside the cluster
                    const int k = own + lane;
                    const bool alive = k < s1;
                    float4 xh = far, xl = zero4;
                    if (alive) {
                        const float4 r = c.xlo[k];
                        grid_split(a.xloc[k], r, c.qround, xh, xl);
                        const int q = __float_as_int(r.w) & 15;     // cell label within the cluster
                        const int w0 = __float_as_int(xh.w);
                        xh.w = __int_as_float((w0 & kSpBits) | kSameBit | (q << 5) | ((w0 & kGhostBit) ? kGhostW : 0));
                        xl.w = __int_as_float(k);
                    }
                    push(alive, xh, xl);
                    own += 32;
                } else if (p0 < total) {
                    // 2b. candidates p0 .. p0 + 31 of the loaded runs: moved into
                    // A's frame, culled against A's box, compacted
                    const int b = inc - p0;
                    const int base = __popc(__ballot_sync(FULL, live && b <= 0));
                    const unsigned M = __reduce_or_sync(FULL, (live && b > 0 && b < 32) ? (1u << b) : 0u);
                    const int p = p0 + lane;
                    bool alive = false;
                    float4 xh = far, xl = zero4;
                    if (p < total) {
                        const int o = base + __popc(M & le);
                        const int l = p + w.eb[o];
                        const float4 dh = w.ed[o], dl = w.el[o];
                        float4 x, y;
                        grid_split(a.xloc[l], c.xlo[l], c.qround, x, y);
                        xh = make_float4(x.x + dh.x, x.y + dh.y, x.z + dh.z, 0.f);
                        const float dx = fmaxf(fmaxf(w.box[0] - xh.x, xh.x - w.box[3]), 0.f);
                        const float dy = fmaxf(fmaxf(w.box[1] - xh.y, xh.y - w.box[4]), 0.f);
                        const float dz = fmaxf(fmaxf(w.box[2] - xh.z, xh.z - w.box[5]), 0.f);
                        alive = dx * dx + dy * dy + dz * dz <= rcut2;
                        const int code = __float_as_int(dl.w) >> 12;
                        const int w0 = __float_as_int(x.w);
                        xh.w = __int_as_float((w0 & kSpBits) | (code != 0 ? kImgBit : 0) | (code << 9) |
                                              ((w0 & kGhostBit) ? kGhostW : 0));
                        xl = make_float4(y.x + dl.x, y.y + dl.y, y.z + dl.z, __int_as_float(l));
                    }
                    push(alive, xh, xl);
                    p0 += 32;
                } else if (eb < e1) {
                    // the next 32 partner runs: candidate counts prefix-summed,
                    // live runs compacted into ed / el / eb
                    const bool has = eb + lane < e1;
                    int js = 0, n = 0;
                    ClRun r;
                    r.dh = zero4;
                    r.dl = zero4;
                    if (has) {
                        r = c.runs[eb + lane];
                        const int cf = __float_as_int(r.dh.w), code = __float_as_int(r.dl.w);
                        js = a.cell_off[cf];
                        n = a.cell_off[cf + (code & 4095)] - js;
                    }
                    inc = n;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int y = __shfl_up_sync(FULL, inc, o);
                        if (lane >= o) inc += y;
                    }
                    total = __shfl_sync(FULL, inc, 31);
                    live = n > 0;
                    const unsigned lbal = __ballot_sync(FULL, live);
                    __syncwarp();                       // the previous runs' readers are done
                    if (live) {
                        const int sl = __popc(lbal & lt);
                        w.ed[sl] = r.dh;
                        w.el[sl] = r.dl;
                        w.eb[sl] = js - (inc - n);
                    }
                    if (lane == 0) w.cnt[1] += (unsigned)total;
                    __syncwarp();
                    eb += 32;
                    p0 = 0;
                } else {
                    more = false;
                    break;
                }
            }
            if (nq > 0) {
                // 3. every tile of A against the buffered survivors; while A's own
                // molecules are all in the buffer (slots 0 .. nA - 1, as in the
                // first flush of a cluster below the fill threshold) the tiles
                // are read there, in the same representation
                __syncwarp();
                const bool own_buf = own_first && own >= s1;
                for (int i0 = 0; i0 < nA; i0 += kNI) {
                    const int ni = min(kNI, nA - i0), k0 = s0 + i0;
                    const float4 *th = own_buf ? &w.sh[i0] : w.ih, *tl = own_buf ? &w.sl[i0] : w.il;
                    if (!own_buf && lane < kNI) {
                        float4 h = make_float4(1e18f, 1e18f, 1e18f, 0.f), lo = zero4;
                        if (lane < ni) {
                            const float4 r = c.xlo[k0 + lane];
                            grid_split(a.xloc[k0 + lane], r, c.qround, h, lo);
                            const int q = __float_as_int(r.w) & 15;
                            const int w0 = __float_as_int(h.w);
                            h.w = __int_as_float((w0 & kSpBits) | (q << 5) | ((w0 & kGhostBit) ? kGhostW : 0));
                        }
                        w.ih[lane] = h;
                        w.il[lane] = lo;
                    }
                    if (lane == 0) w.cnt[0] += (unsigned)(nq * ni);
                    float fi[4 * kNI];
#pragma unroll
                    for (int i = 0; i < 4 * kNI; ++i) fi[i] = 0.f;
                    __syncwarp();
                    for (int jb = 0; jb < nq; jb += 32) {
                        const int j = jb + lane;
                        const bool valid = j < nq;
                        const float4 xh = valid ? w.sh[j] : make_float4(-1e18f, -1e18f, -1e18f, 0.f);
                        const float4 xl = valid ? w.sl[j] : zero4;
                        float4 fj = zero4;
                        unsigned nin = 0, nsame = 0;
                        if (__any_sync(FULL, (__float_as_int(xh.w) & kSameBit) != 0))
                            eval_tile<MULTI, SHIFT, true, GHOST>(a, tab, th, tl, ni, k0, xh, xl, fi, fj, u_acc, nin,
                                                                 nsame, vg, vl, facc);
                        else
                            eval_tile<MULTI, SHIFT, false, GHOST>(a, tab, th, tl, ni, k0, xh, xl, fi, fj, u_acc, nin,
                                                                  nsame, vg, vl, facc);
                        {
                            // within-rc counts per category (same cell, DIL, periodic image),
                            // without branches (nin = nsame = 0 on invalid lanes)
                            const int wq = __float_as_int(xh.w);
                            const unsigned img = (wq & kImgBit) ? nin : 0u;
                            wc0 += nsame;
                            wc1 += nin - nsame - img;
                            wc2 += img;
                        }
                        if (valid && nin) {
                            float4 f = w.sf[j];
                            f.x += fj.x; f.y += fj.y; f.z += fj.z; f.w += fj.w;
                            w.sf[j] = f;
                        }
                    }
                    tile_reduce4(fi, lane);
                    const int t = lane >> 2;
                    if ((lane & 3) == 0 && t < ni) {
                        atomicAdd(facc + k0 + t, make_float4(fi[0], fi[1], fi[2], fi[3]));
                        if (!GHOST) {
                            const float4 x = th[t];
                            vir_add<32>(vl, x.x, x.y, x.z, fi[0], fi[1], fi[2]);
                        }
                    }
                    __syncwarp();
                }
                // 4. survivors' reactions (and the survivor side of the virial, in A's frame)
                for (int j = lane; j < nq; j += 32) {
                    const float4 f = w.sf[j];
                    if (f.x != 0.f || f.y != 0.f || f.z != 0.f || f.w != 0.f) {
                        atomicAdd(facc + __float_as_int(w.sl[j].w), f);
                        if (!GHOST) {
                            const float4 x = w.sh[j];
                            vir_add<32>(vl, x.x, x.y, x.z, f.x, f.y, f.z);
                        }
                    }
                }
                __syncwarp();
                nq = 0;
                own_first = false;
            }
            if (!more) break;
        }
        // FP32 running sums to FP64 once per cluster
        {
            const float su = warp_sum(u_acc);
            u_acc = 0.f;
            float sv[6];
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                sv[i] = warp_sum(GHOST ? vg[i] : vl[32 * i]);
                vg[i] = 0.f;
                if (!GHOST) vl[32 * i] = 0.f;
            }
            if (lane == 0) {
                dsum[0] += (double)su;
                for (int i = 0; i < 6; ++i) dsum[1 + i] += (double)sv[i];
            }
            __syncwarp();
        }
    }
    __syncwarp();
    double fin[7];
#pragma unroll
    for (int i = 0; i < 7; ++i) fin[i] = dsum[i];
    unsigned cv[8] = {0u, 0u, 0u, wc0, wc1, wc2, w.cnt[0], w.cnt[1]};
    if (lane != 0) cv[6] = cv[7] = 0;
    warp_to_stripe(a, blockIdx.x * kCW + wib, fin, cv, lane);
}

// AICA-evaluated pairs of the cell schedule (§2.3's loops count every pair
// of every listed cell pair): a warp per cell, lanes over its runs.
__global__ void __launch_bounds__(256) count_evaluated(const int *cell_off, const int *run_off, const RunEntry *runs,
                                                       int C, double *acc) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    unsigned long long ev[3] = {0, 0, 0};
    for (int I = gw; I < C; I += nw) {
        const long long nI = cell_off[I + 1] - cell_off[I];
        if (nI == 0) continue;
        if (lane == 0) ev[0] += (unsigned long long)(nI * (nI - 1) / 2);
        for (int r = run_off[I] + lane; r < run_off[I + 1]; r += 32) {
            const RunEntry e = runs[r];
            const int len = ((unsigned)e.n >> 24) + 1;
            const long long m = cell_off[e.j + len] - cell_off[e.j];
            ev[(e.n & 0xffffff) != 0 ? 2 : 1] += (unsigned long long)(nI * m);
        }
    }
    double *row = acc + kAccStripes + (size_t)(gw % kStripes) * kParts;
    for (int i = 0; i < 3; ++i) {
        unsigned long long s = ev[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0 && s) atomicAdd(row + 7 + i, (double)s);
    }
}

// grid: enough warps to fill the GPU, at least two cells per warp
int pair_grid(int C) {
    int need = (C + 2 * kWarps - 1) / (2 * kWarps);
    return std::max(1, std::min(need, 152 * 16));
}

aica_status fill_params(aica_mesh *m, const aica_lj *lj, int max_s, PairArgs &a) {
    if (!lj || !lj->eps || !lj->sigma || lj->n_species < 1 || lj->n_species > max_s) {
        set_error("LJ parameters: need 1..%d species with eps and sigma", max_s);
        return AICA_ERR_INVALID_ARG;
    }
    const int S = lj->n_species;
    for (int s = 0; s < S; ++s)
        if (!(lj->eps[s] >= 0) || !(lj->sigma[s] > 0)) {
            set_error("LJ parameters: eps must be >= 0 and sigma > 0");
            return AICA_ERR_INVALID_ARG;
        }
    if (m->max_species >= S) {
        set_error("species index %d >= n_species %d", m->max_species, S);
        return AICA_ERR_INVALID_ARG;
    }
    memset(&a.tab, 0, sizeof(a.tab));
    const double rc2 = m->rc * m->rc;
    for (int i = 0; i < S; ++i)
        for (int j = 0; j < S; ++j) {
            double e = sqrt(lj->eps[i] * lj->eps[j]), sg = 0.5 * (lj->sigma[i] + lj->sigma[j]);
            double s2 = sg * sg, sc = s2 / rc2, sc3 = sc * sc * sc;
            double ush = 4.0 * e * (sc3 * sc3 - sc3);
            a.tab.f[i * kMaxSpecies + j] = make_float4((float)s2, (float)(24.0 * e), (float)(4.0 * e), (float)ush);
            a.tab.d[i * kMaxSpecies + j][0] = s2;
            a.tab.d[i * kMaxSpecies + j][1] = 24.0 * e;
            a.tab.d[i * kMaxSpecies + j][2] = 4.0 * e;
            a.tab.d[i * kMaxSpecies + j][3] = ush;
        }
    a.S = S;
    return AICA_OK;
}

void fill_common(aica_mesh *m, PairArgs &a) {
    a.C = (int)m->n_cells;
    a.cell_off = m->cell_off.as<int>();
    a.work_off = m->work_off.as<int>();
    a.work = m->work.as<WorkEntry>();
    a.orgm = m->orgm.as<int>();
    a.run_off = m->run_off.as<int>();
    a.runs = m->runs.as<RunEntry>();
    a.xf = m->n_xf > 0 ? 1 : 0;
    a.n_xf = m->n_xf;
    a.xft = m->n_xf > 0 ? m->xf_dev.as<XfDev>() : nullptr;
    a.run_d = m->n_xf > 0 ? m->run_d.as<float4>() : nullptr;
    for (int d = 0; d < 3; ++d) {
        double L = m->box.periodic[d] ? m->box.L[d] : 0.0;
        a.Lhi[d] = (float)L;
        a.Llo[d] = (float)(L - (double)a.Lhi[d]);
    }
    a.xloc = m->xloc.as<float4>();
    a.xs64 = m->xs64.as<double>();
    a.sph = m->sph.as<float4>();
    double rc2 = m->rc * m->rc;
    a.rc2_d = rc2;
    a.rc2_lo = (float)(rc2 * (1 - 1e-5));
    a.rc2_hi = (float)(rc2 * (1 + 1e-5));
    {
        const double rp = sqrt(rc2 * (1 + 1e-5)) + 8.0 * ldexp(1.0, -m->qexp);
        a.rc2_pre = (float)(rp * rp);
    }
    for (int d = 0; d < 3; ++d) a.L[d] = m->box.periodic[d] ? m->box.L[d] : 0.0;
    a.facc = m->facc.p;
    a.acc = m->acc.as<double>();
    a.ghosts = m->ghosts ? 1 : 0;
}

aica_status check_flags(aica_mesh *m, cudaStream_t st) {
    unsigned flags = 0;
    AICA_CUDA(cudaMemcpyAsync(&flags, m->flags.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    AICA_CUDA(cudaStreamSynchronize(st));
    if (flags & kFlagSpecies) { set_error("species index out of range"); return AICA_ERR_INVALID_ARG; }
    if (flags & kFlagOutside) { set_error("some molecules lie in no cell"); return AICA_ERR_OUTSIDE_MESH; }
    if (flags & kFlagCapacity) { set_error("a kernel capacity was exceeded"); return AICA_ERR_CAPACITY; }
    return AICA_OK;
}

template <bool XF>
void launch_fwd64(const PairArgs &a, bool multi, bool shift, int grid, cudaStream_t st) {
    if (multi) {
        if (shift) pair_fwd64<true, true, XF><<<grid, kPairThreads, 0, st>>>(a);
        else pair_fwd64<true, false, XF><<<grid, kPairThreads, 0, st>>>(a);
    } else {
        if (shift) pair_fwd64<false, true, XF><<<grid, kPairThreads, 0, st>>>(a);
        else pair_fwd64<false, false, XF><<<grid, kPairThreads, 0, st>>>(a);
    }
}

// Blocks of the persistent FP32 kernel: every SM filled to its occupancy.
template <int NI_, bool MULTI, bool SHIFT, int MINB, bool XF>
int fwd32_grid() {
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    if (!cache[dev]) {
        int sms = 0, per = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, pair_fwd32<NI_, MULTI, SHIFT, MINB, XF>, kThreads32, 0);
        cache[dev] = std::max(1, sms * std::max(1, per));
    }
    return cache[dev];
}

template <int NI_, bool MULTI, bool SHIFT, bool XF>
int launch_fwd32_t(const PairArgs &a, cudaStream_t st) {
    constexpr int MINB = 7;                    // 7 blocks of 4 warps per SM (72 registers)
    const int grid = std::min(fwd32_grid<NI_, MULTI, SHIFT, MINB, XF>(), std::max(1, (a.C + kWarps32 - 1) / kWarps32));
    pair_fwd32<NI_, MULTI, SHIFT, MINB, XF><<<grid, kThreads32, 0, st>>>(a);
    return grid * kWarps32;
}

template <int NI_, bool XF>
int launch_fwd32_x(const PairArgs &a, bool multi, bool shift, cudaStream_t st) {
    if (multi) return shift ? launch_fwd32_t<NI_, true, true, XF>(a, st) : launch_fwd32_t<NI_, true, false, XF>(a, st);
    return shift ? launch_fwd32_t<NI_, false, true, XF>(a, st) : launch_fwd32_t<NI_, false, false, XF>(a, st);
}

// Launch the FP32 kernel; returns the number of warps.
template <int NI_>
int launch_fwd32(const PairArgs &a, bool multi, bool shift, cudaStream_t st) {
    return a.xf ? launch_fwd32_x<NI_, true>(a, multi, shift, st) : launch_fwd32_x<NI_, false>(a, multi, shift, st);
}

// Launch the FP32 adjoint on a persistent grid (every SM filled to its
// occupancy: 7 blocks of 4 warps at 72 registers for chunks of 4, 6 at 80
// for chunks of 8, the most that keep the pair loop free of spills);
// returns the number of blocks.
template <int NI_, bool MULTI, bool XF>
int launch_bwd32_t(const BwdArgs &b, cudaStream_t st) {
    constexpr int MINB = NI_ == 4 ? 7 : 6;
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    if (!cache[dev]) {
        int sms = 0, per = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, pair_bwd32<NI_, MULTI, XF, MINB>, kThreads32, 0);
        cache[dev] = std::max(1, sms * std::max(1, per));
    }
    const int grid = std::min(cache[dev], std::max(1, (b.p.C + kWarps32 - 1) / kWarps32));
    pair_bwd32<NI_, MULTI, XF, MINB><<<grid, kThreads32, 0, st>>>(b);
    return grid;
}

template <int NI_>
int launch_bwd32(const BwdArgs &b, bool multi, cudaStream_t st) {
    if (b.p.xf) return multi ? launch_bwd32_t<NI_, true, true>(b, st) : launch_bwd32_t<NI_, false, true>(b, st);
    return multi ? launch_bwd32_t<NI_, true, false>(b, st) : launch_bwd32_t<NI_, false, false>(b, st);
}

void launch_bwd64(const BwdArgs &b, bool multi, int grid, cudaStream_t st) {
    if (b.p.xf) {
        if (multi) pair_bwd64<true, true><<<grid, kPairThreads, 0, st>>>(b);
        else pair_bwd64<false, true><<<grid, kPairThreads, 0, st>>>(b);
    } else {
        if (multi) pair_bwd64<true, false><<<grid, kPairThreads, 0, st>>>(b);
        else pair_bwd64<false, false><<<grid, kPairThreads, 0, st>>>(b);
    }
}

// The FP32 cluster kernel: a persistent grid, every SM filled to its
// occupancy (dynamic shared memory: the warps' survivor buffers and queues).
template <bool MULTI, bool SHIFT, bool GHOST>
void launch_fwd32c_t(const PairArgs &a, const ClKArgs &c, cudaStream_t st) {
    constexpr int MINB = 5;
    static int cache[64] = {0};
    const size_t shm = sizeof(WarpC) * kCW;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    if (!cache[dev]) {
        cudaFuncSetAttribute(pair_fwd32c<MULTI, SHIFT, GHOST, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
        int sms = 0, per = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, pair_fwd32c<MULTI, SHIFT, GHOST, MINB>, kCT, shm);
        cache[dev] = std::max(1, sms * std::max(1, per));
    }
    const int grid = std::min(cache[dev], std::max(1, (c.ncl + kCW - 1) / kCW));
    pair_fwd32c<MULTI, SHIFT, GHOST, MINB><<<grid, kCT, shm, st>>>(a, c);
}

template <bool GHOST>
void launch_fwd32c_g(const PairArgs &a, const ClKArgs &c, bool multi, bool shift, cudaStream_t st) {
    if (multi) shift ? launch_fwd32c_t<true, true, GHOST>(a, c, st) : launch_fwd32c_t<true, false, GHOST>(a, c, st);
    else shift ? launch_fwd32c_t<false, true, GHOST>(a, c, st) : launch_fwd32c_t<false, false, GHOST>(a, c, st);
}

void launch_fwd32c(const PairArgs &a, const ClKArgs &c, bool multi, bool shift, cudaStream_t st) {
    if (a.ghosts) launch_fwd32c_g<true>(a, c, multi, shift, st);
    else launch_fwd32c_g<false>(a, c, multi, shift, st);
}

}  // namespace
}  // namespace aica

using namespace aica;

extern "C" aica_status aica_forces(aica_mesh *m, const aica_lj *lj, aica_precision prec, void *force_out,
                                   double *ev_out, int64_t *counts_out, void *stream) {
    AICA_RANGE("aica_forces");
    if (!m || (!force_out && m->n_mol > 0)) { set_error("aica_forces: NULL argument"); return AICA_ERR_INVALID_ARG; }
    if (prec != AICA_FP32 && prec != AICA_FP64) { set_error("aica_forces: bad precision"); return AICA_ERR_INVALID_ARG; }
    if (!m->built || !m->binned) { set_error("aica_forces: build the lists and bin the molecules first"); return AICA_ERR_NOT_BUILT; }
    cudaStream_t st = (cudaStream_t)stream;
    PairArgs a{};
    aica_status s = fill_params(m, lj, kMaxSpecies, a);
    if (s != AICA_OK) return s;
    const int grid = pair_grid((int)m->n_cells);
    fill_common(m, a);
    a.next_cell = (unsigned *)(m->acc.as<double>() + 24);
    m->launches = 0;
    const int64_t n = m->n_mol;
    const bool f64 = prec == AICA_FP64;
    if (n > 0) AICA_CUDA(cudaMemsetAsync(m->facc.p, 0, (f64 ? 4 * sizeof(double) : sizeof(float4)) * n, st));
    AICA_CUDA(cudaMemsetAsync(m->acc.p, 0, (kAccStripes + kStripes * kParts) * sizeof(double), st));
    const bool multi = a.S > 1, shift = lj->shift != 0;
    cudaEvent_t tstop;
    AICA_CUDA(timing_begin(m, st, &tstop));
    // FP32 with box periodicity: the cluster kernel when the lists have a
    // cluster schedule (the cell kernel on request, and for general transforms)
    const bool clsched = !f64 && !a.xf && m->n_cl_runs >= 0;
    const bool clpath = clsched && m->fp32_kernel != 1;
    if (m->ghosts && !f64 && !clpath) {
        set_error("aica_forces: portion mode (halo molecules) needs the FP32 cluster kernel");
        return AICA_ERR_INVALID_ARG;
    }
    if (m->ghosts && a.xf) {
        set_error("aica_forces: portion mode (halo molecules) needs box periodicity");
        return AICA_ERR_INVALID_ARG;
    }
    if (!f64) {
        if (clpath) {
            ClKArgs c{};
            c.cl_first = m->cl_first.as<int>();
            c.cl_run_off = m->cl_run_off.as<int>();
            c.runs = m->cl_runs.as<ClRun>();
            c.xlo = m->xlo.as<float4>();
            c.cl_box = m->cl_box.as<float4>();
            c.ncl = (int)m->n_cl;
            c.qround = (float)ldexp(1.5, 23 - m->qexp);
            launch_fwd32c(a, c, multi, shift, st);
        } else {
            // i-chunk width: 4 for cells of a few molecules (tetrahedra), 8 otherwise
            if ((double)n < 5.0 * (double)a.C) launch_fwd32<4>(a, multi, shift, st);
            else launch_fwd32<8>(a, multi, shift, st);
        }
    } else {
        if (a.xf) launch_fwd64<true>(a, multi, shift, grid, st);
        else launch_fwd64<false>(a, multi, shift, grid, st);
    }
    AICA_CUDA(timing_end(tstop, st));
    m->launches = 2;
    double *acc = m->acc.as<double>();
    if (clpath && counts_out && m->count_evaluated && a.C > 0) {
        // the cluster kernel does not walk the cell schedule: count the method's evaluated pairs
        count_evaluated<<<(unsigned)std::min<int64_t>(((int64_t)a.C * 32 + 255) / 256, 152 * 16), 256, 0, st>>>(
            a.cell_off, a.run_off, a.runs, a.C, acc);
        m->launches += 1;
    }
    // FP32 cluster path: molecules whose FP32 force cannot
    // be certified to the tolerance are recomputed in double-single arithmetic
    // (needs the cluster lists)
    const bool refine = clpath && m->refine_tol > 0 && n > 0;
    int *flags = refine ? m->flag_list.as<int>() : nullptr;
    if (refine) AICA_CUDA(cudaMemsetAsync(flags, 0, sizeof(int), st));
    const float kf = refine ? (float)(kRefineScale / m->refine_tol) : 0.f;
    if (n > 0) {
        const unsigned g = (unsigned)((n + 255) / 256);
        if (f64) unsort_forces<double><<<g, 256, 0, st>>>(m->inv.as<int>(), n, m->facc.p, (double *)force_out, 1, acc, ev_out, (long long *)counts_out);
        else unsort_forces<float><<<g, 256, 0, st>>>(m->inv.as<int>(), n, m->facc.p, (float *)force_out, 0, acc, ev_out, (long long *)counts_out);
        if (refine) {
            flag_ill_conditioned<<<g, 256, 0, st>>>((const float4 *)m->facc.p, m->xloc.as<float4>(), (int)n, kf * kf,
                                                    flags);
            m->launches += 1;
        }
    } else {
        finish_sums<<<1, 15 * 32, 0, st>>>(acc, ev_out, (long long *)counts_out);
    }
    if (refine) {
        RefineArgs r{};
        r.flag_list = flags;
        r.cl_first = m->cl_first.as<int>();
        r.cl_of = m->cl_of.as<int>();
        r.full_off = m->cl_full_off.as<int>();
        r.full = m->cl_full.as<unsigned long long>();
        r.order = m->order.as<int>();
        r.xlo = m->xlo.as<float4>();
        r.cl_box = m->cl_box.as<float4>();
        r.out = (float *)force_out;
        r.C = a.C;
        r.orgm = m->orgm.as<int>();
        for (int d = 0; d < 3; ++d) {
            const double L = m->box.periodic[d] ? m->box.L[d] : 0.0;
            // nearest FP32 of L on the 2^-q grid (a multiple of 2^-q whether or not
            // the grid value itself fits 24 bits), remainder against that FP32 value
            r.Lh[d] = (float)(rint(ldexp(L, m->qexp)) * ldexp(1.0, -m->qexp));
            r.Ll[d] = (float)(L - (double)r.Lh[d]);
        }
        r.qround = (float)ldexp(1.5, 23 - m->qexp);
        for (int i = 0; i < kMaxSpecies * kMaxSpecies; ++i) {
            const double *t = a.tab.d[i];
            const float sh = (float)t[0], ch = (float)t[1];
            r.sig2[i][0] = sh;
            r.sig2[i][1] = (float)(t[0] - (double)sh);
            r.c24[i][0] = ch;
            r.c24[i][1] = (float)(t[1] - (double)ch);
        }
        r.rc2h = (float)a.rc2_d;
        r.rc2l = (float)(a.rc2_d - (double)r.rc2h);
        r.next = (unsigned *)(m->acc.as<double>() + 25);      // zeroed with the sums at the call's start
        refine_ds<<<152 * 8, 256, 0, st>>>(a, r);
        m->launches += 1;
    }
    AICA_CUDA(cudaGetLastError());
    if (!m->deferred) return check_flags(m, st);
    return AICA_OK;
}

extern "C" aica_status aica_forces_backward(aica_mesh *m, const aica_lj *lj, aica_precision prec,
                                            const void *grad_force, void *grad_pos, double *grad_eps,
                                            double *grad_sigma, void *stream) {
    AICA_RANGE("aica_forces_backward");
    if (!m || ((!grad_force || !grad_pos) && m->n_mol > 0)) {
        set_error("aica_forces_backward: NULL argument");
        return AICA_ERR_INVALID_ARG;
    }
    if (prec != AICA_FP32 && prec != AICA_FP64) { set_error("aica_forces_backward: bad precision"); return AICA_ERR_INVALID_ARG; }
    if (!m->built || !m->binned) { set_error("aica_forces_backward: build the lists and bin the molecules first"); return AICA_ERR_NOT_BUILT; }
    if (m->ghosts) { set_error("aica_forces_backward: not available in portion mode (halo molecules)"); return AICA_ERR_INVALID_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    BwdArgs b{};
    aica_status s = fill_params(m, lj, kMaxSpecies, b.p);
    if (s != AICA_OK) return s;
    fill_common(m, b.p);
    b.S = b.p.S;
    for (int i = 0; i < b.S; ++i)
        for (int j = 0; j < b.S; ++j) {
            BwdTab &t = b.t[i * kMaxSpecies + j];
            double e = sqrt(lj->eps[i] * lj->eps[j]), sg = 0.5 * (lj->sigma[i] + lj->sigma[j]);
            t.eps = e;
            t.sig2 = sg * sg;
            t.inv_eps = e > 0 ? 1.0 / e : 0.0;
            t.inv_sig = 1.0 / sg;
            // d eps_ab / d eps_a = eps_ab / (2 eps_a)  (both halves when a == b)
            t.fa = lj->eps[i] > 0 ? e / (2.0 * lj->eps[i]) : 0.0;
            t.fb = lj->eps[j] > 0 ? e / (2.0 * lj->eps[j]) : 0.0;
            b.tb[i * kMaxSpecies + j] = make_float4((float)(t.fa * t.inv_eps), (float)(t.fb * t.inv_eps),
                                                    (float)(0.5 * t.inv_sig), 0.f);
        }
    b.e1 = lj->eps[0] > 0 ? 1.0 / lj->eps[0] : 0.0;
    b.s1 = 1.0 / lj->sigma[0];
    b.p.next_cell = (unsigned *)(m->acc.as<double>() + 24);
    m->launches = 0;
    const int64_t n = m->n_mol;
    const bool f64 = prec == AICA_FP64, multi = b.S > 1;
    const size_t esz = f64 ? 4 * sizeof(double) : sizeof(float4);
    int nb = 0;
    AICA_CUDA(cudaMemcpyAsync(&nb, m->cell_off.as<int>() + m->n_cells, sizeof(int), cudaMemcpyDeviceToHost, st));
    AICA_CUDA(cudaStreamSynchronize(st));
    int launches = 0;
    if (n > 0) {
        AICA_CUDA(cudaMemsetAsync(m->facc.p, 0, esz * n, st));
        if (nb > 0) {
            if (f64) gather_grad<double><<<(nb + 255) / 256, 256, 0, st>>>(m->order.as<int>(), nb, (const double *)grad_force, m->vsorted.p, 1);
            else gather_grad<float><<<(nb + 255) / 256, 256, 0, st>>>(m->order.as<int>(), nb, (const float *)grad_force, m->vsorted.p, 0);
            launches++;
        }
    }
    AICA_CUDA(cudaMemsetAsync(m->acc.p, 0, (kAccStripes + kStripes * kParts) * sizeof(double), st));
    b.p.vs = m->vsorted.p;
    cudaEvent_t tstop;
    AICA_CUDA(timing_begin(m, st, &tstop));
    if (f64) {
        launch_bwd64(b, multi, pair_grid(b.p.C), st);
    } else {
        if ((double)n < 5.0 * (double)b.p.C) launch_bwd32<4>(b, multi, st);
        else launch_bwd32<8>(b, multi, st);
    }
    AICA_CUDA(timing_end(tstop, st));
    launches++;
    if (n > 0) {
        if (f64) unsort_forces<double><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(m->inv.as<int>(), n, m->facc.p, (double *)grad_pos, 1);
        else unsort_forces<float><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(m->inv.as<int>(), n, m->facc.p, (float *)grad_pos, 0);
        launches++;
    }
    if (grad_eps || grad_sigma) {
        finish_bwd<<<1, kGradSlots * 32, 0, st>>>(m->acc.as<double>(), b.S, grad_eps, grad_sigma);
        launches++;
    }
    m->launches = launches;
    AICA_CUDA(cudaGetLastError());
    if (!m->deferred) return check_flags(m, st);
    return AICA_OK;
}
