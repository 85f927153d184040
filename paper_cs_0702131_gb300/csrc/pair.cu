// Pair-force kernels (steps a5-a10): the force loops of §2.3 on the binned
// molecules and the per-cell pair schedule built with the lists.
//
// Schedule.  For real cell I the schedule holds its DIL cells (pairs with
// Newton's third law, §2.3 "real-real") and, after work_split[I], every
// referred cell (c, n) whose real-cell list contains I: those pairs act on
// I's molecules only (§2.3 "real-referred"; the source molecules get their
// share from the mirror referred cell).  Same-cell pairs (sorted index
// k' > k) are walked first.  A referred molecule is never copied: it is the
// source molecule read through the cell-pair shift Delta = o_J + n.L - o_I
// (step a5).
//
// Layout.  One warp walks one cell I at a time (cells interleaved over all
// warps of the grid).  Up to NI molecules of I sit in registers; the lanes
// stream the concatenated molecules of the partner cells, 32 at a time (a
// load-balanced expansion of the partner list: warp scan of partner sizes,
// then a 5-step binary search per lane).  Each lane evaluates its partner
// molecule against the NI molecules of I; reactions on the partner molecule
// are summed in registers and added once per (partner molecule, I-chunk)
// with a vector atomic; forces on I's molecules are reduced over the warp.
//
// Precision (FP32 path).  Coordinates are cell-local (dyadic cell origins,
// so o_J - o_I is exact in FP32).  Pairs whose FP32 r^2 falls within 1e-5
// rc^2 of the cut-off are re-decided in FP64 exactly as the all-pairs
// definition computes r^2, so the evaluated-within-rc pair set is the same as
// in FP64.  Energy and virial are summed per cell in FP32, carried across
// cells with compensated (Kahan) summation and reduced in FP64.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "aica_internal.cuh"

namespace aica {
namespace {

constexpr int kPairThreads = 256;
constexpr int NI = 8;

struct SpeciesTab {
    float4 f[kMaxSpecies * kMaxSpecies];    // sig2, 24 eps, 4 eps, u(rc) for FP32
    double d[kMaxSpecies * kMaxSpecies][4]; // same in FP64
};

struct PairArgs {
    int C;
    const int *cell_off, *work_off, *work_split;
    const WorkEntry *work;
    const float4 *work_d32;
    const float4 *xloc;
    const double *xs64;
    float rc2_f, rc2_lo, rc2_hi;
    double rc2_d;
    double L[3];
    int S;
    void *facc;                  // float4 (FP32) or double4 (FP64), binned order
    const void *vs;              // backward: grad_force in binned order (float4 / double4)
    double *acc;                 // [0..6] U, W; [8..13] counters (as unsigned long long); [16..] grads
    SpeciesTab tab;
};

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

template <class R> struct R3 { R x, y, z; };

template <class R> struct CellAcc {
    R u, w[6];
    __device__ void zero() { u = 0; for (int i = 0; i < 6; ++i) w[i] = 0; }
    __device__ void scale(R s) { u *= s; for (int i = 0; i < 6; ++i) w[i] *= s; }
};

// compensated running sum
struct Kahan {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        float y = v - c;
        float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

struct Counters {
    unsigned long long eval[3] = {0, 0, 0};
    unsigned within[3] = {0, 0, 0};
};

// FP64 re-decision of r^2 < rc^2 with the all-pairs definition's operation order
__device__ __noinline__ bool band_in(const PairArgs &a, int k, int l, int np) {
    const double *xk = a.xs64 + 3 * (size_t)k, *xl = a.xs64 + 3 * (size_t)l;
    double dx = __dsub_rn(__dsub_rn(xk[0], xl[0]), __dmul_rn(a.L[0], (double)unpack_n(np, 0)));
    double dy = __dsub_rn(__dsub_rn(xk[1], xl[1]), __dmul_rn(a.L[1], (double)unpack_n(np, 1)));
    double dz = __dsub_rn(__dsub_rn(xk[2], xl[2]), __dmul_rn(a.L[2], (double)unpack_n(np, 2)));
    double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    return r2 < a.rc2_d;
}

// ---------------------------------------------------------------- FP32 pair
template <bool MULTI, bool SHIFT>
__device__ __forceinline__ void pair32(const PairArgs &a, const float4 *tab, float rx, float ry, float rz, float r2,
                                       int spi, int spj, R3<float> &fi, R3<float> &fj, CellAcc<float> &acc,
                                       bool newton) {
    float sig2, c24, c4, ush;
    if (MULTI) {
        float4 t = tab[spi * kMaxSpecies + spj];
        sig2 = t.x; c24 = t.y; c4 = t.z; ush = t.w;
    } else {
        float4 t = tab[0];
        sig2 = t.x; c24 = t.y; c4 = t.z; ush = t.w;
    }
    float inv = rcp_approx(r2);
    float s = sig2 * inv;
    float s3 = s * s * s;
    float fs = (c24 * inv) * s3 * fmaf(2.f, s3, -1.f);
    float fx = fs * rx, fy = fs * ry, fz = fs * rz;
    fi.x += fx; fi.y += fy; fi.z += fz;
    if (newton) { fj.x -= fx; fj.y -= fy; fj.z -= fz; }
    float u = c4 * s3 * (s3 - 1.f);
    if (SHIFT) u -= ush;
    acc.u += u;
    acc.w[0] = fmaf(rx, fx, acc.w[0]);
    acc.w[1] = fmaf(ry, fy, acc.w[1]);
    acc.w[2] = fmaf(rz, fz, acc.w[2]);
    acc.w[3] = fmaf(rx, fy, acc.w[3]);
    acc.w[4] = fmaf(rx, fz, acc.w[4]);
    acc.w[5] = fmaf(ry, fz, acc.w[5]);
}

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

// Stream the partner molecules of entries [e0, e1) against the NI-chunk of I.
template <bool NEWTON, bool MULTI, bool SHIFT>
__device__ __forceinline__ void stream32(const PairArgs &a, const float4 *tab, int e0, int e1, int kbase, int ni,
                                         const float4 (&xi)[NI], R3<float> (&fi)[NI], CellAcc<float> &acc,
                                         Counters &cnt, int lane) {
    float4 *facc = (float4 *)a.facc;
    const int cat = NEWTON ? 1 : 2;
    for (int eb = e0; eb < e1; eb += 32) {
        int e = eb + lane;
        int js = 0, n = 0, np = 0;
        float4 d = make_float4(0.f, 0.f, 0.f, 0.f);
        if (e < e1) {
            WorkEntry we = a.work[e];
            js = a.cell_off[we.j];
            n = a.cell_off[we.j + 1] - js;
            np = we.n;
            d = a.work_d32[e];
        }
        cnt.eval[cat] += (unsigned long long)(n * ni);
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
            bool valid = p < total;
            int l = jsl + (p - exl);
            float4 xl = valid ? a.xloc[l] : make_float4(1e18f, 1e18f, 1e18f, 0.f);
            float xjx = xl.x + dx, xjy = xl.y + dy, xjz = xl.z + dz;
            int spj = __float_as_int(xl.w);
            R3<float> fj = {0.f, 0.f, 0.f};
#pragma unroll
            for (int t = 0; t < NI; ++t) {
                if (t < ni) {
                    float rx = xi[t].x - xjx, ry = xi[t].y - xjy, rz = xi[t].z - xjz;
                    float r2 = fmaf(rz, rz, fmaf(ry, ry, rx * rx));
                    if (r2 < a.rc2_hi) {
                        bool in = r2 < a.rc2_lo || band_in(a, kbase + t, l, npl);
                        if (in) {
                            pair32<MULTI, SHIFT>(a, tab, rx, ry, rz, r2, __float_as_int(xi[t].w), spj, fi[t], fj, acc,
                                                 NEWTON);
                            cnt.within[cat]++;
                        }
                    }
                }
            }
            if (NEWTON && valid && (fj.x != 0.f || fj.y != 0.f || fj.z != 0.f))
                atomicAdd(facc + l, make_float4(fj.x, fj.y, fj.z, 0.f));
        }
    }
}

template <bool MULTI, bool SHIFT>
__global__ void __launch_bounds__(kPairThreads) pair_fwd32(PairArgs a) {
    __shared__ float4 tab[kMaxSpecies * kMaxSpecies];
    __shared__ double red[kPairThreads / 32][16];
    for (int i = threadIdx.x; i < kMaxSpecies * kMaxSpecies; i += blockDim.x) tab[i] = a.tab.f[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nwarps = gridDim.x * (kPairThreads / 32);
    float4 *facc = (float4 *)a.facc;
    Kahan tot[7];
    Counters cnt;
    for (int I = blockIdx.x * (kPairThreads / 32) + wib; I < a.C; I += nwarps) {
        const int sI = a.cell_off[I], nI = a.cell_off[I + 1] - sI;
        if (nI == 0) continue;
        const int e0 = a.work_off[I], es = a.work_split[I], e1 = a.work_off[I + 1];
        CellAcc<float> acc;
        acc.zero();
        for (int pass = 0; pass < 2; ++pass) {       // 0: real-referred (one-sided), 1: same-cell + DIL
            if (pass == 0 && es == e1) continue;
            for (int i0 = 0; i0 < nI; i0 += NI) {
                const int ni = min(NI, nI - i0);
                float4 xi[NI];
                R3<float> fi[NI];
#pragma unroll
                for (int t = 0; t < NI; ++t) {
                    xi[t] = t < ni ? a.xloc[sI + i0 + t] : make_float4(0.f, 0.f, 0.f, 0.f);
                    fi[t] = {0.f, 0.f, 0.f};
                }
                if (pass == 0) {
                    stream32<false, MULTI, SHIFT>(a, tab, es, e1, sI + i0, ni, xi, fi, acc, cnt, lane);
                } else {
                    // same-cell pairs k' > k (sorted order), Newton's third law
                    for (int lb = i0 + 1; lb < nI; lb += 32) {
                        int li = lb + lane;
                        bool valid = li < nI;
                        int l = sI + li;
                        float4 xl = valid ? a.xloc[l] : make_float4(1e18f, 1e18f, 1e18f, 0.f);
                        R3<float> fj = {0.f, 0.f, 0.f};
#pragma unroll
                        for (int t = 0; t < NI; ++t) {
                            if (t < ni && li > i0 + t) {
                                float rx = xi[t].x - xl.x, ry = xi[t].y - xl.y, rz = xi[t].z - xl.z;
                                float r2 = fmaf(rz, rz, fmaf(ry, ry, rx * rx));
                                if (r2 < a.rc2_hi && (r2 < a.rc2_lo || band_in(a, sI + i0 + t, l, 0))) {
                                    pair32<MULTI, SHIFT>(a, tab, rx, ry, rz, r2, __float_as_int(xi[t].w),
                                                         __float_as_int(xl.w), fi[t], fj, acc, true);
                                    cnt.within[0]++;
                                }
                            }
                        }
                        if (valid && (fj.x != 0.f || fj.y != 0.f || fj.z != 0.f))
                            atomicAdd(facc + l, make_float4(fj.x, fj.y, fj.z, 0.f));
                    }
                    stream32<true, MULTI, SHIFT>(a, tab, e0, es, sI + i0, ni, xi, fi, acc, cnt, lane);
                }
                // forces on I's molecules: warp sums, one vector atomic each
#pragma unroll
                for (int t = 0; t < NI; ++t) {
                    if (t < ni) {
                        float x = warp_sum(fi[t].x), y = warp_sum(fi[t].y), z = warp_sum(fi[t].z);
                        if (lane == t) atomicAdd(facc + sI + i0 + t, make_float4(x, y, z, 0.f));
                    }
                }
            }
            if (pass == 0) acc.scale(0.5f);   // each referred pair is evaluated from both sides
        }
        if (lane == 0) cnt.eval[0] += (unsigned long long)nI * (nI - 1) / 2;
        tot[0].add(acc.u);
#pragma unroll
        for (int i = 0; i < 6; ++i) tot[i + 1].add(acc.w[i]);
    }
    // block reduction, then one FP64 / 64-bit atomic per value
    double v[13];
    for (int i = 0; i < 7; ++i) v[i] = warp_sum((double)tot[i].s - (double)tot[i].c);
    for (int i = 0; i < 3; ++i) v[7 + i] = warp_sum((double)cnt.eval[i]);
    for (int i = 0; i < 3; ++i) v[10 + i] = warp_sum((double)cnt.within[i]);
    if (lane == 0)
        for (int i = 0; i < 13; ++i) red[wib][i] = v[i];
    __syncthreads();
    if (threadIdx.x < 13) {
        double s = 0;
        for (int w = 0; w < kPairThreads / 32; ++w) s += red[w][threadIdx.x];
        if (threadIdx.x < 7) atomicAdd(a.acc + threadIdx.x, s);
        else atomicAdd((unsigned long long *)(a.acc + 8) + (threadIdx.x - 7), (unsigned long long)llrint(s));
    }
}

// ---------------------------------------------------------------- FP64 pair
template <bool MULTI, bool SHIFT>
__device__ __forceinline__ void pair64(const double (*tab)[4], double rx, double ry, double rz, double r2, int spi,
                                       int spj, R3<double> &fi, R3<double> &fj, CellAcc<double> &acc, bool newton) {
    const double *t = MULTI ? tab[spi * kMaxSpecies + spj] : tab[0];
    double inv = 1.0 / r2;
    double s = t[0] * inv;
    double s3 = s * s * s;
    double fs = t[1] * inv * s3 * (2.0 * s3 - 1.0);
    double fx = fs * rx, fy = fs * ry, fz = fs * rz;
    fi.x += fx; fi.y += fy; fi.z += fz;
    if (newton) { fj.x -= fx; fj.y -= fy; fj.z -= fz; }
    double u = t[2] * s3 * (s3 - 1.0);
    if (SHIFT) u -= t[3];
    acc.u += u;
    acc.w[0] += rx * fx; acc.w[1] += ry * fy; acc.w[2] += rz * fz;
    acc.w[3] += rx * fy; acc.w[4] += rx * fz; acc.w[5] += ry * fz;
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

template <bool NEWTON, bool MULTI, bool SHIFT>
__device__ __forceinline__ void stream64(const PairArgs &a, const double (*tab)[4], int e0, int e1, int ni,
                                         const double (&xi)[NI][3], const int (&spi)[NI], R3<double> (&fi)[NI],
                                         CellAcc<double> &acc, Counters &cnt, int lane) {
    double *facc = (double *)a.facc;
    const int cat = NEWTON ? 1 : 2;
    for (int eb = e0; eb < e1; eb += 32) {
        int e = eb + lane;
        int js = 0, n = 0, np = 0;
        if (e < e1) {
            WorkEntry we = a.work[e];
            js = a.cell_off[we.j];
            n = a.cell_off[we.j + 1] - js;
            np = we.n;
        }
        cnt.eval[cat] += (unsigned long long)(n * ni);
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
            int npl = __shfl_sync(0xffffffffu, np, o);
            if (p >= total) continue;
            int l = jsl + (p - exl);
            const double *xl = a.xs64 + 3 * (size_t)l;
            int spj = __float_as_int(a.xloc[l].w);
            R3<double> fj = {0, 0, 0};
            bool any = false;
#pragma unroll
            for (int t = 0; t < NI; ++t) {
                if (t < ni) {
                    double rx, ry, rz, r2;
                    sep64(xi[t], xl, a.L, npl, rx, ry, rz, r2);
                    if (r2 < a.rc2_d) {
                        pair64<MULTI, SHIFT>(tab, rx, ry, rz, r2, spi[t], spj, fi[t], fj, acc, NEWTON);
                        cnt.within[cat]++;
                        any = true;
                    }
                }
            }
            if (NEWTON && any) atomic_add3(facc + 4 * (size_t)l, fj.x, fj.y, fj.z);
        }
    }
}

template <bool MULTI, bool SHIFT>
__global__ void __launch_bounds__(kPairThreads) pair_fwd64(PairArgs a) {
    __shared__ double tab[kMaxSpecies * kMaxSpecies][4];
    __shared__ double red[kPairThreads / 32][16];
    for (int i = threadIdx.x; i < kMaxSpecies * kMaxSpecies; i += blockDim.x)
        for (int c = 0; c < 4; ++c) tab[i][c] = a.tab.d[i][c];
    __syncthreads();
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nwarps = gridDim.x * (kPairThreads / 32);
    double *facc = (double *)a.facc;
    CellAcc<double> tot;
    tot.zero();
    Counters cnt;
    for (int I = blockIdx.x * (kPairThreads / 32) + wib; I < a.C; I += nwarps) {
        const int sI = a.cell_off[I], nI = a.cell_off[I + 1] - sI;
        if (nI == 0) continue;
        const int e0 = a.work_off[I], es = a.work_split[I], e1 = a.work_off[I + 1];
        CellAcc<double> acc;
        acc.zero();
        for (int pass = 0; pass < 2; ++pass) {
            if (pass == 0 && es == e1) continue;
            for (int i0 = 0; i0 < nI; i0 += NI) {
                const int ni = min(NI, nI - i0);
                double xi[NI][3];
                int spi[NI];
                R3<double> fi[NI];
#pragma unroll
                for (int t = 0; t < NI; ++t) {
                    int k = sI + i0 + min(t, ni - 1);
                    for (int c = 0; c < 3; ++c) xi[t][c] = a.xs64[3 * (size_t)k + c];
                    spi[t] = __float_as_int(a.xloc[k].w);
                    fi[t] = {0, 0, 0};
                }
                if (pass == 0) {
                    stream64<false, MULTI, SHIFT>(a, tab, es, e1, ni, xi, spi, fi, acc, cnt, lane);
                } else {
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
                                    if (r2 < a.rc2_d) {
                                        pair64<MULTI, SHIFT>(tab, rx, ry, rz, r2, spi[t], spj, fi[t], fj, acc, true);
                                        cnt.within[0]++;
                                        any = true;
                                    }
                                }
                            }
                            if (any) atomic_add3(facc + 4 * (size_t)l, fj.x, fj.y, fj.z);
                        }
                    }
                    stream64<true, MULTI, SHIFT>(a, tab, e0, es, ni, xi, spi, fi, acc, cnt, lane);
                }
#pragma unroll
                for (int t = 0; t < NI; ++t) {
                    if (t < ni) {
                        double x = warp_sum(fi[t].x), y = warp_sum(fi[t].y), z = warp_sum(fi[t].z);
                        if (lane == t) atomic_add3(facc + 4 * (size_t)(sI + i0 + t), x, y, z);
                    }
                }
            }
            if (pass == 0) acc.scale(0.5);
        }
        if (lane == 0) cnt.eval[0] += (unsigned long long)nI * (nI - 1) / 2;
        tot.u += acc.u;
        for (int i = 0; i < 6; ++i) tot.w[i] += acc.w[i];
    }
    double v[13];
    v[0] = warp_sum(tot.u);
    for (int i = 0; i < 6; ++i) v[1 + i] = warp_sum(tot.w[i]);
    for (int i = 0; i < 3; ++i) v[7 + i] = warp_sum((double)cnt.eval[i]);
    for (int i = 0; i < 3; ++i) v[10 + i] = warp_sum((double)cnt.within[i]);
    if (lane == 0)
        for (int i = 0; i < 13; ++i) red[wib][i] = v[i];
    __syncthreads();
    if (threadIdx.x < 13) {
        double s = 0;
        for (int w = 0; w < kPairThreads / 32; ++w) s += red[w][threadIdx.x];
        if (threadIdx.x < 7) atomicAdd(a.acc + threadIdx.x, s);
        else atomicAdd((unsigned long long *)(a.acc + 8) + (threadIdx.x - 7), (unsigned long long)llrint(s));
    }
}

// ---------------------------------------------------------------- unsort
template <class T>
__global__ void __launch_bounds__(256) unsort_forces(const int *inv, int64_t n, const void *facc, T *out, int f64) {
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
        }
    }
    out[3 * k] = (T)x;
    out[3 * k + 1] = (T)y;
    out[3 * k + 2] = (T)z;
}

__global__ void finish_sums(const double *acc, double *ev, long long *counts) {
    int i = threadIdx.x;
    if (ev && i < 7) ev[i] = acc[i];
    if (counts && i < 6) counts[i] = (long long)((const unsigned long long *)(acc + 8))[i];
}

// ---------------------------------------------------------------- adjoint
// Per pair with r = x_k - x_l', f = g(r^2) r, g = 24 e inv s3 (2 s3 - 1):
//   J = df/dr = g I + 2 g' r r^T,  g' = dg/d(r^2) = 24 e inv^2 (4 s3 - 14 s6)
//   with w = v_k - v_l (Newton pairs) or w = v_k (one-sided): dL/dr = J w,
//   x_k gets +J w, the partner (for referred pairs its source molecule) -J w;
//   dL/d eps_ab = g (r.w) / eps_ab,  dL/d sigma_ab = 24 e inv (24 s6 - 6 s3) (r.w) / sigma_ab.
struct BwdTab {
    double eps, sig2, inv_eps, inv_sig, fa, fb;   // fa, fb: d eps_ab / d eps_a, d eps_ab / d eps_b
};

struct BwdArgs {
    PairArgs p;
    BwdTab t[kMaxSpeciesBwd * kMaxSpeciesBwd];
    int S;
};

template <class R> struct BwdLane {
    R ge[kMaxSpeciesBwd], gs[kMaxSpeciesBwd];
};

template <class R>
__device__ __forceinline__ void bwd_pair(const BwdTab *tab, int S, R rx, R ry, R rz, R r2, int spi, int spj, R wx,
                                         R wy, R wz, R3<R> &gi, R3<R> &gj, BwdLane<R> &gl) {
    spi &= kMaxSpeciesBwd - 1;
    spj &= kMaxSpeciesBwd - 1;
    const BwdTab &t = tab[spi * kMaxSpeciesBwd + spj];
    R eps = (R)t.eps;
    R inv = R(1) / r2;
    R s = (R)t.sig2 * inv;
    R s3 = s * s * s, s6 = s3 * s3;
    R g = R(24) * eps * inv * s3 * (R(2) * s3 - R(1));
    R gp = R(24) * eps * inv * inv * (R(4) * s3 - R(14) * s6);
    R rw = rx * wx + ry * wy + rz * wz;
    R c = R(2) * gp * rw;
    R jx = g * wx + c * rx, jy = g * wy + c * ry, jz = g * wz + c * rz;
    gi.x += jx; gi.y += jy; gi.z += jz;
    gj.x -= jx; gj.y -= jy; gj.z -= jz;
    R Ge = g * rw * (R)t.inv_eps;
    R Gs = R(24) * eps * inv * (R(24) * s6 - R(6) * s3) * rw * (R)t.inv_sig;
#pragma unroll
    for (int q = 0; q < kMaxSpeciesBwd; ++q) {
        if (q < S) {
            gl.ge[q] += (spi == q ? Ge * (R)t.fa : R(0)) + (spj == q ? Ge * (R)t.fb : R(0));
            gl.gs[q] += (spi == q ? R(0.5) * Gs : R(0)) + (spj == q ? R(0.5) * Gs : R(0));
        }
    }
}

template <class R> struct Pos;
template <> struct Pos<float> {
    // positions of k (I frame) and partner l (its frame + Delta)
    __device__ static void sep(const PairArgs &a, const float4 &xk, int l, float4 d, int np, int kidx, float &rx,
                               float &ry, float &rz, float &r2, bool &in) {
        float4 xl = a.xloc[l];
        rx = xk.x - (xl.x + d.x);
        ry = xk.y - (xl.y + d.y);
        rz = xk.z - (xl.z + d.z);
        r2 = fmaf(rz, rz, fmaf(ry, ry, rx * rx));
        in = r2 < a.rc2_hi && (r2 < a.rc2_lo || band_in(a, kidx, l, np));
    }
};
template <> struct Pos<double> {
    __device__ static void sep(const PairArgs &a, const float4 &, int l, float4, int np, int kidx, double &rx,
                               double &ry, double &rz, double &r2, bool &in) {
        sep64(a.xs64 + 3 * (size_t)kidx, a.xs64 + 3 * (size_t)l, a.L, np, rx, ry, rz, r2);
        in = r2 < a.rc2_d;
    }
};

template <class R>
__device__ __forceinline__ void ldv(const void *vs, int s, R &x, R &y, R &z) {
    if (sizeof(R) == 4) {
        float4 v = ((const float4 *)vs)[s];
        x = (R)v.x; y = (R)v.y; z = (R)v.z;
    } else {
        const double *v = (const double *)vs + 4 * (size_t)s;
        x = (R)v[0]; y = (R)v[1]; z = (R)v[2];
    }
}
template <class R>
__device__ __forceinline__ void add_grad(void *g, int s, R x, R y, R z) {
    if (sizeof(R) == 4) atomicAdd((float4 *)g + s, make_float4((float)x, (float)y, (float)z, 0.f));
    else atomic_add3((double *)g + 4 * (size_t)s, (double)x, (double)y, (double)z);
}

// Warp per cell I, lanes over (partner molecule, I molecule) pairs of one
// entry batch at a time: simple and exact; the adjoint is not the hot path.
template <class R>
__global__ void __launch_bounds__(kPairThreads) pair_bwd(BwdArgs b) {
    const PairArgs &a = b.p;
    __shared__ BwdTab tab[kMaxSpeciesBwd * kMaxSpeciesBwd];
    __shared__ double red[kPairThreads / 32][2 * kMaxSpeciesBwd];
    for (int i = threadIdx.x; i < kMaxSpeciesBwd * kMaxSpeciesBwd; i += blockDim.x) tab[i] = b.t[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nwarps = gridDim.x * (kPairThreads / 32);
    BwdLane<double> tot;
    for (int q = 0; q < kMaxSpeciesBwd; ++q) tot.ge[q] = tot.gs[q] = 0;
    for (int I = blockIdx.x * (kPairThreads / 32) + wib; I < a.C; I += nwarps) {
        const int sI = a.cell_off[I], nI = a.cell_off[I + 1] - sI;
        if (nI == 0) continue;
        const int e0 = a.work_off[I], es = a.work_split[I], e1 = a.work_off[I + 1];
        BwdLane<R> gl;
        for (int q = 0; q < kMaxSpeciesBwd; ++q) gl.ge[q] = gl.gs[q] = R(0);
        // entry -1: the cell itself (pairs k' > k); then e0..e1
        for (int e = e0 - 1; e < e1; ++e) {
            int J, np = 0;
            float4 d = make_float4(0.f, 0.f, 0.f, 0.f);
            bool newton;
            if (e < e0) {
                J = I;
                newton = true;
            } else {
                WorkEntry we = a.work[e];
                J = we.j;
                np = we.n;
                d = a.work_d32[e];
                newton = e < es;
            }
            const int sJ = a.cell_off[J], nJ = a.cell_off[J + 1] - sJ;
            const int npairs = nI * nJ;
            for (int p = lane; p < npairs; p += 32) {
                int ki = p / nJ, lj = p - ki * nJ;
                if (e < e0 && lj <= ki) continue;
                int k = sI + ki, l = sJ + lj;
                float4 xk = a.xloc[k];
                R rx, ry, rz, r2;
                bool in;
                Pos<R>::sep(a, xk, l, d, np, k, rx, ry, rz, r2, in);
                if (!in) continue;
                R vkx, vky, vkz, vlx, vly, vlz;
                ldv<R>(a.vs, k, vkx, vky, vkz);
                R wx = vkx, wy = vky, wz = vkz;
                if (newton) {
                    ldv<R>(a.vs, l, vlx, vly, vlz);
                    wx -= vlx; wy -= vly; wz -= vlz;
                }
                R3<R> gi = {0, 0, 0}, gj = {0, 0, 0};
                bwd_pair<R>(tab, b.S, rx, ry, rz, r2, __float_as_int(xk.w), __float_as_int(a.xloc[l].w), wx, wy,
                            wz, gi, gj, gl);
                add_grad<R>(a.facc, k, gi.x, gi.y, gi.z);
                add_grad<R>(a.facc, l, gj.x, gj.y, gj.z);
            }
        }
        for (int q = 0; q < kMaxSpeciesBwd; ++q) {
            tot.ge[q] += (double)gl.ge[q];
            tot.gs[q] += (double)gl.gs[q];
        }
    }
    for (int q = 0; q < kMaxSpeciesBwd; ++q) {
        double x = warp_sum(tot.ge[q]), y = warp_sum(tot.gs[q]);
        if (lane == 0) {
            red[wib][q] = x;
            red[wib][kMaxSpeciesBwd + q] = y;
        }
    }
    __syncthreads();
    if (threadIdx.x < 2 * kMaxSpeciesBwd) {
        double s = 0;
        for (int w = 0; w < kPairThreads / 32; ++w) s += red[w][threadIdx.x];
        atomicAdd(a.acc + 16 + threadIdx.x, s);
    }
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

__global__ void finish_bwd(const double *acc, int S, double *ge, double *gs) {
    int i = threadIdx.x;
    if (i < S) {
        if (ge) ge[i] = acc[16 + i];
        if (gs) gs[i] = acc[16 + kMaxSpeciesBwd + i];
    }
}

int pair_grid(int C) {
    int warps = kPairThreads / 32;
    int need = (C + warps - 1) / warps;
    return std::max(1, std::min(need, 152 * 8));
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
    a.work_split = m->work_split.as<int>();
    a.work = m->work.as<WorkEntry>();
    a.work_d32 = m->work_d32.as<float4>();
    a.xloc = m->xloc.as<float4>();
    a.xs64 = m->xs64.as<double>();
    double rc2 = m->rc * m->rc;
    a.rc2_d = rc2;
    a.rc2_f = (float)rc2;
    a.rc2_lo = (float)(rc2 * (1 - 1e-5));
    a.rc2_hi = (float)(rc2 * (1 + 1e-5));
    for (int d = 0; d < 3; ++d) a.L[d] = m->box.periodic[d] ? m->box.L[d] : 0.0;
    a.facc = m->facc.p;
    a.acc = m->acc.as<double>();
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

}  // namespace
}  // namespace aica

using namespace aica;

extern "C" aica_status aica_forces(aica_mesh *m, const aica_lj *lj, aica_precision prec, void *force_out,
                                   double *ev_out, int64_t *counts_out, void *stream) {
    if (!m || !force_out) { set_error("aica_forces: NULL argument"); return AICA_ERR_INVALID_ARG; }
    if (prec != AICA_FP32 && prec != AICA_FP64) { set_error("aica_forces: bad precision"); return AICA_ERR_INVALID_ARG; }
    if (!m->built || !m->binned) { set_error("aica_forces: build the lists and bin the molecules first"); return AICA_ERR_NOT_BUILT; }
    cudaStream_t st = (cudaStream_t)stream;
    PairArgs a{};
    aica_status s = fill_params(m, lj, kMaxSpecies, a);
    if (s != AICA_OK) return s;
    fill_common(m, a);
    m->launches = 0;
    const int64_t n = m->n_mol;
    const bool f64 = prec == AICA_FP64;
    if (n > 0) AICA_CUDA(cudaMemsetAsync(m->facc.p, 0, (f64 ? 4 * sizeof(double) : sizeof(float4)) * n, st));
    AICA_CUDA(cudaMemsetAsync(m->acc.p, 0, 16 * sizeof(double), st));
    const bool multi = a.S > 1, shift = lj->shift != 0;
    const int grid = pair_grid(a.C);
    cudaEvent_t tstop;
    AICA_CUDA(timing_begin(m, st, &tstop));
    if (!f64) {
        if (multi) {
            if (shift) pair_fwd32<true, true><<<grid, kPairThreads, 0, st>>>(a);
            else pair_fwd32<true, false><<<grid, kPairThreads, 0, st>>>(a);
        } else {
            if (shift) pair_fwd32<false, true><<<grid, kPairThreads, 0, st>>>(a);
            else pair_fwd32<false, false><<<grid, kPairThreads, 0, st>>>(a);
        }
    } else {
        if (multi) {
            if (shift) pair_fwd64<true, true><<<grid, kPairThreads, 0, st>>>(a);
            else pair_fwd64<true, false><<<grid, kPairThreads, 0, st>>>(a);
        } else {
            if (shift) pair_fwd64<false, true><<<grid, kPairThreads, 0, st>>>(a);
            else pair_fwd64<false, false><<<grid, kPairThreads, 0, st>>>(a);
        }
    }
    AICA_CUDA(timing_end(tstop, st));
    if (n > 0) {
        if (f64) unsort_forces<double><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(m->inv.as<int>(), n, m->facc.p, (double *)force_out, 1);
        else unsort_forces<float><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(m->inv.as<int>(), n, m->facc.p, (float *)force_out, 0);
    }
    m->launches = n > 0 ? 2 : 1;
    if (ev_out || counts_out) {
        finish_sums<<<1, 32, 0, st>>>(m->acc.as<double>(), ev_out, (long long *)counts_out);
        m->launches++;
    }
    AICA_CUDA(cudaGetLastError());
    if (!m->deferred) return check_flags(m, st);
    return AICA_OK;
}

extern "C" aica_status aica_forces_backward(aica_mesh *m, const aica_lj *lj, aica_precision prec,
                                            const void *grad_force, void *grad_pos, double *grad_eps,
                                            double *grad_sigma, void *stream) {
    if (!m || !grad_force || !grad_pos) { set_error("aica_forces_backward: NULL argument"); return AICA_ERR_INVALID_ARG; }
    if (prec != AICA_FP32 && prec != AICA_FP64) { set_error("aica_forces_backward: bad precision"); return AICA_ERR_INVALID_ARG; }
    if (!m->built || !m->binned) { set_error("aica_forces_backward: build the lists and bin the molecules first"); return AICA_ERR_NOT_BUILT; }
    cudaStream_t st = (cudaStream_t)stream;
    BwdArgs b{};
    aica_status s = fill_params(m, lj, kMaxSpeciesBwd, b.p);
    if (s != AICA_OK) return s;
    fill_common(m, b.p);
    b.S = b.p.S;
    for (int i = 0; i < b.S; ++i)
        for (int j = 0; j < b.S; ++j) {
            BwdTab &t = b.t[i * kMaxSpeciesBwd + j];
            double e = sqrt(lj->eps[i] * lj->eps[j]), sg = 0.5 * (lj->sigma[i] + lj->sigma[j]);
            t.eps = e;
            t.sig2 = sg * sg;
            t.inv_eps = e > 0 ? 1.0 / e : 0.0;
            t.inv_sig = 1.0 / sg;
            // d eps_ab / d eps_a = eps_ab / (2 eps_a)  (both halves when a == b)
            t.fa = lj->eps[i] > 0 ? e / (2.0 * lj->eps[i]) : 0.0;
            t.fb = lj->eps[j] > 0 ? e / (2.0 * lj->eps[j]) : 0.0;
        }
    m->launches = 0;
    const int64_t n = m->n_mol;
    const bool f64 = prec == AICA_FP64;
    const size_t esz = f64 ? 4 * sizeof(double) : sizeof(float4);
    int nb = 0;
    AICA_CUDA(cudaMemcpyAsync(&nb, m->cell_off.as<int>() + m->n_cells, sizeof(int), cudaMemcpyDeviceToHost, st));
    AICA_CUDA(cudaStreamSynchronize(st));
    if (n > 0) {
        AICA_CUDA(cudaMemsetAsync(m->facc.p, 0, esz * n, st));
        if (nb > 0) {
            if (f64) gather_grad<double><<<(nb + 255) / 256, 256, 0, st>>>(m->order.as<int>(), nb, (const double *)grad_force, m->vsorted.p, 1);
            else gather_grad<float><<<(nb + 255) / 256, 256, 0, st>>>(m->order.as<int>(), nb, (const float *)grad_force, m->vsorted.p, 0);
        }
    }
    AICA_CUDA(cudaMemsetAsync(m->acc.as<double>() + 16, 0, 2 * kMaxSpeciesBwd * sizeof(double), st));
    b.p.vs = m->vsorted.p;
    const int grid = pair_grid(b.p.C);
    if (f64) pair_bwd<double><<<grid, kPairThreads, 0, st>>>(b);
    else pair_bwd<float><<<grid, kPairThreads, 0, st>>>(b);
    if (n > 0) {
        if (f64) unsort_forces<double><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(m->inv.as<int>(), n, m->facc.p, (double *)grad_pos, 1);
        else unsort_forces<float><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(m->inv.as<int>(), n, m->facc.p, (float *)grad_pos, 0);
    }
    if (grad_eps || grad_sigma) finish_bwd<<<1, 32, 0, st>>>(m->acc.as<double>(), b.S, grad_eps, grad_sigma);
    m->launches = 5;
    AICA_CUDA(cudaGetLastError());
    if (!m->deferred) return check_flags(m, st);
    return AICA_OK;
}
