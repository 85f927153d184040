// Robust orientation predicates for point location.
//
// O(a, b, c, p) = ((b - a) x (c - a)) . (p - a): positive when p lies on the
// side the right-handed normal of triangle abc points to.  Ties are broken by
// simulation of simplicity on the query point only: p is read as
// p + (e, e^2, e^3) for infinitesimal e > 0, so the sign is the first nonzero
// of (O, N_x, N_y, N_z) with N = (b - a) x (c - a).  Signs are decided by an
// FP32 filter, then an FP64 filter, then exact expansion arithmetic (error-free
// transformations: TwoSum and an FMA-based TwoProduct, summed with zero-
// eliminating expansion growth as in Shewchuk, "Adaptive precision floating-
// point arithmetic and fast robust geometric predicates", 1997).
#pragma once

#include <cuda_runtime.h>

#include <cmath>

// The exact stages also run on the host (mesh checks); host code is built
// with FP contraction off, so every operation rounds as written there too.
#ifdef __CUDA_ARCH__
#define AICA_DADD(a, b) __dadd_rn(a, b)
#define AICA_DSUB(a, b) __dsub_rn(a, b)
#define AICA_DMUL(a, b) __dmul_rn(a, b)
#define AICA_DFMA(a, b, c) __fma_rn(a, b, c)
#else
#define AICA_DADD(a, b) ((a) + (b))
#define AICA_DSUB(a, b) ((a) - (b))
#define AICA_DMUL(a, b) ((a) * (b))
#define AICA_DFMA(a, b, c) std::fma(a, b, c)
#endif

namespace aica {

// ------------------------------------------------------------ exact arithmetic
__host__ __device__ __forceinline__ void two_sum(double a, double b, double &x, double &y) {
    x = AICA_DADD(a, b);
    double bv = AICA_DSUB(x, a);
    double av = AICA_DSUB(x, bv);
    y = AICA_DADD(AICA_DSUB(a, av), AICA_DSUB(b, bv));
}
__host__ __device__ __forceinline__ void two_diff(double a, double b, double &x, double &y) {
    x = AICA_DSUB(a, b);
    double bv = AICA_DSUB(a, x);
    double av = AICA_DADD(x, bv);
    y = AICA_DADD(AICA_DSUB(a, av), AICA_DSUB(bv, b));
}
__host__ __device__ __forceinline__ void two_prod(double a, double b, double &x, double &y) {
    x = AICA_DMUL(a, b);
    y = AICA_DFMA(a, b, -x);
}

// e <- e + b, keeping e a nonoverlapping expansion in increasing magnitude
// with zero components removed.
__host__ __device__ inline void grow(double *e, int &n, double b) {
    if (b == 0.0) return;
    double q = b;
    int m = 0;
    for (int i = 0; i < n; ++i) {
        double s, h;
        two_sum(q, e[i], s, h);
        q = s;
        if (h != 0.0) e[m++] = h;
    }
    if (q != 0.0) e[m++] = q;
    n = m;
}

__host__ __device__ inline int expansion_sign(const double *e, int n) {
    return n == 0 ? 0 : (e[n - 1] > 0 ? 1 : -1);
}

// add s * (x1 + x0) * (y1 + y0) * (z1 + z0) to e (each factor a two-term
// expansion; zero terms, common for inputs on a lattice, are skipped)
__host__ __device__ inline void grow_triple(double *e, int &n, double s, const double x[2], const double y[2],
                                            const double z[2]) {
    for (int i = 0; i < 2; ++i) {
        if (x[i] == 0.0) continue;
        for (int j = 0; j < 2; ++j) {
            if (y[j] == 0.0) continue;
            double p, q;
            two_prod(x[i], y[j], p, q);
            for (int k = 0; k < 2; ++k) {
                if (z[k] == 0.0) continue;
                double r, t;
                two_prod(p, z[k], r, t);
                grow(e, n, s * r);
                grow(e, n, s * t);
                if (q != 0.0) {
                    two_prod(q, z[k], r, t);
                    grow(e, n, s * r);
                    grow(e, n, s * t);
                }
            }
        }
    }
}

// exact sign of det[u; v; w] where u = a - p etc. (rows), FP64 inputs
static __host__ __device__ __noinline__ int exact_det3_sign(const double *a, const double *b, const double *c,
                                                   const double *p) {
    double u[3][2], v[3][2], w[3][2];
    for (int d = 0; d < 3; ++d) {
        two_diff(a[d], p[d], u[d][0], u[d][1]);
        two_diff(b[d], p[d], v[d][0], v[d][1]);
        two_diff(c[d], p[d], w[d][0], w[d][1]);
    }
    double e[200];
    int n = 0;
    // u.(v x w) = ux(vy wz - vz wy) + uy(vz wx - vx wz) + uz(vx wy - vy wx)
    grow_triple(e, n, 1.0, u[0], v[1], w[2]);
    grow_triple(e, n, -1.0, u[0], v[2], w[1]);
    grow_triple(e, n, 1.0, u[1], v[2], w[0]);
    grow_triple(e, n, -1.0, u[1], v[0], w[2]);
    grow_triple(e, n, 1.0, u[2], v[0], w[1]);
    grow_triple(e, n, -1.0, u[2], v[1], w[0]);
    return expansion_sign(e, n);
}

// exact sign of (b_i - a_i)(c_j - a_j) - (b_j - a_j)(c_i - a_i)
static __device__ __noinline__ int exact_det2_sign(const double *a, const double *b, const double *c, int i, int j) {
    double x[2], y[2], z[2], t[2];
    two_diff(b[i], a[i], x[0], x[1]);
    two_diff(c[j], a[j], y[0], y[1]);
    two_diff(b[j], a[j], z[0], z[1]);
    two_diff(c[i], a[i], t[0], t[1]);
    double e[24];
    int n = 0;
    for (int r = 0; r < 2; ++r)
        for (int s = 0; s < 2; ++s) {
            double p, q;
            if (x[r] != 0.0 && y[s] != 0.0) {
                two_prod(x[r], y[s], p, q);
                grow(e, n, p);
                grow(e, n, q);
            }
            if (z[r] != 0.0 && t[s] != 0.0) {
                two_prod(z[r], t[s], p, q);
                grow(e, n, -p);
                grow(e, n, -q);
            }
        }
    return expansion_sign(e, n);
}

// --------------------------------------------------------------- the predicate
// FP64 stage and exact stage of the perturbed orientation sign (FP64 inputs).
static __device__ __noinline__ int orient_sos_slow(const double *a, const double *b, const double *c, const double *p) {
    double u[3], v[3], w[3];
    for (int d = 0; d < 3; ++d) {
        u[d] = a[d] - p[d];
        v[d] = b[d] - p[d];
        w[d] = c[d] - p[d];
    }
    double m0 = v[1] * w[2], m1 = v[2] * w[1], m2 = v[2] * w[0], m3 = v[0] * w[2], m4 = v[0] * w[1], m5 = v[1] * w[0];
    double det = u[0] * (m0 - m1) + u[1] * (m2 - m3) + u[2] * (m4 - m5);
    double perm = fabs(u[0]) * (fabs(m0) + fabs(m1)) + fabs(u[1]) * (fabs(m2) + fabs(m3)) +
                  fabs(u[2]) * (fabs(m4) + fabs(m5));
    int s;
    if (det > 1e-14 * perm) s = 1;
    else if (det < -1e-14 * perm) s = -1;
    else s = exact_det3_sign(a, b, c, p);
    if (s != 0) return -s;   // O = -det[a-p; b-p; c-p]
    // p on the plane: N_x, N_y, N_z of N = (b - a) x (c - a), exactly
    int nx = exact_det2_sign(a, b, c, 1, 2);
    if (nx) return nx;
    int ny = exact_det2_sign(a, b, c, 2, 0);
    if (ny) return ny;
    return exact_det2_sign(a, b, c, 0, 1);
}

// FP32 filter on coordinates local to a common origin.  The local copies
// carry an absolute rounding error of at most 2^-24 of their magnitude each;
// `scale` bounds every local coordinate magnitude involved.  Returns +-1 when
// certain, 0 when the slow path must decide.
__device__ __forceinline__ int orient_f32(float3 a, float3 b, float3 c, float3 p, float scale) {
    float ux = a.x - p.x, uy = a.y - p.y, uz = a.z - p.z;
    float vx = b.x - p.x, vy = b.y - p.y, vz = b.z - p.z;
    float wx = c.x - p.x, wy = c.y - p.y, wz = c.z - p.z;
    float m0 = vy * wz, m1 = vz * wy, m2 = vz * wx, m3 = vx * wz, m4 = vx * wy, m5 = vy * wx;
    float det = ux * (m0 - m1) + uy * (m2 - m3) + uz * (m4 - m5);
    float perm = fabsf(ux) * (fabsf(m0) + fabsf(m1)) + fabsf(uy) * (fabsf(m2) + fabsf(m3)) +
                 fabsf(uz) * (fabsf(m4) + fabsf(m5));
    float su = fabsf(ux) + fabsf(uy) + fabsf(uz), sv = fabsf(vx) + fabsf(vy) + fabsf(vz),
          sw = fabsf(wx) + fabsf(wy) + fabsf(wz);
    float bound = 1e-5f * perm + 1e-6f * scale * (sv * sw + su * sw + su * sv);
    if (det > bound) return -1;
    if (det < -bound) return 1;
    return 0;
}

}  // namespace aica
