// Closest-point distances between points, segments and triangles, templated
// on the scalar type (FP32 filter / FP64 decision).  Point-triangle by the
// Voronoi regions of the triangle's vertices and edges; segment-segment by the
// clamped parametric solution (both as in Ericson, "Real-Time Collision
// Detection", 2005, §5.1.5 and §5.1.9, written here from the geometry).
#pragma once

#include <cuda_runtime.h>

namespace aica {

template <class T> struct V3 { T x, y, z; };

template <class T> __host__ __device__ __forceinline__ V3<T> operator-(V3<T> a, V3<T> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class T> __host__ __device__ __forceinline__ V3<T> operator+(V3<T> a, V3<T> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class T> __host__ __device__ __forceinline__ V3<T> operator*(V3<T> a, T s) { return {a.x * s, a.y * s, a.z * s}; }
template <class T> __host__ __device__ __forceinline__ T dot3(V3<T> a, V3<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

template <class T> __host__ __device__ __forceinline__ T clamp01(T v) { return v < T(0) ? T(0) : (v > T(1) ? T(1) : v); }

// squared distance from p to triangle abc
template <class T>
__host__ __device__ inline T d2_point_triangle(V3<T> p, V3<T> a, V3<T> b, V3<T> c) {
    V3<T> ab = b - a, ac = c - a, ap = p - a;
    T d1 = dot3(ab, ap), d2 = dot3(ac, ap);
    V3<T> q;
    if (d1 <= T(0) && d2 <= T(0)) {
        q = a;
    } else {
        V3<T> bp = p - b;
        T d3 = dot3(ab, bp), d4 = dot3(ac, bp);
        if (d3 >= T(0) && d4 <= d3) {
            q = b;
        } else {
            T vc = d1 * d4 - d3 * d2;
            if (vc <= T(0) && d1 >= T(0) && d3 <= T(0)) {
                q = a + ab * (d1 / (d1 - d3));
            } else {
                V3<T> cp = p - c;
                T d5 = dot3(ab, cp), d6 = dot3(ac, cp);
                if (d6 >= T(0) && d5 <= d6) {
                    q = c;
                } else {
                    T vb = d5 * d2 - d1 * d6;
                    if (vb <= T(0) && d2 >= T(0) && d6 <= T(0)) {
                        q = a + ac * (d2 / (d2 - d6));
                    } else {
                        T va = d3 * d6 - d5 * d4;
                        if (va <= T(0) && (d4 - d3) >= T(0) && (d5 - d6) >= T(0)) {
                            q = b + (c - b) * ((d4 - d3) / ((d4 - d3) + (d5 - d6)));
                        } else {
                            T den = T(1) / (va + vb + vc);
                            q = a + ab * (vb * den) + ac * (vc * den);
                        }
                    }
                }
            }
        }
    }
    V3<T> d = p - q;
    return dot3(d, d);
}

// squared distance between segments p0p1 and q0q1 (non-degenerate)
template <class T>
__host__ __device__ inline T d2_segment_segment(V3<T> p0, V3<T> p1, V3<T> q0, V3<T> q1) {
    V3<T> d1 = p1 - p0, d2 = q1 - q0, r = p0 - q0;
    T a = dot3(d1, d1), e = dot3(d2, d2), f = dot3(d2, r);
    T c = dot3(d1, r), b = dot3(d1, d2);
    T den = a * e - b * b;
    T s = den > T(0) ? clamp01((b * f - c * e) / den) : T(0);
    T t = (b * s + f) / e;
    if (t < T(0)) {
        t = T(0);
        s = clamp01(-c / a);
    } else if (t > T(1)) {
        t = T(1);
        s = clamp01((b - c) / a);
    }
    V3<T> g = (p0 + d1 * s) - (q0 + d2 * t);
    return dot3(g, g);
}

}  // namespace aica
