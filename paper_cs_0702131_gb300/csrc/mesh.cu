// Mesh ingest: validation, fan triangulation, per-cell geometry, dyadic cell
// origins and the point-location bucket grid (step a1 of the hot path; runs
// once, like the list construction it feeds, App. A).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "aica_internal.cuh"
#include "scan.cuh"
#include "predicates.cuh"

namespace {

struct CellTri {
    int64_t cell;
    int64_t a, b, c;
};

template <class T>
cudaError_t upload(aica::DevBuf &buf, const std::vector<T> &h) {
    size_t n = h.size() * sizeof(T);
    cudaError_t e = buf.reserve(n > 0 ? n : sizeof(T));
    if (e != cudaSuccess) return e;
    if (n) e = cudaMemcpy(buf.p, h.data(), n, cudaMemcpyHostToDevice);
    return e;
}

}  // namespace

namespace {
// Sign of O(a, b, c, p) = ((b - a) x (c - a)) . (p - a), exactly: FP64 filter,
// then the exact determinant.
int orient_host(const double *a, const double *b, const double *c, const double *p) {
    double u[3], v[3], w[3];
    for (int d = 0; d < 3; ++d) { u[d] = a[d] - p[d]; v[d] = b[d] - p[d]; w[d] = c[d] - p[d]; }
    double m0 = v[1] * w[2], m1 = v[2] * w[1], m2 = v[2] * w[0], m3 = v[0] * w[2], m4 = v[0] * w[1], m5 = v[1] * w[0];
    double det = u[0] * (m0 - m1) + u[1] * (m2 - m3) + u[2] * (m4 - m5);
    double perm = fabs(u[0]) * (fabs(m0) + fabs(m1)) + fabs(u[1]) * (fabs(m2) + fabs(m3)) +
                  fabs(u[2]) * (fabs(m4) + fabs(m5));
    int s;
    if (det > 1e-14 * perm) s = 1;
    else if (det < -1e-14 * perm) s = -1;
    else s = aica::exact_det3_sign(a, b, c, p);
    return -s;
}
}  // namespace

extern "C" aica_status aica_mesh_create(const double *points, int64_t n_points, const int64_t *face_offsets,
                                        const int64_t *face_vertices, int64_t n_faces, const int64_t *owner,
                                        const int64_t *neighbour, int64_t n_cells, const aica_box *box,
                                        aica_mesh **out) {
    AICA_RANGE("aica_mesh_create");
    using namespace aica;
    if (!out) { set_error("aica_mesh_create: out is NULL"); return AICA_ERR_INVALID_ARG; }
    *out = nullptr;
    if (!points || !face_offsets || !face_vertices || !owner || !neighbour || !box) {
        set_error("aica_mesh_create: NULL input array");
        return AICA_ERR_INVALID_ARG;
    }
    if (n_points < 4 || n_faces < 4 || n_cells < 1 || n_cells > (int64_t)INT32_MAX / 2) {
        set_error("aica_mesh_create: bad sizes (points %lld, faces %lld, cells %lld)", (long long)n_points,
                  (long long)n_faces, (long long)n_cells);
        return AICA_ERR_INVALID_ARG;
    }
    for (int d = 0; d < 3; ++d)
        if (box->periodic[d] && !(box->L[d] > 0 && isfinite(box->L[d]))) {
            set_error("aica_mesh_create: periodic axis %d needs L > 0", d);
            return AICA_ERR_INVALID_ARG;
        }

    // ---- faces -> oriented triangles per cell (fan from the lowest vertex id)
    std::vector<int64_t> tcount(n_cells + 1, 0);
    if (face_offsets[0] != 0) { set_error("face_offsets[0] must be 0"); return AICA_ERR_BAD_MESH; }
    for (int64_t f = 0; f < n_faces; ++f) {
        int64_t k = face_offsets[f + 1] - face_offsets[f];
        if (k < 3) { set_error("face %lld has %lld vertices", (long long)f, (long long)k); return AICA_ERR_BAD_MESH; }
        if (owner[f] < 0 || owner[f] >= n_cells || neighbour[f] < -1 || neighbour[f] >= n_cells ||
            neighbour[f] == owner[f]) {
            set_error("face %lld: bad owner/neighbour", (long long)f);
            return AICA_ERR_BAD_MESH;
        }
        tcount[owner[f] + 1] += k - 2;
        if (neighbour[f] >= 0) tcount[neighbour[f] + 1] += k - 2;
    }
    for (int64_t c = 0; c < n_cells; ++c) tcount[c + 1] += tcount[c];
    int64_t T = tcount[n_cells];
    std::vector<int64_t> tv(3 * T);
    std::vector<int32_t> h_tri_nbr(T);      // the cell on the other side of each triangle (-1: boundary)
    std::vector<int64_t> fillc(n_cells, 0);
    for (int64_t f = 0; f < n_faces; ++f) {
        const int64_t *v = face_vertices + face_offsets[f];
        int64_t k = face_offsets[f + 1] - face_offsets[f];
        int64_t r = 0;
        for (int64_t i = 0; i < k; ++i) {
            if (v[i] < 0 || v[i] >= n_points) { set_error("face %lld: vertex out of range", (long long)f); return AICA_ERR_BAD_MESH; }
            if (v[i] < v[r]) r = i;
        }
        for (int64_t i = 1; i + 1 < k; ++i) {
            int64_t a = v[r], b = v[(r + i) % k], c = v[(r + i + 1) % k];
            int64_t o = tcount[owner[f]] + fillc[owner[f]]++;
            tv[3 * o] = a; tv[3 * o + 1] = b; tv[3 * o + 2] = c;
            h_tri_nbr[o] = (int32_t)neighbour[f];
            if (neighbour[f] >= 0) {
                int64_t q = tcount[neighbour[f]] + fillc[neighbour[f]]++;
                tv[3 * q] = a; tv[3 * q + 1] = c; tv[3 * q + 2] = b;
                h_tri_nbr[q] = (int32_t)owner[f];
            }
        }
    }

    // ---- per-cell checks and geometry
    std::vector<int32_t> h_tri_off(n_cells + 1), h_vtx_off(n_cells + 1), h_edg_off(n_cells + 1), h_ntri(n_cells);
    std::vector<double> h_tri(9 * T), h_ctr(3 * n_cells), h_rad(n_cells), h_lo(3 * n_cells), h_hi(3 * n_cells),
        h_org(3 * n_cells);
    std::vector<double> h_vtx, h_edg;
    std::vector<int32_t> h_orgk(3 * n_cells);
    h_vtx.reserve(3 * T);
    h_edg.reserve(6 * T);
    int max_tri = 0, max_vtx = 0, max_edg = 0;
    std::vector<int64_t> vs, es;
    std::vector<std::pair<int64_t, int64_t>> de;
    h_tri_off[0] = h_vtx_off[0] = h_edg_off[0] = 0;
    for (int64_t c = 0; c < n_cells; ++c) {
        int64_t t0 = tcount[c], t1 = tcount[c + 1];
        int nt = (int)(t1 - t0);
        vs.clear(); de.clear();
        for (int64_t t = t0; t < t1; ++t)
            for (int i = 0; i < 3; ++i) {
                vs.push_back(tv[3 * t + i]);
                de.emplace_back(tv[3 * t + i], tv[3 * t + (i + 1) % 3]);
            }
        std::sort(vs.begin(), vs.end());
        vs.erase(std::unique(vs.begin(), vs.end()), vs.end());
        // closed, consistently oriented surface: every directed edge once, its reverse once
        std::sort(de.begin(), de.end());
        bool closed = nt >= 4;
        for (size_t i = 0; closed && i < de.size(); ++i) {
            if (i + 1 < de.size() && de[i] == de[i + 1]) closed = false;
            if (!std::binary_search(de.begin(), de.end(), std::make_pair(de[i].second, de[i].first))) closed = false;
        }
        if (!closed) { set_error("cell %lld is not a closed oriented surface", (long long)c); return AICA_ERR_BAD_MESH; }
        int ne = (int)de.size() / 2;
        if (nt > kMaxTri || (int)vs.size() > kMaxVtx || ne > kMaxEdg) {
            set_error("cell %lld exceeds %d triangles / %d vertices / %d edges", (long long)c, kMaxTri, kMaxVtx, kMaxEdg);
            return AICA_ERR_CAPACITY;
        }
        max_tri = std::max(max_tri, nt);
        max_vtx = std::max(max_vtx, (int)vs.size());
        max_edg = std::max(max_edg, ne);
        double C[3] = {0, 0, 0}, lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int64_t v : vs)
            for (int d = 0; d < 3; ++d) {
                double x = points[3 * v + d];
                if (!isfinite(x)) { set_error("vertex %lld is not finite", (long long)v); return AICA_ERR_BAD_MESH; }
                C[d] += x;
                lo[d] = std::min(lo[d], x);
                hi[d] = std::max(hi[d], x);
            }
        double rad = 0;
        for (int d = 0; d < 3; ++d) C[d] /= (double)vs.size();
        for (int64_t v : vs) {
            double s = 0;
            for (int d = 0; d < 3; ++d) s += (points[3 * v + d] - C[d]) * (points[3 * v + d] - C[d]);
            rad = std::max(rad, sqrt(s));
            h_vtx.insert(h_vtx.end(), points + 3 * v, points + 3 * v + 3);
        }
        for (int d = 0; d < 3; ++d) {
            if (box->periodic[d] && (lo[d] < -1e-9 * box->L[d] || hi[d] > box->L[d] * (1 + 1e-9))) {
                set_error("cell %lld leaves the periodic box on axis %d", (long long)c, d);
                return AICA_ERR_BAD_MESH;
            }
            h_ctr[3 * c + d] = C[d];
            h_lo[3 * c + d] = lo[d];
            h_hi[3 * c + d] = hi[d];
            h_org[3 * c + d] = rint(C[d] * 1024.0) / 1024.0;   // dyadic: exact in FP32 differences
            if (fabs(h_org[3 * c + d]) > 1e6) { set_error("cell %lld: coordinates beyond 1e6", (long long)c); return AICA_ERR_BAD_MESH; }
            h_orgk[3 * c + d] = (int32_t)rint(C[d] * 1024.0);
        }
        h_rad[c] = rad;
        // star-shaped about C: every (C, triangle) tetrahedron has positive volume
        for (int64_t t = t0; t < t1; ++t) {
            const double *a = points + 3 * tv[3 * t], *b = points + 3 * tv[3 * t + 1], *e = points + 3 * tv[3 * t + 2];
            double u[3], w[3], q[3];
            for (int d = 0; d < 3; ++d) { u[d] = a[d] - C[d]; w[d] = b[d] - C[d]; q[d] = e[d] - C[d]; }
            double vol = u[0] * (w[1] * q[2] - w[2] * q[1]) - u[1] * (w[0] * q[2] - w[2] * q[0]) +
                         u[2] * (w[0] * q[1] - w[1] * q[0]);
            double scale = sqrt((u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) * (w[0] * w[0] + w[1] * w[1] + w[2] * w[2]) *
                                (q[0] * q[0] + q[1] * q[1] + q[2] * q[2]));
            if (!(vol > 1e-12 * scale)) {
                set_error("cell %lld: tetrahedron from the vertex mean to triangle %lld is not positive",
                          (long long)c, (long long)(t - t0));
                return AICA_ERR_BAD_MESH;
            }
            for (int i = 0; i < 3; ++i)
                for (int d = 0; d < 3; ++d) h_tri[9 * t + 3 * i + d] = points[3 * tv[3 * t + i] + d];
        }
        // unique undirected edges (fan diagonals included)
        for (auto &p : de)
            if (p.first < p.second) {
                h_edg.insert(h_edg.end(), points + 3 * p.first, points + 3 * p.first + 3);
                h_edg.insert(h_edg.end(), points + 3 * p.second, points + 3 * p.second + 3);
            }
        h_tri_off[c + 1] = (int32_t)t1;
        h_vtx_off[c + 1] = h_vtx_off[c] + (int32_t)vs.size();
        h_edg_off[c + 1] = h_edg_off[c] + ne;
        // convex: no vertex in front of any face plane (exact).  Binning then
        // decides "outside" at the first face a point is in front of.
        bool convex = true;
        if (nt != 4)
            for (int64_t t = t0; t < t1 && convex; ++t) {
                const double *a = points + 3 * tv[3 * t], *b = points + 3 * tv[3 * t + 1],
                             *e = points + 3 * tv[3 * t + 2];
                for (int64_t v : vs) {
                    if (v == tv[3 * t] || v == tv[3 * t + 1] || v == tv[3 * t + 2]) continue;
                    if (orient_host(a, b, e, points + 3 * v) > 0) { convex = false; break; }
                }
            }
        h_ntri[c] = nt | (convex ? 1 << 16 : 0);
    }
    if (T > INT32_MAX / 2) { set_error("too many triangles"); return AICA_ERR_CAPACITY; }
    std::vector<float> h_tri32(9 * T), h_vtx32(h_vtx.size()), h_edg32(h_edg.size()), h_ctr32(3 * n_cells),
        h_rad32(n_cells), h_box32(6 * n_cells);
    // per triangle, its plane in the cell's frame for the FP32 point-location
    // filter: N = (b - a) x (c - a) and N.a in FP64, both divided by |N|_1 and
    // rounded (16 B per triangle instead of 36 B of vertices)
    std::vector<float> h_pl32(4 * T);
    std::vector<int32_t> h_tric(2 * n_cells);
    double max_local = 0;
    for (int64_t c = 0; c < n_cells; ++c) {
        for (int64_t i = 3 * (int64_t)h_tri_off[c]; i < 3 * (int64_t)h_tri_off[c + 1]; ++i)
            for (int d = 0; d < 3; ++d) {
                double x = h_tri[3 * i + d] - h_org[3 * c + d];
                max_local = std::max(max_local, fabs(x));
                h_tri32[3 * i + d] = (float)x;
            }
        for (int64_t t = h_tri_off[c]; t < h_tri_off[c + 1]; ++t) {
            double v[3][3];
            for (int j = 0; j < 3; ++j)
                for (int d = 0; d < 3; ++d) v[j][d] = h_tri[9 * t + 3 * j + d] - h_org[3 * c + d];
            const double e1[3] = {v[1][0] - v[0][0], v[1][1] - v[0][1], v[1][2] - v[0][2]};
            const double e2[3] = {v[2][0] - v[0][0], v[2][1] - v[0][1], v[2][2] - v[0][2]};
            const double N[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                                 e1[0] * e2[1] - e1[1] * e2[0]};
            const double s1 = fabs(N[0]) + fabs(N[1]) + fabs(N[2]);
            const double g = (fabs(e1[0]) + fabs(e1[1]) + fabs(e1[2])) * (fabs(e2[0]) + fabs(e2[1]) + fabs(e2[2]));
            // a sliver (|N| tiny against its edges, so N's direction carries FP64
            // cancellation) or degenerate triangle gets plane 0: never decided
            const double w = s1 > 1e-6 * g ? 1.0 / s1 : 0.0;
            for (int d = 0; d < 3; ++d) h_pl32[4 * t + d] = (float)(N[d] * w);
            h_pl32[4 * t + 3] = (float)((N[0] * v[0][0] + N[1] * v[0][1] + N[2] * v[0][2]) * w);
        }
        h_tric[2 * c] = h_tri_off[c];
        h_tric[2 * c + 1] = h_ntri[c];
        for (int64_t i = h_vtx_off[c]; i < h_vtx_off[c + 1]; ++i)
            for (int d = 0; d < 3; ++d) h_vtx32[3 * i + d] = (float)(h_vtx[3 * i + d] - h_org[3 * c + d]);
        for (int64_t i = 2 * (int64_t)h_edg_off[c]; i < 2 * (int64_t)h_edg_off[c + 1]; ++i)
            for (int d = 0; d < 3; ++d) h_edg32[3 * i + d] = (float)(h_edg[3 * i + d] - h_org[3 * c + d]);
        for (int d = 0; d < 3; ++d) h_ctr32[3 * c + d] = (float)(h_ctr[3 * c + d] - h_org[3 * c + d]);
        for (int d = 0; d < 3; ++d) {
            h_box32[6 * c + d] = nextafterf((float)(h_lo[3 * c + d] - h_org[3 * c + d]), -INFINITY);
            h_box32[6 * c + 3 + d] = nextafterf((float)(h_hi[3 * c + d] - h_org[3 * c + d]), INFINITY);
        }
        h_rad32[c] = (float)(h_rad[c] * (1 + 1e-6)) + 1e-6f;
    }

    // ---- clusters and molecule frames.  A cluster is a run of consecutive
    // cells whose joint bounding box is hardly larger than the largest box
    // among its cells (the tetrahedra split from one hexahedron, or one cell
    // of a hexahedral mesh): the FP32 pair kernel takes a cluster's molecules
    // as one i-tile and culls partners against their joint box.  A molecule
    // frame (one dyadic origin for the binned FP32 coordinates) is a run of
    // consecutive clusters whose joint box stays within twice the median cell
    // extent, so a run of consecutive partner cells or clusters is one shift.
    std::vector<int32_t> h_orgm(3 * n_cells);
    std::vector<double> h_orgm64(3 * n_cells);
    std::vector<int32_t> h_cl_first, h_cl_of(n_cells);
    double max_mlocal = 0;
    {
        auto vol = [](const double *lo, const double *hi) {
            return std::max(hi[0] - lo[0], 0.0) * std::max(hi[1] - lo[1], 0.0) * std::max(hi[2] - lo[2], 0.0);
        };
        double clo[3] = {0, 0, 0}, chi[3] = {0, 0, 0}, vmax = 0;
        for (int64_t c = 0; c < n_cells; ++c) {
            const double *lo = &h_lo[3 * c], *hi = &h_hi[3 * c];
            bool join = !h_cl_first.empty() && c - h_cl_first.back() < kMaxClusterCells;
            if (join) {
                double jlo[3], jhi[3];
                for (int d = 0; d < 3; ++d) { jlo[d] = std::min(clo[d], lo[d]); jhi[d] = std::max(chi[d], hi[d]); }
                join = vol(jlo, jhi) <= 1.35 * std::max(vmax, vol(lo, hi));
            }
            if (!join) {
                h_cl_first.push_back((int32_t)c);
                vmax = 0;
                for (int d = 0; d < 3; ++d) { clo[d] = lo[d]; chi[d] = hi[d]; }
            }
            for (int d = 0; d < 3; ++d) { clo[d] = std::min(clo[d], lo[d]); chi[d] = std::max(chi[d], hi[d]); }
            vmax = std::max(vmax, vol(lo, hi));
            h_cl_of[c] = (int32_t)h_cl_first.size() - 1;
        }
        h_cl_first.push_back((int32_t)n_cells);
        const int64_t ncl = (int64_t)h_cl_first.size() - 1;

        std::vector<double> ext(n_cells);
        for (int64_t c = 0; c < n_cells; ++c) {
            double e = 0;
            for (int d = 0; d < 3; ++d) e = std::max(e, h_hi[3 * c + d] - h_lo[3 * c + d]);
            ext[c] = e;
        }
        std::vector<double> tmp(ext);
        double emax = 0;
        if (n_cells > 0) {
            std::nth_element(tmp.begin(), tmp.begin() + n_cells / 2, tmp.end());
            emax = 2.0 * tmp[n_cells / 2];
        }
        int64_t g0 = 0;           // first cell of the open frame
        double glo_[3], ghi_[3];
        auto close_group = [&](int64_t g1) {
            for (int d = 0; d < 3; ++d) {
                const int32_t k = (int32_t)rint(0.5 * (glo_[d] + ghi_[d]) * 1024.0);
                for (int64_t c = g0; c < g1; ++c) {
                    h_orgm[3 * c + d] = k;
                    h_orgm64[3 * c + d] = (double)k / 1024.0;
                    max_mlocal = std::max(max_mlocal, std::max(fabs(h_lo[3 * c + d] - (double)k / 1024.0),
                                                               fabs(h_hi[3 * c + d] - (double)k / 1024.0)));
                }
            }
        };
        for (int64_t q = 0; q < ncl; ++q) {
            const int64_t c0 = h_cl_first[q], c1 = h_cl_first[q + 1];
            double qlo[3], qhi[3];
            for (int d = 0; d < 3; ++d) { qlo[d] = INFINITY; qhi[d] = -INFINITY; }
            for (int64_t c = c0; c < c1; ++c)
                for (int d = 0; d < 3; ++d) {
                    qlo[d] = std::min(qlo[d], h_lo[3 * c + d]);
                    qhi[d] = std::max(qhi[d], h_hi[3 * c + d]);
                }
            bool join = c0 > g0 && c1 - g0 <= 64;
            if (join) {
                double e = 0;
                for (int d = 0; d < 3; ++d) e = std::max(e, std::max(ghi_[d], qhi[d]) - std::min(glo_[d], qlo[d]));
                join = e <= emax;
            }
            if (!join) {
                if (c0 > 0) close_group(c0);
                g0 = c0;
                for (int d = 0; d < 3; ++d) { glo_[d] = qlo[d]; ghi_[d] = qhi[d]; }
            } else {
                for (int d = 0; d < 3; ++d) {
                    glo_[d] = std::min(glo_[d], qlo[d]);
                    ghi_[d] = std::max(ghi_[d], qhi[d]);
                }
            }
        }
        if (n_cells > 0) close_group(n_cells);
    }

    // ---- point-location bucket grid over the mesh bounding box
    double glo[3], ghi[3];
    for (int d = 0; d < 3; ++d) {
        glo[d] = INFINITY; ghi[d] = -INFINITY;
        for (int64_t c = 0; c < n_cells; ++c) {
            glo[d] = std::min(glo[d], h_lo[3 * c + d]);
            ghi[d] = std::max(ghi[d], h_hi[3 * c + d]);
        }
    }
    double vol = 1;
    for (int d = 0; d < 3; ++d) vol *= std::max(ghi[d] - glo[d], 1e-300);
    // bucket edge: half the geometric-mean cell bounding-box edge
    double lg = 0;
    for (int64_t c = 0; c < n_cells; ++c)
        for (int d = 0; d < 3; ++d) lg += log(std::max(h_hi[3 * c + d] - h_lo[3 * c + d], 1e-12));
    double h0 = 0.5 * exp(lg / (3.0 * (double)n_cells));
    (void)vol;
    int G[3];
    double gh[3];
    for (int d = 0; d < 3; ++d) {
        G[d] = std::max(1, std::min(1024, (int)floor((ghi[d] - glo[d]) / h0)));
        gh[d] = (ghi[d] - glo[d]) / G[d];
    }
    int64_t nb = (int64_t)G[0] * G[1] * G[2];
    std::vector<int32_t> h_bkt_off(nb + 1, 0);
    std::vector<int32_t> h_bkt_cells;
    auto range = [&](int64_t c, int d, int &i0, int &i1) {
        // tolerance covers the FP32 bucket index of the point-location kernel
        i0 = (int)floor((h_lo[3 * c + d] - glo[d]) / gh[d] - 1e-3);
        i1 = (int)floor((h_hi[3 * c + d] - glo[d]) / gh[d] + 1e-3);
        i0 = std::max(i0, 0);
        i1 = std::min(i1, G[d] - 1);
    };
    for (int pass = 0; pass < 2; ++pass) {
        std::vector<int32_t> fillb(pass ? nb : 0, 0);
        if (pass) h_bkt_cells.resize(h_bkt_off[nb]);
        for (int64_t c = 0; c < n_cells; ++c) {
            int r0[3], r1[3];
            for (int d = 0; d < 3; ++d) range(c, d, r0[d], r1[d]);
            for (int x = r0[0]; x <= r1[0]; ++x)
                for (int y = r0[1]; y <= r1[1]; ++y)
                    for (int z = r0[2]; z <= r1[2]; ++z) {
                        int64_t b = ((int64_t)x * G[1] + y) * G[2] + z;
                        if (!pass) h_bkt_off[b + 1]++;
                        else h_bkt_cells[h_bkt_off[b] + fillb[b]++] = (int32_t)c;
                    }
        }
        if (!pass) {
            for (int64_t b = 0; b < nb; ++b) h_bkt_off[b + 1] += h_bkt_off[b];
            if (h_bkt_off[nb] < 0 || (int64_t)h_bkt_off[nb] > (int64_t)INT32_MAX / 2) {
                set_error("bucket grid too large");
                return AICA_ERR_CAPACITY;
            }
        }
    }

    // face neighbours of each cell (point-location search order after a move)
    std::vector<int32_t> h_nbr_off(n_cells + 1, 0), h_nbr;
    for (int64_t f = 0; f < n_faces; ++f)
        if (neighbour[f] >= 0) {
            h_nbr_off[owner[f] + 1]++;
            h_nbr_off[neighbour[f] + 1]++;
        }
    for (int64_t c = 0; c < n_cells; ++c) h_nbr_off[c + 1] += h_nbr_off[c];
    h_nbr.resize(h_nbr_off[n_cells]);
    {
        std::vector<int32_t> fl(h_nbr_off.begin(), h_nbr_off.end() - 1);
        for (int64_t f = 0; f < n_faces; ++f)
            if (neighbour[f] >= 0) {
                h_nbr[fl[owner[f]]++] = (int32_t)neighbour[f];
                h_nbr[fl[neighbour[f]]++] = (int32_t)owner[f];
            }
    }

    aica_mesh *m = new (std::nothrow) aica_mesh();
    if (!m) { set_error("host allocation failed"); return AICA_ERR_OOM; }
    cudaGetDevice(&m->device);
    m->n_cells = n_cells;
    m->n_points = n_points;
    m->box = *box;
    m->max_tri = max_tri; m->max_vtx = max_vtx; m->max_edg = max_edg;
    m->max_local = max_local;
    m->max_mlocal = max_mlocal;
    m->org32 = true;
    for (int32_t k : h_orgk) m->org32 = m->org32 && k > -(1 << 24) && k < (1 << 24);
    std::vector<float> h_orgf(h_orgk.size());
    for (size_t i = 0; i < h_orgk.size(); ++i) h_orgf[i] = (float)h_orgk[i] * (1.0f / 1024.0f);
    // the FP32 cluster kernel splits binned coordinates at multiples of
    // 2^-qexp: |x - o_m| 2^qexp < 2^22 keeps the parts exact, with room for
    // the shifts of nearby partners
    m->qexp = 22 - (int)ceil(log2(std::max(max_mlocal, 1e-3) * (1 + 1e-9)));
    m->qexp = std::min(m->qexp, 40);
    m->n_cl = (int64_t)h_cl_first.size() - 1;
    m->max_cl_cells = 0;
    for (int64_t q = 0; q < m->n_cl; ++q) m->max_cl_cells = std::max<int>(m->max_cl_cells, h_cl_first[q + 1] - h_cl_first[q]);
    for (int d = 0; d < 3; ++d) { m->G[d] = G[d]; m->glo[d] = glo[d]; m->gh[d] = gh[d]; }
    cudaError_t e = cudaSuccess;
    const char *what = "upload";
    if (e == cudaSuccess) e = upload(m->tri_off, h_tri_off);
    if (e == cudaSuccess) e = upload(m->tri, h_tri);
    if (e == cudaSuccess) e = upload(m->tri_nbr, h_tri_nbr);
    if (e == cudaSuccess) e = upload(m->ntri, h_ntri);
    if (e == cudaSuccess) e = upload(m->box32, h_box32);
    if (e == cudaSuccess) e = upload(m->vtx_off, h_vtx_off);
    if (e == cudaSuccess) e = upload(m->vtx, h_vtx);
    if (e == cudaSuccess) e = upload(m->edg_off, h_edg_off);
    if (e == cudaSuccess) e = upload(m->edg, h_edg);
    if (e == cudaSuccess) e = upload(m->ctr, h_ctr);
    if (e == cudaSuccess) e = upload(m->rad, h_rad);
    if (e == cudaSuccess) e = upload(m->lo, h_lo);
    if (e == cudaSuccess) e = upload(m->hi, h_hi);
    if (e == cudaSuccess) e = upload(m->org, h_org);
    if (e == cudaSuccess) e = upload(m->orgk, h_orgk);
    if (e == cudaSuccess) e = upload(m->orgm, h_orgm);
    if (e == cudaSuccess) e = upload(m->orgm64, h_orgm64);
    if (e == cudaSuccess) e = upload(m->cl_first, h_cl_first);
    if (e == cudaSuccess) e = upload(m->cl_of, h_cl_of);
    if (e == cudaSuccess) e = upload(m->tri32, h_tri32);
    if (e == cudaSuccess) e = upload(m->pl32, h_pl32);
    if (e == cudaSuccess) e = upload(m->tric, h_tric);
    if (e == cudaSuccess) e = upload(m->orgf, h_orgf);
    if (e == cudaSuccess) e = upload(m->vtx32, h_vtx32);
    if (e == cudaSuccess) e = upload(m->edg32, h_edg32);
    if (e == cudaSuccess) e = upload(m->ctr32, h_ctr32);
    if (e == cudaSuccess) e = upload(m->rad32, h_rad32);
    if (e == cudaSuccess) e = upload(m->nbr_off, h_nbr_off);
    if (e == cudaSuccess) e = upload(m->nbr, h_nbr);
    if (e == cudaSuccess) e = upload(m->bkt_off, h_bkt_off);
    if (e == cudaSuccess) e = upload(m->bkt_cells, h_bkt_cells);
    if (e == cudaSuccess) { e = m->flags.reserve(16); what = "flags"; }
    if (e == cudaSuccess) e = cudaMemset(m->flags.p, 0, 16);
    if (e == cudaSuccess) { e = m->acc.reserve(sizeof(double) * (64 + 64 * 16)); what = "acc"; }
    if (e == cudaSuccess) {
        e = m->scan_state.reserve(sizeof(unsigned long long) * aica::scan_lookback_words(m->n_cells));
        what = "scan state";
    }
    if (e == cudaSuccess) e = cudaMemset(m->scan_state.p, 0, m->scan_state.bytes);
    if (e != cudaSuccess) {
        aica_status s = e == cudaErrorMemoryAllocation ? AICA_ERR_OOM : AICA_ERR_CUDA;
        cuda_fail(e, what);
        aica_mesh_destroy(m);
        return s;
    }
    m->h_ctr.swap(h_ctr);
    m->h_rad.swap(h_rad);
    *out = m;
    return AICA_OK;
}

extern "C" void aica_mesh_destroy(aica_mesh *m) {
    if (!m) return;
    aica::DevBuf *bufs[] = {&m->tri_off, &m->tri, &m->tri_nbr, &m->vtx_off, &m->vtx, &m->edg_off, &m->edg, &m->ctr, &m->rad,
                            &m->lo, &m->hi, &m->org, &m->ntri, &m->orgk, &m->orgm, &m->orgm64, &m->cl_first, &m->cl_of, &m->cl_run_off, &m->cl_runs, &m->cl_full_off, &m->cl_full, &m->cl_box, &m->xlo, &m->flag_list, &m->tri32, &m->pl32, &m->tric, &m->orgf, &m->vtx32, &m->edg32, &m->ctr32, &m->rad32, &m->box32, &m->bkt_off, &m->bkt_cells, &m->nbr_off, &m->nbr, &m->dil_off,
                            &m->dil_ids, &m->ref_src, &m->ref_n, &m->ref_off, &m->ref_ids, &m->run_off, &m->runs, &m->xf_dev, &m->run_d, &m->work_off,
                            &m->work, &m->work_split, &m->proc_order, &m->cell_of, &m->order, &m->unsorted, &m->ucell,
                            &m->cell_off, &m->fill, &m->inv, &m->sph, &m->xloc, &m->xs64, &m->facc,
                            &m->vsorted, &m->acc, &m->flags, &m->params, &m->tmp, &m->scan_state};
    for (auto *b : bufs) b->release();
    for (auto *v : {&m->tev, &m->tfree})
        for (auto &p : *v) {
            cudaEventDestroy(p.first);
            cudaEventDestroy(p.second);
        }
    delete m;
}
