// General referring transforms (§2.2.2): periodic boundaries given as
// transforms P' = y + R.P (rotation and translation), their compositions,
// and the referred cells and pair schedule they induce.
//
// The box case (integer image vectors n, R = I) is handled by the list
// builder on the GPU.  With general transforms the referral is built on the
// host once per list build (App. A: allowed to be expensive, done once):
//   1. the closure of the generators and their inverses (compositions of at
//      most kXfDepth, duplicates removed by comparing R and y: App. A.2's
//      duplicate check), keeping the transforms that bring an image of the
//      domain within rc + skin of it;
//   2. for every kept transform T and cell c, the real cells J within
//      rc + skin of T(c) (exact minimum distance between the polyhedra in
//      FP64): referred cell (c, T) with its list (§2.2.1);
//   3. the schedule of each real cell I: its DIL, then every referred cell
//      whose list holds I, evaluated from I's side only (§2.3: real-referred
//      pairs act on the real molecule; each physical pair is met from both
//      of its sides, so energy and virial take half of each).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "aica_internal.cuh"
#include "geom.cuh"

namespace aica {
namespace {

constexpr int kXfDepth = 6;

Xform xf_identity() {
    Xform t{};
    t.R[0] = t.R[4] = t.R[8] = 1.0;
    return t;
}

// a after b: R = Ra Rb, y = ya + Ra yb
Xform xf_compose(const Xform &a, const Xform &b) {
    Xform c{};
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += a.R[3 * i + k] * b.R[3 * k + j];
            c.R[3 * i + j] = s;
        }
        double s = a.y[i];
        for (int k = 0; k < 3; ++k) s += a.R[3 * i + k] * b.y[k];
        c.y[i] = s;
    }
    return c;
}

Xform xf_inverse(const Xform &a) {
    Xform c{};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) c.R[3 * i + j] = a.R[3 * j + i];
    for (int i = 0; i < 3; ++i) {
        double s = 0;
        for (int k = 0; k < 3; ++k) s -= c.R[3 * i + k] * a.y[k];
        c.y[i] = s;
    }
    return c;
}

bool xf_same(const Xform &a, const Xform &b, double ytol) {
    for (int i = 0; i < 9; ++i)
        if (fabs(a.R[i] - b.R[i]) > 1e-9) return false;
    for (int i = 0; i < 3; ++i)
        if (fabs(a.y[i] - b.y[i]) > ytol) return false;
    return true;
}

// y + R p in the operation order of the oracle's image sum
V3<double> xf_apply(const Xform &t, V3<double> p) {
    return {t.y[0] + ((t.R[0] * p.x + t.R[1] * p.y) + t.R[2] * p.z),
            t.y[1] + ((t.R[3] * p.x + t.R[4] * p.y) + t.R[5] * p.z),
            t.y[2] + ((t.R[6] * p.x + t.R[7] * p.y) + t.R[8] * p.z)};
}

template <class T> void download(std::vector<T> &h, const DevBuf &d, size_t n) {
    h.resize(n);
    if (n) cudaMemcpy(h.data(), d.p, sizeof(T) * n, cudaMemcpyDeviceToHost);
}

}  // namespace

// Host side of the list build with general transforms; called by
// aica_build_interaction_list_ex after the device builder produced the DIL
// schedule (no periodic axes).  Replaces the schedule, its runs and the
// referred-cell lists.
aica_status build_transform_referral(aica_mesh *m, double thr, cudaStream_t st) {
    AICA_CUDA(cudaStreamSynchronize(st));
    const int C = (int)m->n_cells;
    std::vector<int> tri_off, vtx_off, edg_off, work_off;
    std::vector<double> tri, vtx, edg, om;
    std::vector<WorkEntry> work;
    download(tri_off, m->tri_off, C + 1);
    download(vtx_off, m->vtx_off, C + 1);
    download(edg_off, m->edg_off, C + 1);
    download(tri, m->tri, 9 * (size_t)tri_off[C]);
    download(vtx, m->vtx, 3 * (size_t)vtx_off[C]);
    download(edg, m->edg, 6 * (size_t)edg_off[C]);
    download(om, m->orgm64, 3 * (size_t)C);
    download(work_off, m->work_off, C + 1);
    download(work, m->work, (size_t)work_off[C]);
    AICA_CUDA(cudaGetLastError());
    const std::vector<double> &ctr = m->h_ctr, &rad = m->h_rad;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY}, rmax = 0;
    for (int c = 0; c < C; ++c) {
        rmax = std::max(rmax, rad[c]);
        for (int d = 0; d < 3; ++d) {
            lo[d] = std::min(lo[d], ctr[3 * c + d] - rad[c]);
            hi[d] = std::max(hi[d], ctr[3 * c + d] + rad[c]);
        }
    }
    double span = 0;
    for (int d = 0; d < 3; ++d) span = std::max(span, hi[d] - lo[d]);
    const double ytol = 1e-9 * std::max(1.0, span);

    // 1. closure of the generators, kept when an image of the domain comes within thr
    std::vector<Xform> base;
    for (const Xform &g : m->xf_gen)
        for (const Xform &h : {g, xf_inverse(g)}) {
            bool dup = false;
            for (const Xform &b : base) dup |= xf_same(h, b, ytol);
            if (!dup) base.push_back(h);
        }
    std::vector<Xform> all{xf_identity()}, frontier{xf_identity()};
    for (int depth = 0; depth < kXfDepth && !frontier.empty(); ++depth) {
        std::vector<Xform> next;
        for (const Xform &t : frontier)
            for (const Xform &g : base) {
                Xform u = xf_compose(g, t);
                bool dup = false;
                for (const Xform &v : all) dup |= xf_same(u, v, ytol);
                if (!dup) {
                    all.push_back(u);
                    next.push_back(u);
                }
            }
        frontier.swap(next);
        if (all.size() > 4096) break;
    }
    std::vector<Xform> xf{xf_identity()};
    for (size_t i = 1; i < all.size(); ++i) {
        // the image of the domain's bounding box (its 8 corners) against the box grown by thr
        double tlo[3] = {INFINITY, INFINITY, INFINITY}, thi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int k = 0; k < 8; ++k) {
            V3<double> p = {(k & 1) ? hi[0] : lo[0], (k & 2) ? hi[1] : lo[1], (k & 4) ? hi[2] : lo[2]};
            V3<double> q = xf_apply(all[i], p);
            const double qq[3] = {q.x, q.y, q.z};
            for (int d = 0; d < 3; ++d) {
                tlo[d] = std::min(tlo[d], qq[d]);
                thi[d] = std::max(thi[d], qq[d]);
            }
        }
        bool near = true;
        for (int d = 0; d < 3; ++d) near &= tlo[d] <= hi[d] + thr && thi[d] >= lo[d] - thr;
        if (near) xf.push_back(all[i]);
    }
    if ((int)xf.size() > kMaxXf) {
        set_error("aica_build_interaction_list: %d referring transforms reach the domain (at most %d)",
                  (int)xf.size(), kMaxXf);
        return AICA_ERR_CAPACITY;
    }

    // 2. referred cells: (c, t) with the real cells J within thr of T_t(c)
    double gh = std::max(thr, 2.0 * rmax);
    int G[3];
    for (int d = 0; d < 3; ++d) G[d] = std::max(1, std::min(512, (int)ceil((hi[d] - lo[d]) / gh)));
    std::vector<int> boff(G[0] * G[1] * G[2] + 1, 0), bcell(C);
    auto bidx = [&](double v, int d) { return std::min(G[d] - 1, std::max(0, (int)floor((v - lo[d]) / gh))); };
    for (int c = 0; c < C; ++c)
        boff[1 + (bidx(ctr[3 * c], 0) * G[1] + bidx(ctr[3 * c + 1], 1)) * G[2] + bidx(ctr[3 * c + 2], 2)]++;
    for (size_t b = 1; b < boff.size(); ++b) boff[b] += boff[b - 1];
    {
        std::vector<int> fill(boff.begin(), boff.end() - 1);
        for (int c = 0; c < C; ++c)
            bcell[fill[(bidx(ctr[3 * c], 0) * G[1] + bidx(ctr[3 * c + 1], 1)) * G[2] + bidx(ctr[3 * c + 2], 2)]++] = c;
    }
    const double thr2 = thr * thr;
    auto ld = [](const double *p) { return V3<double>{p[0], p[1], p[2]}; };
    struct Ref { int src, t; std::vector<int> ids; };
    std::vector<Ref> refs;
    std::vector<std::vector<std::pair<int, int>>> sched(C);   // per real cell: (t, source)
    int64_t ties = 0;
    std::vector<V3<double>> tv, ttri, tedg;
    for (int t = 1; t < (int)xf.size(); ++t)
        for (int c = 0; c < C; ++c) {
            const V3<double> pc = xf_apply(xf[t], ld(&ctr[3 * c]));
            const double R = thr + rad[c] + rmax;
            int b0[3], b1[3];
            const double pp[3] = {pc.x, pc.y, pc.z};
            bool out = false;
            for (int d = 0; d < 3; ++d) {
                if (pp[d] + R < lo[d] || pp[d] - R > hi[d]) out = true;
                b0[d] = bidx(pp[d] - R, d);
                b1[d] = bidx(pp[d] + R, d);
            }
            if (out) continue;
            tv.clear(); ttri.clear(); tedg.clear();
            for (int i = vtx_off[c]; i < vtx_off[c + 1]; ++i) tv.push_back(xf_apply(xf[t], ld(&vtx[3 * i])));
            for (int i = 3 * tri_off[c]; i < 3 * tri_off[c + 1]; ++i) ttri.push_back(xf_apply(xf[t], ld(&tri[3 * i])));
            for (int i = 2 * edg_off[c]; i < 2 * edg_off[c + 1]; ++i) tedg.push_back(xf_apply(xf[t], ld(&edg[3 * i])));
            Ref ref{c, t, {}};
            for (int bx = b0[0]; bx <= b1[0]; ++bx)
                for (int by = b0[1]; by <= b1[1]; ++by)
                    for (int bz = b0[2]; bz <= b1[2]; ++bz) {
                        const int b = (bx * G[1] + by) * G[2] + bz;
                        for (int q = boff[b]; q < boff[b + 1]; ++q) {
                            const int J = bcell[q];
                            const V3<double> dc = ld(&ctr[3 * J]) - pc;
                            const double lb = sqrt(dot3(dc, dc)) - rad[c] - rad[J];
                            if (lb > thr * (1 + 1e-9) + 1e-9) continue;
                            double d2 = INFINITY;
                            for (const V3<double> &p : tv)
                                for (int k = tri_off[J]; k < tri_off[J + 1]; ++k)
                                    d2 = std::min(d2, d2_point_triangle(p, ld(&tri[9 * k]), ld(&tri[9 * k + 3]),
                                                                        ld(&tri[9 * k + 6])));
                            for (int i = vtx_off[J]; i < vtx_off[J + 1]; ++i)
                                for (size_t k = 0; k < ttri.size(); k += 3)
                                    d2 = std::min(d2, d2_point_triangle(ld(&vtx[3 * i]), ttri[k], ttri[k + 1], ttri[k + 2]));
                            for (int i = edg_off[J]; i < edg_off[J + 1]; ++i)
                                for (size_t k = 0; k < tedg.size(); k += 2)
                                    d2 = std::min(d2, d2_segment_segment(ld(&edg[6 * i]), ld(&edg[6 * i + 3]), tedg[k],
                                                                         tedg[k + 1]));
                            if (fabs(d2 - thr2) <= 1e-9 * thr2) ++ties;
                            if (d2 < thr2) ref.ids.push_back(J);
                        }
                    }
            if (!ref.ids.empty()) {
                std::sort(ref.ids.begin(), ref.ids.end());
                for (int J : ref.ids) sched[J].push_back({t, c});
                refs.push_back(std::move(ref));
            }
        }

    // 3. schedule: DIL entries (image 0), then referred entries (transform id in the image field)
    std::vector<int> nwo(C + 1, 0);
    std::vector<WorkEntry> nw;
    nw.reserve(work.size() + refs.size() * 8);
    for (int I = 0; I < C; ++I) {
        nwo[I] = (int)nw.size();
        for (int e = work_off[I]; e < work_off[I + 1]; ++e) nw.push_back(work[e]);
        std::sort(sched[I].begin(), sched[I].end());
        for (auto &p : sched[I]) nw.push_back(WorkEntry{p.second, p.first});
    }
    nwo[C] = (int)nw.size();
    // runs: consecutive partners under one transform and one molecule-frame origin; their shift
    // o = R_t o_J + y_t - o_I in I's molecule frame (FP64, then FP32)
    std::vector<int> ro(C + 1, 0);
    std::vector<RunEntry> runs;
    std::vector<float4> rd;
    for (int I = 0; I < C; ++I) {
        ro[I] = (int)runs.size();
        for (int e = nwo[I]; e < nwo[I + 1]; ++e) {
            const WorkEntry w = nw[e];
            bool cont = false;
            if (e > nwo[I] && !runs.empty()) {
                const RunEntry &r = runs.back();
                const int len = (int)((unsigned)r.n >> 24) + 1;
                cont = w.j == r.j + len && w.n == (r.n & 0xffffff) && len < 256 && om[3 * w.j] == om[3 * r.j] &&
                       om[3 * w.j + 1] == om[3 * r.j + 1] && om[3 * w.j + 2] == om[3 * r.j + 2];
            }
            if (cont) {
                runs.back().n += 1 << 24;
            } else {
                runs.push_back(RunEntry{w.j, w.n & 0xffffff});
                const V3<double> q = xf_apply(xf[w.n], ld(&om[3 * w.j]));
                rd.push_back(make_float4((float)(q.x - om[3 * I]), (float)(q.y - om[3 * I + 1]),
                                         (float)(q.z - om[3 * I + 2]), 0.f));
            }
        }
    }
    ro[C] = (int)runs.size();
    // referred-cell lists (image field: transform id, 0, 0)
    std::vector<int> rsrc, rn, roff{0}, rids;
    for (const Ref &r : refs) {
        rsrc.push_back(r.src);
        rn.push_back(r.t); rn.push_back(0); rn.push_back(0);
        rids.insert(rids.end(), r.ids.begin(), r.ids.end());
        roff.push_back((int)rids.size());
    }
    std::vector<XfDev> tab(xf.size());
    for (size_t t = 0; t < xf.size(); ++t) {
        for (int i = 0; i < 9; ++i) {
            tab[t].R[i] = xf[t].R[i];
            tab[t].Rf[i] = (float)xf[t].R[i];
        }
        for (int i = 0; i < 3; ++i) tab[t].y[i] = xf[t].y[i];
    }
    auto up = [&](DevBuf &d, const void *h, size_t bytes) -> cudaError_t {
        cudaError_t e = d.reserve(std::max<size_t>(bytes, 16));
        if (e == cudaSuccess && bytes) e = cudaMemcpy(d.p, h, bytes, cudaMemcpyHostToDevice);
        return e;
    };
    AICA_CUDA(up(m->work_off, nwo.data(), sizeof(int) * nwo.size()));
    AICA_CUDA(up(m->work, nw.data(), sizeof(WorkEntry) * nw.size()));
    AICA_CUDA(up(m->run_off, ro.data(), sizeof(int) * ro.size()));
    AICA_CUDA(up(m->runs, runs.data(), sizeof(RunEntry) * runs.size()));
    AICA_CUDA(up(m->run_d, rd.data(), sizeof(float4) * rd.size()));
    AICA_CUDA(up(m->ref_src, rsrc.data(), sizeof(int) * rsrc.size()));
    AICA_CUDA(up(m->ref_n, rn.data(), sizeof(int) * rn.size()));
    AICA_CUDA(up(m->ref_off, roff.data(), sizeof(int) * roff.size()));
    AICA_CUDA(up(m->ref_ids, rids.data(), sizeof(int) * rids.size()));
    AICA_CUDA(up(m->xf_dev, tab.data(), sizeof(XfDev) * tab.size()));
    m->n_work = (int64_t)nw.size();
    m->n_runs = (int64_t)runs.size();
    m->n_ref = (int64_t)refs.size();
    m->n_ref_ids = (int64_t)rids.size();
    m->n_ties += ties;
    m->n_xf = (int)xf.size();
    return AICA_OK;
}

}  // namespace aica

using namespace aica;

extern "C" aica_status aica_coupling_transform(const double *n_alpha, const double *c_alpha, const double *n_beta,
                                               const double *c_beta, double *R, double *y) {
    if (!n_alpha || !c_alpha || !n_beta || !c_beta || !R || !y) {
        set_error("aica_coupling_transform: NULL argument");
        return AICA_ERR_INVALID_ARG;
    }
    double a[3], b[3], la = 0, lb = 0;
    for (int d = 0; d < 3; ++d) { la += n_alpha[d] * n_alpha[d]; lb += n_beta[d] * n_beta[d]; }
    if (!(la > 0) || !(lb > 0)) { set_error("aica_coupling_transform: zero normal"); return AICA_ERR_INVALID_ARG; }
    for (int d = 0; d < 3; ++d) { a[d] = n_alpha[d] / sqrt(la); b[d] = n_beta[d] / sqrt(lb); }
    const double c = a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
    if (c > 1.0 - 1e-12) {
        set_error("aica_coupling_transform: parallel face normals (rotation axis undefined)");
        return AICA_ERR_INVALID_ARG;
    }
    // R = -(a.b) I + (1 + a.b) u u + a b - b a,  u = (a x b) / |a x b|  (§2.2.2)
    double u[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
    const double lu = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const bool anti = c < -1.0 + 1e-12;     // antiparallel normals: R = I
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double r = anti ? (i == j ? 1.0 : 0.0)
                            : -c * (i == j ? 1.0 : 0.0) + (1.0 + c) * (u[i] / lu) * (u[j] / lu) + a[i] * b[j] -
                                  b[i] * a[j];
            R[3 * i + j] = r;
        }
    for (int i = 0; i < 3; ++i) y[i] = c_beta[i] - (R[3 * i] * c_alpha[0] + R[3 * i + 1] * c_alpha[1] + R[3 * i + 2] * c_alpha[2]);
    return AICA_OK;
}

extern "C" aica_status aica_mesh_set_transforms(aica_mesh *m, int32_t n, const double *R, const double *y) {
    if (!m || n < 0 || (n > 0 && (!R || !y))) { set_error("aica_mesh_set_transforms: bad arguments"); return AICA_ERR_INVALID_ARG; }
    if (n > 0 && (m->box.periodic[0] || m->box.periodic[1] || m->box.periodic[2])) {
        set_error("aica_mesh_set_transforms: the box must have no periodic axis (give its translations as transforms)");
        return AICA_ERR_INVALID_ARG;
    }
    std::vector<Xform> g;
    for (int k = 0; k < n; ++k) {
        Xform t{};
        memcpy(t.R, R + 9 * k, sizeof(t.R));
        memcpy(t.y, y + 3 * k, sizeof(t.y));
        // rotation: R^T R = I and det R = +1 to 1e-9
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double s = 0;
                for (int q = 0; q < 3; ++q) s += t.R[3 * q + i] * t.R[3 * q + j];
                if (!(fabs(s - (i == j ? 1.0 : 0.0)) <= 1e-9)) {
                    set_error("aica_mesh_set_transforms: transform %d is not a rotation", k);
                    return AICA_ERR_INVALID_ARG;
                }
            }
        const double det = t.R[0] * (t.R[4] * t.R[8] - t.R[5] * t.R[7]) - t.R[1] * (t.R[3] * t.R[8] - t.R[5] * t.R[6]) +
                           t.R[2] * (t.R[3] * t.R[7] - t.R[4] * t.R[6]);
        if (!(fabs(det - 1.0) <= 1e-9) || !isfinite(t.y[0] + t.y[1] + t.y[2])) {
            set_error("aica_mesh_set_transforms: transform %d is not a proper rotation with a finite shift", k);
            return AICA_ERR_INVALID_ARG;
        }
        g.push_back(t);
    }
    m->xf_gen.swap(g);
    m->built = false;
    return AICA_OK;
}
