/*
 * CPU oracle for the AICA pair-force path.  TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow FP64 reference code written from the paper (Macpherson & Reese,
 * "Molecular dynamics in arbitrary geometries: parallel evaluation of pair
 * forces", arXiv cs/0702131).  Only the test suite, the package smoke check
 * and the CPU-baseline leg of the benchmark may load this library.  It shares
 * no code, header or table with the CUDA path.  Built with -ffp-contract=off
 * so every FP64 operation rounds exactly as written.
 *
 * Contents
 *   oracle_lj            all-pairs minimum-image Lennard-Jones sum (the plain
 *                        definition the method reaches, see §2.3)
 *   oracle_cell_pairs    brute-force cell-cell minimum distance between
 *                        triangulated polyhedra, all periodic images (§2.2,
 *                        App. A.1, with the exact-distance criterion), or the
 *                        paper's vertex-vertex distance
 *   oracle_cell_pairs_grid  the same pairs for all cells, candidates from a
 *                        bucket grid of cell centres (full-size lists)
 *   oracle_locate        point location by ray parity with a symbolic
 *                        perturbation tie-break, FP64 with an error filter;
 *                        uncertain cases are flagged for exact resolution
 *   oracle_aica_loop     the real-real and real-referred loops of §2.3 over
 *                        the oracle's own lists and binning
 *   oracle_lj_images     the LJ sum over the images of all molecules under
 *                        general referring transforms (§2.2.2)
 *   oracle_lj_cells      the same LJ sum by the textbook cubic-cell
 *                        algorithm of §2.1 (bins of side >= rc, 27-bin
 *                        stencil): the practical CPU baseline, not a pin
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ LJ pair */
/* The paper names Lennard-Jones molecules (§3) but prints no formula; the
 * 12-6 form, plain truncation at r < rc and Lorentz-Berthelot mixing are the
 * reading used throughout.  f is the force on the first molecule of the pair,
 * d = x_first - x_second. */
static void lj_pair(double r2, double eps_ab, double sig_ab, double *fscal, double *u)
{
    double s = (sig_ab * sig_ab) / r2;
    double s3 = s * s * s;
    double s6 = s3 * s3;
    *fscal = 24.0 * eps_ab * (2.0 * s6 - s3) / r2;
    *u = 4.0 * eps_ab * (s6 - s3);
}

static double min_image(double d, double L, int periodic)
{
    if (periodic) d -= L * nearbyint(d / L);
    return d;
}

/* Forces F[k] = sum_{l != k, r_kl < rc} f_kl for every k in idx (or all k when
 * idx is NULL), with Fabs[k] = sum_l |f_kl|.  ev7 gets U and the virial
 * W_ab = sum_pairs d_a f_b (xx, yy, zz, xy, xz, yz), each pair counted once
 * (half from each of its two molecules); abs2 gets sum_pairs |u| and
 * sum_pairs |r . f|, the scales of those sums.  count gets the number of (k, l)
 * ordered pairs within rc, i.e. twice the pair count when idx is NULL. */
void oracle_lj(int64_t n, const double *pos, const int32_t *species, int S,
               const double *eps, const double *sigma, double rc, const double *L,
               const int32_t *periodic, int shift, const int64_t *idx, int64_t nidx,
               double *F, double *Fabs, double *ev7, double *abs2, int64_t *count)
{
    double rc2 = rc * rc;
    double U = 0, wxx = 0, wyy = 0, wzz = 0, wxy = 0, wxz = 0, wyz = 0, Ua = 0, Va = 0;
    int64_t cnt = 0;
    int64_t m = idx ? nidx : n;
    (void)S;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : U, wxx, wyy, wzz, wxy, wxz, wyz, Ua, Va, cnt)
    for (int64_t t = 0; t < m; ++t) {
        int64_t k = idx ? idx[t] : t;
        double fx = 0, fy = 0, fz = 0, fa = 0;
        int a = species[k];
        for (int64_t l = 0; l < n; ++l) {
            if (l == k) continue;
            double dx = min_image(pos[3 * k + 0] - pos[3 * l + 0], L[0], periodic[0]);
            double dy = min_image(pos[3 * k + 1] - pos[3 * l + 1], L[1], periodic[1]);
            double dz = min_image(pos[3 * k + 2] - pos[3 * l + 2], L[2], periodic[2]);
            double r2 = (dx * dx + dy * dy) + dz * dz;
            if (!(r2 < rc2)) continue;
            int b = species[l];
            double eab = sqrt(eps[a] * eps[b]);
            double sab = 0.5 * (sigma[a] + sigma[b]);
            double fs, u;
            lj_pair(r2, eab, sab, &fs, &u);
            if (shift) {
                double fc, uc;
                lj_pair(rc2, eab, sab, &fc, &uc);
                u -= uc;
            }
            fx += fs * dx;
            fy += fs * dy;
            fz += fs * dz;
            fa += fabs(fs) * sqrt(r2);
            U += 0.5 * u;
            Ua += 0.5 * fabs(u);
            Va += 0.5 * fabs(fs) * r2;
            wxx += 0.5 * dx * (fs * dx);
            wyy += 0.5 * dy * (fs * dy);
            wzz += 0.5 * dz * (fs * dz);
            wxy += 0.5 * dx * (fs * dy);
            wxz += 0.5 * dx * (fs * dz);
            wyz += 0.5 * dy * (fs * dz);
            cnt += 1;
        }
        F[3 * t + 0] = fx;
        F[3 * t + 1] = fy;
        F[3 * t + 2] = fz;
        Fabs[t] = fa;
    }
    ev7[0] = U;
    ev7[1] = wxx; ev7[2] = wyy; ev7[3] = wzz;
    ev7[4] = wxy; ev7[5] = wxz; ev7[6] = wyz;
    abs2[0] = Ua;
    abs2[1] = Va;
    *count = cnt;
}

/* ------------------------------------------------- cell-cell min distance */
typedef struct { double x, y, z; } v3;

static v3 ld(const double *p) { v3 r = {p[0], p[1], p[2]}; return r; }
static v3 ldsh(const double *p, v3 s) { v3 r = {p[0] + s.x, p[1] + s.y, p[2] + s.z}; return r; }
static v3 sub(v3 a, v3 b) { v3 r = {a.x - b.x, a.y - b.y, a.z - b.z}; return r; }
static v3 add(v3 a, v3 b) { v3 r = {a.x + b.x, a.y + b.y, a.z + b.z}; return r; }
static v3 scl(v3 a, double s) { v3 r = {a.x * s, a.y * s, a.z * s}; return r; }
static double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static v3 cross(v3 a, v3 b)
{
    v3 r = {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
    return r;
}

/* squared distance from p to the closed segment [a, b] */
static double d2_point_seg(v3 p, v3 a, v3 b)
{
    v3 ab = sub(b, a);
    double t = dot(sub(p, a), ab) / dot(ab, ab);
    if (t < 0) t = 0;
    if (t > 1) t = 1;
    v3 q = add(a, scl(ab, t));
    v3 d = sub(p, q);
    return dot(d, d);
}

/* squared distance from p to the closed triangle abc: the orthogonal
 * projection when it falls inside, otherwise the nearest edge */
static double d2_point_tri(v3 p, v3 a, v3 b, v3 c)
{
    v3 nrm = cross(sub(b, a), sub(c, a));
    double s0 = dot(cross(sub(b, a), sub(p, a)), nrm);
    double s1 = dot(cross(sub(c, b), sub(p, b)), nrm);
    double s2 = dot(cross(sub(a, c), sub(p, c)), nrm);
    if (s0 >= 0 && s1 >= 0 && s2 >= 0) {
        double h = dot(sub(p, a), nrm);
        return h * h / dot(nrm, nrm);
    }
    double d = d2_point_seg(p, a, b);
    double e = d2_point_seg(p, b, c);
    double f = d2_point_seg(p, c, a);
    if (e < d) d = e;
    if (f < d) d = f;
    return d;
}

/* squared distance between closed segments [p0,p1] and [q0,q1]: either an
 * endpoint is involved, or both closest points are interior and then they are
 * the feet of the common perpendicular of the two lines */
static double d2_seg_seg(v3 p0, v3 p1, v3 q0, v3 q1)
{
    double best = d2_point_seg(p0, q0, q1);
    double t;
    if ((t = d2_point_seg(p1, q0, q1)) < best) best = t;
    if ((t = d2_point_seg(q0, p0, p1)) < best) best = t;
    if ((t = d2_point_seg(q1, p0, p1)) < best) best = t;
    v3 u = sub(p1, p0), v = sub(q1, q0), w = sub(p0, q0);
    double a = dot(u, u), b = dot(u, v), c = dot(v, v), d = dot(u, w), e = dot(v, w);
    double D = a * c - b * b;
    if (D > 1e-14 * a * c) {
        double s = (b * e - c * d) / D;
        double r = (a * e - b * d) / D;
        if (s > 0 && s < 1 && r > 0 && r < 1) {
            v3 g = sub(add(w, scl(u, s)), scl(v, r));
            double gg = dot(g, g);
            if (gg < best) best = gg;
        }
    }
    return best;
}

/* Geometry of cell c: triangles tri[tri_off[c]..tri_off[c+1]) (9 doubles each),
 * vertices vtx[...] (3 doubles), edges edg[...] (6 doubles). */
typedef struct {
    const int64_t *tri_off, *vtx_off, *edg_off;
    const double *tri, *vtx, *edg;
} cellgeo;

/* min squared distance between cell A and cell B translated by sB */
static double cell_d2(const cellgeo *g, int64_t A, int64_t B, v3 sB)
{
    v3 z = {0, 0, 0};
    double best = INFINITY, t;
    for (int64_t i = g->vtx_off[A]; i < g->vtx_off[A + 1]; ++i) {
        v3 p = ld(g->vtx + 3 * i);
        for (int64_t j = g->tri_off[B]; j < g->tri_off[B + 1]; ++j) {
            const double *T = g->tri + 9 * j;
            if ((t = d2_point_tri(p, ldsh(T, sB), ldsh(T + 3, sB), ldsh(T + 6, sB))) < best) best = t;
        }
    }
    for (int64_t i = g->vtx_off[B]; i < g->vtx_off[B + 1]; ++i) {
        v3 p = ldsh(g->vtx + 3 * i, sB);
        for (int64_t j = g->tri_off[A]; j < g->tri_off[A + 1]; ++j) {
            const double *T = g->tri + 9 * j;
            if ((t = d2_point_tri(p, ldsh(T, z), ldsh(T + 3, z), ldsh(T + 6, z))) < best) best = t;
        }
    }
    for (int64_t i = g->edg_off[A]; i < g->edg_off[A + 1]; ++i) {
        const double *E = g->edg + 6 * i;
        v3 p0 = ld(E), p1 = ld(E + 3);
        for (int64_t j = g->edg_off[B]; j < g->edg_off[B + 1]; ++j) {
            const double *Q = g->edg + 6 * j;
            if ((t = d2_seg_seg(p0, p1, ldsh(Q, sB), ldsh(Q + 3, sB))) < best) best = t;
        }
    }
    return best;
}

/* For every query cell A = query[q]: every (B, n) with B a real cell, n an
 * integer image vector (|n_k| <= m[k]; n_k = 0 on non-periodic axes), (B, n)
 * != (A, 0), and min_dist^2(A, B + n.L) < thr^2.  Results per query are in
 * image-major (n lexicographic), then ascending B order, at most cap entries
 * per query (count[q] = -1 if the capacity is exceeded).
 *
 * When use_bound is set a pair is skipped without the exact test if
 * |ctr_A - ctr_B - n.L| - rad_A - rad_B > thr (1 + 1e-9) + 1e-9, where rad_c
 * bounds the distance from ctr_c to every vertex of c; every point of a cell
 * lies in the convex hull of its vertices, so this bound never drops a pair.
 * ties[q] counts decisions with |d^2 - thr^2| <= 1e-9 thr^2. */
/* The paper's own criterion (§2.2, App. A.1): the smallest distance between a
 * vertex of A and a vertex of B (B shifted by sB). */
static double cell_vertex_d2(const cellgeo *g, int64_t A, int64_t B, v3 sB)
{
    double best = INFINITY, t;
    for (int64_t i = g->vtx_off[A]; i < g->vtx_off[A + 1]; ++i) {
        v3 p = ld(g->vtx + 3 * i);
        for (int64_t j = g->vtx_off[B]; j < g->vtx_off[B + 1]; ++j) {
            v3 d = sub(p, ldsh(g->vtx + 3 * j, sB));
            if ((t = dot(d, d)) < best) best = t;
        }
    }
    return best;
}

/* vertex_only selects the vertex-vertex criterion instead of the exact
 * minimum distance between the polyhedra. */
void oracle_cell_pairs(const int64_t *tri_off, const double *tri, const int64_t *vtx_off,
                       const double *vtx, const int64_t *edg_off, const double *edg,
                       const double *ctr, const double *rad, int64_t n_cells,
                       const int64_t *query, int64_t nq, double thr, const int32_t *m,
                       const double *L, int use_bound, int vertex_only, int64_t cap, int64_t *count,
                       int32_t *outB, int32_t *outN, double *outD2, int64_t *ties)
{
    cellgeo g = {tri_off, vtx_off, edg_off, tri, vtx, edg};
    double thr2 = thr * thr;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < nq; ++q) {
        int64_t A = query[q];
        int64_t c = 0, nt = 0;
        for (int nx = -m[0]; nx <= m[0]; ++nx)
            for (int ny = -m[1]; ny <= m[1]; ++ny)
                for (int nz = -m[2]; nz <= m[2]; ++nz) {
                    v3 s = {nx * L[0], ny * L[1], nz * L[2]};
                    for (int64_t B = 0; B < n_cells; ++B) {
                        if (B == A && nx == 0 && ny == 0 && nz == 0) continue;
                        if (use_bound) {
                            v3 dc = {ctr[3 * A] - ctr[3 * B] - s.x, ctr[3 * A + 1] - ctr[3 * B + 1] - s.y,
                                     ctr[3 * A + 2] - ctr[3 * B + 2] - s.z};
                            double lb = sqrt(dot(dc, dc)) - rad[A] - rad[B];
                            if (lb > thr * (1 + 1e-9) + 1e-9) continue;
                        }
                        double d2 = vertex_only ? cell_vertex_d2(&g, A, B, s) : cell_d2(&g, A, B, s);
                        if (fabs(d2 - thr2) <= 1e-9 * thr2) nt++;
                        if (d2 < thr2) {
                            if (c < cap) {
                                int64_t o = q * cap + c;
                                outB[o] = (int32_t)B;
                                outN[3 * o + 0] = nx;
                                outN[3 * o + 1] = ny;
                                outN[3 * o + 2] = nz;
                                outD2[o] = d2;
                            }
                            c++;
                        }
                    }
                }
        count[q] = c > cap ? -1 : c;
        ties[q] = nt;
    }
}

/* The same pairs for every cell as query, found through a uniform grid of
 * buckets over the cell centres instead of a loop over all cells: for query
 * A and image n only the cells whose centre lies within thr + rad_A +
 * max(rad) of c_A - n.L can pass the sphere bound of oracle_cell_pairs, and
 * the buckets searched cover that ball, so the set of cells that reach the
 * bound and the exact distance is unchanged.  The same sphere bound and the
 * same distance then decide.  Only the entries the lists need are written:
 * n = 0 with B > A (the DIL) and every n != 0 (referred cells); ties are
 * counted over all pairs evaluated, as in oracle_cell_pairs.
 *   pass 0: count[q] = entries of query cell query[q]; pass 1: its entries
 *   at off[q] .. off[q] + count[q] (in search order; the caller sorts). */
void oracle_cell_pairs_grid(const int64_t *tri_off, const double *tri, const int64_t *vtx_off,
                            const double *vtx, const int64_t *edg_off, const double *edg,
                            const double *ctr, const double *rad, int64_t n_cells,
                            const int64_t *query, int64_t nq, double thr,
                            const int32_t *m, const double *L, int vertex_only, int pass,
                            const int64_t *bkt_off, const int64_t *bkt_cells, const int64_t *G,
                            const double *glo, double h, int64_t *count, const int64_t *off,
                            int32_t *outB, int8_t *outN, int64_t *ties)
{
    cellgeo g = {tri_off, vtx_off, edg_off, tri, vtx, edg};
    double thr2 = thr * thr, rmax = 0;
    for (int64_t B = 0; B < n_cells; ++B) rmax = rad[B] > rmax ? rad[B] : rmax;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < nq; ++q) {
        const int64_t A = query[q];
        int64_t c = 0, nt = 0;
        /* a cell passing the sphere bound lies within thr (1 + 1e-9) + 1e-9 +
         * rad_A + rad_B of c_A - n.L; the searched ball is wider by far more
         * than the rounding of the bucket arithmetic */
        double R = (thr + rad[A] + rmax) * (1 + 1e-6) + 1e-6;
        for (int nx = -m[0]; nx <= m[0]; ++nx)
            for (int ny = -m[1]; ny <= m[1]; ++ny)
                for (int nz = -m[2]; nz <= m[2]; ++nz) {
                    v3 s = {nx * L[0], ny * L[1], nz * L[2]};
                    double p[3] = {ctr[3 * A] - s.x, ctr[3 * A + 1] - s.y, ctr[3 * A + 2] - s.z};
                    int64_t b0[3], b1[3];
                    int empty = 0;
                    for (int d = 0; d < 3; ++d) {
                        double lo = floor((p[d] - R - glo[d]) / h), hi = floor((p[d] + R - glo[d]) / h);
                        if (hi < 0 || lo > (double)(G[d] - 1)) empty = 1;
                        b0[d] = lo < 0 ? 0 : (int64_t)lo;
                        b1[d] = hi > (double)(G[d] - 1) ? G[d] - 1 : (int64_t)hi;
                    }
                    if (empty) continue;
                    for (int64_t i = b0[0]; i <= b1[0]; ++i)
                        for (int64_t j = b0[1]; j <= b1[1]; ++j)
                            for (int64_t k = b0[2]; k <= b1[2]; ++k) {
                                int64_t bk = (i * G[1] + j) * G[2] + k;
                                for (int64_t t = bkt_off[bk]; t < bkt_off[bk + 1]; ++t) {
                                    int64_t B = bkt_cells[t];
                                    if (B == A && nx == 0 && ny == 0 && nz == 0) continue;
                                    v3 dc = {ctr[3 * A] - ctr[3 * B] - s.x, ctr[3 * A + 1] - ctr[3 * B + 1] - s.y,
                                             ctr[3 * A + 2] - ctr[3 * B + 2] - s.z};
                                    double lb = sqrt(dot(dc, dc)) - rad[A] - rad[B];
                                    if (lb > thr * (1 + 1e-9) + 1e-9) continue;
                                    double d2 = vertex_only ? cell_vertex_d2(&g, A, B, s) : cell_d2(&g, A, B, s);
                                    if (fabs(d2 - thr2) <= 1e-9 * thr2) nt++;
                                    if (!(d2 < thr2)) continue;
                                    int zero = nx == 0 && ny == 0 && nz == 0;
                                    if (zero && B < A) continue;
                                    if (pass == 1) {
                                        int64_t o = off[q] + c;
                                        outB[o] = (int32_t)B;
                                        outN[3 * o] = (int8_t)nx;
                                        outN[3 * o + 1] = (int8_t)ny;
                                        outN[3 * o + 2] = (int8_t)nz;
                                    }
                                    c++;
                                }
                            }
                }
        if (pass == 0) count[q] = c;
        ties[q] = nt;
    }
}

/* -------------------------------------------------------- point location */
/* Signs of orientation determinants for a point perturbed to
 * p_eps = p + (eps, eps^2, eps^3), eps -> 0+.  Each sign is computed in FP64
 * and accepted only when the value clears a bound (>= 30x the worst rounding
 * error); otherwise the caller reports the molecule as uncertain. */
#define UNCERTAIN 2

/* sign of (b_y - a_y)(p_z - a_z) - (b_z - a_z)(p_y - a_y) for p perturbed by
 * (eps^2, eps^3) in (y, z) */
static int orient2_yz_eps(v3 a, v3 b, v3 p)
{
    double t1 = (b.y - a.y) * (p.z - a.z), t2 = (b.z - a.z) * (p.y - a.y);
    double v = t1 - t2, bound = 1e-14 * (fabs(t1) + fabs(t2));
    if (v > bound) return 1;
    if (v < -bound) return -1;
    if (v != 0 || bound != 0) return UNCERTAIN;
    double cy = -(b.z - a.z), cz = (b.y - a.y);
    if (cy != 0) return cy > 0 ? 1 : -1;
    if (cz != 0) return cz > 0 ? 1 : -1;
    return 0;
}

/* sign of N_x with N = (b - a) x (c - a): the triangle's yz-projected area */
static int orient2_yz(v3 a, v3 b, v3 c)
{
    double t1 = (b.y - a.y) * (c.z - a.z), t2 = (b.z - a.z) * (c.y - a.y);
    double v = t1 - t2, bound = 1e-14 * (fabs(t1) + fabs(t2));
    if (v > bound) return 1;
    if (v < -bound) return -1;
    if (v == 0 && bound == 0) return 0;
    return UNCERTAIN;
}

/* sign of N . (p - a): the plane value of p (exact zero -> 0) */
static int orient3(v3 a, v3 b, v3 c, v3 p)
{
    v3 u = sub(b, a), w = sub(c, a), d = sub(p, a);
    double n1 = u.y * w.z, n2 = u.z * w.y, n3 = u.z * w.x, n4 = u.x * w.z, n5 = u.x * w.y, n6 = u.y * w.x;
    double Nx = n1 - n2, Ny = n3 - n4, Nz = n5 - n6;
    double v = (Nx * d.x + Ny * d.y) + Nz * d.z;
    double perm = (fabs(n1) + fabs(n2)) * fabs(d.x) + (fabs(n3) + fabs(n4)) * fabs(d.y) +
                  (fabs(n5) + fabs(n6)) * fabs(d.z);
    double bound = 1e-13 * perm;
    if (v > bound) return 1;
    if (v < -bound) return -1;
    if (v == 0 && perm == 0) return 0;
    return UNCERTAIN;
}

/* Parity of crossings of the ray p_eps + s x^, s > 0, with the closed
 * triangulated surface of a cell.  Returns 1 inside, 0 outside, UNCERTAIN. */
static int inside_ray(const double *tri, int64_t t0, int64_t t1, v3 p)
{
    int parity = 0;
    for (int64_t t = t0; t < t1; ++t) {
        v3 a = ld(tri + 9 * t), b = ld(tri + 9 * t + 3), c = ld(tri + 9 * t + 6);
        int nx = orient2_yz(a, b, c);
        if (nx == UNCERTAIN) return UNCERTAIN;
        if (nx == 0) continue; /* edge-on in the yz projection: never crossed */
        int e0 = orient2_yz_eps(a, b, p), e1 = orient2_yz_eps(b, c, p), e2 = orient2_yz_eps(c, a, p);
        if (e0 == UNCERTAIN || e1 == UNCERTAIN || e2 == UNCERTAIN) return UNCERTAIN;
        if (!(e0 == nx && e1 == nx && e2 == nx)) continue;
        int o = orient3(a, b, c, p);
        if (o == UNCERTAIN) return UNCERTAIN;
        if (o == 0) o = nx; /* on the plane: p_eps sits on the +N_x side */
        if (o == -nx) parity ^= 1;
    }
    return parity;
}

static double wrap_coord(double x, double L)
{
    if (x >= 0 && x < L) return x;
    x = x - L * floor(x / L);
    if (x >= L) x -= L;
    return x;
}

/* For each molecule: wrap periodic coordinates into [0, L), then test every
 * cell whose closed bounding box holds the point (the box test is exact and
 * only skips cells that cannot hold it).  cell[k] = the containing cell,
 * -1 if none, -2 if some decision was uncertain or two cells claimed it.
 * Candidate cells come from a uniform grid over the mesh bounding box. */
void oracle_locate(const int64_t *tri_off, const double *tri, const double *lo, const double *hi,
                   int64_t n_cells, const double *pos, int64_t n, const double *L,
                   const int32_t *periodic, int32_t *cell, double *wrapped)
{
    double glo[3] = {INFINITY, INFINITY, INFINITY}, ghi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t c = 0; c < n_cells; ++c)
        for (int d = 0; d < 3; ++d) {
            if (lo[3 * c + d] < glo[d]) glo[d] = lo[3 * c + d];
            if (hi[3 * c + d] > ghi[d]) ghi[d] = hi[3 * c + d];
        }
    int G[3];
    double h[3];
    double per = cbrt((double)n_cells);
    for (int d = 0; d < 3; ++d) {
        G[d] = (int)per + 1;
        h[d] = (ghi[d] - glo[d]) / G[d];
    }
    size_t nb = (size_t)G[0] * (size_t)G[1] * (size_t)G[2];
    int64_t *boff = calloc(nb + 1, sizeof(int64_t));
    for (int pass = 0; pass < 2; ++pass) {
        int64_t *fill = pass ? calloc(nb, sizeof(int64_t)) : NULL;
        int64_t *lst = pass ? malloc(sizeof(int64_t) * (boff[nb] ? boff[nb] : 1)) : NULL;
        for (int64_t c = 0; c < n_cells; ++c) {
            int i0[3], i1[3];
            for (int d = 0; d < 3; ++d) {
                i0[d] = (int)floor((lo[3 * c + d] - glo[d]) / h[d]) - 1;
                i1[d] = (int)floor((hi[3 * c + d] - glo[d]) / h[d]) + 1;
                if (i0[d] < 0) i0[d] = 0;
                if (i1[d] > G[d] - 1) i1[d] = G[d] - 1;
            }
            for (int x = i0[0]; x <= i1[0]; ++x)
                for (int y = i0[1]; y <= i1[1]; ++y)
                    for (int z = i0[2]; z <= i1[2]; ++z) {
                        int64_t b = ((int64_t)x * G[1] + y) * G[2] + z;
                        if (!pass) boff[b + 1]++;
                        else lst[boff[b] + fill[b]++] = c;
                    }
        }
        if (!pass) {
            for (size_t b = 0; b < nb; ++b) boff[b + 1] += boff[b];
        } else {
#pragma omp parallel for schedule(dynamic, 256)
            for (int64_t k = 0; k < n; ++k) {
                v3 p = ld(pos + 3 * k);
                double *pp = &p.x;
                for (int d = 0; d < 3; ++d)
                    if (periodic[d]) pp[d] = wrap_coord(pp[d], L[d]);
                wrapped[3 * k] = p.x;
                wrapped[3 * k + 1] = p.y;
                wrapped[3 * k + 2] = p.z;
                int ib[3], ok = 1;
                for (int d = 0; d < 3; ++d) {
                    ib[d] = (int)floor((pp[d] - glo[d]) / h[d]);
                    if (ib[d] < 0) ib[d] = 0;
                    if (ib[d] > G[d] - 1) ib[d] = G[d] - 1;
                    if (pp[d] < glo[d] || pp[d] > ghi[d]) ok = 0;
                }
                int32_t found = -1;
                if (ok) {
                    int64_t b = ((int64_t)ib[0] * G[1] + ib[1]) * G[2] + ib[2];
                    for (int64_t i = boff[b]; i < boff[b + 1]; ++i) {
                        int64_t c = lst[i];
                        if (p.x < lo[3 * c] || p.x > hi[3 * c] || p.y < lo[3 * c + 1] || p.y > hi[3 * c + 1] ||
                            p.z < lo[3 * c + 2] || p.z > hi[3 * c + 2])
                            continue;
                        int r = inside_ray(tri, tri_off[c], tri_off[c + 1], p);
                        if (r == UNCERTAIN) { found = -2; break; }
                        if (r == 1) {
                            if (found >= 0) { found = -2; break; }
                            found = (int32_t)c;
                        }
                    }
                }
                cell[k] = found;
            }
            free(fill);
            free(lst);
        }
    }
    free(boff);
}

/* ------------------------------------------------------------- AICA loops */
/* The force loops of §2.3 over the oracle's lists and binning, literally:
 * real-real (DIL cells with Newton's third law, then same-cell pairs with
 * sorted index k' > k) and real-referred (force on the real molecule only).
 * Molecules are in binned order: cell c holds xs[cell_off[c] .. cell_off[c+1]).
 * A referred molecule q of referred cell (src, n) sits at xs[q] + n.L.
 * counts: evaluated {same, dil, referred}, within rc {same, dil, referred}.
 * ev7: U and virial, real-referred pairs weighted 1/2 (each physical pair is
 * evaluated from both of its sides). */
static void pair_eval(const double *xp, const double *xq, const int32_t *n, const double *L, int a, int b,
                      const double *eps, const double *sigma, double rc2, int shift, double *fp, double *fq,
                      double w, double *ev, int64_t *within)
{
    double dx = (xp[0] - xq[0]) - L[0] * n[0];
    double dy = (xp[1] - xq[1]) - L[1] * n[1];
    double dz = (xp[2] - xq[2]) - L[2] * n[2];
    double r2 = (dx * dx + dy * dy) + dz * dz;
    if (!(r2 < rc2)) return;
    double eab = sqrt(eps[a] * eps[b]), sab = 0.5 * (sigma[a] + sigma[b]), fs, u;
    lj_pair(r2, eab, sab, &fs, &u);
    if (shift) {
        double fc, uc;
        lj_pair(rc2, eab, sab, &fc, &uc);
        u -= uc;
    }
    fp[0] += fs * dx; fp[1] += fs * dy; fp[2] += fs * dz;
    if (fq) { fq[0] -= fs * dx; fq[1] -= fs * dy; fq[2] -= fs * dz; }
    ev[0] += w * u;
    ev[1] += w * dx * (fs * dx); ev[2] += w * dy * (fs * dy); ev[3] += w * dz * (fs * dz);
    ev[4] += w * dx * (fs * dy); ev[5] += w * dx * (fs * dz); ev[6] += w * dy * (fs * dz);
    (*within)++;
}

void oracle_aica_loop(int64_t n_cells, const int64_t *cell_off, const double *xs, const int32_t *sp,
                      const double *eps, const double *sigma, double rc, const double *L, int shift,
                      const int64_t *dil_off, const int32_t *dil_ids, int64_t n_ref, const int32_t *ref_src,
                      const int32_t *ref_n, const int64_t *ref_off, const int32_t *ref_ids, double *F,
                      double *ev7, int64_t *counts)
{
    double rc2 = rc * rc;
    int32_t zero[3] = {0, 0, 0};
    memset(ev7, 0, 7 * sizeof(double));
    memset(counts, 0, 6 * sizeof(int64_t));
    /* real-real */
    for (int64_t I = 0; I < n_cells; ++I) {
        for (int64_t k = cell_off[I]; k < cell_off[I + 1]; ++k) {
            for (int64_t e = dil_off[I]; e < dil_off[I + 1]; ++e) {
                int64_t J = dil_ids[e];
                for (int64_t l = cell_off[J]; l < cell_off[J + 1]; ++l) {
                    counts[1]++;
                    pair_eval(xs + 3 * k, xs + 3 * l, zero, L, sp[k], sp[l], eps, sigma, rc2, shift, F + 3 * k,
                              F + 3 * l, 1.0, ev7, &counts[4]);
                }
            }
            for (int64_t k2 = cell_off[I]; k2 < cell_off[I + 1]; ++k2) {
                if (!(k2 > k)) continue;
                counts[0]++;
                pair_eval(xs + 3 * k, xs + 3 * k2, zero, L, sp[k], sp[k2], eps, sigma, rc2, shift, F + 3 * k,
                          F + 3 * k2, 1.0, ev7, &counts[3]);
            }
        }
    }
    /* real-referred */
    for (int64_t M = 0; M < n_ref; ++M) {
        int64_t c = ref_src[M];
        for (int64_t q = cell_off[c]; q < cell_off[c + 1]; ++q) {
            for (int64_t e = ref_off[M]; e < ref_off[M + 1]; ++e) {
                int64_t N = ref_ids[e];
                for (int64_t p = cell_off[N]; p < cell_off[N + 1]; ++p) {
                    counts[2]++;
                    pair_eval(xs + 3 * p, xs + 3 * q, ref_n + 3 * M, L, sp[p], sp[q], eps, sigma, rc2, shift,
                              F + 3 * p, NULL, 0.5, ev7, &counts[5]);
                }
            }
        }
    }
}

/* ------------------------------------------------ cubic-cell baseline (§2.1) */
/* The conventional cell algorithm the paper starts from: the box is cut into
 * cubic bins of side >= rc, and every molecule meets the molecules of its own
 * and the 26 surrounding bins (periodic wrap; a bin met twice through a narrow
 * axis is visited once).  The pair arithmetic is oracle_lj's, so forces equal
 * it up to summation order and counts equal it exactly.  On non-periodic axes
 * the bins span the molecules' extent. */
void oracle_lj_cells(int64_t n, const double *pos, const int32_t *species, const double *eps,
                     const double *sigma, double rc, const double *L, const int32_t *periodic, int shift,
                     double *F, double *Fabs, double *ev7, double *abs2, int64_t *count)
{
    double rc2 = rc * rc, lo[3], side[3];
    int64_t nb[3];
    for (int d = 0; d < 3; ++d) {
        double a = 0, b = L[d];
        if (!periodic[d]) {
            a = INFINITY; b = -INFINITY;
            for (int64_t k = 0; k < n; ++k) { a = fmin(a, pos[3 * k + d]); b = fmax(b, pos[3 * k + d]); }
            if (n == 0) { a = 0; b = 1; }
        }
        lo[d] = a;
        nb[d] = (int64_t)floor((b - a) / rc);
        if (nb[d] < 1) nb[d] = 1;
        side[d] = (b - a) / (double)nb[d];
        if (!periodic[d]) side[d] *= 1.0 + 1e-12;
    }
    int64_t B = nb[0] * nb[1] * nb[2];
    int64_t *bin = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *start = (int64_t *)calloc((size_t)B + 1, sizeof(int64_t));
    int64_t *sorted = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t k = 0; k < n; ++k) {
        int64_t c[3];
        for (int d = 0; d < 3; ++d) {
            double x = pos[3 * k + d];
            if (periodic[d]) x -= L[d] * floor(x / L[d]);
            c[d] = (int64_t)floor((x - lo[d]) / side[d]);
            if (c[d] < 0) c[d] = 0;
            if (c[d] >= nb[d]) c[d] = nb[d] - 1;
        }
        bin[k] = (c[0] * nb[1] + c[1]) * nb[2] + c[2];
        start[bin[k] + 1]++;
    }
    for (int64_t b = 0; b < B; ++b) start[b + 1] += start[b];
    {
        int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(B > 0 ? B : 1));
        memcpy(fill, start, sizeof(int64_t) * (size_t)B);
        for (int64_t k = 0; k < n; ++k) sorted[fill[bin[k]]++] = k;
        free(fill);
    }
    double U = 0, wxx = 0, wyy = 0, wzz = 0, wxy = 0, wxz = 0, wyz = 0, Ua = 0, Va = 0;
    int64_t cnt = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : U, wxx, wyy, wzz, wxy, wxz, wyz, Ua, Va, cnt)
    for (int64_t k = 0; k < n; ++k) {
        int64_t b = bin[k];
        int64_t c[3] = {b / (nb[1] * nb[2]), (b / nb[2]) % nb[1], b % nb[2]};
        int64_t seen[27];
        int ns = 0;
        double fx = 0, fy = 0, fz = 0, fa = 0;
        int a = species[k];
        for (int ox = -1; ox <= 1; ++ox)
            for (int oy = -1; oy <= 1; ++oy)
                for (int oz = -1; oz <= 1; ++oz) {
                    int64_t q[3] = {c[0] + ox, c[1] + oy, c[2] + oz}, ok = 1;
                    for (int d = 0; d < 3; ++d) {
                        if (q[d] < 0 || q[d] >= nb[d]) {
                            if (!periodic[d]) ok = 0;
                            else q[d] = (q[d] + nb[d]) % nb[d];
                        }
                    }
                    if (!ok) continue;
                    int64_t nbin = (q[0] * nb[1] + q[1]) * nb[2] + q[2], dup = 0;
                    for (int i = 0; i < ns; ++i) dup |= seen[i] == nbin;
                    if (dup) continue;
                    seen[ns++] = nbin;
                    for (int64_t s = start[nbin]; s < start[nbin + 1]; ++s) {
                        int64_t l = sorted[s];
                        if (l == k) continue;
                        double dx = min_image(pos[3 * k + 0] - pos[3 * l + 0], L[0], periodic[0]);
                        double dy = min_image(pos[3 * k + 1] - pos[3 * l + 1], L[1], periodic[1]);
                        double dz = min_image(pos[3 * k + 2] - pos[3 * l + 2], L[2], periodic[2]);
                        double r2 = (dx * dx + dy * dy) + dz * dz;
                        if (!(r2 < rc2)) continue;
                        int bs = species[l];
                        double eab = sqrt(eps[a] * eps[bs]);
                        double sab = 0.5 * (sigma[a] + sigma[bs]);
                        double fs, u;
                        lj_pair(r2, eab, sab, &fs, &u);
                        if (shift) {
                            double fc, uc;
                            lj_pair(rc2, eab, sab, &fc, &uc);
                            u -= uc;
                        }
                        fx += fs * dx;
                        fy += fs * dy;
                        fz += fs * dz;
                        fa += fabs(fs) * sqrt(r2);
                        U += 0.5 * u;
                        Ua += 0.5 * fabs(u);
                        Va += 0.5 * fabs(fs) * r2;
                        wxx += 0.5 * dx * (fs * dx);
                        wyy += 0.5 * dy * (fs * dy);
                        wzz += 0.5 * dz * (fs * dz);
                        wxy += 0.5 * dx * (fs * dy);
                        wxz += 0.5 * dx * (fs * dz);
                        wyz += 0.5 * dy * (fs * dz);
                        cnt += 1;
                    }
                }
        F[3 * k + 0] = fx;
        F[3 * k + 1] = fy;
        F[3 * k + 2] = fz;
        Fabs[k] = fa;
    }
    ev7[0] = U;
    ev7[1] = wxx; ev7[2] = wyy; ev7[3] = wzz;
    ev7[4] = wxy; ev7[5] = wxz; ev7[6] = wyz;
    abs2[0] = Ua;
    abs2[1] = Va;
    *count = cnt;
    free(bin);
    free(start);
    free(sorted);
}

/* ------------------------------------------- general referring transforms */
/* Forces on every molecule from all images P' = y_t + R_t . P of all
 * molecules under the given transforms (§2.2.2, Eq. P' = y + R.P), the
 * identity among them (its own image excluded): F_k = sum_t sum_l f(x_k -
 * (y_t + R_t x_l)) over r < rc.  Each physical pair appears once from each
 * side, so U and W take half of every term.  R row-major [nt*9], y [nt*3].
 * With idx only the rows k = idx[0..nidx) are computed (into F[row]). */
void oracle_lj_images(int64_t n, const double *pos, const int32_t *species, const double *eps,
                      const double *sigma, double rc, int64_t nt, const double *R, const double *y,
                      int shift, const int64_t *idx, int64_t nidx, double *F, double *Fabs, double *ev7,
                      double *abs2, int64_t *count)
{
    double rc2 = rc * rc;
    double U = 0, wxx = 0, wyy = 0, wzz = 0, wxy = 0, wxz = 0, wyz = 0, Ua = 0, Va = 0;
    int64_t cnt = 0;
    int64_t rows = idx ? nidx : n;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : U, wxx, wyy, wzz, wxy, wxz, wyz, Ua, Va, cnt)
    for (int64_t row = 0; row < rows; ++row) {
        int64_t k = idx ? idx[row] : row;
        double fx = 0, fy = 0, fz = 0, fa = 0;
        int a = species[k];
        for (int64_t t = 0; t < nt; ++t) {
            const double *Rt = R + 9 * t, *yt = y + 3 * t;
            int ident = Rt[0] == 1 && Rt[4] == 1 && Rt[8] == 1 && Rt[1] == 0 && Rt[2] == 0 && Rt[3] == 0 &&
                        Rt[5] == 0 && Rt[6] == 0 && Rt[7] == 0 && yt[0] == 0 && yt[1] == 0 && yt[2] == 0;
            for (int64_t l = 0; l < n; ++l) {
                if (ident && l == k) continue;
                const double *x = pos + 3 * l;
                double q0 = yt[0] + ((Rt[0] * x[0] + Rt[1] * x[1]) + Rt[2] * x[2]);
                double q1 = yt[1] + ((Rt[3] * x[0] + Rt[4] * x[1]) + Rt[5] * x[2]);
                double q2 = yt[2] + ((Rt[6] * x[0] + Rt[7] * x[1]) + Rt[8] * x[2]);
                double dx = pos[3 * k] - q0, dy = pos[3 * k + 1] - q1, dz = pos[3 * k + 2] - q2;
                double r2 = (dx * dx + dy * dy) + dz * dz;
                if (!(r2 < rc2)) continue;
                int b = species[l];
                double eab = sqrt(eps[a] * eps[b]);
                double sab = 0.5 * (sigma[a] + sigma[b]);
                double fs, u;
                lj_pair(r2, eab, sab, &fs, &u);
                if (shift) {
                    double fc, uc;
                    lj_pair(rc2, eab, sab, &fc, &uc);
                    u -= uc;
                }
                fx += fs * dx;
                fy += fs * dy;
                fz += fs * dz;
                fa += fabs(fs) * sqrt(r2);
                U += 0.5 * u;
                Ua += 0.5 * fabs(u);
                Va += 0.5 * fabs(fs) * r2;
                wxx += 0.5 * dx * (fs * dx);
                wyy += 0.5 * dy * (fs * dy);
                wzz += 0.5 * dz * (fs * dz);
                wxy += 0.5 * dx * (fs * dy);
                wxz += 0.5 * dx * (fs * dz);
                wyz += 0.5 * dy * (fs * dz);
                cnt += 1;
            }
        }
        F[3 * row + 0] = fx;
        F[3 * row + 1] = fy;
        F[3 * row + 2] = fz;
        Fabs[row] = fa;
    }
    ev7[0] = U;
    ev7[1] = wxx; ev7[2] = wyy; ev7[3] = wzz;
    ev7[4] = wxy; ev7[5] = wxz; ev7[6] = wyz;
    abs2[0] = Ua;
    abs2[1] = Va;
    *count = cnt;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
