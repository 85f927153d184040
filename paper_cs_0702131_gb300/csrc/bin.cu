// Molecule-to-cell binning (step a4; §2.2 requires each molecule's cell to be
// known at every step).
//
// Kernels
//   bin_locate   thread per molecule: wrap periodic coordinates, look up the
//                point-location bucket, test candidate cells until one holds
//                p + (e, e^2, e^3): tetrahedra by their four face planes,
//                other (star-shaped) cells by the cone from the vertex mean
//                through each face triangle.  FP32 filter on cell-local
//                coordinates, FP64 and exact slow paths (predicates.cuh).
//   bin_locate_hint / bin_locate_miss   when the same molecules were binned
//                before: test each molecule's previous cell, collect the
//                ones that left it, then search those among the face
//                neighbours of the previous cell and finally the grid.  The
//                previous cell is only a search order: the test is exact.
//   bin_count    warp-aggregated histogram of cells (match_any + one atomic)
//   (scan)       cell offsets
//   bin_scatter  warp-aggregated slot claims
//   bin_fixup    per-cell insertion sort by original index: the binned order
//                is the stable counting sort by (cell, original index)
//   bin_gather   sorted FP64 positions and float4 cell-local coordinates with
//                the species in .w (the pair kernels' input layout)
#include <math.h>

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
    const float *tri32, *ctr32;
    const double *tri, *ctr;
    float max_local;
    int *cell_of;
    unsigned *flags;
};

__device__ __forceinline__ double wrap_coord(double x, double L) {
    if (x >= 0.0 && x < L) return x;
    x = __dsub_rn(x, __dmul_rn(L, floor(__ddiv_rn(x, L))));
    if (x >= L) x = __dsub_rn(x, L);
    return x;
}

__device__ __forceinline__ float3 ld3f(const float *p) { return make_float3(p[0], p[1], p[2]); }

// sign of O(a, b, c, p + (e, e^2, e^3)); FP32 filter then exact slow path
__device__ __forceinline__ int orient(float3 a, float3 b, float3 c, float3 q, float scale, const double *a64,
                                      const double *b64, const double *c64, const double *p64) {
    int s = orient_f32(a, b, c, q, scale);
    if (s) return s;
    return orient_sos_slow(a64, b64, c64, p64);
}

__device__ bool cell_contains(const BinArgs &a, int c, float3 q, const double *p64) {
    int t0 = a.tri_off[c], nt = a.ntri[c];
    float scale = fmaxf(a.max_local, fmaxf(fabsf(q.x), fmaxf(fabsf(q.y), fabsf(q.z))));
    if (nt == 4) {   // tetrahedron: convex, inside iff behind all four faces
        for (int t = t0; t < t0 + 4; ++t) {
            const float *T = a.tri32 + 9 * t;
            const double *D = a.tri + 9 * t;
            if (orient(ld3f(T), ld3f(T + 3), ld3f(T + 6), q, scale, D, D + 3, D + 6, p64) > 0) return false;
        }
        return true;
    }
    float3 C = ld3f(a.ctr32 + 3 * c);
    const double *C64 = a.ctr + 3 * c;
    for (int t = t0; t < t0 + nt; ++t) {
        const float *T = a.tri32 + 9 * t;
        const double *D = a.tri + 9 * t;
        float3 x0 = ld3f(T), x1 = ld3f(T + 3), x2 = ld3f(T + 6);
        // p in the cone from C through triangle (x0, x1, x2)?
        if (orient(C, x0, x1, q, scale, C64, D, D + 3, p64) < 0) continue;
        if (orient(C, x1, x2, q, scale, C64, D + 3, D + 6, p64) < 0) continue;
        if (orient(C, x2, x0, q, scale, C64, D + 6, D, p64) < 0) continue;
        return orient(x0, x1, x2, q, scale, D, D + 3, D + 6, p64) < 0;
    }
    return false;
}

// p relative to the dyadic origin c_k * 2^-10 of cell c, in FP32 (one rounding)
__device__ __forceinline__ float3 local_to(const BinArgs &a, const double *p, int c) {
    return make_float3((float)(p[0] - a.orgk[3 * c] * (1.0 / 1024.0)), (float)(p[1] - a.orgk[3 * c + 1] * (1.0 / 1024.0)),
                       (float)(p[2] - a.orgk[3 * c + 2] * (1.0 / 1024.0)));
}

__device__ __forceinline__ void wrapped_position(const BinArgs &a, int64_t k, double *p, bool &ok) {
    ok = true;
    for (int d = 0; d < 3; ++d) {
        p[d] = a.pos[3 * k + d];
        if (a.per[d]) p[d] = wrap_coord(p[d], a.L[d]);
        if (!(p[d] >= a.glo[d] && p[d] <= a.ghi[d])) ok = false;
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
    if (k >= a.n) return;
    double p[3];
    bool ok;
    wrapped_position(a, k, p, ok);
    const int found = ok ? grid_search(a, p, -1) : -1;
    a.cell_of[k] = found;
    if (found < 0) atomicOr(a.flags, kFlagOutside);
}

// Previous cell first; molecules that left it go to the miss list.
__global__ void __launch_bounds__(256) bin_locate_hint(BinArgs a) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool miss = false;
    if (k < a.n) {
        double p[3];
        bool ok;
        wrapped_position(a, k, p, ok);
        const int h = a.hint[k];
        if (ok && h >= 0 && cell_contains(a, h, local_to(a, p, h), p)) {
            a.cell_of[k] = h;
        } else if (ok) {
            miss = true;
        } else {
            a.cell_of[k] = -1;
            atomicOr(a.flags, kFlagOutside);
        }
    }
    const unsigned bal = __ballot_sync(0xffffffffu, miss);
    const int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == 0 && bal) base = atomicAdd(a.miss, __popc(bal));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (miss) a.miss[1 + base + __popc(bal & ((1u << lane) - 1u))] = (int)k;
}

// Molecules that left their previous cell: one warp per molecule, lanes test
// the previous cell's face neighbours in parallel, then the cells of the
// molecule's bucket.  Exact predicates make at most one cell hold the point.
__global__ void __launch_bounds__(256) bin_locate_miss(BinArgs a) {
    const int lane = threadIdx.x & 31;
    const int nm = a.miss[0];
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nm; i += nw) {
        const int k = a.miss[1 + i];
        double p[3];
        bool ok;
        wrapped_position(a, k, p, ok);
        const int h = a.hint[k];
        int found = -1;
        if (h >= 0) {
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
            if (found < 0) atomicOr(a.flags, kFlagOutside);
        }
    }
}

__global__ void __launch_bounds__(256) bin_count(const int *cell_of, int64_t n, int *cnt) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int c = k < n ? cell_of[k] : -1;
    unsigned same = __match_any_sync(0xffffffffu, c);
    int lane = threadIdx.x & 31;
    if (c >= 0 && lane == __ffs(same) - 1) atomicAdd(cnt + c, __popc(same));
}

__global__ void __launch_bounds__(256) bin_scatter(const int *cell_of, int64_t n, const int *cell_off, int *fill,
                                                   int *order) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int c = k < n ? cell_of[k] : -1;
    unsigned same = __match_any_sync(0xffffffffu, c);
    int lane = threadIdx.x & 31;
    int leader = __ffs(same) - 1;
    int base = 0;
    if (c >= 0 && lane == leader) base = atomicAdd(fill + c, __popc(same));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (c >= 0) order[cell_off[c] + base + __popc(same & ((1u << lane) - 1u))] = (int)k;
}

__global__ void __launch_bounds__(256) bin_fixup(const int *cell_off, int C, int *order) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    int s = cell_off[c], e = cell_off[c + 1];
    for (int i = s + 1; i < e; ++i) {
        int v = order[i], j = i - 1;
        while (j >= s && order[j] > v) {
            order[j + 1] = order[j];
            --j;
        }
        order[j + 1] = v;
    }
}

__global__ void __launch_bounds__(256) bin_gather(BinArgs a, const int *order, const int *cell_off, int C,
                                                  double *xs64, float4 *xloc, int *inv) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int sp = 0;
    if (s < cell_off[C]) {
        int k = order[s];
        inv[k] = (int)s;
        sp = a.species[k];
    int c = a.cell_of[k];
    double p[3];
    for (int d = 0; d < 3; ++d) {
        p[d] = a.pos[3 * (int64_t)k + d];
        if (a.per[d]) p[d] = wrap_coord(p[d], a.L[d]);
        xs64[3 * s + d] = p[d];
    }
    xloc[s] = make_float4((float)(p[0] - a.orgk[3 * c] * (1.0 / 1024.0)), (float)(p[1] - a.orgk[3 * c + 1] * (1.0 / 1024.0)),
                          (float)(p[2] - a.orgk[3 * c + 2] * (1.0 / 1024.0)), __int_as_float(sp & (kMaxSpecies - 1)));
    }
    // largest species index (flags[1]) and out-of-range species (flags[0])
    unsigned bad = (unsigned)sp >= (unsigned)kMaxSpecies;
    int mx = __reduce_max_sync(0xffffffffu, sp < 0 ? kMaxSpecies : sp);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(a.flags, kFlagSpecies);
    if ((threadIdx.x & 31) == 0) atomicMax((int *)a.flags + 1, mx);
}

// Per-cell bounding sphere of its molecules in the cell's local frame:
// centre = mean, radius = max distance, rounded up.  Used by the pair kernels
// to skip cell pairs and partner molecules that cannot be within rc.
__global__ void __launch_bounds__(256) bin_spheres(const int *cell_off, int C, const float4 *xloc, float4 *sph) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    int s = cell_off[c], e = cell_off[c + 1];
    float cx = 0.f, cy = 0.f, cz = 0.f;
    for (int i = s; i < e; ++i) {
        float4 x = xloc[i];
        cx += x.x; cy += x.y; cz += x.z;
    }
    float inv = e > s ? 1.f / (float)(e - s) : 0.f;
    cx *= inv; cy *= inv; cz *= inv;
    float r2 = 0.f;
    for (int i = s; i < e; ++i) {
        float4 x = xloc[i];
        float dx = x.x - cx, dy = x.y - cy, dz = x.z - cz;
        r2 = fmaxf(r2, dx * dx + dy * dy + dz * dz);
    }
    sph[c] = make_float4(cx, cy, cz, sqrtf(r2) * (1.f + 1e-5f) + 1e-5f);
}

}  // namespace
}  // namespace aica

using namespace aica;

extern "C" aica_status aica_bin_molecules(aica_mesh *m, const double *pos, const int32_t *species, int64_t n,
                                          int32_t *cell_of, int32_t *order, int32_t *cell_off, void *stream) {
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
        AICA_CUDA(m->xloc.reserve(sizeof(float4) * cap));
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
    AICA_CUDA(m->scratch_i32.reserve(sizeof(int) * (scan_work_items(C) + 8)));
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
    a.tri32 = m->tri32.as<float>();
    a.ctr32 = m->ctr32.as<float>();
    a.tri = m->tri.as<double>();
    a.ctr = m->ctr.as<double>();
    a.max_local = (float)(m->max_local * (1 + 1e-6));
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
    AICA_CUDA(cudaMemsetAsync(m->flags.p, 0, 16, st));
    AICA_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (C + 1), st));
    unsigned nb = (unsigned)((n + 255) / 256);
    if (n > 0) {
        if (a.hint) {
            AICA_CUDA(cudaMemsetAsync(m->miss.p, 0, sizeof(int), st));
            bin_locate_hint<<<nb, 256, 0, st>>>(a);
            bin_locate_miss<<<152 * 4, 256, 0, st>>>(a);
            m->launches += 2;
        } else {
            bin_locate<<<nb, 256, 0, st>>>(a);
            m->launches += 1;
        }
        bin_count<<<nb, 256, 0, st>>>(a.cell_of, n, cnt);
        m->launches += 1;
    }
    m->launches += exclusive_scan<int, int>(cnt, C, off, m->scratch_i32.as<int>(), st);
    AICA_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (C + 1), st));
    if (n > 0) {
        bin_scatter<<<nb, 256, 0, st>>>(a.cell_of, n, off, cnt, m->order.as<int>());
        bin_fixup<<<(C + 255) / 256, 256, 0, st>>>(off, C, m->order.as<int>());
        AICA_CUDA(cudaMemsetAsync(m->inv.p, 0xff, sizeof(int) * n, st));
        bin_gather<<<nb, 256, 0, st>>>(a, m->order.as<int>(), off, C, m->xs64.as<double>(), m->xloc.as<float4>(),
                                       m->inv.as<int>());
        m->launches += 3;
    }
    bin_spheres<<<(C + 255) / 256, 256, 0, st>>>(off, C, m->xloc.as<float4>(), m->sph.as<float4>());
    m->launches += 1;
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
    AICA_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (C + 1), st));
    const unsigned nb = (unsigned)((n + 255) / 256);
    if (n > 0) bin_count<<<nb, 256, 0, st>>>(cell_of, n, cnt);
    exclusive_scan<int, int>(cnt, C, cell_off, work, st);
    AICA_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (C + 1), st));
    if (n > 0) {
        bin_scatter<<<nb, 256, 0, st>>>(cell_of, n, cell_off, cnt, order);
        bin_fixup<<<(C + 255) / 256, 256, 0, st>>>(cell_off, C, order);
    }
    AICA_CUDA(cudaGetLastError());
    return AICA_OK;
}
