// Internal state and helpers of the AICA library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/aica.h"

struct aica_mesh;

namespace aica {

// Per-cell limits of the list builder and binning kernels.
constexpr int kMaxTri = 32;
constexpr int kMaxVtx = 24;
constexpr int kMaxEdg = 48;
constexpr int kMaxSpecies = 8;
constexpr int kMaxClusterCells = 16;   // cells of one pair-kernel cluster (see mesh.cu)
// Bit of a binned molecule's species word (xloc.w) marking a molecule this
// portion does not own (a halo copy received from the processor that does).
constexpr int kGhostBit = kMaxSpecies;

// Device-side error flags (bitwise OR into mesh->d_flags[0]).
enum : unsigned {
    kFlagOutside = 1u,   // a molecule lies in no cell
    kFlagSpecies = 2u,   // a species index is out of range
    kFlagCapacity = 4u,  // a per-cell capacity of a kernel was exceeded
    kFlagTimeout = 8u,   // a bounded wait between blocks gave up
};

cudaError_t timing_begin(aica_mesh *m, cudaStream_t st, cudaEvent_t *stop);
cudaError_t timing_end(cudaEvent_t stop, cudaStream_t st);

// Thread-local last error message.
void set_error(const char *fmt, ...);
aica_status cuda_fail(cudaError_t e, const char *what);

// NVTX range over one C-ABI call (header-only NVTX v3: free unless a
// profiler is attached).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};
#define AICA_RANGE(name) aica::Range aica_range_(name)

#define AICA_CUDA(call)                                        \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return aica::cuda_fail(e_, #call); \
    } while (0)

// A device buffer that only grows.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaError_t reserve(size_t n) {
        if (n <= bytes) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        cudaError_t e = cudaMalloc(&p, n);
        if (e == cudaSuccess) bytes = n;
        return e;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    template <class T> T *as() const { return static_cast<T *>(p); }
};

// One work entry of the pair schedule: real cell I interacts with the
// molecules of cell j, translated by the image vector n.
struct WorkEntry {
    int32_t j;      // partner cell
    int32_t n;      // image vector, 3 x int8 packed (x in bits 0-7, y 8-15, z 16-23)
};

// One run of the FP32 kernel's schedule: partner cells j .. j + len - 1 (one
// contiguous range of binned molecules under one shift).
struct RunEntry {
    int32_t j;      // first partner cell
    int32_t n;      // image vector in bits 0-23 (as WorkEntry), len - 1 in bits 24-31
};

// One run of the FP32 cluster kernel's schedule: partner molecules of the
// cells c0 .. c0 + ncells - 1 (consecutive clusters under one image and one
// molecule frame), shifted into the owner cluster's frame by dh + dl (dh a
// multiple of 2^-qexp, exact in FP32; dl the FP32 remainder).
//   dh.w: c0 (int bits);  dl.w: ncells | (image n, 3 x 4-bit fields) << 12
struct ClRun {
    float4 dh, dl;
};

// A referring transform P' = y + R.P (§2.2.2), R row-major.
struct Xform {
    double R[9], y[3];
};
// Its device copy: FP64 for exact decisions, FP32 rotation for the FP32 path.
struct XfDev {
    double R[9], y[3];
    float Rf[9], pad[3];
};
constexpr int kMaxXf = 64;          // transforms reaching the domain (identity included)

__host__ __device__ inline int32_t pack_n(int nx, int ny, int nz) {
    return (int32_t)(((unsigned)(nx & 0xff)) | ((unsigned)(ny & 0xff) << 8) | ((unsigned)(nz & 0xff) << 16));
}
__host__ __device__ inline int unpack_n(int32_t p, int axis) {
    return (int)(signed char)((p >> (8 * axis)) & 0xff);
}

}  // namespace aica

struct aica_mesh;
namespace aica {
aica_status build_transform_referral(aica_mesh *m, double thr, cudaStream_t st);
}

struct aica_mesh {
    int device = 0;
    int64_t n_cells = 0, n_points = 0;
    aica_box box{};
    int max_tri = 0, max_vtx = 0, max_edg = 0;

    // Geometry (device, FP64).  Triangles are oriented out of their cell.
    aica::DevBuf tri_off, tri, vtx_off, vtx, edg_off, edg;  // int32 offsets, double coords
    aica::DevBuf tri_nbr;                                    // [T] int32 cell across each triangle (-1: boundary)
    aica::DevBuf ctr, rad, lo, hi, org;                      // [C*3] vertex mean, [C] radius, AABB, origin
    aica::DevBuf ntri;                                       // [C] int32 triangle count | convex << 16
    aica::DevBuf box32;                                      // [C*6] float local AABB (lo, hi), rounded outward
    // FP32 copies local to each cell's dyadic origin org_c = orgk_c * 2^-10.
    aica::DevBuf orgk;                                       // [C*3] int32
    // Molecule frame: binned FP32 coordinates are local to orgm_c * 2^-10, an
    // origin shared by runs of consecutive cells (see mesh.cu).
    aica::DevBuf orgm, orgm64;                               // [C*3] int32, double (exact)
    double max_mlocal = 0;                                   // largest |cell bound - its molecule origin|
    // Clusters (runs of consecutive cells, see mesh.cu): first cell of each
    // cluster [n_cl+1] and cluster of each cell [C].
    int64_t n_cl = 0;
    int max_cl_cells = 0;
    aica::DevBuf cl_first, cl_of;
    aica::DevBuf tri32, vtx32, edg32, ctr32;                 // float, minus org_c
    aica::DevBuf pl32;                  // float4 per triangle: plane n / |n|_1, offset (local to org_c)
    aica::DevBuf tric;                  // int2 per cell: first triangle, count | convex bit
    aica::DevBuf orgf;                  // float x3 per cell: orgk * 2^-10 (exact when org32)
    aica::DevBuf rad32;                                      // [C] float, rad rounded up
    double max_local = 0;                                    // largest |local coordinate|
    bool org32 = false;                 // every cell origin (orgk * 2^-10) exact in FP32 (|orgk| < 2^24)
    // Point-location grid: cells whose bounding box meets a bucket.
    int G[3] = {1, 1, 1};
    double glo[3] = {0, 0, 0}, gh[3] = {1, 1, 1};
    aica::DevBuf bkt_off, bkt_cells;
    aica::DevBuf nbr_off, nbr;                               // face neighbours of each cell (CSR)
    // Host copies kept for the list builder's bucket grid.
    std::vector<double> h_ctr, h_rad;

    // Interaction lists (device), valid when built.
    bool built = false;
    double rc = 0, skin = 0;
    int criterion = 0;                       // aica_dil_criterion of the built lists
    int64_t n_dil = 0, n_ref = 0, n_ref_ids = 0, n_ties = 0, n_work = 0, n_runs = 0;
    aica::DevBuf dil_off, dil_ids, ref_src, ref_n, ref_off, ref_ids;   // int32 (ref_n: 3 int32)
    aica::DevBuf run_off, runs;              // [C+1] int32 first run of each cell; RunEntry
    // Cluster schedule of the FP32 box-periodic kernel: per cluster A the runs
    // of partner clusters B > A (any image) and B = A (lexicographically
    // positive image), as RunEntry over clusters; and the full (symmetric)
    // partner list of every cluster for the FP64 refinement, one entry per
    // (partner cluster, image).
    aica::DevBuf cl_run_off, cl_runs, cl_full_off, cl_full;
    aica::DevBuf cl_box;                     // [n_cl][2] float4: molecule box of each cluster (last FP32 call)
    int64_t n_cl_runs = -1, n_cl_full = 0;    // n_cl_runs < 0: no cluster schedule
    int qexp = 20;                           // cluster kernel: hi parts are multiples of 2^-qexp
    // General referring transforms (empty: box periodicity).  With them the
    // image field of work entries and runs holds a transform index (0 = none).
    std::vector<aica::Xform> xf_gen;         // generators given by the caller
    int n_xf = 0;                            // transforms of the built lists (identity first)
    aica::DevBuf xf_dev;                     // [n_xf] XfDev
    aica::DevBuf run_d;                      // [runs] float4 shift of each run in I's molecule frame
    aica::DevBuf work_off, work;             // [C+1] int32 first entry of each cell; WorkEntry (partner, image)
    aica::DevBuf work_split;                 // [C] int32: first periodic-image entry of each cell
    aica::DevBuf proc_order;                 // [C] int32: cell processing order (spatially local)

    // Binned molecules (device), valid when binned.
    bool binned = false;
    int64_t n_mol = 0, cap_mol = 0;
    aica::DevBuf cell_of, order, cell_off, fill, xloc, xs64, inv;
    aica::DevBuf xlo;                        // [n] float4: x - o_m - xloc (FP32 remainder), binned order
    aica::DevBuf flag_list;                  // FP32 forces: [0] count, [1..] binned molecules to refine in FP64
    double refine_tol = 1e-5;                // FP32 forces: refine a molecule whose error bound exceeds this (0: off)
    bool count_evaluated = true;             // aica_forces: count the AICA-evaluated pairs (an extra pass)
    int fp32_kernel = 0;                     // 0: cluster kernel when available, 1: the cell kernel
    int64_t n_owned = -1;                    // portion mode: molecules [0, n_owned) are owned, the rest halo (-1: all)
    bool ghosts = false;                     // the last binning marked halo molecules
    int64_t n_refined = 0;                   // molecules the last FP32 call recomputed (host copy on demand)
    aica::DevBuf unsorted;                   // [n] binned slots before the in-cell sort (cells of a few molecules)
    aica::DevBuf ucell;                      // [n] the cell of each slot of `unsorted`
    int max_species = -1;                    // from the last checked binning, -1 if unknown
    aica::DevBuf sph;                        // [C] float4 molecule bounding sphere per cell (local frame)
    aica::DevBuf miss;                       // molecules whose previous cell no longer holds them
    aica::DevBuf scan_state;                 // single-pass scan of the cell counts: ticket, epoch, tile words
    int64_t n_mol_prev = -1;                 // molecule count of the previous binning
    bool hint_valid = false;                 // cell_of holds that binning (a search hint)
    aica::DevBuf facc, vsorted;              // force / gradient accumulators in binned order
    aica::DevBuf acc;                        // double[16] sums + uint64 counters
    aica::DevBuf flags;                      // unsigned[4] device error flags
    aica::DevBuf params;                     // per-call parameter block
    aica::DevBuf tmp;                        // general scratch

    bool deferred = false;
    int64_t launches = 0;
    bool timing = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> tev;   // recorded, not yet taken
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> tfree;  // reusable
};
