/*
 * aica.h -- C ABI of the GB300 (sm_103a) AICA pair-force library.
 *
 * AICA, the Arbitrary Interacting Cells Algorithm (Macpherson & Reese,
 * arXiv cs/0702131), evaluates short-range pair forces between molecules
 * binned into the cells of an arbitrary polyhedral mesh: each cell carries a
 * direct interaction list (DIL) of the cells it must interact with (§2.2),
 * built once because the mesh is static, and periodic boundaries are handled
 * by "referred" copies of cells and molecules (§2.2.1).  On one GPU only
 * periodic referral exists.  Every compute step runs in hand-written CUDA
 * kernels; there is no CPU fallback.
 *
 * Conventions
 *   - All functions return an aica_status; on failure aica_last_error() gives
 *     a thread-local message.  No exception crosses this boundary.
 *   - "host" pointers are read during the call and may be freed afterwards.
 *     "device" pointers are CUDA global memory owned by the caller; the
 *     library reads inputs and writes outputs on `stream` (a cudaStream_t, or
 *     NULL for the legacy default stream) and returns before the work ends
 *     unless stated otherwise.
 *   - The library owns the mesh, the interaction lists, the binned molecule
 *     state and its workspaces (device memory allocated on the device that is
 *     current at aica_mesh_create).  A mesh handle is not thread-safe.
 *   - Reduced LJ units; rc and skin are absolute lengths.
 */
#ifndef AICA_H
#define AICA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct aica_mesh aica_mesh; /* opaque, library-owned */

typedef enum {
    AICA_OK = 0,
    AICA_ERR_INVALID_ARG = 1,  /* NULL pointer, negative size, unsupported option   */
    AICA_ERR_BAD_MESH = 2,     /* open cell, inverted or non-star cell, bad index     */
    AICA_ERR_OUTSIDE_MESH = 3, /* a molecule lies in no cell (see aica_bin_molecules) */
    AICA_ERR_NOT_BUILT = 4,    /* forces requested before lists or binning            */
    AICA_ERR_CAPACITY = 5,     /* a fixed per-cell limit of the kernels is exceeded   */
    AICA_ERR_CUDA = 6,         /* a CUDA runtime call failed                          */
    AICA_ERR_OOM = 7           /* device allocation failed                            */
} aica_status;

typedef enum { AICA_FP32 = 0, AICA_FP64 = 1 } aica_precision;

/* Translational periodicity of the domain: an axis with periodic[k] != 0
 * repeats with period L[k]; the mesh must fill [0, L[k]] along it. */
typedef struct {
    double L[3];
    int32_t periodic[3];
} aica_box;

/* Lennard-Jones 12-6 parameters.  The paper names LJ molecules (§3) without
 * printing the potential; this library uses u(r) = 4 eps ((s/r)^12 - (s/r)^6)
 * truncated at r < rc, with Lorentz-Berthelot mixing eps_ab = sqrt(eps_a
 * eps_b), sigma_ab = (sigma_a + sigma_b) / 2 and one absolute rc for every
 * pair (the largest cut-off builds the lists, App. A). */
typedef struct {
    int32_t n_species;   /* S: 1..8                                         */
    const double *eps;   /* host [S]                                       */
    const double *sigma; /* host [S]                                       */
    int32_t shift;       /* nonzero: subtract u(rc) from each pair's energy */
} aica_lj;

typedef struct {
    int64_t n_cells;
    int64_t n_dil;      /* entries of all direct interaction lists         */
    int64_t n_ref;      /* referred cells                                  */
    int64_t n_ref_ids;  /* entries of all referred-cell real-cell lists    */
    int64_t n_ties;     /* cell-pair decisions within 1e-9 (rc+skin)^2     */
    double rc, skin;
    int32_t criterion;  /* aica_dil_criterion the lists were built with     */
} aica_list_info;

/* Create a mesh from a face-based description (OpenFOAM style).  Defines the
 * cells whose DILs §2.2 builds; the cell numbering is the caller's and is
 * what "j > i" in App. A.1 refers to.
 *   points        host [n_points*3] FP64 vertex coordinates
 *   face_offsets  host [n_faces+1]; face f has vertices
 *                 face_vertices[face_offsets[f] .. face_offsets[f+1])
 *   owner         host [n_faces] cell on the side the right-handed normal
 *                 leaves; neighbour host [n_faces] the other cell or -1
 *   box           host; periodic axes of the domain
 * Faces are split into fans from their lowest vertex id, so both cells of a
 * face see the same triangles.  Each cell must be closed and star-shaped
 * about the mean of its vertices (every tetrahedron from that point to a
 * face triangle has positive volume), else AICA_ERR_BAD_MESH.  At most 32
 * triangles, 24 vertices and 48 edges per cell (AICA_ERR_CAPACITY).
 * Synchronous; allocates device memory on the current device. */
aica_status aica_mesh_create(const double *points, int64_t n_points, const int64_t *face_offsets,
                             const int64_t *face_vertices, int64_t n_faces, const int64_t *owner,
                             const int64_t *neighbour, int64_t n_cells, const aica_box *box,
                             aica_mesh **out);

/* Free every library allocation of the mesh.  NULL is ignored. */
void aica_mesh_destroy(aica_mesh *mesh);

/* Build the interaction lists (§2.2, App. A): for cells i < j, j joins DIL(i)
 * iff the minimum distance between the two closed triangulated polyhedra is
 * below rc + skin (vertex-triangle and edge-edge distances, decided in FP64;
 * this replaces the paper's vertex-vertex search and so has no twisted-mesh
 * error).  Periodic referred cells (§2.2.1) are every (c, n), n a nonzero
 * integer image vector, with at least one real cell J within rc + skin of
 * c + n.L; each keeps the ascending list of such J.  Requires rc > 0,
 * skin >= 0 and rc + skin < L/2 on periodic axes.  Runs on `stream` and
 * synchronizes it before returning (the list sizes are needed on the host). */
aica_status aica_build_interaction_list(aica_mesh *mesh, double rc, double skin, void *stream);

/* General periodic boundaries (§2.2.2): the referring transforms P' = y + R.P
 * that carry the domain onto its periodic images (rotation R, row-major
 * [n*9], and shift y [n*3], host arrays; one per coupled boundary, its
 * inverse is implied).  They replace the box periodicity: the mesh's box must
 * have no periodic axis (translations are given as transforms with R = I).
 * The next list build enumerates their compositions (duplicates removed by
 * comparing R and y, App. A.2), keeps those that bring an image of the
 * domain within rc + skin, and builds the referred cells (source cell,
 * transform) with their real cells by the exact minimum distance (on the
 * host, once).  Real-referred pairs are evaluated from the real side only,
 * as §2.3 does (each physical pair is met from both sides; energy and virial
 * take half of each, and the referred pair counts count both sides).  In the
 * referred-cell lists of aica_get_lists, ref_n holds (transform index, 0, 0).
 * Molecules must lie in the mesh (binning does not fold them through a
 * rotated boundary).  The adjoint supports box periodicity only.  Each R
 * must be a proper rotation (R^T R = I, det R = 1, to 1e-9), else
 * AICA_ERR_INVALID_ARG; n = 0 removes the transforms.  At most 64
 * transforms may reach the domain (AICA_ERR_CAPACITY at the list build). */
aica_status aica_mesh_set_transforms(aica_mesh *mesh, int32_t n, const double *R, const double *y);

/* The referring transform of a pair of coupled faces (§2.2.2, Eq. of
 * R_{alpha beta}): R turns -n_alpha into n_beta,
 *   R = -(a.b) I + (1 + a.b) u u + a b - b a,  u = (a x b) / |a x b|,
 * with a, b the unit face normals, and y = C_beta - R.C_alpha from the face
 * centres.  Antiparallel normals give R = I (a translation); parallel
 * normals leave the rotation axis undefined -> AICA_ERR_INVALID_ARG.  Host
 * arrays: n_alpha, c_alpha, n_beta, c_beta [3] in, R [9] (row-major), y [3]
 * out. */
aica_status aica_coupling_transform(const double *n_alpha, const double *c_alpha, const double *n_beta,
                                    const double *c_beta, double *R, double *y);

/* Criterion that lists a cell pair. */
typedef enum {
    AICA_DIL_MIN_DISTANCE = 0,   /* minimum distance between the polyhedra (default) */
    AICA_DIL_VERTEX = 1          /* the paper's own search (§2.2, App. A.1): some vertex
                                    of one cell within rc + skin of a vertex of the
                                    other; can miss pairs of twisted cells (§2.2) */
} aica_dil_criterion;

/* aica_build_interaction_list with a choice of criterion (same lists, same
 * arguments and behaviour for AICA_DIL_MIN_DISTANCE).  With AICA_DIL_VERTEX
 * the DILs and referred cells are those of the paper's vertex-vertex search,
 * decided in FP64 with the same tie report; aica_forces then evaluates the
 * pairs of those lists, which may omit pairs within rc (the twisted-mesh
 * error of §2.2, reduced by a skin: the paper's guard distance).  An unknown
 * criterion -> AICA_ERR_INVALID_ARG. */
aica_status aica_build_interaction_list_ex(aica_mesh *mesh, double rc, double skin,
                                           aica_dil_criterion criterion, void *stream);

/* Sizes of the current lists (host struct).  AICA_ERR_NOT_BUILT before a build. */
aica_status aica_get_list_info(const aica_mesh *mesh, aica_list_info *info);

/* Copy the lists to host buffers sized from aica_get_list_info:
 *   dil_off [n_cells+1], dil_ids [n_dil]      DIL(i) = dil_ids[dil_off[i]..dil_off[i+1]), ascending
 *   ref_src [n_ref], ref_n [n_ref*3]          referred cell m = source cell and image vector n
 *   ref_off [n_ref+1], ref_ids [n_ref_ids]    its real cells, ascending
 * Referred cells are sorted by (source, n) with n lexicographic.  Any
 * pointer may be NULL to skip that array.  Synchronous. */
aica_status aica_get_lists(const aica_mesh *mesh, int64_t *dil_off, int32_t *dil_ids, int32_t *ref_src,
                           int32_t *ref_n, int64_t *ref_off, int32_t *ref_ids);

/* Bin molecules into cells (§2.2: a molecule's cell must always be known).
 *   pos      device [n*3] FP64 positions; periodic coordinates are wrapped
 *            into [0, L) first
 *   species  device [n] int32 in [0, S) (checked by aica_forces)
 *   cell_of  device [n] out, optional: containing cell, -1 if none
 *   order    device [n] out, optional: order[s] = original index of binned
 *            slot s (stable counting sort by cell, then original index)
 *   cell_off device [n_cells+1] out, optional: cell c holds slots
 *            cell_off[c] .. cell_off[c+1])
 * The containing cell is the unique cell that holds p + (e, e^2, e^3) for
 * infinitesimal e > 0, so points on faces, edges and vertices have exactly
 * one cell.  The binned state stays in the mesh for the force calls.  A
 * molecule in no cell gets cell -1, no slot and zero force; the call then
 * returns AICA_ERR_OUTSIDE_MESH (after synchronizing the stream) unless
 * deferred checking is on (aica_set_deferred_checks).  A species index
 * outside [0, 8) gives AICA_ERR_INVALID_ARG.  The cell offsets come from a
 * single-pass scan whose blocks wait on one another with a bounded wait; if
 * a wait gives up the result is wrong and the call returns AICA_ERR_CUDA. */
aica_status aica_bin_molecules(aica_mesh *mesh, const double *pos, const int32_t *species, int64_t n,
                               int32_t *cell_of, int32_t *order, int32_t *cell_off, void *stream);

/* Forces, potential energy and virial over the AICA pair set (§2.3):
 * same-cell pairs, DIL pairs and periodic (real-referred) pairs, for the last
 * binned molecules.  §2.3 evaluates a real-referred pair once from each side,
 * acting on the real molecule only, because its source may live on another
 * processor; on one device each periodic image pair is evaluated once with
 * Newton's third law instead, which gives the same forces.
 *   prec   AICA_FP32: FP32 pair arithmetic on frame-local coordinates
 *          (separations rounded once on the cluster path), FP64
 *          energy/virial sums, r^2 < rc^2 decided in FP64 whenever the
 *          FP32 value lies within 1e-5 rc^2 of the cut-off, and molecules
 *          whose FP32 force may miss AICA_OPT_FP32_REFINE_TOL recomputed
 *          (see aica_set_option);
 *          AICA_FP64: all FP64.
 *   force_out  device [n*3], float (FP32) or double (FP64), original order;
 *              overwritten (may be NULL when no molecules were binned)
 *   ev_out     device double [7], optional: U, Wxx, Wyy, Wzz, Wxy, Wxz, Wyz
 *              with W_ab = sum over pairs of r_a f_b, each physical pair once
 *   counts_out device int64 [6], optional: evaluated pairs {same-cell, DIL,
 *              periodic image} (every molecule pair of every scheduled cell
 *              pair, each physical pair once), then the pairs within rc in
 *              the same order; their sum is the number of pairs within rc.
 * AICA_ERR_NOT_BUILT without lists and binning. */
aica_status aica_forces(aica_mesh *mesh, const aica_lj *lj, aica_precision prec, void *force_out,
                        double *ev_out, int64_t *counts_out, void *stream);

/* Adjoint of aica_forces for a loss L(F): given grad_force = dL/dF (device
 * [n*3], prec's type, original order) compute
 *   grad_pos   device [n*3] prec's type: dL/dx, a Hessian-vector product
 *   grad_eps   device double [S], optional: dL/d eps_s
 *   grad_sigma device double [S], optional: dL/d sigma_s
 * Pair terms are recomputed over the same pair set (nothing is stored by the
 * forward call).  A periodic image pair couples a molecule to the source
 * molecule of the referred copy, so both receive position gradient.  Under
 * general referring transforms (aica_mesh_set_transforms, §2.2.2) a referred
 * pair acts on the real molecule only and the source molecule's gradient is
 * rotated back (-R^T J v).  The cut-off is not differentiated.  FP32 sums
 * per-molecule gradients with FP32 atomics (run-to-run differences in the
 * last bits); the species sums are FP64.  AICA_ERR_INVALID_ARG for bad
 * species parameters (1..8 species), AICA_ERR_NOT_BUILT without lists and
 * binning. */
aica_status aica_forces_backward(aica_mesh *mesh, const aica_lj *lj, aica_precision prec,
                                 const void *grad_force, void *grad_pos, double *grad_eps,
                                 double *grad_sigma, void *stream);

/* One velocity-Verlet step around the per-step hot path, for the paper's
 * verification runs (§3: conservation of momentum and energy, results
 * independent of the mesh and of the decomposition):
 *   v += (dt/2) F(t)/m;  x += dt v;  bin (aica_bin_molecules);
 *   F(t+dt) (aica_forces);  v += (dt/2) F(t+dt)/m.
 *   mass     host double [S] (S = lj->n_species), positive
 *   dt       time step (> 0), in the units of mass, length and energy used
 *   n, species  device int32 [n]
 *   pos, vel device double [n*3], original order, updated in place; pos is
 *            not wrapped (binning wraps periodic coordinates itself)
 *   force    device [n*3], float (FP32) or double (FP64), original order:
 *            F(t) on entry (e.g. from aica_forces after binning pos), F(t+dt)
 *            on return
 *   ev_out   device double [7] or NULL: U and W at t+dt (as aica_forces)
 *   kin_out  device double [4] or NULL: kinetic energy sum m v^2 / 2 and
 *            momentum sum m v at t+dt
 * Errors as aica_bin_molecules and aica_forces (AICA_ERR_OUTSIDE_MESH when a
 * molecule leaves the mesh through a non-periodic side).  Asynchronous on
 * `stream` apart from the synchronizing checks of those two calls. */
aica_status aica_verlet_step(aica_mesh *mesh, const aica_lj *lj, aica_precision prec, const double *mass,
                             double dt, int64_t n, const int32_t *species, double *pos, double *vel,
                             void *force, double *ev_out, double *kin_out, void *stream);

/* Kinetic energy sum m v^2 / 2 and momentum sum m v (device double [4],
 * FP64) of n molecules with device velocities vel [n*3] and species [n];
 * mass host [n_species].  Asynchronous on `stream`. */
aica_status aica_kinetic(const double *mass, int32_t n_species, const int32_t *species, int64_t n,
                         const double *vel, double *kin_out, void *stream);

/* Stable counting sort of molecules by cell that allocates no device memory.
 * The paper has no counterpart; this entry point exists for callers that
 * cannot allocate device memory while they run: code recorded into a CUDA
 * graph or a stream capture (cudaMalloc is not capturable), real-time loops
 * that forbid allocation, and hosts whose device memory belongs to another
 * allocator.  It runs the sort stage of aica_bin_molecules (histogram,
 * prefix sum, scatter, per-cell order by original index) for cells the
 * caller already knows, with its workspace in a fixed device array inside
 * the library instead of allocated memory.
 *   cell_of  device [n] int32: cell of each molecule in [0, n_cells), or -1
 *            (the molecule is left out).  An id >= n_cells is left out the
 *            same way (nothing is read or written outside the arrays given
 *            and the workspace); the call does not synchronize to report
 *            it, so a caller that may pass such ids compares cell_off[n_cells]
 *            with the number of ids >= 0 it passed.
 *   order    device [n] out: order[s] = original index of slot s for
 *            s < cell_off[n_cells]; later entries are not written
 *   cell_off device [n_cells+1] out: cell c holds slots cell_off[c] ..
 *            cell_off[c+1]
 * The results equal those of aica_bin_molecules for the same cells.  Each
 * cell's slots are put in order by a bitonic sort in shared memory for
 * cells of up to 2048 molecules and by a serial insertion sort (time
 * growing with the square of the occupancy) above that.
 * Limits: n_cells <= 1048576 and n <= 2^30, else AICA_ERR_CAPACITY /
 * AICA_ERR_INVALID_ARG before any device work.  The workspace is about 4 MiB
 * of static device memory that every GPU loading this library holds until
 * the process exits.  All calls share it and it keeps the last call's
 * contents (each call clears what must start at zero), so calls that
 * overlap on the GPU (different streams or threads without ordering) race:
 * order them on one stream.  The first call on a device looks up the
 * workspace's device address (cudaGetSymbolAddress); make that first call
 * outside any stream capture.  Never calls cudaMalloc, cudaFree or an
 * allocating library routine.  Asynchronous on `stream`. */
aica_status aica_sort_by_cell_noalloc(const int32_t *cell_of, int64_t n, int64_t n_cells, int32_t *order,
                                      int32_t *cell_off, void *stream);

/* With deferred != 0, aica_bin_molecules and aica_forces do not synchronize
 * to check device-side error flags; the errors of all calls since the last
 * check accumulate and are reported (then cleared) by aica_check_status,
 * which synchronizes `stream`. */
aica_status aica_set_deferred_checks(aica_mesh *mesh, int deferred);
aica_status aica_check_status(aica_mesh *mesh, void *stream);

/* Measurement hook.  With enable != 0 every aica_forces call records a pair
 * of CUDA events on its stream around its pair kernel (no synchronization).
 * aica_take_kernel_times synchronizes on the recorded events, writes up to
 * cap durations in milliseconds (oldest first) to the host array ms, sets *n
 * to the number written and forgets them.  Not for use under stream capture. */
aica_status aica_set_kernel_timing(aica_mesh *mesh, int enable);
aica_status aica_take_kernel_times(aica_mesh *mesh, float *ms, int64_t cap, int64_t *n);

/* Options of a mesh (no counterpart in the paper: precision policy and
 * measurement switches of this implementation).
 *   AICA_OPT_FP32_REFINE_TOL  (default 1e-5) FP32 forces: the per-component
 *       error relative to max(|F_ic|, ||F_i||) that aica_forces targets on
 *       the box-periodic cluster path.  After the FP32 pass, a molecule
 *       whose force is too small against the FP32 error scale of its pair
 *       forces (|F_i| < 1.25e-6 sqrt(sum_l |f_kl|^2) / tol) is recomputed in
 *       double-single arithmetic (about 48 bits; cut-off decisions near rc in
 *       FP64) over the same pair set.  The factor is calibrated against FP64
 *       forces, not a proven bound.  <= 0 turns the recomputation off.
 *   AICA_OPT_COUNT_EVALUATED  (default 1) aica_forces fills counts_out[0..2]
 *       (pairs of every listed cell pair, §2.3) with an extra pass over the
 *       cell schedule when the FP32 cluster kernel runs; 0 skips that pass
 *       and reports 0 there.  The within-rc counts [3..5] are always exact.
 *   AICA_OPT_FP32_KERNEL      (default 0) FP32 box-periodic pair kernel:
 *       0 the cluster kernel when the lists have a cluster schedule, 1 the
 *       cell kernel (for comparison; its forces are not refined).
 *   AICA_OPT_N_OWNED          (default -1) portion of a spatial
 *       decomposition (§2.1, App. A.2): molecules [0, n_owned) of the next
 *       aica_bin_molecules call belong to this processor, the rest are the
 *       halo it received (the molecules of the remote source cells of its
 *       processor-referred cells, at their own positions).  aica_forces then
 *       evaluates a pair of two owned molecules with Newton's third law, a
 *       pair of an owned molecule and a halo molecule one-sidedly (the
 *       force on the owned molecule; half the pair's energy and virial, the
 *       other half being the other processor's), and no pair of two halo
 *       molecules; force rows of halo molecules are unspecified and the
 *       pair counts count each evaluated pair once.  Needs box periodicity
 *       and the minimum-distance lists of the whole mesh on every
 *       processor; aica_forces_backward and the cell kernel refuse it
 *       (AICA_ERR_INVALID_ARG).  -1 returns to a single processor.
 *   AICA_OPT_REFINED          (read only) molecules the last FP32
 *       aica_forces call recomputed (synchronizes `stream`).
 *   AICA_OPT_CLUSTER_PATH     (read only) 1 when the built lists have a
 *       cluster schedule (box periodicity, exact-separation bound met).
 * AICA_ERR_INVALID_ARG for an unknown option or a read-only one set. */
typedef enum {
    AICA_OPT_FP32_REFINE_TOL = 0,
    AICA_OPT_COUNT_EVALUATED = 1,
    AICA_OPT_FP32_KERNEL = 2,
    AICA_OPT_REFINED = 3,
    AICA_OPT_CLUSTER_PATH = 4,
    AICA_OPT_N_OWNED = 5
} aica_option;
aica_status aica_set_option(aica_mesh *mesh, aica_option option, double value);
aica_status aica_get_option(aica_mesh *mesh, aica_option option, double *value, void *stream);

/* Work the last aica_forces call actually performed (host int64 out[2]):
 * out[0] pair distance tests, out[1] bounding-sphere tests of partner cells
 * and molecules.  The kernels skip cells and molecules that cannot be within
 * rc, so out[0] is below the evaluated counts of aica_forces.  Synchronizes
 * `stream`. */
aica_status aica_get_work_counters(aica_mesh *mesh, int64_t *out, void *stream);

/* Measured arithmetic peak of the current device (a measurement helper with
 * no counterpart in the paper): the rate of fused multiply-adds in FP32
 * (fp64 == 0) or FP64 (fp64 != 0), counted as 2 flops each, over a grid
 * that fills every SM with independent FMA chains of `iters` steps per
 * chain.  One untimed launch, then one launch timed with CUDA events on
 * `stream`; synchronizes `stream`.  *flops_per_s (host) receives the rate.
 * Use iters of about 2e4 (FP64) or 1e6 (FP32) for a launch of tens of
 * milliseconds.  iters outside [1, 2^30] -> AICA_ERR_INVALID_ARG.  Allocates
 * no memory. */
aica_status aica_probe_fma_rate(int fp64, int64_t iters, double *flops_per_s, void *stream);

/* Number of kernels the last call on this mesh launched (for accounting). */
int64_t aica_last_launch_count(const aica_mesh *mesh);

/* Thread-local message of the last failure in this thread ("" if none). */
const char *aica_last_error(void);

/* Name of a status code. */
const char *aica_status_string(aica_status status);

#ifdef __cplusplus
}
#endif

#endif /* AICA_H */
