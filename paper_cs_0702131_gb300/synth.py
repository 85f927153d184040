"""Seeded synthetic inputs for the AICA pair-force path.

Builds Lennard-Jones fluids on FCC lattices and face-based polyhedral meshes
(jittered hexahedra, Kuhn/Freudenthal tetrahedra, a slab nanochannel with four
posts removed).  The paper's verification system (27 000 LJ molecules, §3) is
not available as data; these generators stand in for it with the shapes,
densities and mesh types of the workloads it describes (arbitrary polyhedral
cells, periodic boxes, a channel geometry as in §1.1).

This module builds inputs only.  It holds none of the method's arithmetic (no
distances between cells, no point location, no forces) and imports nothing
from the oracle or from the CUDA path: both sides take their inputs from here.

Mesh format (OpenFOAM-like, face based): ``points`` [P,3] f64,
``face_offsets`` [F+1] i64, ``face_vertices`` i64, ``owner`` [F] i64,
``neighbour`` [F] i64 (-1 on boundary faces), ``n_cells``.  Each face's vertex
order gives a right-handed normal pointing out of its owner cell.
Periodicity is translational, by the box lengths ``L`` on axes flagged in
``periodic``; boundary faces of a periodic axis carry ``neighbour = -1``.
"""
from __future__ import annotations

import itertools

import numpy as np

#: FCC lattice constant at reduced density 0.8: 4 / a^3 = 0.8.
A_FCC_08 = (4.0 / 0.8) ** (1.0 / 3.0)

_FCC_BASIS = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])

# Hexahedron local vertex k sits at grid offset (k & 1, (k >> 1) & 1, (k >> 2) & 1).
_HEX_FACES = np.array([[0, 4, 6, 2], [1, 3, 7, 5], [0, 1, 5, 4],
                       [2, 6, 7, 3], [0, 2, 3, 1], [4, 5, 7, 6]])
# Kuhn split of a cube along its main diagonal 0 -> 7: one tet per axis order.
_KUHN_TETS = np.array([[0, p[0], p[0] + p[1], 7] for p in itertools.permutations((1, 2, 4))])
_TET_FACES = np.array([[1, 2, 3], [0, 3, 2], [0, 1, 3], [0, 2, 1]])
_TET_OPPOSITE = np.array([0, 1, 2, 3])


# --------------------------------------------------------------------------- molecules
def fcc_sites(nx, ny, nz, a, iy0=0):
    """FCC sites of nx*ny*nz unit cells (4 per cell), unit-cell-major order."""
    i, j, k = np.meshgrid(np.arange(nx), np.arange(iy0, iy0 + ny), np.arange(nz), indexing="ij")
    cells = np.stack([i, j, k], -1).reshape(-1, 1, 3).astype(np.float64)
    return ((cells + _FCC_BASIS[None]) * a).reshape(-1, 3)


def wrap(pos, L, periodic):
    """Map coordinates on periodic axes into [0, L)."""
    out = np.array(pos, dtype=np.float64, copy=True)
    for ax in range(3):
        if periodic[ax]:
            x = np.mod(out[:, ax], L[ax])
            x[x >= L[ax]] = 0.0
            out[:, ax] = x
    return out


def jitter(pos, std, rng):
    return pos + rng.normal(0.0, std, size=pos.shape)


def random_displacement(pos, dist, rng, L, periodic):
    """Move every molecule by ``dist`` in a uniformly random direction, then wrap."""
    v = rng.normal(size=pos.shape)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return wrap(pos + dist * v, L, periodic)


# --------------------------------------------------------------------------- meshes
def _grid_vertices(shape, lo, hi):
    nx, ny, nz = shape
    axes = [np.linspace(lo[d], hi[d], shape[d] + 1) for d in range(3)]
    X, Y, Z = np.meshgrid(*axes, indexing="ij")
    ref = np.stack([X, Y, Z], -1).reshape(-1, 3)
    ii, jj, kk = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    boundary = ((ii == 0) | (ii == nx) | (jj == 0) | (jj == ny) | (kk == 0) | (kk == nz)).reshape(-1)
    return ref, boundary


def _hex_vertex_ids(shape):
    nx, ny, nz = shape
    ii, jj, kk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    base = np.stack([ii.reshape(-1), jj.reshape(-1), kk.reshape(-1)], -1)
    ids = np.empty((base.shape[0], 8), dtype=np.int64)
    for k in range(8):
        o = np.array([k & 1, (k >> 1) & 1, (k >> 2) & 1])
        g = base + o
        ids[:, k] = (g[:, 0] * (ny + 1) + g[:, 1]) * (nz + 1) + g[:, 2]
    return ids


def _orient_outward(faces, cell_vertices, ref):
    """Reverse faces whose (reference-geometry) normal points into their cell."""
    f = faces.copy()
    p = ref[f]                                    # [nc, nf, nv, 3]
    nv = f.shape[2]
    normal = np.zeros(p.shape[:2] + (3,))
    for v in range(nv):                           # Newell normal
        normal += np.cross(p[:, :, v], p[:, :, (v + 1) % nv])
    fc = p.mean(axis=2)
    cc = ref[cell_vertices].mean(axis=1)[:, None, :]
    inward = np.einsum("cfk,cfk->cf", normal, fc - cc) < 0
    f[inward] = f[inward][:, ::-1]
    return f


def _to_face_mesh(points, cell_faces):
    """Cell-wise oriented faces [nc, nf, nv] -> face-based arrays (owner < neighbour)."""
    nc, nf, nv = cell_faces.shape
    flat = cell_faces.reshape(-1, nv)
    cell_id = np.repeat(np.arange(nc, dtype=np.int64), nf)
    key3 = np.sort(flat, axis=1)[:, :3]          # three vertices identify a face
    shift = int(np.ceil(np.log2(points.shape[0] + 1)))
    if 3 * shift > 62:
        raise ValueError("mesh too large for face keys")
    key = (key3[:, 0] << (2 * shift)) | (key3[:, 1] << shift) | key3[:, 2]
    order = np.argsort(key, kind="stable")
    ks = key[order]
    starts = np.r_[0, np.flatnonzero(np.diff(ks)) + 1]
    counts = np.diff(np.r_[starts, ks.shape[0]])
    if np.any(counts > 2):
        raise ValueError("non-manifold face")
    first = order[starts]
    owner = cell_id[first]
    neighbour = np.full(starts.shape[0], -1, dtype=np.int64)
    two = counts == 2
    neighbour[two] = cell_id[order[starts[two] + 1]]
    fv = flat[first]
    return dict(points=np.ascontiguousarray(points, dtype=np.float64),
                face_offsets=np.arange(fv.shape[0] + 1, dtype=np.int64) * nv,
                face_vertices=np.ascontiguousarray(fv.reshape(-1), dtype=np.int64),
                owner=owner, neighbour=neighbour, n_cells=int(nc))


def hex_mesh(shape, lo, hi, jitter_frac, rng, tets=False, keep=None):
    """Structured grid of hexahedra (optionally Kuhn-split into 6 tets each).

    Interior vertices move by U(+-jitter_frac * w) per component; vertices on
    the outer boundary, and every vertex of a removed hexahedron (``keep`` is a
    boolean mask over hexahedra), stay on the grid.
    """
    shape = tuple(int(s) for s in shape)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    ref, boundary = _grid_vertices(shape, lo, hi)
    hexes = _hex_vertex_ids(shape)
    frozen = boundary.copy()
    if keep is not None:
        frozen[np.unique(hexes[~keep])] = True
        hexes = hexes[keep]
    w = (hi - lo) / np.asarray(shape)
    pts = ref + rng.uniform(-1.0, 1.0, size=ref.shape) * (jitter_frac * w)
    pts[frozen] = ref[frozen]
    if tets:
        cells = hexes[:, _KUHN_TETS].reshape(-1, 4)
        faces = cells[:, _TET_FACES]
    else:
        cells = hexes
        faces = hexes[:, _HEX_FACES]
    faces = _orient_outward(faces, cells, ref)
    mesh = _to_face_mesh(pts, faces)
    mesh["cell_vertices"] = cells
    return mesh


# --------------------------------------------------------------------------- configs
def _box(L, periodic):
    return dict(L=np.asarray(L, dtype=np.float64), periodic=np.asarray(periodic, dtype=np.int32))


def _lj_fluid(n_cells_fcc, a, hex_shape, tets, rc, seed, jitter_std=0.05, hex_jitter=0.15):
    rng = np.random.default_rng(seed)
    L = np.asarray(n_cells_fcc, dtype=np.float64) * a
    box = _box(L, (1, 1, 1))
    pos = wrap(jitter(fcc_sites(*n_cells_fcc, a), jitter_std, rng), box["L"], box["periodic"])
    mesh = hex_mesh(hex_shape, (0, 0, 0), L, hex_jitter, rng, tets=tets)
    n = pos.shape[0]
    return dict(pos=pos, species=np.zeros(n, np.int32), eps=np.array([1.0]), sigma=np.array([1.0]),
                rc=float(rc), box=box, mesh=mesh)


def nanochannel(seed, nfcc=(144, 12, 144), hex_shape=(96, 10, 96), post_radius=5.0, rc=2.5):
    """Slab channel periodic in x and z, walls of two fixed FCC (100) layers each side.

    Fluid: FCC nfcc unit cells at density 0.8, jittered.  Walls continue the
    lattice two half-layers below y = 0 and above y = ny*a.  The mesh spans
    y in [-1.25a, (ny + 0.75)a]; hexahedra whose centroid lies within
    ``post_radius`` of four y-parallel post axes are removed, and molecules
    inside removed hexahedra are dropped.
    """
    rng = np.random.default_rng(seed)
    a = A_FCC_08
    Lx, Lz = nfcc[0] * a, nfcc[2] * a
    y0, y1 = -1.25 * a, (nfcc[1] + 0.75) * a
    nx, ny, nz = hex_shape
    wx, wy, wz = Lx / nx, (y1 - y0) / ny, Lz / nz
    ci = (np.arange(nx) + 0.5) * wx
    ck = (np.arange(nz) + 0.5) * wz
    CX, CK = np.meshgrid(ci, ck, indexing="ij")
    in_post = np.zeros_like(CX, dtype=bool)
    for fx, fz in ((0.25, 0.25), (0.75, 0.25), (0.25, 0.75), (0.75, 0.75)):
        in_post |= (CX - fx * Lx) ** 2 + (CK - fz * Lz) ** 2 < post_radius ** 2
    removed = np.broadcast_to(in_post[:, None, :], (nx, ny, nz)).reshape(-1)
    mesh = hex_mesh(hex_shape, (0.0, y0, 0.0), (Lx, y1, Lz), 0.15, rng, tets=False, keep=~removed)
    sites = fcc_sites(nfcc[0], nfcc[1] + 2, nfcc[2], a, iy0=-1)
    wall = (sites[:, 1] < -1e-9) | (sites[:, 1] > nfcc[1] * a - 1e-9)
    box = _box((Lx, y1 - y0, Lz), (1, 0, 1))
    pos = sites.copy()
    pos[~wall] = jitter(sites[~wall], 0.05, rng)
    pos = wrap(pos, box["L"], box["periodic"])
    hx = np.clip(np.floor(pos[:, 0] / wx).astype(np.int64), 0, nx - 1)
    hy = np.clip(np.floor((pos[:, 1] - y0) / wy).astype(np.int64), 0, ny - 1)
    hz = np.clip(np.floor(pos[:, 2] / wz).astype(np.int64), 0, nz - 1)
    keep_mol = ~removed[(hx * ny + hy) * nz + hz]
    pos, wall = pos[keep_mol], wall[keep_mol]
    n = pos.shape[0]
    return dict(pos=pos, species=np.zeros(n, np.int32), eps=np.array([1.0]), sigma=np.array([1.0]),
                rc=float(rc), box=box, mesh=mesh, wall=wall)


def two_species(seed, nfcc=(16, 32, 32), hex_shape=(16, 16, 16), rc=2.5):
    """Binary LJ mixture 50/50 by seeded permutation; eps1/eps0 = 1.5, sigma1/sigma0 = 0.88."""
    cfg = _lj_fluid(nfcc, A_FCC_08, hex_shape, False, rc, seed)
    rng = np.random.default_rng(seed + 7919)
    n = cfg["pos"].shape[0]
    sp = np.zeros(n, np.int32)
    sp[rng.permutation(n)[: n // 2]] = 1
    cfg.update(species=sp, eps=np.array([1.0, 1.5]), sigma=np.array([1.0, 0.88]))
    return cfg


def wedge(seed, r0=4.0, r1=12.0, nz_sc=8, nr=4, ntheta=6, nz=4, jitter_std=0.05):
    """A 90-degree sector of an annulus, rotationally periodic about the z axis
    and periodic in z: the general (rotated) referral of §2.2.2.

    Cells: hexahedra of a polar grid (planar chord faces).  Molecules: sites
    ((i+1/2)a, (j+1/2)a, (k+1/2)a) of a simple cubic lattice at density 0.8,
    a lattice the quarter turn maps onto itself, jittered, kept where they lie
    inside a cell.  Transforms (R, y): the quarter turn from the coupled faces
    theta = 0 (normal -y) and theta = 90 degrees (normal -x), and the shift
    (0, 0, H).  The box has no periodic axis (z periodicity is a transform).
    """
    rng = np.random.default_rng(seed)
    a = (1.0 / 0.8) ** (1.0 / 3.0)
    H = nz_sc * a
    r = np.linspace(r0, r1, nr + 1)
    th = np.linspace(0.0, 0.5 * np.pi, ntheta + 1)
    z = np.linspace(0.0, H, nz + 1)
    R_, T_, Z_ = np.meshgrid(r, th, z, indexing="ij")
    pts = np.stack([R_ * np.cos(T_), R_ * np.sin(T_), Z_], -1).reshape(-1, 3)
    pts[np.abs(pts) < 1e-12] = 0.0
    vid = lambda i, j, k: (i * (ntheta + 1) + j) * (nz + 1) + k
    cells = []
    for i in range(nr):
        for j in range(ntheta):
            for k in range(nz):
                cells.append([vid(i + (v & 1), j + ((v >> 1) & 1), k + ((v >> 2) & 1)) for v in range(8)])
    mesh = cells_to_mesh(pts, np.array(cells))
    n1 = int(np.ceil(r1 / a)) + 1
    g = (np.arange(n1) + 0.5) * a
    gz = (np.arange(nz_sc) + 0.5) * a
    X, Y, Zs = np.meshgrid(g, g, gz, indexing="ij")
    sites = np.stack([X.ravel(), Y.ravel(), Zs.ravel()], 1)
    rad = np.hypot(sites[:, 0], sites[:, 1])
    sites = sites[(rad > r0 + 0.2) & (rad < r1 * np.cos(0.25 * np.pi / ntheta) - 0.2)]
    pos = sites + rng.normal(scale=jitter_std, size=sites.shape)
    pos[:, 2] = np.clip(pos[:, 2], 1e-6, H - 1e-6)
    keep = (pos[:, 0] > 1e-6) & (pos[:, 1] > 1e-6)
    pos = pos[keep]
    rot = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    transforms = [(rot, np.zeros(3)), (np.eye(3), np.array([0.0, 0.0, H]))]
    box = _box((2 * r1, 2 * r1, H), (0, 0, 0))
    n = pos.shape[0]
    return dict(pos=pos, species=np.zeros(n, np.int32), eps=np.array([1.0]), sigma=np.array([1.0]), rc=2.5,
                box=box, mesh=mesh, transforms=transforms, H=H, skin=1e-3, name=f"wedge-s{seed}")


#: Named workloads.  ``c1``..``c5`` follow the five configurations of the
#: benchmark table; ``t0`` and ``h0`` are small tet/hex cases for full parity.
CONFIGS = {
    "c1": dict(doc="2,048 molecules (FCC 8^3), 6^3 jittered hexes, periodic, rc 2.5",
               make=lambda seed: _lj_fluid((8, 8, 8), A_FCC_08, (6, 6, 6), False, 2.5, seed)),
    "c2": dict(doc="256,000 molecules (FCC 40^3), 24^3 hexes -> 82,944 Kuhn tets, periodic, rc 2.5",
               make=lambda seed: _lj_fluid((40, 40, 40), A_FCC_08, (24, 24, 24), True, 2.5, seed)),
    "c3": dict(doc="~1.16M molecules: nanochannel 144x12x144 FCC fluid + 4 wall layers, 4 posts, rc 2.5",
               make=lambda seed: nanochannel(seed)),
    "c4": dict(doc="65,536 molecules (FCC 16x32x32), 2 species, 16^3 jittered hexes, rc 2.5",
               make=lambda seed: two_species(seed)),
    "c5": dict(doc="8,388,608 molecules (FCC 128^3), 80^3 hexes -> 3,072,000 Kuhn tets, rc 3.0",
               make=lambda seed: _lj_fluid((128, 128, 128), A_FCC_08, (80, 80, 80), True, 3.0, seed)),
    "t0": dict(doc="864 molecules (FCC 6^3), 4^3 hexes -> 384 Kuhn tets, periodic, rc 2.5",
               make=lambda seed: _lj_fluid((6, 6, 6), A_FCC_08, (4, 4, 4), True, 2.5, seed)),
    "h0": dict(doc="4,000 molecules (FCC 10^3), 7^3 jittered hexes, periodic, rc 2.5",
               make=lambda seed: _lj_fluid((10, 10, 10), A_FCC_08, (7, 7, 7), False, 2.5, seed)),
}


def make(name, seed=0):
    """Build a named workload; the seed fixes molecules and mesh jitter."""
    cfg = CONFIGS[name]["make"](seed)
    cfg["name"] = f"{name}-s{seed}"
    cfg.setdefault("skin", 1e-3)
    return cfg


def cells_to_mesh(points, cells):
    """Face-based mesh from explicit hexahedra ([n,8], grid-offset vertex order)
    or tetrahedra ([n,4]); faces are oriented outward from their owner using the
    given coordinates.  For hand-built test geometries."""
    points = np.asarray(points, dtype=np.float64)
    cells = np.asarray(cells, dtype=np.int64)
    faces = cells[:, _HEX_FACES] if cells.shape[1] == 8 else cells[:, _TET_FACES]
    mesh = _to_face_mesh(points, _orient_outward(faces, cells, points))
    mesh["cell_vertices"] = cells
    return mesh


def cube_cells(origins, size=1.0):
    """Points and hexahedra of axis-aligned cubes with the given min corners."""
    origins = np.asarray(origins, dtype=np.float64)
    off = np.array([[k & 1, (k >> 1) & 1, (k >> 2) & 1] for k in range(8)], dtype=np.float64) * size
    pts = (origins[:, None, :] + off[None]).reshape(-1, 3)
    return pts, np.arange(pts.shape[0]).reshape(-1, 8)
