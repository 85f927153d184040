"""CPU oracle for the AICA pair-force path.  TEST INFRASTRUCTURE ONLY.

Plain, slow, FP64 reference implementations written from the paper
(Macpherson & Reese, arXiv cs/0702131).  Only ``tests/``, the package smoke
check and the CPU-baseline leg of ``bench.py`` may import this package; the
product path never does.  It shares no code with the CUDA path and takes its
inputs as plain arrays (from the seeded generators or hand-written fixtures).

Functions and the passage each follows
  lj                 all-pairs minimum-image LJ sum: the set the method reaches
                     (§2.3: real-real plus real-referred covers every pair once)
  cell_geometry      fan triangulation of faces from their lowest vertex id
  cell_lists         direct interaction lists (§2.2, App. A.1, j > i, never
                     self) and periodic referred cells with their real-cell
                     lists (§2.2.1, App. A.2) by brute force over cell pairs
  locate, bin_order  the containing cell of each molecule and the stable
                     binned order (§2.2: a molecule's cell is always known)
  aica_loop          the two force loops of §2.3 over the oracle's own lists
  lj_cells           the same LJ sum by the cubic-cell algorithm of §2.1
                     (CPU baseline)
  verlet             velocity-Verlet trajectories with all-pairs forces, for
                     the verification runs of §3 (conservation, mesh
                     independence)
  torch_ref          autograd-of-oracle reference for the adjoint (torch FP64)

Parity pins live in ``tests/test_oracle_*.py``.  Readings of the paper used
here (none of these is printed in it): LJ 12-6 truncated at r < rc without
shift, Lorentz-Berthelot mixing, cell-cell criterion min_dist < rc + skin
(instead of vertex-vertex distance, see the twisted-mesh error of §2.2),
exact ties resolved by perturbing a point to p + (e, e^2, e^3).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "aica_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None

_f64 = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i64 = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_i32 = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def build(force=False):
    """Compile the C oracle (gcc, OpenMP, no FP contraction)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        vp = ctypes.c_void_p
        L.oracle_lj.argtypes = [ctypes.c_int64, _f64, _i32, ctypes.c_int, _f64, _f64, ctypes.c_double, _f64,
                                _i32, ctypes.c_int, vp, ctypes.c_int64, _f64, _f64, _f64, _f64, _i64]
        L.oracle_cell_pairs.argtypes = [_i64, _f64, _i64, _f64, _i64, _f64, _f64, _f64, ctypes.c_int64, _i64,
                                        ctypes.c_int64, ctypes.c_double, _i32, _f64, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int64, _i64, _i32, _i32, _f64, _i64]
        L.oracle_cell_pairs_grid.argtypes = [_i64, _f64, _i64, _f64, _i64, _f64, _f64, _f64, ctypes.c_int64,
                                             _i64, ctypes.c_int64, ctypes.c_double, _i32, _f64, ctypes.c_int, ctypes.c_int, _i64, _i64,
                                             _i64, _f64, ctypes.c_double, _i64, _i64, _i32,
                                             np.ctypeslib.ndpointer(np.int8, flags="C_CONTIGUOUS"), _i64]
        L.oracle_locate.argtypes = [_i64, _f64, _f64, _f64, ctypes.c_int64, _f64, ctypes.c_int64, _f64, _i32,
                                    _i32, _f64]
        L.oracle_aica_loop.argtypes = [ctypes.c_int64, _i64, _f64, _i32, _f64, _f64, ctypes.c_double, _f64,
                                       ctypes.c_int, _i64, _i32, ctypes.c_int64, _i32, _i32, _i64, _i32, _f64,
                                       _f64, _i64]
        L.oracle_lj_cells.argtypes = [ctypes.c_int64, _f64, _i32, _f64, _f64, ctypes.c_double, _f64, _i32,
                                      ctypes.c_int, _f64, _f64, _f64, _f64, _i64]
        L.oracle_lj_images.argtypes = [ctypes.c_int64, _f64, _i32, _f64, _f64, ctypes.c_double, ctypes.c_int64,
                                       _f64, _f64, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, _f64, _f64, _f64,
                                       _f64, _i64]
        L.oracle_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def num_threads():
    return int(lib().oracle_num_threads())


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


# ----------------------------------------------------------------------------- LJ
def lj(pos, species, eps, sigma, rc, box, shift=False, idx=None):
    """All-pairs minimum-image LJ forces (the plain definition).

    Returns dict(F [m,3], Fabs [m] = sum_l |f_kl|, U, W [6] (xx,yy,zz,xy,xz,yz),
    Uabs = sum |u|, Wabs = sum |r . f| over pairs, row_pairs = number of
    (k, l) within rc over the computed rows, pairs = number of unordered pairs
    within rc (only when idx is None)).
    Requires rc < L/2 on periodic axes, where the minimum image is unique.
    """
    pos = _c(pos, np.float64)
    n = pos.shape[0]
    idx_arr = None if idx is None else _c(idx, np.int64)
    m = n if idx is None else idx_arr.shape[0]
    F = np.zeros((m, 3))
    Fabs = np.zeros(m)
    ev = np.zeros(7)
    ab = np.zeros(2)
    cnt = np.zeros(1, np.int64)
    lib().oracle_lj(n, pos, _c(species, np.int32), len(eps), _c(eps, np.float64), _c(sigma, np.float64),
                    float(rc), _c(box["L"], np.float64), _c(box["periodic"], np.int32), int(bool(shift)),
                    None if idx_arr is None else idx_arr.ctypes.data, m, F, Fabs, ev, ab, cnt)
    out = dict(F=F, Fabs=Fabs, U=ev[0], W=ev[1:].copy(), Uabs=ab[0], Wabs=ab[1], row_pairs=int(cnt[0]))
    if idx is None:
        out["pairs"] = int(cnt[0]) // 2
    return out


def lj_cells(pos, species, eps, sigma, rc, box, shift=False):
    """The same sum as lj() by the cubic-cell algorithm of §2.1 (CPU baseline).

    Returns the keys of lj() for all molecules.  Requires rc < L/2 on periodic
    axes, as lj() does.
    """
    pos = _c(pos, np.float64)
    n = pos.shape[0]
    F = np.zeros((n, 3))
    Fabs = np.zeros(n)
    ev = np.zeros(7)
    ab = np.zeros(2)
    cnt = np.zeros(1, np.int64)
    lib().oracle_lj_cells(n, pos, _c(species, np.int32), _c(eps, np.float64), _c(sigma, np.float64), float(rc),
                          _c(box["L"], np.float64), _c(box["periodic"], np.int32), int(bool(shift)), F, Fabs, ev,
                          ab, cnt)
    return dict(F=F, Fabs=Fabs, U=ev[0], W=ev[1:].copy(), Uabs=ab[0], Wabs=ab[1], row_pairs=int(cnt[0]),
                pairs=int(cnt[0]) // 2)


def lj_images(pos, species, eps, sigma, rc, transforms, shift=False, idx=None):
    """LJ forces from the images y + R.x of all molecules under `transforms`
    (a list of (R, y), the identity included; see oracle.transforms): the
    plain definition of the forces under general periodicity (§2.2.2).
    Returns the keys of lj() for the rows idx (all molecules if None); pairs =
    within-rc (k, image) terms / 2 when all rows are computed."""
    pos = _c(pos, np.float64)
    n = pos.shape[0]
    idx_arr = None if idx is None else _c(idx, np.int64)
    m = n if idx is None else idx_arr.shape[0]
    R = _c(np.array([t[0] for t in transforms]).reshape(-1), np.float64)
    y = _c(np.array([t[1] for t in transforms]).reshape(-1), np.float64)
    F = np.zeros((m, 3))
    Fabs = np.zeros(m)
    ev = np.zeros(7)
    ab = np.zeros(2)
    cnt = np.zeros(1, np.int64)
    lib().oracle_lj_images(n, pos, _c(species, np.int32), _c(eps, np.float64), _c(sigma, np.float64), float(rc),
                           len(transforms), R, y, int(bool(shift)),
                           None if idx_arr is None else idx_arr.ctypes.data, m, F, Fabs, ev, ab, cnt)
    out = dict(F=F, Fabs=Fabs, U=ev[0], W=ev[1:].copy(), Uabs=ab[0], Wabs=ab[1], row_pairs=int(cnt[0]))
    if idx is None:
        out["pairs"] = int(cnt[0]) // 2
    return out


# ------------------------------------------------------------------ cell geometry
def cell_geometry(mesh):
    """Per-cell closed triangulated surfaces.

    Each face is split into a fan from its lowest global vertex id, so the two
    cells sharing a face see the same triangles.  Triangles are oriented out of
    their cell (the face order points out of the owner; the neighbour gets
    the reversed triangles).  Returns CSR arrays of triangle coordinates,
    unique vertices and unique edges (fan diagonals included), plus the vertex
    mean ``ctr``, ``rad`` = max distance from ctr to a vertex, and the
    bounding box ``lo``/``hi`` per cell.
    """
    P = _c(mesh["points"], np.float64)
    fo = _c(mesh["face_offsets"], np.int64)
    fv = _c(mesh["face_vertices"], np.int64)
    own = _c(mesh["owner"], np.int64)
    nei = _c(mesh["neighbour"], np.int64)
    C = int(mesh["n_cells"])
    NV = P.shape[0]
    sizes = np.diff(fo)
    tri_cell, tri_v = [], []
    for k in np.unique(sizes):                       # faces grouped by vertex count
        fs = np.flatnonzero(sizes == k)
        w = fv[fo[fs][:, None] + np.arange(k)]
        r = np.argmin(w, axis=1)
        w = np.take_along_axis(w, (np.arange(k)[None, :] + r[:, None]) % k, axis=1)
        for i in range(1, k - 1):
            t = np.stack([w[:, 0], w[:, i], w[:, i + 1]], 1)
            tri_cell.append(own[fs])
            tri_v.append(t)
            b = nei[fs] >= 0
            tri_cell.append(nei[fs][b])
            tri_v.append(t[b][:, [0, 2, 1]])
    tri_cell = np.concatenate(tri_cell)
    tri_v = np.concatenate(tri_v)
    o = np.lexsort((tri_v[:, 2], tri_v[:, 1], tri_v[:, 0], tri_cell))
    tri_cell, tri_v = tri_cell[o], tri_v[o]
    tri_off = np.zeros(C + 1, np.int64)
    np.add.at(tri_off, tri_cell + 1, 1)
    tri_off = np.cumsum(tri_off)
    kv = np.unique(np.repeat(tri_cell, 3) * NV + tri_v.reshape(-1))
    vcell, vtx_ids = kv // NV, kv % NV
    vtx_off = np.searchsorted(vcell, np.arange(C + 1)).astype(np.int64)
    e = np.concatenate([tri_v[:, [0, 1]], tri_v[:, [1, 2]], tri_v[:, [2, 0]]])
    e = np.sort(e, axis=1)
    ke = np.unique((np.tile(tri_cell, 3) * NV + e[:, 0]) * NV + e[:, 1])
    ecell = ke // (NV * NV)
    edg_ids = np.stack([(ke // NV) % NV, ke % NV], 1)
    edg_off = np.searchsorted(ecell, np.arange(C + 1)).astype(np.int64)
    vtx = P[vtx_ids]
    cell_of_v = np.repeat(np.arange(C), np.diff(vtx_off))
    ctr = np.zeros((C, 3))
    np.add.at(ctr, cell_of_v, vtx)
    ctr /= np.diff(vtx_off)[:, None]
    rad = np.zeros(C)
    np.maximum.at(rad, cell_of_v, np.linalg.norm(vtx - ctr[cell_of_v], axis=1))
    lo = np.full((C, 3), np.inf)
    hi = np.full((C, 3), -np.inf)
    np.minimum.at(lo, cell_of_v, vtx)
    np.maximum.at(hi, cell_of_v, vtx)
    return dict(n_cells=C, tri_off=tri_off, tri=_c(P[tri_v].reshape(-1, 9), np.float64), tri_ids=tri_v,
                vtx_off=vtx_off, vtx=_c(vtx, np.float64), edg_off=edg_off,
                edg=_c(P[edg_ids].reshape(-1, 6), np.float64), ctr=_c(ctr, np.float64), rad=_c(rad, np.float64),
                lo=_c(lo, np.float64), hi=_c(hi, np.float64))


def image_range(thr, box):
    """|n_k| <= ceil(thr / L_k) on periodic axes (two cells inside the box whose
    images are (|n_k| - 1) L_k apart or more cannot be within thr), 0 otherwise."""
    return np.array([int(np.ceil(thr / box["L"][d])) if box["periodic"][d] else 0 for d in range(3)], np.int32)


def cell_pairs(geo, box, thr, queries=None, use_bound=True, cap=8192, criterion="min_distance"):
    """Every (A, B, n) with min_dist(A, B + n.L) < thr for the query cells A.

    With criterion="vertex" the distance is the paper's vertex-vertex one
    (§2.2, App. A.1) instead of the exact minimum distance between the
    polyhedra.  Returns (A, B, n [k,3], d2, ties).  Brute force over all cells
    and images.
    """
    if criterion not in ("min_distance", "vertex"):
        raise ValueError(criterion)
    C = geo["n_cells"]
    q = np.arange(C, dtype=np.int64) if queries is None else _c(queries, np.int64)
    nq = q.shape[0]
    m = image_range(thr, box)
    cnt = np.zeros(nq, np.int64)
    ties = np.zeros(nq, np.int64)
    outB = np.zeros(nq * cap, np.int32)
    outN = np.zeros(nq * cap * 3, np.int32)
    outD = np.zeros(nq * cap, np.float64)
    lib().oracle_cell_pairs(geo["tri_off"], geo["tri"], geo["vtx_off"], geo["vtx"], geo["edg_off"], geo["edg"],
                            geo["ctr"], geo["rad"], C, q, nq, float(thr), m, _c(box["L"], np.float64),
                            int(use_bound), int(criterion == "vertex"), cap, cnt, outB, outN, outD, ties)
    if np.any(cnt < 0):
        raise RuntimeError("oracle_cell_pairs: capacity exceeded")
    sel = np.concatenate([np.arange(i * cap, i * cap + cnt[i]) for i in range(nq)]) if nq else np.zeros(0, int)
    A = np.repeat(q, cnt)
    return A, outB[sel].astype(np.int64), outN.reshape(-1, 3)[sel].astype(np.int64), outD[sel], int(ties.sum())


def cell_lists(mesh, box, rc, skin, queries=None, geo=None, use_bound=True, criterion="min_distance"):
    """Direct interaction lists and periodic referred cells.

    DIL(i) = ascending {j > i : min_dist(i, j) < rc + skin} (§2.2, App. A.1).
    Referred cells: every (c, n), n != 0, |n_k| <= ceil((rc+skin)/L_k), with a
    non-empty list {J : min_dist(J, c + n.L) < rc + skin} (§2.2.1), sorted by
    (c, n) with n lexicographic; lists ascending.  Found from the query cell
    c's side: min_dist(J, c + n.L) = min_dist(c, J - n.L).

    With ``queries`` the lists cover only those cells (as DIL owners and as
    referred-cell sources).  criterion="vertex" replaces min_dist by the
    paper's vertex-vertex distance.  Returns a dict of CSR arrays and ``ties``.
    """
    geo = geo or cell_geometry(mesh)
    thr = rc + skin
    A, B, N, _, ties = cell_pairs(geo, box, thr, queries, use_bound, criterion=criterion)
    C = geo["n_cells"]
    cells = np.arange(C) if queries is None else np.asarray(queries, np.int64)
    zero = ~N.any(axis=1)
    dil = zero & (B > A)
    dil_off, dil_ids = [0], []
    ref_src, ref_n, ref_off, ref_ids = [], [], [0], []
    for c in cells:
        s = A == c
        d = np.sort(B[s & dil])
        dil_ids.append(d)
        dil_off.append(dil_off[-1] + len(d))
        r = s & ~zero
        nn = -N[r]
        bb = B[r]
        if len(bb):
            key = np.lexsort((bb, nn[:, 2], nn[:, 1], nn[:, 0]))
            nn, bb = nn[key], bb[key]
            brk = np.r_[0, np.flatnonzero(np.any(np.diff(nn, axis=0) != 0, axis=1)) + 1, len(bb)]
            for i in range(len(brk) - 1):
                ref_src.append(c)
                ref_n.append(nn[brk[i]])
                ref_ids.append(bb[brk[i]:brk[i + 1]])
                ref_off.append(ref_off[-1] + brk[i + 1] - brk[i])
    cat = lambda xs: np.concatenate(xs).astype(np.int32) if xs else np.zeros(0, np.int32)
    return dict(cells=np.asarray(cells, np.int64), dil_off=np.asarray(dil_off, np.int64), dil_ids=cat(dil_ids),
                ref_src=np.asarray(ref_src, np.int32),
                ref_n=np.asarray(ref_n, np.int32).reshape(-1, 3),
                ref_off=np.asarray(ref_off, np.int64), ref_ids=cat(ref_ids), ties=ties)


def cell_lists_full(mesh, box, rc, skin, queries=None, geo=None, criterion="min_distance"):
    """The lists of cell_lists at full size: the candidate cells of each
    query come from a bucket grid of the cell centres (oracle_cell_pairs_grid)
    instead of a loop over all cells; the sphere bound and the distance that
    decide are the same, so the lists are too (pinned against cell_lists in
    the tests).  Same arguments and dict as cell_lists."""
    if criterion not in ("min_distance", "vertex"):
        raise ValueError(criterion)
    geo = geo or cell_geometry(mesh)
    thr = rc + skin
    C = geo["n_cells"]
    ctr = geo["ctr"].reshape(-1, 3)
    rmax = float(geo["rad"].max()) if C else 0.0
    h = max((thr + 2 * rmax) / 2, 1e-9)
    glo = ctr.min(axis=0) if C else np.zeros(3)
    G = (np.floor((ctr.max(axis=0) - glo) / h).astype(np.int64) + 1) if C else np.ones(3, np.int64)
    ib = np.clip(np.floor((ctr - glo) / h).astype(np.int64), 0, G - 1)
    bk = (ib[:, 0] * G[1] + ib[:, 1]) * G[2] + ib[:, 2]
    order = np.argsort(bk, kind="stable").astype(np.int64)
    bkt_off = np.r_[0, np.cumsum(np.bincount(bk, minlength=int(G.prod())))].astype(np.int64)
    m = image_range(thr, box)
    cells = np.arange(C, dtype=np.int64) if queries is None else np.asarray(queries, np.int64)
    if len(cells) and (not np.all(np.diff(cells) > 0) or cells[0] < 0 or cells[-1] >= C):
        raise ValueError("queries must be ascending, unique cell ids")
    nq = len(cells)
    cnt = np.zeros(nq, np.int64)
    ties = np.zeros(nq, np.int64)
    args = (geo["tri_off"], geo["tri"], geo["vtx_off"], geo["vtx"], geo["edg_off"], geo["edg"], geo["ctr"],
            geo["rad"], C, cells, nq, float(thr), m, _c(box["L"], np.float64), int(criterion == "vertex"))
    grid = (bkt_off, order, G, _c(glo, np.float64), float(h))
    one = np.zeros(1, np.int32)
    one8 = np.zeros(3, np.int8)
    lib().oracle_cell_pairs_grid(*args, 0, *grid, cnt, np.zeros(nq + 1, np.int64), one, one8, ties)
    off = np.r_[0, np.cumsum(cnt)].astype(np.int64)
    E = int(off[-1])
    outB = np.zeros(max(E, 1), np.int32)
    outN = np.zeros(3 * max(E, 1), np.int8)
    lib().oracle_cell_pairs_grid(*args, 1, *grid, cnt, off, outB, outN, ties)
    A = np.repeat(cells, cnt)
    B = outB[:E].astype(np.int64)
    N = outN[:3 * E].reshape(-1, 3).astype(np.int64)
    zero = ~N.any(axis=1)
    dA, dB = A[zero], B[zero]                        # n = 0, B > A
    o = np.lexsort((dB, dA))
    rows = np.searchsorted(cells, dA) if queries is not None else dA      # row of each entry's owner
    dil_off = np.r_[0, np.cumsum(np.bincount(rows, minlength=nq))].astype(np.int64)
    dil_ids = dB[o].astype(np.int32)
    rA, rB, rn = A[~zero], B[~zero], -N[~zero]       # referred cell (source A, image -n)
    o = np.lexsort((rB, rn[:, 2], rn[:, 1], rn[:, 0], rA))
    rA, rB, rn = rA[o], rB[o], rn[o]
    if len(rA):
        new = np.r_[True, (np.diff(rA) != 0) | np.any(np.diff(rn, axis=0) != 0, axis=1)]
        starts = np.flatnonzero(new)
    else:
        starts = np.zeros(0, np.int64)
    return dict(cells=cells, dil_off=dil_off, dil_ids=dil_ids,
                ref_src=rA[starts].astype(np.int32), ref_n=rn[starts].astype(np.int32).reshape(-1, 3),
                ref_off=np.r_[starts, len(rA)].astype(np.int64), ref_ids=rB.astype(np.int32),
                ties=int(ties.sum()))


# ------------------------------------------------------------------- point location
def _exact_sign(x):
    return (x > 0) - (x < 0)


def _inside_exact(tris, p):
    """Ray-parity membership of p + (e, e^2, e^3) in a closed triangulated
    surface, in exact rational arithmetic (slow path for uncertain cases).
    Every FP64 value is a dyadic rational, so all coordinates are scaled to
    integers over one common power-of-two denominator (exactly); the signs of
    the determinants below are those of the rational ones."""
    vals = [float(v) for v in p] + [float(v) for v in np.asarray(tris).reshape(-1)]
    rat = [v.as_integer_ratio() for v in vals]
    D = max(d for _, d in rat)
    ints = [n * (D // d) for n, d in rat]
    P = ints[:3]
    T = ints[3:]
    parity = 0
    for t in range(len(T) // 9):
        q = T[9 * t:9 * t + 9]
        a, b, c = q[0:3], q[3:6], q[6:9]
        nx = _exact_sign((b[1] - a[1]) * (c[2] - a[2]) - (b[2] - a[2]) * (c[1] - a[1]))
        if nx == 0:
            continue
        es = []
        for u, v in ((a, b), (b, c), (c, a)):
            s = _exact_sign((v[1] - u[1]) * (P[2] - u[2]) - (v[2] - u[2]) * (P[1] - u[1]))
            if s == 0:
                s = _exact_sign(-(v[2] - u[2])) or _exact_sign(v[1] - u[1])
            es.append(s)
        if not all(s == nx for s in es):
            continue
        u = [b[i] - a[i] for i in range(3)]
        w = [c[i] - a[i] for i in range(3)]
        N = [u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]]
        o = _exact_sign(sum(N[i] * (P[i] - a[i]) for i in range(3)))
        if o == 0:
            o = nx
        if o == -nx:
            parity ^= 1
    return parity


def _aabb_buckets(lo, hi):
    """Bucket grid over cell bounding boxes (buckets at least as wide as the
    widest box, so a box meets at most 2 buckets per axis): returns
    (origin, width, shape, offsets, cells) with cells[offsets[b]:offsets[b+1]]
    the cells whose box meets bucket b.  A point's bucket lists every cell
    whose box holds the point (floor is monotone)."""
    g0 = lo.min(0)
    h = np.maximum((hi - lo).max(0), 1e-12)
    shape = np.maximum(np.floor((hi.max(0) - g0) / h).astype(np.int64) + 1, 1)
    i0 = np.clip(np.floor((lo - g0) / h).astype(np.int64), 0, shape - 1)
    i1 = np.clip(np.floor((hi - g0) / h).astype(np.int64), 0, shape - 1)
    keys, ids = [], []
    for off in np.ndindex(2, 2, 2):
        b = i0 + np.asarray(off)
        ok = np.all(b <= i1, axis=1)
        keys.append(np.ravel_multi_index(b[ok].T, shape))
        ids.append(np.flatnonzero(ok))
    keys, ids = np.concatenate(keys), np.concatenate(ids)
    srt = np.argsort(keys, kind="stable")
    offsets = np.zeros(int(np.prod(shape)) + 1, np.int64)
    np.add.at(offsets, keys + 1, 1)
    return g0, h, shape, np.cumsum(offsets), ids[srt]


def locate(geo, box, pos):
    """Containing cell of each molecule after wrapping periodic coordinates
    into [0, L).  Returns (cell [n] int32, -1 = outside every cell; wrapped
    positions).  Decisions the FP64 filter cannot certify are redone exactly."""
    pos = _c(pos, np.float64)
    n = pos.shape[0]
    cell = np.zeros(n, np.int32)
    wrapped = np.zeros_like(pos)
    lib().oracle_locate(geo["tri_off"], geo["tri"], geo["lo"], geo["hi"], geo["n_cells"], pos, n,
                        _c(box["L"], np.float64), _c(box["periodic"], np.int32), cell, wrapped)
    undecided = np.flatnonzero(cell == -2)
    if len(undecided):
        g0, h, shape, boff, bcells = _aabb_buckets(geo["lo"], geo["hi"])
        bidx = np.floor((wrapped[undecided] - g0) / h).astype(np.int64)
        inside_grid = np.all((bidx >= 0) & (bidx < shape), axis=1)
        for k, b, ok in zip(undecided, bidx, inside_grid):
            p = wrapped[k]
            cand = []
            if ok:
                bb = np.ravel_multi_index(tuple(b), shape)
                cc = bcells[boff[bb]:boff[bb + 1]]
                cand = cc[np.all((geo["lo"][cc] <= p) & (p <= geo["hi"][cc]), axis=1)]
            hits = [c for c in sorted(cand)
                    if _inside_exact(geo["tri"][geo["tri_off"][c]:geo["tri_off"][c + 1]], p)]
            if len(hits) > 1:
                raise RuntimeError(f"molecule {k} claimed by cells {hits}")
            cell[k] = hits[0] if hits else -1
    return cell, wrapped


def bin_order(cell, n_cells):
    """Counting sort by (cell, original index): order[s] = original index of
    sorted slot s; cell_off[c] = first slot of cell c."""
    order = np.argsort(cell, kind="stable").astype(np.int32)
    cnt = np.bincount(cell, minlength=n_cells)
    cell_off = np.zeros(n_cells + 1, np.int64)
    cell_off[1:] = np.cumsum(cnt)
    return order, cell_off


# ----------------------------------------------------------------------- AICA loops
def aica_loop(lists, cell_off, xs, species_sorted, eps, sigma, rc, box, shift=False):
    """The two force loops of §2.3 (oracle lists, binned molecules).

    Returns dict(F [n,3] in binned order, U, W, counts [6]: evaluated
    {same, dil, referred}, within rc {same, dil, referred})."""
    n = xs.shape[0]
    F = np.zeros((n, 3))
    ev = np.zeros(7)
    counts = np.zeros(6, np.int64)
    C = len(cell_off) - 1
    lib().oracle_aica_loop(C, _c(cell_off, np.int64), _c(xs, np.float64), _c(species_sorted, np.int32),
                           _c(eps, np.float64), _c(sigma, np.float64), float(rc), _c(box["L"], np.float64),
                           int(bool(shift)), _c(lists["dil_off"], np.int64), _c(lists["dil_ids"], np.int32),
                           len(lists["ref_src"]), _c(lists["ref_src"], np.int32),
                           _c(lists["ref_n"], np.int32).reshape(-1), _c(lists["ref_off"], np.int64),
                           _c(lists["ref_ids"], np.int32), F, ev, counts)
    return dict(F=F, U=ev[0], W=ev[1:].copy(), counts=counts)


# ----------------------------------------------------------------- integration
def verlet(pos, vel, species, eps, sigma, mass, rc, box, dt, steps):
    """Velocity-Verlet trajectory with all-pairs FP64 forces (the runs of §3).

    x(t+dt) = x + dt v + dt^2 F(t) / (2m);  v(t+dt) = v + dt (F(t) + F(t+dt)) / (2m).
    Returns dict(pos, vel) at the end and per-step arrays (step 0 = start)
    KE = sum m v^2 / 2, PE = U, P = sum m v.
    """
    x = np.array(pos, dtype=np.float64)
    v = np.array(vel, dtype=np.float64)
    m = np.asarray(mass, dtype=np.float64)[np.asarray(species)][:, None]
    r = lj(x, species, eps, sigma, rc, box)
    F = r["F"]
    KE, PE, P = [0.5 * float((m * v * v).sum())], [r["U"]], [(m * v).sum(0)]
    for _ in range(steps):
        x = x + dt * v + (dt * dt) * F / (2.0 * m)
        r = lj(x, species, eps, sigma, rc, box)
        v = v + dt * (F + r["F"]) / (2.0 * m)
        F = r["F"]
        KE.append(0.5 * float((m * v * v).sum()))
        PE.append(r["U"])
        P.append((m * v).sum(0))
    return dict(pos=x, vel=v, KE=np.array(KE), PE=np.array(PE), P=np.array(P))
