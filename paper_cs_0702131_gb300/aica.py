"""Thin ctypes binding of ``libaica.so`` (argument marshalling only).

The functions below carry the names of the C ABI in ``include/aica.h`` and
forward to it; every compute step runs in the library's CUDA kernels.  Device
arrays are torch CUDA tensors (torch provides device memory and the stream:
calls are issued on ``torch.cuda.current_stream()``).  There is no CPU
fallback: if the library is missing, :func:`lib` raises.

:class:`Mesh` wraps a mesh handle; :class:`LJForce` is the
``torch.autograd.Function`` whose backward is the hand-written adjoint
kernel (``aica_forces_backward``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import build as _build

_lib = None

AICA_FP32, AICA_FP64 = 0, 1
STATUS = {0: "AICA_OK", 1: "AICA_ERR_INVALID_ARG", 2: "AICA_ERR_BAD_MESH", 3: "AICA_ERR_OUTSIDE_MESH",
          4: "AICA_ERR_NOT_BUILT", 5: "AICA_ERR_CAPACITY", 6: "AICA_ERR_CUDA", 7: "AICA_ERR_OOM"}


class AicaError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status
        self.name = STATUS.get(status, str(status))


class Box(ctypes.Structure):
    _fields_ = [("L", ctypes.c_double * 3), ("periodic", ctypes.c_int32 * 3)]


class LJ(ctypes.Structure):
    _fields_ = [("n_species", ctypes.c_int32), ("eps", ctypes.POINTER(ctypes.c_double)),
                ("sigma", ctypes.POINTER(ctypes.c_double)), ("shift", ctypes.c_int32)]


class ListInfo(ctypes.Structure):
    _fields_ = [("n_cells", ctypes.c_int64), ("n_dil", ctypes.c_int64), ("n_ref", ctypes.c_int64),
                ("n_ref_ids", ctypes.c_int64), ("n_ties", ctypes.c_int64), ("rc", ctypes.c_double),
                ("skin", ctypes.c_double), ("criterion", ctypes.c_int32)]


#: every entry point of include/aica.h with its ctypes signature
SIGNATURES = {
    "aica_mesh_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                        ctypes.POINTER(Box), ctypes.POINTER(ctypes.c_void_p)]),
    "aica_mesh_destroy": (None, [ctypes.c_void_p]),
    "aica_build_interaction_list_ex": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                                      ctypes.c_int, ctypes.c_void_p]),
    "aica_build_interaction_list": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                                   ctypes.c_void_p]),
    "aica_get_list_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ListInfo)]),
    "aica_get_lists": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_void_p] * 6),
    "aica_bin_molecules": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "aica_forces": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(LJ), ctypes.c_int, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "aica_forces_backward": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(LJ), ctypes.c_int, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "aica_set_deferred_checks": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "aica_check_status": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "aica_last_launch_count": (ctypes.c_int64, [ctypes.c_void_p]),
    "aica_get_work_counters": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "aica_set_kernel_timing": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "aica_take_kernel_times": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                              ctypes.POINTER(ctypes.c_int64)]),
    "aica_sort_by_cell_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                                                 ctypes.c_void_p, ctypes.c_void_p]),
    "aica_probe_fma_rate": (ctypes.c_int, [ctypes.c_int, ctypes.c_int64, ctypes.POINTER(ctypes.c_double),
                                           ctypes.c_void_p]),
    "aica_verlet_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(LJ), ctypes.c_int, ctypes.c_void_p,
                                        ctypes.c_double, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p]),
    "aica_kinetic": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p]),
    "aica_mesh_set_transforms": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "aica_coupling_transform": (ctypes.c_int, [ctypes.c_void_p] * 6),
    "aica_set_option": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_double]),
    "aica_get_option": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                       ctypes.c_void_p]),
    "aica_last_error": (ctypes.c_char_p, []),
    "aica_status_string": (ctypes.c_char_p, [ctypes.c_int]),
}


def lib_path():
    return _build.LIB


def lib():
    """Load the in-tree CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libaica.so is missing ({path}); run paper_cs_0702131_gb300.build.build()")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status):
    if status != 0:
        raise AicaError(status, lib().aica_last_error().decode())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _dev(t, dtype, shape=None, name="tensor"):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous CUDA tensor of {dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return t


def _lj(eps, sigma, shift):
    e = np.ascontiguousarray(eps, dtype=np.float64)
    s = np.ascontiguousarray(sigma, dtype=np.float64)
    st = LJ(len(e), e.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
            s.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(bool(shift)))
    st._keep = (e, s)
    return st


# ---------------------------------------------------------------- C-ABI names
def aica_mesh_create(points, face_offsets, face_vertices, owner, neighbour, n_cells, L, periodic):
    """Host arrays in, opaque handle out (see include/aica.h)."""
    P = np.ascontiguousarray(points, dtype=np.float64)
    fo = np.ascontiguousarray(face_offsets, dtype=np.int64)
    fv = np.ascontiguousarray(face_vertices, dtype=np.int64)
    ow = np.ascontiguousarray(owner, dtype=np.int64)
    nb = np.ascontiguousarray(neighbour, dtype=np.int64)
    box = Box((ctypes.c_double * 3)(*[float(x) for x in L]), (ctypes.c_int32 * 3)(*[int(x) for x in periodic]))
    h = ctypes.c_void_p()
    _check(lib().aica_mesh_create(P.ctypes.data, P.shape[0], fo.ctypes.data, fv.ctypes.data, ow.shape[0],
                                  ow.ctypes.data, nb.ctypes.data, int(n_cells), ctypes.byref(box), ctypes.byref(h)))
    return h


def aica_mesh_destroy(h):
    lib().aica_mesh_destroy(h)


AICA_DIL_MIN_DISTANCE, AICA_DIL_VERTEX = 0, 1
_CRITERIA = {"min_distance": AICA_DIL_MIN_DISTANCE, "vertex": AICA_DIL_VERTEX}


def aica_build_interaction_list(h, rc, skin=1e-3):
    _check(lib().aica_build_interaction_list(h, float(rc), float(skin), _stream()))


def aica_build_interaction_list_ex(h, rc, skin=1e-3, criterion="min_distance"):
    """criterion: "min_distance" (default) or "vertex" (the paper's vertex-vertex search)."""
    _check(lib().aica_build_interaction_list_ex(h, float(rc), float(skin), _CRITERIA[criterion], _stream()))


def aica_get_list_info(h):
    info = ListInfo()
    _check(lib().aica_get_list_info(h, ctypes.byref(info)))
    return info


def aica_get_lists(h):
    info = aica_get_list_info(h)
    C, nd, nr, nri = info.n_cells, info.n_dil, info.n_ref, info.n_ref_ids
    out = dict(dil_off=np.zeros(C + 1, np.int64), dil_ids=np.zeros(max(nd, 1), np.int32),
               ref_src=np.zeros(max(nr, 1), np.int32), ref_n=np.zeros((max(nr, 1), 3), np.int32),
               ref_off=np.zeros(nr + 1, np.int64), ref_ids=np.zeros(max(nri, 1), np.int32))
    _check(lib().aica_get_lists(h, *[out[k].ctypes.data for k in
                                     ("dil_off", "dil_ids", "ref_src", "ref_n", "ref_off", "ref_ids")]))
    out["dil_ids"] = out["dil_ids"][:nd]
    out["ref_src"] = out["ref_src"][:nr]
    out["ref_n"] = out["ref_n"][:nr]
    out["ref_ids"] = out["ref_ids"][:nri]
    out["ties"] = info.n_ties
    return out


def aica_bin_molecules(h, pos, species, cell_of=None, order=None, cell_off=None):
    n = pos.shape[0]
    _dev(pos, torch.float64, (n, 3), "pos")
    _dev(species, torch.int32, (n,), "species")
    _check(lib().aica_bin_molecules(h, _ptr(pos), _ptr(species), n, _ptr(cell_of), _ptr(order), _ptr(cell_off),
                                    _stream()))


def aica_forces(h, eps, sigma, prec, force_out, ev_out=None, counts_out=None, shift=False):
    lj = _lj(eps, sigma, shift)
    _check(lib().aica_forces(h, ctypes.byref(lj), int(prec), _ptr(force_out), _ptr(ev_out), _ptr(counts_out),
                             _stream()))


def aica_forces_backward(h, eps, sigma, prec, grad_force, grad_pos, grad_eps=None, grad_sigma=None):
    lj = _lj(eps, sigma, False)
    _check(lib().aica_forces_backward(h, ctypes.byref(lj), int(prec), _ptr(grad_force), _ptr(grad_pos),
                                      _ptr(grad_eps), _ptr(grad_sigma), _stream()))


def aica_verlet_step(h, eps, sigma, prec, mass, dt, species, pos, vel, force, ev_out=None, kin_out=None,
                     shift=False):
    lj = _lj(eps, sigma, shift)
    ms = np.ascontiguousarray(mass, dtype=np.float64)
    if len(ms) != lj.n_species:
        raise ValueError("need one mass per species")
    _check(lib().aica_verlet_step(h, ctypes.byref(lj), int(prec), ms.ctypes.data, float(dt), pos.shape[0],
                                  _ptr(species), _ptr(pos), _ptr(vel), _ptr(force), _ptr(ev_out), _ptr(kin_out),
                                  _stream()))


def aica_kinetic(mass, species, vel, kin_out):
    ms = np.ascontiguousarray(mass, dtype=np.float64)
    _check(lib().aica_kinetic(ms.ctypes.data, len(ms), _ptr(species), vel.shape[0], _ptr(vel), _ptr(kin_out),
                              _stream()))


def aica_mesh_set_transforms(h, transforms):
    """transforms: list of (R [3,3], y [3]) referring transforms P' = y + R.P."""
    R = np.ascontiguousarray(np.array([t[0] for t in transforms], dtype=np.float64).reshape(-1))
    y = np.ascontiguousarray(np.array([t[1] for t in transforms], dtype=np.float64).reshape(-1))
    _check(lib().aica_mesh_set_transforms(h, len(transforms), R.ctypes.data if len(transforms) else None,
                                          y.ctypes.data if len(transforms) else None))


def aica_coupling_transform(n_alpha, c_alpha, n_beta, c_beta):
    """(R [3,3], y [3]) of the coupled faces (normals, centres) by §2.2.2."""
    args = [np.ascontiguousarray(v, dtype=np.float64) for v in (n_alpha, c_alpha, n_beta, c_beta)]
    R = np.zeros(9)
    y = np.zeros(3)
    _check(lib().aica_coupling_transform(*[a.ctypes.data for a in args], R.ctypes.data, y.ctypes.data))
    return R.reshape(3, 3), y


def aica_sort_by_cell_noalloc(cell_of, n_cells, order, cell_off):
    """Counting sort by cell with no device allocation (see include/aica.h)."""
    n = cell_of.shape[0]
    _dev(cell_of, torch.int32, (n,), "cell_of")
    _dev(order, torch.int32, (n,), "order")
    _dev(cell_off, torch.int32, (int(n_cells) + 1,), "cell_off")
    _check(lib().aica_sort_by_cell_noalloc(_ptr(cell_of), n, int(n_cells), _ptr(order), _ptr(cell_off), _stream()))


OPTIONS = {"fp32_refine_tol": 0, "count_evaluated": 1, "fp32_kernel": 2, "refined": 3, "cluster_path": 4,
           "n_owned": 5}


def aica_set_option(h, name, value):
    _check(lib().aica_set_option(h, OPTIONS[name], float(value)))


def aica_get_option(h, name):
    v = ctypes.c_double(0)
    _check(lib().aica_get_option(h, OPTIONS[name], ctypes.byref(v), _stream()))
    return v.value


def aica_set_deferred_checks(h, deferred):
    _check(lib().aica_set_deferred_checks(h, int(bool(deferred))))


def aica_check_status(h):
    _check(lib().aica_check_status(h, _stream()))


def aica_last_launch_count(h):
    return int(lib().aica_last_launch_count(h))


def aica_get_work_counters(h):
    out = np.zeros(2, np.int64)
    _check(lib().aica_get_work_counters(h, out.ctypes.data, _stream()))
    return out


def aica_set_kernel_timing(h, enable):
    _check(lib().aica_set_kernel_timing(h, int(bool(enable))))


def aica_take_kernel_times(h, cap=1 << 16):
    ms = np.zeros(cap, np.float32)
    n = ctypes.c_int64()
    _check(lib().aica_take_kernel_times(h, ms.ctypes.data, cap, ctypes.byref(n)))
    return ms[: n.value].copy()


def aica_probe_fma_rate(fp64, iters):
    """Measured FMA rate of the current device in flop/s (FP64 if fp64)."""
    out = ctypes.c_double()
    _check(lib().aica_probe_fma_rate(int(bool(fp64)), int(iters), ctypes.byref(out), _stream()))
    return out.value


# ---------------------------------------------------------------- convenience
def _prec(p):
    if p in ("fp32", AICA_FP32, torch.float32):
        return AICA_FP32, torch.float32
    if p in ("fp64", AICA_FP64, torch.float64):
        return AICA_FP64, torch.float64
    raise ValueError(f"precision must be fp32 or fp64, got {p!r}")


class Mesh:
    """A library-owned mesh with its lists and binned molecules.

    ``mesh`` is the face-based dict of :mod:`paper_cs_0702131_gb300.synth`
    (points, face_offsets, face_vertices, owner, neighbour, n_cells) and
    ``box`` a dict with ``L`` and ``periodic``.
    """

    def __init__(self, mesh, box):
        self.n_cells = int(mesh["n_cells"])
        self.box = box
        self.h = aica_mesh_create(mesh["points"], mesh["face_offsets"], mesh["face_vertices"], mesh["owner"],
                                  mesh["neighbour"], self.n_cells, box["L"], box["periodic"])
        self.n = 0
        self.rc = None
        self.generation = 0
        self.deferred = False

    def close(self):
        if getattr(self, "h", None):
            aica_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_transforms(self, transforms):
        """General periodic boundaries: list of (R, y) referring transforms."""
        aica_mesh_set_transforms(self.h, transforms)

    def build_lists(self, rc, skin=1e-3, criterion="min_distance"):
        if criterion == "min_distance":
            aica_build_interaction_list(self.h, rc, skin)
        else:
            aica_build_interaction_list_ex(self.h, rc, skin, criterion)
        self.rc = float(rc)

    def lists(self):
        return aica_get_lists(self.h)

    def bin(self, pos, species, outputs=True):
        """Bin molecules; returns (cell_of, order, cell_off) device tensors if outputs."""
        n = pos.shape[0]
        outs = (None, None, None)
        if outputs:
            dev = pos.device
            outs = (torch.empty(n, dtype=torch.int32, device=dev), torch.empty(n, dtype=torch.int32, device=dev),
                    torch.empty(self.n_cells + 1, dtype=torch.int32, device=dev))
        aica_bin_molecules(self.h, pos, species, *outs)
        self.n = n
        self.generation += 1
        return outs if outputs else None

    def forces(self, eps, sigma, prec="fp32", shift=False, out=None, ev=None, counts=None):
        """Forces (original order), energy + virial (7, FP64) and pair counts (6, int64)."""
        p, dt = _prec(prec)
        dev = torch.device("cuda", torch.cuda.current_device())
        F = out if out is not None else torch.empty((self.n, 3), dtype=dt, device=dev)
        ev = ev if ev is not None else torch.empty(7, dtype=torch.float64, device=dev)
        counts = counts if counts is not None else torch.empty(6, dtype=torch.int64, device=dev)
        aica_forces(self.h, eps, sigma, p, F, ev, counts, shift)
        return F, ev, counts

    def forces_backward(self, eps, sigma, grad_force, prec="fp32"):
        p, dt = _prec(prec)
        g = _dev(grad_force.contiguous(), dt, (self.n, 3), "grad_force")
        gp = torch.empty_like(g)
        S = len(np.atleast_1d(eps))
        ge = torch.empty(S, dtype=torch.float64, device=g.device)
        gs = torch.empty(S, dtype=torch.float64, device=g.device)
        aica_forces_backward(self.h, eps, sigma, p, g, gp, ge, gs)
        return gp, ge, gs

    def verlet_step(self, eps, sigma, mass, dt, pos, vel, species, force, prec="fp64", ev=None, kin=None,
                    shift=False):
        """One velocity-Verlet step (aica_verlet_step): pos, vel (FP64, device,
        original order) updated in place; force holds F(t) on entry and
        F(t + dt) on return (float32 for "fp32", float64 for "fp64")."""
        p, dt_ = _prec(prec)
        pos = _dev(pos, torch.float64, (self.n, 3), "pos")
        vel = _dev(vel, torch.float64, (self.n, 3), "vel")
        force = _dev(force, dt_, (self.n, 3), "force")
        species = _dev(species, torch.int32, (self.n,), "species")
        aica_verlet_step(self.h, eps, sigma, p, mass, dt, species, pos, vel, force, ev, kin, shift)

    def set_deferred(self, deferred=True):
        """Deferred device-side checks: errors accumulate until check()."""
        aica_set_deferred_checks(self.h, deferred)
        self.deferred = bool(deferred)

    def set_option(self, name, value):
        aica_set_option(self.h, name, value)

    def get_option(self, name):
        return aica_get_option(self.h, name)

    def set_kernel_timing(self, enable=True):
        aica_set_kernel_timing(self.h, enable)

    def last_stats(self):
        """[pair distance tests, sphere tests] of the last forces call."""
        return aica_get_work_counters(self.h)

    def take_kernel_times(self):
        """Durations (ms) of the pair kernels recorded since the last take."""
        return aica_take_kernel_times(self.h)

    def check(self):
        aica_check_status(self.h)


class LJForce(torch.autograd.Function):
    """F(pos, eps, sigma) over the AICA pair set; backward = adjoint kernel.

    ``pos`` is [N,3] float64 on the GPU (binning input); ``eps``/``sigma`` are
    per-species CPU or GPU tensors.  The returned forces have the dtype of
    ``prec``.
    """

    @staticmethod
    def forward(ctx, pos, eps, sigma, mesh, species, prec):
        e = eps.detach().double().cpu().numpy()
        s = sigma.detach().double().cpu().numpy()
        mesh.bin(pos.detach().contiguous(), species, outputs=False)
        F, ev, counts = mesh.forces(e, s, prec)
        ctx.mesh, ctx.prec, ctx.e, ctx.s = mesh, prec, e, s
        ctx.gen = mesh.generation
        ctx.species = species
        ctx.save_for_backward(pos)
        ctx.dev = (eps.device, sigma.device, eps.dtype)
        return F

    @staticmethod
    def backward(ctx, gF):
        (pos,) = ctx.saved_tensors
        mesh = ctx.mesh
        if mesh.generation != ctx.gen:          # the mesh was re-binned since forward
            mesh.bin(pos.detach().contiguous(), ctx.species, outputs=False)
        _, dt = _prec(ctx.prec)
        gp, ge, gs = mesh.forces_backward(ctx.e, ctx.s, gF.to(dt).contiguous(), ctx.prec)
        edev, sdev, edt = ctx.dev
        return gp.to(pos.dtype), ge.to(edev, edt), gs.to(sdev, edt), None, None, None
