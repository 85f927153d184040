"""Helpers shared by the GPU parity tests: run the CUDA path through the
binding, and build the oracle's answers for the same seeded inputs."""
import numpy as np
import torch

import oracle
from paper_cs_0702131_gb300.aica import Mesh

DEV = "cuda"


def gpu_setup(cfg, skin=None):
    m = Mesh(cfg["mesh"], cfg["box"])
    m.build_lists(cfg["rc"], cfg["skin"] if skin is None else skin)
    pos = torch.tensor(cfg["pos"], dtype=torch.float64, device=DEV)
    sp = torch.tensor(cfg["species"], dtype=torch.int32, device=DEV)
    cell_of, order, cell_off = m.bin(pos, sp)
    return m, pos, sp, (cell_of.cpu().numpy(), order.cpu().numpy(), cell_off.cpu().numpy())


def oracle_all(cfg, lists=True):
    geo = oracle.cell_geometry(cfg["mesh"])
    out = dict(geo=geo)
    cell, wrapped = oracle.locate(geo, cfg["box"], cfg["pos"])
    order, off = oracle.bin_order(cell, geo["n_cells"])
    out.update(cell=cell, order=order, cell_off=off, xs=wrapped[order])
    if lists:
        L = oracle.cell_lists(cfg["mesh"], cfg["box"], cfg["rc"], cfg["skin"], geo=geo)
        out["lists"] = L
        out["loop"] = oracle.aica_loop(L, off, out["xs"], cfg["species"][order], cfg["eps"], cfg["sigma"],
                                       cfg["rc"], cfg["box"])
    return out


def force_errors(F, ref, idx=None):
    """Per-component force errors against the oracle: the stated tolerance's
    normalisation |dF_ic| / max(|F_ic|, ||F_i||_2), and |dF_ic| / sum_l |f_kl|
    (the condition scale of the sum), as arrays [n, 3]."""
    Fr = ref["F"]
    F = F if idx is None else F[idx]
    d = np.abs(F - Fr)
    norm = np.maximum(np.abs(Fr), np.linalg.norm(Fr, axis=1)[:, None])
    return d / np.maximum(norm, 1e-300), d / np.maximum(ref["Fabs"], 1e-300)[:, None]


def assert_forces(F, ref, tol, idx=None):
    """|F - F_ref| per component <= tol * max(|F_ic|, ||F_i||) for every
    molecule and component (the stated tolerance).  Returns the largest
    error under both normalisations."""
    e_norm, e_abs = force_errors(F, ref, idx)
    bad = np.flatnonzero((e_norm > tol).any(axis=1))
    assert len(bad) == 0, (f"{len(bad)} molecules beyond tol {tol}: max {e_norm.max():.3e} "
                           f"(relative to sum |f|: {e_abs.max():.3e})")
    return e_norm.max(), e_abs.max()


def assert_forces_sum_abs(F, ref, tol, idx=None):
    """|F - F_ref| per component <= tol * sum_l |f_kl|: for paths whose
    forces the library does not certify to the stated tolerance (the cell
    kernel under general referring transforms or the vertex criterion)."""
    e_norm, e_abs = force_errors(F, ref, idx)
    assert e_abs.max() <= tol, f"max force error {e_abs.max():.3e} of sum |f| > {tol}"
    return e_abs.max()


def compare_lists(g, o, cells=None):
    """GPU lists (full) against oracle lists (full, or rows for `cells`)."""
    if cells is None:
        for k in ("dil_off", "dil_ids", "ref_src", "ref_n", "ref_off", "ref_ids"):
            np.testing.assert_array_equal(np.asarray(g[k]).reshape(-1), np.asarray(o[k]).reshape(-1), err_msg=k)
        return
    for j, c in enumerate(cells):
        np.testing.assert_array_equal(g["dil_ids"][g["dil_off"][c]:g["dil_off"][c + 1]],
                                      o["dil_ids"][o["dil_off"][j]:o["dil_off"][j + 1]], err_msg=f"DIL({c})")
    gsel = np.flatnonzero(np.isin(g["ref_src"], cells))
    osel = np.arange(len(o["ref_src"]))
    np.testing.assert_array_equal(g["ref_src"][gsel], o["ref_src"][osel])
    np.testing.assert_array_equal(g["ref_n"][gsel], o["ref_n"][osel])
    for a, b in zip(gsel, osel):
        np.testing.assert_array_equal(g["ref_ids"][g["ref_off"][a]:g["ref_off"][a + 1]],
                                      o["ref_ids"][o["ref_off"][b]:o["ref_off"][b + 1]])
