"""Processor referral plan (§2.1, App. A.2) on CPU: the partition, the
per-processor plan against the serial lists, and serial = parallel forces
with the halo exchange run by gloo ranks (the paper's criterion that a
decomposed run reproduces the serial one)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_cs_0702131_gb300 import decomp, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _setup(name="t0", seed=3):
    c = synth.make(name, seed)
    geo = oracle.cell_geometry(c["mesh"])
    lists = oracle.cell_lists(c["mesh"], c["box"], c["rc"], c["skin"], geo=geo)
    cell, pos = oracle.locate(geo, c["box"], c["pos"])
    return c, geo, lists, cell, pos


def test_partition_is_balanced_and_deterministic():
    rng = np.random.default_rng(0)
    cen = rng.uniform(0, 10, size=(1001, 3))
    for P in (1, 2, 3, 4, 7):
        part = decomp.partition(cen, P)
        counts = np.bincount(part, minlength=P)
        assert counts.max() - counts.min() <= 1 and counts.sum() == len(cen)
        np.testing.assert_array_equal(part, decomp.partition(cen, P))
    # a slab splits across its longest extent
    cen = np.stack([np.linspace(0, 100, 50), np.zeros(50), np.zeros(50)], 1)
    part = decomp.partition(cen, 2)
    assert np.all(part[:25] == 0) and np.all(part[25:] == 1)


@pytest.mark.parametrize("P", [2, 3])
def test_halo_molecules_hold_every_partner_of_the_owned(P):
    """Each molecule within rc of an owned molecule (minimum image) is owned
    or in the halo the processor receives, and the halo holds exactly the
    molecules of the plan's received cells."""
    c, geo, lists, cell, pos = _setup()
    part = decomp.partition(geo["ctr"], P)
    L = np.asarray(c["box"]["L"], float)
    d = pos[:, None, :] - pos[None, :, :]
    d -= L * np.rint(d / L)
    near = (d ** 2).sum(-1) < c["rc"] ** 2
    np.fill_diagonal(near, False)
    for r in range(P):
        plan = decomp.halo_plan(lists, part, r)
        owned = part[cell] == r
        halo = decomp.halo_molecules(plan, cell)
        recv = np.concatenate(list(plan["recv"].values())) if plan["recv"] else np.zeros(0, np.int64)
        np.testing.assert_array_equal(halo, np.flatnonzero(np.isin(cell, recv)))
        assert not owned[halo].any()
        have = owned.copy()
        have[halo] = True
        partners = near[owned].any(axis=0)
        assert np.all(have[partners]), f"rank {r}: {int((partners & ~have).sum())} partners missing"


def test_plans_cover_every_interaction_once():
    c, geo, lists, _, _ = _setup()
    P = 3
    part = decomp.partition(geo["ctr"], P)
    plans = [decomp.halo_plan(lists, part, r) for r in range(P)]
    a = np.repeat(np.arange(len(lists["dil_off"]) - 1), np.diff(lists["dil_off"]))
    b = np.asarray(lists["dil_ids"], np.int64)
    entries = {}
    for r, p in enumerate(plans):
        np.testing.assert_array_equal(p["local"], np.flatnonzero(part == r))
        for i, j in zip(p["dil_a"], p["dil_b"]):
            entries[("dil", int(i), int(j))] = entries.get(("dil", int(i), int(j)), 0) + 1
        for k in range(len(p["ref_src"])):
            for J in p["ref_ids"][p["ref_off"][k]:p["ref_off"][k + 1]]:
                key = ("ref", int(p["ref_src"][k]), *map(int, p["ref_n"][k]), int(J))
                assert part[J] == r
                entries[key] = entries.get(key, 0) + 1
        owners = p["ref_owner"]
        for s, cells in p["recv"].items():
            assert s != r
            np.testing.assert_array_equal(cells, np.unique(p["ref_src"][owners == s]))
    expected = {}
    for i, j in zip(a, b):
        if part[i] == part[j]:
            expected[("dil", int(i), int(j))] = 1
        else:                      # one-sided on each side, as a referred cell with n = 0
            expected[("ref", int(j), 0, 0, 0, int(i))] = 1
            expected[("ref", int(i), 0, 0, 0, int(j))] = 1
    for k in range(len(lists["ref_src"])):
        for J in lists["ref_ids"][lists["ref_off"][k]:lists["ref_off"][k + 1]]:
            expected[("ref", int(lists["ref_src"][k]), *map(int, lists["ref_n"][k]), int(J))] = 1
    assert entries == expected
    # what a processor sends is what the others receive from it
    for r in range(P):
        for dest, cells in decomp.send_lists(plans, r).items():
            np.testing.assert_array_equal(cells, plans[dest]["recv"][r])
            assert np.all(part[cells] == r)


def _pair_terms(xp, sp, xq, sq, eps, sig, rc, upper):
    """Forces on the first set, energy and virial of all pairs within rc (the
    second set already shifted into place); upper: only k < l (one cell)."""
    d = xp[:, None, :] - xq[None, :, :]
    r2 = (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]
    m = r2 < rc * rc
    if upper:
        m &= np.triu(np.ones(m.shape, bool), 1)
    e = np.sqrt(eps[sp][:, None] * eps[sq][None, :])
    s = 0.5 * (sig[sp][:, None] + sig[sq][None, :])
    with np.errstate(divide="ignore", invalid="ignore"):
        q = np.where(m, s * s / np.where(m, r2, 1.0), 0.0)
        q3 = q * q * q
        fs = np.where(m, 24.0 * e * (2.0 * q3 * q3 - q3) / np.where(m, r2, 1.0), 0.0)
        u = np.where(m, 4.0 * e * (q3 * q3 - q3), 0.0)
    f = fs[..., None] * d
    w = np.array([(d[..., 0] * f[..., 0]).sum(), (d[..., 1] * f[..., 1]).sum(), (d[..., 2] * f[..., 2]).sum(),
                  (d[..., 0] * f[..., 1]).sum(), (d[..., 0] * f[..., 2]).sum(), (d[..., 1] * f[..., 2]).sum()])
    return f.sum(axis=1), f.sum(axis=0), u.sum(), w


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    c, geo, lists, cell, pos = _setup()
    eps, sig, rc, L = c["eps"], c["sigma"], c["rc"], c["box"]["L"]
    sp_all = np.asarray(c["species"])
    part = decomp.partition(geo["ctr"], world)
    plans = [decomp.halo_plan(lists, part, r) for r in range(world)]
    plan = plans[rank]
    # this processor holds the molecules of its own cells only
    mine = {int(k): np.flatnonzero(cell == k) for k in plan["local"]}
    # halo exchange: per destination, the molecule counts of the sent cells, then positions and species
    reqs, keep = [], []
    for dest, cells in decomp.send_lists(plans, rank).items():
        idx = np.concatenate([mine[int(k)] for k in cells]) if len(cells) else np.zeros(0, np.int64)
        cnt = torch.tensor([len(mine[int(k)]) for k in cells], dtype=torch.int64)
        xs = torch.tensor(pos[idx], dtype=torch.float64)
        ss = torch.tensor(sp_all[idx], dtype=torch.int64)
        keep += [cnt, xs, ss]
        reqs += [dist.isend(cnt, dest), dist.isend(torch.tensor([len(idx)], dtype=torch.int64), dest)]
    halo = {}
    for src, cells in plan["recv"].items():
        cnt = torch.empty(len(cells), dtype=torch.int64)
        tot = torch.empty(1, dtype=torch.int64)
        dist.recv(cnt, src)
        dist.recv(tot, src)
        halo[src] = (cells, cnt, int(tot.item()))
    for r_ in reqs:
        r_.wait()
    reqs = []
    for k, dest in enumerate(decomp.send_lists(plans, rank)):
        _, xs, ss = keep[3 * k:3 * k + 3]
        reqs += [dist.isend(xs, dest), dist.isend(ss, dest)]
    remote = {}
    for src, (cells, cnt, tot) in halo.items():
        xs = torch.empty((tot, 3), dtype=torch.float64)
        ss = torch.empty(tot, dtype=torch.int64)
        dist.recv(xs, src)
        dist.recv(ss, src)
        o = 0
        for cc, n in zip(cells, cnt.tolist()):
            remote[int(cc)] = (xs[o:o + n].numpy(), ss[o:o + n].numpy())
            o += n
    for r_ in reqs:
        r_.wait()

    def molecules(cc):
        cc = int(cc)
        if cc in mine:
            return pos[mine[cc]], sp_all[mine[cc]]
        return remote[cc]

    F = {k: np.zeros((len(v), 3)) for k, v in mine.items()}
    U, W = 0.0, np.zeros(6)
    for k, idx in mine.items():              # same-cell pairs, Newton's third law
        x, s = pos[idx], sp_all[idx]
        fp, fq, u, w = _pair_terms(x, s, x, s, eps, sig, rc, upper=True)
        F[k] += fp - fq
        U += u
        W += w
    for i, j in zip(plan["dil_a"], plan["dil_b"]):   # local DIL pairs, Newton's third law
        fp, fq, u, w = _pair_terms(pos[mine[int(i)]], sp_all[mine[int(i)]], pos[mine[int(j)]], sp_all[mine[int(j)]],
                                   eps, sig, rc, upper=False)
        F[int(i)] += fp
        F[int(j)] -= fq
        U += u
        W += w
    for r_ in range(len(plan["ref_src"])):     # referred cells: one-sided, half the energy and virial
        xq, sq = molecules(plan["ref_src"][r_])
        xq = xq + plan["ref_n"][r_] * L
        for J in plan["ref_ids"][plan["ref_off"][r_]:plan["ref_off"][r_ + 1]]:
            fp, _, u, w = _pair_terms(pos[mine[int(J)]], sp_all[mine[int(J)]], xq, sq, eps, sig, rc, upper=False)
            F[int(J)] += fp
            U += 0.5 * u
            W += 0.5 * w
    sums = torch.tensor([U, *W], dtype=torch.float64)
    dist.all_reduce(sums)
    gathered = [None] * world
    dist.all_gather_object(gathered, {int(g): f for k, idx in mine.items() for g, f in zip(idx, F[k])})
    if rank == 0:
        out["F"] = {g: f for part_ in gathered for g, f in part_.items()}
        out["sums"] = sums.numpy()
        out["halo_cells"] = sum(len(v) for v in plan["recv"].values())
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_serial_equals_parallel(world):
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    c = synth.make("t0", 3)
    ref = oracle.lj(c["pos"], c["species"], c["eps"], c["sigma"], c["rc"], c["box"])
    F = np.array([out["F"][g] for g in range(len(c["pos"]))])
    assert np.abs(F - ref["F"]).max() <= 1e-12 * ref["Fabs"].max()
    assert abs(out["sums"][0] - ref["U"]) <= 1e-12 * ref["Uabs"]
    assert np.all(np.abs(out["sums"][1:] - ref["W"]) <= 1e-12 * ref["Wabs"])
    assert out["halo_cells"] > 0
