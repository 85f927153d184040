"""Processor referral plan for a spatial decomposition (§2.1, App. A.2).

Host-side logic of the multi-GPU path: the mesh's cells are split into
portions, one per processor, and each processor evaluates the forces on the
molecules of its own cells.  A cell pair of the direct interaction lists
whose cells lie on two processors becomes, on each side, a processor-
referred cell (the remote cell, image n = 0) acting on the local cell only;
a periodic referred cell (c, n) stays a referred cell on the processor that
owns its real cells, whether its source c is local or remote.  One-sided
evaluations carry half the pair's energy and virial (§2.3), so the sums over
processors equal the serial ones.  Each step the owner of every source cell
sends its molecules to the processors that refer it (the halo exchange;
there is no reverse force exchange).

The plan is derived here from the interaction lists of the whole mesh (the
CSR arrays of ``aica_get_lists`` / ``Mesh.lists()``), so the paper's
iterative referral between processors reduces to set operations: a referred
cell is keyed by (source cell, n), which makes App. A.2's duplicate check
hold by construction.

On the GPU a portion is evaluated by the library itself: every processor
holds the whole mesh and its lists, bins its own molecules followed by the
halo it received (the molecules of ``recv``'s cells, at their own
positions) with the option ``n_owned`` set to the number of its own, and
``aica_forces`` evaluates owned-owned pairs with Newton's third law and
owned-halo pairs one-sidedly with half their energy and virial (the
referred pairs of this plan).  The exchange between processors needs more
than one GPU; it is exercised on CPU ranks (gloo) in the tests, and the GPU
evaluation of every portion in one process.
"""
from __future__ import annotations

import numpy as np


def partition(centroids, n_parts):
    """Recursive coordinate bisection of the cell centroids into n_parts
    portions whose cell counts differ by at most one; returns the portion of
    every cell (int32).  Each split cuts the current set along its longest
    extent at the position that gives the two halves their share of parts."""
    c = np.asarray(centroids, dtype=np.float64).reshape(-1, 3)
    if n_parts < 1:
        raise ValueError("n_parts must be >= 1")
    part = np.zeros(len(c), np.int32)

    def split(idx, first, k):
        if k == 1 or len(idx) == 0:
            part[idx] = first
            return
        ext = c[idx].max(axis=0) - c[idx].min(axis=0)
        ax = int(np.argmax(ext))
        order = idx[np.lexsort((idx, c[idx, ax]))]      # ties by cell id: deterministic
        k1 = k // 2
        cut = (len(order) * k1) // k
        split(order[:cut], first, k1)
        split(order[cut:], first + k1, k - k1)

    split(np.arange(len(c)), 0, int(n_parts))
    return part


def _dil_pairs(lists):
    off = np.asarray(lists["dil_off"], np.int64)
    a = np.repeat(np.arange(len(off) - 1), np.diff(off))
    return a, np.asarray(lists["dil_ids"], np.int64)


def halo_plan(lists, part, rank):
    """What processor `rank` evaluates and receives each step.

    Returns a dict:
      local      ascending local cells
      dil_a, dil_b   DIL pairs with both cells local (Newton's third law)
      ref_src, ref_n, ref_owner   referred cells (source cell, image vector,
                 owner of the source), sorted by (source, n)
      ref_off, ref_ids   CSR: the ascending local cells each referred cell
                 acts on (one-sided)
      recv       {source processor: ascending source cells to receive}
    """
    part = np.asarray(part)
    a, b = _dil_pairs(lists)
    pa, pb = part[a], part[b]
    both = (pa == rank) & (pb == rank)
    refs = {}
    # cross-processor DIL pairs: the remote cell is referred with n = 0, on each side
    for i, j in zip(a[(pa == rank) & (pb != rank)], b[(pa == rank) & (pb != rank)]):
        refs.setdefault((int(j), 0, 0, 0), set()).add(int(i))
    for i, j in zip(a[(pb == rank) & (pa != rank)], b[(pb == rank) & (pa != rank)]):
        refs.setdefault((int(i), 0, 0, 0), set()).add(int(j))
    # periodic referred cells whose real cells are local
    ref_src = np.asarray(lists["ref_src"], np.int64)
    ref_n = np.asarray(lists["ref_n"], np.int64).reshape(-1, 3)
    ref_off = np.asarray(lists["ref_off"], np.int64)
    ref_ids = np.asarray(lists["ref_ids"], np.int64)
    for r in range(len(ref_src)):
        J = ref_ids[ref_off[r]:ref_off[r + 1]]
        J = J[part[J] == rank]
        if len(J):
            refs.setdefault((int(ref_src[r]), *map(int, ref_n[r])), set()).update(map(int, J))
    keys = sorted(refs)
    src = np.array([k[0] for k in keys], np.int64)
    nvec = np.array([k[1:] for k in keys], np.int64).reshape(-1, 3)
    ids = [np.array(sorted(refs[k]), np.int64) for k in keys]
    off = np.concatenate([[0], np.cumsum([len(x) for x in ids])]).astype(np.int64)
    owner = part[src] if len(src) else np.zeros(0, part.dtype)
    recv = {}
    for s in sorted(set(int(o) for o in owner) - {int(rank)}):
        recv[s] = np.unique(src[owner == s])
    return dict(local=np.flatnonzero(part == rank), dil_a=a[both], dil_b=b[both], ref_src=src, ref_n=nvec,
                ref_owner=owner, ref_off=off, ref_ids=np.concatenate(ids) if ids else np.zeros(0, np.int64),
                recv=recv)


def halo_molecules(plan, cell_of):
    """Indices of the molecules `rank` receives (those of the cells in
    plan["recv"]), from every molecule's cell."""
    cells = np.concatenate(list(plan["recv"].values())) if plan["recv"] else np.zeros(0, np.int64)
    return np.flatnonzero(np.isin(np.asarray(cell_of), cells))


def send_lists(plans, rank):
    """{destination processor: ascending cells of `rank` it receives}, from
    every processor's plan (what `rank` must send each step)."""
    out = {}
    for dest, p in enumerate(plans):
        if dest != rank and rank in p["recv"]:
            out[dest] = p["recv"][rank]
    return out
