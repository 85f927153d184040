"""Referring transforms of §2.2.2 (TEST INFRASTRUCTURE ONLY).

Plain numpy restatements of the paper's transform algebra, for the oracle of
general (rotational and translational) periodicity:

  rotation(n_a, n_b)   the tensor R_{a b} of §2.2.2 that turns -n_a into n_b,
                       from the coupled faces' unit normals
  coupling(n_a, c_a, n_b, c_b)   the referring transform P' = y + R.P of the
                       coupled faces (y = C_b - R.C_a)
  compose(T2, T1)      T2 after T1: y* = y2 + R2.y1, R* = R2.R1
  inverse(T)           (R^T, -R^T y)
  closure(gens, depth) every distinct composition of at most `depth`
                       generators and their inverses, the identity first

Readings (the paper is silent or the formula degenerates): "(u)^2" is the
outer product u u of u = (n_a x n_b) / |n_a x n_b|; for antiparallel normals
(n_a . n_b = -1) the cross product vanishes and the factor (1 + n_a . n_b)
multiplying it is 0, so R = I; parallel normals (n_a . n_b = +1, a half turn
about an undefined axis) are rejected.  Two transforms are the same when R
and y agree to 1e-9 (the duplicate check of App. A.2).
"""
from __future__ import annotations

import numpy as np

IDENTITY = (np.eye(3), np.zeros(3))


def rotation(n_a, n_b):
    na = np.asarray(n_a, dtype=np.float64)
    nb = np.asarray(n_b, dtype=np.float64)
    na = na / np.linalg.norm(na)
    nb = nb / np.linalg.norm(nb)
    c = float(na @ nb)
    if c > 1.0 - 1e-12:
        raise ValueError("parallel face normals: the rotation axis is undefined")
    if c < -1.0 + 1e-12:
        return np.eye(3)
    u = np.cross(na, nb)
    u = u / np.linalg.norm(u)
    return -c * np.eye(3) + (1.0 + c) * np.outer(u, u) + np.outer(na, nb) - np.outer(nb, na)


def coupling(n_a, c_a, n_b, c_b):
    R = rotation(n_a, n_b)
    return R, np.asarray(c_b, dtype=np.float64) - R @ np.asarray(c_a, dtype=np.float64)


def apply(T, P):
    R, y = T
    return y + np.asarray(P, dtype=np.float64) @ R.T


def compose(T2, T1):
    R2, y2 = T2
    R1, y1 = T1
    return R2 @ R1, y2 + R2 @ y1


def inverse(T):
    R, y = T
    return R.T, -(R.T @ y)


def same(T1, T2, tol=1e-9):
    return np.abs(T1[0] - T2[0]).max() <= tol and np.abs(T1[1] - T2[1]).max() <= tol


def closure(gens, depth):
    """Distinct compositions of at most `depth` generators or their inverses."""
    base = []
    for g in gens:
        for h in (g, inverse(g)):
            if not any(same(h, b) for b in base):
                base.append(h)
    out = [IDENTITY]
    frontier = [IDENTITY]
    for _ in range(depth):
        nxt = []
        for T in frontier:
            for g in base:
                U = compose(g, T)
                if not any(same(U, V) for V in out):
                    out.append(U)
                    nxt.append(U)
        frontier = nxt
    return out
