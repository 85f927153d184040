"""Autograd-of-oracle reference for the adjoint.  TEST INFRASTRUCTURE ONLY.

Plain PyTorch FP64 CPU ops: the minimum-image LJ force on every molecule as
a differentiable function of positions and the per-species eps and sigma
(Lorentz-Berthelot mixing), so ``torch.autograd.grad`` gives the reference
vector-Jacobian product that the hand-written adjoint must reproduce.  The
set of pairs within rc is chosen once (without gradient) from the given
positions; the gradient of the truncated potential is that of its smooth
part, as for the kernel.  ``image_vjp`` does the same for the force sum over
the images of all molecules under general referring transforms (§2.2.2).
"""
from __future__ import annotations

import numpy as np
import torch


def pair_list(pos, rc, box):
    """Unordered pairs (i < j) within rc under the minimum image (no gradient)."""
    x = torch.as_tensor(np.asarray(pos), dtype=torch.float64)
    L = torch.as_tensor(np.asarray(box["L"], dtype=np.float64))
    per = torch.as_tensor(np.asarray(box["periodic"]).astype(bool))
    n = x.shape[0]
    I, J = [], []
    for s in range(0, n, 512):
        d = x[s:s + 512, None, :] - x[None, :, :]
        d = torch.where(per, d - L * torch.round(d / L), d)
        r2 = (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]
        i, j = torch.nonzero(r2 < rc * rc, as_tuple=True)
        i = i + s
        keep = i < j
        I.append(i[keep])
        J.append(j[keep])
    return torch.cat(I), torch.cat(J)


def forces(pos, species, eps, sigma, box, pairs):
    """F [n,3] as a differentiable function of pos [n,3], eps [S], sigma [S]."""
    I, J = pairs
    L = torch.as_tensor(np.asarray(box["L"], dtype=np.float64))
    per = torch.as_tensor(np.asarray(box["periodic"]).astype(bool))
    sp = torch.as_tensor(np.asarray(species), dtype=torch.long)
    d = pos[I] - pos[J]
    d = torch.where(per, d - L * torch.round(d.detach() / L), d)
    r2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
    a, b = sp[I], sp[J]
    eab = torch.sqrt(eps[a] * eps[b])
    sab = 0.5 * (sigma[a] + sigma[b])
    s = sab * sab / r2
    s3 = s * s * s
    fs = 24.0 * eab * (2.0 * s3 * s3 - s3) / r2
    f = fs[:, None] * d
    F = torch.zeros_like(pos)
    F = F.index_add(0, I, f)
    F = F.index_add(0, J, -f)
    return F


def vjp(pos, species, eps, sigma, rc, box, v):
    """d(sum v . F)/d(pos, eps, sigma) by autograd, FP64."""
    x = torch.tensor(np.asarray(pos), dtype=torch.float64, requires_grad=True)
    e = torch.tensor(np.asarray(eps), dtype=torch.float64, requires_grad=True)
    s = torch.tensor(np.asarray(sigma), dtype=torch.float64, requires_grad=True)
    pairs = pair_list(pos, rc, box)
    F = forces(x, species, e, s, box, pairs)
    vv = torch.as_tensor(np.asarray(v), dtype=torch.float64)
    gx, ge, gs = torch.autograd.grad((F * vv).sum(), (x, e, s))
    return gx.numpy(), ge.numpy(), gs.numpy(), F.detach().numpy()


# ------------------------------------------------------- general transforms
def _is_identity(R, y):
    return bool(np.all(np.asarray(R) == np.eye(3)) and np.all(np.asarray(y) == 0))


def image_terms(pos, rc, transforms):
    """Ordered terms (k, l, t) with |x_k - (y_t + R_t x_l)| < rc, the identity's
    k == l excluded (no gradient): the pair set of the force sum over images
    under general referring transforms (§2.2.2)."""
    x = torch.as_tensor(np.asarray(pos), dtype=torch.float64)
    n = x.shape[0]
    K, Lx, T = [], [], []
    for t, (R, y) in enumerate(transforms):
        Rt = torch.as_tensor(np.asarray(R), dtype=torch.float64)
        yt = torch.as_tensor(np.asarray(y), dtype=torch.float64)
        q = x @ Rt.T + yt
        ident = _is_identity(R, y)
        for s in range(0, n, 512):
            d = x[s:s + 512, None, :] - q[None, :, :]
            r2 = (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]
            k, l = torch.nonzero(r2 < rc * rc, as_tuple=True)
            k = k + s
            if ident:
                keep = k != l
                k, l = k[keep], l[keep]
            K.append(k)
            Lx.append(l)
            T.append(torch.full_like(k, t))
    return torch.cat(K), torch.cat(Lx), torch.cat(T)


def image_forces(pos, species, eps, sigma, transforms, terms):
    """F [n,3] = sum over the terms of f(x_k - (y_t + R_t x_l)) on molecule k, a
    differentiable function of pos, eps and sigma."""
    K, Lx, T = terms
    R = torch.as_tensor(np.array([np.asarray(t[0]) for t in transforms]), dtype=torch.float64)
    y = torch.as_tensor(np.array([np.asarray(t[1]) for t in transforms]), dtype=torch.float64)
    sp = torch.as_tensor(np.asarray(species), dtype=torch.long)
    q = torch.einsum("tij,tj->ti", R[T], pos[Lx]) + y[T]
    d = pos[K] - q
    r2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
    a, b = sp[K], sp[Lx]
    eab = torch.sqrt(eps[a] * eps[b])
    sab = 0.5 * (sigma[a] + sigma[b])
    s = sab * sab / r2
    s3 = s * s * s
    fs = 24.0 * eab * (2.0 * s3 * s3 - s3) / r2
    return torch.zeros_like(pos).index_add(0, K, fs[:, None] * d)


def image_vjp(pos, species, eps, sigma, rc, transforms, v):
    """d(sum v . F)/d(pos, eps, sigma) for the force sum over images, FP64."""
    x = torch.tensor(np.asarray(pos), dtype=torch.float64, requires_grad=True)
    e = torch.tensor(np.asarray(eps), dtype=torch.float64, requires_grad=True)
    s = torch.tensor(np.asarray(sigma), dtype=torch.float64, requires_grad=True)
    F = image_forces(x, species, e, s, transforms, image_terms(pos, rc, transforms))
    vv = torch.as_tensor(np.asarray(v), dtype=torch.float64)
    gx, ge, gs = torch.autograd.grad((F * vv).sum(), (x, e, s))
    return gx.numpy(), ge.numpy(), gs.numpy(), F.detach().numpy()


def vjp_rows(pos, species, eps, sigma, rc, box, v, idx):
    """Rows idx of d(sum v . F)/d pos under the minimum image, for large n:
    only the pairs (k, l) of molecule k depend on x_k, and they add
    (v_k - v_l) . f(x_k - x_l) to sum v . F, so each row is the autograd
    gradient of that sum with the other molecules held fixed."""
    x = torch.as_tensor(np.asarray(pos), dtype=torch.float64)
    vv = torch.as_tensor(np.asarray(v), dtype=torch.float64)
    L = torch.as_tensor(np.asarray(box["L"], dtype=np.float64))
    per = torch.as_tensor(np.asarray(box["periodic"]).astype(bool))
    sp = torch.as_tensor(np.asarray(species), dtype=torch.long)
    e = torch.as_tensor(np.asarray(eps), dtype=torch.float64)
    s = torch.as_tensor(np.asarray(sigma), dtype=torch.float64)
    out = np.zeros((len(idx), 3))
    for row, k in enumerate(np.asarray(idx)):
        d0 = x[k] - x
        d0 = torch.where(per, d0 - L * torch.round(d0 / L), d0)
        r2 = (d0[:, 0] * d0[:, 0] + d0[:, 1] * d0[:, 1]) + d0[:, 2] * d0[:, 2]
        near = torch.nonzero(r2 < rc * rc).flatten()
        near = near[near != int(k)]
        xk = x[k].clone().requires_grad_(True)
        d = xk - x[near]
        d = torch.where(per, d - L * torch.round(d.detach() / L), d)
        r2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
        a, b = sp[k], sp[near]
        eab = torch.sqrt(e[a] * e[b])
        sab = 0.5 * (s[a] + s[b])
        q = sab * sab / r2
        q3 = q * q * q
        fs = 24.0 * eab * (2.0 * q3 * q3 - q3) / r2
        phi = ((vv[k] - vv[near]) * (fs[:, None] * d)).sum()
        (g,) = torch.autograd.grad(phi, xk)
        out[row] = g.numpy()
    return out
