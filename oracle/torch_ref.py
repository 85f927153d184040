"""Autograd-of-oracle reference for the adjoint.  TEST INFRASTRUCTURE ONLY.

Plain PyTorch FP64 CPU ops: the minimum-image LJ force on every molecule as
a differentiable function of positions and the per-species eps and sigma
(Lorentz-Berthelot mixing), so ``torch.autograd.grad`` gives the reference
vector-Jacobian product that the hand-written adjoint must reproduce.  The
set of pairs within rc is chosen once (without gradient) from the given
positions; the gradient of the truncated potential is that of its smooth
part, as for the kernel.
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
