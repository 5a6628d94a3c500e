"""Error measures for computed P1 solutions (evaluation only, no solver code).

``h1_error`` integrates |grad(U - u)|^2 over the Kuhn simplices of the
structured mesh, with U the piecewise-linear function of the nodal values and u
the exact solution; it is the H^1 seminorm that the paper's success criterion
uses for Poisson (Sec. 7.1, eqs. experiment-successful and
experiment-successful-order with m = 1).  Quadrature: the 6-point degree-4
Dunavant rule on triangles and the 5-point degree-3 rule on tetrahedra
(centroid weight -4/5, four points (1/2,1/6,1/6,1/6) of weight 9/20).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

_TRI = []
for a, w in ((0.445948490915965, 0.223381589678011), (0.091576213509771, 0.109951743655322)):
    for perm in ((a, a, 1 - 2 * a), (a, 1 - 2 * a, a), (1 - 2 * a, a, a)):
        _TRI.append((perm, w))
_TET = [((0.25, 0.25, 0.25, 0.25), -0.8)]
for k in range(4):
    b = [1.0 / 6.0] * 4
    b[k] = 0.5
    _TET.append((tuple(b), 0.45))


def _padded(U: np.ndarray, dim: int) -> np.ndarray:
    """Nodal values including the zero Dirichlet boundary."""
    if dim == 2:
        U = U.reshape(U.shape[-2], U.shape[-1])
        return np.pad(U, 1)
    return np.pad(U, 1)


def h1_seminorm_sq(U: np.ndarray, dim: int) -> float:
    """|U|_{H^1}^2 of the P1 function, equal to U^T A U for the FEM stiffness."""
    V = _padded(U, dim)
    h = 1.0 / (V.shape[-1] - 1)
    tot = 0.0
    for ax in range(dim):
        dif = np.diff(V, axis=ax) / h
        tot += float(np.sum(dif * dif))
    return tot * h ** dim / (1 if dim == 2 else 1) * (1.0)


def h1_error(prob, U: np.ndarray, level: int, zchunk: int = 16) -> float:
    """|U - u|_{H^1} for nodal values U on level ``level`` (interior nodes)."""
    dim = prob.dim
    V = _padded(U, dim)
    n = (1 << level)
    h = 1.0 / n
    grad = prob.exact_grad
    total = 0.0
    if dim == 2:
        V = V  # index [j, i] = y, x
        j0, i0 = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        for path in ((0, 1), (1, 0)):  # axis order of the Kuhn path: 0 = x, 1 = y
            # vertices of the simplex in (x, y) offsets
            verts = [(0, 0)]
            for ax in path:
                v = list(verts[-1])
                v[ax] += 1
                verts.append(tuple(v))
            vals = [V[j0 + vy, i0 + vx] for (vx, vy) in verts]
            G = [None, None]
            for k, ax in enumerate(path):
                G[ax] = (vals[k + 1] - vals[k]) / h
            for bary, w in _TRI:
                px = sum(bary[k] * verts[k][0] for k in range(3))
                py = sum(bary[k] * verts[k][1] for k in range(3))
                gx, gy = grad((i0 + px) * h, (j0 + py) * h)
                total += w * float(np.sum((G[0] - gx) ** 2 + (G[1] - gy) ** 2))
        return math.sqrt(total * h * h / 2.0)
    # 3-D: V indexed [k, j, i] = z, y, x
    for z0 in range(0, n, zchunk):
        z1 = min(n, z0 + zchunk)
        k0, j0, i0 = np.meshgrid(np.arange(z0, z1), np.arange(n), np.arange(n), indexing="ij")
        for path in itertools.permutations(range(3)):
            verts = [(0, 0, 0)]
            for ax in path:
                v = list(verts[-1])
                v[ax] += 1
                verts.append(tuple(v))
            vals = [V[k0 + vz, j0 + vy, i0 + vx] for (vx, vy, vz) in verts]
            G = [None, None, None]
            for k, ax in enumerate(path):
                G[ax] = (vals[k + 1] - vals[k]) / h
            for bary, w in _TET:
                p = [sum(bary[k] * verts[k][a] for k in range(4)) for a in range(3)]
                gx, gy, gz = grad((i0 + p[0]) * h, (j0 + p[1]) * h, (k0 + p[2]) * h)
                total += w * float(np.sum((G[0] - gx) ** 2 + (G[1] - gy) ** 2 + (G[2] - gz) ** 2))
    return math.sqrt(total * h ** 3 / 6.0)


def exact_on_grid(prob, level: int) -> np.ndarray:
    """Exact solution at the interior nodes of ``level`` (shape (1,n,n) or (n,n,n))."""
    n = (1 << level) - 1
    x = (np.arange(n) + 1.0) * 2.0 ** -level
    if prob.dim == 2:
        Y, X = np.meshgrid(x, x, indexing="ij")
        return prob.exact_u(X, Y)[None]
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    return prob.exact_u(X, Y, Z)


def nodal_rel_l2(prob, U: np.ndarray, level: int) -> float:
    ue = exact_on_grid(prob, level)
    return float(np.sqrt(np.mean((U.reshape(ue.shape) - ue) ** 2)) / np.sqrt(np.mean(ue ** 2)))


def h1_error_slabs(prob, decode, level: int, zchunk: int = 8) -> float:
    """``h1_error`` for a 3-D problem, streamed over slabs of z-planes with torch.

    ``decode(z0, nz)`` returns the interior nodal values of planes z0 .. z0+nz-1
    as a float64 torch tensor of shape (nz, n, n) (on the GPU for the full-size
    solutions, which are never held whole); the quadrature is that of
    ``h1_error``, evaluated on the tensor's device.
    """
    import torch
    assert prob.dim == 3
    n = 1 << level  # cubes per axis; padded planes 0 .. n, interior planes 1 .. n-1
    h = 1.0 / n
    total = 0.0
    dev = None
    for z0 in range(0, n, zchunk):
        z1 = min(n, z0 + zchunk)  # cubes z0 .. z1-1 use padded planes z0 .. z1
        lo, hi = max(z0, 1) - 1, min(z1, n - 1) - 1  # interior planes among them
        U = decode(lo, hi - lo + 1)
        dev = U.device
        V = torch.zeros((z1 - z0 + 1, n + 1, n + 1), dtype=torch.float64, device=dev)
        V[lo + 1 - z0: hi + 2 - z0, 1:n, 1:n] = U.reshape(hi - lo + 1, n - 1, n - 1)
        ar = torch.arange(n, dtype=torch.float64, device=dev)
        i0, j0 = ar.view(1, 1, n), ar.view(1, n, 1)
        k0 = torch.arange(z0, z1, dtype=torch.float64, device=dev).view(-1, 1, 1)
        nz = z1 - z0
        for path in itertools.permutations(range(3)):
            verts = [(0, 0, 0)]
            for ax in path:
                v = list(verts[-1])
                v[ax] += 1
                verts.append(tuple(v))
            vals = [V[vz:vz + nz, vy:vy + n, vx:vx + n] for (vx, vy, vz) in verts]
            G = [None, None, None]
            for k, ax in enumerate(path):
                G[ax] = (vals[k + 1] - vals[k]) / h
            for bary, w in _TET:
                p = [sum(bary[k] * verts[k][a] for k in range(4)) for a in range(3)]
                gx, gy, gz = prob.exact_grad((i0 + p[0]) * h, (j0 + p[1]) * h, (k0 + p[2]) * h)
                total += w * float(((G[0] - gx) ** 2 + (G[1] - gy) ** 2 + (G[2] - gz) ** 2).sum())
    return math.sqrt(total * h ** 3 / 6.0)
