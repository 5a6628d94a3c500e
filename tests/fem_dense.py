"""Dense finite-element matrices for tiny grids, built from first principles.

Independent of the oracle's stencil code: the stiffness matrix is assembled
element by element from barycentric gradients of the Kuhn simplices, and the
prolongation evaluates the coarse piecewise-linear function at the fine nodes by
locating the containing coarse simplex.  Used only to pin the oracle.
"""
from __future__ import annotations

import itertools
from fractions import Fraction

import numpy as np


def interior_index(dim: int, level: int):
    """Map from interior node numbers (I, J[, K]) (1-based) to the oracle's dense index."""
    n = (1 << level) - 1

    def f(I):
        if any(c < 1 or c > n for c in I):
            return None
        if dim == 2:
            return (I[1] - 1) * n + (I[0] - 1)
        return ((I[2] - 1) * n + (I[1] - 1)) * n + (I[0] - 1)

    return f, n ** dim


def kuhn_paths(dim: int):
    return list(itertools.permutations(range(dim)))


def simplex_vertices(corner, path):
    v = [tuple(corner)]
    for ax in path:
        c = list(v[-1])
        c[ax] += 1
        v.append(tuple(c))
    return v


def stiffness(dim: int, level: int) -> np.ndarray:
    """P1 stiffness matrix on the Kuhn triangulation of the unit square/cube."""
    n = 1 << level
    h = 1.0 / n
    f, N = interior_index(dim, level)
    K = np.zeros((N, N))
    for corner in itertools.product(range(n), repeat=dim):
        for path in kuhn_paths(dim):
            verts = simplex_vertices(corner, path)
            X = np.array(verts, dtype=float) * h
            M = np.hstack([np.ones((dim + 1, 1)), X])
            G = np.linalg.inv(M)[1:, :]  # gradients of barycentric functions, columns
            vol = abs(np.linalg.det(M)) / (2 if dim == 2 else 6)
            Kl = vol * G.T @ G
            ids = [f(v) for v in verts]
            for a in range(dim + 1):
                for b in range(dim + 1):
                    if ids[a] is not None and ids[b] is not None:
                        K[ids[a], ids[b]] += Kl[a, b]
    return K


def prolongation(dim: int, level: int) -> np.ndarray:
    """P_level: interpolate the coarse (level-1) P1 function at the fine nodes."""
    ff, Nf = interior_index(dim, level)
    fc, Nc = interior_index(dim, level - 1)
    nf = (1 << level) - 1
    P = np.zeros((Nf, Nc))
    for I in itertools.product(range(1, nf + 1), repeat=dim):
        row = ff(I)
        xi = [Fraction(c, 2) for c in I]  # coarse-grid coordinates
        cube = [min(int(x), (1 << (level - 1)) - 1) for x in xi]
        loc = [xi[a] - cube[a] for a in range(dim)]
        order = sorted(range(dim), key=lambda a: -loc[a])  # Kuhn simplex containing the point
        lam = [1 - loc[order[0]]] + [loc[order[k]] - loc[order[k + 1]] for k in range(dim - 1)] + \
              [loc[order[-1]]]
        verts = simplex_vertices(cube, order)
        for v, l in zip(verts, lam):
            col = fc(v)
            if col is not None and l != 0:
                P[row, col] += float(l)
    return P


def load_vector_exact(tables, scale_exp: int, dim: int, Lmax: int, L: int):
    """h_L^d * F(x) with F the exact integer table sum, rounded to 50 bits below
    the bound sum_t prod_a max|T| (Python integers; ties to even)."""
    nterms = tables.shape[0]
    bound = 0
    for t in range(nterms):
        p = 1
        for a in range(dim):
            p *= int(np.max(np.abs(tables[t, a].astype(np.int64))))
        bound += p
    B = bound.bit_length()
    sh = max(0, B - 50)
    n = (1 << L) - 1
    stride = 1 << (Lmax - L)
    out = np.zeros(n ** dim)
    f, _ = interior_index(dim, L)
    for I in itertools.product(range(1, n + 1), repeat=dim):
        F = 0
        for t in range(nterms):
            p = 1
            for a in range(dim):
                p *= int(tables[t, a, I[a] * stride - 1])
            F += p
        q = F >> sh
        rem = F - (q << sh)
        if sh > 0:
            half = 1 << (sh - 1)
            if rem > half or (rem == half and (q & 1)):
                q += 1
        out[f(I)] = float(Fraction(q) * Fraction(2) ** (scale_exp + sh - dim * L))
    return out
