"""Seeded synthetic problems for the compact full multigrid (CMG) solver.

This module is shared input data, not solver code: it produces the separable
right-hand-side tables that both the CUDA path and the CPU oracle consume,
plus closed-form exact solutions used to measure discretization error.  It
holds none of the method's arithmetic (no stencil, no prolongation, no
rounding to block floating point, no assembly of the load vector).

Right-hand-side format
----------------------
The continuous right-hand side is a sum of separable terms,

    F(x) = sum_t  prod_a  g_{t,a}(x_a),

sampled at the interior nodes x_a = (i + 1) * 2**-Lmax, i = 0 .. 2**Lmax - 2,
of the finest grid.  Each 1-D factor is delivered as an int32 table that holds
g_{t,a}(x_i) in fixed point: all terms of axis a share one exponent, so that

    F(x) ~= 2**scale_exp * sum_t prod_a T[t, a, i_a]      (exact integers).

The integer form makes the sampled right-hand side an exact dyadic rational
that both sides can reproduce bit for bit.  The paper manufactures every
workload analytically (Sec. 7.1), so no dataset is involved.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Tuple

import numpy as np

TABLE_BITS = 30  # |T| <= 2**30, so a 3-factor product stays below 2**90

_M64 = (1 << 64) - 1


def splitmix64(seed: int):
    """Generator of 64-bit outputs of SplitMix64 (Steele, Lea, Flood 2014)."""
    state = seed & _M64
    while True:
        state = (state + 0x9E3779B97F4A7C15) & _M64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        yield z ^ (z >> 31)


class SeededRNG:
    """Uniform and Box-Muller normal deviates driven by SplitMix64."""

    def __init__(self, seed: int):
        self._g = splitmix64(seed)

    def uniform(self) -> float:
        # 53 high bits -> [0, 1)
        return (next(self._g) >> 11) * (1.0 / (1 << 53))

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi]."""
        return lo + int(self.uniform() * (hi - lo + 1))

    def normal(self) -> float:
        u1 = 1.0 - self.uniform()  # (0, 1]
        u2 = self.uniform()
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)


@dataclasses.dataclass
class SeparableProblem:
    """A Poisson problem -Lap u = F on the unit square/cube, zero Dirichlet."""

    name: str
    dim: int
    Lmax: int
    tables: np.ndarray  # int32 [nterms, dim, 2**Lmax - 1]
    scale_exp: int
    exact_u: Callable[..., np.ndarray]  # vectorised u(x, y[, z])
    description: str
    exact_grad: Callable[..., Tuple[np.ndarray, ...]] = None  # vectorised grad u

    @property
    def nterms(self) -> int:
        return int(self.tables.shape[0])

    @property
    def n1(self) -> int:
        return (1 << self.Lmax) - 1

    def rhs_float(self, coords: Tuple[np.ndarray, ...]) -> np.ndarray:
        """F at given finest-grid node indices, from the quantised tables (float)."""
        acc = 0.0
        for t in range(self.nterms):
            term = 1.0
            for a in range(self.dim):
                term = term * self.tables[t, a, coords[a]].astype(np.float64)
            acc = acc + term
        return np.ldexp(acc, self.scale_exp)


def _sin(a):  # the closed forms below take numpy arrays or torch tensors (device diagnostics)
    return a.sin() if hasattr(a, "sin") else np.sin(a)


def _cos(a):
    return a.cos() if hasattr(a, "cos") else np.cos(a)


def _nodes(Lmax: int) -> np.ndarray:
    n1 = (1 << Lmax) - 1
    return (np.arange(n1, dtype=np.float64) + 1.0) * (2.0 ** -Lmax)


def quantise_tables(funcs: List[List[np.ndarray]], dim: int) -> Tuple[np.ndarray, int]:
    """Fixed-point int32 tables with one exponent per axis (shared by all terms)."""
    nterms = len(funcs)
    n1 = funcs[0][0].shape[0]
    tables = np.zeros((nterms, dim, n1), dtype=np.int32)
    scale_exp = 0
    for a in range(dim):
        amax = max(float(np.max(np.abs(funcs[t][a]))) for t in range(nterms))
        if amax == 0.0:
            raise ValueError("axis table identically zero")
        _, E = math.frexp(amax)  # amax < 2**E
        q = np.rint(np.ldexp(np.stack([funcs[t][a] for t in range(nterms)]), TABLE_BITS - E))
        assert np.max(np.abs(q)) <= (1 << TABLE_BITS)
        tables[:, a, :] = q.astype(np.int32)
        scale_exp += E - TABLE_BITS
    return tables, scale_exp


def poisson2d_manufactured(Lmax: int) -> SeparableProblem:
    """u = sin(pi x) sin(pi y) (1 + x^2 y) on the unit square (2-D, 257^2 at Lmax=8).

    -Lap u splits into three separable terms:
        2 pi^2 S(x) S(y)
      + [2 pi^2 x^2 S(x) - 4 pi x C(x) - 2 S(x)] * y S(y)
      - 2 pi x^2 S(x) * C(y)
    with S(t) = sin(pi t), C(t) = cos(pi t).
    """
    x = _nodes(Lmax)
    pi = math.pi
    S, C = np.sin(pi * x), np.cos(pi * x)
    funcs = [
        [2 * pi * pi * S, S],
        [2 * pi * pi * x * x * S - 4 * pi * x * C - 2 * S, x * S],
        [-2 * pi * x * x * S, C],
    ]
    tables, se = quantise_tables(funcs, 2)

    def exact_u(X, Y):
        return _sin(pi * X) * _sin(pi * Y) * (1.0 + X * X * Y)

    def exact_grad(X, Y):
        sx, sy, cx, cy = _sin(pi * X), _sin(pi * Y), _cos(pi * X), _cos(pi * Y)
        g = 1.0 + X * X * Y
        return (pi * cx * sy * g + sx * sy * 2 * X * Y,
                sx * (pi * cy * g + sy * X * X))

    return SeparableProblem("poisson2d_manufactured", 2, Lmax, tables, se, exact_u,
                            "u=sin(pi x)sin(pi y)(1+x^2 y)", exact_grad)


def poisson3d_manufactured(Lmax: int) -> SeparableProblem:
    """u = sin(pi x) sin(pi y) sin(pi z) (1 + x^2 y z) on the unit cube.

    -Lap u splits into four separable terms:
        3 pi^2 S(x) S(y) S(z)
      + [3 pi^2 x^2 S(x) - 4 pi x C(x) - 2 S(x)] * y S(y) * z S(z)
      - 2 pi x^2 S(x) * C(y) * z S(z)
      - 2 pi x^2 S(x) * y S(y) * C(z)
    """
    x = _nodes(Lmax)
    pi = math.pi
    S, C = np.sin(pi * x), np.cos(pi * x)
    funcs = [
        [3 * pi * pi * S, S, S],
        [3 * pi * pi * x * x * S - 4 * pi * x * C - 2 * S, x * S, x * S],
        [-2 * pi * x * x * S, C, x * S],
        [-2 * pi * x * x * S, x * S, C],
    ]
    tables, se = quantise_tables(funcs, 3)

    def exact_u(X, Y, Z):
        return _sin(pi * X) * _sin(pi * Y) * _sin(pi * Z) * (1.0 + X * X * Y * Z)

    def exact_grad(X, Y, Z):
        sx, sy, sz = _sin(pi * X), _sin(pi * Y), _sin(pi * Z)
        cx, cy, cz = _cos(pi * X), _cos(pi * Y), _cos(pi * Z)
        g = 1.0 + X * X * Y * Z
        sss = sx * sy * sz
        return (pi * cx * sy * sz * g + sss * 2 * X * Y * Z,
                pi * sx * cy * sz * g + sss * X * X * Z,
                pi * sx * sy * cz * g + sss * X * X * Y)

    return SeparableProblem("poisson3d_manufactured", 3, Lmax, tables, se, exact_u,
                            "u=sin(pi x)sin(pi y)sin(pi z)(1+x^2 y z)", exact_grad)


def poisson3d_fourier(Lmax: int, seed: int = 0, nmodes: int = 8, kmax: int = 8) -> SeparableProblem:
    """F = sum_j a_j sin(k1 pi x) sin(k2 pi y) sin(k3 pi z), a_j ~ N(0,1), k in {1..kmax}.

    The exact solution is u = sum_j a_j / (pi^2 |k_j|^2) prod sin(.) .
    """
    rng = SeededRNG(seed)
    modes = []
    for _ in range(nmodes):
        a = rng.normal()
        k = tuple(rng.randint(1, kmax) for _ in range(3))
        modes.append((a, k))
    x = _nodes(Lmax)
    pi = math.pi
    funcs = [[a * np.sin(k[0] * pi * x), np.sin(k[1] * pi * x), np.sin(k[2] * pi * x)]
             for a, k in modes]
    tables, se = quantise_tables(funcs, 3)

    def exact_u(X, Y, Z):
        out = 0.0
        for a, k in modes:
            out = out + a / (pi * pi * (k[0] ** 2 + k[1] ** 2 + k[2] ** 2)) * \
                _sin(k[0] * pi * X) * _sin(k[1] * pi * Y) * _sin(k[2] * pi * Z)
        return out

    def exact_grad(X, Y, Z):
        gx = gy = gz = 0.0
        for a, k in modes:
            c = a / (pi * pi * (k[0] ** 2 + k[1] ** 2 + k[2] ** 2))
            sx, sy, sz = _sin(k[0] * pi * X), _sin(k[1] * pi * Y), _sin(k[2] * pi * Z)
            gx = gx + c * k[0] * pi * _cos(k[0] * pi * X) * sy * sz
            gy = gy + c * k[1] * pi * sx * _cos(k[1] * pi * Y) * sz
            gz = gz + c * k[2] * pi * sx * sy * _cos(k[2] * pi * Z)
        return gx, gy, gz

    desc = "sum of %d modes, seed %d: %s" % (nmodes, seed, ", ".join(
        "%.4f*(%d,%d,%d)" % (a, *k) for a, k in modes))
    return SeparableProblem("poisson3d_fourier", 3, Lmax, tables, se, exact_u, desc, exact_grad)


def poisson2d_fourier(Lmax: int, seed: int = 0, nmodes: int = 8, kmax: int = 8) -> SeparableProblem:
    """2-D analogue of :func:`poisson3d_fourier` (used for small parity cases)."""
    rng = SeededRNG(seed)
    modes = []
    for _ in range(nmodes):
        a = rng.normal()
        k = tuple(rng.randint(1, kmax) for _ in range(2))
        modes.append((a, k))
    x = _nodes(Lmax)
    pi = math.pi
    funcs = [[a * np.sin(k[0] * pi * x), np.sin(k[1] * pi * x)] for a, k in modes]
    tables, se = quantise_tables(funcs, 2)

    def exact_u(X, Y):
        out = 0.0
        for a, k in modes:
            out = out + a / (pi * pi * (k[0] ** 2 + k[1] ** 2)) * \
                _sin(k[0] * pi * X) * _sin(k[1] * pi * Y)
        return out

    def exact_grad(X, Y):
        gx = gy = 0.0
        for a, k in modes:
            c = a / (pi * pi * (k[0] ** 2 + k[1] ** 2))
            gx = gx + c * k[0] * pi * _cos(k[0] * pi * X) * _sin(k[1] * pi * Y)
            gy = gy + c * k[1] * pi * _sin(k[0] * pi * X) * _cos(k[1] * pi * Y)
        return gx, gy

    return SeparableProblem("poisson2d_fourier", 2, Lmax, tables, se, exact_u,
                            "2-D sum of %d modes, seed %d" % (nmodes, seed), exact_grad)


def make_problem(name: str, Lmax: int, seed: int = 0) -> SeparableProblem:
    if name == "poisson2d_manufactured":
        return poisson2d_manufactured(Lmax)
    if name == "poisson3d_manufactured":
        return poisson3d_manufactured(Lmax)
    if name == "poisson3d_fourier":
        return poisson3d_fourier(Lmax, seed)
    if name == "poisson2d_fourier":
        return poisson2d_fourier(Lmax, seed)
    if name in ("diffusion3d_grf", "diffusion2d_grf"):
        from .diffusion import diffusion_grf
        return diffusion_grf(3 if name.startswith("diffusion3d") else 2, Lmax, seed=seed if seed else 1)
    raise KeyError(name)


def random_block_values(n: int, seed: int, spread_bits: int = 20, zero_frac: float = 0.05) -> np.ndarray:
    """Seeded FP64 test vector for codec checks: mixed magnitudes, exact zeros,
    ties at small widths and a few all-zero 32-blocks."""
    rng = np.random.default_rng(seed)
    mant = rng.integers(-(1 << 20), 1 << 20, size=n).astype(np.float64)
    expo = rng.integers(-spread_bits, spread_bits + 1, size=n)
    x = np.ldexp(mant, expo - 20)
    x[rng.random(n) < zero_frac] = 0.0
    nb = (n + 31) // 32
    if nb >= 4:
        zb = rng.choice(nb, size=max(1, nb // 16), replace=False)
        for b in zb:
            x[32 * b: min(n, 32 * b + 32)] = 0.0
    return x
