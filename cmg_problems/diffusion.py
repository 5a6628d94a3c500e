"""Seeded variable-coefficient diffusion problems (input data only).

-div(k grad u) = f on the unit square / cube, u = 0 on the boundary, f = 1, and
k = exp(g) with g a Gaussian random field of standard deviation sigma and
squared-exponential covariance with correlation length corr, drawn as random
Fourier features:

    g(x) = sigma sqrt(2/M) sum_j cos(omega_j . x + phi_j),
    omega_j ~ N(0, corr^-2 I),  phi_j ~ U(0, 2 pi)

(then E[g(x) g(y)] = sigma^2 exp(-|x - y|^2 / (2 corr^2))).  The field is
evaluated separably, cos(omega . x + phi) = Re(e^(i phi) prod_a e^(i omega_a
x_a)), from complex 1-D tables, and stored in binary32: that binary32 nodal
field, boundary nodes included, is the problem's coefficient.  f = 1 is given as
one separable term of unit tables, so the right-hand side machinery of the
Poisson problems applies unchanged.

This module holds no arithmetic of the solver; it only draws inputs.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Tuple

import numpy as np

from . import SeededRNG


@dataclasses.dataclass
class DiffusionProblem:
    name: str
    dim: int
    Lmax: int
    tables: np.ndarray  # int32 [1, dim, 2**Lmax - 1], all ones: f = 1
    scale_exp: int
    seed: int
    sigma: float
    corr: float
    nmodes: int
    description: str
    coef: int = 1

    @property
    def nterms(self) -> int:
        return 1

    def modes(self) -> Tuple[np.ndarray, np.ndarray]:
        """(omega [M, dim], phi [M]) drawn from the seeded SplitMix64 stream."""
        rng = SeededRNG(self.seed)
        om = np.zeros((self.nmodes, self.dim))
        ph = np.zeros(self.nmodes)
        for j in range(self.nmodes):
            for a in range(self.dim):
                om[j, a] = rng.normal() / self.corr
            ph[j] = 2.0 * math.pi * rng.uniform()
        return om, ph

    def g_field(self, device: Optional[str] = None) -> np.ndarray:
        """g at every node x_I = I 2^-Lmax, I = 0..2^Lmax, as FP64 (numpy), or on a
        torch device for large grids (returned as a torch tensor)."""
        om, ph = self.modes()
        N = (1 << self.Lmax) + 1
        x = np.arange(N, dtype=np.float64) * 2.0 ** -self.Lmax
        amp = self.sigma * math.sqrt(2.0 / self.nmodes)
        c = amp * np.exp(1j * ph)  # [M]
        E = [np.exp(1j * np.outer(om[:, a], x)) for a in range(self.dim)]  # [M, N] per axis
        if device is None:
            if self.dim == 2:
                G = np.einsum("j,jy,jx->yx", c, E[1], E[0], optimize=True)
            else:
                G = np.einsum("j,jz,jy,jx->zyx", c, E[2], E[1], E[0], optimize=True)
            return np.ascontiguousarray(G.real)
        import torch
        ct = torch.tensor(c, dtype=torch.complex128, device=device)
        Et = [torch.tensor(e, dtype=torch.complex128, device=device) for e in E]
        if self.dim == 2:
            A = Et[1] * ct[:, None]  # [M, y]
            return (A.transpose(0, 1) @ Et[0]).real  # [y, x]
        out = torch.empty((N, N, N), dtype=torch.float64, device=device)
        step = 32
        for z0 in range(0, N, step):
            z1 = min(N, z0 + step)
            A = (Et[2][:, z0:z1, None] * Et[1][:, None, :]) * ct[:, None, None]  # [M, zc, y]
            out[z0:z1] = (A.reshape(self.nmodes, -1).transpose(0, 1) @ Et[0]).real.reshape(z1 - z0, N, N)
        return out

    def kfield(self, device: Optional[str] = None):
        """k = exp(g) in binary32 on the finest grid, boundary included, x fastest."""
        g = self.g_field(device)
        if device is None:
            return np.exp(g).astype(np.float32)
        import torch
        return torch.exp(g).to(torch.float32)

    def exact_u(self, *coords):  # no closed form; the diagnostics use a reference solve
        return None


def diffusion_grf(dim: int, Lmax: int, seed: int = 1, sigma: float = 1.0, corr: float = 0.1,
                  nmodes: int = 256) -> DiffusionProblem:
    n1 = (1 << Lmax) - 1
    tables = np.ones((1, dim, n1), dtype=np.int32)
    return DiffusionProblem("diffusion%dd_grf" % dim, dim, Lmax, tables, 0, seed, sigma, corr, nmodes,
                            "%d-D -div(exp(g) grad u) = 1, g a GRF (sigma %g, correlation %g, %d Fourier "
                            "features, seed %d)" % (dim, sigma, corr, nmodes, seed))
