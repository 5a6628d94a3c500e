"""The seeded input generators (cmg_problems) against their stated recipes (CPU).

- The manufactured right-hand sides are -Lap u of the stated u. That is
  derived here symbolically, independently of the hand-expanded separable
  terms in the generator, and must match the quantised tables to their 30-bit
  precision.
- The Fourier-mode right-hand sides are read back by a sine transform: at
  most 8 modes, wavenumbers in 1..8, and -Lap u = f mode by mode.
- The diffusion coefficient's field g is a Gaussian random field with standard
  deviation sigma and squared-exponential covariance
  sigma^2 exp(-r^2 / (2 corr^2)). Its sample variance and correlation over
  seeds must match, and k = exp(g) rounded to binary32.
"""
import math

import numpy as np
import pytest

import cmg_problems as P
from cmg_problems.diffusion import diffusion_grf

sympy = pytest.importorskip("sympy")

X, Y, Z = sympy.symbols("x y z")
STATED_U = {
    "poisson2d_manufactured": (2, sympy.sin(sympy.pi * X) * sympy.sin(sympy.pi * Y) * (1 + X**2 * Y)),
    "poisson3d_manufactured": (3, sympy.sin(sympy.pi * X) * sympy.sin(sympy.pi * Y) * sympy.sin(sympy.pi * Z)
                               * (1 + X**2 * Y * Z)),
}


@pytest.mark.parametrize("name", sorted(STATED_U))
def test_manufactured_rhs_is_minus_laplacian_of_the_stated_u(name):
    dim, u = STATED_U[name]
    syms = (X, Y, Z)[:dim]
    f = sympy.lambdify(syms, -sum(sympy.diff(u, s, 2) for s in syms), "numpy")
    uf = sympy.lambdify(syms, u, "numpy")
    Lmax = 8
    prob = P.make_problem(name, Lmax)
    rng = np.random.default_rng(7)
    idx = tuple(rng.integers(0, prob.n1, size=400) for _ in range(dim))
    x = tuple((i + 1.0) * 2.0 ** -Lmax for i in idx)
    want = f(*x)
    got = prob.rhs_float(idx)
    scale = np.max(np.abs(want))
    assert np.max(np.abs(got - want)) <= 1e-7 * scale
    # the closure the diagnostics use is the stated u
    assert np.allclose(prob.exact_u(*x), uf(*x), rtol=0, atol=1e-15)


@pytest.mark.parametrize("sigma", [1.0, 0.5])
def test_grf_variance_and_correlation(sigma):
    L, corr = 5, 0.1
    h = 2.0 ** -L
    lag = 3  # r = 3 h = 0.09375, close to the correlation length
    r = lag * h
    var, cov = [], []
    for seed in range(1, 13):
        g = diffusion_grf(3, L, seed=seed, sigma=sigma, corr=corr).g_field()
        assert g.shape == ((1 << L) + 1,) * 3
        var.append(np.mean(g * g))
        cov.append(np.mean(g[:, :, lag:] * g[:, :, :-lag]))
        cov.append(np.mean(g[:, lag:, :] * g[:, :-lag, :]))
        cov.append(np.mean(g[lag:, :, :] * g[:-lag, :, :]))
    assert abs(np.mean(var) / sigma**2 - 1.0) < 0.1
    rho = np.mean(cov) / np.mean(var)
    assert abs(rho - math.exp(-r * r / (2 * corr * corr))) < 0.06
    # far apart the field decorrelates
    g = diffusion_grf(3, L, seed=1, sigma=sigma, corr=corr).g_field()
    far = np.mean(g[:, :, 16:] * g[:, :, :-16]) / np.mean(g * g)
    assert abs(far) < 0.2


def test_coefficient_is_exp_g_in_binary32():
    prob = diffusion_grf(3, 4, seed=2, sigma=0.5)
    g = prob.g_field()
    k = prob.kfield()
    assert k.dtype == np.float32 and k.shape == g.shape
    assert np.array_equal(k, np.exp(g).astype(np.float32))
    assert np.all(k > 0)


@pytest.mark.parametrize("name,dim", [("poisson3d_fourier", 3), ("poisson2d_fourier", 2)])
def test_fourier_modes_by_sine_transform(name, dim):
    """C2's recipe (f = sum of 8 modes a_j prod sin(k pi x), k in 1..8; u with
    -Lap u = f) read back from the nodal values by a DST-I, which represents
    every sin(k pi x), k < 2^L, exactly on the interior nodes."""
    from scipy.fft import dstn
    L = 5
    prob = P.make_problem(name, L)
    idx = np.meshgrid(*([np.arange(prob.n1)] * dim), indexing="ij")
    F = prob.rhs_float(tuple(idx))
    U = prob.exact_u(*[(i + 1.0) * 2.0 ** -L for i in idx])
    Fh, Uh = dstn(F, type=1), dstn(U, type=1)
    tol = 1e-6 * np.max(np.abs(Fh))
    on = np.abs(Fh) > tol
    assert 1 <= on.sum() <= 8
    k = np.argwhere(on) + 1  # wavenumbers of the modes present
    assert k.min() >= 1 and k.max() <= 8
    ksq = (k * k).sum(axis=1)
    ratio = Fh[on] / Uh[on]
    assert np.allclose(ratio, math.pi**2 * ksq, rtol=1e-6)
    assert np.max(np.abs(Uh[~on])) <= 1e-6 * np.max(np.abs(Uh))
