"""Pins of the oracle's diffusion operator -div(k grad u) (variable coefficient).

The operator uses face coefficients (k_p + k_q) / 2 of the nodal binary32 field
k, injected onto coarse levels.  Pinned by: k = 1 reproduces the Poisson
operator exactly; the matrix is exactly symmetric for dyadic k; the stencil is
a second-order consistent discretisation of -div(k grad u) for smooth k and u;
and compact FMG with the FP32 cycle converges to the dense direct solution of
the same discrete system.
"""
import math

import numpy as np
import pytest

import cmg_problems as P
import oracle


def make(dim, L, kfield, **kw):
    prob = P.make_problem("diffusion%dd_grf" % dim, L)
    base = dict(b1=5, b2=4, N=3, nu1=2, nu2=2, omega=0.75)
    base.update(kw)
    return prob, oracle.Oracle(dim, L, prob.tables, prob.scale_exp, arith=1, coef=1, kfield=kfield, **base)


@pytest.mark.parametrize("dim,L", [(2, 4), (3, 3)])
def test_unit_coefficient_is_the_poisson_operator(dim, L):
    n = (1 << L) + 1
    _, o = make(dim, L, np.ones(n ** dim, dtype=np.float32))
    rng = np.random.default_rng(3)
    for lev in range(1, L + 1):
        npts = ((1 << lev) - 1) ** dim
        x = rng.integers(-1000, 1000, size=npts).astype(np.float64)
        a = o.apply_A_diffusion(lev, x)
        b = np.zeros_like(x)
        oracle.lib().cmgo_apply_A(dim, lev, oracle._p(x), oracle._p(b))
        assert np.array_equal(a, b)


def dense(o, dim, lev):
    npts = ((1 << lev) - 1) ** dim
    M = np.zeros((npts, npts))
    for i in range(npts):
        e = np.zeros(npts)
        e[i] = 1.0
        M[:, i] = o.apply_A_diffusion(lev, e)
    return M


@pytest.mark.parametrize("dim,L", [(2, 3), (3, 2)])
def test_symmetric_for_dyadic_coefficients(dim, L):
    n = (1 << L) + 1
    rng = np.random.default_rng(9)
    k = rng.choice(np.array([0.5, 1.0, 2.0, 3.0, 0.25], dtype=np.float32), size=n ** dim)
    _, o = make(dim, L, k)
    for lev in range(1, L + 1):
        M = dense(o, dim, lev)
        assert np.array_equal(M, M.T)
        assert np.all(np.linalg.eigvalsh(M) > 0)


def test_second_order_consistency():
    # k = 1 + x^2 y, u = sin(pi x) sin(pi y):  -div(k grad u) at the nodes
    errs = []
    for L in (5, 6, 7):
        n = (1 << L) + 1
        x = np.arange(n) / (n - 1.0)
        X, Y = np.meshgrid(x, x, indexing="xy")
        k = (1.0 + X * X * Y).astype(np.float32)
        _, o = make(2, L, k.ravel())
        xi = x[1:-1]
        XI, YI = np.meshgrid(xi, xi, indexing="xy")
        pi = math.pi
        u = np.sin(pi * XI) * np.sin(pi * YI)
        Au = o.apply_A_diffusion(L, u.ravel()).reshape(u.shape)
        kk = 1.0 + XI * XI * YI
        kx, ky = 2 * XI * YI, XI * XI
        ux, uy = pi * np.cos(pi * XI) * np.sin(pi * YI), pi * np.sin(pi * XI) * np.cos(pi * YI)
        lap = -2 * pi * pi * u
        f = -(kk * lap + kx * ux + ky * uy)
        h = 2.0 ** -L
        errs.append(np.max(np.abs(Au / (h * h) - f)))
    # the binary32 field perturbs k by ~2^-24 relative; the O(h^2) term dominates
    assert 3.6 < errs[0] / errs[1] < 4.4
    assert 3.6 < errs[1] / errs[2] < 4.4


@pytest.mark.parametrize("dim,L", [(2, 5), (3, 3)])
def test_fmg_reaches_the_dense_solution(dim, L):
    prob = P.make_problem("diffusion%dd_grf" % dim, L)
    k = prob.kfield().ravel()
    # Jacobi V(2,2) with injected coarse coefficients contracts by about 1/2 per
    # iteration on this rough field (k spans e^+-3), so 20 IR iterations per level
    prob, o = make(dim, L, k, b1=16, b2=10, N=20)
    o.fmg()
    assert o.status == 0
    u = np.asarray(o.decode_solution()).ravel()
    M = dense(o, dim, L)
    f = np.full(M.shape[0], 2.0 ** (-dim * L))
    ud = np.linalg.solve(M, f)
    assert np.max(np.abs(u - ud)) / np.max(np.abs(ud)) < 1e-5
