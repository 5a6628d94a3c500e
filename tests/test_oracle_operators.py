"""Pins for the oracle's operators against first-principles FEM matrices.

Sec. 3.1 defines A_l (FEM stiffness), P_l (canonical prolongation from the
nesting V_(l-1) in V_l) and R_l = P_l^T; the Galerkin identity
A_(l-1) = R_l A_l P_l holds for nested P1 spaces on the Kuhn refinement.
The dense matrices come from tests/fem_dense.py, which shares no code with the
oracle's stencil, odd-set interpolation or restriction loops.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import cmg_problems as P
from exact_ref import bfp, matvec, pack, snap
from fem_dense import load_vector_exact, prolongation, stiffness

CASES = [(2, 2), (2, 3), (2, 4), (3, 2), (3, 3)]


@pytest.mark.parametrize("dim,level", CASES)
def test_stencil_equals_assembled_stiffness(dim, level):
    K = stiffness(dim, level)
    rng = np.random.default_rng(level)
    x = rng.integers(-1000, 1000, size=K.shape[0]).astype(float)
    assert np.allclose(oracle.apply_A(dim, level, x), K @ x, rtol=0, atol=1e-9)


@pytest.mark.parametrize("dim,level", CASES)
def test_prolongation_equals_interpolation(dim, level):
    Pm = prolongation(dim, level)
    rng = np.random.default_rng(10 + level)
    xc = rng.integers(-1000, 1000, size=Pm.shape[1]).astype(float)
    assert np.array_equal(oracle.prolong(dim, level, xc), Pm @ xc)


@pytest.mark.parametrize("dim,level", CASES)
def test_restriction_is_transpose(dim, level):
    Pm = prolongation(dim, level)
    rng = np.random.default_rng(20 + level)
    xf = rng.integers(-1000, 1000, size=Pm.shape[0]).astype(float)
    assert np.array_equal(oracle.restrict(dim, level, xf), Pm.T @ xf)


@pytest.mark.parametrize("dim,level", [(2, 3), (2, 4), (3, 3)])
def test_galerkin_coarse_operator(dim, level):
    Kf, Kc, Pm = stiffness(dim, level), stiffness(dim, level - 1), prolongation(dim, level)
    assert np.allclose(Pm.T @ Kf @ Pm, Kc, rtol=0, atol=1e-12)


@pytest.mark.parametrize("name,Lmax,L", [("poisson2d_manufactured", 4, 3),
                                         ("poisson2d_manufactured", 4, 4),
                                         ("poisson3d_fourier", 3, 3),
                                         ("poisson3d_manufactured", 3, 2)])
def test_load_vector_exact(name, Lmax, L):
    prob = P.make_problem(name, Lmax)
    o = oracle.Oracle.for_problem(prob, b1=5, b2=4, N=1, nu1=1, nu2=1, omega=0.75)
    ref = load_vector_exact(prob.tables, prob.scale_exp, prob.dim, Lmax, L)
    assert np.array_equal(o.rhs(L).reshape(-1), ref)
    # and it approximates h^d F(x) of the continuous right-hand side
    h = 2.0 ** -L
    n = (1 << L) - 1
    x = (np.arange(n) + 1) * h
    stride = 1 << (Lmax - L)
    idx = np.arange(1, n + 1) * stride - 1
    grids = np.meshgrid(*([idx] * prob.dim), indexing="ij")[::-1]
    F = prob.rhs_float(tuple(grids)).reshape(-1)
    assert np.allclose(ref, h ** prob.dim * F, rtol=1e-12, atol=0)


@pytest.mark.parametrize("name,Lmax", [("poisson2d_manufactured", 4), ("poisson3d_fourier", 3)])
def test_residual_matches_dense_formula(name, Lmax):
    """Algorithm 2: t_L = f_L - A_L (u~_L + P_L (u~_(L-1) + ... )) before rounding."""
    prob = P.make_problem(name, Lmax)
    o = oracle.Oracle.for_problem(prob, b1=5, b2=4, N=2, nu1=2, nu2=2, omega=0.75)
    o.fmg()  # leaves nonzero sections on every level
    dim = prob.dim
    uhat = None
    for l in range(1, Lmax + 1):
        sec = o.get_section(oracle.U, l, words=False)[2].reshape(-1)
        uhat = sec if l == 1 else sec + prolongation(dim, l) @ uhat
    o.residual()
    t = o.last_t().reshape(-1)
    f = load_vector_exact(prob.tables, prob.scale_exp, dim, Lmax, Lmax)
    expect = f - stiffness(dim, Lmax) @ uhat
    assert np.allclose(t, expect, rtol=0, atol=1e-12 * np.max(np.abs(f)))
    # exactly: t_L equals the dense formula in rationals, and r_L is that t_L
    # rounded into the b2-bit BFP format of the finest level (independent rounder
    # and packer), compared code for code and exponent for exponent
    Km = snap(stiffness(dim, Lmax), (1 << Lmax) * 12)
    t_exact = [Fraction(float(a)) - b for a, b in
               zip(f, matvec(Km, [Fraction(float(v)) for v in uhat]))]
    assert [Fraction(float(v)) for v in t] == t_exact
    W = o.width(oracle.R, Lmax)
    _, e, codes = bfp(t_exact, (1 << Lmax) - 1, W)
    wr_, er, rv = o.get_section(oracle.R, Lmax)
    assert np.array_equal(er.astype(int), np.array(e))
    assert np.array_equal(wr_, pack(codes, W))
    assert any(c != 0 for blk in codes for c in blk)
