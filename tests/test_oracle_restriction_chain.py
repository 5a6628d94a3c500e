"""Pin of the oracle's restriction chain in fmgResidual (Algorithm 2 without
pre-smoothing, the red-black V(0,1) cycle's source of every coarse right-hand side).

Algorithm 2 decodes u^_L, forms t_L = f_L - A_L u^_L, rounds r_L from it, and
restricts t down the hierarchy.  Table 1 gives t^ in fmgResidual the precision
(p+1)L + b1 bits; the oracle reads that as 32-value BFP blocks of width
Wt = (p+1)L + b1 (the reading is argued in the design notes):

    r_L   = round_{Wr(L)}(t_L)                 (from the exact t_L)
    t^_L  = round_{Wt}(t_L)
    t^_l  = round_{Wt}(R_(l+1) t^_(l+1)),      l = L-1 .. 1
    r_l   = round_{Wr(l)}(t^_l)

This file restates the chain with exact rationals (fractions.Fraction), the
first-principles FEM matrices of tests/fem_dense.py (element-by-element P1
stiffness, prolongation by locating the containing coarse simplex, R = P^T),
the load vector of tests/fem_dense.py, and its own BFP rounder and bit packer
(Sec. 4: round to nearest, ties to even; Sec. 6.1.3: BFP).  It shares no code
with the oracle.  Every r_l the oracle stores must equal the restatement bit for
bit (exponents and packed words), at the production widths and at widths where
r is wider than t^.  In the wide case three plausible mistakes change the coarse
r_l and would be caught: r_l rounded from the unrounded chain R^(L-l) t_L, t^
kept at the finest solution width b1 instead of Wt, and t^ rounded value by
value (floating point) instead of in BFP blocks.  At the production widths the
value-by-value reading changes at most 1 % of the coarse r codes.
"""
from fractions import Fraction

import numpy as np
import pytest

import cmg_problems as P
import oracle
from exact_ref import bfp, matvec, pack, per_value, snap, transpose
from fem_dense import load_vector_exact, prolongation, stiffness


# production widths (Table 2's 2-D constants; the 3-D red-black ones) and a wide-r
# case (b2 = 10 > b1 = 2), in which r_l keeps t^_l's bits, so that the rounding of
# the chain itself is visible in the stored r_l
CASES = [("poisson2d_manufactured", 5, 4, 4), ("poisson3d_manufactured", 4, 5, 4)]
WIDE = [("poisson2d_manufactured", 5, 2, 10), ("poisson3d_manufactured", 4, 2, 10)]


def chain_case(name, L, b1, b2):
    prob = P.make_problem(name, L)
    dim = prob.dim
    o = oracle.Oracle.for_problem(prob, b1=b1, b2=b2, N=3, nu1=0, nu2=1, omega=1.0 if dim == 2 else 0.75,
                                  smoother=1)
    o.fmg()  # nonzero u~ sections on every level
    assert o.status == 0
    o.residual()  # the chain from the final solution
    assert o.status == 0 and o.inexact == 0
    h_den = (1 << L) * 12
    Pm = {l: snap(prolongation(dim, l), 2) for l in range(2, L + 1)}
    Rm = {l: transpose(Pm[l], ((1 << (l - 1)) - 1) ** dim) for l in range(2, L + 1)}
    K = snap(stiffness(dim, L), h_den)
    uhat = None
    for l in range(1, L + 1):
        u = [Fraction(float(v)) for v in o.get_section(oracle.U, l, words=False)[2].ravel()]
        uhat = u if l == 1 else [a + b for a, b in zip(u, matvec(Pm[l], uhat))]
    f = [Fraction(float(v)) for v in load_vector_exact(prob.tables, prob.scale_exp, dim, L, L)]
    t = [a - b for a, b in zip(f, matvec(K, uhat))]
    return prob, o, dim, Rm, t


def wr(L, l, b2):
    return (L - l) + b2


@pytest.mark.parametrize("name,L,b1,b2", CASES + WIDE)
def test_restriction_chain_equals_rational_restatement(name, L, b1, b2):
    prob, o, dim, Rm, t = chain_case(name, L, b1, b2)
    Wt = 2 * L + b1  # (p+1) L + b1 with p = 1
    n = lambda l: (1 << l) - 1  # noqa: E731
    expect = {}
    _, e, q = bfp(t, n(L), wr(L, L, b2))
    expect[L] = (e, q)
    th, _, _ = bfp(t, n(L), Wt)
    for l in range(L - 1, 0, -1):
        th, _, _ = bfp(matvec(Rm[l + 1], th), n(l), Wt)
        _, e, q = bfp(th, n(l), wr(L, l, b2))
        expect[l] = (e, q)
    for l in range(1, L + 1):
        w, eo, _ = o.get_section(oracle.R, l)
        W = o.width(oracle.R, l)
        assert W == wr(L, l, b2)
        e, q = expect[l]
        assert np.array_equal(eo.astype(int), np.array(e)), "exponents of r_%d" % l
        assert np.array_equal(w, pack(q, W)), "codes of r_%d" % l
        if l < L:  # the coarse right-hand sides are not trivially zero
            assert any(ee != -128 for ee in e)


def coarse_r_of_chain(t, Rm, L, b2, t_round):
    n = lambda l: (1 << l) - 1  # noqa: E731
    out = {}
    th = t_round(t, n(L))
    for l in range(L - 1, 0, -1):
        th = t_round(matvec(Rm[l + 1], th), n(l))
        out[l] = np.array([float(v) for v in bfp(th, n(l), wr(L, l, b2))[0]])
    return out


@pytest.mark.parametrize("name,L,b1,b2", WIDE)
def test_restriction_chain_pin_detects_plausible_mistakes(name, L, b1, b2):
    """With r wider than t^, three other chains give different coarse r_l, so the
    bit-exact comparison above would catch each: r_l from the unrounded chain
    R^(L-l) t_L, t^ kept at the finest solution width b1 instead of Wt, and t^
    rounded value by value (floating point) instead of in BFP blocks."""
    prob, o, dim, Rm, t = chain_case(name, L, b1, b2)
    got = {l: o.get_section(oracle.R, l, words=False)[2].ravel() for l in range(1, L)}
    Wt = 2 * L + b1
    for t_round in (lambda v, m: v, lambda v, m: bfp(v, m, b1)[0], lambda v, m: per_value(v, Wt)):
        alt = coarse_r_of_chain(t, Rm, L, b2, t_round)
        ndiff = sum(int(np.sum(alt[l] != got[l])) for l in got)
        assert ndiff >= 0.1 * sum(got[l].size for l in got)
    same = coarse_r_of_chain(t, Rm, L, b2, lambda v, m: bfp(v, m, Wt)[0])
    assert all(np.array_equal(same[l], got[l]) for l in got)


@pytest.mark.parametrize("name,L,b1,b2", CASES)
def test_chain_readings_agree_at_production_widths(name, L, b1, b2):
    """At the widths the solver runs with, r_l (Wr(l) = L - l + b2 bits) is far
    narrower than t^ (Wt = 2L + b1 bits): the value-by-value reading of Table 1's
    t^ and the unrounded chain change at most 1 % of the coarse r codes."""
    prob, o, dim, Rm, t = chain_case(name, L, b1, b2)
    got = {l: o.get_section(oracle.R, l, words=False)[2].ravel() for l in range(1, L)}
    ntot = sum(got[l].size for l in got)
    for t_round in (lambda v, m: v, lambda v, m: per_value(v, 2 * L + b1)):
        alt = coarse_r_of_chain(t, Rm, L, b2, t_round)
        assert sum(int(np.sum(alt[l] != got[l])) for l in got) <= 0.01 * ntot
