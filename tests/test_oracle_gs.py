"""Pins of the oracle's red-black Gauss-Seidel smoother and the paper's V(0,1) cycle.

* One red-black sweep of the up-leg equals a sequential, in-place Gauss-Seidel
  sweep that visits all red nodes and then all black nodes, the section being
  rounded into BFP after each colour (brute force with dense matrices; exact
  arithmetic on the short dyadic values).
* V(0,1) with Gauss-Seidel contracts faster than V(0,1) with Jacobi.
* Paper-faithful configuration (Algorithm 1 as V(0,1) with one Gauss-Seidel
  sweep per level, Table 2's 2-D p = 1 constants b1 = 4, b2 = 4, N = 3, omega =
  1): compact FMG meets the Sec. 7.1 success criterion.
"""
import numpy as np
import pytest

import cmg_problems as P
import oracle
from cmg_problems.diagnostics import h1_error


def dense(fn, n_in, n_out):
    M = np.zeros((n_out, n_in))
    for i in range(n_in):
        e = np.zeros(n_in)
        e[i] = 1.0
        M[:, i] = fn(e)
    return M


def A_dense(dim, level):
    n = ((1 << level) - 1) ** dim

    def f(x):
        out = np.zeros_like(x)
        oracle.lib().cmgo_apply_A(dim, level, oracle._p(x), oracle._p(out))
        return out
    return dense(f, n, n)


def P_dense(dim, level):
    nf, nc = ((1 << level) - 1) ** dim, ((1 << (level - 1)) - 1) ** dim

    def f(x):
        out = np.zeros(nf)
        oracle.lib().cmgo_prolong(dim, level, oracle._p(np.ascontiguousarray(x)), oracle._p(out))
        return out
    return dense(f, nc, nf)


@pytest.mark.parametrize("name,L", [("poisson2d_manufactured", 4), ("poisson3d_manufactured", 3)])
def test_red_black_sweep_is_sequential_gauss_seidel(name, L):
    prob = P.make_problem(name, L)
    dim = prob.dim
    omega = 1.0 if dim == 2 else 0.75
    # BFP widths: every value is a short dyadic, so the arithmetic is exact (certified)
    # and the order of evaluation is immaterial; each half-sweep re-rounds the section
    o = oracle.Oracle.for_problem(prob, b1=5, b2=4, N=1, nu1=0, nu2=1, omega=omega, smoother=1)
    o.start()
    for _ in range(L - 1):
        o.next_level()
    o.residual()
    for l in range(L, 1, -1):
        o.down(l)
    o.coarse()
    for l in range(2, L + 1):
        w = np.zeros(((1 << (l - 1)) - 1) ** dim)
        oracle.lib().cmgo_last_w(o._ctx, l - 1, oracle._p(w))
        _, _, rc = o.get_section(oracle.RC, l, words=False)
        rc = rc.ravel()
        A = A_dense(dim, l)
        z = P_dense(dim, l) @ w
        c = omega / (2 * dim) * 2.0 ** ((dim - 2) * l)
        n = (1 << l) - 1
        coords = np.array(list(np.ndindex(*((n,) * dim))))[:, ::-1]  # (x, y[, z]) per flat index
        colour = (coords + 1).sum(axis=1) & 1
        W = o.width(oracle.Y, l)

        def rnd(v):  # BFP rounding of the level's rows (one 32-value block per row here)
            rows = np.zeros((n ** (dim - 1), 32))
            rows[:, :n] = v.reshape(-1, n)
            w2, e2, st = oracle.encode(rows.ravel(), W)
            assert st == 0
            return oracle.decode(w2, e2, rows.size, W)[0].reshape(-1, 32)[:, :n].ravel()

        y = np.zeros(n ** dim)
        for col in (0, 1):  # sequential, in place: all red nodes, then all black nodes
            for p in np.nonzero(colour == col)[0]:
                y[p] += c * (rc[p] - A[p] @ (y + z))
            y = rnd(y)
        o.up(l)
        _, _, ygot = o.get_section(oracle.Y, l, words=False)
        assert np.array_equal(ygot.ravel(), y), "level %d" % l
    assert o.inexact == 0


def _ir_error(prob, smoother, iters):
    """Nodal error to the discrete solution after `iters` lossless IR iterations at L."""
    L = prob.Lmax
    o = oracle.Oracle.for_problem(prob, b1=0, b2=0, N=1, nu1=0, nu2=1, omega=1.0, smoother=smoother)
    o.start()
    for _ in range(L - 1):
        o.next_level()
    ref = oracle.Oracle.for_problem(prob, b1=0, b2=0, N=30, nu1=2, nu2=2, omega=0.75)
    ref.fmg()
    u_ref = np.asarray(ref.decode_solution()).ravel()
    errs = []
    for _ in range(iters):
        o.ir_iteration()
        errs.append(np.max(np.abs(np.asarray(o.decode_solution()).ravel() - u_ref)))
    return np.array(errs)


def test_gauss_seidel_contracts_faster_than_jacobi():
    prob = P.make_problem("poisson2d_manufactured", 6)
    gs = _ir_error(prob, 1, 6)
    ja = _ir_error(prob, 0, 6)
    rate_gs = (gs[-1] / gs[1]) ** (1 / 4)
    rate_ja = (ja[-1] / ja[1]) ** (1 / 4)
    assert rate_gs < rate_ja < 1.0


def test_paper_configuration_meets_the_success_criterion():
    """Algorithm 1 as V(0,1) with Gauss-Seidel and Table 2's constants (2-D, p = 1)."""
    name, Lmax = "poisson2d_manufactured", 7
    prob = P.make_problem(name, Lmax)

    def h1s(**cfg):
        o = oracle.Oracle.for_problem(prob, **cfg)
        o.start()
        errs = []
        for L in range(2, Lmax + 1):
            o.next_level()
            for _ in range(cfg["N"]):
                o.ir_iteration()
            errs.append(h1_error(prob, o.decode_solution(), L))
        return np.array(errs), o

    ref, _ = h1s(b1=0, b2=0, N=12, nu1=2, nu2=2, omega=0.75)
    err, o = h1s(b1=4, b2=4, N=3, nu1=0, nu2=1, omega=1.0, smoother=1)
    Ls = np.arange(2, Lmax + 1)
    assert np.all(err[Ls >= 4] <= 2 * ref[Ls >= 4])
    order = -np.log2(err[1:] / err[:-1])
    assert np.all(order[Ls[1:] >= 4] >= 0.95)
    assert o.inexact == 0
