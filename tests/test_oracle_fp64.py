"""Pins of the oracle's binary64 V-cycle (arith = 2, the plain FP64 form).

The binary64 cycle is the binary32 cycle's operation sequence (one source,
oracle/cycle_real.inc, instantiated for both types) with every intermediate
rounded to binary64 instead.  These tests fix it against what the mathematics
gives:

* where no binary64 operation rounds (every sum and product of the Poisson
  cycle spans fewer than 53 bits at these widths and sizes, including 2-D
  L = 10 where binary32 does round), it equals the exact cycle bit for bit, for
  Jacobi V(2,2) and red-black V(0,1), with the inexactness counter at zero;
* on a residual whose rows spread over 60 binary orders, one down-leg equals a
  numpy binary64 restatement (an IEEE implementation independent of the
  oracle's C) with the restriction formed in exact rationals, and binary64
  rounding is shown to happen in that sweep;
* on a problem where binary32 departs from the exact cycle (2-D L = 10) the
  binary64 solution is the exact cycle's, at its discretization error.
"""
from fractions import Fraction

import numpy as np
import pytest

import cmg_problems as P
import oracle
from cmg_problems import random_block_values
from exact_ref import bfp

F64 = np.float64


def make(name, L, arith, **over):
    prob = P.make_problem(name, L)
    kw = dict(b1=5, b2=3, N=3, nu1=2, nu2=2, omega=0.75) if prob.dim == 3 else \
        dict(b1=4, b2=4, N=3, nu1=2, nu2=2, omega=0.75)
    kw.update(over)
    return prob, oracle.Oracle.for_problem(prob, arith=arith, **kw)


@pytest.mark.parametrize("name,L,over", [("poisson2d_manufactured", 7, {}), ("poisson3d_fourier", 5, {}),
                                         ("poisson2d_manufactured", 10, {}),
                                         ("poisson3d_manufactured", 6, {"nu1": 0, "nu2": 1, "smoother": 1,
                                                                        "b2": 4})])
def test_fp64_cycle_equals_exact_cycle_where_nothing_rounds(name, L, over):
    outs = []
    for arith in (0, 2):
        prob, o = make(name, L, arith, **over)
        o.fmg()
        assert o.status == 0 and o.inexact == 0
        outs.append([o.get_section(oracle.U, l)[:2] for l in range(1, L + 1)])
    for (w0, e0), (w1, e1) in zip(*outs):
        assert np.array_equal(w0, w1) and np.array_equal(e0, e1)


def stencil(F, level):
    """3-D A F in binary64: 6 F_p, minus -x, +x, -y, +y, -z, +z neighbours, times h."""
    pad = np.pad(F, 1)
    acc = F64(6) * pad[1:-1, 1:-1, 1:-1]
    for nb in (pad[1:-1, 1:-1, :-2], pad[1:-1, 1:-1, 2:], pad[1:-1, :-2, 1:-1], pad[1:-1, 2:, 1:-1],
               pad[:-2, 1:-1, 1:-1], pad[2:, 1:-1, 1:-1]):
        acc = acc - nb
    return acc * F64(2.0 ** -level)


def stencil_exact(F, level):
    n = F.shape[0]
    q = [[[Fraction(float(F[k, j, i])) for i in range(n)] for j in range(n)] for k in range(n)]

    def at(k, j, i):
        return q[k][j][i] if 0 <= k < n and 0 <= j < n and 0 <= i < n else Fraction(0)
    out = np.empty((n, n, n), dtype=object)
    for k in range(n):
        for j in range(n):
            for i in range(n):
                s = 6 * at(k, j, i) - at(k, j, i - 1) - at(k, j, i + 1) - at(k, j - 1, i) - at(k, j + 1, i) \
                    - at(k - 1, j, i) - at(k + 1, j, i)
                out[k, j, i] = s / 2 ** level
    return out


def bfp_rows(v, W):
    n = v.shape[-1]
    vals, _, _ = bfp([Fraction(float(x)) for x in v.ravel()], n, W)
    return np.array([float(x) for x in vals]).reshape(v.shape)


def test_fp64_down_leg_matches_binary64_restatement():
    L = 3
    prob, o = make("poisson3d_manufactured", L, 2, b2=30)
    o.start()
    for _ in range(L - 1):
        o.next_level()
    n = (1 << L) - 1
    W = o.width(oracle.R, L)
    rng = np.random.default_rng(11)
    x = random_block_values(n ** 3, seed=78, spread_bits=20) * np.repeat(
        2.0 ** rng.integers(-60, 0, size=n * n), n)
    rc = bfp_rows(x.reshape(n, n, n), W)
    vals, e, q = bfp([Fraction(float(v)) for v in rc.ravel()], n, W)
    from exact_ref import pack
    o.set_section(oracle.R, L, W, pack(q, W), np.array(e, dtype=np.int8))
    o.down(L)
    assert o.status == 0
    Wy = o.width(oracle.Y, L)
    c = F64(2.0 ** L / 8)  # omega / (2d h^(d-2)) = (3/4) / 6 * 2^L
    y = bfp_rows(c * rc, Wy)
    S = stencil(y, L)
    y2 = bfp_rows(y + c * (rc - S), Wy)
    _, _, ygot = o.get_section(oracle.Y, L, words=False)
    assert np.array_equal(ygot.reshape(n, n, n), y2)
    # binary64 rounding happened in this sweep's stencil
    Sx = stencil_exact(y, L)
    assert any(Fraction(float(S[idx])) != Sx[idx] for idx in np.ndindex(S.shape))
    # restriction: d = fl(rc - A y) in binary64, R d exact, rounded into rc_(L-1)
    d = rc - stencil(y2, L)
    dq = [[[Fraction(float(d[k, j, i])) for i in range(n)] for j in range(n)] for k in range(n)]

    def at(I, J, K):
        if 1 <= I <= n and 1 <= J <= n and 1 <= K <= n:
            return dq[K - 1][J - 1][I - 1]
        return Fraction(0)
    nc = (1 << (L - 1)) - 1
    odd = [(1, 0, 0), (0, 1, 0), (1, 1, 0), (0, 0, 1), (1, 0, 1), (0, 1, 1), (1, 1, 1)]
    Rd = []
    for K in range(1, nc + 1):
        for J in range(1, nc + 1):
            for I in range(1, nc + 1):
                s = sum(at(2 * I - a, 2 * J - b, 2 * K - cc) + at(2 * I + a, 2 * J + b, 2 * K + cc)
                        for a, b, cc in odd)
                Rd.append(at(2 * I, 2 * J, 2 * K) + s / 2)
    want, _, _ = bfp(Rd, nc, o.width(oracle.RC, L - 1))
    _, _, rcgot = o.get_section(oracle.RC, L - 1, words=False)
    assert [Fraction(float(v)) for v in rcgot.ravel()] == list(want)


def test_fp64_cycle_keeps_discretization_accuracy():
    # 2-D L = 10: binary32 rounds and departs from the exact cycle; binary64 does not
    name, L = "poisson2d_manufactured", 10
    res = {}
    for arith in (0, 1, 2):
        prob, o = make(name, L, arith)
        o.fmg()
        assert o.status == 0 and o.inexact == 0
        res[arith] = np.asarray(o.decode_solution()).ravel()
    n = (1 << L) - 1
    xs = (np.arange(n) + 1.0) / (n + 1)
    X, Y = np.meshgrid(xs, xs, indexing="xy")
    ue = prob.exact_u(X, Y).ravel()
    err = {a: np.max(np.abs(res[a] - ue)) / np.max(np.abs(ue)) for a in res}
    assert np.array_equal(res[2], res[0])  # binary64 holds every intermediate here
    assert np.max(np.abs(res[1] - res[0])) > 0
    assert err[2] == err[0] and err[1] < 1.1 * err[0]
