"""Pins of the oracle's FP32 V-cycle (binary32 cycle inside exact iterative refinement).

The FP32 cycle is defined by its operation order (oracle/cmg_oracle.c, "FP32
V-cycle"; the precision split of Table 1).  These tests restate one cycle's
down-leg with numpy binary32 arithmetic, an independent IEEE implementation,
and exact rationals for the restriction, and check that the oracle produces
the same stored sections; they also check that the FP32 cycle reduces to the
exact one where no binary32 operation rounds, and that it keeps the solution
at discretization accuracy.
"""
from fractions import Fraction

import numpy as np
import pytest

import cmg_problems as P
import oracle
from cmg_problems import random_block_values

F32 = np.float32


def make(name, L, arith, **over):
    prob = P.make_problem(name, L)
    kw = dict(b1=5, b2=3, N=3, nu1=2, nu2=2, omega=0.75) if prob.dim == 3 else \
        dict(b1=4, b2=4, N=3, nu1=2, nu2=2, omega=0.75)
    kw.update(over)
    return prob, oracle.Oracle.for_problem(prob, arith=arith, **kw)


def stencil_f32(F, dim, level):
    """A F in binary32: (2d) F_p, minus -x, +x, -y, +y, -z, +z neighbours, times h^(d-2)."""
    pad = np.pad(F, 1)
    if dim == 2:
        c = pad[1:-1, 1:-1]
        acc = F32(4) * c
        for nb in (pad[1:-1, :-2], pad[1:-1, 2:], pad[:-2, 1:-1], pad[2:, 1:-1]):
            acc = (acc - nb).astype(F32)
        return acc
    c = pad[1:-1, 1:-1, 1:-1]
    acc = (F32(6) * c).astype(F32)
    for nb in (pad[1:-1, 1:-1, :-2], pad[1:-1, 1:-1, 2:], pad[1:-1, :-2, 1:-1], pad[1:-1, 2:, 1:-1],
               pad[:-2, 1:-1, 1:-1], pad[2:, 1:-1, 1:-1]):
        acc = (acc - nb).astype(F32)
    return (acc * F32(2.0 ** -level)).astype(F32)


def bfp_round_exact(vals, W):
    """RNE of exact rationals into 32-value BFP blocks along x (Sec. 4, Sec. 6.1.3)."""
    out = []
    n = len(vals)
    for b0 in range(0, n, 32):
        blk = vals[b0:b0 + 32]
        M = max(abs(v) for v in blk)
        if M == 0:
            out += [Fraction(0)] * len(blk)
            continue
        e = 0
        while Fraction(2) ** e <= M:
            e += 1
        while Fraction(2) ** (e - 1) > M:
            e -= 1
        for _ in range(2):
            scale = Fraction(2) ** (W - 1 - e)
            qs = []
            for v in blk:
                x = v * scale
                fl = x.numerator // x.denominator
                rem = x - fl
                q = fl + (1 if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2) else 0)
                qs.append(q)
            if max(abs(q) for q in qs) >= 2 ** (W - 1):
                e += 1
                continue
            break
        out += [Fraction(q) * Fraction(2) ** (e - W + 1) for q in qs]
    return out


def test_down_leg_matches_binary32_restatement():
    dim, L = 3, 3
    prob, o = make("poisson3d_manufactured", L, 1)
    o.start()
    for _ in range(L - 1):
        o.next_level()
    # a residual section with block exponents spread over ~40 bits, so that
    # binary32 sums of neighbours round
    n = (1 << L) - 1
    W = o.width(oracle.R, L)

    # the section layout: every x-row of n values is one 32-value block
    def encode_rows(v, width):
        rows = np.zeros((n * n, 32))
        rows[:, :n] = np.asarray(v, dtype=np.float64).reshape(n * n, n)
        w2, e2, s2 = oracle.encode(rows.ravel(), width)
        assert s2 == 0
        return w2, e2

    def decode_rows(w2, e2, width):
        vals, s2 = oracle.decode(w2, e2, n * n * 32, width)
        assert s2 == 0
        return vals.reshape(n * n, 32)[:, :n].reshape(n, n, n)

    rng = np.random.default_rng(5)
    x = random_block_values(n ** 3, seed=77)
    scale = np.repeat(2.0 ** rng.integers(-40, 0, size=n * n).astype(np.float64), n)
    words, e = encode_rows(x * scale, W)
    o.set_section(oracle.R, L, W, words, e)
    o.down(L)
    rc64 = decode_rows(words, e, W)
    rc = rc64.astype(F32)
    assert np.array_equal(rc.astype(np.float64), rc64)
    c = F32(2.0 ** L / 8)  # omega / (2d h^(d-2)) = (3/4) / 6 * 2^L
    Wy = o.width(oracle.Y, L)

    def rnd(v):
        w2, e2 = encode_rows(v, Wy)
        return decode_rows(w2, e2, Wy).astype(F32)

    y = rnd((F32(0) + (c * (rc - F32(0))).astype(F32)).astype(F32))
    S = stencil_f32(y, 3, L)
    y2 = rnd((y + (c * (rc - S).astype(F32)).astype(F32)).astype(F32))
    # binary32 rounding really happened somewhere in this sweep
    S64 = 6 * y.astype(np.float64)
    assert not np.array_equal(S.astype(np.float64) * 2.0 ** L,
                              S64 - np.pad(y, 1)[1:-1, 1:-1, :-2] - np.pad(y, 1)[1:-1, 1:-1, 2:]
                              - np.pad(y, 1)[1:-1, :-2, 1:-1] - np.pad(y, 1)[1:-1, 2:, 1:-1]
                              - np.pad(y, 1)[:-2, 1:-1, 1:-1] - np.pad(y, 1)[2:, 1:-1, 1:-1])
    _, _, ygot = o.get_section(oracle.Y, L, words=False)
    assert np.array_equal(ygot.reshape(n, n, n), y2.astype(np.float64))
    # restriction: d = fl(rc - A y) in binary32, R d exact, rounded into rc_(L-1)
    d = (rc - stencil_f32(y2, 3, L)).astype(F32)
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
    want = []
    for row in range(nc * nc):
        want += bfp_round_exact(Rd[row * nc:(row + 1) * nc], o.width(oracle.RC, L - 1))
    _, _, rcgot = o.get_section(oracle.RC, L - 1, words=False)
    assert [Fraction(float(v)) for v in rcgot.ravel()] == want


@pytest.mark.parametrize("name,L", [("poisson2d_manufactured", 7), ("poisson3d_fourier", 5),
                                    ("poisson3d_manufactured", 6)])
def test_fp32_cycle_equals_exact_cycle_when_nothing_rounds(name, L):
    outs = []
    for arith in (0, 1):
        prob, o = make(name, L, arith)
        o.fmg()
        assert o.status == 0
        outs.append([o.get_section(oracle.U, l)[:2] for l in range(1, L + 1)])
    for (w0, e0), (w1, e1) in zip(*outs):
        assert np.array_equal(w0, w1) and np.array_equal(e0, e1)


def test_fp32_cycle_keeps_discretization_accuracy():
    # at 2-D L = 10 the binary32 cycle rounds (the corrections span more than 24
    # bits) and its solution differs from the exact path's, within the error
    name, L = "poisson2d_manufactured", 10
    res = {}
    for arith in (0, 1):
        prob, o = make(name, L, arith)
        o.fmg()
        assert o.status == 0 and o.inexact == 0
        res[arith] = np.asarray(o.decode_solution()).ravel()
    n = (1 << L) - 1
    x = (np.arange(n) + 1.0) / (n + 1)
    X, Y = np.meshgrid(x, x, indexing="xy")
    ue = prob.exact_u(X, Y).ravel()
    err = {a: np.max(np.abs(res[a] - ue)) / np.max(np.abs(ue)) for a in res}
    diff = np.max(np.abs(res[1] - res[0])) / np.max(np.abs(res[0]))
    assert diff > 0
    assert diff < 0.5 * err[0]
    assert err[1] < 1.1 * err[0]
