"""Pins of the oracle's floating-point diffusion down-leg (the variable-coefficient cycle).

The diffusion cycle runs in IEEE binary32 (arith = 1) or binary64 (arith = 2,
the plain FP64 form) in one fixed order (the precision split of Table 1: the
cycle in progressive(+m, b4), which binary32 already holds):

    per node p and neighbour q in the order -x, +x, -y, +y, -z, +z:
        kf   = fl(fl(k_q + k_p) * 0.5)
        acc  = fl(acc + fl(kf * fl(F_p - F_q)))        (F = y~, zero outside)
        dsum = fl(dsum + kf)
    S = fl(acc h^(d-2)),  D_p = fl(dsum h^(d-2)),  c_p = fl(omega / D_p)
    y~' = round_BFP(fl(y~ + fl(c_p fl(rc - S))))       (one Jacobi sweep)
    d = fl(rc - S(y~)),  R d in binary32: sum over S = {x}, {y}, {x,y}, {z},
        {x,z}, {y,z}, {x,y,z} of fl(sum + d(2I - e_S)) then fl(sum + d(2I + e_S)),
        R d = fl(d(2I) + fl(sum * 0.5)),  rc_(l-1) = round_BFP(R d).

This file restates two Jacobi sweeps and the restriction of one down-leg with
numpy binary32 / binary64 arithmetic (an IEEE implementation independent of the
oracle's C) and the exact-rational BFP rounder of exact_ref.py, on a seeded
coefficient field and a residual whose block exponents spread over 40 binary
orders (so that the operations round: checked against exact rationals), and
requires the oracle's stored y~_L and rc_(L-1) to equal it bit for bit.  Two
plausible mistakes, the Poisson factor c = omega / (2d h^(d-2)) in place of
omega / D_p and the restriction summed in another order, are shown to change
the binary32 result on data whose sections are wide enough (20-bit residual
and correction) to keep binary32's last bits; both cycles are one source
instantiated twice, so that order pin holds for the binary64 cycle as well.
"""
from fractions import Fraction

import numpy as np
import pytest

import cmg_problems as P
import oracle
from cmg_problems import random_block_values
from exact_ref import bfp, pack

F32 = np.float32
ODD = [(1, 0, 0), (0, 1, 0), (1, 1, 0), (0, 0, 1), (1, 0, 1), (0, 1, 1), (1, 1, 1)]


def flux_sum(F, k, L, dt=F32):
    """(S, D) of the diffusion stencil in type dt at every interior node (3-D
    arrays in (z, y, x) order; F interior, k on the closed grid)."""
    k = k.astype(dt)
    Fp = np.pad(F, 1)
    c = (slice(1, -1),) * 3
    kp = k[c]
    acc = np.zeros_like(F)
    dsum = np.zeros_like(F)
    # -x, +x, -y, +y, -z, +z in (z, y, x) indexing
    shifts = [(0, 0, -1), (0, 0, 1), (0, -1, 0), (0, 1, 0), (-1, 0, 0), (1, 0, 0)]
    for dz, dy, dx in shifts:
        sl = (slice(1 + dz, Fp.shape[0] - 1 + dz), slice(1 + dy, Fp.shape[1] - 1 + dy),
              slice(1 + dx, Fp.shape[2] - 1 + dx))
        ks = (k[sl] + kp).astype(dt)
        kf = (ks * dt(0.5)).astype(dt)
        du = (F - Fp[sl]).astype(dt)
        acc = (acc + (kf * du).astype(dt)).astype(dt)
        dsum = (dsum + kf).astype(dt)
    hs = dt(2.0 ** -L)
    return (acc * hs).astype(dt), (dsum * hs).astype(dt)


def restrict_f32(d):
    dt = d.dtype.type
    n = d.shape[0]
    nc = (n - 1) // 2
    dp = np.pad(d, 1)  # 1-based node (I, J, K) at dp[K, J, I]
    out = np.zeros((nc, nc, nc), dtype=dt)
    for K in range(1, nc + 1):
        for J in range(1, nc + 1):
            for I in range(1, nc + 1):
                s = dt(0)
                for ex, ey, ez in ODD:
                    s = dt(s + dp[2 * K - ez, 2 * J - ey, 2 * I - ex])
                    s = dt(s + dp[2 * K + ez, 2 * J + ey, 2 * I + ex])
                out[K - 1, J - 1, I - 1] = dt(dp[2 * K, 2 * J, 2 * I] + dt(s * dt(0.5)))
    return out


def bfp_levels(v, W):
    n = v.shape[-1]
    vals, e, q = bfp([Fraction(float(x)) for x in v.ravel()], n, W)
    return np.array([float(x) for x in vals]).reshape(v.shape), e, q


def setup(b2, spread=40, L=3, arith=1):
    prob = P.make_problem("diffusion3d_grf", L)
    k = np.ascontiguousarray(prob.kfield(), dtype=np.float32).reshape((1 << L) + 1, (1 << L) + 1, (1 << L) + 1)
    o = oracle.Oracle(3, L, prob.tables, prob.scale_exp, b1=6, b2=b2, N=1, nu1=2, nu2=2, omega=0.75,
                      arith=arith, coef=1, kfield=k.ravel())
    o.start()
    for _ in range(L - 1):
        o.next_level()
    n = (1 << L) - 1
    W = o.width(oracle.R, L)
    rng = np.random.default_rng(5)
    x = random_block_values(n ** 3, seed=77, spread_bits=min(spread, 20)) * np.repeat(
        2.0 ** rng.integers(-spread, 0, size=n * n), n)
    rc64, e, q = bfp_levels(x.reshape(n, n, n), W)
    o.set_section(oracle.R, L, W, pack(q, W), np.array(e, dtype=np.int8))
    return o, k, rc64, L, n


def one_down_leg(k, rc, L, factor=None, restrict=restrict_f32, Wy=None, Wrc=None):
    """Two Jacobi sweeps from y~ = 0 and the restriction in rc's type; factor(D)
    is the Jacobi factor (default fl(omega / D_p))."""
    dt = rc.dtype.type
    if factor is None:
        def factor(D):
            return (dt(0.75) / D).astype(dt)
    y = np.zeros_like(rc)
    for _ in range(2):
        S, D = flux_sum(y, k, L, dt)
        cp = factor(D)
        y2 = (y + (cp * (rc - S).astype(dt)).astype(dt)).astype(dt)
        y = bfp_levels(y2, Wy)[0].astype(dt)
    S, _ = flux_sum(y, k, L, dt)
    d = (rc - S).astype(dt)
    Rd = restrict(d)
    return y, bfp_levels(Rd, Wrc)


@pytest.mark.parametrize("b2,arith", [(4, 1), (16, 1), (4, 2), (16, 2), (30, 2)])
def test_diffusion_down_leg_equals_restatement(b2, arith):
    dt = F32 if arith == 1 else np.float64
    o, k, rc64, L, n = setup(b2, arith=arith)
    rc = rc64.astype(dt)
    assert np.array_equal(rc.astype(np.float64), rc64)
    o.down(L)
    assert o.status == 0
    Wy, Wrc = o.width(oracle.Y, L), o.width(oracle.RC, L - 1)
    y, (rcv, e, q) = one_down_leg(k, rc, L, Wy=Wy, Wrc=Wrc)
    _, _, ygot = o.get_section(oracle.Y, L, words=False)
    assert np.array_equal(ygot.reshape(n, n, n), y.astype(np.float64))
    w, eo, _ = o.get_section(oracle.RC, L - 1)
    assert np.array_equal(eo.astype(int), np.array(e))
    assert np.array_equal(w, pack(q, Wrc))
    # rounding happened in the flux sums of this sweep: the exact rational flux
    # differs from the one in dt at some node
    Sdt, _ = flux_sum(y, k, L, dt)
    yq = np.pad(y.astype(np.float64), 1)
    shifts = [(0, 0, -1), (0, 0, 1), (0, -1, 0), (0, 1, 0), (-1, 0, 0), (1, 0, 0)]
    differs = 0
    for z in range(n):
        for yy in range(n):
            for x in range(n):
                acc = Fraction(0)
                for dz, dy, dx in shifts:
                    kf = (Fraction(float(k[z + 1 + dz, yy + 1 + dy, x + 1 + dx])) + Fraction(float(k[z + 1, yy + 1, x + 1]))) / 2
                    acc += kf * (Fraction(float(yq[z + 1, yy + 1, x + 1])) - Fraction(float(yq[z + 1 + dz, yy + 1 + dy, x + 1 + dx])))
                differs += Fraction(float(Sdt[z, yy, x])) != acc / 2 ** L
    assert differs > 0


def restrict_in_order(order, minus_first=True):
    def r(d):
        nc = (d.shape[0] - 1) // 2
        dp = np.pad(d, 1)
        out = np.zeros((nc, nc, nc), dtype=F32)
        for K in range(1, nc + 1):
            for J in range(1, nc + 1):
                for I in range(1, nc + 1):
                    s = F32(0)
                    for ex, ey, ez in order:
                        a, b = dp[2 * K - ez, 2 * J - ey, 2 * I - ex], dp[2 * K + ez, 2 * J + ey, 2 * I + ex]
                        if not minus_first:
                            a, b = b, a
                        s = F32(s + a)
                        s = F32(s + b)
                    out[K - 1, J - 1, I - 1] = F32(dp[2 * K, 2 * J, 2 * I] + F32(s * F32(0.5)))
        return out
    return r


def test_diffusion_down_leg_pin_detects_plausible_mistakes():
    # b2 = 20 and residual rows spread over 8 binary orders: the stored sections keep
    # binary32's last bits and the restriction's partial sums round, so an operation
    # order that rounds differently shows in them
    o, k, rc64, L, n = setup(20, spread=8)
    rc = rc64.astype(F32)
    o.down(L)
    Wy, Wrc = o.width(oracle.Y, L), o.width(oracle.RC, L - 1)
    _, _, ygot = o.get_section(oracle.Y, L, words=False)
    _, _, rcgot = o.get_section(oracle.RC, L - 1, words=False)
    _, (rc_ref, _, _) = one_down_leg(k, rc, L, Wy=Wy, Wrc=Wrc)
    assert np.array_equal(rcgot.reshape(rc_ref.shape), rc_ref)
    # the Poisson Jacobi factor instead of omega / D_p
    y_bad, _ = one_down_leg(k, rc, L, factor=lambda D: np.full_like(D, F32(0.75 / 6 * 2.0 ** L)), Wy=Wy, Wrc=Wrc)
    assert not np.array_equal(ygot.reshape(n, n, n), y_bad.astype(np.float64))
    # the restriction with plus before minus, and with the odd sets in reverse order
    for wrong in (restrict_in_order(ODD, minus_first=False), restrict_in_order(ODD[::-1])):
        _, (rc_bad, _, _) = one_down_leg(k, rc, L, restrict=wrong, Wy=Wy, Wrc=Wrc)
        assert not np.array_equal(rcgot.reshape(rc_bad.shape), rc_bad)
