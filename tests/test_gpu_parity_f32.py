"""GPU parity of the floating-point V-cycles inside exact iterative refinement.

The CUDA path with arith = CMG_ARITH_FP32 / CMG_ARITH_FP64 against the oracle
with arith = 1 / 2: bit-exact sections after every step, including inputs on
which binary32 operations round (a residual whose rows span about 32 binary
orders), and whole solves at sizes where the binary32 cycle departs from the
exact one (where the binary64 cycle does not).
"""
import numpy as np
import pytest

import cmg_problems as P
import oracle
from cmg_problems import random_block_values

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cmg():
    from paper_2511_19036_gb300 import cmg as m
    return m


def make_pair(cmg, name, Lmax, arith=1, **over):
    prob = P.make_problem(name, Lmax)
    cfg = cmg.config_for(name, Lmax, arith=arith)
    for k, v in over.items():
        setattr(cfg, k, v)
    s = cmg.Solver(cfg)
    s.set_rhs(prob.tables, prob.scale_exp)
    o = oracle.Oracle.for_problem(prob, b1=cfg.b1, b2=cfg.b2, N=cfg.N_ir, nu1=cfg.nu1, nu2=cfg.nu2,
                                  omega=cfg.omega, arith=arith)
    return prob, cfg, s, o


def same_section(cmg, s, o, which_g, which_o, level, what=""):
    gw, ge = s.get_section(which_g, level)
    ow, oe, _ = o.get_section(which_o, level)
    assert s.width(which_g, level) == o.width(which_o, level)
    assert np.array_equal(ge, oe), "exponents differ: %s level %d (%d blocks)" % (
        what, level, int(np.sum(ge != oe)))
    assert np.array_equal(gw, ow), "words differ: %s level %d (%d words)" % (what, level, int(np.sum(gw != ow)))


FMG_CASES = [("poisson2d_manufactured", 8, 1, {}),
             ("poisson2d_manufactured", 10, 1, {}),   # the binary32 cycle rounds here
             ("poisson3d_fourier", 6, 1, {}),
             ("poisson3d_manufactured", 6, 1, {"nu1": 1, "nu2": 1}),
             ("poisson2d_fourier", 7, 1, {"nu1": 0, "nu2": 1}),
             ("poisson2d_manufactured", 10, 2, {}),
             ("poisson3d_fourier", 6, 2, {}),
             ("poisson3d_manufactured", 6, 2, {"nu1": 1, "nu2": 1, "b2": 12})]


@pytest.mark.parametrize("name,Lmax,arith,over", FMG_CASES)
def test_fmg_parity_fp(cmg, name, Lmax, arith, over):
    prob, cfg, s, o = make_pair(cmg, name, Lmax, arith, **over)
    s.fmg_solve()
    o.fmg()
    assert o.status == 0 and o.inexact == 0
    for l in range(1, Lmax + 1):
        same_section(cmg, s, o, cmg.SEC_U, oracle.U, l, "fmg fp32")
    assert np.array_equal(s.decode_solution().cpu().numpy(), o.decode_solution())


def _rows_encode(dim, L, vals, W):
    n = (1 << L) - 1
    rows = np.zeros((n ** (dim - 1), 32 * ((n + 31) // 32)))
    rows[:, :n] = vals.reshape(n ** (dim - 1), n)
    w, e, st = oracle.encode(rows.ravel(), W)
    assert st == 0
    return w, e


@pytest.mark.parametrize("name,L,arith", [("poisson3d_manufactured", 5, 1), ("poisson2d_manufactured", 6, 1),
                                          ("poisson3d_manufactured", 5, 2), ("poisson2d_manufactured", 6, 2)])
def test_cycle_steps_where_binary32_rounds(cmg, name, L, arith):
    prob, cfg, s, o = make_pair(cmg, name, L, arith)
    s.start()
    o.start()
    for _ in range(L - 1):
        s.prolongate()
        o.next_level()
    n = (1 << L) - 1
    npts = n ** prob.dim
    W = o.width(oracle.R, L)
    # rows scaled over 24 binary orders (values within a row over 8): neighbours
    # differ by more than binary32's 24 bits, while R d still fits the exact
    # int64 accumulation (a span of at most 57 bits)
    rng = np.random.default_rng(11)
    x = random_block_values(npts, seed=91, spread_bits=4) * np.repeat(
        2.0 ** rng.integers(-24, 0, size=npts // n).astype(np.float64), n)
    words, e = _rows_encode(prob.dim, L, x, W)
    s.set_section(cmg.SEC_R, L, W, words, e)
    o.set_section(oracle.R, L, W, words, e)
    # the exact cycle on the same input: binary32 must round somewhere here
    o64 = oracle.Oracle.for_problem(prob, b1=cfg.b1, b2=cfg.b2, N=cfg.N_ir, nu1=cfg.nu1, nu2=cfg.nu2,
                                    omega=cfg.omega, arith=0)
    o64.start()
    for _ in range(L - 1):
        o64.next_level()
    o64.set_section(oracle.R, L, W, words, e)
    o64.down(L)
    for l in range(L, 1, -1):
        s.down(l)
        o.down(l)
        same_section(cmg, s, o, cmg.SEC_Y, oracle.Y, l, "down")
        same_section(cmg, s, o, cmg.SEC_RC, oracle.RC, l - 1, "restrict")
        if l == L and prob.dim == 3:  # binary32 rounds; binary64 holds these spans
            assert (arith == 1) != np.array_equal(o.get_section(oracle.RC, l - 1, words=False)[2],
                                      o64.get_section(oracle.RC, l - 1, words=False)[2])
    s.coarse()
    o.coarse()
    same_section(cmg, s, o, cmg.SEC_Y, oracle.Y, 1, "coarse")
    for l in range(2, L + 1):
        s.up(l)
        o.up(l)
        same_section(cmg, s, o, cmg.SEC_Y, oracle.Y, l, "up")
    assert o.status == 0


def test_fp32_needs_widths_within_binary32(cmg):
    cfg = cmg.config_for("poisson3d_fourier", 14, arith=1)
    cfg.b2 = 12  # r / y~ on level 1 would need 13 + 12 bits plus the Jacobi numerator
    assert cmg.params_check(cfg) == cmg.ERANGE
    assert cmg.params_check(cmg.config_for("poisson3d_fourier", 11, arith=1)) == cmg.OK
    bad = cmg.config_for("poisson3d_fourier", 5, arith=3)
    assert cmg.params_check(bad) == cmg.EINVAL
    for arith, want in ((1, cmg.ERANGE), (2, cmg.OK)):  # binary64 holds these widths
        cfg = cmg.config_for("poisson3d_fourier", 11, arith=arith)
        cfg.b2 = 16
        assert cmg.params_check(cfg) == want
