"""The exact path's kernel choices give one result (GPU).

* The specialised 3-D kernels (cmg_fast.cu) and the generic kernels
  (cmg_stencil.cu), each on its own, give the oracle's sections bit for bit,
  for the red-black V(0,1) and the Jacobi V(2,2) cycles.
* On the finest FMG level the level-(L-1) sources w and u^ can be formed on the
  fly from the level-(L-1) section and the level-(L-2) temporary (no int64
  copy of level L_max - 1, cmg_set_two_level): the solve equals the oracle
  with and without, the report's temporary bytes drop by those two int64
  arrays, and the switch works between solves in both directions.
* Operands whose footprints exceed the specialised kernels' 32-bit proofs send
  tiles to the generic kernels (the fallback list), and the result is
  unchanged.
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


def sections(s, cmg, L):
    return [s.get_section(cmg.SEC_U, l) for l in range(1, L + 1)]


@pytest.mark.parametrize("name,L,smoother", [("poisson3d_manufactured", 6, 1), ("poisson3d_fourier", 6, 0),
                                             ("poisson3d_manufactured", 7, 1), ("poisson2d_manufactured", 7, 0)])
def test_fast_and_generic_kernels_agree_with_the_oracle(cmg, name, L, smoother):
    prob = P.make_problem(name, L)
    cfg = cmg.config_for(name, L, smoother=smoother)
    got = []
    for fast, two in ((True, True), (False, True), (True, False), (False, False)):
        s = cmg.Solver(cfg, fast=fast, two_level=two)
        s.set_rhs(prob.tables, prob.scale_exp)
        s.fmg_solve()
        got.append((sections(s, cmg, L), s.decode_solution().cpu().numpy()))
        if fast and prob.dim == 3:
            st = s.fast_stats()
            assert st["top"]["ctas"] > 0  # the specialised kernels ran on the finest level
    o = oracle.Oracle.for_problem(prob, b1=cfg.b1, b2=cfg.b2, N=cfg.N_ir, nu1=cfg.nu1, nu2=cfg.nu2,
                                  omega=cfg.omega, smoother=smoother)
    o.fmg()
    assert o.status == 0 and o.inexact == 0
    for (secs, u) in got:
        for l in range(1, L + 1):
            ow, oe, _ = o.get_section(oracle.U, l)
            assert np.array_equal(secs[l - 1][1], oe) and np.array_equal(secs[l - 1][0], ow), l
        assert np.array_equal(u, o.decode_solution())


def test_two_level_path_drops_the_level_below_the_finest_temporaries(cmg):
    name, L = "poisson3d_fourier", 6
    prob = P.make_problem(name, L)
    rep = {}
    for two in (True, False):
        s = cmg.Solver(cmg.config_for(name, L), two_level=two)
        s.set_rhs(prob.tables, prob.scale_exp)
        rep[two] = s.fmg_solve()
        secs = sections(s, cmg, L)
        if two:
            ref = secs
        else:
            assert all(np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) for a, b in zip(ref, secs))
    n = (1 << (L - 1)) - 1
    R = 32 * ((n + 31) // 32)
    assert rep[False]["temp_bytes"] - rep[True]["temp_bytes"] == 2 * 8 * n * n * R
    # switching between solves, both ways, on one context
    s = cmg.Solver(cmg.config_for(name, L), two_level=True)
    s.set_rhs(prob.tables, prob.scale_exp)
    for two in (False, True, False):
        s.set_two_level(two)
        s.fmg_solve()
        assert all(np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
                   for a, b in zip(ref, sections(s, cmg, L)))
    # the binary32 cycle has no two-level path
    f = cmg.Solver(cmg.config_for(name, L, arith=1))
    with pytest.raises(cmg.CmgError) as ei:
        f.set_two_level(True)
    assert ei.value.status == cmg.EUNSUPPORTED


def _rows(x, n, npts):
    rows = np.zeros((npts // n, 32 * ((n + 31) // 32)))
    rows[:, :n] = x.reshape(npts // n, n)
    return rows.ravel()


@pytest.mark.parametrize("two", [True, False])
def test_wide_operands_take_the_fallback_tiles(cmg, two):
    # a residual whose rows span 36 binary orders: |c rc| on the tile's finest
    # grid exceeds the red half-sweep's 32-bit proof on some tiles, which the
    # generic kernel then runs from the fallback list (red-black V(0,1), whose
    # red half-sweep from y~ = 0 is specialised; two-level source on L_max)
    name, L = "poisson3d_manufactured", 6
    prob = P.make_problem(name, L)
    cfg = cmg.config_for(name, L, smoother=1)
    s = cmg.Solver(cfg, two_level=two)
    s.set_rhs(prob.tables, prob.scale_exp)
    o = oracle.Oracle.for_problem(prob, b1=cfg.b1, b2=cfg.b2, N=cfg.N_ir, nu1=cfg.nu1, nu2=cfg.nu2,
                                  omega=cfg.omega, smoother=1)
    s.start()
    o.start()
    for _ in range(L - 1):
        s.prolongate()
        o.next_level()
        for _ in range(cfg.N_ir):
            s.ir_iteration()
            o.ir_iteration()
    s.residual()
    o.residual()
    n = (1 << L) - 1
    W = o.width(oracle.R, L)
    rng = np.random.default_rng(3)
    x = random_block_values(n ** 3, seed=23, spread_bits=8) * np.repeat(
        2.0 ** rng.integers(-50, -14, size=n * n).astype(np.float64), n)
    words, e, st = oracle.encode(_rows(x, n, n ** 3), W)
    assert st == 0
    s.set_section(cmg.SEC_R, L, W, words, e)
    o.set_section(oracle.R, L, W, words, e)
    before = s.fast_stats()["top"]["fallback_ctas"]
    for l in range(L, 1, -1):
        s.down(l)
        o.down(l)
    s.coarse()
    o.coarse()
    for l in range(2, L + 1):
        s.up(l)
        o.up(l)
        gw, ge = s.get_section(cmg.SEC_Y, l)
        ow, oe, _ = o.get_section(oracle.Y, l)
        assert np.array_equal(ge, oe) and np.array_equal(gw, ow), l
    assert s.fast_stats()["top"]["fallback_ctas"] > before
    s.correct()
    o.correct()
    assert o.status == 0 and o.inexact == 0
    for l in range(1, L + 1):
        ow, oe, _ = o.get_section(oracle.U, l)
        gw, ge = s.get_section(cmg.SEC_U, l)
        assert np.array_equal(ge, oe) and np.array_equal(gw, ow), l
    assert np.array_equal(s.decode_solution().cpu().numpy(), o.decode_solution())
