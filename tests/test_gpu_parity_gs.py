"""GPU parity of the red-black Gauss-Seidel V(0, nu2) cycle.

The CUDA path with smoother = CMG_SMOOTHER_RBGS (each post-smoothing sweep a
red half-sweep, then a black one fused with the correction, w_l and u^_l)
against the oracle with smoother = 1: bit-exact sections after every step of
the cycle and for whole solves, in exact arithmetic (2-D omega = 1, plain
Gauss-Seidel; 3-D omega = 3/4, so that omega/6 stays dyadic) and in the
binary32 cycle.
"""
import numpy as np
import pytest

import cmg_problems as P
import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cmg():
    from paper_2511_19036_gb300 import cmg as m
    return m


def make_pair(cmg, name, Lmax, arith=0, **over):
    prob = P.make_problem(name, Lmax)
    cfg = cmg.config_for(name, Lmax, arith=arith, smoother=1)
    for k, v in over.items():
        setattr(cfg, k, v)
    s = cmg.Solver(cfg)
    s.set_rhs(prob.tables, prob.scale_exp)
    o = oracle.Oracle.for_problem(prob, b1=cfg.b1, b2=cfg.b2, N=cfg.N_ir, nu1=cfg.nu1, nu2=cfg.nu2,
                                  omega=cfg.omega, arith=arith, smoother=1)
    return prob, cfg, s, o


def same_section(cmg, s, o, which_g, which_o, level, what=""):
    gw, ge = s.get_section(which_g, level)
    ow, oe, _ = o.get_section(which_o, level)
    assert s.width(which_g, level) == o.width(which_o, level)
    assert np.array_equal(ge, oe), "exponents differ: %s level %d (%d blocks)" % (
        what, level, int(np.sum(ge != oe)))
    assert np.array_equal(gw, ow), "words differ: %s level %d (%d words)" % (what, level, int(np.sum(gw != ow)))


STEP_CASES = [("poisson2d_manufactured", 6, 0, {}), ("poisson3d_fourier", 5, 0, {}),
              ("poisson3d_manufactured", 4, 0, {"nu2": 2}), ("poisson2d_fourier", 7, 1, {}),
              ("poisson3d_fourier", 5, 1, {"nu2": 2}), ("poisson3d_fourier", 5, 2, {}),
              ("poisson2d_manufactured", 6, 2, {})]


@pytest.mark.parametrize("name,Lmax,arith,over", STEP_CASES)
def test_step_parity_red_black(cmg, name, Lmax, arith, over):
    prob, cfg, s, o = make_pair(cmg, name, Lmax, arith, **over)
    s.start()
    o.start()
    for L in range(2, Lmax + 1):
        s.prolongate()
        o.next_level()
        for it in range(2):
            s.residual()
            o.residual()
            for l in range(L, 1, -1):
                s.down(l)
                o.down(l)
                same_section(cmg, s, o, cmg.SEC_RC, oracle.RC, l - 1, "restrict L=%d" % L)
            s.coarse()
            o.coarse()
            same_section(cmg, s, o, cmg.SEC_Y, oracle.Y, 1, "coarse L=%d" % L)
            for l in range(2, L + 1):
                s.up(l)
                o.up(l)
                same_section(cmg, s, o, cmg.SEC_Y, oracle.Y, l, "up L=%d" % L)
            s.correct()
            o.correct()
            for l in range(1, L + 1):
                same_section(cmg, s, o, cmg.SEC_U, oracle.U, l, "correct L=%d" % L)
    assert o.status == 0 and o.inexact == 0


FMG_CASES = [("poisson2d_manufactured", 8, 0, {}),   # Table 2's 2-D constants, 257^2
             ("poisson3d_fourier", 8, 0, {}),        # the 257^3 configuration, whole
             ("poisson2d_fourier", 3, 0, {}),
             ("poisson3d_fourier", 6, 0, {}),
             ("poisson3d_manufactured", 5, 0, {"nu2": 2, "N_ir": 4}),
             ("poisson2d_manufactured", 10, 1, {}),  # binary32 rounds in the cycle
             ("poisson3d_fourier", 6, 1, {}),
             ("poisson2d_manufactured", 10, 2, {}),  # binary64 cycle
             ("poisson3d_fourier", 6, 2, {})]


@pytest.mark.parametrize("name,Lmax,arith,over", FMG_CASES)
def test_fmg_parity_red_black(cmg, name, Lmax, arith, over):
    prob, cfg, s, o = make_pair(cmg, name, Lmax, arith, **over)
    s.fmg_solve()
    o.fmg()
    assert o.status == 0 and o.inexact == 0
    for l in range(1, Lmax + 1):
        same_section(cmg, s, o, cmg.SEC_U, oracle.U, l, "fmg red-black")
    assert np.array_equal(s.decode_solution().cpu().numpy(), o.decode_solution())


def test_fused_ir_iteration_red_black(cmg):
    """The production IR iteration (black half-sweep fused with u~, w, u^) against the oracle."""
    prob, cfg, s, o = make_pair(cmg, "poisson3d_manufactured", 5)
    s.start()
    o.start()
    for L in range(2, 6):
        s.prolongate()
        o.next_level()
        for _ in range(cfg.N_ir):
            s.ir_iteration()
            o.ir_iteration()
        for l in range(1, L + 1):
            same_section(cmg, s, o, cmg.SEC_U, oracle.U, l, "ir L=%d" % L)
