"""GPU parity of the variable-coefficient diffusion path.

-div(k grad u) = 1 with k = exp(GRF): the CUDA path (FP64 outer residual,
binary32 cycle, FP64 level-1 solve, each in its fixed order) against the
oracle's diffusion mode on the same binary32 coefficient array, bit-exact
after every step and for whole solves.
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


def make_pair(cmg, dim, L, **over):
    name = "diffusion%dd_grf" % dim
    prob = P.make_problem(name, L)
    k = np.ascontiguousarray(prob.kfield().ravel())
    cfg = cmg.config_for(name, L)
    for key, v in over.items():
        setattr(cfg, key, v)
    s = cmg.Solver(cfg)
    s.set_rhs(prob.tables, prob.scale_exp)
    s.set_coefficient(torch.from_numpy(k).cuda())
    o = oracle.Oracle(dim, L, prob.tables, prob.scale_exp, b1=cfg.b1, b2=cfg.b2, N=cfg.N_ir, nu1=cfg.nu1,
                      nu2=cfg.nu2, omega=cfg.omega, arith=1, coef=1, kfield=k)
    return prob, cfg, s, o


def same_section(cmg, s, o, which_g, which_o, level, what=""):
    gw, ge = s.get_section(which_g, level)
    ow, oe, _ = o.get_section(which_o, level)
    assert s.width(which_g, level) == o.width(which_o, level)
    assert np.array_equal(ge, oe), "exponents differ: %s level %d (%d blocks)" % (
        what, level, int(np.sum(ge != oe)))
    assert np.array_equal(gw, ow), "words differ: %s level %d (%d words)" % (what, level, int(np.sum(gw != ow)))


@pytest.mark.parametrize("dim,L,over", [(3, 4, {}), (3, 6, {}), (2, 7, {}), (3, 5, {"nu1": 1, "nu2": 1, "N_ir": 4})])
def test_fmg_parity_diffusion(cmg, dim, L, over):
    prob, cfg, s, o = make_pair(cmg, dim, L, **over)
    s.fmg_solve()
    o.fmg()
    assert o.status == 0
    for l in range(1, L + 1):
        same_section(cmg, s, o, cmg.SEC_U, oracle.U, l, "fmg diffusion")
    assert np.array_equal(s.decode_solution().cpu().numpy(), o.decode_solution())


@pytest.mark.parametrize("dim,L", [(3, 5), (2, 6)])
def test_cycle_steps_diffusion(cmg, dim, L):
    prob, cfg, s, o = make_pair(cmg, dim, L)
    s.start()
    o.start()
    same_section(cmg, s, o, cmg.SEC_U, oracle.U, 1, "start")
    for Lc in range(2, L + 1):
        s.prolongate()
        o.next_level()
        s.residual()
        o.residual()
        same_section(cmg, s, o, cmg.SEC_R, oracle.R, Lc, "residual L=%d" % Lc)
        for l in range(Lc, 1, -1):
            s.down(l)
            o.down(l)
            same_section(cmg, s, o, cmg.SEC_Y, oracle.Y, l, "down L=%d" % Lc)
            same_section(cmg, s, o, cmg.SEC_RC, oracle.RC, l - 1, "restrict L=%d" % Lc)
        s.coarse()
        o.coarse()
        same_section(cmg, s, o, cmg.SEC_Y, oracle.Y, 1, "coarse L=%d" % Lc)
        for l in range(2, Lc + 1):
            s.up(l)
            o.up(l)
            same_section(cmg, s, o, cmg.SEC_Y, oracle.Y, l, "up L=%d" % Lc)
        s.correct()
        o.correct()
        for l in range(1, Lc + 1):
            same_section(cmg, s, o, cmg.SEC_U, oracle.U, l, "correct L=%d" % Lc)
    assert o.status == 0


def test_diffusion_needs_the_fp32_cycle_and_a_coefficient(cmg):
    cfg = cmg.config_for("diffusion3d_grf", 5)
    cfg.arith = 0
    assert cmg.params_check(cfg) == cmg.EINVAL
    cfg = cmg.config_for("diffusion3d_grf", 5)
    cfg.nu1 = 0
    assert cmg.params_check(cfg) == cmg.EINVAL
    s = cmg.Solver(cmg.config_for("diffusion3d_grf", 4))
    prob = P.make_problem("diffusion3d_grf", 4)
    s.set_rhs(prob.tables, prob.scale_exp)
    with pytest.raises(cmg.CmgError):
        s.fmg_solve()  # no coefficient set
    with pytest.raises(cmg.CmgError):
        s.set_coefficient(torch.ones(10, dtype=torch.float32, device="cuda"))  # wrong size
