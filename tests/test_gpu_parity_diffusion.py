"""GPU parity of the variable-coefficient diffusion path.

-div(k grad u) = 1 with k = exp(GRF): the CUDA path (FP64 outer residual,
binary32 or binary64 cycle, FP64 level-1 solve, each in its fixed order)
against the oracle's diffusion mode on the same binary32 coefficient array,
bit-exact after every step and for whole solves, including a solve at widths
where the binary64 cycle's roundings reach the stored sections (its result
differs from the binary32 cycle's).
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


def make_pair(cmg, dim, L, arith=1, **over):
    name = "diffusion%dd_grf" % dim
    prob = P.make_problem(name, L)
    k = np.ascontiguousarray(prob.kfield().ravel())
    cfg = cmg.config_for(name, L, arith=arith)
    for key, v in over.items():
        setattr(cfg, key, v)
    s = cmg.Solver(cfg)
    s.set_rhs(prob.tables, prob.scale_exp)
    s.set_coefficient(torch.from_numpy(k).cuda())
    o = oracle.Oracle(dim, L, prob.tables, prob.scale_exp, b1=cfg.b1, b2=cfg.b2, N=cfg.N_ir, nu1=cfg.nu1,
                      nu2=cfg.nu2, omega=cfg.omega, arith=arith, coef=1, kfield=k)
    return prob, cfg, s, o


def same_section(cmg, s, o, which_g, which_o, level, what=""):
    gw, ge = s.get_section(which_g, level)
    ow, oe, _ = o.get_section(which_o, level)
    assert s.width(which_g, level) == o.width(which_o, level)
    assert np.array_equal(ge, oe), "exponents differ: %s level %d (%d blocks)" % (
        what, level, int(np.sum(ge != oe)))
    assert np.array_equal(gw, ow), "words differ: %s level %d (%d words)" % (what, level, int(np.sum(gw != ow)))


@pytest.mark.parametrize("dim,L,arith,over", [(3, 4, 1, {}), (3, 6, 1, {}), (2, 7, 1, {}),
                                              (3, 5, 1, {"nu1": 1, "nu2": 1, "N_ir": 4}),
                                              (3, 6, 2, {}), (2, 7, 2, {}), (3, 5, 2, {"nu1": 1, "nu2": 1, "N_ir": 4})])
def test_fmg_parity_diffusion(cmg, dim, L, arith, over):
    prob, cfg, s, o = make_pair(cmg, dim, L, arith, **over)
    s.fmg_solve()
    o.fmg()
    assert o.status == 0
    for l in range(1, L + 1):
        same_section(cmg, s, o, cmg.SEC_U, oracle.U, l, "fmg diffusion")
    assert np.array_equal(s.decode_solution().cpu().numpy(), o.decode_solution())


@pytest.mark.parametrize("dim,L,arith", [(3, 5, 1), (2, 6, 1), (3, 5, 2), (2, 6, 2)])
def test_cycle_steps_diffusion(cmg, dim, L, arith):
    prob, cfg, s, o = make_pair(cmg, dim, L, arith)
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


@pytest.mark.parametrize("dim,L", [(3, 6), (2, 8)])
def test_fp64_cycle_where_its_roundings_show(cmg, dim, L):
    # wide sections keep the low bits of the cycle: the binary64 and binary32
    # cycles give different solutions, and the GPU matches the oracle in both
    wide = {"b1": 14, "b2": 10}
    prob, cfg, s, o = make_pair(cmg, dim, L, 2, **wide)
    s.fmg_solve()
    o.fmg()
    assert o.status == 0
    for l in range(1, L + 1):
        same_section(cmg, s, o, cmg.SEC_U, oracle.U, l, "fmg diffusion fp64 wide")
    _, _, s32, o32 = make_pair(cmg, dim, L, 1, **wide)
    s32.fmg_solve()
    o32.fmg()
    u64, u32 = o.decode_solution(), o32.decode_solution()
    assert not np.array_equal(u64, u32)
    assert np.array_equal(s32.decode_solution().cpu().numpy(), u32)


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
