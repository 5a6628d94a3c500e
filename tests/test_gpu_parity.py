"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

The bar is bit-exact: codes, exponents and packed words of every section after
every step, and the decoded solution.  Exact arithmetic on both sides (the
oracle certifies zero inexact FP64 operations) makes this the correct bar.
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


def make_pair(cmg, name, Lmax, **over):
    prob = P.make_problem(name, Lmax)
    cfg = cmg.config_for(name, Lmax)
    for k, v in over.items():
        setattr(cfg, k, v)
    s = cmg.Solver(cfg)
    s.set_rhs(prob.tables, prob.scale_exp)
    o = oracle.Oracle.for_problem(prob, b1=cfg.b1, b2=cfg.b2, N=cfg.N_ir, nu1=cfg.nu1, nu2=cfg.nu2,
                                  omega=cfg.omega)
    return prob, cfg, s, o


def same_section(cmg, s, o, which_g, which_o, level, what=""):
    gw, ge = s.get_section(which_g, level)
    ow, oe, _ = o.get_section(which_o, level)
    assert s.width(which_g, level) == o.width(which_o, level)
    assert np.array_equal(ge, oe), "exponents differ: %s level %d (%d blocks)" % (
        what, level, int(np.sum(ge != oe)))
    assert np.array_equal(gw, ow), "words differ: %s level %d (%d words)" % (what, level, int(np.sum(gw != ow)))


# ---------------------------------------------------------------- codec
@pytest.mark.parametrize("W", [2, 3, 4, 5, 7, 8, 13, 16, 25, 31, 32])
@pytest.mark.parametrize("n", [0, 1, 31, 32, 33, 32 * 257 + 5])
def test_codec_bit_exact(cmg, W, n):
    x = random_block_values(n, seed=1000 + W + n)
    ow, oe, st = oracle.encode(x, W)
    assert st == 0
    xt = torch.tensor(x, dtype=torch.float64, device="cuda")
    gw, ge = cmg.encode(xt, W)
    torch.cuda.synchronize()
    assert np.array_equal(ge.cpu().numpy(), oe)
    assert np.array_equal(gw.cpu().numpy().view(np.uint32), ow)
    y = cmg.decode(gw, ge, n, W).cpu().numpy()
    yo, _ = oracle.decode(ow, oe, n, W)
    assert np.array_equal(y, yo)


def test_codec_ties_and_edges(cmg):
    x = np.zeros(64)
    x[:6] = [1.5, 0.25, 0.75, -0.25, -0.75, 1.9]
    x[32:36] = [2.0 ** -120, -(2.0 ** -121), 3 * 2.0 ** -122, 0.0]
    for W in (2, 3, 4):
        ow, oe, _ = oracle.encode(x, W)
        gw, ge = cmg.encode(torch.tensor(x, device="cuda"), W)
        assert np.array_equal(ge.cpu().numpy(), oe)
        assert np.array_equal(gw.cpu().numpy().view(np.uint32), ow)


def test_codec_errors(cmg):
    big = torch.zeros(32, dtype=torch.float64, device="cuda")
    big[0] = 2.0 ** 200
    with pytest.raises(cmg.CmgError) as ei:
        cmg.encode(big, 8)
    assert ei.value.status == cmg.ERANGE
    bad = torch.zeros(32, dtype=torch.float64, device="cuda")
    bad[3] = float("nan")
    with pytest.raises(cmg.CmgError) as ei:
        cmg.encode(bad, 8)
    assert ei.value.status == cmg.EINVAL
    words = torch.zeros(4, dtype=torch.int32, device="cuda")
    words[0] = 0b1000
    exps = torch.zeros(1, dtype=torch.int8, device="cuda")
    with pytest.raises(cmg.CmgError) as ei:
        cmg.decode(words, exps, 32, 4)
    assert ei.value.status == cmg.ECORRUPT


# ---------------------------------------------------------------- steps
STEP_CASES = [("poisson2d_manufactured", 6, {}), ("poisson3d_fourier", 5, {}),
              ("poisson3d_manufactured", 4, {"nu1": 0, "nu2": 1}),
              ("poisson2d_fourier", 6, {"nu1": 1, "nu2": 2}),
              ("poisson3d_fourier", 4, {"nu1": 3, "nu2": 1})]


@pytest.mark.parametrize("name,Lmax,over", STEP_CASES)
def test_step_parity(cmg, name, Lmax, over):
    prob, cfg, s, o = make_pair(cmg, name, Lmax, **over)
    s.start()
    o.start()
    same_section(cmg, s, o, cmg.SEC_U, oracle.U, 1, "start")
    for L in range(2, Lmax + 1):
        s.prolongate()
        o.next_level()
        for l in range(1, L + 1):
            same_section(cmg, s, o, cmg.SEC_U, oracle.U, l, "prolongate L=%d" % L)
        for it in range(2):
            s.residual()
            o.residual()
            same_section(cmg, s, o, cmg.SEC_R, oracle.R, L, "residual L=%d" % L)
            if cfg.nu1 == 0:
                for l in range(1, L):
                    same_section(cmg, s, o, cmg.SEC_R, oracle.R, l, "residual chain L=%d" % L)
            for l in range(L, 1, -1):
                s.down(l)
                o.down(l)
                same_section(cmg, s, o, cmg.SEC_Y, oracle.Y, l, "down L=%d" % L)
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
    assert o.inexact == 0


# ---------------------------------------------------------------- full solves
FMG_CASES = [("poisson2d_manufactured", 8, {}),       # 257^2, the 2-D workload
             ("poisson2d_manufactured", 3, {}),
             ("poisson2d_fourier", 7, {"nu1": 0, "nu2": 1}),
             ("poisson3d_fourier", 2, {}),
             ("poisson3d_fourier", 6, {}),
             ("poisson3d_fourier", 8, {}),          # the 257^3 configuration, whole
             ("poisson3d_manufactured", 6, {"nu1": 1, "nu2": 1}),
             ("poisson3d_fourier", 5, {"nu1": 0, "nu2": 2, "N_ir": 4})]


@pytest.mark.parametrize("name,Lmax,over", FMG_CASES)
def test_fmg_parity(cmg, name, Lmax, over):
    prob, cfg, s, o = make_pair(cmg, name, Lmax, **over)
    s.fmg_solve()
    o.fmg()
    assert o.inexact == 0
    for l in range(1, Lmax + 1):
        same_section(cmg, s, o, cmg.SEC_U, oracle.U, l, "fmg")
    u = s.decode_solution().cpu().numpy()
    assert np.array_equal(u, o.decode_solution())


def test_fmg_repeatable(cmg):
    prob, cfg, s, o = make_pair(cmg, "poisson3d_fourier", 6)
    s.fmg_solve()
    a = [s.get_section(cmg.SEC_U, l) for l in range(1, 7)]
    s.fmg_solve()
    b = [s.get_section(cmg.SEC_U, l) for l in range(1, 7)]
    for (w1, e1), (w2, e2) in zip(a, b):
        assert np.array_equal(w1, w2) and np.array_equal(e1, e2)


def test_ir_iteration_matches_oracle(cmg):
    """The fused production IR iteration equals the oracle's residual + cycle + correction."""
    prob, cfg, s, o = make_pair(cmg, "poisson3d_fourier", 5)
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


def test_checkpoint_roundtrip(cmg):
    prob, cfg, s, o = make_pair(cmg, "poisson2d_manufactured", 6)
    s.fmg_solve()
    blob = s.state_save()
    s2 = cmg.Solver(cfg)
    s2.set_rhs(prob.tables, prob.scale_exp)
    s2.state_load(blob)
    assert s2.level == 6
    assert np.array_equal(s.decode_solution().cpu().numpy(), s2.decode_solution().cpu().numpy())
    # a further IR iteration continues identically on both
    s.ir_iteration()
    s2.ir_iteration()
    for l in range(1, 7):
        a, b = s.get_section(cmg.SEC_U, l), s2.get_section(cmg.SEC_U, l)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_invalid_parameters(cmg):
    bad = [dict(dim=4), dict(L_max=0), dict(L_max=15), dict(b1=1), dict(nu2=0), dict(N_ir=0),
           dict(omega_num=4, omega_log2den=2)]  # 4/4 / 6 is not dyadic in 3-D
    for over in bad:
        cfg = cmg.config_for("poisson3d_fourier", 5)
        for k, v in over.items():
            setattr(cfg, k, v)
        assert cmg.params_check(cfg) in (cmg.EINVAL, cmg.ERANGE)
        with pytest.raises(cmg.CmgError):
            cmg.Solver(cfg)
    cfg = cmg.config_for("poisson3d_fourier", 14)
    cfg.b1 = 12  # u~ on level 1 would need 2*13 + 12 > 32 bits
    assert cmg.params_check(cfg) == cmg.ERANGE


def test_solve_without_rhs_is_rejected(cmg):
    s = cmg.Solver(cmg.config_for("poisson2d_manufactured", 4))
    with pytest.raises(cmg.CmgError) as ei:
        s.fmg_solve()
    assert ei.value.status == cmg.EINVAL


# ---------------------------------------------------------------- wide operands
def _rows(x, n, npts):
    rows = np.zeros((npts // n, 32 * ((n + 31) // 32)))
    rows[:, :n] = x.reshape(npts // n, n)
    return rows.ravel()


@pytest.mark.parametrize("name,L,smoother", [("poisson3d_manufactured", 5, 0), ("poisson3d_manufactured", 5, 1),
                                             ("poisson2d_manufactured", 6, 0), ("poisson2d_manufactured", 6, 1)])
def test_cycle_on_operands_wider_than_32_bits(cmg, name, L, smoother):
    """Sections whose rows are scaled over 16-36 binary orders (u~_L before the
    residual, r~_L before the down-leg, y~_L before the finest up-sweep): the
    stencil kernels meet footprints whose exact operands need more than 31 bits
    (the 64-bit march) next to footprints that fit (the 32-bit march).  The
    magnitudes keep every oracle operation exact; the bar is bit-exact."""
    prob = P.make_problem(name, L)
    cfg = cmg.config_for(name, L, smoother=smoother)
    s = cmg.Solver(cfg)
    s.set_rhs(prob.tables, prob.scale_exp)
    o = oracle.Oracle.for_problem(prob, b1=cfg.b1, b2=cfg.b2, N=cfg.N_ir, nu1=cfg.nu1, nu2=cfg.nu2,
                                  omega=cfg.omega, smoother=smoother)
    s.start()
    o.start()
    for _ in range(L - 1):
        s.prolongate()
        o.next_level()
        for _ in range(cfg.N_ir):
            s.ir_iteration()
            o.ir_iteration()
    n = (1 << L) - 1
    npts = n ** prob.dim
    rng = np.random.default_rng(5)

    def put(which_g, which_o, seed, lo, hi):
        W = o.width(which_o, L)
        x = random_block_values(npts, seed=seed, spread_bits=8) * np.repeat(
            2.0 ** rng.integers(lo, hi, size=npts // n).astype(np.float64), n)
        words, e, st = oracle.encode(_rows(x, n, npts), W)
        assert st == 0
        s.set_section(which_g, L, W, words, e)
        o.set_section(which_o, L, W, words, e)

    put(cmg.SEC_U, oracle.U, 17, -38, -22)
    s.residual()
    o.residual()
    same_section(cmg, s, o, cmg.SEC_R, oracle.R, L, "residual")
    put(cmg.SEC_R, oracle.R, 23, -50, -14)
    for l in range(L, 1, -1):
        s.down(l)
        o.down(l)
        same_section(cmg, s, o, cmg.SEC_RC, oracle.RC, l - 1, "restrict")
    s.coarse()
    o.coarse()
    for l in range(2, L):
        s.up(l)
        o.up(l)
        same_section(cmg, s, o, cmg.SEC_Y, oracle.Y, l, "up")
    put(cmg.SEC_Y, oracle.Y, 29, -50, -14)
    s.up(L)
    o.up(L)
    same_section(cmg, s, o, cmg.SEC_Y, oracle.Y, L, "up, finest")
    s.correct()
    o.correct()
    for l in range(1, L + 1):
        same_section(cmg, s, o, cmg.SEC_U, oracle.U, l, "correct")
    s.ir_iteration()
    o.ir_iteration()
    for l in range(1, L + 1):
        same_section(cmg, s, o, cmg.SEC_U, oracle.U, l, "fused iteration")
    assert o.status == 0 and o.inexact == 0


# ---------------------------------------------------------------- smoothing and restriction calls
@pytest.mark.parametrize("name,Lmax,smoother", [("poisson3d_fourier", 5, 0), ("poisson2d_manufactured", 6, 0),
                                                ("poisson3d_manufactured", 5, 1)])
def test_smooth_and_restrict_calls_match_the_cycle(cmg, name, Lmax, smoother):
    """cmg_smooth(l, nu1, 0) + cmg_restrict(l) is the down-leg and cmg_smooth(l, nu2, 1)
    the up-leg: bit-exact against the oracle's cycle steps."""
    prob = P.make_problem(name, Lmax)
    cfg = cmg.config_for(name, Lmax, smoother=smoother)
    s = cmg.Solver(cfg)
    s.set_rhs(prob.tables, prob.scale_exp)
    o = oracle.Oracle.for_problem(prob, b1=cfg.b1, b2=cfg.b2, N=cfg.N_ir, nu1=cfg.nu1, nu2=cfg.nu2,
                                  omega=cfg.omega, smoother=smoother)
    s.start()
    o.start()
    for L in range(2, Lmax + 1):
        s.prolongate()
        o.next_level()
        for it in range(cfg.N_ir):
            s.residual()
            o.residual()
            for l in range(L, 1, -1):
                if cfg.nu1 > 0:
                    s.smooth(l, cfg.nu1, False)
                    s.restrict(l)
                else:
                    s.down(l)
                o.down(l)
                same_section(cmg, s, o, cmg.SEC_RC, oracle.RC, l - 1, "restrict L=%d" % L)
            s.coarse()
            o.coarse()
            for l in range(2, L + 1):
                s.smooth(l, cfg.nu2, True)
                o.up(l)
                same_section(cmg, s, o, cmg.SEC_Y, oracle.Y, l, "up L=%d" % L)
            s.correct()
            o.correct()
        for l in range(1, L + 1):
            same_section(cmg, s, o, cmg.SEC_U, oracle.U, l, "L=%d" % L)
    assert o.status == 0 and o.inexact == 0
    if smoother:
        with pytest.raises(cmg.CmgError) as ei:
            s.smooth(Lmax, 1, False)
        assert ei.value.status == cmg.EUNSUPPORTED
        with pytest.raises(cmg.CmgError) as ei:
            s.restrict(Lmax)
        assert ei.value.status == cmg.EUNSUPPORTED
    with pytest.raises(cmg.CmgError):
        s.smooth(1, 1, True)


@pytest.mark.parametrize("name", ["poisson3d_fourier", "poisson2d_manufactured"])
def test_one_level_hierarchy(cmg, name):
    """L_max = 1, one unknown: the FMG is the coarse solve u~_1 = round(f_1 / A_1); a
    cycle on it is refused."""
    prob, cfg, s, o = make_pair(cmg, name, 1)
    s.fmg_solve()
    o.fmg()
    assert o.status == 0
    same_section(cmg, s, o, cmg.SEC_U, oracle.U, 1, "L_max = 1")
    assert np.array_equal(s.decode_solution().cpu().numpy(), o.decode_solution())
    with pytest.raises(cmg.CmgError) as ei:
        s.ir_iteration()
    assert ei.value.status == cmg.EINVAL
    with pytest.raises(cmg.CmgError) as ei:
        s.coarse()
    assert ei.value.status == cmg.EUNSUPPORTED


def test_values_beyond_62_bits_raise_erange(cmg):
    """u~_L with rows scaled over 120 binary orders: the residual's exact operand
    would need more than 62 bits; the kernels flag it and the call reports
    CMG_ERANGE (the values never wrap)."""
    name, L = "poisson3d_fourier", 4
    prob, cfg, s, o = make_pair(cmg, name, L)
    s.start()
    for _ in range(L - 1):
        s.prolongate()
    n = (1 << L) - 1
    npts = n ** 3
    W = s.width(cmg.SEC_U, L)
    rng = np.random.default_rng(3)
    x = random_block_values(npts, seed=5, spread_bits=4) * np.repeat(
        2.0 ** rng.integers(-120, 0, size=npts // n).astype(np.float64), n)
    rows = np.zeros((npts // n, 32 * ((n + 31) // 32)))
    rows[:, :n] = x.reshape(npts // n, n)
    words, e, st = oracle.encode(rows.ravel(), W)
    assert st == 0
    s.set_section(cmg.SEC_U, L, W, words, e)
    with pytest.raises(cmg.CmgError) as ei:
        s.residual()
        s.sync()
    assert ei.value.status == cmg.ERANGE


@pytest.mark.parametrize("level_from_top", [0, 1])
def test_invalid_code_in_a_section_raises_ecorrupt(cmg, level_from_top):
    """A code -2^(W-1) (never written by an encoder) in u~ is reported as
    CMG_ECORRUPT by cmg_decode_solution, on the finest section (decode kernel)
    and on a coarse one (decode chain)."""
    prob, cfg, s, o = make_pair(cmg, "poisson3d_manufactured", 5)
    s.fmg_solve()
    l = 5 - level_from_top
    w, e = s.get_section(cmg.SEC_U, l)
    W = s.width(cmg.SEC_U, l)
    w = w.copy()
    blk = int(np.flatnonzero(e != -128)[0])
    stream = 0
    for k in range(W):
        stream |= int(w[blk * W + k]) << (32 * k)
    stream = (stream & ~((1 << W) - 1)) | (1 << (W - 1))
    for k in range(W):
        w[blk * W + k] = (stream >> (32 * k)) & 0xFFFFFFFF
    s.set_section(cmg.SEC_U, l, W, w, e)
    with pytest.raises(cmg.CmgError) as ei:
        s.decode_solution()
    assert ei.value.status == cmg.ECORRUPT
