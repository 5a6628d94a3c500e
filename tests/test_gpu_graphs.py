"""The solve replayed as one CUDA graph gives the eager solve's bits (GPU).

cmg_fmg_solve runs the first solve of new inputs eagerly, captures the second
into a CUDA graph and launches that graph for later solves, restoring the host
state of the captured solve before each launch.  These tests check that every
replay gives the eager solve's sections bit for bit (and the oracle's), that
the statistics of a replay equal those of an eager solve, and that a change of
input or configuration drops the graph while an unchanged right-hand side
keeps it.
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


def sections(s, cmg, L):
    return [s.get_section(cmg.SEC_U, l) for l in range(1, L + 1)]


def same_sections(a, b):
    return all(np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1]) for x, y in zip(a, b))


def launch_counts(st):
    return {k: v["launches"] for k, v in st.items()}


@pytest.mark.parametrize("name,L,smoother", [("poisson3d_manufactured", 6, 1), ("poisson3d_fourier", 5, 0),
                                             ("poisson2d_manufactured", 7, 1)])
def test_graph_replays_equal_the_eager_solve_and_the_oracle(cmg, name, L, smoother):
    prob = P.make_problem(name, L)
    cfg = cmg.config_for(name, L, smoother=smoother)
    eager = cmg.Solver(cfg, stream=torch.cuda.Stream(), timing=True, graphs=False)
    eager.set_rhs(prob.tables, prob.scale_exp)
    erep = eager.fmg_solve()
    ref = sections(eager, cmg, L)
    ref_u = eager.decode_solution().cpu().numpy()
    ref_stats = launch_counts(eager.kernel_stats())
    assert eager.graph_stats() == {"captures": 0, "graph_solves": 0}

    o = oracle.Oracle.for_problem(prob, b1=cfg.b1, b2=cfg.b2, N=cfg.N_ir, nu1=cfg.nu1, nu2=cfg.nu2,
                                  omega=cfg.omega, smoother=smoother)
    o.fmg()
    assert o.status == 0 and o.inexact == 0
    for l in range(1, L + 1):
        ow, oe, _ = o.get_section(oracle.U, l)
        assert np.array_equal(ref[l - 1][0], ow) and np.array_equal(ref[l - 1][1], oe), l

    s = cmg.Solver(cfg, stream=torch.cuda.Stream(), timing=True)
    s.set_rhs(prob.tables, prob.scale_exp)
    for it in range(4):  # eager, capture + launch, two replays
        rep = s.fmg_solve()
        assert same_sections(sections(s, cmg, L), ref), it
        assert np.array_equal(s.decode_solution().cpu().numpy(), ref_u), it
        assert rep["launches"] == erep["launches"] and rep["alg_bytes"] == erep["alg_bytes"]
        assert launch_counts(s.kernel_stats()) == ref_stats
        if prob.dim == 3:
            assert s.fast_stats() == eager.fast_stats()
    assert s.graph_stats() == {"captures": 1, "graph_solves": 3}
    # the replay's per-kernel times come from event records inside the graph
    ks = s.kernel_stats()
    assert ks["sweep_top"]["ms"] > 0 and ks["residual_top"]["ms"] > 0
    assert rep["sweep_ms_total"] > 0 and rep["solve_ms"] > 0


def test_inputs_and_settings_drop_the_graph(cmg):
    name, L = "poisson3d_manufactured", 5
    pa = P.make_problem(name, L)
    pb = P.make_problem("poisson3d_fourier", L)
    cfg = cmg.config_for(name, L)
    cfg_b = cmg.config_for("poisson3d_fourier", L)
    assert (cfg_b.b1, cfg_b.b2, cfg_b.N_ir, cfg_b.smoother) == (cfg.b1, cfg.b2, cfg.N_ir, cfg.smoother)

    def eager_solution(prob):
        e = cmg.Solver(cfg, stream=torch.cuda.Stream(), graphs=False)
        e.set_rhs(prob.tables, prob.scale_exp)
        e.fmg_solve()
        return sections(e, cmg, L)

    ref_a, ref_b = eager_solution(pa), eager_solution(pb)
    assert not same_sections(ref_a, ref_b)
    s = cmg.Solver(cfg, stream=torch.cuda.Stream())
    s.set_rhs(pa.tables, pa.scale_exp)
    for _ in range(3):
        s.fmg_solve()
    assert s.graph_stats() == {"captures": 1, "graph_solves": 2}
    # the same tables again (the end-to-end loop): the graph stays
    s.set_rhs(pa.tables, pa.scale_exp)
    s.fmg_solve()
    assert s.graph_stats() == {"captures": 1, "graph_solves": 3}
    assert same_sections(sections(s, cmg, L), ref_a)
    # other tables: eager, then a new capture, each with the new solution
    s.set_rhs(pb.tables, pb.scale_exp)
    for it in range(3):
        s.fmg_solve()
        assert same_sections(sections(s, cmg, L), ref_b), it
    assert s.graph_stats() == {"captures": 2, "graph_solves": 5}
    # settings that change the launches drop it too
    for setter in (lambda: s.set_two_level(True), lambda: cmg.lib().cmg_set_fast_kernels(s._h, 0),
                   lambda: cmg.lib().cmg_set_timing(s._h, 1), lambda: s.set_two_level(False)):
        setter()
        before = s.graph_stats()
        s.fmg_solve()  # eager
        assert s.graph_stats() == before
        for _ in range(2):
            s.fmg_solve()
            assert same_sections(sections(s, cmg, L), ref_b)
        assert s.graph_stats()["captures"] == before["captures"] + 1
    # a step call between solves: the next solve runs eagerly from the start
    s.start()
    before = s.graph_stats()
    s.fmg_solve()
    assert s.graph_stats() == before and same_sections(sections(s, cmg, L), ref_b)
    # graphs off: eager solves only
    s.set_graphs(False)
    for _ in range(3):
        s.fmg_solve()
    assert s.graph_stats() == before and same_sections(sections(s, cmg, L), ref_b)


def test_no_graph_on_the_legacy_default_stream(cmg):
    name, L = "poisson3d_fourier", 4
    prob = P.make_problem(name, L)
    s = cmg.Solver(cmg.config_for(name, L), stream=0)
    s.set_rhs(prob.tables, prob.scale_exp)
    for _ in range(3):
        s.fmg_solve()
    assert s.graph_stats() == {"captures": 0, "graph_solves": 0}


def test_diffusion_replays_read_the_coefficient_through_its_pointer(cmg):
    # the binary32 cycle of the diffusion problem: the graph keeps the borrowed
    # coefficient pointer, so new values at the same address need no new graph
    name, L = "diffusion3d_grf", 5
    prob = P.make_problem(name, L)
    cfg = cmg.config_for(name, L)
    k0 = prob.kfield(device="cuda").reshape(-1).contiguous()
    k1 = (k0 * 1.5).contiguous()
    torch.cuda.synchronize()  # the fields are made on torch's stream, the solvers use their own

    def eager(k):
        e = cmg.Solver(cfg, stream=torch.cuda.Stream(), graphs=False)
        e.set_rhs(prob.tables, prob.scale_exp)
        e.set_coefficient(k)
        e.fmg_solve()
        return sections(e, cmg, L)

    ref0, ref1 = eager(k0), eager(k1)
    assert not same_sections(ref0, ref1)
    kf = k0.clone()
    s = cmg.Solver(cfg, stream=torch.cuda.Stream())
    s.set_rhs(prob.tables, prob.scale_exp)
    s.set_coefficient(kf)
    torch.cuda.synchronize()
    for it in range(3):
        s.fmg_solve()
        assert same_sections(sections(s, cmg, L), ref0), it
    kf.copy_(k1)
    torch.cuda.synchronize()
    s.set_coefficient(kf)
    s.fmg_solve()
    assert same_sections(sections(s, cmg, L), ref1)
    assert s.graph_stats() == {"captures": 1, "graph_solves": 3}


def test_finest_level_timing_mode(cmg):
    # cmg_set_timing mode 2: events around the level-L_max launches only, also
    # inside the graph; the launch counts of every level stay
    name, L = "poisson3d_manufactured", 6
    prob = P.make_problem(name, L)
    s = cmg.Solver(cmg.config_for(name, L, smoother=1), stream=torch.cuda.Stream(), timing="top")
    s.set_rhs(prob.tables, prob.scale_exp)
    for it in range(3):
        rep = s.fmg_solve()
        ks = s.kernel_stats()
        assert ks["sweep_top"]["ms"] > 0 and ks["residual_top"]["ms"] > 0, it
        assert ks["sweep_lower"]["ms"] == 0 and ks["sweep_lower"]["launches"] > 0, it
        assert rep["sweep_ms_total"] > 0 and rep["resid_ms_total"] > 0, it
    assert s.graph_stats() == {"captures": 1, "graph_solves": 2}
    assert cmg.lib().cmg_set_timing(s._h, 3) == cmg.EINVAL
