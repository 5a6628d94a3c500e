"""GPU adjoint (NEXT-2): gradients of J = |u - u_obs|^2 / 2 for the diffusion problem.

* the gradient kernel is bit-exact against the oracle's node formula;
* forward and adjoint compact solves with a nodal right-hand side are bit-exact
  against the oracle, and so are the resulting gradients, with the binary32
  cycle and with the plain binary64 cycle;
* the torch.autograd path (compact checkpoint, adjoint CMG solve, gradient
  kernel) agrees with central finite differences of J on the exact discrete
  system (dense FP64 solves), to the accuracy of the compact solves.
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


def make_oracle(prob, cfg, k):
    return oracle.Oracle(prob.dim, prob.Lmax, prob.tables, prob.scale_exp, b1=cfg.b1, b2=cfg.b2, N=cfg.N_ir,
                         nu1=cfg.nu1, nu2=cfg.nu2, omega=cfg.omega, arith=cfg.arith, coef=1, kfield=k)


@pytest.mark.parametrize("dim,L", [(3, 4), (2, 6)])
def test_gradient_kernel_matches_oracle(cmg, dim, L):
    prob = P.make_problem("diffusion%dd_grf" % dim, L)
    k = np.ascontiguousarray(prob.kfield().ravel())
    cfg = cmg.config_for(prob.name, L)
    s = cmg.Solver(cfg)
    s.set_coefficient(torch.from_numpy(k).cuda())
    rng = np.random.default_rng(2)
    n = ((1 << L) - 1) ** dim
    u = rng.standard_normal(n)
    lam = rng.standard_normal(n)
    dk, dg = s.gradient(torch.from_numpy(u).cuda(), torch.from_numpy(lam).cuda())
    o = make_oracle(prob, cfg, k)
    assert np.array_equal(dk.cpu().numpy(), o.gradient_k(u, lam))
    assert np.array_equal(dg.cpu().numpy(), np.ldexp(lam, -dim * L))


@pytest.mark.parametrize("dim,L,arith", [(3, 5, 1), (2, 6, 1), (3, 5, 2), (2, 6, 2)])
def test_forward_adjoint_and_gradients_match_oracle(cmg, dim, L, arith):
    prob = P.make_problem("diffusion%dd_grf" % dim, L)
    k = np.ascontiguousarray(prob.kfield().ravel())
    cfg = cmg.config_for(prob.name, L, arith=arith)
    n = ((1 << L) - 1) ** dim
    rng = np.random.default_rng(8)
    g = np.ones(n)
    uobs = 0.5 * rng.standard_normal(n) * 1e-3
    # forward
    s = cmg.Solver(cfg)
    s.set_coefficient(torch.from_numpy(k).cuda())
    gt = torch.from_numpy(g).cuda()
    s.set_rhs_nodal(gt)
    s.fmg_solve()
    o = make_oracle(prob, cfg, k)
    o.set_rhs_nodal(g)
    o.fmg()
    assert o.status == 0
    u_gpu = s.decode_solution().reshape(-1).cpu().numpy()
    u_orc = np.asarray(o.decode_solution()).ravel()
    assert np.array_equal(u_gpu, u_orc)
    # adjoint with the right-hand side 2^(dL) (u - u_obs): the library applies the
    # power-of-two scale; the oracle gets the scaled values
    rhs = np.ldexp(u_orc - uobs, dim * L)
    sa = cmg.Solver(cfg)
    sa.set_coefficient(torch.from_numpy(k).cuda())
    rt = torch.from_numpy(u_orc - uobs).cuda()
    sa.set_rhs_nodal(rt, dim * L)
    sa.fmg_solve()
    oa = make_oracle(prob, cfg, k)
    oa.set_rhs_nodal(rhs)
    oa.fmg()
    lam_gpu = sa.decode_solution().reshape(-1)
    lam_orc = np.asarray(oa.decode_solution()).ravel()
    assert np.array_equal(lam_gpu.cpu().numpy(), lam_orc)
    dk, dg = s.gradient(s.decode_solution().reshape(-1), lam_gpu)
    assert np.array_equal(dk.cpu().numpy(), o.gradient_k(u_orc, lam_orc))


def dense_assembly(k, dim, L):
    N = (1 << L) + 1
    n = N - 2
    kk = np.asarray(k, dtype=np.float64).reshape((N,) * dim)
    idx = -np.ones((N,) * dim, dtype=np.int64)
    idx[tuple(slice(1, -1) for _ in range(dim))] = np.arange(n ** dim).reshape((n,) * dim)
    A = np.zeros((n ** dim, n ** dim))
    h = 2.0 ** -L
    for p in np.ndindex(*((n,) * dim)):
        P1 = tuple(c + 1 for c in p)
        for a in range(dim):
            for sgn in (-1, 1):
                Q = list(P1)
                Q[a] += sgn
                Q = tuple(Q)
                kf = 0.5 * (kk[P1] + kk[Q])
                A[idx[P1], idx[P1]] += kf * h ** (dim - 2)
                if idx[Q] >= 0:
                    A[idx[P1], idx[Q]] -= kf * h ** (dim - 2)
    return A


def test_autograd_matches_central_differences(cmg):
    from paper_2511_19036_gb300.adjoint import diffusion_solve
    dim, L = 3, 4
    prob = P.make_problem("diffusion3d_grf", L)
    k = np.ascontiguousarray(prob.kfield().ravel())
    cfg = cmg.config_for(prob.name, L)
    cfg.b1, cfg.b2, cfg.N_ir = 14, 10, 16  # compact solves accurate to ~1e-6
    N, n = (1 << L) + 1, ((1 << L) - 1) ** dim
    rng = np.random.default_rng(13)
    g = np.ones(n) + 0.2 * rng.standard_normal(n)
    uobs = 1e-3 * rng.standard_normal(n)
    kt = torch.from_numpy(k).cuda().requires_grad_(True)
    gt = torch.from_numpy(g).cuda().requires_grad_(True)
    u = diffusion_solve(kt, gt, cfg)
    J = 0.5 * torch.sum((u - torch.from_numpy(uobs).cuda()) ** 2)
    dk, dg = torch.autograd.grad(J, (kt, gt))
    dk, dg = dk.double().cpu().numpy(), dg.cpu().numpy()
    h = 2.0 ** -L

    def Jexact(kv, gv):
        uu = np.linalg.solve(dense_assembly(kv, dim, L), h ** dim * gv)
        return 0.5 * np.sum((uu - uobs) ** 2)

    eps = 1e-6
    for _ in range(3):
        d1 = rng.standard_normal(N ** dim)
        fd = (Jexact(k.astype(np.float64) + eps * d1, g) - Jexact(k.astype(np.float64) - eps * d1, g)) / (2 * eps)
        assert abs(fd - dk @ d1) <= 2e-4 * abs(fd)
        d2 = rng.standard_normal(n)
        fd = (Jexact(k, g + eps * d2) - Jexact(k, g - eps * d2)) / (2 * eps)
        assert abs(fd - dg @ d2) <= 2e-4 * abs(fd)


def test_adjoint_workload_257_whole(cmg):
    """The 257^3 adjoint configuration whole: k = exp(m), m a GRF (sigma 0.5, seed 2),
    u_obs from m + a GRF (sigma 0.1, seed 3); forward solve, adjoint solve with the
    right-hand side 2^(dL) (u - u_obs), and both gradients, bit-exact against the oracle."""
    from cmg_problems.diffusion import diffusion_grf
    dim, L = 3, 8
    prob = diffusion_grf(dim, L, seed=2, sigma=0.5)
    pert = diffusion_grf(dim, L, seed=3, sigma=0.1)
    m = prob.g_field()
    k = np.exp(m).astype(np.float32).ravel()
    k_obs = np.exp(m + pert.g_field()).astype(np.float32).ravel()
    cfg = cmg.config_for("diffusion3d_grf", L)
    n = ((1 << L) - 1) ** dim
    g = np.ones(n)

    def solve_pair(kk, rhs, scale_log2=0):
        s = cmg.Solver(cfg)
        s.set_coefficient(torch.from_numpy(kk).cuda())
        s.set_rhs_nodal(torch.from_numpy(rhs).cuda(), scale_log2)
        s.fmg_solve()
        o = make_oracle(prob, cfg, kk)
        o.set_rhs_nodal(np.ldexp(rhs, scale_log2))
        o.fmg()
        assert o.status == 0
        ug = s.decode_solution().reshape(-1).cpu().numpy()
        uo = np.asarray(o.decode_solution()).ravel()
        assert np.array_equal(ug, uo)
        return s, o, uo

    _, _, uobs = solve_pair(k_obs, g)
    s, o, u = solve_pair(k, g)
    _, _, lam = solve_pair(k, u - uobs, dim * L)
    dk, dg = s.gradient(torch.from_numpy(u).cuda(), torch.from_numpy(lam).cuda())
    assert np.array_equal(dk.cpu().numpy(), o.gradient_k(u, lam))
    assert np.array_equal(dg.cpu().numpy(), np.ldexp(lam, -dim * L))


def test_forward_keeps_only_the_compact_checkpoint(cmg):
    """After forward returns, no solver context is alive (its residual, correction
    and temporaries are freed); the saved state is the compact u~ sections alone,
    and backward rebuilt from it gives the same gradient as the oracle path."""
    import gc
    from paper_2511_19036_gb300 import adjoint
    dim, L = 3, 4
    prob = P.make_problem("diffusion3d_grf", L)
    k = np.ascontiguousarray(prob.kfield().ravel())
    cfg = cmg.config_for(prob.name, L)
    n = ((1 << L) - 1) ** dim
    kt = torch.from_numpy(k).cuda().requires_grad_(True)
    gt = torch.ones(n, dtype=torch.float64, device="cuda").requires_grad_(True)
    live_before = sum(1 for o in gc.get_objects() if isinstance(o, cmg.Solver) and o._h)
    u = adjoint.diffusion_solve(kt, gt, cfg)
    gc.collect()
    live_after = sum(1 for o in gc.get_objects() if isinstance(o, cmg.Solver) and o._h)
    assert live_after == live_before
    node = u.grad_fn
    ck = node.checkpoint
    assert isinstance(ck, bytes)
    # header + per level: width, exponents, words of u~ only
    sec_bytes = sum(4 + int(cmg.lib().cmg_section_blocks(dim, l)) * (1 + 4 * (cfg.k_u * (L - l) + cfg.b1))
                    for l in range(1, L + 1))
    assert 0 < len(ck) - sec_bytes < 256
    J = 0.5 * torch.sum(u ** 2)
    dk, dg = torch.autograd.grad(J, (kt, gt))
    assert node.checkpoint is None  # released after backward
    assert torch.isfinite(dk).all() and torch.isfinite(dg).all()
