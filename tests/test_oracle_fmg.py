"""Pins for the oracle's compact FMG (Algorithms 1-3) against what the paper and
the mathematics fix: the coarse solve, the exact discrete solution on tiny
grids, equivalence of the compact cycle with a textbook correction-scheme
V-cycle, the success criteria of Sec. 7.1, linear storage (Sec. 6.1.1) and the
exactness of the arithmetic."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import cmg_problems as P
from cmg_problems.diagnostics import exact_on_grid, h1_error
from fem_dense import load_vector_exact, prolongation, stiffness

CFG2 = dict(b1=4, b2=4, N=3, nu1=2, nu2=2, omega=0.75)   # 2-D widths (Table 2, Poisson 2D, p=1)
CFG3 = dict(b1=5, b2=3, N=3, nu1=2, nu2=2, omega=0.75)   # 3-D widths tuned by the Sec. 7.1 search


def rne_fraction(x: Fraction, W: int):
    """Reference BFP rounding of a single value block (pure rationals)."""
    if x == 0:
        return Fraction(0), -128
    M = abs(x)
    e = 0
    while Fraction(2) ** e <= M:
        e += 1
    while Fraction(2) ** (e - 1) > M:
        e -= 1
    for _ in range(2):
        s = Fraction(2) ** (e - W + 1)
        v = x / s
        q = int(v // 1)
        r = v - q
        if r > Fraction(1, 2) or (r == Fraction(1, 2) and q % 2 == 1):
            q += 1
        if abs(q) >= 2 ** (W - 1):
            e += 1
            continue
        return q * s, e
    raise AssertionError


@pytest.mark.parametrize("name,Lmax", [("poisson2d_manufactured", 3), ("poisson3d_fourier", 3),
                                       ("poisson3d_manufactured", 2)])
def test_coarsest_level_solve(name, Lmax):
    """Algorithm 3 starts with u~_1 = round(A_1^-1 f_1); A_1 = 4 (2-D) or 3 (3-D)."""
    prob = P.make_problem(name, Lmax)
    cfg = CFG2 if prob.dim == 2 else CFG3
    o = oracle.Oracle.for_problem(prob, **cfg)
    o.start()
    f1 = Fraction(load_vector_exact(prob.tables, prob.scale_exp, prob.dim, Lmax, 1)[0])
    A1 = 4 if prob.dim == 2 else 3
    v, e = rne_fraction(f1 / A1, cfg["b1"])
    _, eo, vo = o.get_section(oracle.U, 1)
    assert eo[0] == e and Fraction(vo.reshape(-1)[0]) == v


@pytest.mark.parametrize("name,Lmax", [("poisson2d_manufactured", 4), ("poisson2d_fourier", 4),
                                       ("poisson3d_fourier", 3)])
def test_lossless_fmg_reaches_direct_solve(name, Lmax):
    prob = P.make_problem(name, Lmax)
    o = oracle.Oracle.for_problem(prob, b1=0, b2=0, N=25, nu1=2, nu2=2, omega=0.75)
    o.fmg()
    K = stiffness(prob.dim, Lmax)
    f = load_vector_exact(prob.tables, prob.scale_exp, prob.dim, Lmax, Lmax)
    u = np.linalg.solve(K, f)
    got = o.decode_solution().reshape(-1)
    assert np.max(np.abs(got - u)) <= 1e-10 * np.max(np.abs(u))  # FP64 rounding, lossless storage


@pytest.mark.parametrize("name,Lmax", [("poisson2d_manufactured", 5), ("poisson3d_manufactured", 4)])
def test_quantised_fmg_near_direct_solve(name, Lmax):
    """With the production widths the IR fixed point is the discrete solution up
    to the quantisation of the finest section (a few units of its last bit)."""
    prob = P.make_problem(name, Lmax)
    cfg = dict(CFG2 if prob.dim == 2 else CFG3)
    cfg["N"] = 20
    o = oracle.Oracle.for_problem(prob, **cfg)
    o.fmg()
    K = stiffness(prob.dim, Lmax)
    f = load_vector_exact(prob.tables, prob.scale_exp, prob.dim, Lmax, Lmax)
    u = np.linalg.solve(K, f)
    got = o.decode_solution().reshape(-1)
    _, eL, _ = o.get_section(oracle.U, Lmax)
    ulp = 2.0 ** (int(eL.max()) - cfg["b1"] + 1)
    assert np.max(np.abs(got - u)) <= 8 * ulp
    assert o.inexact == 0


def textbook_cs_vcycle(Ks, Ps, r, omega, nu1, nu2, dim):
    """Correction-scheme V(nu1, nu2) cycle with weighted Jacobi (supplement,
    Sec. SM1.1), written with dense matrices; returns the fine correction."""
    L = len(Ks) - 1

    def cyc(l, b):
        if l == 1:
            return b / Ks[1][0, 0]
        D = np.diag(Ks[l])
        y = np.zeros_like(b)
        for _ in range(nu1):
            y = y + omega / D * (b - Ks[l] @ y)
        d = cyc(l - 1, Ps[l].T @ (b - Ks[l] @ y))
        y = y + Ps[l] @ d
        for _ in range(nu2):
            y = y + omega / D * (b - Ks[l] @ y)
        return y

    return cyc(L, r)


@pytest.mark.parametrize("dim,Lmax,nu1,nu2", [(2, 4, 2, 2), (2, 4, 0, 1), (2, 5, 1, 2), (3, 3, 2, 2),
                                              (3, 3, 0, 1)])
def test_compact_cycle_equals_textbook_cs(dim, Lmax, nu1, nu2):
    """With lossless storage one compact cycle (eq. cfas, Algorithm 1 generalised to
    V(nu1, nu2)) yields the same correction as the textbook CS V-cycle."""
    prob = P.make_problem("poisson2d_fourier" if dim == 2 else "poisson3d_fourier", Lmax)
    o = oracle.Oracle.for_problem(prob, b1=0, b2=0, N=1, nu1=nu1, nu2=nu2, omega=0.75)
    o.start()
    for _ in range(2, Lmax + 1):
        o.next_level()
    o.residual()
    r = o.get_section(oracle.R, Lmax, words=False)[2].reshape(-1)
    o.vcycle()
    Ks = [None] + [stiffness(dim, l) for l in range(1, Lmax + 1)]
    Ps = [None, None] + [prolongation(dim, l) for l in range(2, Lmax + 1)]
    ycomp = None
    for l in range(1, Lmax + 1):
        yl = o.get_section(oracle.Y, l, words=False)[2].reshape(-1)
        ycomp = yl if l == 1 else yl + Ps[l] @ ycomp
    ycs = textbook_cs_vcycle(Ks, Ps, r, 0.75, nu1, nu2, dim)
    assert np.max(np.abs(ycomp - ycs)) <= 1e-13 * np.max(np.abs(ycs))
    # the cycle's w_L is the same sum, formed level by level
    assert np.max(np.abs(o.last_w(Lmax).reshape(-1) - ycs)) <= 1e-13 * np.max(np.abs(ycs))


def _h1_errors(prob, Lmax, **cfg):
    o = oracle.Oracle.for_problem(prob, **cfg)
    o.start()
    errs = []
    for L in range(2, Lmax + 1):
        o.next_level()
        for _ in range(cfg["N"]):
            o.ir_iteration()
        errs.append(h1_error(prob, o.decode_solution(), L))
    return np.array(errs), o


# Algorithm 1's V(0,1) with one red-black Gauss-Seidel sweep (3-D: b2 one bit wider
# than the Jacobi V(2,2) configuration; at b2 = 3 the order from L = 3 to 4 is 0.949)
CFG3_RB = dict(CFG3, b2=4, nu1=0, nu2=1, smoother=1)


@pytest.mark.parametrize("name,Lmax,cfg", [("poisson2d_manufactured", 7, CFG2),
                                           ("poisson3d_manufactured", 5, CFG3),
                                           ("poisson3d_manufactured", 7, CFG3_RB)])
def test_success_criteria(name, Lmax, cfg):
    """Sec. 7.1: |u~_L - u|_H1 <= 2 |u_L - u|_H1 and order >= p - m + 1 - 0.05 for
    L >= 4, with u_L the discrete solution (here: lossless FMG, 12 IR iterations)."""
    prob = P.make_problem(name, Lmax)
    ref, _ = _h1_errors(prob, Lmax, b1=0, b2=0, N=12, nu1=2, nu2=2, omega=0.75)
    err, o = _h1_errors(prob, Lmax, **cfg)
    Ls = np.arange(2, Lmax + 1)
    assert np.all(err[Ls >= 4] <= 2 * ref[Ls >= 4])
    order = -np.log2(err[1:] / err[:-1])
    assert np.all(order[Ls[1:] >= 4] >= 0.95)
    assert o.inexact == 0


def test_nonuniform_weight_reports_inexact():
    """A non-dyadic Jacobi weight cannot be carried exactly: the checker notices."""
    prob = P.make_problem("poisson2d_manufactured", 4)
    o = oracle.Oracle.for_problem(prob, b1=4, b2=4, N=2, nu1=2, nu2=2, omega=0.8)
    o.fmg()
    assert o.inexact > 0


@pytest.mark.parametrize("dim,Lmax,bound", [(2, 7, 0.32), (3, 7, 0.5)])
def test_vcycle_convergence_factor_h_independent(dim, Lmax, bound):
    """Lossless IR with one V(2,2) cycle per iteration contracts the residual by a
    factor that levels off as h decreases (weighted Jacobi, omega = 3/4)."""
    rates = []
    for L in range(4, Lmax + 1):
        prob = P.make_problem("poisson2d_fourier" if dim == 2 else "poisson3d_fourier", L)
        o = oracle.Oracle.for_problem(prob, b1=0, b2=0, N=1, nu1=2, nu2=2, omega=0.75)
        o.start()
        for _ in range(2, L + 1):
            o.next_level()
        norms = []
        for _ in range(9):
            o.residual()
            norms.append(np.linalg.norm(o.last_t()))
            o.vcycle()
            o.correct()
        rates.append((norms[-1] / norms[3]) ** (1 / 5))
    assert max(rates) < bound
    steps = np.diff(rates)
    assert steps[-1] < 0.05 and steps[-1] < 0.7 * steps[-2] + 1e-3


def test_storage_is_linear():
    """Sec. 6.1.1: sum_l n_l (k (L-l) + b) < (2^d/(2^d-1) b + 2^d/(2^d-1)^2 k) n_L.
    Padded BFP storage (32-value blocks, one exponent byte) stays within a
    bounded factor of that and its bits per finest DoF converge as L grows."""
    for dim, b, k in [(2, 4, 2), (2, 4, 1), (3, 5, 2), (3, 3, 1)]:
        prev = None
        for L in range(3, 12 if dim == 2 else 11):
            nL = ((1 << L) - 1) ** dim
            mant = sum(((1 << l) - 1) ** dim * (k * (L - l) + b) for l in range(1, L + 1))
            c = 2 ** dim / (2 ** dim - 1)
            assert mant < (c * b + c / (2 ** dim - 1) * k) * nL
            padded = sum(oracle.nblocks(dim, l) * (32 * (k * (L - l) + b) + 8) for l in range(1, L + 1))
            per = padded / nL
            if prev is not None and L >= 8:
                assert abs(per - prev) < 0.5
            prev = per
        assert per < 1.1 * (c * b + c / (2 ** dim - 1) * k) + 8 / 32 + 1.0


def test_slab_h1_error_equals_the_whole_array_one():
    """The slab-streamed H^1 error (used on the GPU at full size) equals the
    whole-array one on the same nodal values."""
    torch = pytest.importorskip("torch")
    from cmg_problems.diagnostics import h1_error_slabs
    prob = P.make_problem("poisson3d_manufactured", 5)
    n = (1 << 5) - 1
    rng = np.random.default_rng(1)
    U = np.asarray(prob.exact_u(*np.meshgrid(*(np.arange(1, n + 1) / 32.0,) * 3, indexing="ij")[::-1]))
    U = U + 1e-3 * rng.standard_normal(U.shape)
    Ut = torch.from_numpy(U)
    a = h1_error(prob, U, 5)
    b = h1_error_slabs(prob, lambda z0, nz: Ut[z0:z0 + nz], 5, zchunk=3)
    assert abs(a - b) <= 1e-12 * a


@pytest.mark.parametrize("name,levels", [("poisson2d_manufactured", (5, 6, 7, 8)),
                                         ("poisson3d_manufactured", (4, 5, 6))])
def test_nodal_error_is_second_order(name, levels):
    """The discrete solution (lossless FMG, 12 IR iterations) converges to the
    manufactured u at the nodes with order 2 (P1 on the uniform Kuhn mesh): a
    dropped term or a wrong sign in the operator or in f breaks it."""
    errs = []
    for L in levels:
        prob = P.make_problem(name, L)
        o = oracle.Oracle.for_problem(prob, b1=0, b2=0, N=12, nu1=2, nu2=2, omega=0.75)
        o.fmg()
        U = np.asarray(o.decode_solution()).reshape(-1)
        ue = np.asarray(exact_on_grid(prob, L)).reshape(-1)
        errs.append(np.max(np.abs(U - ue)))
    orders = -np.log2(np.array(errs[1:]) / np.array(errs[:-1]))
    assert np.all(orders > 1.9), orders


@pytest.mark.parametrize("name,Lmax,cfg", [("poisson2d_manufactured", 5, CFG2),
                                           ("poisson3d_manufactured", 4, CFG3),
                                           ("poisson3d_fourier", 4, CFG3_RB)])
def test_fmg_level_step_is_p1_interpolation(name, Lmax, cfg):
    """Algorithm 3's level step in the compact representation (eq.
    compact-to-standard): a zero finest section and coarser sections widened by
    k_u = p + 1 zero bits, so the decoded solution on the new level is exactly
    the P1 interpolation of the previous level's solution."""
    prob = P.make_problem(name, Lmax)
    o = oracle.Oracle.for_problem(prob, **cfg)
    o.start()
    for L in range(2, Lmax + 1):
        if L > 2:
            for _ in range(cfg["N"]):
                o.ir_iteration()
        coarse = o.decode_solution().ravel()
        before = [o.get_section(0, l)[2].copy() for l in range(1, L)]
        widths = [o.width(0, l) for l in range(1, L)]
        o.next_level()
        assert o.level == L
        fine = o.decode_solution().ravel()
        assert np.array_equal(fine, prolongation(prob.dim, L) @ coarse)
        _, e, vals = o.get_section(0, L)
        assert not vals.any() and np.all(e == -128)
        for l in range(1, L):
            assert o.width(0, l) == widths[l - 1] + 2
            assert np.array_equal(o.get_section(0, l)[2], before[l - 1])
    assert o.inexact == 0
