"""Pins of the oracle's adjoint gradient for the diffusion problem.

J = 1/2 |u - u_obs|^2 with A(k) u = h^d g.  The adjoint state solves
A lam = u - u_obs (A is symmetric), dJ/dg = h^d lam and
dJ/dk_i = -lam^T (dA/dk_i) u, which the oracle evaluates node by node
(cmgo_gradient_k).  Pinned by: the node formula equals -lam^T (dA/dk_i) u with
dA/dk_i taken from the assembled matrix (A is affine in k, so a dyadic step is
exact); a dense assembly in FP64 written from the operator's definition equals
the oracle's operator; and central finite differences of J through dense
solves match the adjoint gradients for both k and g.
"""
import numpy as np
import pytest

import cmg_problems as P
import oracle


def make(dim, L, k, **kw):
    prob = P.make_problem("diffusion%dd_grf" % dim, L)
    base = dict(b1=5, b2=4, N=3, nu1=2, nu2=2, omega=0.75)
    base.update(kw)
    return oracle.Oracle(dim, L, prob.tables, prob.scale_exp, arith=1, coef=1, kfield=k, **base)


def dense_oracle(o, dim, L):
    npts = ((1 << L) - 1) ** dim
    M = np.zeros((npts, npts))
    for i in range(npts):
        e = np.zeros(npts)
        e[i] = 1.0
        M[:, i] = o.apply_A_diffusion(L, e)
    return M


def dense_assembly(k, dim, L):
    """A from its definition: h^(d-2) sum over the neighbour faces of (k_p + k_q)/2 (u_p - u_q)."""
    N = (1 << L) + 1
    n = N - 2
    kk = np.asarray(k, dtype=np.float64).reshape((N,) * dim)
    idx = -np.ones((N,) * dim, dtype=np.int64)
    inner = tuple(slice(1, -1) for _ in range(dim))
    idx[inner] = np.arange(n ** dim).reshape((n,) * dim)
    A = np.zeros((n ** dim, n ** dim))
    h = 2.0 ** -L
    for p in np.ndindex(*((n,) * dim)):
        P1 = tuple(c + 1 for c in p)
        ip = idx[P1]
        for a in range(dim):
            for s in (-1, 1):
                Q = list(P1)
                Q[a] += s
                Q = tuple(Q)
                kf = 0.5 * (kk[P1] + kk[Q])
                A[ip, ip] += kf * h ** (dim - 2)
                if idx[Q] >= 0:
                    A[ip, idx[Q]] -= kf * h ** (dim - 2)
    return A


@pytest.mark.parametrize("dim,L", [(2, 3), (3, 2)])
def test_node_formula_equals_the_matrix_derivative(dim, L):
    N = (1 << L) + 1
    rng = np.random.default_rng(4)
    k = rng.choice(np.array([0.5, 1.0, 1.5, 2.0, 3.0], dtype=np.float32), size=N ** dim)
    npts = ((1 << L) - 1) ** dim
    u = rng.integers(-8, 9, size=npts).astype(np.float64)
    lam = rng.integers(-8, 9, size=npts).astype(np.float64)
    o = make(dim, L, k)
    M0 = dense_oracle(o, dim, L)
    G = o.gradient_k(u, lam)
    for i in range(N ** dim):
        k2 = k.copy()
        k2[i] += np.float32(0.25)
        M1 = dense_oracle(make(dim, L, k2), dim, L)
        dA = (M1 - M0) / 0.25
        assert G[i] == -(lam @ dA @ u), i


@pytest.mark.parametrize("dim,L", [(2, 4), (3, 3)])
def test_dense_assembly_matches_the_operator(dim, L):
    prob = P.make_problem("diffusion%dd_grf" % dim, L)
    k = prob.kfield().ravel()
    o = make(dim, L, k)
    A = dense_assembly(k, dim, L)
    M = dense_oracle(o, dim, L)
    assert np.allclose(A, M, rtol=1e-14, atol=0)


@pytest.mark.parametrize("dim,L", [(2, 4), (3, 3)])
def test_adjoint_gradients_match_central_differences(dim, L):
    prob = P.make_problem("diffusion%dd_grf" % dim, L)
    k = prob.kfield().ravel()
    N = (1 << L) + 1
    npts = ((1 << L) - 1) ** dim
    rng = np.random.default_rng(21)
    g = rng.standard_normal(npts)
    u_obs = 0.01 * rng.standard_normal(npts)
    h = 2.0 ** -L

    def J(kv, gv):
        u = np.linalg.solve(dense_assembly(kv, dim, L), h ** dim * gv)
        return 0.5 * np.sum((u - u_obs) ** 2)

    A = dense_assembly(k, dim, L)
    u = np.linalg.solve(A, h ** dim * g)
    lam = np.linalg.solve(A, u - u_obs)
    o = make(dim, L, k)
    Gk = o.gradient_k(u, lam)
    Gg = h ** dim * lam
    eps = 1e-6
    for trial in range(3):
        dk = rng.standard_normal(N ** dim)
        fd = (J(k.astype(np.float64) + eps * dk, g) - J(k.astype(np.float64) - eps * dk, g)) / (2 * eps)
        assert abs(fd - Gk @ dk) <= 1e-6 * abs(fd) + 1e-14
        dg = rng.standard_normal(npts)
        fd = (J(k, g + eps * dg) - J(k, g - eps * dg)) / (2 * eps)
        assert abs(fd - Gg @ dg) <= 1e-6 * abs(fd) + 1e-14
