"""Compact FMG on a slab partition of ranks (test infrastructure).

Runs Algorithm 3 with the red-black V(0,1) cycle of Algorithm 1 and the
restriction chain of Algorithm 2 (the bench's default cycle) on one rank of a
SlabPlan, exchanging planes through the product's Exchanger.  Every array is a
full level array, but a rank computes and keeps only the planes it owns: after
every step the other planes are cleared, so a step that read a plane the plan
did not deliver would change the result.  The arithmetic is plain float64 on
dyadic values (exact here, as in the oracle), the operators P_l and R_l are the
oracle's dense ones applied to the masked arrays, and the BFP rounding of rows
is written out from the format's definition (Sec. 4, Sec. 6.1.3).

The gathered sections must equal the single-rank oracle bit for bit.
"""
from __future__ import annotations

import numpy as np

import oracle
from fem_dense import load_vector_exact
from paper_2511_19036_gb300.partition import Exchanger, SlabPlan, planes_of


def shape_of(dim, l):
    n = planes_of(l)
    return (n, n, n) if dim == 3 else (n, n)


def bfp_rows(x, W):
    """Rows (last axis) rounded into 32-value BFP blocks of width W."""
    n = x.shape[-1]
    nbx = (n + 31) // 32
    pad = np.zeros(x.shape[:-1] + (32 * nbx,))
    pad[..., :n] = x
    b = pad.reshape(x.shape[:-1] + (nbx, 32))
    M = np.max(np.abs(b), axis=-1)
    _, E = np.frexp(M)  # 2^(E-1) <= M < 2^E
    q = np.rint(np.ldexp(b, (W - 1 - E)[..., None]))
    bump = np.any(np.abs(q) >= 2.0 ** (W - 1), axis=-1)
    E = E + bump
    q = np.rint(np.ldexp(b, (W - 1 - E)[..., None]))
    v = np.ldexp(q, (E - W + 1)[..., None])
    v[M == 0] = 0.0
    return v.reshape(pad.shape)[..., :n]


def apply_A(x, dim, l):
    """A_l x = h^(d-2) (2d x - sum of the 2d axis neighbours), zero outside."""
    p = np.pad(x, 1)
    c = (slice(1, -1),) * dim
    acc = (2 * dim) * p[c]
    for ax in range(dim):
        for sh in (-1, 1):
            sl = list(c)
            sl[ax] = slice(1 + sh, p.shape[ax] - 1 + sh)
            acc = acc - p[tuple(sl)]
    return acc * 2.0 ** (-(dim - 2) * l)


class SlabFMG:
    def __init__(self, prob, plan: SlabPlan, ex: Exchanger, b1, b2, N, omega):
        self.prob, self.plan, self.ex = prob, plan, ex
        self.dim, self.Lmax = prob.dim, prob.Lmax
        self.b1, self.b2, self.N, self.omega = b1, b2, N, omega
        self.rank = ex.rank
        d = self.dim
        self.f = {l: load_vector_exact(prob.tables, prob.scale_exp, d, self.Lmax, l).reshape(shape_of(d, l))
                  for l in range(1, self.Lmax + 1)}
        z = {l: np.zeros(shape_of(d, l)) for l in range(1, self.Lmax + 1)}
        self.u = {l: v.copy() for l, v in z.items()}
        self.r = {l: v.copy() for l, v in z.items()}
        self.y = {l: v.copy() for l, v in z.items()}
        self.w = {l: v.copy() for l, v in z.items()}
        self.L = 1

    # ------------------------------------------------------------ helpers
    def own(self, l):
        return self.plan.owned(l, self.rank)

    def keep_own(self, x, l):
        """x with every plane this rank does not own cleared."""
        out = np.zeros_like(x)
        o = self.own(l)
        out[o.start:o.stop] = x[o.start:o.stop]
        return out

    def Wu(self, l):
        return 2 * (self.L - l) + self.b1

    def Wr(self, l):
        return (self.L - l) + self.b2

    def prolong(self, xc, l):
        return oracle.prolong(self.dim, l, xc).reshape(shape_of(self.dim, l))

    def restrict(self, xf, l):
        return oracle.restrict(self.dim, l, xf).reshape(shape_of(self.dim, l - 1))

    def colour(self, l, c):
        n = planes_of(l)
        idx = np.indices(shape_of(self.dim, l)).sum(axis=0) + self.dim  # 1-based sum
        return (idx & 1) == c

    # ------------------------------------------------------------ Algorithm 3
    def start(self):
        A1 = 2.0 * self.dim * 2.0 ** (2 - self.dim)
        self.L = 1
        self.u[1] = self.keep_own(bfp_rows(self.f[1] / A1, self.Wu(1)), 1)

    def next_level(self):
        self.L += 1  # widening appends zero bits: values unchanged; u~_L = 0

    def residual(self):
        L, d, ex = self.L, self.dim, self.ex
        uh = self.u[1].copy()
        for l in range(2, L + 1):
            ex.prolong_source(uh, l)
            uh = self.keep_own(self.u[l] + self.prolong(uh, l), l)
        ex.halo(uh, L)
        t = self.keep_own(self.f[L] - apply_A(uh, d, L), L)
        self.r[L] = self.keep_own(bfp_rows(t, self.Wr(L)), L)
        Wt = 2 * L + self.b1  # t^ of Table 1: (p+1) L + b1 bits
        th = self.keep_own(bfp_rows(t, Wt), L)
        for l in range(L - 1, 0, -1):
            acc = self.restrict(th, l + 1)
            ex.reduce_to_owners(acc, l + 1)
            th = self.keep_own(bfp_rows(self.keep_own(acc, l), Wt), l)
            self.r[l] = self.keep_own(bfp_rows(th, self.Wr(l)), l)

    def half_sweep(self, l, z, colour):
        d = self.dim
        cl = self.omega / (2 * d) * 2.0 ** ((d - 2) * l)
        y = self.y[l]
        res = (self.r[l] - apply_A(z, d, l)) - apply_A(y, d, l)
        yn = np.where(self.colour(l, colour), y + cl * res, y)
        self.y[l] = self.keep_own(bfp_rows(self.keep_own(yn, l), self.Wr(l)), l)

    def vcycle(self):
        L, ex = self.L, self.ex
        for l in range(1, L + 1):
            self.y[l] = np.zeros_like(self.y[l])
        A1 = 2.0 * self.dim * 2.0 ** (2 - self.dim)
        self.y[1] = self.keep_own(bfp_rows(self.r[1] / A1, self.Wr(1)), 1)
        self.w[1] = self.y[1].copy()
        for l in range(2, L + 1):
            wc = self.w[l - 1].copy()
            ex.prolong_source(wc, l)
            z = self.prolong(wc, l)  # valid on own planes and the stencil halo
            z = z * self.mask_own_and_halo(l)
            ex.halo(self.y[l], l)
            self.half_sweep(l, z, 0)  # red
            ex.halo(self.y[l], l)
            self.half_sweep(l, z, 1)  # black
            self.w[l] = self.keep_own(self.y[l] + z, l)

    def mask_own_and_halo(self, l):
        m = np.zeros(shape_of(self.dim, l))
        o = self.own(l)
        m[o.start:o.stop] = 1.0
        for zp in self.plan.stencil_halo(l, self.rank):
            m[zp] = 1.0
        return m

    def correct(self):
        for l in range(1, self.L + 1):
            self.u[l] = self.keep_own(bfp_rows(self.u[l] + self.y[l], self.Wu(l)), l)

    def fmg(self):
        self.start()
        for _ in range(2, self.Lmax + 1):
            self.next_level()
            for _ in range(self.N):
                self.residual()
                self.vcycle()
                self.correct()

    def gather(self, l):
        """u~_l on rank 0 (every rank must call it)."""
        x = self.u[l].copy()
        n = planes_of(l)
        needs = [list(range(n))] + [[] for _ in range(1, self.plan.world)]
        self.ex.fetch(x, l, needs)
        return x
