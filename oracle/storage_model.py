"""Storage model of compact multigrid -- TEST INFRASTRUCTURE ONLY.

Plain exact-integer restatement of Secs. 6.1.1 and 6.1.4 of "Multigrid with Linear Storage
Complexity" (mantissas of regressive-precision vectors; comparison with
progressive-precision FMG in BFP arithmetic, "BFPMG").  Only the tests may
import it; it shares no code with the library.

Levels are numbered as in the solver: level l = 1..L holds (2^l - 1)^d interior
values and corresponds to the paper's level l - 1, so the paper's
regressive(+k, b) precision gives k (L - l) + b bits on level l and its
progressive(+k, b) precision k (l - 1) + b bits (eq. regressive; the
definition of progressive precision next to it).

Readings (the paper plots the comparison without listing its formulas):
  * CMG stores u~ (regressive(+p+1, b1)) and r, y~ (regressive(+m, b2)) on
    every level (Table 1);
  * BFPMG stores, as the paper assumes for a memory-efficient implementation,
    u_L (progressive(+p+1, b1)), r_L and r_(L-1) (progressive(+m, b2)) and the
    correction y on every level (progressive(+m, b2)), with the same increments
    and constants;
  * mantissa bits only, sign included (Table 2 caption); exponents and the
    sublinear temporaries are left out, as the paper does for the plot.

Pins: tests/test_storage_model.py (the closed-form bound of Sec. 6.1.1 and its
constants 2, 4/3, 8/7, brute-force enumeration on tiny grids, the paper's
"around an order of magnitude" claim).
"""
from __future__ import annotations

from fractions import Fraction
from typing import Dict, List, Tuple


def level_sizes(d: int, L: int) -> List[Tuple[int, int]]:
    """(level, interior values) for levels 1..L."""
    return [(l, (2 ** l - 1) ** d) for l in range(1, L + 1)]


def regressive_bits(k: int, b: int, L: int, l: int) -> int:
    """Bits per value of a regressive(+k, b) vector on level l of L (eq. regressive)."""
    return k * (L - l) + b


def progressive_bits(k: int, b: int, l: int) -> int:
    """Bits per value of a progressive(+k, b) vector on level l (coarsest level 1)."""
    return k * (l - 1) + b


def cmg_vector_bits(d: int, L: int, k_u: int, b1: int) -> int:
    """Sec. 6.1.1: N = sum over levels of n_l (k (L - l) + b) for the compact u~."""
    return sum(n * regressive_bits(k_u, b1, L, l) for l, n in level_sizes(d, L))


def cmg_fmg_bits(d: int, L: int, k_u: int, k_r: int, b1: int, b2: int) -> int:
    """u~, r and y~ of CMG on all levels (Table 1 precisions)."""
    r = sum(n * regressive_bits(k_r, b2, L, l) for l, n in level_sizes(d, L))
    return cmg_vector_bits(d, L, k_u, b1) + 2 * r


def bfpmg_vector_bits(d: int, L: int, k_u: int, b1: int) -> int:
    """The standard-representation solution u_L in progressive(+p+1, b1)."""
    n_L = (2 ** L - 1) ** d
    return n_L * progressive_bits(k_u, b1, L)


def bfpmg_fmg_bits(d: int, L: int, k_u: int, k_r: int, b1: int, b2: int) -> int:
    """u_L, r_L, r_(L-1) and y_1..L of BFPMG in progressive precision."""
    sizes = dict(level_sizes(d, L))
    total = bfpmg_vector_bits(d, L, k_u, b1)
    total += sizes[L] * progressive_bits(k_r, b2, L)
    if L >= 2:
        total += sizes[L - 1] * progressive_bits(k_r, b2, L - 1)
    total += sum(n * progressive_bits(k_r, b2, l) for l, n in sizes.items())
    return total


def model(d: int, L: int, k_u: int, k_r: int, b1: int, b2: int) -> Dict[str, Fraction]:
    """All quantities of the comparison, exact."""
    cv = cmg_vector_bits(d, L, k_u, b1)
    cf = cmg_fmg_bits(d, L, k_u, k_r, b1, b2)
    bv = bfpmg_vector_bits(d, L, k_u, b1)
    bf = bfpmg_fmg_bits(d, L, k_u, k_r, b1, b2)
    return {"dofs": Fraction((2 ** L - 1) ** d), "cmg_vector_bits": Fraction(cv),
            "cmg_fmg_bits": Fraction(cf), "bfpmg_vector_bits": Fraction(bv),
            "bfpmg_fmg_bits": Fraction(bf), "vector_saving": Fraction(bv, cv),
            "fmg_saving": Fraction(bf, cf)}


def linear_bound_coefficient(d: int, k: int, b: int) -> Fraction:
    """Sec. 6.1.1: N < (2^d/(2^d-1) b + 2^d/(2^d-1)^2 k) n_L, with n_L ~ 2^(d L)."""
    q = Fraction(2 ** d, 2 ** d - 1)
    return q * b + Fraction(2 ** d, (2 ** d - 1) ** 2) * k
