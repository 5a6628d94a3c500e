"""Storage model of Secs. 6.1.1 and 6.1.4 (CMG regressive vs BFPMG progressive mantissa bits).

The oracle (oracle/storage_model.py) is pinned to what the paper fixes: the
closed-form linear bound of Sec. 6.1.1 and its constants 2, 4/3, 8/7, brute-force
enumeration of every stored value on tiny grids, and the plotted claim of
savings around an order of magnitude at ~1e15 DoF.  The library's
cmg_storage_model (host arithmetic behind the C ABI) must agree with it.
"""
import itertools
from fractions import Fraction

import pytest

from oracle import storage_model as sm

# Table 2 constants (p = 1 Poisson; p = 3 biharmonic), increments k_u = p + 1, k_r = m
POISSON_1D = dict(d=1, k_u=2, k_r=1, b1=5, b2=3)
POISSON_2D = dict(d=2, k_u=2, k_r=1, b1=4, b2=4)
BIHARM_1D = dict(d=1, k_u=4, k_r=2, b1=4, b2=4)


def test_paper_constants_of_the_linear_bound():
    # Sec. 6.1.1: 2^d / (2^d - 1) is 2 in 1-D, 4/3 in 2-D and 8/7 in 3-D
    assert sm.linear_bound_coefficient(1, 0, 1) == 2
    assert sm.linear_bound_coefficient(2, 0, 1) == Fraction(4, 3)
    assert sm.linear_bound_coefficient(3, 0, 1) == Fraction(8, 7)


@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("k,b", [(0, 1), (1, 4), (2, 4), (2, 5), (4, 12)])
def test_linear_storage_below_the_bound_and_tight(d, k, b):
    for L in range(1, 31):
        N = sm.cmg_vector_bits(d, L, k, b)
        bound = sm.linear_bound_coefficient(d, k, b) * 2 ** (d * L)
        assert N < bound, (d, L)
    # the bound is the L -> infinity limit of N / 2^(d L)
    L = 40
    ratio = Fraction(sm.cmg_vector_bits(d, L, k, b), 2 ** (d * L))
    assert abs(float(ratio / sm.linear_bound_coefficient(d, k, b)) - 1.0) < 1e-9


def _enumerate(d, L, width_of_level, levels):
    """Brute force: one entry per stored value of every listed level."""
    total = 0
    for l in levels:
        side = 2 ** l - 1
        for _ in itertools.product(range(side), repeat=d):
            total += width_of_level(l)
    return total


@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("L", [1, 2, 3, 4])
def test_brute_force_on_tiny_hierarchies(d, L):
    k_u, k_r, b1, b2 = 2, 1, 5, 3
    levels = range(1, L + 1)
    u_reg = _enumerate(d, L, lambda l: k_u * (L - l) + b1, levels)
    r_reg = _enumerate(d, L, lambda l: k_r * (L - l) + b2, levels)
    assert sm.cmg_vector_bits(d, L, k_u, b1) == u_reg
    assert sm.cmg_fmg_bits(d, L, k_u, k_r, b1, b2) == u_reg + 2 * r_reg
    u_pro = _enumerate(d, L, lambda l: k_u * (l - 1) + b1, [L])
    r_top = _enumerate(d, L, lambda l: k_r * (l - 1) + b2, [L] + ([L - 1] if L >= 2 else []))
    y_pro = _enumerate(d, L, lambda l: k_r * (l - 1) + b2, levels)
    assert sm.bfpmg_vector_bits(d, L, k_u, b1) == u_pro
    assert sm.bfpmg_fmg_bits(d, L, k_u, k_r, b1, b2) == u_pro + r_top + y_pro


def _level_for_dofs(d, dofs):
    L = 1
    while (2 ** L - 1) ** d < dofs:
        L += 1
    return L


@pytest.mark.parametrize("cfg", [POISSON_1D, POISSON_2D, BIHARM_1D])
def test_savings_about_an_order_of_magnitude_at_1e15_dofs(cfg):
    # Sec. 6.1.4 / the memory-comparison figure: ~10x where a supercomputer's
    # memory becomes prohibitive (the plot's axis ends at 15x)
    c = dict(cfg)
    d = c.pop("d")
    L = _level_for_dofs(d, 1e15)
    m = sm.model(d, L, **c)
    assert 4 <= m["vector_saving"] <= 15
    assert 4 <= m["fmg_saving"] <= 15


def test_savings_grow_with_size_and_with_m():
    prev = 0
    for L in range(3, 60):
        s = sm.model(1, L, **{k: v for k, v in POISSON_1D.items() if k != "d"})["fmg_saving"]
        assert s > prev
        prev = s
    # larger residual/correction increment m: larger FMG saving (Sec. 6.1.4)
    L = 50
    pois = sm.model(1, L, **{k: v for k, v in POISSON_1D.items() if k != "d"})["fmg_saving"]
    biha = sm.model(1, L, **{k: v for k, v in BIHARM_1D.items() if k != "d"})["fmg_saving"]
    assert biha > pois


def test_library_matches_the_oracle():
    from paper_2511_19036_gb300 import cmg
    for d in (1, 2, 3):
        for L in list(range(1, 14)) + [20, 30, 40]:
            for (k_u, k_r, b1, b2) in [(2, 1, 4, 4), (2, 1, 5, 3), (4, 2, 4, 4), (0, 0, 1, 1)]:
                got = cmg.storage_model(d, L, k_u, k_r, b1, b2)
                want = sm.model(d, L, k_u, k_r, b1, b2)
                for key, v in want.items():
                    assert got[key] == pytest.approx(float(v), rel=1e-12, abs=0), (d, L, key)


def test_library_rejects_bad_arguments():
    from paper_2511_19036_gb300 import cmg
    for args in [(0, 5, 2, 1, 4, 4), (4, 5, 2, 1, 4, 4), (2, 0, 2, 1, 4, 4), (2, 41, 2, 1, 4, 4),
                 (2, 5, -1, 1, 4, 4), (2, 5, 2, 1, 0, 4)]:
        with pytest.raises(cmg.CmgError):
            cmg.storage_model(*args)
