"""Pins for the oracle's BFP codec (Sec. 4 rounding rules, Sec. 6.1.3 BFP).

Expected codes and words below are worked out by hand from the format's
definition (value = q * 2^(e-W+1), e the smallest integer with max|x| < 2^e,
round to nearest with ties to even, bump the exponent when a code reaches
2^(W-1), code i at bits [iW, iW+W) of the block's little-endian word stream).
"""
import numpy as np
import pytest

import oracle
from cmg_problems import random_block_values


def codes_of(words, W, nvals=32):
    bits = 0
    for k, w in enumerate(words):
        bits |= int(w) << (32 * k)
    out = []
    for i in range(nvals):
        c = (bits >> (i * W)) & ((1 << W) - 1)
        if c >> (W - 1):
            c -= 1 << W
        out.append(c)
    return out


def test_hand_worked_block_w4():
    x = np.zeros(32)
    x[:3] = [0.75, -0.5, 0.125]
    words, e, st = oracle.encode(x, 4)
    assert st == 0
    # max 0.75 < 2^0 -> e = 0, step 2^-3: codes 6, -4, 1
    assert e.tolist() == [0]
    # 6 = 0b0110 at bits 0..3, -4 = 0b1100 at bits 4..7, 1 at bits 8..11
    assert int(words[0]) == 0x1C6
    assert words[1:].tolist() == [0, 0, 0]
    y, st = oracle.decode(words, e, 32, 4)
    assert st == 0 and np.array_equal(y, x)


def test_ties_to_even_w3():
    x = np.zeros(32)
    x[:5] = [1.5, 0.25, 0.75, -0.25, -0.75]
    words, e, st = oracle.encode(x, 3)
    # max 1.5 -> e = 1, step 2^-1: 3, tie 0.5->0, tie 1.5->2, tie -0.5->0, tie -1.5->-2
    assert e.tolist() == [1]
    assert codes_of(words, 3)[:5] == [3, 0, 2, 0, -2]
    y, _ = oracle.decode(words, e, 32, 3)
    assert y[:5].tolist() == [1.5, 0.0, 1.0, 0.0, -1.0]


def test_exponent_bump_on_round_up():
    x = np.zeros(32)
    x[:2] = [1.9, 0.3]
    words, e, st = oracle.encode(x, 3)
    # e = 1 gives 1.9/0.5 = 3.8 -> 4 = 2^(W-1): bump to e = 2, step 1: 1.9->2, 0.3->0
    assert e.tolist() == [2]
    assert codes_of(words, 3)[:2] == [2, 0]


def test_code_straddles_word_boundary_w5():
    x = np.zeros(32)
    x[0] = 15.0  # e = 4, step 2^0 -> code 15
    x[6] = -11.0  # code -11 = 0b10101 at bits 30..34
    words, e, _ = oracle.encode(x, 5)
    assert e.tolist() == [4]
    assert int(words[0]) == (15 | ((0b10101 & 0b11) << 30))
    assert int(words[1]) == (0b10101 >> 2)


def test_zero_block_and_padding():
    x = np.zeros(37)
    x[33] = -3.0
    words, e, _ = oracle.encode(x, 6)
    assert e.tolist() == [-128, 2]
    assert not words[:6].any()
    y, _ = oracle.decode(words, e, 37, 6)
    assert np.array_equal(y, x)
    # padding lanes 37..63 carry code 0
    assert codes_of(words[6:12], 6)[5:] == [0] * 27


@pytest.mark.parametrize("W", [2, 3, 4, 5, 7, 8, 13, 16, 24, 31, 32])
def test_round_trip_error_bound(W):
    x = random_block_values(32 * 40 + 7, seed=W)
    words, e, st = oracle.encode(x, W)
    assert st == 0
    y, st = oracle.decode(words, e, x.size, W)
    assert st == 0
    for b in range(e.size):
        blk = slice(32 * b, min(x.size, 32 * b + 32))
        if e[b] == -128:
            assert not x[blk].any() and not y[blk].any()
            continue
        M = np.max(np.abs(x[blk]))
        assert 2.0 ** (e[b] - 2) <= M < 2.0 ** e[b]  # at most one bump above the natural exponent
        assert np.max(np.abs(y[blk] - x[blk])) <= 2.0 ** (e[b] - W)  # half a unit of the block
        codes = codes_of(words[b * W:(b + 1) * W], W)
        assert max(abs(c) for c in codes) <= 2 ** (W - 1) - 1


@pytest.mark.parametrize("W", [2, 3, 4])
def test_exhaustive_small_width_idempotent(W):
    """Every representable block value re-encodes to itself (all codes, both signs)."""
    lim = 2 ** (W - 1) - 1
    codes = np.arange(-lim, lim + 1)
    for top in (lim, -lim):  # force the exponent with a full-scale entry
        for start in range(0, codes.size, 31):
            q = np.zeros(32)
            q[0] = top
            chunk = codes[start:start + 31]
            q[1:1 + chunk.size] = chunk
            x = np.ldexp(q, -3 - W + 1)  # exponent -3: full scale is below 2^-3
            words, e, _ = oracle.encode(x, W)
            y, _ = oracle.decode(words, e, 32, W)
            assert np.array_equal(x, y)
            if lim >= 2:
                assert e[0] == -3


def test_widening_appends_zero_bits():
    x = random_block_values(32 * 8, seed=5)
    w5, e5, _ = oracle.encode(x, 5)
    y5, _ = oracle.decode(w5, e5, x.size, 5)
    w7, e7, _ = oracle.encode(y5, 7)  # already on the 5-bit grid: exact at 7 bits
    assert np.array_equal(e5, e7)
    for b in range(e5.size):
        c5 = codes_of(w5[5 * b:5 * b + 5], 5)
        c7 = codes_of(w7[7 * b:7 * b + 7], 7)
        assert c7 == [4 * c for c in c5]


def test_errors():
    x = np.zeros(32)
    x[0] = 2.0 ** 200
    assert oracle.encode(x, 8)[2] == oracle.ERANGE
    assert oracle.encode(np.zeros(32), 1)[2] == oracle.EINVAL
    assert oracle.encode(np.zeros(32), 33)[2] == oracle.EINVAL
    words = np.zeros(4, dtype=np.uint32)
    words[0] = 0b1000  # code -8 = -2^(W-1) for W = 4 is not a valid code
    _, st = oracle.decode(words, np.array([0], dtype=np.int8), 32, 4)
    assert st == oracle.ECORRUPT
