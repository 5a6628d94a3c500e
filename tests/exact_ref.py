"""Exact-rational reference pieces for the oracle pins (test infrastructure).

Sparse matrices of Fractions snapped from the first-principles FEM matrices of
fem_dense.py, and a BFP rounder and bit packer written from the format's
definition (Sec. 4: round to nearest, ties to even; Sec. 6.1.3: blocks sharing
one exponent): a block of values x gets e, the smallest integer with
max|x| < 2^e, and codes q = RNE(x 2^(W-1-e)); a code reaching 2^(W-1) raises e
by one; an all-zero block stores e = -128; code i occupies bits [iW, iW+W) of
the block's little-endian stream of W 32-bit words.  Nothing here is shared
with the oracle or the CUDA path.
"""
from fractions import Fraction

import numpy as np


def snap(M, denom):
    """Dense float matrix -> sparse rows of exact Fractions on the grid 1/denom
    (the assembled entries are dyadic up to float round-off in cancelled terms)."""
    rows = []
    for i in range(M.shape[0]):
        nz = np.flatnonzero(np.abs(M[i]) > 1e-9)
        row = []
        for j in nz:
            q = int(round(M[i, j] * denom))
            assert abs(M[i, j] * denom - q) < 1e-6
            if q:
                row.append((int(j), Fraction(q, denom)))
        rows.append(row)
    return rows


def matvec(rows, x):
    return [sum((a * x[j] for j, a in row), Fraction(0)) for row in rows]


def transpose(rows, ncols):
    out = [[] for _ in range(ncols)]
    for i, row in enumerate(rows):
        for j, a in row:
            out[j].append((i, a))
    return out


def round_block(blk, W):
    """(e, codes) of one block: e the smallest integer with max|x| < 2^e,
    codes RNE(x 2^(W-1-e)); a code reaching 2^(W-1) raises e by one."""
    M = max(abs(v) for v in blk)
    if M == 0:
        return -128, [0] * len(blk)
    e = 0
    while Fraction(2) ** e <= M:
        e += 1
    while Fraction(2) ** (e - 1) > M:
        e -= 1
    for _ in range(2):
        codes = []
        for v in blk:
            x = v * Fraction(2) ** (W - 1 - e)
            fl = x.numerator // x.denominator
            rem = x - fl
            codes.append(fl + (1 if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2) else 0))
        if max(abs(q) for q in codes) >= 2 ** (W - 1):
            e += 1
            continue
        return e, codes
    raise AssertionError("second bump")


def bfp(vals, n, W):
    """Round a dense level array (x fastest, rows of n) into 32-value blocks per row.
    Returns (rounded values, exponents per block, codes per block, padded to 32)."""
    out, exps, codes = [], [], []
    for r0 in range(0, len(vals), n):
        row = vals[r0:r0 + n]
        for b0 in range(0, n, 32):
            blk = row[b0:b0 + 32]
            e, q = round_block(blk, W)
            exps.append(e)
            codes.append(q + [0] * (32 - len(q)))
            out += [Fraction(c) * Fraction(2) ** (e - W + 1) if e != -128 else Fraction(0) for c in q]
    return out, exps, codes


def per_value(vals, W):
    """Each value rounded alone (a one-value block): floating point with W - 1 bits
    of significand and the sign, the paper's FP reading of a temporary."""
    out = []
    for v in vals:
        e, q = round_block([v], W)
        out.append(Fraction(q[0]) * Fraction(2) ** (e - W + 1) if e != -128 else Fraction(0))
    return out


def pack(codes, W):
    """Code i at bits [iW, iW+W) of the block's little-endian stream of W words."""
    words = []
    for blk in codes:
        s = 0
        for i, q in enumerate(blk):
            s |= (q & ((1 << W) - 1)) << (i * W)
        words += [(s >> (32 * k)) & 0xFFFFFFFF for k in range(W)]
    return np.array(words, dtype=np.uint32)
