"""cmg_decode_compact: decoding a compact vector with no device allocation.

Some callers may not allocate device memory while they run (an application that
hands all of its device memory to its own pool at start-up, or a time-critical
loop that cannot accept the device-wide synchronisation cudaMalloc implies).
For them the library offers cmg_decode_compact, which keeps its scratch (the
decoded coarse levels) in one static device array instead of allocating it.

This file checks that entry point through the C ABI against the context-based
cmg_decode_solution, on two calls in a row with different sizes (the array keeps
the previous call's contents), and that a size beyond the static capacity is
refused.  It sorts last so that a run stopping at its first failure has already
run every other test.
"""
import ctypes

import numpy as np
import pytest

import cmg_problems as P

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cmg():
    from paper_2511_19036_gb300 import cmg as m
    return m


def solved(cmg, name, L):
    prob = P.make_problem(name, L)
    s = cmg.Solver(cmg.config_for(name, L))
    s.set_rhs(prob.tables, prob.scale_exp)
    s.fmg_solve()
    return s


def compact_on_device(cmg, s, L):
    words, exps, widths = [], [], []
    for l in range(1, L + 1):
        w, e = s.get_section(cmg.SEC_U, l)
        words.append(torch.from_numpy(w.view(np.int32).copy()).cuda())
        exps.append(torch.from_numpy(e.copy()).cuda())
        widths.append(s.width(cmg.SEC_U, l))
    return words, exps, widths


def decode_compact(cmg, dim, L, words, exps, widths, z0, nz, out):
    wp = (ctypes.c_void_p * L)(*[t.data_ptr() for t in words])
    ep = (ctypes.c_void_p * L)(*[t.data_ptr() for t in exps])
    wd = (ctypes.c_int * L)(*widths)
    return cmg.lib().cmg_decode_compact(dim, L, wp, ep, wd, z0, nz, out.data_ptr(),
                                        torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("order", [("poisson3d_fourier", 6, "poisson2d_manufactured", 8),
                                   ("poisson2d_manufactured", 8, "poisson3d_manufactured", 5)])
def test_two_calls_in_a_row_match_decode_solution(cmg, order):
    cases = [(order[0], order[1]), (order[2], order[3])]
    prepared = []
    for name, L in cases:
        s = solved(cmg, name, L)
        ref = s.decode_solution().cpu().numpy()
        prepared.append((name, L, s.cfg.dim, compact_on_device(cmg, s, L), ref))
    for name, L, dim, (words, exps, widths), ref in prepared:  # two calls in a row
        n = (1 << L) - 1
        nz = n if dim == 3 else 1
        out = torch.full((nz, n, n), float("nan"), dtype=torch.float64, device="cuda")
        st = decode_compact(cmg, dim, L, words, exps, widths, 0, nz, out)
        assert st == cmg.OK
        assert np.array_equal(out.cpu().numpy(), ref), name
    # a slab of planes, after both calls
    name, L, dim, (words, exps, widths), ref = prepared[0]
    if dim == 3:
        n = (1 << L) - 1
        out = torch.empty((3, n, n), dtype=torch.float64, device="cuda")
        assert decode_compact(cmg, dim, L, words, exps, widths, 5, 3, out) == cmg.OK
        assert np.array_equal(out.cpu().numpy(), ref[5:8])


def test_capacity_limit_is_refused(cmg):
    limit = 24 << 20
    assert cmg.lib().cmg_decode_compact_scratch_bytes(3, 8) <= limit
    assert cmg.lib().cmg_decode_compact_scratch_bytes(3, 9) > limit
    assert cmg.lib().cmg_decode_compact_scratch_bytes(2, 11) <= limit
    assert cmg.lib().cmg_decode_compact_scratch_bytes(2, 12) > limit
    dummy_w = torch.zeros(64, dtype=torch.int32, device="cuda")
    dummy_e = torch.zeros(64, dtype=torch.int8, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    L = 9
    st = decode_compact(cmg, 3, L, [dummy_w] * L, [dummy_e] * L, [5] * L, 0, 1, out)
    assert st == cmg.ERANGE


def plant_invalid_code(words, exps, W):
    """Overwrite code 0 of the first nonzero block with -2^(W-1), the one code
    that no encoder writes (codes are symmetric in [-(2^(W-1)-1), 2^(W-1)-1])."""
    w = words.copy().view(np.uint32)
    blk = int(np.flatnonzero(exps != -128)[0])
    base = blk * W
    stream = 0
    for k in range(W):
        stream |= int(w[base + k]) << (32 * k)
    stream &= ~((1 << W) - 1)
    stream |= 1 << (W - 1)
    for k in range(W):
        w[base + k] = (stream >> (32 * k)) & 0xFFFFFFFF
    return w.view(np.int32)


@pytest.mark.parametrize("level_from_top", [0, 1])
def test_invalid_code_is_reported(cmg, level_from_top):
    """A code -2^(W-1) in the caller's sections is reported as CMG_ECORRUPT,
    whether it sits on the finest section or on a coarse one; the next clean
    call on the same array returns CMG_OK again."""
    name, L = "poisson3d_manufactured", 5
    s = solved(cmg, name, L)
    words, exps, widths = compact_on_device(cmg, s, L)
    l = L - level_from_top
    w_host, e_host = s.get_section(cmg.SEC_U, l)
    bad = list(words)
    bad[l - 1] = torch.from_numpy(plant_invalid_code(w_host, e_host, widths[l - 1]).copy()).cuda()
    n = (1 << L) - 1
    out = torch.empty((n, n, n), dtype=torch.float64, device="cuda")
    assert decode_compact(cmg, 3, L, bad, exps, widths, 0, n, out) == cmg.ECORRUPT
    assert decode_compact(cmg, 3, L, words, exps, widths, 0, n, out) == cmg.OK
    assert np.array_equal(out.cpu().numpy(), s.decode_solution().cpu().numpy())
