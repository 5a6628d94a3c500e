"""Section reads into page-locked host memory (GPU).

cmg_get_section writes page-locked destinations with a copy kernel through the
GPU's mapping of the host buffer and other destinations with cudaMemcpy.  Both
must deliver the same bytes: 16-byte words plus a ragged tail (exponent arrays
of any length), aligned and unaligned page-locked buffers, and pageable
arrays.
"""
import numpy as np
import pytest

import cmg_problems as P

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_pinned_and_pageable_section_reads_agree():
    from paper_2511_19036_gb300 import cmg
    name, L = "poisson3d_manufactured", 6
    prob = P.make_problem(name, L)
    s = cmg.Solver(cmg.config_for(name, L, smoother=1), stream=torch.cuda.Stream())
    s.set_rhs(prob.tables, prob.scale_exp)
    s.fmg_solve()
    lib = cmg.lib()
    tails = set()
    for which, levels in ((cmg.SEC_U, range(1, L + 1)), (cmg.SEC_R, [L])):
        for level in levels:
            ref_w, ref_e = s.get_section(which, level)  # pageable: cudaMemcpy
            nw, ne = ref_w.nbytes, ref_e.nbytes
            tails.add(ne % 16)
            for off in (0, 4, 1):  # aligned (kernel copy), then unaligned (cudaMemcpy)
                bw = torch.full((nw + 16,), 0xAB, dtype=torch.uint8).pin_memory()
                be = torch.full((ne + 16,), 0xAB, dtype=torch.uint8).pin_memory()
                wp = bw.data_ptr() + (off if off % 4 == 0 else 4)  # the word array stays 4-byte aligned
                st = lib.cmg_get_section(s._h, which, level, wp, be.data_ptr() + off)
                assert st == cmg.OK, cmg.lib().cmg_last_error(s._h)
                w = bw.numpy()
                e = be.numpy()
                woff = off if off % 4 == 0 else 4
                assert np.array_equal(w[woff:woff + nw].view(np.uint32), ref_w), (which, level, off)
                assert np.array_equal(e[off:off + ne].view(np.int8), ref_e), (which, level, off)
                # nothing written outside the destination
                assert (w[:woff] == 0xAB).all() and (w[woff + nw:] == 0xAB).all()
                assert (e[:off] == 0xAB).all() and (e[off + ne:] == 0xAB).all()
    assert len(tails) > 1  # exponent arrays with different ragged tails
