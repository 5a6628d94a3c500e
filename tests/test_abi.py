"""The C-ABI library loads and exports every entry point that include/cmg.h
declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions(header):
    src = open(header).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(cmg_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2511_19036_gb300 import _build
    try:
        return _build.build()
    except (RuntimeError, FileNotFoundError) as e:  # nvcc missing on this host
        pytest.skip("nvcc unavailable: %s" % e)


def test_header_declares_the_boundary():
    names = declared_functions(os.path.join(ROOT, "include", "cmg.h"))
    for need in ("cmg_encode", "cmg_decode", "cmg_create", "cmg_fmg_solve", "cmg_residual",
                 "cmg_down", "cmg_up", "cmg_prolongate", "cmg_vcycle", "cmg_decode_solution"):
        assert need in names
    assert len(names) >= 25


def test_library_exports_every_declared_symbol(libpath):
    names = declared_functions(os.path.join(ROOT, "include", "cmg.h"))
    lib = ctypes.CDLL(libpath)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(cmg_\w+)", out))
    assert set(names) <= exported


def test_binding_covers_every_symbol(libpath):
    from paper_2511_19036_gb300 import cmg
    names = declared_functions(os.path.join(ROOT, "include", "cmg.h"))
    assert set(names) <= set(cmg.exported_symbols())


def test_host_side_parameter_validation(libpath):
    from paper_2511_19036_gb300 import cmg
    good = cmg.config_for("poisson3d_fourier", 11)
    assert cmg.params_check(good) == cmg.OK
    assert cmg.params_check(cmg.config_for("poisson2d_manufactured", 8)) == cmg.OK
    for k, v in [("dim", 1), ("L_max", 0), ("b2", 1), ("nu2", 0), ("omega_num", 0), ("omega_num", 2)]:
        bad = cmg.config_for("poisson3d_fourier", 8)
        setattr(bad, k, v)
        assert cmg.params_check(bad) == cmg.EINVAL, k
    # red-black Gauss-Seidel: only as V(0, nu2) post-smoothing of the Poisson problem
    rb = cmg.config_for("poisson3d_fourier", 8)
    rb.smoother, rb.nu1, rb.nu2 = 1, 0, 1
    assert cmg.params_check(rb) == cmg.OK
    for k, v in [("nu1", 1), ("smoother", 2), ("smoother", -1)]:
        bad = cmg.config_for("poisson3d_fourier", 8)
        bad.smoother, bad.nu1, bad.nu2 = 1, 0, 1
        setattr(bad, k, v)
        assert cmg.params_check(bad) == cmg.EINVAL, k
    diff = cmg.config_for("diffusion3d_grf", 8)
    diff.smoother = 1
    assert cmg.params_check(diff) == cmg.EINVAL
    wide = cmg.config_for("poisson3d_fourier", 14)
    wide.b1 = 12
    assert cmg.params_check(wide) == cmg.ERANGE
    assert cmg.lib().cmg_section_blocks(3, 8) == 255 * 255 * 8
    assert cmg.lib().cmg_section_blocks(2, 8) == 255 * 8
    assert cmg.lib().cmg_section_blocks(4, 8) == -1


def test_host_side_parameter_validation_edges(libpath):
    from paper_2511_19036_gb300 import cmg

    def check(name, L, **kw):
        c = cmg.config_for(name, L, smoother=kw.pop("smoother", 0))
        for k, v in kw.items():
            setattr(c, k, v)
        return cmg.params_check(c)

    # binary32 cycle: every r~ / y~ code must be exact in binary32
    assert check("poisson3d_manufactured", 11, arith=1) == cmg.OK
    assert check("poisson3d_manufactured", 11, arith=1, b2=14) == cmg.ERANGE
    # diffusion runs only with a floating-point cycle (binary32 or binary64), with pre-smoothing
    assert check("diffusion3d_grf", 8) == cmg.OK
    assert check("diffusion3d_grf", 8, arith=2) == cmg.OK
    assert check("poisson3d_manufactured", 11, arith=2, b2=14) == cmg.OK
    assert check("diffusion3d_grf", 8, arith=0) == cmg.EINVAL
    assert check("diffusion3d_grf", 8, nu1=0) == cmg.EINVAL
    for k, v in [("arith", 3), ("coef", 2), ("omega_log2den", 31), ("omega_log2den", -1), ("N_ir", 0),
                 ("nu1", 65), ("b1", 1), ("k_u", -1)]:
        assert check("poisson3d_fourier", 8, **{k: v}) == cmg.EINVAL, k
    # without pre-smoothing t^ carries (p+1) L + b1 bits, at most 32
    assert check("poisson3d_manufactured", 11, smoother=1) == cmg.OK
    assert check("poisson3d_manufactured", 11, smoother=1, b1=10) == cmg.OK  # 32 bits
    assert check("poisson3d_manufactured", 11, smoother=1, b1=11) == cmg.ERANGE  # 33 bits
    assert check("poisson3d_manufactured", 11, b1=11) == cmg.OK  # Jacobi V(2,2): no chain
    # 3-D: omega / 6 must be dyadic
    assert check("poisson3d_fourier", 8, omega_num=1, omega_log2den=0) == cmg.EINVAL
    # block and plane indices of the finest level fit 31 bits: 3-D L = 12 does, L = 13 not
    assert check("poisson3d_fourier", 12, b1=4) == cmg.OK
    assert check("poisson3d_fourier", 13, b1=4, b2=2, k_u=1) == cmg.ERANGE
    assert check("poisson3d_fourier", 15) == cmg.EINVAL  # above the deepest hierarchy


def test_section_blocks_agree_with_the_oracle(libpath):
    """The BFP layout's block count (rows of ceil((2^l - 1)/32) blocks), from the
    library and from the oracle, on every level the library accepts."""
    import oracle
    from paper_2511_19036_gb300 import cmg
    for dim in (2, 3):
        for level in range(1, 15):
            n = (1 << level) - 1
            want = (n if dim == 3 else 1) * n * ((n + 31) // 32)
            assert cmg.lib().cmg_section_blocks(dim, level) == want
            if level <= 9:
                assert oracle.nblocks(dim, level) == want
