"""The committed ncu summaries under profiles/ (CPU only).

Each ncu summary names the kernel sources it was taken on (source_sha). Every ncu
command it gives leaves the GPU clocks alone (--clock-control none) and runs
only committed files (bench.py). The per-unit figures the bench reads parse
whenever the summary matches the current kernel sources.
"""
import glob
import os
import re

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FILES = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))


def commands(txt):
    """The ncu command lines of a summary, continuation lines joined."""
    out, cur = [], None
    for line in txt.splitlines():
        s = line.strip()
        if cur is not None:
            cur += " " + s.rstrip("\\").strip()
            if not s.endswith("\\"):
                out.append(cur)
                cur = None
        elif line.startswith("    ncu "):  # indented command blocks only
            cur = s.rstrip("\\").strip()
            if not s.endswith("\\"):
                out.append(cur)
                cur = None
    return out


def test_there_are_summaries():
    assert len(FILES) >= 8


@pytest.mark.parametrize("path", FILES, ids=[os.path.basename(f) for f in FILES])
def test_summary_is_well_formed(path):
    txt = open(path).read()
    if not os.path.basename(path).startswith("clocks_"):  # nvidia-smi samples, not ncu
        assert re.search(r"^source_sha: [0-9a-f]{16}$", txt, re.M), "no source_sha line"
    assert len(txt) < 8192, "summaries stay short"
    for cmd in commands(txt):
        assert "--clock-control none" in cmd, cmd
        assert " python bench.py " in " " + cmd + " ", cmd


@pytest.mark.parametrize("kernel,workload", [("k_fast_sweep", "poisson3d_2049_rbgs"),
                                             ("k_sweep", "poisson3d_2049_jacobi")])
def test_bench_figures_parse_for_current_sources(kernel, workload):
    path = os.path.join(ROOT, "profiles", "%s_%s.md" % (kernel, workload))
    if not os.path.exists(path):
        pytest.skip("no summary for this kernel and workload; the bench reports traffic null")
    sha = re.search(r"source_sha:\s*([0-9a-f]+)", open(path).read()).group(1)
    if sha != bench.source_sha():
        pytest.skip("summary predates the current kernel sources; the bench reports traffic null")
    traffic = bench.read_traffic(kernel, workload)
    inst = bench.read_profile(kernel, workload, "warp_inst_per_row")
    # a few bytes per DoF and a few hundred warp-instructions per 32-value row
    assert traffic is not None and 1.0 < traffic < 5.0
    assert inst is not None and 100 < inst < 1000
