"""Pins against the paper's printed parameters (Table 2, Sec. 7.2).

The fixture tests/golden/table2_parameters.txt holds Table 2 and two
statements the paper makes about it elsewhere. The tests check:

- the transcription against those statements;
- the oracle's storage model (oracle/storage_model.py) against the Table 2
  caption, which says b1 and b2 are the bits per DoF on the finest FMG level;
- the 2-D configuration used here against Table 2's 2-D Poisson p = 1 column.
"""
import os

import pytest

from oracle import storage_model as sm
from paper_2511_19036_gb300.cmg_config import config_for

FIXTURE = os.path.join(os.path.dirname(__file__), "golden", "table2_parameters.txt")


def load():
    table, claims = {}, {}
    for line in open(FIXTURE):
        line = line.split("#", 1)[0].split()
        if not line:
            continue
        if line[0] == "claim":
            claims[line[1]] = line[2:]
            continue
        prob, m, row, vals = line[0], int(line[1]), line[2], line[3:]
        assert len(vals) == 7, line
        for p, v in enumerate(vals, start=1):
            if v != "-":
                table.setdefault((prob, p), {"m": m})[row] = int(v)
    return table, claims


TABLE, CLAIMS = load()


def test_fixture_shape():
    # 5 + 5 + 5 (p = 1..5, Poisson 1-D and 2-D; p = 3..7 biharmonic) columns
    assert len(TABLE) == 15
    for key, rec in TABLE.items():
        assert set(rec) == {"m", "N", "b1", "b2", "b3", "b4"}, key


def test_transcription_matches_the_papers_statements():
    lo1, hi1 = map(int, CLAIMS["range_b1"])
    lo2, hi2 = map(int, CLAIMS["range_b2"])
    b1s = [r["b1"] for r in TABLE.values()]
    b2s = [r["b2"] for r in TABLE.values()]
    assert (min(b1s), max(b1s)) == (lo1, hi1)
    assert (min(b2s), max(b2s)) == (lo2, hi2)
    prob, p, bits = CLAIMS["bits_per_point"]
    rec = TABLE[(prob, int(p))]
    assert rec["b1"] + 2 * rec["b2"] == int(bits)
    # about one sixth of a binary64 value
    assert abs(int(bits) / 64 - 1 / 6) < 0.01


@pytest.mark.parametrize("key", sorted(TABLE))
def test_storage_model_finest_level_bits_are_b1_and_b2(key):
    rec = TABLE[key]
    p, m = key[1], rec["m"]
    k_u, k_r = p + 1, m  # increments of the regressive widths (Table 1)
    d = 2 if key[0] == "poisson2d" else 1
    for L in (3, 10, 22):
        assert sm.regressive_bits(k_u, rec["b1"], L, L) == rec["b1"]
        assert sm.regressive_bits(k_r, rec["b2"], L, L) == rec["b2"]
        # the finest level's share of the FMG storage: u~, r and y~ at b1, b2, b2
        n_L = dict(sm.level_sizes(d, L))[L]
        finest = n_L * (sm.regressive_bits(k_u, rec["b1"], L, L) + 2 * sm.regressive_bits(k_r, rec["b2"], L, L))
        coarser = sum(n * (sm.regressive_bits(k_u, rec["b1"], L, l) + 2 * sm.regressive_bits(k_r, rec["b2"], L, l))
                      for l, n in sm.level_sizes(d, L) if l < L)
        assert sm.cmg_fmg_bits(d, L, k_u, k_r, rec["b1"], rec["b2"]) == finest + coarser
        assert finest == n_L * (rec["b1"] + 2 * rec["b2"])


@pytest.mark.parametrize("smoother", [0, 1])
def test_2d_configuration_is_table2_poisson_2d_p1(smoother):
    rec = TABLE[("poisson2d", 1)]
    cfg = config_for("poisson2d_manufactured", 8, smoother=smoother)
    assert (cfg.N_ir, cfg.b1, cfg.b2) == (rec["N"], rec["b1"], rec["b2"])
    assert (cfg.k_u, cfg.k_r) == (1 + 1, rec["m"])
