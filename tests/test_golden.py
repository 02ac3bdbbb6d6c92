"""Stored fixtures: facts the paper states (tests/golden/paper_facts.txt) and
oracle regression values written by tests/golden/make_golden.py (oracle only)."""
import json
import os

import numpy as np
import pytest

import pot3d_synth as syn

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def paper_facts():
    facts = {}
    with open(os.path.join(GOLD, "paper_facts.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                k, v = [s.strip() for s in line.split("=")]
                facts[k] = v
    return facts


def test_cell_centred_count_matches_paper(oracle_mod):
    """Sec. 4.1 counts N_r x N_theta x N_phi as grid cells (more than 2e8 for
    its mesh): the unknowns are cell centres, one per (i, j, k)."""
    f = paper_facts()
    nr, nt, np_ = [int(v) for v in f["paper_mesh"].split()]
    assert nr * nt * np_ > int(f["paper_cells_min"])
    g = oracle_mod.Grid(3, 4, 5)
    assert g.n == 3 * 4 * 5 and g.rc.size == 3 and g.tc.size == 4 and g.pc.size == 5


def test_pole_epsilon_half_cell(oracle_mod):
    """Eq. 3: the polar average is taken half a cell from the pole, which is
    where the first theta centre sits."""
    eps = float(paper_facts()["pole_epsilon_cells"])
    g = oracle_mod.Grid(2, 9, 4)
    w = g.tf[1] - g.tf[0]
    assert abs(g.tc[0] - eps * w) < 1e-15 and abs((np.pi - g.tc[-1]) - eps * w) < 1e-15


@pytest.mark.parametrize("name", ["ylm32_40x40x80", "bip_13x21x37_g1.05", "bip_24x33x65_g1.02"])
def test_oracle_regression(oracle_mod, name):
    with open(os.path.join(GOLD, "oracle_small.json")) as f:
        case = json.load(f)[name]
    g = oracle_mod.Grid(*case["shape"], ratio=case["ratio"])
    if case["br"] == "ylm":
        br = syn.ylm_br(case["shape"][1], case["shape"][2], 3, 2)[0]
    else:
        br = syn.bipole_br(case["shape"][1], case["shape"][2], seed=1709, n_bipoles=40)
    x, it, st = g.solve(br, case["tol"])
    assert st == case["status"]
    assert abs(it - case["iters"]) <= 1
    np.testing.assert_allclose(x.ravel()[case["sample_index"]], case["sample_phi"], rtol=1e-9,
                               atol=1e-12 * np.abs(x).max())
