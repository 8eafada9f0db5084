"""Values printed in the paper (tests/golden/paper_values.json, each cited)."""
import json
import math
import os

import numpy as np
import pytest

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_default_weight_parameters_match_paper(orc):
    p = orc.default_params(2, 0)
    g = GOLD["weights"]
    assert (p[0], p[1], p[2], p[3]) == (g["eps"], g["r"], g["lambda0"], g["lambda_s"])


@pytest.mark.parametrize("case", GOLD["stencil_sizes"]["cases"])
def test_stencil_sizes(orc, wl, case):
    mesh = wl.tri_mesh(8) if case["dim"] == 2 else wl.tet_mesh(5)
    o = orc.Oracle(mesh, case["M"] + 1)
    assert o.ne == case["ne"]
    S0, sec = o.stencil(3)
    assert len(S0) == case["ne"]
    assert sec.shape[1] + 1 == case["sector_cells"]


@pytest.mark.parametrize("case", GOLD["dof_per_cell"]["cases"] + GOLD["total_dofs"]["cases"])
def test_dof_counts(orc, wl, case):
    mesh = wl.tri_mesh(8) if case["dim"] == 2 else wl.tet_mesh(5)
    o = orc.Oracle(mesh, case["M"] + 1)
    if "Mcal" in case:
        assert o.Mc == case["Mcal"]
    else:
        assert case["elements"] * o.Mc == case["dofs"]


def test_memory_ratio_formula():
    g = GOLD["memory_ratio"]
    for d, approx in ((2, g["approx_2d"]), (3, g["approx_3d"])):
        M = 50  # "sufficiently high polynomial degree"
        Mc = math.comb(M + d, d)
        ratio = (d * Mc ** 2 + (d + 1) ** 3) / ((1 + 2 * (d + 1)) * d * Mc ** 2)
        assert abs(ratio - approx) < 1e-3
