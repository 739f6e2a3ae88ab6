"""Pins against numbers the paper prints (tests/golden/*.json, each with its citation)."""
import json
import os

import numpy as np
import pytest

from oracle import basis, cg, topology
from tests import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_unique_dofs_per_cell_five_tet_split(p):
    """N(n) is a cubic polynomial in the number n of subcubes per direction (n even keeps the
    alternating 5-tet pattern periodic); its leading coefficient over the 5 cells per subcube is the
    paper's unique-DoFs-per-cell figure."""
    want = load("unique_dofs_5tet_split.json")["values"][str(p)]
    ns = [2, 4, 6, 8]
    Ns = []
    for n in ns:
        xyz, cells = brute.five_tet_cube(n)
        _, keys = topology.cg_numbering(cells, p)
        Ns.append(keys.shape[0])
    coef = np.polyfit(np.array(ns, float), np.array(Ns, float), 3)
    assert abs(coef[0] / 5.0 - want) < 1e-9


def test_interpolation_matrix_shape_p3():
    g = load("interpolation_matrix_p3.json")
    xq, wq, G, V = cg.tables(g["p"])
    assert G.shape[0] * G.shape[2] == g["rows"]
    assert G.shape[1] == g["cols"] == basis.num_dofs(3)
