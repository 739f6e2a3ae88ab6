"""Pins for the oracle's Grundmann-Moeller rules: exact rational monomial integrals."""
from fractions import Fraction
from itertools import product
from math import factorial

import numpy as np
import pytest

from oracle import quadrature


def exact_monomial(exps):
    """int over the unit n-simplex of prod x_k^{a_k} = prod a_k! / (sum a + n)!."""
    num = 1
    for a in exps:
        num *= factorial(a)
    return Fraction(num, factorial(sum(exps) + len(exps)))


@pytest.mark.parametrize("n", [2, 3])
@pytest.mark.parametrize("s", [0, 1, 2, 3, 4])
def test_exact_to_degree_2s_plus_1(s, n):
    pts, wts = quadrature.gm_rule_exact(s, n)
    deg = 2 * s + 1
    for exps in product(range(deg + 1), repeat=n):
        if sum(exps) > deg:
            continue
        q = sum(w * np.prod([p[k + 1] ** exps[k] for k in range(n)]) for p, w in zip(pts, wts))
        assert q == exact_monomial(exps), (s, n, exps)


@pytest.mark.parametrize("n", [2, 3])
@pytest.mark.parametrize("s", [1, 2, 3])
def test_not_exact_beyond_degree(s, n):
    """Degree 2s+2 is generally not integrated exactly (the rule is not accidentally a higher one)."""
    pts, wts = quadrature.gm_rule_exact(s, n)
    deg = 2 * s + 2
    errs = []
    for exps in product(range(deg + 1), repeat=n):
        if sum(exps) != deg:
            continue
        q = sum(w * np.prod([p[k + 1] ** exps[k] for k in range(n)]) for p, w in zip(pts, wts))
        errs.append(q != exact_monomial(exps))
    assert any(errs)


def test_point_counts():
    assert [len(quadrature.gm_rule_exact(s, 3)[1]) for s in (1, 2, 3, 4)] == [5, 15, 35, 70]
    assert [len(quadrature.gm_rule_exact(s, 2)[1]) for s in (1, 2, 3, 4)] == [4, 10, 20, 35]


def test_worked_example_s1_tet():
    """s=1 on the tetrahedron: weight 3/40 at the four points with one barycentric 1/2, -2/15 at the centroid."""
    pts, wts = quadrature.gm_rule_exact(1, 3)
    assert wts[:4] == (Fraction(3, 40),) * 4
    assert wts[4] == Fraction(-2, 15)
    for j, p in enumerate(pts[:4]):
        # beta lexicographic ascending: (0,0,0,1), (0,0,1,0), (0,1,0,0), (1,0,0,0)
        expect = [Fraction(1, 6)] * 4
        expect[3 - j] = Fraction(1, 2)
        assert list(p) == expect
    assert list(pts[4]) == [Fraction(1, 4)] * 4


def test_float_rule_matches_exact():
    x, w = quadrature.tet_rule(3)
    pts, wts = quadrature.gm_rule_exact(3, 3)
    assert x.shape == (35, 3)
    assert np.allclose(w, [float(v) for v in wts], rtol=0, atol=1e-16)
    assert abs(w.sum() - 1.0 / 6.0) < 1e-15
    xt, wt = quadrature.tri_rule(2)
    assert abs(wt.sum() - 0.5) < 1e-15 and xt.shape == (10, 2)
