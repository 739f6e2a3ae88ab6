"""Pins for the modified cell integration of Sec. 3.3 in the oracle: a rule exact to degree 2p-2
integrates the Laplace stiffness of an affine cell exactly, so with it the element matrices still
equal the brute-force (exact monomial) integrals, and the operator, its diagonal and the load
vector equal those of the standard rule; the same holds for a coefficient linear in x (degree
2p-1 integrand)."""
import numpy as np
import pytest

import synth
from oracle import cg, dg, quadrature, topology
from tests import brute


def test_modified_rule_sizes():
    assert [quadrature.tet_rule(p, modified=True)[0].shape[0] for p in (1, 2, 3, 4)] == [1, 5, 15, 35]
    x, w = quadrature.tet_rule(1, modified=True)
    assert np.allclose(x, [[0.25, 0.25, 0.25]], rtol=0, atol=1e-16) and abs(w[0] - 1.0 / 6.0) < 1e-16


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_modified_element_matrix_brute_force(p):
    rng = np.random.default_rng(20 + p)
    xyz = rng.normal(size=(8, 3))
    cells = np.array([[0, 1, 2, 3], [4, 5, 6, 7]])
    nd = (p + 1) * (p + 2) * (p + 3) // 6
    for c in range(cells.shape[0]):
        K = brute.stiffness(xyz[cells[c]], p)
        cols = cg.element_apply(xyz, np.repeat(cells[c:c + 1], nd, 0), np.eye(nd), p, modified=True)
        assert np.allclose(cols.T, K, rtol=0, atol=1e-12 * np.abs(K).max())


@pytest.mark.parametrize("p", [1, 2, 3])
def test_modified_operator_diagonal_rhs_equal_standard(p):
    xyz, cells = synth.kuhn_cube(2, jitter=0.2, seed=5)
    dofs, keys = topology.cg_numbering(cells, p)
    N = keys.shape[0]
    u = synth.uniform_vector(N, 1)
    y = cg.apply(xyz, cells, u, p, dofs=dofs)
    ym = cg.apply(xyz, cells, u, p, dofs=dofs, modified=True)
    assert np.abs(ym - y).max() <= 1e-12 * np.abs(y).max()
    d = cg.diagonal(xyz, cells, p, N, dofs=dofs)
    assert np.allclose(cg.diagonal(xyz, cells, p, N, dofs=dofs, modified=True), d, rtol=1e-12, atol=0)
    b = cg.rhs_const(xyz, cells, p, N, dofs=dofs)
    assert np.abs(cg.rhs_const(xyz, cells, p, N, dofs=dofs, modified=True) - b).max() <= 1e-12 * np.abs(b).max()


@pytest.mark.parametrize("p", [1, 2, 3])
def test_modified_rule_exact_for_linear_coefficient(p):
    """k(x) = 1.5 + a . x sampled at each rule's own points gives the same operator."""
    xyz, cells = synth.kuhn_cube(2, jitter=0.2, seed=6)
    dofs, keys = topology.cg_numbering(cells, p)
    u = synth.uniform_vector(keys.shape[0], 2)
    a = np.array([0.4, -0.3, 0.2])
    X = xyz[cells]

    def k_at(modified):
        xq = quadrature.tet_rule(p, modified)[0]
        lam = np.concatenate([1.0 - xq.sum(axis=1, keepdims=True), xq], axis=1)  # barycentric [nq, 4]
        pts = np.einsum("qv,cvd->cqd", lam, X)
        return 1.5 + pts @ a

    y = cg.apply(xyz, cells, u, p, k=k_at(False), dofs=dofs)
    ym = cg.apply(xyz, cells, u, p, k=k_at(True), dofs=dofs, modified=True)
    assert np.abs(ym - y).max() <= 1e-12 * np.abs(y).max()


def test_modified_rule_differs_for_quadratic_coefficient():
    """The modified rule is genuinely smaller: a quadratic coefficient exposes it at p = 2."""
    p = 2
    xyz, cells = synth.kuhn_cube(2, jitter=0.2, seed=6)
    dofs, keys = topology.cg_numbering(cells, p)
    u = synth.uniform_vector(keys.shape[0], 2)
    X = xyz[cells]

    def k_at(modified):
        xq = quadrature.tet_rule(p, modified)[0]
        lam = np.concatenate([1.0 - xq.sum(axis=1, keepdims=True), xq], axis=1)
        pts = np.einsum("qv,cvd->cqd", lam, X)
        return 1.0 + (pts ** 2).sum(axis=2)

    y = cg.apply(xyz, cells, u, p, k=k_at(False), dofs=dofs)
    ym = cg.apply(xyz, cells, u, p, k=k_at(True), dofs=dofs, modified=True)
    assert np.abs(ym - y).max() > 1e-8 * np.abs(y).max()


@pytest.mark.parametrize("p", [1, 2])
def test_dg_modified_cell_rule_equal_standard(p):
    xyz, cells = synth.kuhn_cube(2, jitter=0.2, seed=7)
    nd = (p + 1) * (p + 2) * (p + 3) // 6
    u = synth.uniform_vector(cells.shape[0] * nd, 3)
    y = dg.apply(xyz, cells, u, p)
    ym = dg.apply(xyz, cells, u, p, modified=True)
    assert np.abs(ym - y).max() <= 1e-12 * np.abs(y).max()
