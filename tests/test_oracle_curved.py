"""Pins for the oracle's curved (second-order geometry, Sec. 3.2) operator: it reduces to the affine
operator when the nodes lie on an affine image of the straight cells; on the cube deformed by a map
that fixes the boundary (the domain stays the unit cube, boundary faces stay flat) it keeps
A 1 = 0, symmetry, and u^T A u = |a|^2 for u = a . x (exactly representable for p >= 2, integrand
|a|^2 |det J| of degree 3 integrated exactly); the load vector integrates to |Omega| = 1."""
import numpy as np
import pytest

import synth
from oracle import basis, cg, topology


def test_node_order_is_the_p2_basis_order():
    assert [tuple(b) for b in basis.nodes_beta(2)] == synth.mesh._BETA2


@pytest.mark.parametrize("p", [1, 2, 3])
def test_affine_nodes_reproduce_the_affine_operator(p):
    xyz, cells = synth.kuhn_cube(2, jitter=0.2, seed=3)
    B = np.array([[1.2, 0.3, -0.1], [0.0, 0.9, 0.2], [0.1, -0.2, 1.1]])
    xyz2 = xyz @ B.T + np.array([0.3, -0.4, 2.0])
    nodes = synth.curved_nodes(xyz, cells, 0.0) @ B.T + np.array([0.3, -0.4, 2.0])
    dofs, keys = topology.cg_numbering(cells, p)
    u = synth.uniform_vector(keys.shape[0], 1)
    y = cg.apply(xyz2, cells, u, p, dofs=dofs)
    yc = cg.apply(xyz2, cells, u, p, dofs=dofs, nodes=nodes)
    assert np.abs(yc - y).max() <= 1e-12 * np.abs(y).max()
    N = keys.shape[0]
    assert np.allclose(cg.diagonal(xyz2, cells, p, N, dofs=dofs, nodes=nodes), cg.diagonal(xyz2, cells, p, N, dofs=dofs),
                       rtol=1e-12, atol=0)
    b = cg.rhs_const(xyz2, cells, p, N, dofs=dofs)
    assert np.abs(cg.rhs_const(xyz2, cells, p, N, dofs=dofs, nodes=nodes) - b).max() <= 1e-12 * np.abs(b).max()


def dof_positions(nodes, cells, p, dofs, N):
    """Physical position of every canonical DoF: its reference node pushed through the cell map."""
    xhat = np.array(basis.nodes_beta(p), dtype=np.float64)[:, 1:] / p  # (beta_1, beta_2, beta_3) / p
    phi2 = basis.values(2, xhat)                                       # [nd, 10]
    X = np.einsum("jn,cnd->cjd", phi2, nodes)
    out = np.empty((N, 3))
    out[dofs.ravel()] = X.reshape(-1, 3)
    return out


@pytest.mark.parametrize("p", [2, 3])
def test_curved_closed_forms(p):
    xyz, cells = synth.kuhn_cube(3, jitter=0.2, seed=4)
    nodes = synth.curved_nodes(xyz, cells, 0.05)
    dofs, keys = topology.cg_numbering(cells, p)
    N = keys.shape[0]
    A = lambda v: cg.apply(xyz, cells, v, p, dofs=dofs, nodes=nodes)
    assert np.abs(A(np.ones(N))).max() < 1e-12
    X = dof_positions(nodes, cells, p, dofs, N)
    a = np.array([0.3, -1.2, 0.7])
    u = X @ a + 0.4
    assert abs(u @ A(u) - a @ a) < 1e-11
    v = synth.uniform_vector(N, 2)
    w = synth.uniform_vector(N, 3)
    assert abs(v @ A(w) - w @ A(v)) < 1e-12 * abs(v @ A(w))
    assert abs(cg.rhs_const(xyz, cells, p, N, dofs=dofs, nodes=nodes).sum() - 1.0) < 1e-12
    # and the deformation is not trivial: the operator differs from the straight one
    y0 = cg.apply(xyz, cells, w, p, dofs=dofs)
    assert np.abs(A(w) - y0).max() > 1e-3 * np.abs(y0).max()
