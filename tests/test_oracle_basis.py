"""Pins for the oracle's Lagrange basis: Kronecker property, partition of unity,
polynomial reproduction, gradients against central differences and against the
independent Silvester construction in tests/brute.py."""
import numpy as np
import pytest

from oracle import basis
from tests import brute


def random_points(m, seed=0):
    rng = np.random.default_rng(seed)
    x = rng.dirichlet(np.ones(4), size=m)
    return x[:, 1:]


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_kronecker(p):
    nodes = np.array([[b[1], b[2], b[3]] for b in basis.nodes_beta(p)], dtype=float) / p
    V = basis.values(p, nodes)
    assert V.shape == (basis.num_dofs(p),) * 2
    assert np.allclose(V, np.eye(V.shape[0]), atol=1e-12)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_partition_of_unity_and_zero_gradient_sum(p):
    x = random_points(50)
    assert np.allclose(basis.values(p, x).sum(-1), 1.0, atol=1e-12)
    assert np.allclose(basis.gradients(p, x).sum(-2), 0.0, atol=1e-11)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_polynomial_reproduction(p):
    nodes = np.array([[b[1], b[2], b[3]] for b in basis.nodes_beta(p)], dtype=float) / p
    x = random_points(40, seed=1)
    rng = np.random.default_rng(2)
    c = rng.normal(size=4)
    f = lambda z: (c[0] + c[1] * z[..., 0] + c[2] * z[..., 1] + c[3] * z[..., 2]) ** p
    interp = basis.values(p, x) @ f(nodes)
    assert np.allclose(interp, f(x), atol=1e-11)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_gradient_central_difference(p):
    x = random_points(10, seed=3) * 0.8 + 0.05
    G = basis.gradients(p, x)
    h = 1e-6
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        fd = (basis.values(p, x + e) - basis.values(p, x - e)) / (2 * h)
        assert np.allclose(G[..., k], fd, atol=1e-7)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_matches_silvester(p):
    x = random_points(20, seed=4)
    lam = np.concatenate([1 - x.sum(1, keepdims=True), x], axis=1)
    sil = brute.silvester_basis(p)
    ref = np.array([[sum(float(c) * np.prod(l ** np.array(e)) for e, c in poly.items()) for poly in sil] for l in lam])
    assert np.allclose(basis.values(p, x), ref, atol=1e-12)
