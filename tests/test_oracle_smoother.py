"""Pins for the oracle's Chebyshev-Jacobi smoother and power iteration: on a diagonal operator the
error after m steps is the scaled Chebyshev polynomial T_m((theta - lambda) / delta) / T_m(theta /
delta) (evaluated here with numpy's Chebyshev series) times the initial error, componentwise; the
power iteration finds a known largest eigenvalue; on the FE operator the smoother reduces the
residual for every degree."""
import numpy as np
import pytest
from numpy.polynomial import chebyshev as npcheb

import synth
from oracle import cg, smoother, topology


@pytest.mark.parametrize("degree", [1, 2, 3, 5, 8])
def test_error_polynomial_on_a_diagonal_operator(degree):
    rng = np.random.default_rng(degree)
    a = rng.uniform(0.05, 2.0, size=40)
    b = rng.normal(size=40)
    lam_max, lam_min = 2.1, 0.3
    x = smoother.chebyshev(lambda v: a * v, np.ones(40), b, np.zeros(40), degree, lam_max, lam_min)
    theta, delta = 0.5 * (lam_max + lam_min), 0.5 * (lam_max - lam_min)
    Tm = np.zeros(degree + 1)
    Tm[degree] = 1.0
    P = npcheb.chebval((theta - a) / delta, Tm) / npcheb.chebval(theta / delta, Tm)
    xs = b / a
    assert np.allclose(xs - x, P * xs, rtol=0, atol=1e-12 * np.abs(xs).max())


def test_jacobi_scaling_is_applied():
    """With D = A (diagonal) the preconditioned spectrum is {1}: one step on [0.5, 1.5] is exact."""
    a = np.linspace(1.0, 50.0, 30)
    b = np.cos(np.arange(30.0))
    x = smoother.chebyshev(lambda v: a * v, a, b, np.zeros(30), 1, 1.5, 0.5)
    assert np.allclose(x, b / a, rtol=1e-14, atol=0)


def test_power_iteration_known_eigenvalue():
    a = np.array([1.0, 3.0, 7.0, 2.0, 5.0])
    d = np.array([1.0, 1.0, 2.0, 1.0, 1.0])
    lam = smoother.lambda_max(lambda v: a * v, d, np.ones(5), 200)
    assert abs(lam - 5.0) < 1e-10  # largest of a / d = (1, 3, 3.5, 2, 5)


@pytest.mark.parametrize("degree", [2, 5])
def test_smoother_reduces_residual_on_the_fe_operator(degree):
    p = 2
    xyz, cells = synth.kuhn_cube(3, jitter=0.2, seed=1)
    dofs, keys = topology.cg_numbering(cells, p)
    N = keys.shape[0]
    mask = topology.dirichlet_mask(cells, p, keys)
    A = lambda v: cg.apply(xyz, cells, v, p, dirichlet_mask=mask, dofs=dofs)
    d = cg.diagonal(xyz, cells, p, N, dirichlet_mask=mask, dofs=dofs)
    lam = smoother.lambda_max(A, d, synth.uniform_vector(N, 2), 40)
    b = synth.uniform_vector(N, 1)
    x = smoother.chebyshev(A, d, b, np.zeros(N), degree, 1.2 * lam, 1.2 * lam / 15.0)
    assert np.linalg.norm(b - A(x)) < 0.7 * np.linalg.norm(b)
