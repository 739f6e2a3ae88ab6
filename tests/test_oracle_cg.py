"""Pins for the oracle's continuous operator (Eq. 3): brute-force element matrices,
closed forms of the Neumann Laplacian, the 7-point stencil, symmetry, the adjoint,
the coefficient gradient and the Dirichlet set."""
import numpy as np
import pytest

import synth
from oracle import cg, topology
from tests import brute


def jittered(n, jitter=0.2, seed=0):
    return synth.kuhn_cube(n, jitter=jitter, seed=seed)


def dof_xyz(xyz, cells, p):
    dofs, keys = topology.cg_numbering(cells, p)
    return dofs, keys, xyz[keys].mean(axis=1)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_element_matrix_brute_force(p):
    rng = np.random.default_rng(10 + p)
    xyz = rng.normal(size=(8, 3))
    cells = np.array([[0, 1, 2, 3], [4, 5, 6, 7], [1, 0, 2, 3]])
    nd = (p + 1) * (p + 2) * (p + 3) // 6
    for c in range(cells.shape[0]):
        K = brute.stiffness(xyz[cells[c]], p)
        cols = cg.element_apply(xyz, np.repeat(cells[c:c + 1], nd, 0), np.eye(nd), p)
        assert np.allclose(cols.T, K, rtol=0, atol=1e-12 * np.abs(K).max())


@pytest.mark.parametrize("p", [1, 2, 3])
def test_neumann_row_sums_zero(p):
    xyz, cells = jittered(3)
    dofs, keys = topology.cg_numbering(cells, p)
    y = cg.apply(xyz, cells, np.ones(keys.shape[0]), p, dofs=dofs)
    assert np.abs(y).max() < 1e-13


@pytest.mark.parametrize("p", [1, 2, 3])
def test_energy_of_linear_field(p):
    """u = a.x + b on the unit cube: u^T A u = |Omega| |a|^2 = |a|^2."""
    xyz, cells = jittered(3)
    dofs, keys, X = dof_xyz(xyz, cells, p)
    a = np.array([0.3, -1.2, 0.7])
    u = X @ a + 0.4
    y = cg.apply(xyz, cells, u, p, dofs=dofs)
    assert abs(u @ y - a @ a) < 1e-12


@pytest.mark.parametrize("p", [2, 3])
def test_energy_of_quadratic_field(p):
    """u = x^2 (exactly represented for p >= 2): int |grad u|^2 = int 4 x^2 = 4/3."""
    xyz, cells = jittered(2)
    dofs, keys, X = dof_xyz(xyz, cells, p)
    u = X[:, 0] ** 2
    y = cg.apply(xyz, cells, u, p, dofs=dofs)
    assert abs(u @ y - 4.0 / 3.0) < 1e-12


def test_p1_kuhn_seven_point_stencil():
    n = 4
    h = 1.0 / n
    xyz, cells = synth.kuhn_cube(n)
    dofs, keys = topology.cg_numbering(cells, 1)
    N = keys.shape[0]
    i, j, k = 2, 2, 2
    vid = i + (n + 1) * (j + (n + 1) * k)
    row = np.searchsorted(keys[:, 0], vid)
    e = np.zeros(N)
    e[row] = 1.0
    col = cg.apply(xyz, cells, e, 1, dofs=dofs)  # symmetric: column == row
    expect = np.zeros(N)
    expect[row] = 6 * h
    for d in [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]:
        nb = (i + d[0]) + (n + 1) * ((j + d[1]) + (n + 1) * (k + d[2]))
        expect[np.searchsorted(keys[:, 0], nb)] = -h
    assert np.allclose(col, expect, atol=1e-14)


@pytest.mark.parametrize("p", [1, 2])
def test_matches_brute_force_assembly(p):
    xyz, cells = jittered(2, seed=5)
    A, nodes = brute.assemble_cg(xyz, cells, p)
    dofs, keys, X = dof_xyz(xyz, cells, p)
    # match brute-force DoFs (by coordinate) to canonical DoFs
    order = [int(np.argmin(np.linalg.norm(nodes - x, axis=1))) for x in X]
    u = np.random.default_rng(0).uniform(-1, 1, size=X.shape[0])
    ub = np.empty_like(u)
    ub[order] = u
    y = cg.apply(xyz, cells, u, p, dofs=dofs)
    yb = (A @ ub)[order]
    assert np.allclose(y, yb, atol=1e-13)
    d = cg.diagonal(xyz, cells, p, X.shape[0], dofs=dofs)
    assert np.allclose(d, np.diag(A)[order], atol=1e-13)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_symmetry_and_adjoint_variable_k(p):
    xyz, cells = jittered(2, seed=1)
    dofs, keys = topology.cg_numbering(cells, p)
    N = keys.shape[0]
    nq = cg.tables(p)[1].shape[0]
    k = synth.lognormal_coefficients((cells.shape[0], nq), seed=3)
    u = synth.uniform_vector(N, 1)
    v = synth.uniform_vector(N, 2)
    Au = cg.apply(xyz, cells, u, p, k=k, dofs=dofs)
    Atv = cg.apply_adjoint(xyz, cells, v, p, k=k, dofs=dofs)
    assert abs(v @ Au - Atv @ u) < 1e-12 * abs(v @ Au) + 1e-14
    Av = cg.apply(xyz, cells, v, p, k=k, dofs=dofs)
    assert abs(v @ Au - u @ Av) < 1e-12 * abs(v @ Au) + 1e-14


def test_coefficient_scaling():
    """A(c k) = c A(k): the coefficient enters linearly at every quadrature point."""
    xyz, cells = jittered(2, seed=2)
    p = 2
    dofs, keys = topology.cg_numbering(cells, p)
    nq = cg.tables(p)[1].shape[0]
    u = synth.uniform_vector(keys.shape[0], 1)
    y1 = cg.apply(xyz, cells, u, p, dofs=dofs)
    y3 = cg.apply(xyz, cells, u, p, k=np.full((cells.shape[0], nq), 3.0), dofs=dofs)
    assert np.allclose(y3, 3.0 * y1, atol=1e-13)


@pytest.mark.parametrize("p", [1, 2])
def test_coeff_grad_identities(p):
    xyz, cells = jittered(2, seed=3)
    dofs, keys = topology.cg_numbering(cells, p)
    N = keys.shape[0]
    nq = cg.tables(p)[1].shape[0]
    k = synth.lognormal_coefficients((cells.shape[0], nq), seed=3)
    u = synth.uniform_vector(N, 1)
    g = synth.uniform_vector(N, 2)
    L = lambda kk: g @ cg.apply(xyz, cells, u, p, k=kk, dofs=dofs)
    grad_u, dk = cg.coeff_grad(xyz, cells, u, g, p, k=k, dofs=dofs)
    L0 = L(k)
    # Euler identity: L is linear (homogeneous of degree 1) in k
    assert abs((k * dk).sum() - L0) < 1e-12 * abs(L0)
    # L = <grad_u, u> since L is linear in u
    assert abs(grad_u @ u - L0) < 1e-12 * abs(L0)
    # central differences in k (exact up to roundoff since L is linear in k)
    rng = np.random.default_rng(7)
    for _ in range(5):
        e, q = rng.integers(cells.shape[0]), rng.integers(nq)
        kp, km = k.copy(), k.copy()
        kp[e, q] += 1e-6
        km[e, q] -= 1e-6
        fd = (L(kp) - L(km)) / 2e-6
        assert abs(fd - dk[e, q]) < 1e-8 * max(1.0, abs(dk[e, q]))
    # central differences in u
    for _ in range(3):
        i = rng.integers(N)
        up, um = u.copy(), u.copy()
        up[i] += 1e-6
        um[i] -= 1e-6
        fd = (g @ cg.apply(xyz, cells, up, p, k=k, dofs=dofs) - g @ cg.apply(xyz, cells, um, p, k=k, dofs=dofs)) / 2e-6
        assert abs(fd - grad_u[i]) < 1e-7


@pytest.mark.parametrize("p", [1, 2, 3])
def test_dof_count_and_lattice_numbering(p):
    """Unjittered Kuhn mesh: DoFs are exactly the (pn+1)^3 lattice points at spacing h/p."""
    n = 3
    xyz, cells = synth.kuhn_cube(n)
    dofs, keys, X = dof_xyz(xyz, cells, p)
    assert keys.shape[0] == (p * n + 1) ** 3
    lattice = np.round(X * p * n).astype(int)
    assert np.allclose(lattice, X * p * n, atol=1e-9)
    ids = lattice[:, 0] + (p * n + 1) * (lattice[:, 1] + (p * n + 1) * lattice[:, 2])
    assert np.array_equal(np.sort(ids), np.arange((p * n + 1) ** 3))


@pytest.mark.parametrize("p", [1, 2, 3])
def test_dirichlet_mask_counts(p):
    n = 3
    xyz, cells = synth.kuhn_cube(n, jitter=0.2, seed=0)
    dofs, keys = topology.cg_numbering(cells, p)
    mask = topology.dirichlet_mask(cells, p, keys)
    m = p * n + 1
    assert mask.sum() == m ** 3 - (m - 2) ** 3
    xyz0, _ = synth.kuhn_cube(n)
    X = xyz0[keys].mean(axis=1)
    on_bnd = np.any((X < 1e-12) | (X > 1 - 1e-12), axis=1)
    assert np.array_equal(mask, on_bnd)


def test_dirichlet_operator_structure():
    p = 2
    xyz, cells = jittered(2, seed=4)
    dofs, keys = topology.cg_numbering(cells, p)
    mask = topology.dirichlet_mask(cells, p, keys)
    u = synth.uniform_vector(keys.shape[0], 1)
    y = cg.apply(xyz, cells, u, p, dirichlet_mask=mask, dofs=dofs)
    assert np.array_equal(y[mask], u[mask])
    u2 = u.copy()
    u2[mask] = 0.0
    y2 = cg.apply(xyz, cells, u2, p, dofs=dofs)
    assert np.allclose(y[~mask], y2[~mask], atol=1e-14)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_rhs_total_mass(p):
    """sum_i b_i = int_Omega f = 1 for f = 1 (partition of unity), and b = M 1."""
    xyz, cells = jittered(2, seed=6)
    dofs, keys = topology.cg_numbering(cells, p)
    b = cg.rhs_const(xyz, cells, p, keys.shape[0], dofs=dofs)
    assert abs(b.sum() - 1.0) < 1e-13
