"""The pins catch plausible mistakes: each test plants one mistake in the oracle (CPU only, via
monkeypatch) and checks that a pin from test_oracle_*.py then fails."""
import numpy as np
import pytest

import synth
from oracle import basis, cg, dg, quadrature, topology
from tests import brute


def _linear_energy_error(p=2):
    xyz, cells = synth.kuhn_cube(2, jitter=0.2, seed=0)
    dofs, keys = topology.cg_numbering(cells, p)
    X = xyz[keys].mean(axis=1)
    a = np.array([0.3, -1.2, 0.7])
    u = X @ a + 0.4
    return abs(u @ cg.apply(xyz, cells, u, p, dofs=dofs) - a @ a)


def _element_matrix_error(p=2):
    rng = np.random.default_rng(12)
    xyz = rng.normal(size=(4, 3))
    cells = np.array([[0, 1, 2, 3]])
    nd = basis.num_dofs(p)
    K = brute.stiffness(xyz, p)
    cols = cg.element_apply(xyz, np.repeat(cells, nd, 0), np.eye(nd), p)
    return np.abs(cols.T - K).max() / np.abs(K).max()


def test_unplanted_oracle_passes():
    assert _linear_energy_error() < 1e-12
    assert _element_matrix_error() < 1e-12


def test_transposed_inverse_jacobian_is_caught(monkeypatch):
    orig = cg.geometry

    def wrong(xyz, cells):
        J, det, Jinv = orig(xyz, cells)
        return J, det, np.transpose(Jinv, (0, 2, 1))

    monkeypatch.setattr(cg, "geometry", wrong)
    assert _element_matrix_error() > 1e-3


def test_signed_determinant_is_caught(monkeypatch):
    """Forgetting |.| on det J (half of the Kuhn cells have det J < 0)."""
    import types

    proxy = types.SimpleNamespace(**{k: getattr(np, k) for k in dir(np) if not k.startswith("__")})
    proxy.abs = lambda v: v
    monkeypatch.setattr(cg, "np", proxy)
    assert _linear_energy_error() > 1e-3


def test_dropped_quadrature_point_is_caught(monkeypatch):
    orig = quadrature.tet_rule

    def wrong(p, modified=False):
        x, w = orig(p, modified)
        return x[:-1], w[:-1]

    monkeypatch.setattr(quadrature, "tet_rule", wrong)
    assert _element_matrix_error() > 1e-3


def test_wrong_node_order_is_caught(monkeypatch):
    orig = basis.nodes_beta

    def wrong(p):
        return list(reversed(orig(p)))

    basis._coefficients.cache_clear()
    monkeypatch.setattr(basis, "nodes_beta", wrong)
    try:
        err = _element_matrix_error()
    finally:
        monkeypatch.undo()
        basis._coefficients.cache_clear()
    assert err > 1e-3


def _dg_penalty_pin(p=1):
    xyz, cells = synth.kuhn_cube(2, jitter=0.2, seed=4)
    nd = basis.num_dofs(p)
    c = synth.uniform_vector(cells.shape[0], 5)
    u = np.repeat(c, nd)
    y = dg.apply(xyz, cells, u, p)
    from tests.test_oracle_dg import face_table

    faces_, vol, area = face_table(xyz, cells)
    eta = (p + 1) * (p + 3)
    expect = 0.0
    for tri, cs in faces_.items():
        F = area(tri)
        tau = eta / min(3 * vol(k) / F for k in cs)
        expect += tau * F * (c[cs[0]] - c[cs[1]]) ** 2 if len(cs) == 2 else 2 * tau * F * c[cs[0]] ** 2
    return abs(u @ y - expect) / expect


def test_dg_penalty_mistakes_are_caught(monkeypatch):
    assert _dg_penalty_pin() < 1e-11
    monkeypatch.setattr(dg, "default_penalty", lambda p: float((p + 1) * (p + 2)))
    assert _dg_penalty_pin() > 1e-3


def test_dg_normal_sign_is_caught(monkeypatch):
    """A normal pointing into the owner cell breaks the closed form of the boundary terms."""
    from tests.test_oracle_dg import test_linear_field_with_boundary_terms

    test_linear_field_with_boundary_terms()
    orig = dg._face_geometry

    def wrong(xyz, cells, c, m, p):
        pts, W, n, area = orig(xyz, cells, c, m, p)
        return pts, W, -n, area

    monkeypatch.setattr(dg, "_face_geometry", wrong)
    with pytest.raises(AssertionError):
        test_linear_field_with_boundary_terms()


def test_too_small_modified_rule_is_caught(monkeypatch):
    """A modified rule one order too small (s = p - 2, exact to 2p - 3) fails the brute-force pin."""
    from tests.test_oracle_modified_rule import test_modified_element_matrix_brute_force

    test_modified_element_matrix_brute_force(3)
    orig = quadrature.tet_rule
    monkeypatch.setattr(quadrature, "tet_rule", lambda p, modified=False: orig(p - 1 if modified else p, modified))
    with pytest.raises(AssertionError):
        test_modified_element_matrix_brute_force(3)


def test_wrong_chebyshev_recurrence_is_caught(monkeypatch):
    """rho_k = 1 / (2 sigma + rho_{k-1}) instead of 1 / (2 sigma - rho_{k-1}) fails the error-polynomial pin."""
    from oracle import smoother
    from tests.test_oracle_smoother import test_error_polynomial_on_a_diagonal_operator

    test_error_polynomial_on_a_diagonal_operator(5)

    def wrong(degree, lam_max, lam_min):
        theta, delta = 0.5 * (lam_max + lam_min), 0.5 * (lam_max - lam_min)
        sigma = theta / delta
        out, rho = [(0.0, 1.0 / theta)], 1.0 / sigma
        for _ in range(degree - 1):
            rho_new = 1.0 / (2.0 * sigma + rho)
            out.append((rho_new * rho, 2.0 * rho_new / delta))
            rho = rho_new
        return out

    monkeypatch.setattr(smoother, "step_coefficients", wrong)
    with pytest.raises(AssertionError):
        test_error_polynomial_on_a_diagonal_operator(5)


def test_wrong_transfer_table_is_caught(monkeypatch):
    """Fine nodes taken in reverse order when tabulating the coarse basis breaks polynomial reproduction."""
    import types

    from oracle import transfer
    from tests.test_oracle_transfer import test_prolongation_reproduces_coarse_polynomials

    test_prolongation_reproduces_coarse_polynomials(3, 1)
    proxy = types.SimpleNamespace(nodes_beta=lambda p: list(reversed(basis.nodes_beta(p))), values=basis.values)
    monkeypatch.setattr(transfer, "basis", proxy)
    with pytest.raises(AssertionError):
        test_prolongation_reproduces_coarse_polynomials(3, 1)
