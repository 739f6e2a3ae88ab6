"""Pins for the oracle's p-transfer: prolongation reproduces polynomials of the coarse degree at the
fine nodes; the coarse operator is the Galerkin product P^T A_fine P (nested spaces, exact
quadrature), with and without Dirichlet constraints."""
import numpy as np
import pytest

import synth
from oracle import basis, cg, topology, transfer
from tests import brute


def setup(pf, pc, n=2, seed=3):
    xyz, cells = synth.kuhn_cube(n, jitter=0.2, seed=seed)
    df, kf = topology.cg_numbering(cells, pf)
    dc, kc = topology.cg_numbering(cells, pc)
    P = transfer.prolongation_matrix(cells, pf, pc, df, dc, kf.shape[0], kc.shape[0])
    return xyz, cells, df, kf, dc, kc, P


@pytest.mark.parametrize("pf,pc", [(2, 1), (3, 1), (3, 2), (4, 2)])
def test_prolongation_reproduces_coarse_polynomials(pf, pc):
    xyz, cells, df, kf, dc, kc, P = setup(pf, pc)
    f = lambda X: 0.3 + X @ np.array([1.0, -2.0, 0.5]) + (0.7 * X[:, 0] * X[:, 2] if pc >= 2 else 0.0)
    uc = f(xyz[kc].mean(axis=1))
    uf = transfer.prolongate(P, uc)
    assert np.abs(uf - f(xyz[kf].mean(axis=1))).max() < 1e-13


@pytest.mark.parametrize("pf,pc", [(2, 1), (3, 1), (3, 2)])
def test_galerkin_coarse_operator(pf, pc):
    xyz, cells, df, kf, dc, kc, P = setup(pf, pc)
    Nf, Nc = kf.shape[0], kc.shape[0]
    Af = np.column_stack([cg.apply(xyz, cells, e, pf, dofs=df) for e in np.eye(Nf)])
    Ac = np.column_stack([cg.apply(xyz, cells, e, pc, dofs=dc) for e in np.eye(Nc)])
    assert np.abs(P.T @ Af @ P - Ac).max() < 1e-12 * np.abs(Ac).max()


def test_restriction_is_the_transpose_with_dirichlet():
    pf, pc = 3, 1
    xyz, cells, df, kf, dc, kc, P = setup(pf, pc)
    mf = topology.dirichlet_mask(cells, pf, kf)
    mc = topology.dirichlet_mask(cells, pc, kc)
    uc = synth.uniform_vector(kc.shape[0], 1)
    rf = synth.uniform_vector(kf.shape[0], 2)
    lhs = transfer.prolongate(P, np.where(mc, 0.0, uc), mf) @ rf
    rhs = np.where(mc, 0.0, uc) @ transfer.restrict(P, rf, mf, mc)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # a constrained coarse DoF never feeds an unconstrained fine one through the boundary trace
    uf = transfer.prolongate(P, np.where(mc, 0.0, uc))
    assert np.abs(uf[mf]).max() < 1e-14
