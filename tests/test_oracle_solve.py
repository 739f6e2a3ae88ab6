"""Pins for the oracle's Jacobi-PCG: agreement with a sparse direct solve of the
brute-force assembled matrix, and the residual criterion."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla
import scipy.sparse as sp

import synth
from oracle import cg, solve, topology
from tests import brute


@pytest.mark.parametrize("p", [1, 2])
def test_dirichlet_poisson_matches_direct_solve(p):
    xyz, cells = synth.kuhn_cube(2, jitter=0.2, seed=0)
    dofs, keys = topology.cg_numbering(cells, p)
    N = keys.shape[0]
    mask = topology.dirichlet_mask(cells, p, keys)
    b = cg.rhs_const(xyz, cells, p, N, dirichlet_mask=mask, dofs=dofs)
    d = cg.diagonal(xyz, cells, p, N, dirichlet_mask=mask, dofs=dofs)
    op = lambda x: cg.apply(xyz, cells, x, p, dirichlet_mask=mask, dofs=dofs)
    x, it, rel = solve.jacobi_pcg(op, d, b, rtol=1e-13)
    assert rel < 1e-12
    # independent direct solve: brute-force matrix with identity rows/cols on the boundary
    A, nodes = brute.assemble_cg(xyz, cells, p)
    X = xyz[keys].mean(axis=1)
    order = [int(np.argmin(np.linalg.norm(nodes - z, axis=1))) for z in X]
    Ac = A[np.ix_(order, order)]
    Ac[mask, :] = 0.0
    Ac[:, mask] = 0.0
    Ac[mask, mask] = 1.0
    xd = spla.spsolve(sp.csr_matrix(Ac), b)
    assert np.allclose(x, xd, atol=1e-11 * np.abs(xd).max())
    # the load vector itself: b_i = int phi_i, so sum over free DoFs of b_i < 1
    assert 0 < b.sum() < 1
