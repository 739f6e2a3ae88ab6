"""GPU parity of the Chebyshev-Jacobi smoother and of the power iteration that tunes it, through the
C ABI, against the FP64 oracle on the same inputs (CG P2 8^3 and P3 6^3, homogeneous Dirichlet)."""
import numpy as np
import pytest

import synth
from oracle import cg, smoother, topology
from tests.gpu_util import TOL, assert_close, require_gpu, to_dev, to_host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


def problem(n, p):
    from paper_2509_10226_gb300.fem import FemSpace

    xyz, cells = synth.kuhn_cube(n, jitter=0.2, seed=1)
    sp = FemSpace(xyz, cells, kind="cg", degree=p, dirichlet=True, device=0)
    dofs, keys = topology.cg_numbering(cells, p)
    mask = topology.dirichlet_mask(cells, p, keys)
    A = lambda v: cg.apply(xyz, cells, v, p, dirichlet_mask=mask, dofs=dofs)
    d = cg.diagonal(xyz, cells, p, keys.shape[0], dirichlet_mask=mask, dofs=dofs)
    return sp, A, d, sp.dof_permutation()


@pytest.mark.parametrize("p,n", [(2, 8), (3, 6)])
def test_lambda_max_fp64(p, n):
    sp, A, d, perm = problem(n, p)
    v0 = synth.uniform_vector(sp.n_dofs, 2)
    lam_ref = smoother.lambda_max(A, d, v0, 30)
    lam = sp.lambda_max(to_dev(d[perm], "fp64"), to_dev(v0[perm], "fp64"), iterations=30, prec="fp64")
    assert abs(lam - lam_ref) <= 1e-10 * lam_ref


# the smoother chains `degree` applies; the stated per-apply tolerance is allowed to add up over them
@pytest.mark.parametrize("p,n", [(2, 8), (3, 6)])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32", "bf16", "tf32x3"])
def test_chebyshev(p, n, prec):
    sp, A, d, perm = problem(n, p)
    degree = 5
    lam = 1.2 * smoother.lambda_max(A, d, synth.uniform_vector(sp.n_dofs, 2), 30)
    b = synth.uniform_vector(sp.n_dofs, 1)
    x0 = 0.1 * synth.uniform_vector(sp.n_dofs, 3)
    x_ref = smoother.chebyshev(A, d, b, x0, degree, lam, lam / 15.0)
    x = to_dev(x0[perm], prec)
    sp.chebyshev(to_dev(b[perm], prec), x, to_dev(d[perm], prec), degree=degree, lam_max=lam, ratio=15.0, prec=prec)
    err = np.linalg.norm(to_host(x) - x_ref[perm]) / np.linalg.norm(x_ref)
    assert err <= (1 if prec == "fp64" else degree) * TOL[prec], err
    # a smoother: the residual drops
    assert np.linalg.norm(b - A(x_ref)) < 0.7 * np.linalg.norm(b - A(x0))
