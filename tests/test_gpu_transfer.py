"""GPU parity of the p-transfer (prolongation and restriction between CG spaces of two degrees on
one mesh) against the FP64 oracle, with and without Dirichlet constraints, and the Galerkin
identity P^T A_fine P u = A_coarse u through the library."""
import numpy as np
import pytest

import synth
from oracle import topology, transfer
from tests.gpu_util import assert_close, require_gpu, to_dev, to_host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


def spaces(pf, pc, dirichlet, n=4):
    from paper_2509_10226_gb300.fem import FemSpace, Transfer

    xyz, cells = synth.kuhn_cube(n, jitter=0.2, seed=2)
    f = FemSpace(xyz, cells, kind="cg", degree=pf, dirichlet=dirichlet, device=0)
    c = FemSpace(xyz, cells, kind="cg", degree=pc, dirichlet=dirichlet, device=0)
    return xyz, cells, f, c, Transfer(f, c)


@pytest.mark.parametrize("pf,pc", [(2, 1), (3, 1), (3, 2), (4, 1), (4, 2), (4, 3)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("dirichlet", [False, True])
def test_transfer(pf, pc, prec, dirichlet):
    xyz, cells, f, c, t = spaces(pf, pc, dirichlet)
    df, kf = topology.cg_numbering(cells, pf)
    dc, kc = topology.cg_numbering(cells, pc)
    P = transfer.prolongation_matrix(cells, pf, pc, df, dc, kf.shape[0], kc.shape[0])
    mf = topology.dirichlet_mask(cells, pf, kf) if dirichlet else None
    mc = topology.dirichlet_mask(cells, pc, kc) if dirichlet else None
    pfm, pcm = f.dof_permutation(), c.dof_permutation()
    uc = synth.uniform_vector(c.n_dofs, 1)
    uf = to_host(t.prolongate(to_dev(uc[pcm], prec), prec=prec))
    ref = transfer.prolongate(P, uc if mc is None else np.where(mc, 0.0, uc), mf)
    assert_close(uf, ref[pfm], prec, "prolongate")
    rf = synth.uniform_vector(f.n_dofs, 2)
    rc = to_host(t.restrict(to_dev(rf[pfm], prec), prec=prec))
    assert_close(rc, transfer.restrict(P, rf, mf, mc)[pcm], prec, "restrict")


def test_galerkin_identity_through_the_library():
    xyz, cells, f, c, t = spaces(3, 1, False, n=3)
    u = to_dev(synth.uniform_vector(c.n_dofs, 3), "fp64")
    lhs = t.restrict(f.apply(t.prolongate(u)))
    rhs = c.apply(u)
    assert_close(to_host(lhs), to_host(rhs), "fp64", "P^T A P = A_c")
