"""GPU parity of the curved-cell operator (second-order geometry, metric per quadrature point,
Sec. 3.2) against the FP64 oracle: apply in every offered precision, diagonal, load vector, an
IR solve, and the combinations that are refused."""
import numpy as np
import pytest

import synth
from oracle import cg, topology
from tests.gpu_util import TOL, assert_close, require_gpu, to_dev, to_host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

AMPLITUDE = 0.05


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


def curved(n, p, dirichlet=False, seed=5):
    from paper_2509_10226_gb300.fem import FemSpace

    xyz, cells = synth.kuhn_cube(n, jitter=0.2, seed=seed)
    nodes = synth.curved_nodes(xyz, cells, AMPLITUDE)
    sp = FemSpace(xyz, cells, kind="cg", degree=p, dirichlet=dirichlet, device=0, cell_nodes=nodes)
    dofs, keys = topology.cg_numbering(cells, p)
    return sp, xyz, cells, nodes, dofs, keys


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32", "bf16"])
def test_curved_apply(p, prec):
    sp, xyz, cells, nodes, dofs, keys = curved(3, p)
    perm = sp.dof_permutation()
    u = synth.uniform_vector(sp.n_dofs, 1)
    y = to_host(sp.apply(to_dev(u[perm], prec), prec=prec))
    assert_close(y, cg.apply(xyz, cells, u, p, dofs=dofs, nodes=nodes)[perm], prec, f"curved p={p}")
    assert sp.device_status() == 0


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_curved_tensor_cores_many_tiles(prec):
    """8^3 cube: 24 tiles, several per warpgroup."""
    p = 3
    sp, xyz, cells, nodes, dofs, keys = curved(8, p)
    perm = sp.dof_permutation()
    u = synth.uniform_vector(sp.n_dofs, 1)
    y = to_host(sp.apply(to_dev(u[perm], prec), prec=prec))
    assert_close(y, cg.apply(xyz, cells, u, p, dofs=dofs, nodes=nodes)[perm], prec, "curved 8^3")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_curved_diagonal_and_rhs(prec):
    p = 2
    sp, xyz, cells, nodes, dofs, keys = curved(4, p)
    perm = sp.dof_permutation()
    d = to_host(sp.diagonal(prec=prec))
    assert_close(d, cg.diagonal(xyz, cells, p, sp.n_dofs, dofs=dofs, nodes=nodes)[perm], prec, "diag")
    b = to_host(sp.rhs_const(1.0))
    assert_close(b, cg.rhs_const(xyz, cells, p, sp.n_dofs, dofs=dofs, nodes=nodes)[perm], "fp64", "rhs")


def test_curved_ir_solve():
    p = 2
    sp, xyz, cells, nodes, dofs, keys = curved(6, p, dirichlet=True)
    mask = topology.dirichlet_mask(cells, p, keys)
    perm = sp.dof_permutation()
    b = sp.rhs_const(1.0)
    x, st = sp.solve(b, mode="ir", inner_prec="tf32", rtol=1e-10, inner_rtol=1e-3)
    assert st["converged"]
    x_can = np.empty(sp.n_dofs)
    x_can[perm] = to_host(x)
    b_can = cg.rhs_const(xyz, cells, p, sp.n_dofs, dirichlet_mask=mask, dofs=dofs, nodes=nodes)
    r = b_can - cg.apply(xyz, cells, x_can, p, dirichlet_mask=mask, dofs=dofs, nodes=nodes)
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b_can)


def test_curved_refusals():
    from paper_2509_10226_gb300 import FemError
    from paper_2509_10226_gb300.fem import FemSpace

    sp, xyz, cells, nodes, dofs, keys = curved(3, 2)
    u = to_dev(np.ones(sp.n_dofs), "tf32")
    k = to_dev(np.ones(sp.n_cells * sp.n_qpoints), "tf32")
    with pytest.raises(FemError):
        sp.apply(u, k=k, prec="tf32")
    with pytest.raises(FemError):
        sp.apply(u, prec="tf32x3")
    with pytest.raises(FemError):
        sp.csr_build()
    with pytest.raises(FemError):
        FemSpace(xyz, cells, kind="dg", degree=2, device=0, cell_nodes=nodes)
