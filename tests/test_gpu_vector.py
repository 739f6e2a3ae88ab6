"""GPU parity of the vector Laplacian (independent components, components-batched on the FMA units,
one pass per component on the tensor cores) against the FP64 oracle."""
import numpy as np
import pytest

import synth
from oracle import cg, topology
from tests.gpu_util import assert_close, require_gpu, to_dev, to_host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


@pytest.mark.parametrize("p", [1, 3])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32", "bf16"])
@pytest.mark.parametrize("dirichlet", [False, True])
def test_vector_apply(p, prec, dirichlet):
    from paper_2509_10226_gb300.fem import FemSpace

    xyz, cells = synth.kuhn_cube(4, jitter=0.2, seed=p)
    sp = FemSpace(xyz, cells, kind="cg", degree=p, dirichlet=dirichlet, device=0)
    dofs, keys = topology.cg_numbering(cells, p)
    mask = topology.dirichlet_mask(cells, p, keys) if dirichlet else None
    perm = sp.dof_permutation()
    U = np.stack([synth.uniform_vector(sp.n_dofs, s) for s in (1, 2, 3)])
    Y = to_host(sp.apply_vector(to_dev(U[:, perm], prec), prec=prec))
    Y_ref = cg.apply_vector(xyz, cells, U, p, dirichlet_mask=mask, dofs=dofs)[:, perm]
    for c in range(3):
        assert_close(Y[c], Y_ref[c], prec, f"component {c}")


def test_vector_apply_colour_mode():
    from paper_2509_10226_gb300.fem import FemSpace

    p = 2
    xyz, cells = synth.kuhn_cube(4, jitter=0.2, seed=7)
    sp = FemSpace(xyz, cells, kind="cg", degree=p, device=0, scatter="colour")
    dofs, keys = topology.cg_numbering(cells, p)
    perm = sp.dof_permutation()
    U = np.stack([synth.uniform_vector(sp.n_dofs, s) for s in (1, 2)])
    Y = to_host(sp.apply_vector(to_dev(U[:, perm], "fp64"), prec="fp64"))
    Y_ref = cg.apply_vector(xyz, cells, U, p, dofs=dofs)[:, perm]
    for c in range(2):
        assert_close(Y[c], Y_ref[c], "fp64", f"component {c}")
