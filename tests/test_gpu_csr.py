"""Assembled CSR comparator (Sec. 3.2) against the oracle and against the matrix-free apply."""
import numpy as np
import pytest

import synth
from oracle import cg, topology
from tests import brute
from tests.gpu_util import assert_close, require_gpu, to_dev, to_host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("dirichlet", [False, True])
def test_csr_matches_oracle(p, dirichlet):
    from paper_2509_10226_gb300.fem import FemSpace

    xyz, cells = synth.kuhn_cube(3, jitter=0.2, seed=p)
    sp = FemSpace(xyz, cells, degree=p, dirichlet=dirichlet, device=0)
    nnz = sp.csr_build()
    dofs, keys = topology.cg_numbering(cells, p)
    mask = topology.dirichlet_mask(cells, p, keys) if dirichlet else None
    perm = sp.dof_permutation()
    u = synth.uniform_vector(sp.n_dofs, 1)
    y_ref = cg.apply(xyz, cells, u, p, dirichlet_mask=mask, dofs=dofs)[perm]
    for prec in ("fp64", "fp32"):
        y = to_host(sp.csr_apply(to_dev(u[perm], prec), prec=prec))
        assert_close(y, y_ref, prec, f"csr p={p}")
    if not dirichlet and p <= 2:
        # stored entries = structurally coupled DoF pairs (two DoFs share a cell)
        A, _ = brute.assemble_cg(xyz, cells, p)
        X = xyz[keys].mean(axis=1)
        pairs = set()
        for c in range(cells.shape[0]):
            d = dofs[c]
            pairs.update((int(a), int(b)) for a in d for b in d)
        assert nnz == len(pairs)


def test_csr_cg_p3_64cubed_full_size():
    """P3 64^3 (314M stored entries): every entry of the FP64 and FP32 CSR SpMV against the oracle's
    matrix-free y = A u (the same operator)."""
    from paper_2509_10226_gb300.fem import FemSpace
    from tests import fullsize

    p = 3
    xyz, cells, u_canon, y_canon = fullsize.cg_p3_64()
    sp = FemSpace(xyz, cells, degree=p, device=0)
    nnz = sp.csr_build()
    assert 40 * sp.n_dofs < nnz < 50 * sp.n_dofs
    perm = sp.dof_permutation()
    for prec in ("fp64", "fp32"):
        y = to_host(sp.csr_apply(to_dev(u_canon[perm], prec), prec=prec))
        assert_close(y, y_canon[perm], prec, "csr CG P3 64^3")
