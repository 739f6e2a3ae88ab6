"""GPU parity of the SIPG operator (Eq. 2 / Eq. 5) through the C ABI against the FP64 oracle."""
import numpy as np
import pytest

import synth
from oracle import dg
from tests.gpu_util import assert_close, require_gpu, to_dev, to_host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


def lib_to_user(sp, v_lib):
    nd = sp.dofs_per_cell
    cperm = sp.cell_permutation()
    out = np.empty_like(v_lib)
    out.reshape(-1, nd)[cperm] = v_lib.reshape(-1, nd)
    return out


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32", "bf16"])
def test_dg_degrees(p, prec):
    from paper_2509_10226_gb300.fem import FemSpace

    xyz, cells = synth.kuhn_cube(3, jitter=0.2, seed=p)
    xyz, cells, _ = synth.shuffle_mesh(xyz, cells, seed=4)
    sp = FemSpace(xyz, cells, kind="dg", degree=p, device=0)
    u_lib = synth.uniform_vector(sp.n_dofs, 1)
    y = lib_to_user(sp, to_host(sp.apply(to_dev(u_lib, prec), prec=prec)))
    y_ref = dg.apply(xyz, cells, lib_to_user(sp, u_lib), p)
    assert_close(y, y_ref, prec, f"dg p={p}")


def test_dg_custom_penalty_and_adjoint():
    from paper_2509_10226_gb300.fem import FemSpace

    p = 2
    xyz, cells = synth.kuhn_cube(4, jitter=0.2, seed=9)
    sp = FemSpace(xyz, cells, kind="dg", degree=p, penalty=30.0, device=0)
    u = synth.uniform_vector(sp.n_dofs, 1)
    v = synth.uniform_vector(sp.n_dofs, 2)
    y = lib_to_user(sp, to_host(sp.apply(to_dev(u, "fp64"))))
    assert_close(y, dg.apply(xyz, cells, lib_to_user(sp, u), p, penalty_factor=30.0), "fp64", "penalty 30")
    at = to_host(sp.apply_adjoint(to_dev(v, "fp64")))
    au = to_host(sp.apply(to_dev(u, "fp64")))
    assert abs(v @ au - at @ u) < 1e-12 * abs(v @ au)


def user_to_lib(sp, v_user):
    nd = sp.dofs_per_cell
    cperm = sp.cell_permutation()
    return np.ascontiguousarray(v_user.reshape(-1, nd)[cperm].ravel())


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32", "bf16"])
def test_dg_p2_48cubed_full_size(prec):
    """DG SIPG P2 on the 48^3 Kuhn cube (663,552 cells, 1,313,280 interior + 27,648 boundary faces),
    the launch the benchmark times: every entry of y against the oracle."""
    from paper_2509_10226_gb300.fem import FemSpace
    from tests import fullsize

    p = 2
    xyz, cells, u_user, y_ref = fullsize.dg_p2_48()
    sp = FemSpace(xyz, cells, kind="dg", degree=p, device=0)
    assert sp.n_dofs == 6635520
    assert (sp.n_interior_faces, sp.n_boundary_faces) == (1313280, 27648)
    y_user = lib_to_user(sp, to_host(sp.apply(to_dev(user_to_lib(sp, u_user), prec), prec=prec)))
    assert_close(y_user, y_ref, prec, "DG P2 48^3")
    assert sp.device_status() == 0


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_dg_tensor_core_ragged_and_status(prec):
    """Tensor-core DG on a mesh whose cell count is not a multiple of 128 and whose face groups
    leave partial tiles, against the oracle; the device status word stays clean; a linear field (no
    jumps, small interior flux) also matches the oracle to the stated tolerance."""
    from paper_2509_10226_gb300.fem import FemSpace

    p = 2
    xyz, cells = synth.kuhn_cube(5, jitter=0.2, seed=3)  # 750 cells
    sp = FemSpace(xyz, cells, kind="dg", degree=p, device=0)
    assert sp.n_cells % 128 != 0
    u = synth.uniform_vector(sp.n_dofs, 1)
    y = to_host(sp.apply(to_dev(u, prec), prec=prec))
    y_ref = dg.apply(xyz, cells, lib_to_user(sp, u), p)
    assert_close(lib_to_user(sp, y), y_ref, prec, "ragged")
    assert sp.device_status() == 0
    # smooth data: u(x) = a . x + b interpolated per cell (continuous across faces)
    from oracle import basis

    nodes = np.array(basis.nodes_beta(p), dtype=np.float64) / p  # barycentric weights of the nodes
    perm = sp.cell_permutation()
    X = np.einsum("nk,ckd->cnd", nodes, xyz[cells[perm]])  # library cell order
    a = np.array([0.3, -1.1, 0.6])
    ul = (X @ a + 0.25).ravel()
    yl = to_host(sp.apply(to_dev(ul, prec), prec=prec))
    yl_ref = dg.apply(xyz, cells, lib_to_user(sp, ul), p)
    assert_close(lib_to_user(sp, yl), yl_ref, prec, "linear field")
