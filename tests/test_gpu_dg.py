"""GPU parity of the SIPG operator (Eq. 2 / Eq. 5) through the C ABI against the FP64 oracle."""
import numpy as np
import pytest

import synth
from oracle import dg, topology
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
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
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


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_config3_dg_p2_48cubed_sampled(prec):
    """DG SIPG P2 on the 48^3 Kuhn cube (663,552 cells, 1,313,280 interior + 27,648 boundary faces):
    256 sampled cells against the oracle evaluated on the sampled cells and their face neighbours."""
    from paper_2509_10226_gb300.fem import FemSpace

    p = 2
    xyz, cells = synth.kuhn_cube(48, jitter=0.2, seed=synth.SEEDS["jitter"])
    sp = FemSpace(xyz, cells, kind="dg", degree=p, device=0)
    assert sp.n_dofs == 6635520
    assert (sp.n_interior_faces, sp.n_boundary_faces) == (1313280, 27648)
    u_lib = synth.uniform_vector(sp.n_dofs, synth.SEEDS["u"])
    y_user = lib_to_user(sp, to_host(sp.apply(to_dev(u_lib, prec), prec=prec)))
    u_user = lib_to_user(sp, u_lib)
    nd = sp.dofs_per_cell
    rng = np.random.default_rng(12)
    sample = rng.choice(cells.shape[0], 256, replace=False)
    interior, _ = topology.faces(cells)
    pairs = interior[:, :, 0]
    hit = np.isin(pairs, sample).any(axis=1)
    sub = np.unique(np.concatenate([sample, pairs[hit].ravel()]))
    u_sub = u_user.reshape(-1, nd)[sub].ravel()
    y_sub = dg.apply(xyz, cells[sub], u_sub, p).reshape(-1, nd)
    y_ref = y_sub[np.searchsorted(sub, sample)]
    assert_close(y_user.reshape(-1, nd)[sample], y_ref, prec, "config3 sampled")
