"""GPU parity of the continuous operator (Eq. 3) through the C ABI against the FP64 oracle."""
import numpy as np
import pytest

import synth
from oracle import cg, topology
from tests.gpu_util import TOL, assert_close, require_gpu, sampled_rows, to_dev, to_host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def make(n, p, jitter=0.2, shuffle=False, reorder=True, dirichlet=False, seed=0):
    from paper_2509_10226_gb300.fem import FemSpace

    xyz, cells = synth.kuhn_cube(n, jitter=jitter, seed=seed)
    if shuffle:
        xyz, cells, _ = synth.shuffle_mesh(xyz, cells, seed=4)
    sp = FemSpace(xyz, cells, kind="cg", degree=p, dirichlet=dirichlet, reorder=reorder, device=0)
    dofs, keys = topology.cg_numbering(cells, p)
    return sp, xyz, cells, dofs, keys


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_cg_p2_8cubed(prec):
    """CG P2 on the 8^3 Kuhn cube (3072 cells, 24 tiles), jitter 0.2h, u ~ U[-1,1]."""
    sp, xyz, cells, dofs, keys = make(8, 2)
    assert sp.n_dofs == 4913
    perm = sp.dof_permutation()
    u = synth.uniform_vector(sp.n_dofs, synth.SEEDS["u"])
    y_ref = cg.apply(xyz, cells, u, 2, dofs=dofs)
    y = to_host(sp.apply(to_dev(u[perm], prec), prec=prec))
    assert_close(y, y_ref[perm], prec, "CG P2 8^3")


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("reorder", [True, False])
def test_degrees_shuffled_ragged(p, prec, reorder):
    """3^3 cube = 162 cells: one full tile and a ragged tail of 34 cells; shuffled mesh order."""
    sp, xyz, cells, dofs, keys = make(3, p, shuffle=True, reorder=reorder, seed=p)
    perm = sp.dof_permutation()
    u = synth.uniform_vector(sp.n_dofs, 1)
    y_ref = cg.apply(xyz, cells, u, p, dofs=dofs)
    y = to_host(sp.apply(to_dev(u[perm], prec), prec=prec))
    assert_close(y, y_ref[perm], prec, f"p={p}")


def test_single_cell():
    from paper_2509_10226_gb300.fem import FemSpace

    xyz = np.array([[0, 0, 0], [1, 0.1, 0], [0.2, 1, 0], [0.1, 0.3, 0.9]], dtype=float)
    cells = np.array([[0, 1, 2, 3]], dtype=np.int32)
    for p in (1, 3):
        sp = FemSpace(xyz, cells, degree=p, device=0)
        dofs, keys = topology.cg_numbering(cells, p)
        perm = sp.dof_permutation()
        u = synth.uniform_vector(sp.n_dofs, 2)
        y = to_host(sp.apply(to_dev(u[perm], "fp64")))
        assert_close(y, cg.apply(xyz, cells, u, p, dofs=dofs)[perm], "fp64", "single cell")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_variable_coefficient_adjoint_and_gradient(prec):
    """Variable coefficient on 6^3 (1296 cells): k ~ lognormal(0, 0.5) per quadrature point."""
    p = 2
    sp, xyz, cells, dofs, keys = make(6, p, seed=3)
    perm, cperm = sp.dof_permutation(), sp.cell_permutation()
    nq = sp.n_qpoints
    k_user = synth.lognormal_coefficients((cells.shape[0], nq), synth.SEEDS["k"])
    u = synth.uniform_vector(sp.n_dofs, synth.SEEDS["u"])
    w = synth.uniform_vector(sp.n_dofs, synth.SEEDS["w"])
    kd = to_dev(k_user[cperm].ravel(), prec)
    ud, wd = to_dev(u[perm], prec), to_dev(w[perm], prec)
    y = to_host(sp.apply(ud, k=kd, prec=prec))
    assert_close(y, cg.apply(xyz, cells, u, p, k=k_user, dofs=dofs)[perm], prec, "A(k)u")
    at = to_host(sp.apply_adjoint(wd, k=kd, prec=prec))
    assert_close(at, cg.apply_adjoint(xyz, cells, w, p, k=k_user, dofs=dofs)[perm], prec, "A(k)^T w")
    gu, dk = sp.coeff_grad(ud, wd, k=kd, prec=prec)
    gu_ref, dk_ref = cg.coeff_grad(xyz, cells, u, w, p, k=k_user, dofs=dofs)
    assert_close(to_host(gu), gu_ref[perm], prec, "grad_u")
    assert_close(to_host(dk).reshape(-1, nq), dk_ref[cperm], prec, "dk")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_dirichlet_diag_rhs(prec):
    p = 3
    sp, xyz, cells, dofs, keys = make(4, p, dirichlet=True, seed=5)
    perm = sp.dof_permutation()
    mask = topology.dirichlet_mask(cells, p, keys)
    assert np.array_equal(sp.dirichlet_mask(), mask[perm])
    u = synth.uniform_vector(sp.n_dofs, 1)
    y = to_host(sp.apply(to_dev(u[perm], prec), prec=prec))
    assert_close(y, cg.apply(xyz, cells, u, p, dirichlet_mask=mask, dofs=dofs)[perm], prec, "dirichlet")
    d = to_host(sp.diagonal(prec=prec))
    assert_close(d, cg.diagonal(xyz, cells, p, sp.n_dofs, dirichlet_mask=mask, dofs=dofs)[perm], prec, "diag")
    if prec == "fp64":
        b = to_host(sp.rhs_const(1.0))
        assert_close(b, cg.rhs_const(xyz, cells, p, sp.n_dofs, dirichlet_mask=mask, dofs=dofs)[perm], prec, "rhs")


def test_autograd_function():
    from paper_2509_10226_gb300.fem import fem_apply

    p = 2
    sp, xyz, cells, dofs, keys = make(4, p, seed=6)
    perm, cperm = sp.dof_permutation(), sp.cell_permutation()
    k_user = synth.lognormal_coefficients((cells.shape[0], sp.n_qpoints), 3)
    u = synth.uniform_vector(sp.n_dofs, 1)
    w = synth.uniform_vector(sp.n_dofs, 2)
    ud = to_dev(u[perm], "fp64").requires_grad_(True)
    kd = to_dev(k_user[cperm].ravel(), "fp64").requires_grad_(True)
    wd = to_dev(w[perm], "fp64")
    L = (fem_apply(sp, ud, kd) * wd).sum()
    L.backward()
    gu_ref, dk_ref = cg.coeff_grad(xyz, cells, u, w, p, k=k_user, dofs=dofs)
    assert_close(to_host(ud.grad), gu_ref[perm], "fp64", "autograd u")
    assert_close(to_host(kd.grad).reshape(-1, sp.n_qpoints), dk_ref[cperm], "fp64", "autograd k")
    # central differences of L in one coefficient, through the GPU forward (exact: L is linear in k)
    e = int(np.argmax(np.abs(dk_ref[cperm]).ravel()))
    with torch.no_grad():
        kp, km = kd.detach().clone(), kd.detach().clone()
        kp[e] += 1e-6
        km[e] -= 1e-6
        fd = ((sp.apply(ud.detach(), k=kp) - sp.apply(ud.detach(), k=km)) @ wd).item() / 2e-6
    assert abs(fd - kd.grad[e].item()) < 1e-8 * max(1.0, abs(fd))


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32", "bf16", "tf32x3"])
def test_cg_p3_64cubed_full_size(prec):
    """CG P3 on the 64^3 Kuhn cube (1,572,864 cells, 7,189,057 DoFs), Morton order, the launch the
    benchmark times: every entry of y against the oracle, plus A 1 = 0 and u^T A u = |a|^2."""
    from paper_2509_10226_gb300.fem import FemSpace
    from tests import fullsize

    p = 3
    xyz, cells, u_canon, y_canon = fullsize.cg_p3_64()
    sp = FemSpace(xyz, cells, degree=p, device=0)
    assert sp.n_dofs == 7189057
    perm = sp.dof_permutation()
    y = to_host(sp.apply(to_dev(u_canon[perm], prec), prec=prec))
    assert_close(y, y_canon[perm], prec, "CG P3 64^3")
    # properties that hold at any size
    ones = to_host(sp.apply(to_dev(np.ones(sp.n_dofs), prec), prec=prec))
    term = np.abs(y).max()
    assert np.abs(ones).max() <= 10 * TOL[prec] * term
    X = xyz[sp.dof_keys()].mean(axis=1)
    a = np.array([0.3, -0.5, 0.8])
    lin = X @ a
    ylin = to_host(sp.apply(to_dev(lin, prec), prec=prec))
    assert abs(lin @ ylin - a @ a) <= 10 * TOL[prec] * (a @ a) + 1e-9
    assert sp.device_status() == 0


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("prec", ["tf32", "bf16", "tf32x3"])
def test_tensor_core_degrees_ragged(p, prec):
    """tcgen05 path, p = 1..4, 3^3 cube (one full tile + a 34-cell tail), shuffled input order."""
    sp, xyz, cells, dofs, keys = make(3, p, shuffle=True, seed=p)
    perm = sp.dof_permutation()
    u = synth.uniform_vector(sp.n_dofs, 1)
    if prec == "tf32x3" and p == 4:
        from paper_2509_10226_gb300 import FemError

        with pytest.raises(FemError, match="degrees 1 to 3"):
            sp.apply(to_dev(u[perm], prec), prec=prec)
        return
    y_ref = cg.apply(xyz, cells, u, p, dofs=dofs)
    y = to_host(sp.apply(to_dev(u[perm], prec), prec=prec))
    assert_close(y, y_ref[perm], prec, f"p={p}")
    assert sp.device_status() == 0


@pytest.mark.parametrize("prec", ["tf32", "bf16", "tf32x3"])
def test_tensor_core_p2_8cubed_variable_k_dirichlet(prec):
    """The 8^3 mesh (3072 cells, 24 tiles) on the tensor cores: plain, with k ~ lognormal(0, 0.5), and with
    Dirichlet rows; several tiles per persistent CTA are exercised on the 64^3 test below."""
    p = 2
    sp, xyz, cells, dofs, keys = make(8, p)
    perm, cperm = sp.dof_permutation(), sp.cell_permutation()
    u = synth.uniform_vector(sp.n_dofs, 1)
    y = to_host(sp.apply(to_dev(u[perm], prec), prec=prec))
    assert_close(y, cg.apply(xyz, cells, u, p, dofs=dofs)[perm], prec, "CG P2 8^3")
    k_user = synth.lognormal_coefficients((cells.shape[0], sp.n_qpoints), 3)
    y = to_host(sp.apply(to_dev(u[perm], prec), k=to_dev(k_user[cperm].ravel(), prec), prec=prec))
    assert_close(y, cg.apply(xyz, cells, u, p, k=k_user, dofs=dofs)[perm], prec, "variable k")
    spd, xyz, cells, dofs, keys = make(8, p, dirichlet=True)
    perm = spd.dof_permutation()
    mask = topology.dirichlet_mask(cells, p, keys)
    y = to_host(spd.apply(to_dev(u[perm], prec), prec=prec))
    assert_close(y, cg.apply(xyz, cells, u, p, dirichlet_mask=mask, dofs=dofs)[perm], prec, "dirichlet")
    assert sp.device_status() == 0 and spd.device_status() == 0


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_cg_p2_32cubed_variable_k_backward(prec):
    """CG P2 on the 32^3 cube (196,608 cells), k ~ lognormal(0, 0.5) per quadrature point,
    L = <w, A(k) u>: forward rows, grad_u = A(k)^T w rows and dL/dk on sampled cells against the
    oracle; central differences of L in k through the GPU forward."""
    from oracle import cg as ocg
    from paper_2509_10226_gb300.fem import FemSpace, fem_apply

    p = 2
    xyz, cells = synth.kuhn_cube(32, jitter=0.2, seed=synth.SEEDS["jitter"])
    sp = FemSpace(xyz, cells, degree=p, device=0)
    assert (sp.n_cells, sp.n_dofs) == (196608, 274625)
    cperm = sp.cell_permutation()
    nq = sp.n_qpoints
    k_user = synth.lognormal_coefficients((cells.shape[0], nq), synth.SEEDS["k"])
    k_lib = k_user[cperm]
    u = synth.uniform_vector(sp.n_dofs, synth.SEEDS["u"])
    w = synth.uniform_vector(sp.n_dofs, synth.SEEDS["w"])
    dt = torch.float64 if prec == "fp64" else torch.float32
    ud = torch.as_tensor(u, dtype=dt, device="cuda").requires_grad_(True)
    kd = torch.as_tensor(k_lib.ravel(), dtype=dt, device="cuda").requires_grad_(True)
    wd = torch.as_tensor(w, dtype=dt, device="cuda")
    y = fem_apply(sp, ud, kd, prec=prec)
    L = (y * wd).sum()
    L.backward()
    rng = np.random.default_rng(15)
    rows = rng.choice(sp.n_dofs, 256, replace=False)
    assert_close(to_host(y)[rows], sampled_rows(sp, xyz, cells, p, u, rows, k_user=k_user), prec, "A(k)u")
    assert_close(to_host(ud.grad)[rows], sampled_rows(sp, xyz, cells, p, w, rows, k_user=k_user), prec, "grad_u")
    # dL/dk of sampled library cells: the oracle evaluates those cells alone
    from oracle import topology as otop

    lc = rng.choice(sp.n_cells, 256, replace=False)
    uc = cells[cperm[lc]]
    dofs_loc, keys_loc = otop.cg_numbering(uc, p)
    lib_keys = sp.dof_keys()
    from tests.gpu_util import encode_keys

    code = encode_keys(lib_keys, xyz.shape[0])
    order = np.argsort(code)
    lib_of = order[np.searchsorted(code, encode_keys(keys_loc, xyz.shape[0]), sorter=order)]
    _, dk_ref = ocg.coeff_grad(xyz, uc, u[lib_of], w[lib_of], p, k=k_lib[lc], dofs=dofs_loc)
    assert_close(to_host(kd.grad).reshape(-1, nq)[lc], dk_ref, prec, "dL/dk")
    if prec == "fp64":
        e = int(lc[0]) * nq + 3
        with torch.no_grad():
            kp, km = kd.detach().clone(), kd.detach().clone()
            kp[e] += 1e-6
            km[e] -= 1e-6
            fd = ((sp.apply(ud.detach(), k=kp) - sp.apply(ud.detach(), k=km)) @ wd).item() / 2e-6
        assert abs(fd - kd.grad[e].item()) <= 1e-8 * max(1.0, abs(fd))


@pytest.mark.parametrize("p", [2, 3])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_colour_scatter_parity_and_reproducibility(p, prec):
    """Colour mode: parity with the oracle, and bitwise-identical results over repeated applies
    (the atomic mode is not bitwise reproducible in general)."""
    from paper_2509_10226_gb300.fem import FemSpace

    xyz, cells = synth.kuhn_cube(8, jitter=0.2, seed=2)
    sp = FemSpace(xyz, cells, kind="cg", degree=p, device=0, scatter="colour")
    dofs, keys = topology.cg_numbering(cells, p)
    perm = sp.dof_permutation()
    u = synth.uniform_vector(sp.n_dofs, 1)
    ud = to_dev(u[perm], prec)
    y0 = sp.apply(ud, prec=prec).clone()
    assert_close(to_host(y0), cg.apply(xyz, cells, u, p, dofs=dofs)[perm], prec, "colour")
    for _ in range(5):
        assert torch.equal(sp.apply(ud, prec=prec), y0)
    g = sp.apply_adjoint(ud, prec=prec)
    assert torch.equal(g, y0)
