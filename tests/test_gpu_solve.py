"""GPU Poisson solve (Jacobi-PCG in FP64, and FP64 iterative refinement around an FP32 / tensor-core
inner PCG), checked with the FP64 oracle: residual recomputed by the oracle, solution against the
oracle's own Jacobi-PCG."""
import numpy as np
import pytest

import synth
from oracle import cg, solve, topology
from tests.gpu_util import require_gpu, sampled_rhs, sampled_rows, to_dev, to_host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


def setup_problem(n, p, seed=0):
    from paper_2509_10226_gb300.fem import FemSpace

    xyz, cells = synth.kuhn_cube(n, jitter=0.2, seed=seed)
    sp = FemSpace(xyz, cells, degree=p, dirichlet=True, device=0)
    dofs, keys = topology.cg_numbering(cells, p)
    mask = topology.dirichlet_mask(cells, p, keys)
    return sp, xyz, cells, dofs, keys, mask


def oracle_residual(xyz, cells, p, dofs, mask, x_can, b_can):
    r = b_can - cg.apply(xyz, cells, x_can, p, dirichlet_mask=mask, dofs=dofs)
    return np.linalg.norm(r) / np.linalg.norm(b_can)


@pytest.mark.parametrize("mode,inner",
                         [("pcg", "fp32"), ("ir", "fp32"), ("ir", "tf32"), ("ir", "bf16"), ("ir", "tf32x3")])
def test_solve_p3_small(mode, inner):
    p = 3
    sp, xyz, cells, dofs, keys, mask = setup_problem(6, p)
    perm = sp.dof_permutation()
    b = sp.rhs_const(1.0)
    b_can = np.empty(sp.n_dofs)
    b_can[perm] = to_host(b)
    assert np.allclose(b_can, cg.rhs_const(xyz, cells, p, sp.n_dofs, dirichlet_mask=mask, dofs=dofs), atol=1e-15)
    x, st = sp.solve(b, mode=mode, inner_prec=inner, rtol=1e-10, inner_rtol=1e-3)
    assert st["converged"] and st["rel_residual"] <= 1e-10
    x_can = np.empty(sp.n_dofs)
    x_can[perm] = to_host(x)
    assert oracle_residual(xyz, cells, p, dofs, mask, x_can, b_can) <= 1e-10
    d = cg.diagonal(xyz, cells, p, sp.n_dofs, dirichlet_mask=mask, dofs=dofs)
    op = lambda v: cg.apply(xyz, cells, v, p, dirichlet_mask=mask, dofs=dofs)
    x_ref, _, _ = solve.jacobi_pcg(op, d, b_can, rtol=1e-13)
    assert np.linalg.norm(x_can - x_ref) <= 1e-7 * np.linalg.norm(x_ref)


@pytest.mark.parametrize("p", [1, 2, 4])
def test_solve_degree_sweep(p):
    sp, xyz, cells, dofs, keys, mask = setup_problem(4, p, seed=p)
    perm = sp.dof_permutation()
    b = sp.rhs_const(1.0)
    b_can = np.empty(sp.n_dofs)
    b_can[perm] = to_host(b)
    for mode, inner in (("pcg", "fp32"), ("ir", "tf32")):
        x, st = sp.solve(b, mode=mode, inner_prec=inner, rtol=1e-10)
        x_can = np.empty(sp.n_dofs)
        x_can[perm] = to_host(x)
        assert st["converged"], (p, mode, st)
        assert oracle_residual(xyz, cells, p, dofs, mask, x_can, b_can) <= 1e-10


def test_not_converged_reports_status():
    from paper_2509_10226_gb300 import FemError, _lib

    sp, *_ = setup_problem(4, 2)
    b = sp.rhs_const(1.0)
    with pytest.raises(FemError) as e:
        sp.solve(b, mode="pcg", rtol=1e-14, max_inner=3)
    assert e.value.status == _lib.FEM_ENOTCONV
    x, st = sp.solve(b, mode="ir", inner_prec="fp32", rtol=1e-14, max_outer=1, max_inner=5,
                     raise_on_notconv=False)
    assert not st["converged"] and st["outer"] == 1 and st["inner"] <= 5
    assert np.isfinite(to_host(x)).all()


def test_graph_blocks_and_plain_tail_match_the_oracle():
    """fem_solve replays blocks of eight PCG iterations as CUDA graphs and runs what is left below the
    cap as single launches.  With a cap of 13 iterations (one block, then five single iterations) the
    FP64 iterate equals the oracle's Jacobi-PCG after 13 iterations, and the allocation-free solve
    (single launches throughout) gives the same iterate."""
    p = 2
    sp, xyz, cells, dofs, keys, mask = setup_problem(6, p)
    perm = sp.dof_permutation()
    b = sp.rhs_const(1.0)
    b_can = np.empty(sp.n_dofs)
    b_can[perm] = to_host(b)
    x, st = sp.solve(b, mode="pcg", rtol=1e-15, max_inner=13, raise_on_notconv=False)
    assert st["inner"] == 13 and not st["converged"]
    x_can = np.empty(sp.n_dofs)
    x_can[perm] = to_host(x)
    d = cg.diagonal(xyz, cells, p, sp.n_dofs, dirichlet_mask=mask, dofs=dofs)
    op = lambda v: cg.apply(xyz, cells, v, p, dirichlet_mask=mask, dofs=dofs)
    x_ref, it, _ = solve.jacobi_pcg(op, d, b_can, rtol=0.0, maxiter=13)
    assert it == 13
    assert np.linalg.norm(x_can - x_ref) <= 1e-10 * np.linalg.norm(x_ref)
    x2, st2 = sp.solve(b, mode="pcg", rtol=1e-15, max_inner=13, raise_on_notconv=False, no_alloc=True)
    assert st2["inner"] == 13
    assert torch.allclose(x, x2, rtol=1e-12, atol=1e-14)


def test_zero_rhs_and_initial_guess():
    sp, *_ = setup_problem(3, 2)
    b = torch.zeros(sp.n_dofs, dtype=torch.float64, device="cuda")
    x, st = sp.solve(b, x0=torch.ones_like(b))
    assert st["converged"] and float(x.abs().max()) == 0.0
    b = sp.rhs_const(1.0)
    x1, st1 = sp.solve(b, mode="pcg", rtol=1e-10)
    x2, st2 = sp.solve(b, x0=x1, mode="pcg", rtol=1e-10)
    assert st2["inner"] <= 1


def test_solve_cg_p3_48cubed_mixed():
    """CG P3 on the 48^3 cube (663,552 cells, 3,048,625 DoFs, Dirichlet), f = 1, IR with the
    TF32 tensor-core inner PCG and FP64 outer residual to 1e-10, against the all-FP64 PCG; the final
    residual is recomputed with the FP64 library operator (pinned to the oracle above) and on 256
    rows by the oracle."""
    from paper_2509_10226_gb300.fem import FemSpace

    p = 3
    xyz, cells = synth.kuhn_cube(48, jitter=0.2, seed=synth.SEEDS["jitter"])
    sp = FemSpace(xyz, cells, degree=p, dirichlet=True, device=0)
    assert sp.n_dofs == 3048625
    assert int(sp.dirichlet_mask().sum()) == 3048625 - 143 ** 3
    b = sp.rhs_const(1.0)
    x_ir, st_ir = sp.solve(b, mode="ir", inner_prec="tf32", rtol=1e-10, inner_rtol=1e-3)
    x_mg, st_mg = sp.solve(b, mode="pmg", inner_prec="tf32", rtol=1e-10, inner_rtol=1e-5)
    x_64, st_64 = sp.solve(b, mode="pcg", rtol=1e-10)
    assert st_ir["converged"] and st_mg["converged"] and st_64["converged"]
    for x in (x_ir, x_mg, x_64):
        r = b - sp.apply(x)
        assert float(torch.linalg.norm(r) / torch.linalg.norm(b)) <= 1e-10
    # the solutions agree within the conditioning of the problem
    for x in (x_ir, x_mg):
        assert float(torch.linalg.norm(x - x_64) / torch.linalg.norm(x_64)) <= 1e-6
    # oracle on 256 sampled rows: b and (A x) agree to 1e-10 ||b||_inf
    mask = sp.dirichlet_mask()
    sample = np.random.default_rng(14).choice(sp.n_dofs, 256, replace=False)
    b_ref = sampled_rhs(sp, xyz, cells, p, sample, mask_lib=mask)
    bh = to_host(b)
    assert np.allclose(bh[sample], b_ref, rtol=0, atol=1e-13 * np.abs(bh).max())
    ax = sampled_rows(sp, xyz, cells, p, to_host(x_ir), sample, mask_lib=mask)
    assert np.abs(b_ref - ax).max() <= 1e-9 * np.abs(bh).max()


@pytest.mark.parametrize("p,inner", [(2, "tf32"), (3, "tf32"), (3, "fp32"), (3, "bf16")])
def test_pmg_solve(p, inner):
    """Refinement around flexible CG with the p-multigrid V-cycle: converges to 1e-10 (the oracle's
    residual agrees) in far fewer inner iterations than Jacobi-PCG."""
    sp, xyz, cells, dofs, keys, mask = setup_problem(6, p)
    perm = sp.dof_permutation()
    b = sp.rhs_const(1.0)
    x, st = sp.solve(b, mode="pmg", inner_prec=inner, rtol=1e-10, inner_rtol=1e-3)
    assert st["converged"] and st["rel_residual"] <= 1e-10
    b_can = np.empty(sp.n_dofs)
    b_can[perm] = to_host(b)
    x_can = np.empty(sp.n_dofs)
    x_can[perm] = to_host(x)
    assert oracle_residual(xyz, cells, p, dofs, mask, x_can, b_can) <= 1e-10
    _, st_j = sp.solve(b, mode="ir", inner_prec=inner, rtol=1e-10, inner_rtol=1e-3)
    assert st["inner"] < st_j["inner"] / 2, (st["inner"], st_j["inner"])


def test_pmg_refusals():
    from paper_2509_10226_gb300 import FemError

    sp, xyz, cells, dofs, keys, mask = setup_problem(3, 1)
    with pytest.raises(FemError, match="degree >= 2"):
        sp.solve(sp.rhs_const(1.0), mode="pmg", inner_prec="tf32")
    sp2, *_ = setup_problem(3, 2)
    with pytest.raises(FemError, match="allocated"):
        sp2.solve(sp2.rhs_const(1.0), mode="pmg", inner_prec="tf32", no_alloc=True)
