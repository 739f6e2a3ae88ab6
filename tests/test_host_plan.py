"""Host-side plan of the library (device = -1, no GPU needed): numbering against
the oracle's canonical numbering (bit-exact), Dirichlet set, reordering and the
error paths of fem_create."""
import numpy as np
import pytest

import synth
from oracle import topology
from paper_2509_10226_gb300 import FemError, _lib
from paper_2509_10226_gb300.fem import FemSpace


def space(xyz, cells, **kw):
    kw.setdefault("device", -1)
    return FemSpace(xyz, cells, **kw)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("reorder", [True, False])
def test_cg_numbering_matches_oracle(p, reorder):
    xyz, cells = synth.kuhn_cube(3, jitter=0.2, seed=0)
    xyz, cells, _ = synth.shuffle_mesh(xyz, cells, seed=4)
    sp = space(xyz, cells, degree=p, reorder=reorder)
    dofs, keys = topology.cg_numbering(cells, p)
    assert sp.n_dofs == keys.shape[0]
    assert sp.n_qpoints == [5, 15, 35, 70][p - 1]
    perm = sp.dof_permutation()
    assert np.array_equal(np.sort(perm), np.arange(sp.n_dofs))
    lib_keys = sp.dof_keys()
    assert np.array_equal(lib_keys, keys[perm])
    cperm = sp.cell_permutation()
    assert np.array_equal(np.sort(cperm), np.arange(cells.shape[0]))
    if not reorder:
        assert np.array_equal(cperm, np.arange(cells.shape[0]))


@pytest.mark.parametrize("p", [1, 2, 3])
def test_dirichlet_mask_matches_oracle(p):
    xyz, cells = synth.kuhn_cube(3, jitter=0.2, seed=1)
    sp = space(xyz, cells, degree=p, dirichlet=True)
    dofs, keys = topology.cg_numbering(cells, p)
    mask = topology.dirichlet_mask(cells, p, keys)
    assert np.array_equal(sp.dirichlet_mask(), mask[sp.dof_permutation()])


def test_dg_numbering_and_faces():
    p = 2
    xyz, cells = synth.kuhn_cube(3, jitter=0.2, seed=2)
    sp = space(xyz, cells, kind="dg", degree=p)
    nd = 10
    assert sp.n_dofs == cells.shape[0] * nd
    cperm = sp.cell_permutation()
    perm = sp.dof_permutation()
    expect = (cperm[:, None].astype(np.int64) * nd + np.arange(nd)[None, :]).ravel()
    assert np.array_equal(perm, expect)
    interior, boundary = topology.faces(cells)
    assert sp.n_interior_faces == interior.shape[0]
    assert sp.n_boundary_faces == boundary.shape[0]


@pytest.mark.parametrize("p", [1, 2, 3])
def test_dof_coordinates(p):
    """CG: on the unjittered Kuhn cube the nodes are exactly the (p n + 1)^3 lattice (each once);
    on a jittered, shuffled mesh each node is the mean of its key's vertices.  DG: the nodes of
    each cell are its barycentric points beta / p in the user's vertex order."""
    from oracle import basis

    n = 3
    xyz, cells = synth.kuhn_cube(n, jitter=0.0, seed=0)
    X = space(xyz, cells, degree=p).dof_coordinates()
    lat = np.rint(X * p * n)
    assert np.abs(X * p * n - lat).max() < 1e-9
    codes = (lat[:, 0] * (p * n + 1) + lat[:, 1]) * (p * n + 1) + lat[:, 2]
    assert np.array_equal(np.sort(codes), np.arange((p * n + 1) ** 3))
    xyz, cells = synth.kuhn_cube(n, jitter=0.2, seed=2)
    xyz, cells, _ = synth.shuffle_mesh(xyz, cells, seed=4)
    sp = space(xyz, cells, degree=p)
    assert np.allclose(sp.dof_coordinates(), xyz[sp.dof_keys()].mean(axis=1), rtol=0, atol=1e-14)
    sp = space(xyz, cells, kind="dg", degree=p)
    nodes = np.array(basis.nodes_beta(p), dtype=np.float64) / p
    expect = np.einsum("nk,ckd->cnd", nodes, xyz[cells[sp.cell_permutation()]]).reshape(-1, 3)
    assert np.allclose(sp.dof_coordinates(), expect, rtol=0, atol=1e-14)


@pytest.mark.parametrize("p", [1, 3])
def test_colouring_is_valid(p):
    """Colour mode: the colour ranges cover every library cell once and no two cells of one colour
    share a global DoF (checked with the oracle's numbering of the user cells)."""
    xyz, cells = synth.kuhn_cube(4, jitter=0.2, seed=3)
    sp = space(xyz, cells, degree=p, scatter="colour")
    starts = sp.colour_starts()
    assert starts[0] == 0 and starts[-1] == cells.shape[0] and np.all(np.diff(starts) > 0)
    dofs, _ = topology.cg_numbering(cells, p)
    cperm = sp.cell_permutation()
    for k in range(len(starts) - 1):
        d = dofs[cperm[starts[k]:starts[k + 1]]].ravel()
        assert np.unique(d).size == d.size, f"colour {k} shares a DoF"
    assert len(starts) - 1 < 256
    assert space(xyz, cells, degree=p).colour_starts().size == 0


def test_morton_reorder_improves_locality():
    """Reordering a shuffled mesh makes the cells of a 128-cell batch share vertices (Sec. 2.5)."""
    xyz, cells = synth.kuhn_cube(8, jitter=0.2, seed=0)
    xyz, cells, _ = synth.shuffle_mesh(xyz, cells, seed=4)

    def distinct_vertices_per_batch(order):
        c = cells[order]
        nb = len(c) // 128
        return np.mean([len(np.unique(c[128 * b:128 * (b + 1)])) for b in range(nb)])

    sp_m = space(xyz, cells, degree=1, reorder=True)
    sp_n = space(xyz, cells, degree=1, reorder=False)
    morton = distinct_vertices_per_batch(sp_m.cell_permutation())
    shuffled = distinct_vertices_per_batch(sp_n.cell_permutation())
    assert morton < 0.4 * shuffled, (morton, shuffled)


def test_errors():
    xyz, cells = synth.kuhn_cube(2)
    bad = cells.copy()
    bad[3, 2] = xyz.shape[0] + 5
    with pytest.raises(FemError) as e:
        space(xyz, bad, degree=1)
    assert e.value.status == _lib.FEM_EMESH
    flat = cells.copy()
    flat[0] = [0, 1, 2, 2]
    with pytest.raises(FemError) as e:
        space(xyz, flat, degree=1)
    assert e.value.status == _lib.FEM_EMESH
    with pytest.raises(FemError) as e:
        space(xyz, cells, degree=5)
    assert e.value.status == _lib.FEM_EUNSUPPORTED
    # a face shared by three cells
    extra = np.vstack([cells, cells[:1]])
    with pytest.raises(FemError) as e:
        space(xyz, extra, degree=1)
    assert e.value.status == _lib.FEM_EMESH
    with pytest.raises(FemError) as e:
        space(xyz, cells, kind="dg", degree=1, dirichlet=True)
    assert e.value.status == _lib.FEM_EINVAL


def test_host_only_plan_rejects_device_calls():
    import torch

    xyz, cells = synth.kuhn_cube(2)
    sp = space(xyz, cells, degree=1)
    L = _lib.lib()
    assert L.fem_apply(sp._h, 0, 1, 2, None, None) == _lib.FEM_EINVAL
    assert b"host-only" in L.fem_last_error()


def test_host_only_plan_rejects_host_buffer_and_diagnostic_calls():
    import ctypes

    xyz, cells = synth.kuhn_cube(2)
    sp = space(xyz, cells, degree=1)
    L = _lib.lib()
    u = np.zeros(sp.n_dofs, dtype=np.float32)
    ptrs = (ctypes.c_void_p * 1)(u.ctypes.data)
    assert L.fem_apply_host(sp._h, _lib.FEM_FP32, 1, ptrs, ptrs) == _lib.FEM_EINVAL
    assert b"host-only" in L.fem_last_error()
    waited = (ctypes.c_int64 * 2)()
    assert L.fem_selftest_wait(sp._h, 1000000, waited) == _lib.FEM_EINVAL
    assert b"host-only" in L.fem_last_error()
    # argument checks come before any device work as well
    assert L.fem_apply_host(None, _lib.FEM_FP32, 1, ptrs, ptrs) == _lib.FEM_EINVAL


def test_apply_host_binding_checks_arguments_before_the_call():
    import torch

    xyz, cells = synth.kuhn_cube(2)
    sp = space(xyz, cells, degree=1)
    good = torch.zeros(sp.n_dofs, dtype=torch.float32)
    with pytest.raises(ValueError):
        sp.apply_host([], [], prec="fp32")                      # empty
    with pytest.raises(ValueError):
        sp.apply_host([good, good], [good], prec="fp32")        # lengths differ
    with pytest.raises(ValueError):
        sp.apply_host([good], [good.double()], prec="fp32")     # wrong vector type
    with pytest.raises(ValueError):
        sp.apply_host([good[:-1].contiguous()], [good], prec="fp32")  # wrong length
    with pytest.raises(ValueError):
        sp.apply_host([torch.zeros(2 * sp.n_dofs)[::2]], [good], prec="fp32")  # not contiguous
    # well-formed arguments reach the library, which refuses a host-only context
    with pytest.raises(FemError) as e:
        sp.apply_host([good], [good], prec="fp32")
    assert e.value.status == _lib.FEM_EINVAL


def test_empty_and_oversized_meshes_are_rejected():
    xyz, cells = synth.kuhn_cube(1)
    for kind in ("cg", "dg"):
        with pytest.raises(FemError) as e:
            space(xyz, np.zeros((0, 4), dtype=np.int32), kind=kind, degree=2)
        assert e.value.status == _lib.FEM_EINVAL
    with pytest.raises(FemError) as e:
        space(np.zeros((0, 3)), np.zeros((0, 4), dtype=np.int32), degree=1)
    assert e.value.status == _lib.FEM_EINVAL
    # a cell count above the documented limit is refused before any array is read
    import ctypes
    desc = _lib.MeshDesc(4, xyz.ctypes.data, 1 << 25, cells.ctypes.data, None)
    sd = _lib.SpaceDesc(_lib.FEM_CG, 1, 0, 1, 0.0, -1, 0, 0)
    h = ctypes.c_void_p()
    assert _lib.lib().fem_create(ctypes.byref(desc), ctypes.byref(sd), ctypes.byref(h)) == _lib.FEM_EINVAL
