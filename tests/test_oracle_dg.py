"""Pins for the oracle's SIPG operator (Eq. 2 evaluated as Eq. 5): symmetry,
consistency on continuous fields, the Galerkin identity with the continuous
operator, and closed forms of the penalty terms computed here from face areas
and cell heights."""
import numpy as np
import pytest

import synth
from oracle import cg, dg, topology


def mesh(n=2, seed=0):
    return synth.kuhn_cube(n, jitter=0.2, seed=seed)


def cg_to_dg(u, dofs):
    return u[dofs].reshape(-1)


def face_table(xyz, cells):
    """Independent face enumeration: {sorted vertex triple: [cells]}, plus per-face area and heights."""
    out = {}
    for c, tet in enumerate(cells):
        for m in range(4):
            tri = tuple(sorted(int(v) for i, v in enumerate(tet) if i != m))
            out.setdefault(tri, []).append(c)
    vol = lambda c: abs(np.linalg.det((xyz[cells[c, 1:]] - xyz[cells[c, 0]]))) / 6
    area = lambda t: 0.5 * np.linalg.norm(np.cross(xyz[t[1]] - xyz[t[0]], xyz[t[2]] - xyz[t[0]]))
    return out, vol, area


@pytest.mark.parametrize("p", [1, 2, 3])
def test_symmetry(p):
    xyz, cells = mesh(2, seed=1)
    nd = (p + 1) * (p + 2) * (p + 3) // 6
    n = cells.shape[0] * nd
    u, v = synth.uniform_vector(n, 1), synth.uniform_vector(n, 2)
    a = v @ dg.apply(xyz, cells, u, p)
    b = u @ dg.apply(xyz, cells, v, p)
    assert abs(a - b) < 1e-12 * abs(a)


@pytest.mark.parametrize("p", [1, 2])
def test_interior_only_consistency(p):
    """Without boundary faces: constants are in the kernel and a linear field has energy |a|^2."""
    xyz, cells = mesh(2, seed=2)
    dofs, keys = topology.cg_numbering(cells, p)
    X = xyz[keys].mean(axis=1)
    one = np.ones(cells.shape[0] * dofs.shape[1])
    assert np.abs(dg.apply(xyz, cells, one, p, include_boundary=False)).max() < 1e-12
    a = np.array([0.5, 0.25, -1.0])
    u = cg_to_dg(X @ a - 0.3, dofs)
    y = dg.apply(xyz, cells, u, p, include_boundary=False)
    assert abs(u @ y - a @ a) < 1e-12


@pytest.mark.parametrize("p", [1, 2, 3])
def test_galerkin_identity_with_cg(p):
    """u, v continuous and zero on the boundary: every face term vanishes, v^T A_DG u = v^T A_CG u."""
    xyz, cells = mesh(2, seed=3)
    dofs, keys = topology.cg_numbering(cells, p)
    mask = topology.dirichlet_mask(cells, p, keys)
    N = keys.shape[0]
    u = np.where(mask, 0.0, synth.uniform_vector(N, 1))
    v = np.where(mask, 0.0, synth.uniform_vector(N, 2))
    lhs = cg_to_dg(v, dofs) @ dg.apply(xyz, cells, cg_to_dg(u, dofs), p)
    rhs = v @ cg.apply(xyz, cells, u, p, dofs=dofs)
    assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(rhs))


@pytest.mark.parametrize("p", [1, 2])
def test_piecewise_constant_penalty_energy(p):
    """u = c_K per cell: only penalty terms remain,
    u^T A u = sum_interior tau_F |F| (c- - c+)^2 + sum_boundary 2 tau_F |F| c^2,
    tau_F = (p+1)(p+3) / min_K (3|K|/|F|)."""
    xyz, cells = mesh(2, seed=4)
    nd = (p + 1) * (p + 2) * (p + 3) // 6
    c = synth.uniform_vector(cells.shape[0], 5)
    u = np.repeat(c, nd)
    y = dg.apply(xyz, cells, u, p)
    faces_, vol, area = face_table(xyz, cells)
    eta = (p + 1) * (p + 3)
    expect = 0.0
    for tri, cs in faces_.items():
        F = area(tri)
        h = min(3 * vol(k) / F for k in cs)
        tau = eta / h
        if len(cs) == 2:
            expect += tau * F * (c[cs[0]] - c[cs[1]]) ** 2
        else:
            expect += 2 * tau * F * c[cs[0]] ** 2
    assert abs(u @ y - expect) < 1e-11 * expect


def test_linear_field_with_boundary_terms():
    """u = a.x + b continuous: u^T A u = |a|^2 - 2 int_dOmega u (a.n) + 2 sum_F tau_F int_F u^2."""
    p = 1
    xyz, cells = mesh(2, seed=5)
    dofs, keys = topology.cg_numbering(cells, p)
    X = xyz[keys].mean(axis=1)
    a, b0 = np.array([0.7, -0.2, 0.4]), 0.3
    u = cg_to_dg(X @ a + b0, dofs)
    y = dg.apply(xyz, cells, u, p)
    faces_, vol, area = face_table(xyz, cells)
    eta = (p + 1) * (p + 3)
    expect = a @ a
    for tri, cs in faces_.items():
        if len(cs) != 1:
            continue
        F = area(tri)
        P = xyz[list(tri)]
        uv = P @ a + b0
        nrm = np.cross(P[1] - P[0], P[2] - P[0])
        nrm /= np.linalg.norm(nrm)
        centre = xyz[cells[cs[0]]].mean(axis=0)
        if nrm @ (P[0] - centre) < 0:
            nrm = -nrm
        int_u = F * uv.mean()
        int_u2 = F / 6.0 * (uv @ uv + uv[0] * uv[1] + uv[1] * uv[2] + uv[2] * uv[0])
        tau = eta / (3 * vol(cs[0]) / F)
        expect += -2.0 * int_u * (a @ nrm) + 2.0 * tau * int_u2
    assert abs(u @ y - expect) < 1e-11 * abs(expect)


def test_face_counts():
    n = 3
    xyz, cells = synth.kuhn_cube(n)
    interior, boundary = topology.faces(cells)
    assert boundary.shape[0] == 6 * 2 * n * n
    assert 4 * cells.shape[0] == 2 * interior.shape[0] + boundary.shape[0]
    assert np.all(interior[:, 0, 0] < interior[:, 1, 0])
