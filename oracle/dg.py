"""Symmetric interior penalty (SIPG) DG Laplace operator, Eq. 2 evaluated as Eq. 5.

    a_DG(u, v) = (grad u, grad v)_Omega_h - ({{d_n v}}, [[u]]) - ([[v]], {{d_n u}} - tau [[u]])

with [[.]] = (.)^- - (.)^+ and {{.}} = ((.)^- + (.)^+)/2 on interior faces.  The
operator applied to a vector is the cell loop of Eq. 3 on per-cell DoFs plus a
loop over faces (Eq. 5).

Readings where the paper is silent (Sec. 2.1 says only that the boundary is
"suitably modified"):
  * face owner: the minus side K^- is the adjacent cell with the smaller user id;
    n is the unit normal pointing out of K^-;
  * boundary faces: homogeneous Dirichlet by the mirror principle u^+ = -u^-,
    grad u^+ = grad u^-; only the minus test function exists there;
  * penalty: tau_F = eta / h_F, eta = (p+1)(p+3) by default, and
    h_F = min over the adjacent cells K of 3|K|/|F| (the height of K over F).

Face terms are evaluated directly: each face quadrature point is mapped to
physical space through K^-'s face and pulled back into both adjacent cells by
inverting their affine maps.  No orientation tables are used.
"""
from __future__ import annotations

import numpy as np

from . import basis, quadrature, topology
from .cg import element_apply, geometry

CHUNK = 16384


def default_penalty(p: int) -> float:
    return float((p + 1) * (p + 3))


def _side_eval(xyz, cells, c, x, p):
    """Values [F,q,ndof] and physical gradients [F,q,ndof,3] of cell c's shape functions at points x [F,q,3]."""
    _, det, Jinv = geometry(xyz, cells[c])
    X0 = xyz[cells[c, 0]]
    xhat = np.einsum("fak,fqk->fqa", Jinv, x - X0[:, None, :])
    vals = basis.values(p, xhat)
    gref = basis.gradients(p, xhat)
    gphys = np.einsum("fak,fqja->fqjk", Jinv, gref)
    return vals, gphys, np.abs(det) / 6.0


def _face_geometry(xyz, cells, c, m, p):
    """Points [F,q,3], weights w_q*2|F| [F,q], outward unit normal of cell c [F,3], area [F]."""
    fv = np.array(topology.FACE_VERTICES, dtype=np.int64)[m]      # F,3 local vertex ids
    V = xyz[cells[c[:, None], fv]]                                 # F,3,3
    xq2, wq2 = quadrature.tri_rule(p)
    lam = np.stack([1.0 - xq2[:, 0] - xq2[:, 1], xq2[:, 0], xq2[:, 1]], axis=1)  # q,3
    pts = np.einsum("qi,fik->fqk", lam, V)
    cr = np.cross(V[:, 1] - V[:, 0], V[:, 2] - V[:, 0])
    two_area = np.linalg.norm(cr, axis=1)
    n = cr / two_area[:, None]
    opp = xyz[cells[c, m]]
    flip = np.einsum("fk,fk->f", n, opp - V[:, 0]) > 0
    n[flip] *= -1.0
    return pts, wq2[None, :] * two_area[:, None], n, 0.5 * two_area


def apply(xyz, cells, u, p, penalty_factor=None, include_boundary=True, modified=False):
    """y = A_DG u with u in canonical DG numbering (cell-major, e * ndof + j).  modified selects the
    cell rule of Sec. 3.3 for the cell term; face integrals keep the standard rule."""
    xyz = np.asarray(xyz, dtype=np.float64)
    cells = np.asarray(cells, dtype=np.int64)
    eta = default_penalty(p) if penalty_factor is None else float(penalty_factor)
    nd = basis.num_dofs(p)
    C = cells.shape[0]
    ue = np.asarray(u, dtype=np.float64).reshape(C, nd)
    y = element_apply(xyz, cells, ue, p, modified=modified)  # cell term, Eq. 3 on discontinuous DoFs
    interior, boundary = topology.faces(cells)

    for s in range(0, interior.shape[0], CHUNK):
        f = interior[s:s + CHUNK]
        cm, fm, cp = f[:, 0, 0], f[:, 0, 1], f[:, 1, 0]
        pts, W, n, area = _face_geometry(xyz, cells, cm, fm, p)
        vm, gm, volm = _side_eval(xyz, cells, cm, pts, p)
        vp, gp, volp = _side_eval(xyz, cells, cp, pts, p)
        tau = eta / np.minimum(3.0 * volm / area, 3.0 * volp / area)
        um = np.einsum("fqj,fj->fq", vm, ue[cm])
        up = np.einsum("fqj,fj->fq", vp, ue[cp])
        dnm_phi = np.einsum("fqjk,fk->fqj", gm, n)
        dnp_phi = np.einsum("fqjk,fk->fqj", gp, n)
        dnm = np.einsum("fqj,fj->fq", dnm_phi, ue[cm])
        dnp = np.einsum("fqj,fj->fq", dnp_phi, ue[cp])
        jump = um - up
        avg_dn = 0.5 * (dnm + dnp)
        flux = avg_dn - tau[:, None] * jump
        cm_contrib = np.einsum("fq,fqj->fj", W * (-0.5 * jump), dnm_phi) + np.einsum("fq,fqj->fj", W * (-flux), vm)
        cp_contrib = np.einsum("fq,fqj->fj", W * (-0.5 * jump), dnp_phi) + np.einsum("fq,fqj->fj", W * (+flux), vp)
        np.add.at(y, cm, cm_contrib)
        np.add.at(y, cp, cp_contrib)

    if include_boundary:
        for s in range(0, boundary.shape[0], CHUNK):
            f = boundary[s:s + CHUNK]
            cm, fm = f[:, 0], f[:, 1]
            pts, W, n, area = _face_geometry(xyz, cells, cm, fm, p)
            vm, gm, volm = _side_eval(xyz, cells, cm, pts, p)
            tau = eta / (3.0 * volm / area)
            um = np.einsum("fqj,fj->fq", vm, ue[cm])
            dnm_phi = np.einsum("fqjk,fk->fqj", gm, n)
            dnm = np.einsum("fqj,fj->fq", dnm_phi, ue[cm])
            # mirror principle: u+ = -u-, grad u+ = grad u-
            jump = 2.0 * um
            avg_dn = dnm
            flux = avg_dn - tau[:, None] * jump
            contrib = np.einsum("fq,fqj->fj", W * (-0.5 * jump), dnm_phi) + np.einsum("fq,fqj->fj", W * (-flux), vm)
            np.add.at(y, cm, contrib)
    return y.reshape(-1)
