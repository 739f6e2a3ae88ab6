"""Continuous Galerkin Laplace operator, written as the cell loop of Eq. 3.

    A(u) = sum_e G_e^T E^T D_e E G_e u                               (Eq. 3)

E is the 3 nq x ndof table of reference gradients at the quadrature points
(Eq. 4, row 3i+k holds d_k phi_j(x_i)).  D_e acts at each quadrature point q as
described below Eq. 4 (on curved cells, Sec. 3.2, with the Jacobian of the second-order map taken
at each point): apply the inverse-transpose Jacobian J^-T (reference to
physical gradient), multiply by the quadrature weight times |det J| (and by the
coefficient k_q when one is given), then apply J^-1.  J = [x1-x0 | x2-x0 | x3-x0]
is built from the user's vertex order of each cell.

All arithmetic is FP64.  Cells are processed in chunks only to bound memory;
each cell's contribution is independent of the chunking.
"""
from __future__ import annotations

import numpy as np

from . import basis, quadrature, topology

CHUNK = 16384


def geometry(xyz: np.ndarray, cells: np.ndarray):
    """Affine map data per cell: J [C,3,3], det J [C], J^-1 [C,3,3]."""
    X = np.asarray(xyz, dtype=np.float64)[np.asarray(cells, dtype=np.int64)]  # C,4,3
    J = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], axis=2)  # columns
    det = np.linalg.det(J)
    Jinv = np.linalg.inv(J)
    return J, det, Jinv


def geometry_curved(nodes: np.ndarray, xq: np.ndarray):
    """Per-point geometry of a second-order cell map x(x_hat) = sum_j X_j phi_j(x_hat), phi the P2
    Lagrange basis and X_j [C, 10, 3] its nodes: J [C, nq, 3, 3] with J[c, q, :, k] = d x / d x_hat_k
    at point q, det J [C, nq], J^-1 [C, nq, 3, 3]."""
    G2 = basis.gradients(2, xq)  # [nq, 10, 3]
    J = np.einsum("cjd,qjk->cqdk", np.asarray(nodes, dtype=np.float64), G2)
    return J, np.linalg.det(J), np.linalg.inv(J)


def tables(p: int, modified: bool = False):
    """(x_hat [nq,3], w [nq], E as grad table [nq, ndof, 3], values [nq, ndof]); modified selects the
    cell rule of Sec. 3.3."""
    xq, wq = quadrature.tet_rule(p, modified)
    return xq, wq, basis.gradients(p, xq), basis.values(p, xq)


def _qp_operator(Jinv, det, wq, k, transpose=False):
    """D_e at every quadrature point as explicit 3x3 matrices [C, nq, 3, 3].

    D_q = J^-1 (k_q w_q |det J|) J^-T; with transpose=True its transpose is
    formed explicitly (the adjoint chain of Eq. 3 applies D_e^T).
    """
    scale = wq[None, :] * np.abs(det)[:, None]
    if k is not None:
        scale = scale * k
    JinvT = np.transpose(Jinv, (0, 2, 1))
    D = np.einsum("cab,q,cbd->cqad", Jinv, np.ones(wq.shape[0]), JinvT) * scale[:, :, None, None]
    if transpose:
        D = np.transpose(D, (0, 1, 3, 2))
    return D


def element_apply(xyz, cells, ue, p, k=None, transpose=False, modified=False, nodes=None):
    """Local products y_e = E^T D_e E u_e for every cell; ue [C, ndof] -> [C, ndof].  With nodes
    [C, 10, 3] the cells are curved (second-order map) and J^-T, |det J| are taken per point."""
    xq, wq, G, _ = tables(p, modified)
    C = ue.shape[0]
    out = np.empty_like(ue, dtype=np.float64)
    for s in range(0, C, CHUNK):
        e = slice(s, min(C, s + CHUNK))
        grad_ref = np.einsum("qjk,cj->cqk", G, ue[e])            # E u_e
        if nodes is not None:
            _, detq, Jq = geometry_curved(nodes[e], xq)          # per point
            scale = wq[None, :] * np.abs(detq)
            if k is not None:
                scale = scale * k[e]
            # J^-T, then JxW (and k), then J^-1, point by point; D_q is symmetric, so the adjoint
            # chain is the same
            t = np.einsum("cqak,cqa->cqk", Jq, grad_ref) * scale[:, :, None]
            t_ref = np.einsum("cqak,cqk->cqa", Jq, t)
            out[e] = np.einsum("qjk,cqk->cj", G, t_ref)
            continue
        _, det, Jinv = geometry(xyz, cells[e])
        if not transpose:
            # D_e in the order stated below Eq. 4: J^-T, then JxW (and k), then J^-1
            grad_phys = np.einsum("cak,cqa->cqk", Jinv, grad_ref)  # J^-T g_hat
            scale = wq[None, :] * np.abs(det)[:, None]
            if k is not None:
                scale = scale * k[e]
            t = grad_phys * scale[:, :, None]
            t_ref = np.einsum("cak,cqk->cqa", Jinv, t)            # J^-1 t
        else:
            D = _qp_operator(Jinv, det, wq, None if k is None else k[e], transpose=True)
            t_ref = np.einsum("cqab,cqb->cqa", D, grad_ref)
        out[e] = np.einsum("qjk,cqk->cj", G, t_ref)              # E^T
    return out


def _scatter(dofs, ye, n):
    y = np.zeros(n, dtype=np.float64)
    np.add.at(y, dofs.ravel(), ye.ravel())
    return y


def apply(xyz, cells, u, p, k=None, dirichlet_mask=None, dofs=None, modified=False, nodes=None):
    """y = A(k) u in canonical numbering.

    With a Dirichlet mask P (True = constrained) the operator is P A P + (I - P):
    constrained entries of u are skipped on gather, their rows are identity.
    """
    if dofs is None:
        dofs, _ = topology.cg_numbering(cells, p)
    u = np.asarray(u, dtype=np.float64)
    uu = u if dirichlet_mask is None else np.where(dirichlet_mask, 0.0, u)
    y = _scatter(dofs, element_apply(xyz, cells, uu[dofs], p, k, modified=modified, nodes=nodes), u.shape[0])
    if dirichlet_mask is not None:
        y = np.where(dirichlet_mask, u, y)
    return y


def apply_vector(xyz, cells, U, p, dirichlet_mask=None, dofs=None):
    """Vector Laplacian with independent components (the vector-valued Poisson problem of Sec. 3.1):
    row c of the result is A applied to row c of U [ncomp, N]."""
    return np.stack([apply(xyz, cells, U[c], p, dirichlet_mask=dirichlet_mask, dofs=dofs) for c in range(U.shape[0])])


def apply_adjoint(xyz, cells, g, p, k=None, dirichlet_mask=None, dofs=None, modified=False):
    """A(k)^T g: the transposed chain G_e^T E^T D_e^T E G_e summed over cells."""
    if dofs is None:
        dofs, _ = topology.cg_numbering(cells, p)
    g = np.asarray(g, dtype=np.float64)
    gg = g if dirichlet_mask is None else np.where(dirichlet_mask, 0.0, g)
    out = _scatter(dofs, element_apply(xyz, cells, gg[dofs], p, k, transpose=True, modified=modified), g.shape[0])
    if dirichlet_mask is not None:
        out = np.where(dirichlet_mask, g, out)
    return out


def coeff_grad(xyz, cells, u, g, p, k=None, dofs=None, modified=False):
    """Backward of L = <g, A(k) u>: (dL/du = A(k)^T g, dL/dk [C, nq]).

    dL/dk_{e,q} = w_q |det J_e| (grad u(x_q) . grad g(x_q)) with physical
    gradients grad = J^-T grad_hat.
    """
    if dofs is None:
        dofs, _ = topology.cg_numbering(cells, p)
    xq, wq, G, _ = tables(p, modified)
    C = cells.shape[0]
    dk = np.empty((C, wq.shape[0]))
    for s in range(0, C, CHUNK):
        e = slice(s, min(C, s + CHUNK))
        _, det, Jinv = geometry(xyz, cells[e])
        gu = np.einsum("cak,cqa->cqk", Jinv, np.einsum("qjk,cj->cqk", G, u[dofs[e]]))
        gg = np.einsum("cak,cqa->cqk", Jinv, np.einsum("qjk,cj->cqk", G, g[dofs[e]]))
        dk[e] = wq[None, :] * np.abs(det)[:, None] * np.einsum("cqk,cqk->cq", gu, gg)
    return apply_adjoint(xyz, cells, g, p, k, dofs=dofs, modified=modified), dk


def diagonal(xyz, cells, p, n, k=None, dirichlet_mask=None, dofs=None, modified=False, nodes=None):
    """diag(A): sum over cells and quadrature points of (J^-T grad phi_i)^T k w |detJ| (J^-T grad phi_i)."""
    if dofs is None:
        dofs, _ = topology.cg_numbering(cells, p)
    xq, wq, G, _ = tables(p, modified)
    C = cells.shape[0]
    de = np.empty((C, G.shape[1]))
    for s in range(0, C, CHUNK):
        e = slice(s, min(C, s + CHUNK))
        if nodes is not None:
            _, detq, Jq = geometry_curved(nodes[e], xq)
            gp = np.einsum("cqak,qja->cqjk", Jq, G)
            scale = wq[None, :] * np.abs(detq)
        else:
            _, det, Jinv = geometry(xyz, cells[e])
            gp = np.einsum("cak,qja->cqjk", Jinv, G)  # physical gradient of each shape function
            scale = wq[None, :] * np.abs(det)[:, None]
        if k is not None:
            scale = scale * k[e]
        de[e] = np.einsum("cq,cqjk,cqjk->cj", scale, gp, gp)
    d = _scatter(dofs, de, n)
    if dirichlet_mask is not None:
        d = np.where(dirichlet_mask, 1.0, d)
    return d


def rhs_const(xyz, cells, p, n, f=1.0, dirichlet_mask=None, dofs=None, modified=False, nodes=None):
    """b_i = sum_e sum_q w_q |det J| phi_i(x_q) f for a constant source f (Sec. 2.1 weak form)."""
    if dofs is None:
        dofs, _ = topology.cg_numbering(cells, p)
    xq, wq, _, V = tables(p, modified)
    if nodes is not None:
        _, detq, _ = geometry_curved(nodes, xq)
        be = f * (np.abs(detq) * wq[None, :]) @ V
    else:
        _, det, _ = geometry(xyz, cells)
        be = f * np.abs(det)[:, None] * (wq @ V)[None, :]
    b = _scatter(dofs, be, n)
    if dirichlet_mask is not None:
        b = np.where(dirichlet_mask, 0.0, b)
    return b
