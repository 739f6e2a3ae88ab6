"""Transfer between continuous Lagrange spaces of two degrees on one mesh (the p-levels of the
paper's hybrid multigrid, Sec. 4.1).

Prolongation P: a coarse function (degree pc) is evaluated at the fine nodes (degree p >= pc),
which is exact because P_pc is contained in P_p on every cell.  Restriction is the transpose
P^T.  P is built explicitly, one row per fine DoF from any cell that contains it (the coarse
function is continuous, so every such cell gives the same row).  Plain FP64 numpy, test
infrastructure only.
"""
from __future__ import annotations

import numpy as np

from . import basis


def prolongation_matrix(cells, p_fine, p_coarse, dofs_fine, dofs_coarse, n_fine, n_coarse):
    """Dense P [n_fine, n_coarse] (small meshes only)."""
    xhat = np.array(basis.nodes_beta(p_fine), dtype=np.float64)[:, 1:] / p_fine  # fine reference nodes
    T = basis.values(p_coarse, xhat)                                           # [nd_fine, nd_coarse]
    P = np.zeros((n_fine, n_coarse))
    done = np.zeros(n_fine, dtype=bool)
    for e in range(cells.shape[0]):
        for i, gi in enumerate(dofs_fine[e]):
            if done[gi]:
                continue
            P[gi, :] = 0.0
            P[gi, dofs_coarse[e]] = T[i]
            done[gi] = True
    return P


def prolongate(P, u_coarse, mask_fine=None):
    u = P @ u_coarse
    return u if mask_fine is None else np.where(mask_fine, 0.0, u)


def restrict(P, r_fine, mask_fine=None, mask_coarse=None):
    r = r_fine if mask_fine is None else np.where(mask_fine, 0.0, r_fine)
    rc = P.T @ r
    return rc if mask_coarse is None else np.where(mask_coarse, 0.0, rc)
