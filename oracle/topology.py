"""Mesh topology for the oracle: canonical DoF numbering, faces and the Dirichlet set.

Canonical continuous DoF numbering (the gather operator G_e of Eq. 3): the node
beta of a cell with user vertices (v0, v1, v2, v3) is identified by its key, the
sorted p-tuple holding v_i repeated beta_i times.  Nodes of different cells with
equal keys are the same global DoF.  Global DoFs are numbered by the
lexicographic order of their keys.

Discontinuous DoFs (Eq. 5) belong to one cell each: DoF (e, j) has canonical
number e * ndof + j.
"""
from __future__ import annotations

import numpy as np

from .basis import nodes_beta

# local face m is opposite local vertex m; its vertices in increasing local order
FACE_VERTICES = ((1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2))


def dof_keys(cells: np.ndarray, p: int) -> np.ndarray:
    """Keys [C, ndof, p] int64 (sorted vertex multisets) for every cell node."""
    cells = np.asarray(cells, dtype=np.int64)
    betas = nodes_beta(p)
    keys = np.empty((cells.shape[0], len(betas), p), dtype=np.int64)
    for j, beta in enumerate(betas):
        cols = []
        for i in range(4):
            cols += [cells[:, i]] * beta[i]
        keys[:, j, :] = np.sort(np.stack(cols, axis=1), axis=1)
    return keys


def cg_numbering(cells: np.ndarray, p: int):
    """(dofs [C, ndof] int64 canonical global numbers, keys_unique [N, p])."""
    keys = dof_keys(cells, p)
    flat = keys.reshape(-1, p)
    uniq, inverse = np.unique(flat, axis=0, return_inverse=True)
    return inverse.reshape(keys.shape[0], keys.shape[1]), uniq


def faces(cells: np.ndarray):
    """Match cell faces.

    Returns (interior [F_i, 2, 2], boundary [F_b, 2]) where interior[f] =
    ((cell_minus, local_face_minus), (cell_plus, local_face_plus)) with the
    owner cell_minus < cell_plus, and boundary[f] = (cell, local_face).
    Raises ValueError if a face is shared by more than two cells.
    """
    cells = np.asarray(cells, dtype=np.int64)
    C = cells.shape[0]
    tri = np.stack([np.sort(cells[:, list(fv)], axis=1) for fv in FACE_VERTICES], axis=1)  # C,4,3
    flat = tri.reshape(-1, 3)
    uniq, inverse, counts = np.unique(flat, axis=0, return_inverse=True, return_counts=True)
    if np.any(counts > 2):
        raise ValueError("non-manifold mesh: a face is shared by more than two cells")
    owner = np.repeat(np.arange(C), 4)
    local = np.tile(np.arange(4), C)
    order = np.argsort(inverse, kind="stable")
    inv_sorted = inverse[order]
    starts = np.searchsorted(inv_sorted, np.arange(len(uniq)))
    one = counts == 1
    r = order[starts[one]]
    boundary = np.stack([owner[r], local[r]], axis=1)
    two = counts == 2
    a = order[starts[two]]
    b = order[starts[two] + 1]
    swap = owner[b] < owner[a]
    a, b = np.where(swap, b, a), np.where(swap, a, b)
    interior = np.stack([np.stack([owner[a], local[a]], axis=1), np.stack([owner[b], local[b]], axis=1)], axis=1)
    return interior.reshape(-1, 2, 2).astype(np.int64), boundary.reshape(-1, 2).astype(np.int64)


def boundary_vertex_sets(cells: np.ndarray):
    """Sets of boundary vertices, boundary edges (frozensets) and boundary faces."""
    cells = np.asarray(cells, dtype=np.int64)
    _, bnd = faces(cells)
    bv, be, bf = set(), set(), set()
    for c, m in bnd:
        tri = [int(cells[c, i]) for i in FACE_VERTICES[m]]
        bf.add(frozenset(tri))
        for i in range(3):
            bv.add(tri[i])
            be.add(frozenset((tri[i], tri[(i + 1) % 3])))
    return bv, be, bf


def dirichlet_mask(cells: np.ndarray, p: int, keys_unique: np.ndarray) -> np.ndarray:
    """True for DoFs on the boundary: the distinct vertices of the key lie on one boundary face."""
    bv, be, bf = boundary_vertex_sets(cells)
    mask = np.zeros(keys_unique.shape[0], dtype=bool)
    for i, key in enumerate(keys_unique):
        s = frozenset(int(v) for v in key)
        if len(s) == 1:
            mask[i] = next(iter(s)) in bv
        elif len(s) == 2:
            mask[i] = s in be
        elif len(s) == 3:
            mask[i] = s in bf
    return mask
