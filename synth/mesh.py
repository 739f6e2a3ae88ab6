"""Kuhn-split unit-cube meshes with seeded interior-vertex jitter.

The unit cube is divided into n^3 subcubes of edge h = 1/n.  Every subcube is
split into 6 tetrahedra, one per permutation s of the axes: the path
v0, v0+e_s0, v0+e_s0+e_s1, v0+e_s0+e_s1+e_s2 (the Kuhn / Freudenthal split).
Neighbouring subcubes use the same diagonal, so the mesh is conforming.  Half of
the cells come out with negative orientation; consumers use |det J|.

Cells are emitted in the natural generator order: subcube index i fastest, then
j, then k, and the six permutations in lexicographic order inside a subcube.
"""
from __future__ import annotations

import itertools

import numpy as np

_PERMS = list(itertools.permutations(range(3)))


def _vertex_id(i, j, k, n):
    return i + (n + 1) * (j + (n + 1) * k)


def kuhn_cube(n: int, jitter: float = 0.0, seed: int = 0):
    """Return (xyz [nv,3] float64, cells [nc,4] int32) for the Kuhn-split cube.

    jitter: each coordinate of each interior vertex is moved independently by
    U[-jitter*h, +jitter*h] using numpy's PCG64 generator seeded with `seed`.
    Boundary vertices stay fixed, so the domain is exactly the unit cube.
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    h = 1.0 / n
    g = np.arange(n + 1, dtype=np.float64) * h
    kk, jj, ii = np.meshgrid(g, g, g, indexing="ij")
    xyz = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1)

    ci, cj, ck = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    # subcube order: i fastest, then j, then k
    ci = ci.transpose(2, 1, 0).ravel()
    cj = cj.transpose(2, 1, 0).ravel()
    ck = ck.transpose(2, 1, 0).ravel()
    base = np.stack([ci, cj, ck], axis=1)  # [nsub, 3]
    cells = np.empty((base.shape[0], 6, 4), dtype=np.int64)
    unit = np.eye(3, dtype=np.int64)
    for t, perm in enumerate(_PERMS):
        cur = base.copy()
        cells[:, t, 0] = _vertex_id(cur[:, 0], cur[:, 1], cur[:, 2], n)
        for step in range(3):
            cur = cur + unit[perm[step]]
            cells[:, t, step + 1] = _vertex_id(cur[:, 0], cur[:, 1], cur[:, 2], n)
    cells = cells.reshape(-1, 4).astype(np.int32)
    if jitter:
        xyz = jitter_interior(xyz, n, jitter, seed)
    return xyz, cells


def jitter_interior(xyz: np.ndarray, n: int, jitter: float, seed: int) -> np.ndarray:
    """Move every coordinate of every interior lattice vertex by U[-jitter*h, jitter*h]."""
    h = 1.0 / n
    rng = np.random.default_rng(seed)
    delta = rng.uniform(-jitter * h, jitter * h, size=xyz.shape)
    eps = 1e-12
    interior = np.all((xyz > eps) & (xyz < 1.0 - eps), axis=1)
    out = xyz.copy()
    out[interior] += delta[interior]
    return out


def shuffle_mesh(xyz: np.ndarray, cells: np.ndarray, seed: int):
    """Randomly renumber vertices and cells (an 'unordered' mesh as a generator may emit it).

    Returns (xyz', cells', cell_perm) with cells'[i] = relabelled cells[cell_perm[i]].
    The vertex order inside each cell is kept, so orientation and reference maps
    are unchanged.
    """
    rng = np.random.default_rng(seed)
    nv = xyz.shape[0]
    vperm = rng.permutation(nv)  # new id -> old id
    inv = np.empty(nv, dtype=np.int64)
    inv[vperm] = np.arange(nv)
    cperm = rng.permutation(cells.shape[0])
    new_cells = inv[cells[cperm]].astype(np.int32)
    return xyz[vperm].copy(), new_cells, cperm


# Second-order geometry nodes of a cell: the ten points sum_a beta_a x_a / 2 over the multi-indices
# beta in N^4, |beta| = 2, in lexicographic ascending order (relative to the cell's vertex order).
_BETA2 = [b for b in itertools.product(range(3), repeat=4) if sum(b) == 2]


def curved_nodes(xyz: np.ndarray, cells: np.ndarray, amplitude: float) -> np.ndarray:
    """Geometry nodes [nc, 10, 3] of a curved version of the mesh: the straight cells' second-order
    nodes moved by the smooth map x -> x + amplitude * sin(pi x) sin(pi y) sin(pi z) * (1, 1, 1),
    which is the identity on the boundary of the unit cube (boundary faces stay flat, the domain
    stays the unit cube) and is evaluated once per node (shared nodes coincide)."""
    X = np.asarray(xyz, dtype=np.float64)[np.asarray(cells, dtype=np.int64)]  # [nc, 4, 3]
    B = np.array(_BETA2, dtype=np.float64) / 2.0                              # [10, 4]
    P = np.einsum("na,cad->cnd", B, X)
    s = np.sin(np.pi * P[..., 0]) * np.sin(np.pi * P[..., 1]) * np.sin(np.pi * P[..., 2])
    return P + amplitude * s[..., None]
