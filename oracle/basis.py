"""Lagrange P_p shape functions on the reference tetrahedron.

Reference tet: vertex 0 at the origin, vertex k at e_k.  Nodes are the
equispaced points x_hat_beta = (beta_1, beta_2, beta_3) / p for beta in N^4 with
|beta| = p; the local order is beta lexicographic ascending (beta_0 is the
weight of vertex 0).  The number of shape functions is (p+1)(p+2)(p+3)/6
(Sec. 2.3).

The oracle builds the basis the plain way: expand every shape function in the
monomials x^a y^b z^c (a+b+c <= p) and solve the Vandermonde system
V[node, monomial] C = I.  The table E of Eq. 4 is the derivative of these
polynomials at quadrature points.
"""
from __future__ import annotations

from functools import lru_cache

import numpy as np

from .quadrature import compositions


def nodes_beta(p: int):
    """Multi-indices beta in N^4, |beta| = p, lexicographic ascending."""
    return compositions(p, 4)


def monomials(p: int):
    """Exponents (a, b, c) with a+b+c <= p."""
    return [(a, b, c) for a in range(p + 1) for b in range(p + 1 - a) for c in range(p + 1 - a - b)]


def num_dofs(p: int) -> int:
    return (p + 1) * (p + 2) * (p + 3) // 6


@lru_cache(maxsize=None)
def _coefficients(p: int):
    betas = nodes_beta(p)
    mons = monomials(p)
    nodes = np.array([[b[1], b[2], b[3]] for b in betas], dtype=np.float64) / p
    V = np.empty((len(betas), len(mons)))
    for m, (a, b, c) in enumerate(mons):
        V[:, m] = nodes[:, 0] ** a * nodes[:, 1] ** b * nodes[:, 2] ** c
    C = np.linalg.solve(V, np.eye(len(betas)))  # column j = coefficients of phi_j
    C.setflags(write=False)
    return C


def values(p: int, x: np.ndarray) -> np.ndarray:
    """phi_j(x) for points x [..., 3] -> [..., ndof]."""
    C = _coefficients(p)
    mons = monomials(p)
    x = np.asarray(x, dtype=np.float64)
    M = np.stack([x[..., 0] ** a * x[..., 1] ** b * x[..., 2] ** c for (a, b, c) in mons], axis=-1)
    return M @ C


def gradients(p: int, x: np.ndarray) -> np.ndarray:
    """Reference gradients d phi_j / d x_hat_k at points x [..., 3] -> [..., ndof, 3]."""
    C = _coefficients(p)
    mons = monomials(p)
    x = np.asarray(x, dtype=np.float64)

    def dpow(v, e):
        return e * v ** (e - 1) if e > 0 else np.zeros_like(v)

    dx = np.stack([dpow(x[..., 0], a) * x[..., 1] ** b * x[..., 2] ** c for (a, b, c) in mons], axis=-1)
    dy = np.stack([x[..., 0] ** a * dpow(x[..., 1], b) * x[..., 2] ** c for (a, b, c) in mons], axis=-1)
    dz = np.stack([x[..., 0] ** a * x[..., 1] ** b * dpow(x[..., 2], c) for (a, b, c) in mons], axis=-1)
    return np.stack([dx @ C, dy @ C, dz @ C], axis=-1)
